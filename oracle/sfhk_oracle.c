/*
 * SFHK oracle — plain, slow, FP64 CPU restatement of the strong-field
 * Herman–Kluk (SFHK) trajectory path of arXiv 2601.17164.
 *
 * THIS IS TEST INFRASTRUCTURE.  Only tests/, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library; the only common
 * ingredient is the published Philox4x64-10 definition, which each side
 * implements on its own.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 *
 * What it computes, in the paper's order:
 *   laser field  A(t), E(t) = -dA/dt            (Eq. EfieldTDSE, Sec. II.2)
 *   SFA birth    saddle point t_s = t0 + i t_t  (Eq. SAPeq), S_down^0, tunnel
 *                exit q0 = Re int A, p0 = k     (App. A, Eq. Int)
 *                amplitude                      (Eq. SFHKwf, App. B.1 / B.2)
 *   ADK birth    ADK rate, quasi-static exit, renormalised to the SFA rate
 *                at the two sub-peaks           (Sec. III.C)
 *   propagation  Hamilton's equations, stability blocks, action
 *                                                (App. A, after Eq. HKpropa)
 *   prefactor    C = sqrt(det Z), continuous branch, removal |C|^2 > D_t
 *                                                (Eq. C_HK, Sec. III.A)
 *   dipole       <psi0|z|p,q,gamma>, <psi0|k_z|p,q,gamma> (App. C),
 *                D(t) = -<psi0 e^{iIp t}|z|psi_c> + c.c. (Eq. D_t, V_t)
 *   spectrum     Hanning-windowed Fourier transform (App. D)
 *
 * Readings where the paper is silent or garbled (each one is listed in the
 * design notes): sin^2 pulse centred at t=0 spanning N optical cycles zero to
 * zero, defined through A; classical RK4 with fixed step; births on the
 * integrator grid with measure dt0 d^2k_perp; smallest positive t_t with
 * s = -sign E(t0); recombination phase e^{-i Ip t}; causal removal checked at
 * the output bins; branch of sqrt(det Z) followed at every grid point (the
 * sign closest to the previous grid point's C).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Parameter records (mirrored by ctypes in oracle/oracle.py).              */
/* ------------------------------------------------------------------------ */
typedef struct {
    double E0;      /* peak field, a.u.                                    */
    double omega;   /* carrier angular frequency, a.u.                     */
    double Tp;      /* zero-to-zero duration (sin^2) ; unused for CW       */
    double cep;     /* carrier-envelope phase, rad                         */
    int32_t kind;   /* 0: sin^2 pulse centred at t=0 ; 1: CW, no envelope  */
    int32_t pad;
} or_pulse;

enum { OR_POT_ZERO = 0, OR_POT_SOFTCORE = 1, OR_POT_TONGLIN = 2, OR_POT_HARMONIC = 3 };

typedef struct {
    int32_t pot;          /* potential kind                                 */
    int32_t gto_l;        /* 0: s-type GTO sum ; 1: p_z-type GTO sum        */
    int32_t n_gto;
    int32_t amp_kind;     /* 0: standard SPA (Eq. SFHKwf) ; 1: modified SPA ; 2: ADK */
    double pot_param[8];  /* softcore: a ; tonglin: Zc,a1..a6 ; harmonic: w */
    double ip;            /* ionisation potential, a.u.                     */
    double c[32];         /* GTO coefficients c_j                           */
    double alpha[32];     /* GTO exponents alpha_j                          */
} or_target;

typedef struct {
    double t_start;   /* time of grid index 0                               */
    double dt;        /* RK4 step                                           */
    int64_t n_steps;  /* last grid index                                    */
    int64_t n_out;    /* output bin every n_out steps                       */
    double gamma;     /* coherent-state width                               */
    double d_t;       /* removal threshold on |C|^2                         */
    int32_t removal_whole; /* 1: a removed trajectory contributes nothing   */
    int32_t pw_mask;  /* partial-wave filter: bit c keeps class c (0: no filter) */
    double pw_radius; /* radius of the near-core sphere of the filter        */
} or_grid;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition.  */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B97F4A7C15ULL; k1 += 0xBB67AE8584CAA73BULL; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Units (atomic units; the paper states only "atomic units").              */
/* ------------------------------------------------------------------------ */
double or_E0_from_intensity(double wcm2) { return sqrt(wcm2 / 3.50944758e16); }
double or_omega_from_lambda(double nm) { return 45.5633525 / nm; }

/* ------------------------------------------------------------------------ */
/* Laser field.  sin^2 pulse:                                               */
/*   A(t) = -(E0/w) cos^2(pi t/Tp) sin(w t + phi),  |t| <= Tp/2, else 0     */
/*   E(t) = -dA/dt                                                          */
/* CW: A(t) = -(E0/w) sin(w t + phi), E = E0 cos(w t + phi).                */
/* Complex arguments are used for the saddle point (analytic continuation   */
/* of the in-pulse expression).                                              */
/* ------------------------------------------------------------------------ */
static cplx field_A(const or_pulse* P, cplx t) {
    double w = P->omega;
    if (P->kind == 1) return -(P->E0 / w) * csin(w * t + P->cep);
    cplx env = ccos(OR_PI * t / P->Tp);
    return -(P->E0 / w) * env * env * csin(w * t + P->cep);
}

static cplx field_E(const or_pulse* P, cplx t) {
    double w = P->omega;
    if (P->kind == 1) return P->E0 * ccos(w * t + P->cep);
    /* product rule on -(E0/w) cos^2(x) sin(wt+phi), x = pi t/Tp */
    cplx x = OR_PI * t / P->Tp;
    cplx d_env = -2.0 * ccos(x) * csin(x) * (OR_PI / P->Tp);  /* d/dt cos^2 x */
    cplx env = ccos(x) * ccos(x);
    cplx dA = -(P->E0 / w) * (d_env * csin(w * t + P->cep) + env * w * ccos(w * t + P->cep));
    return -dA;
}

static int in_pulse(const or_pulse* P, double t) {
    return P->kind == 1 || fabs(t) <= 0.5 * P->Tp;
}

static double field_E_real(const or_pulse* P, double t) {
    if (!in_pulse(P, t)) return 0.0;
    return creal(field_E(P, t));
}

/* Sinusoid decomposition of A used for its closed-form integrals:
 *   A(t) = sum_j a_j sin(w_j t + phi).                                      */
static int field_modes(const or_pulse* P, double a[3], double wv[3]) {
    double w = P->omega;
    if (P->kind == 1) { a[0] = -P->E0 / w; wv[0] = w; return 1; }
    double Om = 2.0 * OR_PI / P->Tp;
    /* cos^2(pi t/Tp) = (1 + cos(Om t))/2 ; sin(u)cos(v) = [sin(u+v)+sin(u-v)]/2 */
    a[0] = -P->E0 / (2.0 * w); wv[0] = w;
    a[1] = -P->E0 / (4.0 * w); wv[1] = w + Om;
    a[2] = -P->E0 / (4.0 * w); wv[2] = w - Om;
    return 3;
}

/* int_0^t cos(w s + th) ds */
static cplx int_cos(double w, double th, cplx t) {
    if (fabs(w) < 1e-14) return t * cos(th);
    return (csin(w * t + th) - sin(th)) / w;
}
/* int_0^t sin(w s + th) ds */
static cplx int_sin(double w, double th, cplx t) {
    if (fabs(w) < 1e-14) return t * sin(th);
    return (cos(th) - ccos(w * t + th)) / w;
}

/* F(t) = int_0^t A */
static cplx field_F(const or_pulse* P, cplx t) {
    double a[3], wv[3];
    int m = field_modes(P, a, wv);
    cplx s = 0;
    for (int j = 0; j < m; ++j) s += a[j] * int_sin(wv[j], P->cep, t);
    return s;
}

/* G(t) = int_0^t A^2 ;  sin(u)sin(v) = [cos(u-v) - cos(u+v)]/2 */
static cplx field_G(const or_pulse* P, cplx t) {
    double a[3], wv[3];
    int m = field_modes(P, a, wv);
    cplx s = 0;
    for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k)
            s += 0.5 * a[j] * a[k] * (int_cos(wv[j] - wv[k], 0.0, t) - int_cos(wv[j] + wv[k], 2.0 * P->cep, t));
    return s;
}

/* Array exports for the pins. which: 0 A, 1 E, 2 F, 3 G (complex t).
 * Real in-pulse expressions are used for any t (no cut at the pulse edges). */
void or_field_eval(const or_pulse* P, int which, int64_t n, const double* t_re, const double* t_im,
                   double* out_re, double* out_im) {
    for (int64_t i = 0; i < n; ++i) {
        cplx t = t_re[i] + I * t_im[i];
        cplx v = 0;
        switch (which) {
            case 0: v = field_A(P, t); break;
            case 1: v = field_E(P, t); break;
            case 2: v = field_F(P, t); break;
            default: v = field_G(P, t); break;
        }
        out_re[i] = creal(v);
        out_im[i] = cimag(v);
    }
}

/* E on real times with the pulse-edge cut (what the integrator sees). */
void or_field_E_grid(const or_pulse* P, int64_t n, const double* t, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = field_E_real(P, t[i]);
}

/* ------------------------------------------------------------------------ */
/* Ground state psi0 = sum_j c_j e^{-alpha_j r^2}   (l=0)                   */
/*             psi0 = z sum_j c_j e^{-alpha_j r^2}  (l=1, p_z)               */
/* Tunnelling element (App. B.1), with the plane wave <k|r> =               */
/* (2 pi)^{-3/2} e^{-i k.r}, analytic in complex k:                          */
/*   m(k) = (2pi)^{-3/2} int e^{-i k.r} z psi0(r) d^3r                      */
/* ------------------------------------------------------------------------ */
static cplx tunnel_element(const or_target* T, const cplx k[3]) {
    cplx k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    double pw = pow(2.0 * OR_PI, -1.5);
    double pi32 = pow(OR_PI, 1.5);
    cplx s = 0;
    for (int j = 0; j < T->n_gto; ++j) {
        double al = T->alpha[j];
        cplx g = cexp(-k2 / (4.0 * al));
        if (T->gto_l == 0) {
            /* int z e^{-al r^2 - i k.r} = -i (pi^{3/2}/2) k_z al^{-5/2} e^{-k^2/4al} */
            s += T->c[j] * (-I * 0.5 * pi32) * k[2] * pow(al, -2.5) * g;
        } else {
            /* int z^2 e^{-al r^2 - i k.r} = (pi^{3/2}/4) al^{-7/2} (2 al - k_z^2) e^{-k^2/4al} */
            s += T->c[j] * (0.25 * pi32) * pow(al, -3.5) * (2.0 * al - k[2] * k[2]) * g;
        }
    }
    return pw * s;
}

void or_tunnel_element(const or_target* T, const double* k_re, const double* k_im, double* out) {
    cplx k[3] = {k_re[0] + I * k_im[0], k_re[1] + I * k_im[1], k_re[2] + I * k_im[2]};
    cplx v = tunnel_element(T, k);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* Recombination elements (App. C) for the normalised coherent state
 *   <r|p,q,gamma> = (2 gamma/pi)^{3/4} e^{-gamma (r-q)^2 + i p.(r-q)}.
 * d_len = <psi0| z |p,q,gamma>,  d_vel = <psi0| k_z |p,q,gamma>.            */
static void dipole_elements(const or_target* T, double gam, const double p[3], const double q[3],
                            cplx* d_len, cplx* d_vel) {
    double N = pow(2.0 * gam / OR_PI, 0.75);
    double pi32 = pow(OR_PI, 1.5);
    double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    double pq = p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
    cplx bz = 2.0 * gam * q[2] + I * p[2];   /* (2 gamma q_z + i p_z)       */
    cplx uz = p[2] - 2.0 * I * gam * q[2];   /* (p_z - 2 i gamma q_z)       */
    cplx sl = 0, sv = 0;
    for (int j = 0; j < T->n_gto; ++j) {
        double al = T->alpha[j];
        double be = gam + al;
        cplx X = (-p2 - 4.0 * al * (gam * q2 + I * pq)) / (4.0 * be);
        cplx eX = cexp(X);
        if (T->gto_l == 0) {
            sl += T->c[j] * pow(be, -2.5) * eX;
            sv += T->c[j] * al * pow(be, -2.5) * eX;
        } else {
            sl += T->c[j] * pow(be, -3.5) * eX * (bz * bz + 2.0 * be);
            sv += T->c[j] * al * pow(be, -3.5) * eX * (uz * uz / (2.0 * gam) + be / al);
        }
    }
    if (T->gto_l == 0) {
        *d_len = N * (0.5 * pi32) * bz * sl;
        *d_vel = N * pi32 * uz * sv;
    } else {
        *d_len = N * (0.25 * pi32) * sl;
        *d_vel = N * pi32 * (I * gam) * sv;
    }
}

void or_dipole_elements(const or_target* T, double gam, const double* p, const double* q, double* out) {
    cplx dl, dv;
    dipole_elements(T, gam, p, q, &dl, &dv);
    out[0] = creal(dl); out[1] = cimag(dl); out[2] = creal(dv); out[3] = cimag(dv);
}

/* ------------------------------------------------------------------------ */
/* SFA birth (App. A): saddle point, kz, tunnel exit, S_down^0, amplitude.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double kz, qz, tt;
    double S_re, S_im;      /* S_down^0                                    */
    double amp_re, amp_im;  /* amplitude without the Monte-Carlo weight    */
    int32_t valid;
    int32_t pad;
} or_birth_out;

/* Smallest tt > 0 with Im A(t0 + i tt) = s kappa, by a fine scan followed by
 * bisection.  Returns 0 when no root exists below tt_max.                 */
static int solve_tt(const or_pulse* P, double t0, double target, double* tt_out) {
    double a[3], wv[3];
    int m = field_modes(P, a, wv);
    double wmax = 0;
    for (int j = 0; j < m; ++j) if (fabs(wv[j]) > wmax) wmax = fabs(wv[j]);
    double h = 0.01 / wmax, tmax = 25.0 / wmax;
    double f_prev = cimag(field_A(P, t0)) - target;  /* = -target at tt = 0 */
    double lo = 0.0, hi = -1.0;
    for (double tt = h; tt <= tmax; tt += h) {
        double f = cimag(field_A(P, t0 + I * tt)) - target;
        if ((f > 0) != (f_prev > 0)) { lo = tt - h; hi = tt; break; }
        f_prev = f;
    }
    if (hi < 0) return 0;
    double flo = cimag(field_A(P, t0 + I * lo)) - target;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        double mid = 0.5 * (lo + hi);
        double fm = cimag(field_A(P, t0 + I * mid)) - target;
        if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    *tt_out = 0.5 * (lo + hi);
    return 1;
}

/* ------------------------------------------------------------------------ */
/* ADK births (Sec. III.C): the tunnelling theory's rate in place of the     */
/* SFA amplitude's modulus.  The paper names the ADK rate, the ADK tunnel    */
/* exit, and a renormalisation to the SFA rate near the two sub-peaks; the   */
/* rest is read as follows (each reading listed in the design notes):        */
/*  - static ADK rate for Z_c = 1, m = 0, kappa = sqrt(2 Ip), l = gto_l,     */
/*    without the constant C_l^2 of the orbital's tail (the renormalisation  */
/*    absorbs it):                                                           */
/*      w(F) = (2l+1)/2 kappa^{1-2/kappa} (2 kappa^3/F)^{2/kappa-1}           */
/*             exp(-2 kappa^3 / (3F)),                                       */
/*    with the transverse distribution (kappa/(pi F)) exp(-kappa k^2/F), so  */
/*    rho(t0, k) = w(|E(t0)|) (kappa/(pi |E|)) exp(-kappa k_perp^2/|E|) is the */
/*    rate per unit time and per d^2 k_perp;                                */
/*  - exit q0 = -Ip/E(t0) z, p0 = (kx, ky, 0) (the quasi-static exit);       */
/*  - phase: Re S_down^0 of the SFA saddle of the same (t0, k_perp), so      */
/*    e^{i(Re S + p0.q0)} with p0.q0 = 0;                                    */
/*  - amplitude N sqrt(rho) e^{i Re S}, N^2 = sum_j R(t_j) / sum_j w(|E(t_j)|) */
/*    over the two sub-peaks t_j = ((k* + j) pi - phi)/w, j = -1, +1, the     */
/*    carrier crests next to the one nearest the envelope's peak,            */
/*    k* = floor(phi/pi + 1/2), with R(t) the SFA rate by composite Simpson  */
/*    over k in [0, 6 sqrt(F/kappa)] with 128 intervals (F = |E(t)|):         */
/*      R(t) = 2 pi (h/3) sum_{i=1..128} c_i k_i |a(t, k_i)|^2,  k_i = i h,    */
/*      c_i = 4 for odd i, 2 for even i < 128, 1 for i = 128 (the k = 0 term   */
/*      vanishes), h = 6 sqrt(F/kappa)/128;                                  */
/*    a the standard saddle-point amplitude (no Monte Carlo measure).        */
/* ------------------------------------------------------------------------ */
static double adk_rate(const or_target* T, double F) {
    if (!(F > 0.0)) return 0.0;
    double kappa = sqrt(2.0 * T->ip);
    double l = (double)T->gto_l;
    return 0.5 * (2.0 * l + 1.0) * pow(kappa, 1.0 - 2.0 / kappa) * pow(2.0 * kappa * kappa * kappa / F, 2.0 / kappa - 1.0) *
           exp(-2.0 * kappa * kappa * kappa / (3.0 * F));
}

static double adk_density(const or_target* T, double F, double kperp2) {
    if (!(F > 0.0)) return 0.0;
    double kappa = sqrt(2.0 * T->ip);
    return adk_rate(T, F) * kappa / (OR_PI * F) * exp(-kappa * kperp2 / F);
}

void or_adk_subpeaks(const or_pulse* P, double* t2) {
    double ks = floor(P->cep / OR_PI + 0.5);
    t2[0] = ((ks - 1.0) * OR_PI - P->cep) / P->omega;
    t2[1] = ((ks + 1.0) * OR_PI - P->cep) / P->omega;
}

double or_adk_rate(const or_target* T, double F) { return adk_rate(T, F); }
double or_adk_density(const or_target* T, double F, double kperp2) { return adk_density(T, F, kperp2); }

static or_birth_out birth_one(const or_pulse* P, const or_target* T, double t0, double kx, double ky, double adk_n2);

double or_adk_norm2(const or_pulse* P, const or_target* T) {
    or_target Ts = *T;
    Ts.amp_kind = 0;
    double t2[2], num = 0.0, den = 0.0;
    or_adk_subpeaks(P, t2);
    double kappa = sqrt(2.0 * T->ip);
    for (int j = 0; j < 2; ++j) {
        double F = fabs(creal(field_E(P, t2[j])));
        if (!(F > 0.0)) continue;
        double h = 6.0 * sqrt(F / kappa) / 128.0;
        double R = 0.0;
        for (int i = 1; i <= 128; ++i) {
            double k = (double)i * h;
            double c = (i == 128) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
            or_birth_out b = birth_one(P, &Ts, t2[j], k, 0.0, 0.0);
            if (b.valid) R += c * k * (b.amp_re * b.amp_re + b.amp_im * b.amp_im);
        }
        num += 2.0 * OR_PI * (h / 3.0) * R;
        den += adk_rate(T, F);
    }
    double n2 = num / den;
    return (den > 0.0 && isfinite(n2)) ? n2 : 0.0;
}

static or_birth_out birth_one(const or_pulse* P, const or_target* T, double t0, double kx, double ky, double adk_n2) {
    or_birth_out b;
    memset(&b, 0, sizeof(b));
    double ip = T->ip;
    double Et0 = creal(field_E(P, t0));
    if (Et0 == 0.0) return b;
    double kperp2 = kx * kx + ky * ky;
    double kappa = sqrt(2.0 * ip + kperp2);
    double s = (Et0 > 0) ? -1.0 : 1.0;  /* s = -sign E(t0) */
    double tt;
    if (!solve_tt(P, t0, s * kappa, &tt)) return b;
    cplx ts = t0 + I * tt;
    double A0 = creal(field_A(P, t0));
    cplx Ats = field_A(P, ts);
    /* saddle point (Eq. SAPeq): kz + A(ts) - A(t0) = i s kappa */
    double kz = A0 - creal(Ats);
    /* tunnel exit q0 = Re int_{ts}^{t0} A (Eq. Int and text after it) */
    double qz = creal(field_F(P, t0) - field_F(P, ts));
    /* S_down^0 = Ip ts - int_{ts}^{t0} [k + A(t'') - A(t0)]^2 / 2 dt''   */
    double cc = kz - A0;
    cplx integral = 0.5 * ((kperp2 + cc * cc) * (t0 - ts)
                           + 2.0 * cc * (field_F(P, t0) - field_F(P, ts))
                           + (field_G(P, t0) - field_G(P, ts)));
    cplx S = ip * ts - integral;
    /* velocity at the saddle, v_s = k + A(ts) - A(t0) */
    cplx vs[3] = {kx, ky, kz + Ats - A0};
    cplx Ets = field_E(P, ts);
    cplx EdotV = Ets * vs[2];
    cplx amp;
    double p0q0 = kz * qz;  /* p0 = (kx, ky, kz), q0 = (0, 0, qz) */
    if (T->amp_kind == 0) {
        /* standard SPA: <v_s| r.E(ts) |psi0> / sqrt(E(ts).v_s) e^{i(S + p0.q0)} */
        cplx M = Ets * tunnel_element(T, vs);
        amp = M / csqrt(EdotV) * cexp(I * (S + p0q0));
    } else if (T->amp_kind == 1) {
        /* modified SPA (App. B.2): e^{i(S + p0.q0)} / (E(ts).v_s) */
        amp = cexp(I * (S + p0q0)) / EdotV;
    } else {
        /* ADK (Sec. III.C): quasi-static exit, ADK modulus, the saddle's real action */
        kz = 0.0;
        qz = -ip / Et0;
        amp = sqrt(adk_n2 * adk_density(T, fabs(Et0), kperp2)) * cexp(I * creal(S));
    }
    b.kz = kz; b.qz = qz; b.tt = tt;
    b.S_re = creal(S); b.S_im = cimag(S);
    b.amp_re = creal(amp); b.amp_im = cimag(amp);
    b.valid = isfinite(b.amp_re) && isfinite(b.amp_im);
    return b;
}

void or_birth(const or_pulse* P, const or_target* T, int64_t n, const double* t0, const double* kx,
              const double* ky, or_birth_out* out) {
    const double n2 = T->amp_kind == 2 ? or_adk_norm2(P, T) : 0.0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) out[i] = birth_one(P, T, t0[i], kx[i], ky[i], n2);
}

/* ------------------------------------------------------------------------ */
/* Birth sampling.                                                           */
/*  mode 0 (grid): n_t birth steps at the midpoints of n_t equal strata of   */
/*    the grid x n_k midpoints of k_perp in [0, kmax] with ky = 0; measure   */
/*    2 pi k dk dt0 (rotational symmetry about the polarisation axis).       */
/*  mode 1 (uniform t0, gaussian k_perp): birth i takes the Philox draw      */
/*    counter (i,0,0,0), key (seed,0); n0 = 1 + floor((i + r/2^32) M / N)   */
/*    with M = n_steps-1 (stratified uniform), k_perp ~ N(0, sigma^2)        */
/*    by Box-Muller; weight 1/(N pdf).                                      */
/* Output is sorted by n0 by construction.  Invalid births get amp = 0.    */
/* ------------------------------------------------------------------------ */
static void sample_one(const or_pulse* P, const or_target* T, const or_grid* G, int32_t mode, int64_t n,
                       int32_t n_t, int32_t n_k, double sigma, double kmax, uint64_t seed, int64_t i,
                       int32_t* n0, double* t0, double* px, double* py, double* pz, double* qz,
                       double* amp_re, double* amp_im, double adk_n2) {
    int64_t M = G->n_steps - 1;
    int64_t nb;
    double kx, ky, w;
    if (mode == 0) {
        int64_t it = i / n_k, ik = i % n_k;
        nb = (int64_t)floor(((double)it + 0.5) * (double)G->n_steps / (double)n_t);
        if (nb < 1) nb = 1;
        if (nb > M) nb = M;
        double dk = kmax / n_k;
        kx = ((double)ik + 0.5) * dk;
        ky = 0.0;
        double dt0 = (double)G->n_steps * G->dt / (double)n_t;
        w = 2.0 * OR_PI * kx * dk * dt0;
    } else {
        uint64_t ctr[4] = {(uint64_t)i, 0, 0, 0}, key[2] = {seed, 0}, x[4];
        or_philox4x64(ctr, key, x);
        uint64_t r = x[0] >> 32;
        unsigned __int128 num = ((unsigned __int128)(uint64_t)i << 32) + (unsigned __int128)r;
        num *= (unsigned __int128)(uint64_t)M;
        unsigned __int128 den = (unsigned __int128)(uint64_t)n << 32;
        nb = 1 + (int64_t)(num / den);
        double u1 = ((double)((x[1] >> 11) + 1)) * 0x1.0p-53;  /* (0,1] */
        double u2 = ((double)(x[2] >> 11)) * 0x1.0p-53;        /* [0,1) */
        double rad = sigma * sqrt(-2.0 * log(u1));
        kx = rad * cos(2.0 * OR_PI * u2);
        ky = rad * sin(2.0 * OR_PI * u2);
        double kp2 = kx * kx + ky * ky;
        double pdf_k = exp(-kp2 / (2.0 * sigma * sigma)) / (2.0 * OR_PI * sigma * sigma);
        double pdf_t = 1.0 / ((double)M * G->dt);
        w = 1.0 / ((double)n * pdf_k * pdf_t);
    }
    double tb = G->t_start + (double)nb * G->dt;
    or_birth_out b = birth_one(P, T, tb, kx, ky, adk_n2);
    *n0 = (int32_t)nb;
    *t0 = tb;
    *px = kx; *py = ky; *pz = b.kz; *qz = b.qz;
    *amp_re = b.valid ? w * b.amp_re : 0.0;
    *amp_im = b.valid ? w * b.amp_im : 0.0;
}

void or_sample_births(const or_pulse* P, const or_target* T, const or_grid* G, int32_t mode, int64_t n,
                      int32_t n_t, int32_t n_k, double sigma, double kmax, uint64_t seed,
                      int32_t* n0, double* t0, double* px, double* py, double* pz, double* qz,
                      double* amp_re, double* amp_im) {
    const double n2 = T->amp_kind == 2 ? or_adk_norm2(P, T) : 0.0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i)
        sample_one(P, T, G, mode, n, n_t, n_k, sigma, kmax, seed, i, n0 + i, t0 + i, px + i, py + i, pz + i,
                   qz + i, amp_re + i, amp_im + i, n2);
}

/* The same births, for the listed indices only (sampled checks at full size). */
void or_sample_births_at(const or_pulse* P, const or_target* T, const or_grid* G, int32_t mode, int64_t n,
                         int32_t n_t, int32_t n_k, double sigma, double kmax, uint64_t seed,
                         const int64_t* idx, int64_t m, int32_t* n0, double* t0, double* px, double* py,
                         double* pz, double* qz, double* amp_re, double* amp_im) {
    const double n2 = T->amp_kind == 2 ? or_adk_norm2(P, T) : 0.0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < m; ++j)
        sample_one(P, T, G, mode, n, n_t, n_k, sigma, kmax, seed, idx[j], n0 + j, t0 + j, px + j, py + j,
                   pz + j, qz + j, amp_re + j, amp_im + j, n2);
}

/* ------------------------------------------------------------------------ */
/* Atomic potential, radial form V(r), V'(r), V''(r).                       */
/* ------------------------------------------------------------------------ */
static void potential_radial(const or_target* T, double r, double* V, double* V1, double* V2) {
    const double* a = T->pot_param;
    switch (T->pot) {
        case OR_POT_SOFTCORE: {
            /* V = -1/sqrt(r^2 + a^2) */
            double s2 = r * r + a[0] * a[0];
            double s = sqrt(s2);
            *V = -1.0 / s;
            *V1 = r / (s2 * s);
            *V2 = (a[0] * a[0] - 2.0 * r * r) / (s2 * s2 * s);
            break;
        }
        case OR_POT_TONGLIN: {
            /* V = -(Zc + a1 e^{-a2 r} + a3 r e^{-a4 r} + a5 e^{-a6 r}) / r */
            double Zc = a[0], a1 = a[1], a2 = a[2], a3 = a[3], a4 = a[4], a5 = a[5], a6 = a[6];
            double e2 = exp(-a2 * r), e4 = exp(-a4 * r), e6 = exp(-a6 * r);
            double Y = Zc + a1 * e2 + a3 * r * e4 + a5 * e6;            /* numerator      */
            double Y1 = -a1 * a2 * e2 + a3 * (1.0 - a4 * r) * e4 - a5 * a6 * e6;
            double Y2 = a1 * a2 * a2 * e2 + a3 * (a4 * a4 * r - 2.0 * a4) * e4 + a5 * a6 * a6 * e6;
            /* V = -Y/r ; V' = Y/r^2 - Y'/r ; V'' = -2Y/r^3 + 2Y'/r^2 - Y''/r */
            *V = -Y / r;
            *V1 = Y / (r * r) - Y1 / r;
            *V2 = -2.0 * Y / (r * r * r) + 2.0 * Y1 / (r * r) - Y2 / r;
            break;
        }
        case OR_POT_HARMONIC: {
            double w = a[0];
            *V = 0.5 * w * w * r * r;
            *V1 = w * w * r;
            *V2 = w * w;
            break;
        }
        default:
            *V = 0; *V1 = 0; *V2 = 0;
    }
}

void or_potential_radial(const or_target* T, int64_t n, const double* r, double* out3) {
    for (int64_t i = 0; i < n; ++i) potential_radial(T, r[i], &out3[3 * i], &out3[3 * i + 1], &out3[3 * i + 2]);
}

/* V, grad V and Hess V at q: H_ij = V'' qh_i qh_j + (V'/r)(delta_ij - qh_i qh_j). */
static void potential(const or_target* T, const double q[3], double* V, double g[3], double H[3][3]) {
    double r = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    double V0, V1, V2;
    if (r == 0.0) {
        /* only smooth potentials reach r = 0: V'(0)=0, Hessian = V''(0) I */
        potential_radial(T, 0.0, &V0, &V1, &V2);
        *V = V0;
        for (int i = 0; i < 3; ++i) { g[i] = 0; for (int j = 0; j < 3; ++j) H[i][j] = (i == j) ? V2 : 0.0; }
        return;
    }
    potential_radial(T, r, &V0, &V1, &V2);
    double qh[3] = {q[0] / r, q[1] / r, q[2] / r};
    *V = V0;
    for (int i = 0; i < 3; ++i) {
        g[i] = V1 * qh[i];
        for (int j = 0; j < 3; ++j)
            H[i][j] = V2 * qh[i] * qh[j] + (V1 / r) * ((i == j ? 1.0 : 0.0) - qh[i] * qh[j]);
    }
}

/* ------------------------------------------------------------------------ */
/* Trajectory state, 43 reals (layout shared with the C-ABI contract):       */
/*   y[0..2] q, y[3..5] p,                                                  */
/*   y[6..14]  Mqq = dq/dq0, y[15..23] Mqp = dq/dp0,                         */
/*   y[24..32] Mpq = dp/dq0, y[33..41] Mpp = dp/dp0   (row-major, [i][j] =   */
/*   d(.)_i / d(.)0_j), y[42] S.                                              */
/* ------------------------------------------------------------------------ */
#define NY 43
#define IQ 0
#define IP 3
#define IMQQ 6
#define IMQP 15
#define IMPQ 24
#define IMPP 33
#define IS 42

/* Right-hand side: Hamilton's equations with H = p^2/2 + V(q) + q.E(t) z,
 * the stability equations dM_q./dt = M_p., dM_p./dt = -Hess V M_q., and
 * dS/dt = p.qdot - H.                                                        */
static void rhs(const or_target* T, double Et, const double* y, double* f) {
    double V, g[3], H[3][3];
    potential(T, y + IQ, &V, g, H);
    for (int i = 0; i < 3; ++i) {
        f[IQ + i] = y[IP + i];
        f[IP + i] = -g[i] - (i == 2 ? Et : 0.0);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            f[IMQQ + 3 * i + j] = y[IMPQ + 3 * i + j];
            f[IMQP + 3 * i + j] = y[IMPP + 3 * i + j];
            double sq = 0, sp = 0;
            for (int k = 0; k < 3; ++k) {
                sq += H[i][k] * y[IMQQ + 3 * k + j];
                sp += H[i][k] * y[IMQP + 3 * k + j];
            }
            f[IMPQ + 3 * i + j] = -sq;
            f[IMPP + 3 * i + j] = -sp;
        }
    double p2 = y[IP] * y[IP] + y[IP + 1] * y[IP + 1] + y[IP + 2] * y[IP + 2];
    double Hm = 0.5 * p2 + V + y[IQ + 2] * Et;
    f[IS] = p2 - Hm;  /* p.qdot - H with qdot = p */
}

/* Classical RK4: nodes 0, 1/2, 1/2, 1 ; weights 1/6, 1/3, 1/3, 1/6.       */
static void rk4_step(const or_target* T, const or_pulse* P, double t, double h, double* y) {
    double k1[NY], k2[NY], k3[NY], k4[NY], yt[NY];
    double Ea = field_E_real(P, t), Eb = field_E_real(P, t + 0.5 * h), Ec = field_E_real(P, t + h);
    rhs(T, Ea, y, k1);
    for (int i = 0; i < NY; ++i) yt[i] = y[i] + 0.5 * h * k1[i];
    rhs(T, Eb, yt, k2);
    for (int i = 0; i < NY; ++i) yt[i] = y[i] + 0.5 * h * k2[i];
    rhs(T, Eb, yt, k3);
    for (int i = 0; i < NY; ++i) yt[i] = y[i] + h * k3[i];
    rhs(T, Ec, yt, k4);
    for (int i = 0; i < NY; ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* det Z with Z = 1/2 (Mpp + Mqq - 2 i gamma Mqp - (1/(2 i gamma)) Mpq)  (Eq. C_HK) */
static cplx det_Z(const double* y, double gam) {
    cplx Z[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Z[i][j] = 0.5 * (y[IMPP + 3 * i + j] + y[IMQQ + 3 * i + j] - 2.0 * I * gam * y[IMQP + 3 * i + j]
                             - y[IMPQ + 3 * i + j] / (2.0 * I * gam));
    return Z[0][0] * (Z[1][1] * Z[2][2] - Z[1][2] * Z[2][1])
         - Z[0][1] * (Z[1][0] * Z[2][2] - Z[1][2] * Z[2][0])
         + Z[0][2] * (Z[1][0] * Z[2][1] - Z[1][1] * Z[2][0]);
}

void or_det_Z(const double* y43, double gam, double* out) {
    cplx d = det_Z(y43, gam);
    out[0] = creal(d); out[1] = cimag(d);
}

static int all_finite(const double* y) {
    for (int i = 0; i < NY; ++i) if (!isfinite(y[i])) return 0;
    return 1;
}

/* Neumaier-compensated accumulator */
typedef struct { double s, c; } nsum;
static void nadd(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x; else a->c += (x - t) + a->s;
    a->s = t;
}

enum { OR_FLAG_REMOVED = 1, OR_FLAG_NONFINITE = 2, OR_FLAG_BRANCH_GUARD = 4, OR_FLAG_INVALID = 8 };

typedef struct {
    int64_t removed, nonfinite, branch_guard;
    double traj_steps;
} or_stats;

/* One trajectory from grid index n0 to n_end.  The prefactor is followed at
 * every grid point: C = +-sqrt(det Z), the sign closest to the C of the
 * previous grid point (C(t0) = 1), so that C is continuous in time.  At every
 * output index (n % n_out == 0) and at n_end the trajectory is removed the
 * first time |C|^2 = |det Z| exceeds D_t (it contributes from then on
 * nothing); otherwise, if contrib != NULL, its recombination terms are
 * written there (per bin, 2 reals: D and v).  The branch guard flags a grid
 * step over which arg det Z moved by more than pi/2.  With a partial-wave
 * filter (pw_mask != 0) the trajectory is labelled at every grid point where
 * it enters r < pw_radius (birth counts as an entry when born inside) by
 * L = |q x p| there: class 0 (s) L < 0.5, 1 (p) L < 1.5, 2 (d) L < 2.5, 3
 * otherwise; it contributes at a bin only when it has been labelled and bit
 * (latest class) of pw_mask is set.                                        */
static int run_traj(const or_pulse* P, const or_target* T, const or_grid* G, int64_t n0, int64_t n_end,
                    const double q0[3], const double p0[3], cplx amp, double* y, cplx* C_out,
                    double* contrib, double* steps_out) {
    int flags = 0;
    memset(y, 0, NY * sizeof(double));
    for (int i = 0; i < 3; ++i) {
        y[IQ + i] = q0[i];
        y[IP + i] = p0[i];
        y[IMQQ + 4 * i] = 1.0;
        y[IMPP + 4 * i] = 1.0;
    }
    cplx C_prev = 1.0, det_prev = 1.0;   /* M = identity at birth: det Z = 1 */
    cplx C_acc = 1.0;                    /* last C accepted at an evaluation */
    double gam = G->gamma;
    double steps = 0;
    int pw_cls = -1, pw_in = 0;          /* class at the latest entry into the sphere; inside now */
    int64_t n;
    for (n = n0; n <= n_end; ++n) {
        double t = G->t_start + (double)n * G->dt;
        int on_bin = (n % G->n_out) == 0;
        if (n > n0) {
            if (!all_finite(y)) { flags |= OR_FLAG_NONFINITE | OR_FLAG_REMOVED; break; }
            cplx d = det_Z(y, gam);
            cplx C = csqrt(d);
            if (creal(C * conj(C_prev)) < 0.0) C = -C;
            if (creal(d * conj(det_prev)) < 0.0) flags |= OR_FLAG_BRANCH_GUARD;
            C_prev = C;
            det_prev = d;
        }
        if (G->pw_mask) {
            /* Sec. III.A-B partial waves: near the core the angular momentum
             * L = |q x p| is nearly conserved; a trajectory is labelled, each
             * time it enters r < pw_radius, by the partial wave of L there */
            const double* q = y + IQ;
            const double* p = y + IP;
            int in = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] < G->pw_radius * G->pw_radius;
            if (in && !pw_in) {
                double lx = q[1] * p[2] - q[2] * p[1];
                double ly = q[2] * p[0] - q[0] * p[2];
                double lz = q[0] * p[1] - q[1] * p[0];
                double L = sqrt(lx * lx + ly * ly + lz * lz);
                pw_cls = L < 0.5 ? 0 : (L < 1.5 ? 1 : (L < 2.5 ? 2 : 3));
            }
            pw_in = in;
        }
        if (on_bin || n == n_end) {
            if (!(cabs(det_prev) <= G->d_t)) {
                flags |= OR_FLAG_REMOVED;
                if (!isfinite(cabs(det_prev))) flags |= OR_FLAG_NONFINITE;
                break;
            }
            C_acc = C_prev;
            if (contrib && on_bin && G->pw_mask && !(pw_cls >= 0 && ((G->pw_mask >> pw_cls) & 1))) {
                int64_t k = n / G->n_out;   /* filtered out: no contribution at this bin */
                contrib[2 * k] = 0.0;
                contrib[2 * k + 1] = 0.0;
            } else if (contrib && on_bin) {
                cplx dl, dv;
                dipole_elements(T, gam, y + IP, y + IQ, &dl, &dv);
                /* e^{-i Ip t} <psi0|z|p_t,q_t> C e^{i S} amp ; D += -2 Re(.)  */
                cplx ph = cexp(I * (y[IS] - T->ip * t)) * C_prev * amp;
                int64_t k = n / G->n_out;
                contrib[2 * k] = -2.0 * creal(dl * ph);
                contrib[2 * k + 1] = -2.0 * creal(dv * ph);
            }
        }
        if (n == n_end) break;
        rk4_step(T, P, t, G->dt, y);
        steps += 1;
    }
    *C_out = C_acc;
    if (steps_out) *steps_out = steps;
    return flags;
}

/* Endpoints: integrate births from n0[i] to n_end with q0, p0 given in 3D.
 * state_out is [43][n] (SoA), C_out is [2][n] (re, im), flags_out [n].      */
void or_propagate(const or_pulse* P, const or_target* T, const or_grid* G, int64_t n, const int32_t* n0,
                  const double* q0, /* [3][n] */ const double* p0, /* [3][n] */ int64_t n_end,
                  double* state_out, double* C_out, int32_t* flags_out) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        double y[NY];
        double q[3] = {q0[i], q0[n + i], q0[2 * n + i]};
        double p[3] = {p0[i], p0[n + i], p0[2 * n + i]};
        cplx C;
        int f = run_traj(P, T, G, n0[i], n_end, q, p, 1.0, y, &C, NULL, NULL);
        for (int c = 0; c < NY; ++c) state_out[(int64_t)c * n + i] = y[c];
        C_out[i] = creal(C);
        C_out[n + i] = cimag(C);
        flags_out[i] = f;
    }
}

/* Whole path of one trajectory (for the classical-return pin): the state at
 * every grid index n0..n_end, [n_end-n0+1][43].  No removal, no prefactor.  */
void or_trajectory(const or_pulse* P, const or_target* T, const or_grid* G, int64_t n0, int64_t n_end,
                   const double* q0, const double* p0, double* path) {
    double y[NY];
    memset(y, 0, sizeof(y));
    for (int i = 0; i < 3; ++i) {
        y[IQ + i] = q0[i]; y[IP + i] = p0[i]; y[IMQQ + 4 * i] = 1.0; y[IMPP + 4 * i] = 1.0;
    }
    for (int64_t n = n0; n <= n_end; ++n) {
        memcpy(path + (n - n0) * NY, y, sizeof(y));
        if (n == n_end) break;
        rk4_step(T, P, G->t_start + (double)n * G->dt, G->dt, y);
    }
}

/* Induced dipole D(t_k) and dipole velocity v(t_k) on the output bins
 * k = 0 .. n_steps/n_out, summed over births (Neumaier).  Births carry
 * p0 = (px,py,pz), q0 = (0,0,qz) and their complex amplitude.               */
void or_dipole(const or_pulse* P, const or_target* T, const or_grid* G, int64_t n, const int32_t* n0,
               const double* px, const double* py, const double* pz, const double* qz,
               const double* amp_re, const double* amp_im, double* d_len, double* d_vel, or_stats* st) {
    int64_t nb = G->n_steps / G->n_out + 1;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    nsum* part = (nsum*)calloc((size_t)nthr * 2 * nb, sizeof(nsum));
    int64_t removed = 0, nonfinite = 0, guard = 0;
    double steps_tot = 0;
#pragma omp parallel reduction(+ : removed, nonfinite, guard, steps_tot)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        nsum* mine = part + (size_t)tid * 2 * nb;
        double* contrib = (double*)malloc(sizeof(double) * 2 * nb);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < n; ++i) {
            cplx amp = amp_re[i] + I * amp_im[i];
            if (amp == 0.0) continue;
            for (int64_t k = 0; k < 2 * nb; ++k) contrib[k] = 0.0;
            double y[NY], q[3] = {0, 0, qz[i]}, p[3] = {px[i], py[i], pz[i]}, steps;
            cplx C;
            int f = run_traj(P, T, G, n0[i], G->n_steps, q, p, amp, y, &C, contrib, &steps);
            steps_tot += steps;
            if (f & OR_FLAG_REMOVED) removed++;
            if (f & OR_FLAG_NONFINITE) nonfinite++;
            if (f & OR_FLAG_BRANCH_GUARD) guard++;
            if ((f & OR_FLAG_REMOVED) && G->removal_whole) continue;
            for (int64_t k = n0[i] / G->n_out; k < nb; ++k) {
                nadd(&mine[2 * k], contrib[2 * k]);
                nadd(&mine[2 * k + 1], contrib[2 * k + 1]);
            }
        }
        free(contrib);
    }
    for (int64_t k = 0; k < nb; ++k) {
        nsum a = {0, 0}, b = {0, 0};
        for (int t = 0; t < nthr; ++t) {
            nadd(&a, part[(size_t)t * 2 * nb + 2 * k].s);
            nadd(&a, part[(size_t)t * 2 * nb + 2 * k].c);
            nadd(&b, part[(size_t)t * 2 * nb + 2 * k + 1].s);
            nadd(&b, part[(size_t)t * 2 * nb + 2 * k + 1].c);
        }
        d_len[k] += a.s + a.c;
        d_vel[k] += b.s + b.c;
    }
    free(part);
    if (st) {
        st->removed += removed;
        st->nonfinite += nonfinite;
        st->branch_guard += guard;
        st->traj_steps += steps_tot;
    }
}

/* Hanning-windowed Fourier transform (App. D), rectangle rule on the bins:
 *   X(w) = sum_k x(t_k) W_H(t_k) e^{i w t_k} dt_out,
 *   W_H(t) = (1 + cos(pi t / tau_H)) / 2 for |t| <= tau_H, else 0.          */
void or_spectrum(const double* x, int64_t n_bins, double t0, double dt_out, double tau_h,
                 const double* omega, int64_t n_omega, double* out_re, double* out_im) {
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < n_omega; ++m) {
        nsum re = {0, 0}, im = {0, 0};
        for (int64_t k = 0; k < n_bins; ++k) {
            double t = t0 + (double)k * dt_out;
            double W = (fabs(t) <= tau_h) ? 0.5 * (1.0 + cos(OR_PI * t / tau_h)) : 0.0;
            cplx e = cexp(I * omega[m] * t) * (x[k] * W * dt_out);
            nadd(&re, creal(e));
            nadd(&im, cimag(e));
        }
        out_re[m] = re.s + re.c;
        out_im[m] = im.s + im.c;
    }
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
