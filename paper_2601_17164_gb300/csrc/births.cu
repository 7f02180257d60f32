// SFA births on the GPU (App. A, Eq. SAPeq / Eq. SFAwf / Eq. Int / Eq. SFHKwf;
// App. B.1 tunnelling matrix elements; App. B.2 modified SPA; Sec. III.C ADK
// births renormalised to the SFA rate at the pulse's two sub-peaks).
//
// One thread per birth, FP64.  The birth draws (grid or Philox) are integer
// exact; the saddle point is the smallest t_t > 0 with
// Im A(t0 + i t_t) = s kappa, s = -sign E(t0), found by a scan with an
// exponential recurrence for sinh, then a Newton iteration kept inside the
// bracket (bisection whenever a step would leave it).
#include "sfhk_device.cuh"

namespace sfhk {
namespace {

// Tunnelling element m(k) = (2pi)^{-3/2} int e^{-i k.r} z psi0 d^3r for complex k
// (GTO closed forms: s: -i pi^{3/2}/2 k_z a^{-5/2} e^{-k^2/4a};
//                    p: pi^{3/2}/4 a^{-7/2} (2a - k_z^2) e^{-k^2/4a}).
__device__ cd tunnel_element(const TargetDev& t, cd kx, cd ky, cd kz) {
    cd k2 = kx * kx + ky * ky + kz * kz;
    const double pw = 0.063493635934240969;          // (2 pi)^{-3/2}
    const double pi32 = 5.5683279968317078;          // pi^{3/2}
    cd s = mk(0, 0);
    for (int j = 0; j < t.n_gto; ++j) {
        double a = t.alpha[j];
        cd g = c_exp((-0.25 / a) * k2);
        if (t.gto_l == 0) {
            double c = t.c[j] * 0.5 * pi32 / (a * a * sqrt(a));
            s = s + c * (kz * g);
        } else {
            double c = t.c[j] * 0.25 * pi32 / (a * a * a * sqrt(a));
            s = s + c * ((mk(2.0 * a, 0) - kz * kz) * g);
        }
    }
    if (t.gto_l == 0) s = mk(0, -1) * s;   // factor -i of the s-type element
    return pw * s;
}

// Smallest root of f(tau) = sum_j c_j sinh(w_j tau) - target on (0, tau_max].
__device__ bool solve_tt(const FieldDev& f, double t0, double target, double* tt) {
    double c[3], w[3], e[3], eh[3];
    double wmax = 0.0;
    for (int j = 0; j < f.n_modes; ++j) {
        c[j] = f.a[j] * cos(f.w[j] * t0 + f.cep);
        w[j] = f.w[j];
        wmax = fmax(wmax, fabs(w[j]));
    }
    if (wmax == 0.0) return false;
    const double h = 0.02 / wmax, tmax = 25.0 / wmax;
    double ie[3], ieh[3];   // e^{-w_j tau} by its own recurrence: no division per scan point
    for (int j = 0; j < f.n_modes; ++j) {
        e[j] = 1.0;
        ie[j] = 1.0;
        eh[j] = exp(w[j] * h);
        ieh[j] = exp(-w[j] * h);
    }
    double fprev = -target, tau = 0.0, lo = -1.0, hi = -1.0;
    const int nscan = (int)(tmax / h);
    for (int it = 1; it <= nscan; ++it) {
        tau = it * h;
        double v = -target;
        for (int j = 0; j < f.n_modes; ++j) {
            e[j] *= eh[j];
            ie[j] *= ieh[j];
            v += c[j] * 0.5 * (e[j] - ie[j]);
        }
        if ((v > 0) != (fprev > 0)) {
            lo = tau - h;
            hi = tau;
            break;
        }
        fprev = v;
    }
    if (hi < 0) return false;
    auto fv = [&](double x) {
        double v = -target;
        for (int j = 0; j < f.n_modes; ++j) v += c[j] * sinh(w[j] * x);
        return v;
    };
    double flo = fv(lo);
    if ((flo > 0) == (fv(hi) > 0)) {
        // recurrence and direct values disagree at the bracket: rescan the cell finely
        double x0 = lo, f0 = flo;
        bool found = false;
        for (int k = 1; k <= 64; ++k) {
            double x1 = lo + (hi - lo) * k / 64.0, f1 = fv(x1);
            if ((f1 > 0) != (f0 > 0)) {
                lo = x0;
                hi = x1;
                flo = f0;
                found = true;
                break;
            }
            x0 = x1;
            f0 = f1;
        }
        if (!found) return false;
    }
    // safeguarded Newton inside the bracket (bisection when a step leaves it)
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 100; ++it) {
        double v = -target, d = 0.0;
        for (int j = 0; j < f.n_modes; ++j) {
            const double e = exp(w[j] * x), ie = 1.0 / e;
            v += c[j] * 0.5 * (e - ie);          // sinh
            d += c[j] * w[j] * 0.5 * (e + ie);   // derivative: w cosh
        }
        if ((v > 0) == (flo > 0)) lo = x; else hi = x;
        double xn = (d != 0.0) ? x - v / d : 0.5 * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        const bool done = fabs(xn - x) <= 1e-15 * fabs(xn) || hi - lo <= 1e-15 * hi;
        x = xn;
        if (done) break;
    }
    *tt = x;
    return true;
}

// The saddle of a birth (t0, kx, ky) and its amplitude without the Monte Carlo
// measure: kind 0 standard SPA, 1 modified SPA, 2 ADK (modulus sqrt(adk_n2 rho),
// phase Re S, exit q0 = -Ip/E(t0), kz = 0).  Returns false where no saddle exists.
__device__ bool birth_amp(const FieldDev& f, const TargetDev& t, double t0, double kx, double ky, int kind,
                          double adk_n2, double* kz_out, double* qz_out, cd* amp_out);

// ADK rate per unit time (Z_c = 1, m = 0, l = gto_l; the tail constant C_l^2 left out):
//   w(F) = (2l+1)/2 kappa^{1-2/kappa} (2 kappa^3/F)^{2/kappa-1} exp(-2 kappa^3/(3F)),
// and per d^2 k_perp: rho = w(F) (kappa/(pi F)) exp(-kappa k_perp^2/F).
__device__ double adk_rate(const TargetDev& t, double F) {
    if (!(F > 0.0)) return 0.0;
    const double kappa = sqrt(2.0 * t.ip), k3 = kappa * kappa * kappa;
    return 0.5 * (2.0 * t.gto_l + 1.0) * pow(kappa, 1.0 - 2.0 / kappa) * pow(2.0 * k3 / F, 2.0 / kappa - 1.0) *
           exp(-2.0 * k3 / (3.0 * F));
}
__device__ double adk_density(const TargetDev& t, double F, double kperp2) {
    if (!(F > 0.0)) return 0.0;
    const double kappa = sqrt(2.0 * t.ip);
    return adk_rate(t, F) * kappa / (kPi * F) * exp(-kappa * kperp2 / F);
}

__device__ bool birth_amp(const FieldDev& f, const TargetDev& t, double t0, double kx, double ky, int kind,
                          double adk_n2, double* kz_out, double* qz_out, cd* amp_out) {
    *kz_out = 0.0;
    *qz_out = 0.0;
    *amp_out = mk(0, 0);
    const FieldAt at0 = field_at(f, mk(t0, 0));
    const double Et0 = at0.E.re;
    if (Et0 == 0.0) return false;
    const double kp2 = kx * kx + ky * ky;
    const double kappa = sqrt(2.0 * t.ip + kp2);
    const double s = Et0 > 0 ? -1.0 : 1.0;
    double tt;
    if (!solve_tt(f, t0, s * kappa, &tt)) return false;
    const cd ts = mk(t0, tt);
    const FieldAt ats = field_at(f, ts);
    const double A0 = at0.A.re;
    const cd Ats = ats.A;
    double kz = A0 - Ats.re;
    const cd F0 = at0.F, Fs = ats.F;
    double qz = (F0 - Fs).re;
    const double cc = kz - A0;
    const cd G0 = at0.G, Gs = ats.G;
    // int_{ts}^{t0} v^2/2 with v = k + A - A(t0): constant, linear and quadratic parts
    const cd dt0 = mk(0.0, -tt);  // t0 - ts
    cd integ = 0.5 * ((kp2 + cc * cc) * dt0 + 2.0 * cc * (F0 - Fs) + (G0 - Gs));
    const cd S = t.ip * ts - integ;
    cd amp;
    if (kind == 2) {
        // ADK (Sec. III.C): quasi-static exit, ADK modulus, the saddle's real action
        kz = 0.0;
        qz = -t.ip / Et0;
        amp = sqrt(adk_n2 * adk_density(t, fabs(Et0), kp2)) * c_exp(mk(0.0, S.re));
    } else {
        const cd vz = mk(kz - A0, 0.0) + Ats;
        const cd Ets = ats.E;
        const cd EdotV = Ets * vz;
        const cd ph = c_exp(mk(-S.im, S.re + kz * qz));   // e^{i(S + p0.q0)}
        if (kind == 0) {
            cd m = tunnel_element(t, mk(kx, 0), mk(ky, 0), vz);
            amp = cdiv(Ets * m, c_sqrt(EdotV)) * ph;
        } else {
            amp = cdiv(ph, EdotV);
        }
    }
    if (!isfinite(amp.re) || !isfinite(amp.im)) amp = mk(0, 0);
    *kz_out = kz;
    *qz_out = qz;
    *amp_out = amp;
    return true;
}

// ADK renormalisation N^2 (Sec. III.C), evaluated by every block of 128 threads
// (the same sum in the same order, so every block gets the same value): the SFA
// rate over the ADK rate summed over the two sub-peaks t_j = ((k* + j) pi - phi)/w,
// j = -1, +1, k* = floor(phi/pi + 1/2); the SFA rate by composite Simpson over
// k_perp in [0, 6 sqrt(F/kappa)], 128 intervals: thread (j, m) takes the nodes
// i = 2m + 1 and 2m + 2 of sub-peak j.
__device__ double adk_norm2_block(const FieldDev& f, const TargetDev& t, double* s_part) {
    const int tid = threadIdx.x, j = tid >> 6, m = tid & 63;
    const double ks = floor(f.cep / kPi + 0.5);
    const double tj = ((ks + (j == 0 ? -1.0 : 1.0)) * kPi - f.cep) / f.omega;
    const double F = fabs(field_E(f, mk(tj, 0)).re);
    const double kappa = sqrt(2.0 * t.ip);
    const double h = 6.0 * sqrt(F / kappa) / 128.0;
    double part = 0.0;
    if (F > 0.0) {
        for (int q = 0; q < 2; ++q) {
            const int i = 2 * m + 1 + q;
            const double k = (double)i * h;
            const double c = (i == 128) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
            double kz, qz;
            cd a;
            if (birth_amp(f, t, tj, k, 0.0, 0, 0.0, &kz, &qz, &a)) part += c * k * (a.re * a.re + a.im * a.im);
        }
    }
    s_part[tid] = part;
    __syncthreads();
    double num = 0.0, den = 0.0;
    for (int jj = 0; jj < 2; ++jj) {
        const double tq = ((ks + (jj == 0 ? -1.0 : 1.0)) * kPi - f.cep) / f.omega;
        const double Fq = fabs(field_E(f, mk(tq, 0)).re);
        if (!(Fq > 0.0)) continue;
        double R = 0.0;
        for (int q = 0; q < 64; ++q) R += s_part[64 * jj + q];
        num += 2.0 * kPi * ((6.0 * sqrt(Fq / kappa) / 128.0) / 3.0) * R;
        den += adk_rate(t, Fq);
    }
    const double n2 = num / den;
    return (den > 0.0 && isfinite(n2)) ? n2 : 0.0;
}

__global__ void __launch_bounds__(128) births_kernel(FieldDev f, TargetDev t, BirthArgs a) {
    __shared__ double s_part[128];
    const double adk_n2 = t.amp == 2 ? adk_norm2_block(f, t, s_part) : 0.0;   // every thread takes part
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // output index
    if (o >= a.count) return;
    const int64_t i = a.first + o;                                       // birth index
    int64_t nb;
    double kx, ky, w;
    const int64_t M = f.n_steps - 1;
    if (a.mode == 0) {
        int64_t it = i / a.n_k, ik = i % a.n_k;
        nb = (int64_t)floor(((double)it + 0.5) * (double)f.n_steps / (double)a.n_t);
        nb = nb < 1 ? 1 : (nb > M ? M : nb);
        double dk = a.kmax / a.n_k;
        kx = ((double)ik + 0.5) * dk;
        ky = 0.0;
        w = 2.0 * kPi * kx * dk * ((double)f.n_steps * f.dt / (double)a.n_t);
    } else {
        uint64_t x[4] = {(uint64_t)i, 0, 0, 0};
        philox4x64_10(x, a.seed, 0);
        unsigned __int128 num = (((unsigned __int128)(uint64_t)i) << 32) + (unsigned __int128)(x[0] >> 32);
        num *= (unsigned __int128)(uint64_t)M;
        unsigned __int128 den = ((unsigned __int128)(uint64_t)a.n) << 32;
        nb = 1 + (int64_t)(num / den);
        double u1 = (double)((x[1] >> 11) + 1) * 0x1.0p-53;
        double u2 = (double)(x[2] >> 11) * 0x1.0p-53;
        double rad = a.sigma * sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        kx = rad * cs;
        ky = rad * sn;
        double s2 = a.sigma * a.sigma;
        // w = 1/(n pdf),  pdf = e^{-k^2/2s^2}/(2 pi s^2) * 1/(M dt)
        w = 2.0 * kPi * s2 * exp((kx * kx + ky * ky) / (2.0 * s2)) * ((double)M * f.dt) / (double)a.n;
    }
    const double t0 = f.t_start + (double)nb * f.dt;
    double kz = 0.0, qz = 0.0;
    cd amp = mk(0, 0);
    birth_amp(f, t, t0, kx, ky, t.amp, adk_n2, &kz, &qz, &amp);
    a.n0[o] = (int32_t)nb;
    a.t0[o] = t0;
    a.px[o] = kx;
    a.py[o] = ky;
    a.pz[o] = kz;
    a.qz[o] = qz;
    a.amp_re[o] = w * amp.re;
    a.amp_im[o] = w * amp.im;
}

}  // namespace

cudaError_t launch_births(const FieldDev& f, const TargetDev& t, const BirthArgs& a, cudaStream_t s) {
    if (a.count == 0) return cudaSuccess;
    const int block = 128;   // the ADK renormalisation spreads its 2 x 64 Simpson pairs over 128 threads
    const int64_t grid = (a.count + block - 1) / block;
    births_kernel<<<(unsigned)grid, block, 0, s>>>(f, t, a);
    return cudaGetLastError();
}

}  // namespace sfhk
