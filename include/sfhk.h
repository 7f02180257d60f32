/*
 * sfhk.h — C ABI of the GB300 SFHK trajectory library.
 *
 * The library computes the hot path of the semiclassical strong-field
 * Herman–Kluk (SFHK) method for high-harmonic generation (arXiv 2601.17164):
 * strong-field-approximation births, classical propagation of coherent-state
 * centres with their 3x3 stability blocks and action, the Herman–Kluk
 * prefactor with continuous branch tracking, the time-binned induced dipole
 * and dipole velocity, and the Hanning-windowed spectrum.
 *
 * Conventions shared by every call
 *   - Atomic units throughout.  Linear polarisation along z.
 *   - Handles (sfhk_field, sfhk_target) are owned by the library: create and
 *     destroy them in pairs.  A handle belongs to the CUDA device that was
 *     current when it was created; use it only with that device current.
 *     Handles are read-only after creation and may be shared across streams.
 *   - Every array argument is caller-owned DEVICE memory on that device
 *     unless stated otherwise; the library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous with respect to the host unless
 *     stated otherwise.
 *   - Every call validates its arguments and returns a status.  A non-OK
 *     status leaves a thread-local message for sfhk_last_error().  Errors
 *     raised by kernels still running surface at sfhk_sync() or the next
 *     call.  No C++ exception crosses this boundary.
 *   - Output bins are ACCUMULATED into (so chunks, shards and configurations
 *     can be summed); the caller zeroes them first.
 *   - Some calls use scratch memory the library keeps per device (grown on
 *     demand with cudaMalloc): sfhk_dipole with deterministic bins or with
 *     escalation, sfhk_resample_births.  Such calls must not overlap on the GPU
 *     (issue them on one stream, or order the streams).
 */
#ifndef SFHK_H
#define SFHK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFHK_OK = 0,
    SFHK_EINVAL = 1,        /* bad argument (size, pointer, non-finite value)   */
    SFHK_ENOMEM = 2,        /* device or host allocation failed                 */
    SFHK_ECUDA = 3,         /* CUDA runtime error                               */
    SFHK_ETIMEOUT = 4,      /* a bounded device wait ran out                     */
    SFHK_ENUMERIC = 5,      /* reserved: non-finite result where none is allowed */
    SFHK_EUNSUPPORTED = 6   /* device or option not supported                    */
} sfhk_status;

/* Thread-local message for the last non-OK status of this thread ("" if none). */
const char* sfhk_last_error(void);
/* Library version string. */
const char* sfhk_version(void);
/* Waits for `stream`, then reports any asynchronous error of this library's
 * kernels (device status word) or of the CUDA runtime. */
sfhk_status sfhk_sync(void* stream);

/* ------------------------------------------------------------------------
 * Laser field (Sec. II.2, Eq. EfieldTDSE; App. A: E = -dA/dt).
 * One linearly polarised sin^2 pulse centred at t = 0, `cycles` optical
 * cycles from zero to zero:
 *   A(t) = -(E0/w) cos^2(pi t/Tp) sin(w t + cep),  |t| <= Tp/2 ;  0 outside,
 *   E0 = sqrt(I / 3.50944758e16 W/cm^2),  w = 45.5633525 / lambda[nm],
 *   Tp = cycles * 2 pi / w.
 * The integrator grid is t_n = -Tp/2 + n dt, n = 0..n_steps with
 * n_steps = ceil(Tp/dt); output bins are t_k = -Tp/2 + k t_out_step,
 * k = 0..n_bins-1, n_bins = n_steps/n_out + 1, n_out = t_out_step/dt, which
 * must be an integer (|n_out dt - t_out_step| < 1e-12).
 * The handle holds device tables of E at the RK4 half steps (FP64 and FP32).
 * ---------------------------------------------------------------------- */
typedef struct {
    double intensity_wcm2;   /* peak intensity, W/cm^2 (> 0, or 0 for no field) */
    double lambda_nm;        /* carrier wavelength, nm (> 0)                     */
    double cycles;           /* optical cycles zero to zero (> 0)                */
    double cep_rad;          /* carrier-envelope phase                           */
    int32_t envelope;        /* 0 = sin^2 (the only envelope)                    */
    int32_t reserved;
} sfhk_pulse;

typedef struct sfhk_field sfhk_field;

typedef struct {
    double E0, omega, Tp, t_start, dt, t_out;
    int64_t n_steps, n_out, n_bins;
} sfhk_field_info;

/* Builds the field tables on the current device.  Host pointers in, handle out.
 * Errors: SFHK_EINVAL (non-finite or out-of-range parameters, non-integer
 * n_out, more than 2^30 steps), SFHK_ENOMEM, SFHK_ECUDA. */
sfhk_status sfhk_make_field(const sfhk_pulse* pulse, double dt, double t_out_step, sfhk_field** out);
sfhk_status sfhk_field_get_info(const sfhk_field* field, sfhk_field_info* info /* host */);
void sfhk_field_destroy(sfhk_field* field);

/* ------------------------------------------------------------------------
 * Target: atomic potential V_a and ground state psi0 as GTOs (Sec. II.1,
 * App. A Hamiltonian H = p^2/2 + V_a(q) + q.E(t); App. B.1 GTO expansion).
 *   potential 0 ZERO       V = 0                        (Lewenstein limit)
 *             1 SOFTCORE   V = -1/sqrt(r^2 + a^2)       pot_param[0] = a
 *             2 TONGLIN    V = -(Zc + a1 e^{-a2 r} + a3 r e^{-a4 r}
 *                               + a5 e^{-a6 r}) / r     pot_param[0..6] = Zc,a1..a6
 *             3 HARMONIC   V = w^2 r^2 / 2              pot_param[0] = w
 *   gto_l 0: psi0 = sum_j c_j e^{-alpha_j r^2};  1: psi0 = z sum_j c_j e^{-alpha_j r^2}
 *   amp   0: standard SPA birth amplitude (App. A, Eq. SFHKwf)
 *         1: modified SPA (App. B.2, Eq. SFHKmodSPA)
 *         2: ADK births (Sec. III.C): the tunnelling theory's rate replaces the
 *            SFA modulus, renormalised to the SFA rate at the pulse's two
 *            sub-peaks (see sfhk_sample_births)
 * gto_c / gto_alpha are HOST arrays of n_gto (1..32) values, copied.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t potential;
    int32_t gto_l;
    int32_t n_gto;
    int32_t amp;
    double pot_param[8];
    double ip;                 /* ionisation potential Ip > 0                 */
    const double* gto_c;       /* host, n_gto                                */
    const double* gto_alpha;   /* host, n_gto, each > 0                      */
} sfhk_target_desc;

typedef struct sfhk_target sfhk_target;

sfhk_status sfhk_make_target(const sfhk_target_desc* desc, sfhk_target** out);
void sfhk_target_destroy(sfhk_target* target);

/* ------------------------------------------------------------------------
 * Births (App. A, Eq. SAPeq, Eq. SFAwf, Eq. Int, Eq. SFHKwf).
 * For a birth step n0 (t0 = -Tp/2 + n0 dt) and transverse momentum
 * (kx, ky): kappa = sqrt(2 Ip + kx^2 + ky^2), s = -sign E(t0), t_t = the
 * smallest t_t > 0 with Im A(t0 + i t_t) = s kappa; then
 *   kz = A(t0) - Re A(t_s),  p0 = (kx, ky, kz),  q0 = (0, 0, Re[F(t0) - F(t_s)]),
 *   S0 = Ip t_s - int_{t_s}^{t0} [k + A(t'') - A(t0)]^2/2 dt''   (F = int A),
 *   amp = w * <v_s| r.E(t_s) |psi0> / sqrt(E(t_s).v_s) * e^{i(S0 + p0.q0)}
 *   (v_s = k + A(t_s) - A(t0); modified SPA: e^{i(S0+p0.q0)} / (E(t_s).v_s)),
 * w = the Monte-Carlo measure of the birth.  Births without such a root get
 * amp = 0.
 * ADK births (target amp 2; Sec. III.C): the same saddle, but kz = 0, the
 * quasi-static exit q0 = (0, 0, -Ip/E(t0)) and
 *   amp = w * N sqrt(rho(t0, k)) * e^{i Re S0},
 *   rho = w_ADK(F) (kappa/(pi F)) e^{-kappa k^2/F},  F = |E(t0)|, kappa = sqrt(2 Ip),
 *   w_ADK(F) = (2l+1)/2 kappa^{1-2/kappa} (2 kappa^3/F)^{2/kappa-1} e^{-2 kappa^3/(3F)}
 * (Z_c = 1, m = 0, l = gto_l, the orbital's tail constant left out), and
 *   N^2 = sum_j R(t_j) / sum_j w_ADK(|E(t_j)|)
 * over the two sub-peaks t_j = ((k* + j) pi - cep)/w, j = -1, +1,
 * k* = floor(cep/pi + 1/2) (the carrier crests next to the one nearest the
 * envelope's peak), R(t) the SFA rate: 2 pi int k |a(t, k)|^2 dk over the
 * standard-SPA amplitude without measure, by composite Simpson over
 * [0, 6 sqrt(F/kappa)] with 128 intervals.  N = 0 (all amplitudes 0) when
 * both sub-peaks fall outside the pulse.
 *   mode 0 GRID: n = n_t * n_k births; birth i = it*n_k + ik has
 *      n0 = clamp(floor((it + 1/2) n_steps / n_t), 1, n_steps-1),
 *      kx = (ik + 1/2) kmax/n_k, ky = 0, w = 2 pi kx (kmax/n_k)(n_steps dt/n_t)
 *      (rotational symmetry about z).
 *   mode 1 UNIFORM_T_GAUSS_K: birth i draws Philox4x64-10 with counter
 *      (i,0,0,0), key (seed,0) -> words x0..x3;
 *      n0 = 1 + floor(((i << 32) + (x0 >> 32)) * M / (n << 32)), M = n_steps-1
 *      (stratified uniform, exact integer arithmetic);
 *      u1 = ((x1 >> 11) + 1) 2^-53, u2 = (x2 >> 11) 2^-53,
 *      (kx, ky) = sigma sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2);
 *      w = 1 / (n pdf), pdf = e^{-k^2/2 sigma^2} / (2 pi sigma^2 M dt).
 * In both modes the output is sorted by n0.  A chunk [first, first+count) of
 * the n-birth sample can be produced on its own (streaming in birth-time
 * order); birth i lands at output index i - first.
 * Output arrays (device, capacity >= count): n0 int32; t0, p0x, p0y, p0z, q0z,
 * amp_re, amp_im double.  q0x / q0y are optional (NULL: taken as 0 by the
 * propagation calls; never written here).
 * ---------------------------------------------------------------------- */
typedef struct {
    int64_t n;           /* number of births (mode 0: must equal n_t*n_k)  */
    int32_t mode;        /* 0 GRID, 1 UNIFORM_T_GAUSS_K                     */
    int32_t n_t, n_k;    /* grid sizes (mode 0)                             */
    int32_t reserved;
    double sigma_k;      /* gaussian sigma (mode 1), > 0                    */
    double kmax;         /* grid extent (mode 0), > 0                       */
    uint64_t seed;       /* Philox key (mode 1)                             */
    int64_t first;       /* index of the first birth produced (streaming)  */
    int64_t count;       /* births produced: first .. first+count-1 of the
                            n-birth sample (0: n - first)                  */
} sfhk_birth_params;

typedef struct {
    int32_t* n0;
    double *t0, *p0x, *p0y, *p0z, *q0z, *amp_re, *amp_im;
    double *q0x, *q0y;   /* optional, may be NULL                          */
    int64_t capacity;
} sfhk_births;

sfhk_status sfhk_sample_births(const sfhk_field* field, const sfhk_target* target,
                               const sfhk_birth_params* params, const sfhk_births* births, void* stream);

/* ------------------------------------------------------------------------
 * Importance sampling in proportion to |I0| (App. A, Eq. Int: a momentum that
 * solves the saddle-point equation enters with weight |I0|, which makes the
 * Monte Carlo sum an importance sampling).  Systematic resampling of a
 * proposal pool of m births (e.g. from sfhk_sample_births, whose amplitudes
 * already carry |I0| times the proposal weight) down to n births:
 *   w_i = sqrt(re_i * re_i + im_i * im_i) (no fused multiply-add), A = max w_i,
 *   q_i = floor(w_i * (2^B / A)), B = 62 - ceil(log2 max(2, m)), Q = sum q_i;
 *   U = high 32 bits of word 0 of Philox4x64-10, counter (0,0,0,0), key
 *   (seed, 1); thresholds t_j = floor((j 2^32 + U) Q / (n 2^32)), j < n;
 *   birth i is drawn m_i = #{j : C_{i-1} <= t_j < C_i} times (C_i = q_0+..+q_i).
 * Output (capacity >= n): the r births with m_i > 0 in pool order (so sorted
 * by n0 when the pool is), amplitude a_i * ((m_i Q) / (n q_i)) with each
 * operation correctly rounded, then n - r padding entries that repeat the
 * last drawn birth (the pool's first when r = 0) with amplitude 0, which the
 * dipole calls skip.  The sum of the output amplitudes is an unbiased
 * estimate of the pool's over U.  A pool whose largest |a| is 0, infinite or
 * NaN draws nothing (r = 0).  Integer steps are exact: the result is the
 * same bit for bit on any device and launch configuration.
 *   pool: m entries (device; q0x / q0y are neither read nor written);
 *   n_distinct: optional device int64, receives r.
 * Uses the library's per-device scratch (about 28 bytes per pool entry);
 * calls that use it must not overlap on the GPU (as sfhk_dipole).
 * Errors: SFHK_EINVAL for NULL arrays, m < 1 (with n > 0), m or n >= 2^31,
 * capacities below m or n, or pool and out sharing arrays.  n = 0 writes
 * r = 0 and nothing else.
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_resample_births(const sfhk_births* pool, int64_t m, int64_t n, uint64_t seed,
                                 const sfhk_births* out, int64_t* n_distinct, void* stream);

/* ------------------------------------------------------------------------
 * Propagation (App. A: Hamilton's equations, the stability-matrix equations
 * for dq/dz, dp/dz with z = p0 or q0, the action S = int (p.qdot - H) dt;
 * Eq. C_HK: C = sqrt(det[(Mpp + Mqq - 2 i gamma Mqp - Mpq/(2 i gamma))/2])).
 * Classical RK4 with the grid step on the 43-component state; E is read at
 * t, t + dt/2, t + dt from the field's half-step table.  At every output
 * index (n % n_out == 0) and at the end, C is re-evaluated: C = +-sqrt(det Z),
 * the sign closer to the previous C (C(t0) = 1).  A trajectory is removed
 * (stops integrating and contributing) the first time |C|^2 = |det Z|
 * exceeds d_t, or when its state is not finite (Sec. III.A, Kay's removal).
 *   precision 0 FP64: everything in double.
 *   precision 2 DF (dipole, planar form only): double-float arithmetic on the
 *     FP32 pipe (48-bit significand, float exponent range) for the state;
 *     det Z and the recombination terms as in MIXED.  Regular trajectories
 *     agree with FP64 to ~1e-7 on the bins; chaotic ones drift further (see
 *     esc_precision), so it is no substitute for FP64 where they matter.
 *   precision 1 MIXED: stepping and stability blocks in float (FMA, rsqrt
 *     force, Kahan-compensated increments); action as a compensated two-float
 *     sum reduced mod 2 pi; det Z at the output bins from Z's float entries
 *     without cancellation loss (planar form: compensated float products,
 *     as accurate as twice the float precision; 3D form: FP64); recombination
 *     terms in float, accumulated in double; in the planar dipole pass the
 *     branch is followed with a float det every fifth step and at each bin
 *     (a turn by more than pi/2 between two evaluations counts as a branch
 *     guard event, see esc_ratio).  Births whose amplitude underflows float
 *     are not integrated.
 * deterministic: 0 = one double atomic add per bin per block (run-to-run
 * rounding order varies); 1 = per-block partial bins reduced in block order
 * (bit-reproducible; uses library-owned scratch of n_blocks*n_bins*16 bytes).
 * esc_ratio (MIXED dipole only; <= 0 disables): a float trajectory is
 * escalated at the first output bin where (a) |det Z| exceeds esc_ratio times
 * the free-particle spreading (1 + gamma^2 (t - t0)^2)^{3/2}, (b) the float
 * per-step det Z differs from the accurate one by more than 10%, or (c) a branch
 * guard event occurred.  It then stops; a high-precision pass over the
 * compacted list of escalated births recomputes them from birth and
 * contributes from that bin on (library-owned scratch: ~13 bytes per birth).
 * Measured against the FP64 path (H 800 nm, 8 cycles, 1e6 births; plateau
 * yields / phases): esc_ratio 30: 1e-5 / 1e-5 rad, 100: 4e-5 / 7e-5 rad,
 * 300: 1.1e-4 / 1.7e-4 rad, 1000: 5e-4 / 4e-4 rad; Ar 1600 nm 6 cycles, 2e5
 * births: below 1e-9 at all four.  The Python layer uses esc_ratio 200 with
 * esc_ratio_big 40 above esc_big 1000 (below) and esc_floor 1e-2: on a
 * 4096-birth H sample against the oracle, 2.7e-5 in the plateau yields (100
 * alone: 9.8e-4, the sample's weakest harmonics carried by one trajectory of
 * growth 40..45; 250 with the second ratio: 6.1e-4), with 12,112 escalations
 * at 1e6 births; on five 1e6-birth H samples at most 9.7e-5 / 2.4e-4 rad
 * against FP64.
 * The escalation pass runs in FP64 (esc_precision 0: in the planar form
 * without deterministic bins, a kernel that splits each step of 32
 * trajectories over four warps, same arithmetic; otherwise one thread per
 * trajectory), in double-float (esc_precision 1, planar form only; FP64 in the
 * 3D form), or in FP64 with one thread per trajectory always (esc_precision
 * 2).  Double-float carries ~48 significant bits: on chaotic trajectories its
 * results drift from FP64 (measured: 1.6e-3 in H plateau yields at 1e6
 * births), so FP64 is the default.  In every form the redo recomputes the
 * trajectory, stability blocks, prefactor and branch, and forms the
 * recombination terms of its bins in float from that state rounded to float
 * (the action reduced mod 2 pi first), as the float pass does for the other
 * trajectories.
 * esc_overlap (MIXED with escalation, not deterministic): how the redo
 * overlaps the float pass.  0: the births are cut into 8 chunks in birth
 * order, each chunk's float pass, compaction and redo chained on its own side
 * stream (earlier chunks at higher priority).  1: the float pass runs in 8
 * time segments (whole field windows) with every live trajectory's float
 * state saved in library-owned device memory between them (60 words per birth
 * in the planar form, 92 in 3D), and each segment's escalations are redone
 * at once on a side stream.  2: one float pass, then one compaction and one
 * redo of all escalated births, in order on the caller's stream.  Same
 * arithmetic and results in all three.
 * esc_floor (>= 0, finite): a flagged trajectory is escalated only while
 * |amp| |C| >= esc_floor * max_i |amp_i| (the maximum over the n births of
 * the call, reduced on the device); below the floor it goes on in float.
 * Trajectories whose contribution is negligible are then not redone; 0
 * escalates every flagged trajectory.
 * esc_big, esc_ratio_big (>= 0, finite; MIXED): a second growth threshold for
 * large contributions: where |amp| |C| >= esc_big * max_i |amp_i| (esc_big > 0),
 * criterion (a) uses esc_ratio_big in place of esc_ratio (when esc_ratio_big >
 * 0).  A few trajectories that carry a large part of the signal then leave
 * float at a smaller growth than the many that carry little.
 * pw_mask, pw_radius (dipole only; Sec. III.A-B partial-wave analysis): a
 * trajectory is labelled at every grid point where it enters r < pw_radius
 * (its birth counts when born inside) by its angular momentum L = |q x p|
 * there: class 0 (s) L < 0.5, 1 (p) 0.5 <= L < 1.5, 2 (d) 1.5 <= L < 2.5,
 * 3 otherwise.  With pw_mask != 0 (bits 0..3) it contributes at an output
 * bin only when it has been labelled and bit (latest class) of pw_mask is
 * set.  The label is taken in the working precision (float in MIXED).
 * geometry (dipole only): with the field along z and a central potential, a
 * birth at q0 = (0, 0, qz) moves in the plane of z and its transverse
 * momentum; 0 integrates such births in that plane (the monodromy matrix
 * splits into a 4x4 in-plane and a 2x2 out-of-plane block: 25 reals, same RK4
 * arithmetic, det Z = det(in-plane block of Z) * Z_yy) whenever q0x and q0y
 * are NULL; 1 always integrates the full 43-component state.  Endpoints
 * (sfhk_propagate) always use the full state.
 * block: threads per block (0 = library choice, 128; else 64 or 128).
 * chunk_steps: steps per shared-memory field window (0 = library choice;
 * else a multiple of n_out, 64..8192).
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t precision;       /* 0 FP64, 1 MIXED                              */
    int32_t deterministic;   /* 0 or 1                                       */
    double gamma;            /* coherent-state width (> 0)                   */
    double d_t;              /* removal threshold on |C|^2 (> 1)             */
    int32_t block;
    int32_t chunk_steps;
    double esc_ratio;        /* MIXED dipole only: escalation threshold (<= 0: off)  */
    int32_t geometry;        /* 0 auto (planar form when q0x = q0y = NULL), 1 full 3D */
    int32_t esc_precision;   /* escalation pass: 0 FP64, 1 double-float (planar form), 2 FP64 one thread per trajectory */
    double esc_floor;        /* MIXED escalation: amplitude floor relative to max |amp| (0: none) */
    double pw_radius;        /* partial-wave filter: radius of the near-core sphere (> 0)      */
    int32_t pw_mask;         /* partial-wave filter: bit c keeps class c (0: no filter)         */
    int32_t esc_overlap;     /* MIXED escalation schedule: 0 birth chunks, 1 time segments, 2 sequential */
    double esc_ratio_big;    /* MIXED: growth ratio for large contributions (see esc_big; <= 0: esc_ratio) */
    double esc_big;          /* MIXED: |amp| |C| >= esc_big * max|amp| marks a large contribution (0: none) */
} sfhk_prop_params;

/* Endpoints of sfhk_propagate (device arrays, n entries each):
 *   state  [43][n] double, component-major: q(3), p(3), Mqq(9), Mqp(9),
 *          Mpq(9), Mpp(9) (each row-major, [i][j] = d(.)_i/d(.)0_j), S;
 *          a removed trajectory keeps the state of its removal bin;
 *   c_re, c_im   the branch-tracked prefactor at the last accepted evaluation;
 *   flags  uint8: 1 removed, 2 non-finite, 4 branch guard (|d arg det Z| > pi/2
 *          between two evaluations: one grid step in FP64), 8 not integrated
 *          (amplitude zero).
 * n_end: grid index to integrate to (each birth from its n0; n0 <= n_end <= n_steps). */
typedef struct {
    double* state;
    double* c_re;
    double* c_im;
    uint8_t* flags;
    int64_t n_end;
} sfhk_endpoints;

/* Device-side counters, accumulated into (caller zeroes): */
typedef struct {
    unsigned long long removed;
    unsigned long long nonfinite;
    unsigned long long branch_guard;
    unsigned long long skipped;        /* births not integrated (zero amplitude) */
    unsigned long long traj_steps;     /* RK4 steps of live trajectories          */
    unsigned long long escalated;      /* MIXED: trajectories redone in high precision */
    unsigned long long esc_steps;      /* MIXED: RK4 steps of the high-precision redo  */
    unsigned long long esc_steps_pre;  /* MIXED: the part of esc_steps before the escalation bin
                                          (recomputed steps that contribute nothing) */
} sfhk_stats;

/* Integrates births [0, n) to endpoints.  `stats` is a DEVICE pointer or NULL. */
sfhk_status sfhk_propagate(const sfhk_field* field, const sfhk_target* target, const sfhk_births* births,
                           int64_t n, const sfhk_prop_params* params, const sfhk_endpoints* out,
                           sfhk_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Induced dipole (App. C, Eq. D_t and Eq. V_t) accumulated on the output bins:
 *   D(t_k) += -2 Re sum_traj e^{-i Ip t_k} <psi0| z |p_t,q_t,gamma> C e^{i S} amp
 *   v(t_k) += -2 Re sum_traj e^{-i Ip t_k} <psi0| k_z |p_t,q_t,gamma> C e^{i S} amp
 * over the trajectories alive at t_k >= t0, with the normalised coherent state
 * (2 gamma/pi)^{3/4} e^{-gamma (r-q)^2 + i p.(r-q)}.  d_len, d_vel: device
 * double[n_bins], accumulated into.  `stats`: device pointer or NULL.
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_dipole(const sfhk_field* field, const sfhk_target* target, const sfhk_births* births,
                        int64_t n, const sfhk_prop_params* params, double* d_len, double* d_vel,
                        sfhk_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Phase timing (measurement facility, no paper counterpart).  While enabled,
 * sfhk_dipole records CUDA timing events on its stream around its launches:
 * start of the call, after the trajectory pass (float pass on the mixed path),
 * after the escalation compaction, after the high-precision redo.  Per-phase
 * times are recorded for the sequential escalation schedule (esc_overlap 2),
 * deterministic bins and calls without escalation; the overlapped schedules
 * record the whole call only (phases = 0).  Nothing is recorded while the
 * stream is being captured into a CUDA graph.
 *   sfhk_set_phase_timing(on): 1 enables, 0 disables (process-wide).
 *   sfhk_get_phase_times(out): waits for the events of the last timed call on
 *     the current device and writes the device times in ms (host pointer).
 *     SFHK_EINVAL if no call has been timed on this device.
 * The events are library-owned, one set per device, reused by every call.
 * ---------------------------------------------------------------------- */
typedef struct {
    float traj_ms;      /* trajectory pass (with the amplitude maximum and clears before it) */
    float compact_ms;   /* escalation compaction (0 without escalation)                      */
    float redo_ms;      /* high-precision redo and the partial-bin reduction (0 without)      */
    float total_ms;     /* the whole call                                                     */
    int32_t phases;     /* 1: the three phases are valid; 0: only total_ms                    */
    int32_t reserved;
} sfhk_phase_times;
sfhk_status sfhk_set_phase_timing(int32_t on);
sfhk_status sfhk_get_phase_times(sfhk_phase_times* out);

/* ------------------------------------------------------------------------
 * Autotuner (library facility, no paper counterpart): times sfhk_dipole on the
 * first n_sample births for blocks of 64 and 128 trajectories and field
 * windows of 25, 50, 100, 200 and 400 output bins (chunk_steps = bins * n_out,
 * which also sets the shared-memory bin tile), escalation off, one warm-up and
 * one timed run each; keeps the fastest for (device, precision, planar form,
 * potential).  Later calls with block = chunk_steps = 0 use it.  Writes the
 * choice to best_block / best_chunk / best_ms (host pointers, may be NULL).
 * Synchronous; allocates 2 n_bins doubles for the duration of the call.
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_autotune(const sfhk_field* field, const sfhk_target* target, const sfhk_births* births,
                          int64_t n_sample, const sfhk_prop_params* params, int32_t* best_block, int32_t* best_chunk,
                          double* best_ms, void* stream);

/* ------------------------------------------------------------------------
 * Batched configurations (many laser configurations with uneven trajectory
 * counts and durations in one persistent launch).  sfhk_batch_create builds a
 * plan: per configuration its field, target, births (array of n_cfg records),
 * count n[c] and output bins d_len[c], d_vel[c] (device, accumulated into),
 * with common propagation parameters (precision 0 FP64 or 1 MIXED; block 0 or
 * 128; chunk_steps 0 (= 1000) must be a multiple of every configuration's
 * n_out).  It uploads one record per configuration and a work list of
 * (configuration, 128-birth block) items ordered by estimated remaining steps,
 * longest first, and allocates the escalation scratch (about 13 bytes per
 * birth).  `stats` (device pointer or NULL) receives the counters of every run.
 * sfhk_batch_run launches, on `stream`: the persistent kernel (grid = SMs x
 * resident blocks; each CTA takes the next item from an atomic counter), then,
 * for the mixed path, per configuration the compaction and escalation pass on
 * side streams joined back into `stream`.  A run allocates nothing and can be
 * captured in a CUDA graph once the plan exists.  The plan refers to the
 * caller's arrays; they must outlive it.
 * ---------------------------------------------------------------------- */
typedef struct sfhk_batch sfhk_batch;
sfhk_status sfhk_batch_create(int32_t n_cfg, const sfhk_field* const* fields, const sfhk_target* const* targets,
                              const sfhk_births* births, const int64_t* n, const sfhk_prop_params* params,
                              double* const* d_len, double* const* d_vel, sfhk_stats* stats, sfhk_batch** out);
sfhk_status sfhk_batch_run(sfhk_batch* batch, void* stream);
void sfhk_batch_destroy(sfhk_batch* batch);
/* One-shot form of the above (a batch of dipole configurations in one call):
 * creates the plan, runs it on `stream`, waits for the stream, destroys the
 * plan.  Synchronous; allocates and frees the plan's device memory itself, so
 * it is not for stream capture.  Arguments and errors as sfhk_batch_create. */
sfhk_status sfhk_dipole_batch(int32_t n_cfg, const sfhk_field* const* fields, const sfhk_target* const* targets,
                              const sfhk_births* births, const int64_t* n, const sfhk_prop_params* params,
                              double* const* d_len, double* const* d_vel, sfhk_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free dipole (the paper has no counterpart; this is a library
 * facility).  Same result as sfhk_dipole with deterministic = 1 (per-block
 * partial bins reduced in block order), for callers that cannot allocate
 * device memory at call time — e.g. a host whose device memory belongs to
 * another allocator that must account for every byte, or a latency-critical
 * loop that cannot afford cudaMalloc/cudaFree (they may synchronise the
 * device).  The partial bins live in a fixed 8 MiB __device__ array inside the
 * library (2^20 doubles; every GPU that loads the library holds it until the
 * process exits); nothing is allocated by this call.
 *   - Requires ceil(n / block) * 2 * n_bins <= 2^20, else SFHK_EINVAL; block
 *     is the one sfhk_dipole would launch with (params->block, else the
 *     autotuned block stored by sfhk_autotune for this configuration, else
 *     128), and so is the field window.  Escalation is not available here:
 *     with MIXED, esc_ratio must be <= 0 (else SFHK_EINVAL);
 *     params->deterministic is ignored (always deterministic).
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress); make that first call
 *     before any stream capture.
 *   - Every call shares the array and clears the part it uses; calls whose
 *     work overlaps on the GPU (e.g. on unordered streams) race on it.
 * Arguments and errors otherwise as sfhk_dipole.
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_dipole_static_scratch(const sfhk_field* field, const sfhk_target* target,
                                       const sfhk_births* births, int64_t n, const sfhk_prop_params* params,
                                       double* d_len, double* d_vel, sfhk_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Spectrum (App. D): X(w_m) = sum_k x(t_k) W_H(t_k) e^{i w_m t_k} dt_out with
 * t_k = t0 + k dt_out and W_H(t) = (1 + cos(pi t/tau_h))/2 for |t| <= tau_h,
 * else 0.  bins, omega: device double[n_bins], double[n_omega];
 * out_re, out_im: device double[n_omega] (overwritten).
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_spectrum(const double* bins, int64_t n_bins, double t0, double dt_out, double tau_h,
                          const double* omega, int64_t n_omega, double* out_re, double* out_im, void* stream);

/* ------------------------------------------------------------------------
 * Gabor time-frequency map (Sec. III.A, the map of the dipole velocity whose
 * bursts give the emission times):
 *   G(t_j, w_m) = sum_k x(t_k) exp(-(t_k - t_j)^2 / (2 sigma^2)) e^{i w_m t_k} dt_out
 * with t_k = t0 + k dt_out, summed over |t_k - t_j| <= 9 sigma (the window is
 * below e^{-40} beyond).  The paper gives no window width; 1/(3 w0), w0 the
 * laser frequency, is the customary choice.
 * bins: device double[n_bins]; times: device double[n_times]; omega: device
 * double[n_omega]; out_re, out_im: device double[n_times * n_omega], row j
 * holds time t_j (overwritten).  SFHK_EINVAL for negative sizes, NULL arrays,
 * dt_out <= 0 or sigma <= 0 or non-finite.
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_gabor(const double* bins, int64_t n_bins, double t0, double dt_out, double sigma,
                       const double* times, int64_t n_times, const double* omega, int64_t n_omega, double* out_re,
                       double* out_im, void* stream);

/* ------------------------------------------------------------------------
 * Emission time of a burst (Sec. III.A: the centre of a burst of the Gabor
 * map as a function of the harmonic energy).  For each frequency m, over the
 * analysis times t_j in [t_a, t_b] (times ascending):
 *   centroid[m] = sum_j t_j |G_jm|^2 / sum_j |G_jm|^2;
 *   peak[m]     = the t_j of the largest |G_jm|^2, moved to the vertex of the
 *                 parabola through ln|G|^2 at t_{j-1}, t_j, t_{j+1} when both
 *                 neighbours are in the window, equally spaced, and the
 *                 parabola opens downwards (exact for a Gaussian burst).
 * NaN where the window holds no time or |G| vanishes on it.
 * g_re, g_im: device double[n_times * n_omega] as written by sfhk_gabor;
 * times: device double[n_times]; centroid, peak: device double[n_omega].
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_emission_time(const double* g_re, const double* g_im, int64_t n_times, int64_t n_omega,
                               const double* times, double t_a, double t_b, double* centroid, double* peak,
                               void* stream);

/* ------------------------------------------------------------------------
 * Verification utility (Eq. C_HK, planar form; no counterpart of its own in the
 * paper): det Z = det(2x2 in-plane block of Z) * Z_yy from float entries, as
 * the MIXED float pass evaluates it at every output bin (power-of-two scaling
 * and error-free products and sums: the in-plane determinant is as accurate as
 * if evaluated in twice the float precision, then rounded to float).
 *   z: device float[10][n], component-major: Re Z00, Re Z01, Re Z10, Re Z11,
 *      Im Z00, Im Z01, Im Z10, Im Z11, Re Z_yy, Im Z_yy;
 *   re, im, e: device double[n], double[n], int32[n] (overwritten):
 *      det Z = (re + i im) 2^(2 e), re and im the float results widened.
 * Entries of magnitude >= 1e38 or non-finite give NaN in re.  Errors:
 * SFHK_EINVAL for n < 0 or NULL arrays with n > 0.
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_det_z_planar_f32(const float* z, int64_t n, double* re, double* im, int32_t* e, void* stream);

/* ------------------------------------------------------------------------
 * Measurement utility (no counterpart in the paper): FMA-issue throughput of
 * the current device, kind 0 = FP32 FFMA, 1 = FP64 DFMA, from dependent
 * FMA chains with 8-way ILP over 8 blocks of 256 threads per SM; best of
 * three timed launches after one warm-up.  Writes TFLOP/s (2 flops per FMA)
 * and the launch time in ms (host pointers).  Synchronous; allocates 16 bytes.
 * ---------------------------------------------------------------------- */
sfhk_status sfhk_peak_flops(int32_t kind, double* tflops, float* ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SFHK_H */
