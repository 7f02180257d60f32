// Internal declarations of the SFHK CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "sfhk.h"

namespace sfhk {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kMaxGto = 32;

// Error plumbing: every C entry point funnels failures through fail().
sfhk_status fail(sfhk_status s, const char* fmt, ...);
sfhk_status check_cuda(cudaError_t e, const char* what);
sfhk_status check_launch(const char* what);
// Library-owned device status word per device (bounded waits report here).
unsigned int* device_status();
// An NVTX range named after a C-ABI entry point, open for the entry's lifetime
// (seen by profilers on the host timeline; no cost without one attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Step-size constants of the classical RK4 step and of the planar step matrix:
// h, h/2, h/6, h^2/6, h^3/12, h^4/24, each evaluated left to right in R.  Made
// once on the host (float and FP64 copies in the field record) so that the step
// loops read them from the kernel parameters instead of re-deriving them.
template <typename R>
struct StepK {
    R h, hh, h6, c2, c3, c4;
};

// Field: sin^2 pulse, grid and device half-step tables.
struct FieldDev {
    double E0, omega, Tp, cep;
    double t_start, dt, t_out;
    float dt32;               // dt rounded to float, made on the host (the float kernels read it as a parameter)
    StepK<float> k32;         // step constants from dt32 in float arithmetic
    StepK<double> k64;        // step constants from dt in FP64
    int64_t n_steps, n_out, n_bins;
    int n_modes;              // A(t) = sum_j a_j sin(w_j t + cep)
    double a[3], w[3];
    const double* E64;        // E(t_start + j dt/2), j = 0..2 n_steps (+ padding)
    const float* E32;
    int64_t table_len;        // allocated entries (>= 2 n_steps + 1)
};

struct TargetDev {
    int pot, gto_l, n_gto, amp;
    double pot_param[8];
    float pot_param32[8];     // pot_param rounded to float, and a2_32 = (float)(pot_param[0]^2),
    float a2_32;              // made on the host so that the float kernels convert nothing
    double ip;
    double c[kMaxGto], alpha[kMaxGto];
};

}  // namespace sfhk

struct sfhk_field {
    int device;
    sfhk::FieldDev f;
    double* d_E64;
    float* d_E32;
};

struct sfhk_target {
    int device;
    sfhk::TargetDev t;
};

namespace sfhk {

// ---- argument checks shared by the entry points (api.cu) ----------------------
sfhk_status check_handles(const sfhk_field* f, const sfhk_target* t);
// births arrays for n births (amplitudes too when need_amp)
sfhk_status check_births(const sfhk_births* b, int64_t n, bool need_amp);
// propagation parameters; writes the requested block and field-window steps
sfhk_status check_prop(const sfhk_prop_params* pp, const FieldDev& f, int* block, int* chunk);
// the autotuned shape for (device, precision, planar form, potential) when the
// caller leaves block = chunk_steps = 0 and sfhk_autotune has stored one
void tuned_shape(const sfhk_prop_params* pp, const FieldDev& f, int pot, int planar, int* block, int* chunk);

// ---- launches implemented in the .cu files ---------------------------------
struct BirthArgs {
    int64_t n;            // births in the whole sample
    int64_t first, count; // produced range
    int mode, n_t, n_k;
    double sigma, kmax;
    uint64_t seed;
    int32_t* n0;
    double *t0, *px, *py, *pz, *qz, *amp_re, *amp_im;
};
cudaError_t launch_births(const FieldDev& f, const TargetDev& t, const BirthArgs& a, cudaStream_t s);
// |I0| resampling of a pool of m births to n (resample.cu)
int resample_scale_bits(int64_t m);
size_t resample_scratch_bytes(int64_t m);
cudaError_t launch_resample(const BirthArgs& pool, int64_t m, int64_t n, uint64_t seed, const BirthArgs& out,
                            unsigned char* scratch, int64_t* n_distinct, cudaStream_t s);

// Precomputed recombination constants for a target and coherent-state width.
struct GtoTerms {
    int n, l;
    double kp[kMaxGto];   // -1/(4 beta_j)          (multiplies p^2)
    double kq[kMaxGto];   // -alpha_j gamma/beta_j  (multiplies q^2)
    double kx[kMaxGto];   // -alpha_j/beta_j        (multiplies p.q, imaginary part)
    double w0[kMaxGto], w1[kMaxGto], w2[kMaxGto], w3[kMaxGto];
    double nl, nv;        // length / velocity prefactors (normalisation)
    // the same in float for the float recombination terms (no conversions in the loop)
    float kpf[kMaxGto], kqf[kMaxGto], kxf[kMaxGto], w0f[kMaxGto], w1f[kMaxGto], w2f[kMaxGto], w3f[kMaxGto];
    float nlf, nvf;
};
GtoTerms make_gto_terms(const TargetDev& t, double gamma);

struct TrajArgs {
    // births
    int64_t n;
    const int32_t* n0;
    const double *px, *py, *pz, *qx, *qy, *qz, *amp_re, *amp_im;
    // physics
    double gamma, d_t;
    float gamma32, qg32;  // (float)gamma and (float)(1/(4 gamma)), made on the host
    double qg64;          // 1/(4 gamma) in FP64, made on the host
    // outputs
    int mode;             // 0 endpoints, 1 dipole
    int64_t n_last;       // last grid index
    double *d_len, *d_vel;
    double* part;         // deterministic partial bins [grid][2][n_bins] or null
    double *st_out, *c_re, *c_im;
    uint8_t* flags;
    sfhk_stats* stats;
    int block, chunk;
    // escalation: the mixed pass writes, per birth, the first output bin at which
    // the trajectory left the float regime (-1: never); the FP64 pass takes the
    // compacted list (idx, k_from, *count) and contributes from bin k_from on
    int32_t* esc_bin;
    double esc_ratio;
    // escalate only when |amp| |C| >= esc_floor * sqrt(*esc_amax2) (esc_amax2: device max |amp|^2
    // over the births of the call; null: no floor)
    const double* esc_amax2;
    double esc_floor;
    // second growth threshold esc_ratio_big for |amp| |C| >= esc_big * max|amp| (esc_big 0: off)
    double esc_ratio_big, esc_big;
    // made on the host: log2 of esc_ratio, of the ratio of large contributions and of the
    // smaller of the two, and the weight thresholds log2(esc_floor^2) (-1e30: no floor) and
    // log2(esc_big^2) (1e30: none)
    float esc_l2, esc_l2_big, esc_l2_lo, esc_l2_floor, esc_l2_bigw;
    const int32_t* idx;
    const int32_t* k_from;
    const int32_t* count;
    int planar;           // 1: births at q0 = (0,0,qz) in dipole mode, integrated in the planar form
    int float_bins;       // FP64 escalation redo: recombination terms in float, as the float pass forms them
    int pw_mask;          // partial-wave filter (bit c keeps class c; 0 none) and its sphere radius
    double pw_radius;
    // time segment of a segmented float pass: grid points [seg_lo, seg_hi] (seg_lo a
    // multiple of chunk); trajectories born before seg_lo resume from `state`
    // (kStateWords 32-bit words per birth, word-major with stride n), and the state at
    // seg_hi + 1 is saved there unless seg_hi >= n_last.  state == null: one launch.
    int64_t seg_lo, seg_hi;
    uint32_t* state;
    // four-warp FP64 redo: the number of group lists (the SM count) and
    // redo_scratch_words(n) ints of device scratch: one counter per list (the launch
    // clears them), then the plan that assigns the list's groups to the lists
    int redo_lists;
    int* redo_ctr;
};
cudaError_t launch_traj(const FieldDev& f, const TargetDev& t, int precision, const TrajArgs& a,
                        cudaStream_t s);
// 32-bit words of saved state per birth in a segmented float pass (planar or 3D form)
int state_words(int planar);
// FP64 redo of an escalation list (planar form, atomic bins) with the work of each
// step split across the four warps of a block (redo.cu); blocks of 32 list entries
cudaError_t launch_redo(const FieldDev& f, const TargetDev& t, const TrajArgs& a, cudaStream_t s);
// group lists of the four-warp redo: one per SM of the current device, at most kRedoLists
constexpr int kRedoLists = 256;
int redo_lists();
// ints of device scratch the four-warp redo of a list of up to n births needs
inline size_t redo_scratch_words(int64_t n) { return 3 * (size_t)kRedoLists + 2 * (size_t)((n + 31) / 32 + 1); }
int64_t redo_blocks(int64_t n);
// The high-precision pass over an escalation list: esc_precision 0 FP64 (the split
// kernel where it applies: planar form, atomic bins), 1 double-float (planar form;
// FP64 in the 3D form), 2 FP64 with one thread per trajectory.
// The redo recomputes the trajectory, prefactor and branch in FP64 and forms the
// recombination terms of its bins in float, from the FP64 state rounded to float
// (the action reduced mod 2 pi in FP64 first), as the float pass does for every
// other trajectory.
inline cudaError_t launch_escalation(const FieldDev& f, const TargetDev& t, int esc_precision, const TrajArgs& a,
                                     cudaStream_t s) {
    TrajArgs e = a;
    e.float_bins = 1;
    if (esc_precision == 0 && e.planar && e.part == nullptr && e.mode == 1) return launch_redo(f, t, e, s);
    if (esc_precision == 1 && e.planar) return launch_traj(f, t, 2, e, s);
    return launch_traj(f, t, 0, e, s);
}
cudaError_t launch_compact(const int32_t* esc_bin, int64_t n, int32_t* blk, int32_t* idx, int32_t* k_from,
                           int32_t* count, cudaStream_t s, int32_t k_lo = 0, int32_t k_hi = INT32_MAX);
int64_t compact_blocks(int64_t n);
cudaError_t launch_amp_max(const double* amp_re, const double* amp_im, int64_t n, double* out, cudaStream_t s);
cudaError_t launch_reduce_partials(const double* part, int64_t n_blocks, int64_t n_bins, double* d_len,
                                   double* d_vel, cudaStream_t s);
cudaError_t launch_spectrum(const double* bins, int64_t n_bins, double t0, double dt_out, double tau_h,
                            const double* omega, int64_t n_omega, double* out_re, double* out_im,
                            cudaStream_t s);
cudaError_t launch_gabor(const double* bins, int64_t n_bins, double t0, double dt_out, double sigma,
                         const double* times, int64_t n_t, const double* omega, int64_t n_omega, double* out_re,
                         double* out_im, cudaStream_t s);
cudaError_t launch_emission_time(const double* g_re, const double* g_im, int64_t n_t, int64_t n_omega,
                                 const double* times, double t_a, double t_b, double* centroid, double* peak,
                                 cudaStream_t s);

}  // namespace sfhk
