// Launches of the trajectory block (traj_block.cuh) over one configuration:
// the trajectory kernel, the deterministic reduction of per-block partial
// bins, and the recombination constants of a target.
#include "traj_block.cuh"

namespace sfhk {
namespace {

template <typename R, int POT, bool PLANAR>
__global__ void __launch_bounds__(128, std::is_same<R, float>::value ? (PLANAR ? 4 : 3) : (PLANAR ? 2 : 1))
    traj_kernel(FieldDev f, TargetDev tg, GtoTerms gt, TrajArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_nmin;
    traj_block<R, POT, PLANAR>(f, tg, gt, a, (int64_t)blockIdx.x, smem, s_nmin);
}

__global__ void reduce_partials_kernel(const double* part, int64_t n_blocks, int64_t n_bins, double* d_len,
                                       double* d_vel) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_bins) return;
    double sl = 0.0, sv = 0.0;
    for (int64_t b = 0; b < n_blocks; ++b) {
        sl += part[(b * 2) * n_bins + k];
        sv += part[(b * 2 + 1) * n_bins + k];
    }
    d_len[k] += sl;
    d_vel[k] += sv;
}

template <typename R, int POT, bool PLANAR>
cudaError_t launch_one(const FieldDev& f, const TargetDev& t, const GtoTerms& gt, const TrajArgs& a,
                       cudaStream_t s) {
    const int block = a.block;
    const int nw = block / 32;
    const int nbw = a.chunk / (int)f.n_out;
    using RC = typename std::conditional<std::is_same<R, dfloat>::value, float, R>::type;
    size_t smem = ((size_t)(2 * a.chunk + 2) * sizeof(R) + 15) / 16 * 16 + (size_t)nw * 2 * nbw * sizeof(double) +
                  (size_t)nbw * sizeof(Cx<RC>);
    auto kern = traj_kernel<R, POT, PLANAR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (a.n + block - 1) / block;
    kern<<<(unsigned)grid, block, smem, s>>>(f, t, gt, a);
    return cudaGetLastError();
}

template <typename R, bool PLANAR>
cudaError_t launch_geo(const FieldDev& f, const TargetDev& t, const GtoTerms& gt, const TrajArgs& a,
                       cudaStream_t s) {
    switch (t.pot) {
        case POT_SOFTCORE: return launch_one<R, POT_SOFTCORE, PLANAR>(f, t, gt, a, s);
        case POT_TONGLIN: return launch_one<R, POT_TONGLIN, PLANAR>(f, t, gt, a, s);
        case POT_HARMONIC: return launch_one<R, POT_HARMONIC, PLANAR>(f, t, gt, a, s);
        default: return launch_one<R, POT_ZERO, PLANAR>(f, t, gt, a, s);
    }
}

template <typename R>
cudaError_t launch_prec(const FieldDev& f, const TargetDev& t, const GtoTerms& gt, const TrajArgs& a,
                        cudaStream_t s) {
    return a.planar ? launch_geo<R, true>(f, t, gt, a, s) : launch_geo<R, false>(f, t, gt, a, s);
}

}  // namespace

GtoTerms make_gto_terms(const TargetDev& t, double gamma) {
    GtoTerms g{};
    g.n = t.n_gto;
    g.l = t.gto_l;
    const double pi32 = 5.5683279968317078;                 // pi^{3/2}
    const double N = pow(2.0 * gamma / kPi, 0.75);           // coherent-state normalisation
    for (int j = 0; j < t.n_gto; ++j) {
        double al = t.alpha[j], be = gamma + al;
        g.kp[j] = -0.25 / be;
        g.kq[j] = -al * gamma / be;
        g.kx[j] = -al / be;
        double b52 = pow(be, -2.5), b72 = pow(be, -3.5);
        if (t.gto_l == 0) {
            g.w0[j] = t.c[j] * b52;            // sum c b^{-5/2} e^X
            g.w1[j] = t.c[j] * al * b52;       // sum c a b^{-5/2} e^X
        } else {
            g.w0[j] = t.c[j] * b72;            // b_z^2 sum c b^{-7/2} e^X
            g.w1[j] = 2.0 * be * t.c[j] * b72; // + sum 2 b c b^{-7/2} e^X
            g.w2[j] = t.c[j] * al * b72;       // u_z^2/(2 gamma) sum c a b^{-7/2} e^X
            g.w3[j] = t.c[j] * b52;            // + sum c b^{-5/2} e^X
        }
    }
    g.nl = N * pi32 * (t.gto_l == 0 ? 0.5 : 0.25);
    g.nv = N * pi32;
    for (int j = 0; j < t.n_gto; ++j) {
        g.kpf[j] = (float)g.kp[j];
        g.kqf[j] = (float)g.kq[j];
        g.kxf[j] = (float)g.kx[j];
        g.w0f[j] = (float)g.w0[j];
        g.w1f[j] = (float)g.w1[j];
        g.w2f[j] = (float)g.w2[j];
        g.w3f[j] = (float)g.w3[j];
    }
    g.nlf = (float)g.nl;
    g.nvf = (float)g.nv;
    return g;
}

// the kernel scalars (flags word, Dp, sgn, zc) and every member of the float trajectory
static_assert(sizeof(TrajP<float, POT_ZERO>) == 55 * 4, "planar float state layout");
static_assert(sizeof(Traj<float, POT_ZERO>) == 87 * 4, "3D float state layout");
int state_words(int planar) {
    return 5 + (int)((planar ? sizeof(TrajP<float, POT_ZERO>) : sizeof(Traj<float, POT_ZERO>)) / 4);
}

cudaError_t launch_traj(const FieldDev& f, const TargetDev& t, int precision, const TrajArgs& a,
                        cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    GtoTerms gt = make_gto_terms(t, a.gamma);
    if (precision == 2) {   // double-float, planar form only
        switch (t.pot) {
            case POT_SOFTCORE: return launch_one<dfloat, POT_SOFTCORE, true>(f, t, gt, a, s);
            case POT_TONGLIN: return launch_one<dfloat, POT_TONGLIN, true>(f, t, gt, a, s);
            case POT_HARMONIC: return launch_one<dfloat, POT_HARMONIC, true>(f, t, gt, a, s);
            default: return launch_one<dfloat, POT_ZERO, true>(f, t, gt, a, s);
        }
    }
    return precision == 0 ? launch_prec<double>(f, t, gt, a, s) : launch_prec<float>(f, t, gt, a, s);
}

cudaError_t launch_reduce_partials(const double* part, int64_t n_blocks, int64_t n_bins, double* d_len,
                                   double* d_vel, cudaStream_t s) {
    const int block = 256;
    reduce_partials_kernel<<<(unsigned)((n_bins + block - 1) / block), block, 0, s>>>(part, n_blocks, n_bins,
                                                                                      d_len, d_vel);
    return cudaGetLastError();
}

}  // namespace sfhk
