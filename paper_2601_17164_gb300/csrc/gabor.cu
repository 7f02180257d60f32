// Gabor time-frequency analysis of the dipole bins and emission times of a
// burst (Sec. III.A, the time-frequency maps of the dipole velocity and the
// burst centres as functions of the harmonic energy).
//
//   G(t_j, w_m) = sum_k x(t_k) exp(-(t_k - t_j)^2 / (2 sigma^2)) e^{i w_m t_k} dt_out
//
// summed over the bins with |t_k - t_j| <= 9 sigma (the window is below
// e^{-40} beyond).  Block = one analysis time t_j x 128 frequencies; the
// windowed bins of t_j are staged in shared memory in tiles; e^{i w t_k}
// advances by a complex rotation, re-anchored with an exact sincos every 64
// bins.  Emission time: one thread per frequency scans |G(t_j, w)|^2 over the
// analysis times in [t_a, t_b] for the centroid and the peak (vertex of the
// parabola through ln|G|^2 at the maximum and its two neighbours).
#include "sfhk_device.cuh"

namespace sfhk {
namespace {

constexpr int kGTile = 1024;
constexpr double kGaborCut = 9.0;   // window half-width in units of sigma

__global__ void gabor_kernel(const double* __restrict__ x, int64_t n_bins, double t0, double dt, double sigma,
                             const double* __restrict__ times, int64_t n_t, const double* __restrict__ omega,
                             int64_t n_omega, double* out_re, double* out_im) {
    __shared__ double sx[kGTile];
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double w = m < n_omega ? omega[m] : 0.0;
    double rs, rc;
    sincos(w * dt, &rs, &rc);                       // rotation per bin
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    for (int64_t j = blockIdx.y; j < n_t; j += gridDim.y) {
        const double tj = times[j];
        double lo = ceil((tj - kGaborCut * sigma - t0) / dt), hi = floor((tj + kGaborCut * sigma - t0) / dt);
        lo = fmax(lo, 0.0);
        hi = fmin(hi, (double)(n_bins - 1));
        double sr = 0.0, si = 0.0;
        if (lo <= hi) {
            const int64_t k_lo = (int64_t)lo, k_hi = (int64_t)hi;
            for (int64_t k0 = k_lo; k0 <= k_hi; k0 += kGTile) {
                const int nt = (int)((k_hi - k0 + 1) < kGTile ? (k_hi - k0 + 1) : kGTile);
                __syncthreads();
                for (int u = threadIdx.x; u < nt; u += blockDim.x) {
                    const double d = (t0 + (double)(k0 + u) * dt) - tj;
                    sx[u] = x[k0 + u] * exp(-d * d * inv2s2) * dt;
                }
                __syncthreads();
                double er = 0.0, ei = 0.0;
                for (int u = 0; u < nt; ++u) {
                    if ((u & 63) == 0) sincos(w * (t0 + (double)(k0 + u) * dt), &ei, &er);
                    const double v = sx[u];
                    sr = fma(v, er, sr);
                    si = fma(v, ei, si);
                    const double nr = fma(er, rc, -ei * rs);
                    ei = fma(er, rs, ei * rc);
                    er = nr;
                }
            }
        }
        if (m < n_omega) {
            out_re[j * n_omega + m] = sr;
            out_im[j * n_omega + m] = si;
        }
    }
}

__global__ void emission_kernel(const double* __restrict__ g_re, const double* __restrict__ g_im, int64_t n_t,
                                int64_t n_omega, const double* __restrict__ times, double t_a, double t_b,
                                double* centroid, double* peak) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_omega) return;
    auto P = [&](int64_t j) {
        const double r = g_re[j * n_omega + m], i = g_im[j * n_omega + m];
        return r * r + i * i;
    };
    double s0 = 0.0, s1 = 0.0, pmax = -1.0;
    int64_t jmax = -1, j_first = -1, j_last = -1;
    for (int64_t j = 0; j < n_t; ++j) {
        const double t = times[j];
        if (!(t >= t_a && t <= t_b)) continue;
        if (j_first < 0) j_first = j;
        j_last = j;
        const double p = P(j);
        s0 += p;
        s1 = fma(t, p, s1);
        if (p > pmax) {
            pmax = p;
            jmax = j;
        }
    }
    double cen = nan(""), pk = nan("");
    if (jmax >= 0 && s0 > 0.0) {
        cen = s1 / s0;
        pk = times[jmax];
        if (jmax > j_first && jmax < j_last) {
            const double pm = P(jmax - 1), pp = P(jmax + 1);
            if (pm > 0.0 && pp > 0.0) {
                const double ym = log(pm), y0 = log(pmax), yp = log(pp);
                const double h = times[jmax + 1] - times[jmax];
                const double curv = ym - 2.0 * y0 + yp;
                if (curv < 0.0 && fabs(times[jmax] - times[jmax - 1] - h) <= 1e-9 * fabs(h))
                    pk = times[jmax] + 0.5 * h * (ym - yp) / curv;
            }
        }
    }
    centroid[m] = cen;
    peak[m] = pk;
}

}  // namespace

cudaError_t launch_gabor(const double* bins, int64_t n_bins, double t0, double dt_out, double sigma,
                         const double* times, int64_t n_t, const double* omega, int64_t n_omega, double* out_re,
                         double* out_im, cudaStream_t s) {
    if (n_omega == 0 || n_t == 0) return cudaSuccess;
    const int block = 128;
    const unsigned gx = (unsigned)((n_omega + block - 1) / block);
    const unsigned gy = (unsigned)(n_t < 65535 ? n_t : 65535);
    gabor_kernel<<<dim3(gx, gy), block, 0, s>>>(bins, n_bins, t0, dt_out, sigma, times, n_t, omega, n_omega,
                                                out_re, out_im);
    return cudaGetLastError();
}

cudaError_t launch_emission_time(const double* g_re, const double* g_im, int64_t n_t, int64_t n_omega,
                                 const double* times, double t_a, double t_b, double* centroid, double* peak,
                                 cudaStream_t s) {
    if (n_omega == 0) return cudaSuccess;
    const int block = 128;
    emission_kernel<<<(unsigned)((n_omega + block - 1) / block), block, 0, s>>>(g_re, g_im, n_t, n_omega, times,
                                                                                 t_a, t_b, centroid, peak);
    return cudaGetLastError();
}

}  // namespace sfhk
