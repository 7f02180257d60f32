// Hanning-windowed Fourier transform of the dipole bins (App. D):
//   X(w_m) = sum_k x(t_k) W_H(t_k) e^{i w_m t_k} dt_out,
//   W_H(t) = (1 + cos(pi t / tau_H)) / 2 for |t| <= tau_H, else 0.
// One frequency per thread; the windowed bins are staged in shared memory in
// tiles shared by the block; e^{i w t_k} advances by a complex rotation and is
// re-anchored with an exact sincos every 64 bins.
#include "sfhk_device.cuh"

namespace sfhk {
namespace {

constexpr int kTile = 1024;

__global__ void spectrum_kernel(const double* __restrict__ x, int64_t n_bins, double t0, double dt, double tau,
                                const double* __restrict__ omega, int64_t n_omega, double* out_re,
                                double* out_im) {
    __shared__ double sx[kTile];
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double w = m < n_omega ? omega[m] : 0.0;
    double sr = 0.0, si = 0.0;
    double rs, rc;
    sincos(w * dt, &rs, &rc);                 // rotation per bin
    for (int64_t k0 = 0; k0 < n_bins; k0 += kTile) {
        const int nt = (int)((n_bins - k0) < kTile ? (n_bins - k0) : kTile);
        __syncthreads();
        for (int u = threadIdx.x; u < nt; u += blockDim.x) {
            double t = t0 + (double)(k0 + u) * dt;
            double W = fabs(t) <= tau ? 0.5 * (1.0 + cospi(t / tau)) : 0.0;
            sx[u] = x[k0 + u] * W * dt;
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
    if (m < n_omega) {
        out_re[m] = sr;
        out_im[m] = si;
    }
}

}  // namespace

cudaError_t launch_spectrum(const double* bins, int64_t n_bins, double t0, double dt_out, double tau_h,
                            const double* omega, int64_t n_omega, double* out_re, double* out_im,
                            cudaStream_t s) {
    if (n_omega == 0) return cudaSuccess;
    const int block = 128;
    spectrum_kernel<<<(unsigned)((n_omega + block - 1) / block), block, 0, s>>>(bins, n_bins, t0, dt_out, tau_h,
                                                                                 omega, n_omega, out_re, out_im);
    return cudaGetLastError();
}

}  // namespace sfhk
