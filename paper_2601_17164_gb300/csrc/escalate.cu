// Order-preserving compaction of the escalated births of a mixed-precision
// pass: from esc_bin[i] (first bin in high precision, or -1), restricted to
// escalation bins in [k_lo, k_hi], to the list
// idx[0..count), k_from[0..count) in increasing birth index (hence n0) order,
// so that the FP64 pass over the list keeps its blocks in lockstep.
// Three launches: per-block counts, one-block exclusive scan, scatter.
#include "sfhk_internal.cuh"

namespace sfhk {
namespace {

// births per compaction block (= threads): small blocks, so that a compaction
// launched beside a running float pass fits into the registers one finished
// trajectory block frees (a 1024-thread block would wait for the pass to drain)
constexpr int kB = 128;

// max_i |amp_i|^2 over the births into *out (non-negative doubles order as
// their bit patterns, so an integer atomicMax suffices); *out starts at 0
__global__ void amp_max_kernel(const double* __restrict__ re, const double* __restrict__ im, int64_t n,
                               unsigned long long* out) {
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a2 = re[i] * re[i] + im[i] * im[i];
        if (a2 > m) m = a2;     // NaN never wins
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__device__ __forceinline__ bool listed(int32_t e, int32_t k_lo, int32_t k_hi) { return e >= k_lo && e <= k_hi; }

__global__ void count_kernel(const int32_t* __restrict__ esc, int64_t n, int32_t* blk, int32_t k_lo, int32_t k_hi) {
    const int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x;
    const int c = __syncthreads_count(i < n && listed(esc[i], k_lo, k_hi));
    if (threadIdx.x == 0) blk[blockIdx.x] = c;
}

// exclusive scan of blk[0..nb) in place; total to *count
__global__ void scan_kernel(int32_t* blk, int64_t nb, int32_t* count) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += kB) {
        const int64_t k = base + threadIdx.x;
        const int32_t v = k < nb ? blk[k] : 0;
        int32_t x = v;   // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            int32_t t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;   // inclusive over warps
        }
        __syncthreads();
        const int32_t before = carry + (w > 0 ? warp_tot[w - 1] : 0) + x - v;
        if (k < nb) blk[k] = before;
        __syncthreads();
        if (threadIdx.x == kB - 1) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = carry;
}

__global__ void scatter_kernel(const int32_t* __restrict__ esc, int64_t n, const int32_t* __restrict__ blk,
                               int32_t* idx, int32_t* k_from, int32_t k_lo, int32_t k_hi) {
    __shared__ int32_t warp_cnt[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x;
    const bool f = i < n && listed(esc[i], k_lo, k_hi);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_cnt[w] = __popc(m);
    __syncthreads();
    int32_t off = blk[blockIdx.x];
    for (int k = 0; k < w; ++k) off += warp_cnt[k];
    off += __popc(m & ((1u << lane) - 1u));
    if (f) {
        idx[off] = (int32_t)i;
        k_from[off] = esc[i];
    }
}

}  // namespace

cudaError_t launch_amp_max(const double* amp_re, const double* amp_im, int64_t n, double* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
    if (e != cudaSuccess || n == 0) return e;
    const int64_t want = (n + 255) / 256;
    const unsigned grid = (unsigned)(want < 1216 ? want : 1216);   // 8 blocks per SM at most
    amp_max_kernel<<<grid, 256, 0, s>>>(amp_re, amp_im, n, reinterpret_cast<unsigned long long*>(out));
    return cudaGetLastError();
}

int64_t compact_blocks(int64_t n) { return (n + kB - 1) / kB; }

cudaError_t launch_compact(const int32_t* esc_bin, int64_t n, int32_t* blk, int32_t* idx, int32_t* k_from,
                           int32_t* count, cudaStream_t s, int32_t k_lo, int32_t k_hi) {
    const int64_t nb = compact_blocks(n);
    if (nb == 0) return cudaMemsetAsync(count, 0, sizeof(int32_t), s);
    count_kernel<<<(unsigned)nb, kB, 0, s>>>(esc_bin, n, blk, k_lo, k_hi);
    scan_kernel<<<1, kB, 0, s>>>(blk, nb, count);
    scatter_kernel<<<(unsigned)nb, kB, 0, s>>>(esc_bin, n, blk, idx, k_from, k_lo, k_hi);
    return cudaGetLastError();
}

}  // namespace sfhk
