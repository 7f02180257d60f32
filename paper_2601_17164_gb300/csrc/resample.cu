// Importance sampling of births in proportion to |I0| (App. A, Eq. Int: the
// weight |I0| of a momentum that solves the saddle-point equation turns the
// Monte Carlo integral into importance sampling), as systematic resampling of
// a proposal pool of m births down to n.
//
//   w_i = |a_i| (a_i = the pool amplitude, |I0| times the proposal weight),
//   q_i = floor(w_i 2^B / max w) with B = 62 - ceil(log2 m), Q = sum q_i < 2^62,
//   one uniform U in [0, 2^32) (Philox4x64-10, key (seed, 1), counter 0, the
//   high half of word 0), thresholds t_j = floor((j 2^32 + U) Q / (n 2^32)),
//   m_i = #{j : C_{i-1} <= t_j < C_i} with C_i = q_0 + ... + q_i,
//   output: the births with m_i > 0 in pool order, amplitude a_i m_i Q / (n q_i).
//
// Every integer step is exact (64-bit sums, 128-bit threshold counts) and the
// few floating-point steps are single correctly rounded operations, so the
// result does not depend on the launch configuration.  The count of
// thresholds below c has the closed form
//   J(c) = clamp(ceil((ceil(c n 2^32 / Q) - U) / 2^32), 0, n),
// so m_i = J(C_i) - J(C_{i-1}) needs only the inclusive prefix sum of q.
//
// Launches: weights and their maximum; quantisation with per-block sums; a
// one-block scan of the block sums; multiplicities (block-local scan plus the
// block offset); the order-preserving compaction of the drawn births; the
// gather with the amplitude rescaling and the zero-amplitude padding.
#include "sfhk_device.cuh"
#include "sfhk_internal.cuh"

namespace sfhk {
namespace {

constexpr int kRB = 1024;   // pool entries per block of the scan kernels (= threads)

__global__ void weight_kernel(const double* __restrict__ re, const double* __restrict__ im, int64_t m,
                              double* __restrict__ w, unsigned long long* amax_bits) {
    unsigned long long mb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        // separate products and sum (no fused multiply-add), correctly rounded root
        const double x = __dsqrt_rn(__dadd_rn(__dmul_rn(re[i], re[i]), __dmul_rn(im[i], im[i])));
        w[i] = x;
        // non-negative doubles order as their bit patterns; a NaN (either sign) is above them all
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        if (b > mb) mb = b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o);
        if (t > mb) mb = t;
    }
    if ((threadIdx.x & 31) == 0 && mb) atomicMax(amax_bits, mb);
}

// 2^B / A (one correctly rounded division); 0 when A is zero, infinite or NaN
__device__ __forceinline__ double quant_scale(unsigned long long amax_bits, int B) {
    const double A = __longlong_as_double((long long)amax_bits);
    if (!(A > 0.0) || !isfinite(A)) return 0.0;
    return __ddiv_rn(ldexp(1.0, B), A);
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sh) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wp] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    return t;
}

__global__ void quant_kernel(const double* __restrict__ w, int64_t m, const unsigned long long* amax_bits, int B,
                             unsigned long long* __restrict__ q, unsigned long long* __restrict__ blk) {
    __shared__ unsigned long long sh[32];
    const double s = quant_scale(*amax_bits, B);
    const int64_t i = (int64_t)blockIdx.x * kRB + threadIdx.x;
    unsigned long long v = 0;
    if (i < m) {
        if (s > 0.0) v = (unsigned long long)floor(__dmul_rn(w[i], s));
        q[i] = v;
    }
    const unsigned long long t = block_sum_u64(v, sh);
    if (threadIdx.x == 0) blk[blockIdx.x] = t;
}

// inclusive scan of 1024 values per block (warp scans, then the warp totals)
__device__ __forceinline__ unsigned long long block_incl_scan_u64(unsigned long long v, unsigned long long* wt) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[wp] = x;
    __syncthreads();
    if (wp == 0) {
        unsigned long long t = wt[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wt[lane] = t;
    }
    __syncthreads();
    return x + (wp > 0 ? wt[wp - 1] : 0ull);
}

// exclusive scan of blk[0..nb) in place; the total Q into blk[nb]
__global__ void scan_u64_kernel(unsigned long long* blk, int64_t nb) {
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kRB) {
        const int64_t k = base + threadIdx.x;
        const unsigned long long v = k < nb ? blk[k] : 0ull;
        const unsigned long long incl = block_incl_scan_u64(v, wt);
        const unsigned long long c = carry;
        if (k < nb) blk[k] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == kRB - 1) carry = c + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) blk[nb] = carry;
}

// J(c) = #{j : t_j < c} in closed form (128-bit intermediate, c n 2^32 < 2^125)
__device__ __forceinline__ int64_t thresholds_below(unsigned long long c, unsigned long long Q, int64_t n,
                                                    unsigned long long U) {
    const unsigned __int128 num = ((unsigned __int128)c * (unsigned __int128)(unsigned long long)n) << 32;
    const unsigned __int128 L = (num + (unsigned __int128)(Q - 1)) / (unsigned __int128)Q;   // ceil(c n 2^32 / Q)
    if (L <= (unsigned __int128)U) return 0;
    const unsigned __int128 k = (L - (unsigned __int128)U + (((unsigned __int128)1 << 32) - 1)) >> 32;
    return k >= (unsigned __int128)(unsigned long long)n ? n : (int64_t)k;
}

__device__ __forceinline__ unsigned long long resample_uniform(uint64_t seed) {
    uint64_t c[4] = {0, 0, 0, 0};
    philox4x64_10(c, seed, 1);
    return (unsigned long long)(c[0] >> 32);
}

// m_i into mult[i] (-1 where m_i = 0)
__global__ void mult_kernel(const unsigned long long* __restrict__ q, int64_t m, const unsigned long long* blk,
                            int64_t nb, int64_t n, uint64_t seed, int32_t* __restrict__ mult) {
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long sU;
    if (threadIdx.x == 0) sU = resample_uniform(seed);
    const int64_t i = (int64_t)blockIdx.x * kRB + threadIdx.x;
    const unsigned long long v = i < m ? q[i] : 0ull;
    const unsigned long long incl = block_incl_scan_u64(v, wt);   // (its barriers publish sU)
    if (i >= m) return;
    const unsigned long long Q = blk[nb];
    int32_t r = -1;
    if (Q > 0 && v > 0) {
        const unsigned long long c = blk[blockIdx.x] + incl;
        const int64_t k = thresholds_below(c, Q, n, sU) - thresholds_below(c - v, Q, n, sU);
        if (k > 0) r = (int32_t)k;
    }
    mult[i] = r;
}

__global__ void gather_kernel(BirthArgs pool, int64_t n, const int32_t* __restrict__ idx,
                              const int32_t* __restrict__ times_drawn, const int32_t* count,
                              const unsigned long long* __restrict__ q, const unsigned long long* Qp, BirthArgs out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t r = *count;
    if (j < r) {
        const int64_t i = idx[j];
        const double f = __ddiv_rn(__dmul_rn((double)times_drawn[j], __ull2double_rn(*Qp)),
                                   __dmul_rn((double)n, __ull2double_rn(q[i])));
        out.n0[j] = pool.n0[i];
        out.t0[j] = pool.t0[i];
        out.px[j] = pool.px[i];
        out.py[j] = pool.py[i];
        out.pz[j] = pool.pz[i];
        out.qz[j] = pool.qz[i];
        out.amp_re[j] = __dmul_rn(pool.amp_re[i], f);
        out.amp_im[j] = __dmul_rn(pool.amp_im[i], f);
    } else {
        // padding: the last drawn birth (or the pool's first) with zero amplitude
        const int64_t i = r > 0 ? (int64_t)idx[r - 1] : 0;
        out.n0[j] = pool.n0[i];
        out.t0[j] = pool.t0[i];
        out.px[j] = pool.px[i];
        out.py[j] = pool.py[i];
        out.pz[j] = pool.pz[i];
        out.qz[j] = pool.qz[i];
        out.amp_re[j] = 0.0;
        out.amp_im[j] = 0.0;
    }
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

int resample_scale_bits(int64_t m) {
    int k = 0;   // ceil(log2 max(2, m)), at least 1
    while (((int64_t)1 << k) < (m < 2 ? 2 : m)) ++k;
    return 62 - (k < 1 ? 1 : k);
}

size_t resample_scratch_bytes(int64_t m) {
    const int64_t nb = (m + kRB - 1) / kRB;
    return al256((size_t)m * 8) * 2 + al256((size_t)(nb + 1) * 8) + al256((size_t)m * 4) * 3 +
           al256((size_t)(compact_blocks(m) + 16) * 4) + 512;
}

cudaError_t launch_resample(const BirthArgs& pool, int64_t m, int64_t n, uint64_t seed, const BirthArgs& out,
                            unsigned char* scratch, int64_t* n_distinct, cudaStream_t s) {
    const int64_t nb = (m + kRB - 1) / kRB;
    unsigned char* p = scratch;
    double* w = reinterpret_cast<double*>(p);
    p += al256((size_t)m * 8);
    unsigned long long* q = reinterpret_cast<unsigned long long*>(p);
    p += al256((size_t)m * 8);
    unsigned long long* blk = reinterpret_cast<unsigned long long*>(p);
    p += al256((size_t)(nb + 1) * 8);
    int32_t* mult = reinterpret_cast<int32_t*>(p);
    p += al256((size_t)m * 4);
    int32_t* idx = reinterpret_cast<int32_t*>(p);
    p += al256((size_t)m * 4);
    int32_t* kf = reinterpret_cast<int32_t*>(p);
    p += al256((size_t)m * 4);
    int32_t* cblk = reinterpret_cast<int32_t*>(p);
    p += al256((size_t)(compact_blocks(m) + 16) * 4);
    int32_t* count = reinterpret_cast<int32_t*>(p);
    unsigned long long* amax = reinterpret_cast<unsigned long long*>(p + 256);

    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t want = (m + 255) / 256;
    weight_kernel<<<(unsigned)(want < 1216 ? want : 1216), 256, 0, s>>>(pool.amp_re, pool.amp_im, m, w, amax);
    quant_kernel<<<(unsigned)nb, kRB, 0, s>>>(w, m, amax, resample_scale_bits(m), q, blk);
    scan_u64_kernel<<<1, kRB, 0, s>>>(blk, nb);
    mult_kernel<<<(unsigned)nb, kRB, 0, s>>>(q, m, blk, nb, n, seed, mult);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // births with m_i >= 1, in pool order: idx = pool index, kf = m_i, *count = distinct draws
    e = launch_compact(mult, m, cblk, idx, kf, count, s, 1, INT32_MAX);
    if (e != cudaSuccess) return e;
    gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pool, n, idx, kf, count, q, blk + nb, out);
    e = cudaGetLastError();
    if (e != cudaSuccess || n_distinct == nullptr) return e;
    e = cudaMemsetAsync(n_distinct, 0, sizeof(int64_t), s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(n_distinct, count, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);   // little-endian low word
}

}  // namespace sfhk
