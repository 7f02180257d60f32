// FMA-throughput microbenchmarks: the measured FP32 / FP64 issue peaks that
// the trajectory kernels' roofline fractions are quoted against.
//
// Each thread runs 8 independent dependent-FMA chains (enough ILP to hide the
// FMA latency); the grid fills every SM several times over.  The result is
// flops = 2 * threads * 8 chains * iterations / elapsed time.
#include "sfhk_internal.cuh"

namespace sfhk {
namespace {

template <typename R>
__global__ void fma_chains(R* out, int iters, R a, R b) {
    R x0 = (R)threadIdx.x, x1 = x0 + R(1), x2 = x0 + R(2), x3 = x0 + R(3);
    R x4 = x0 + R(4), x5 = x0 + R(5), x6 = x0 + R(6), x7 = x0 + R(7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    R s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == R(-12345.678)) out[0] = s;   // keeps the chains alive
}

}  // namespace
}  // namespace sfhk

using namespace sfhk;

extern "C" sfhk_status sfhk_peak_flops(int32_t kind, double* tflops, float* ms_out, void* stream) {
    if (!tflops || (kind != 0 && kind != 1)) return fail(SFHK_EINVAL, "kind must be 0 (fp32) or 1 (fp64)");
    int dev, sms;
    sfhk_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    st = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int block = 256;
    const int grid = sms * 8;
    const int iters = kind == 0 ? 4096 : 128;
    void* out = nullptr;
    st = check_cuda(cudaMalloc(&out, 16), "alloc");
    if (st) return st;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        if (kind == 0)
            fma_chains<float><<<grid, block, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
        else
            fma_chains<double><<<grid, block, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;   // first launch is warm-up
    }
    st = check_cuda(cudaGetLastError(), "peak kernel");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (st) return st;
    double flops = 2.0 * (double)grid * block * 8.0 * 16.0 * iters;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return SFHK_OK;
}
