// Verification utility: the mixed path's planar det Z from given float entries.
//
// The float pass evaluates det Z (Eq. C_HK; planar form: the 2x2 in-plane block
// of Z times Z_yy) at every output bin from Z's float entries with error-free
// transformations (power-of-two scaling, TwoProd by FMA, TwoSum), so that the
// in-plane determinant carries no cancellation loss.  This entry runs that
// same device function on caller-given entries, so that a test can hold it
// against the exact determinant of the same float values.
#include <algorithm>

#include "sfhk_internal.cuh"
#include "traj_block.cuh"

namespace sfhk {
namespace {

__global__ void detz_kernel(const float* __restrict__ z, int64_t n, double* re, double* im, int32_t* ex) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float zr[2][2], zi[2][2];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            zr[k >> 1][k & 1] = z[(size_t)k * n + i];
            zi[k >> 1][k & 1] = z[(size_t)(4 + k) * n + i];
        }
        const ScaledDet d = det_planar_comp(zr, zi, z[(size_t)8 * n + i], z[(size_t)9 * n + i]);
        re[i] = (double)d.re;
        im[i] = (double)d.im;
        ex[i] = d.e;
    }
}

}  // namespace
}  // namespace sfhk

using namespace sfhk;

extern "C" sfhk_status sfhk_det_z_planar_f32(const float* z, int64_t n, double* re, double* im, int32_t* e,
                                             void* stream) {
    if (n < 0) return fail(SFHK_EINVAL, "n must be >= 0");
    if (n >= ((int64_t)1 << 40)) return fail(SFHK_EINVAL, "n too large");
    if (n == 0) return SFHK_OK;
    if (!z || !re || !im || !e) return fail(SFHK_EINVAL, "NULL array");
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    detz_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(z, n, re, im, e);
    return check_launch("det Z launch");
}
