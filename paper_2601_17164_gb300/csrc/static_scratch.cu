// Allocation-free variant of the deterministic dipole reduction.
//
// Some callers cannot allocate device memory at call time: a host whose device
// memory is owned by another allocator that must account for every byte (a
// framework's caching allocator, a fixed memory budget handed out at start-up),
// or a latency-critical loop that cannot afford cudaMalloc / cudaFree, which
// may synchronise the whole device.  sfhk_dipole_static_scratch() serves them:
// the per-block partial bins of the deterministic reduction live in a
// file-scope __device__ array of fixed size (8 MiB, held by every GPU that
// loads the library until the process exits) instead of library-allocated
// scratch.  The device address of that array is looked up once per device
// (cudaGetSymbolAddress) the first time the entry point runs with that device
// current; nothing is allocated, by this file or by the launches it makes.
//
// The array is shared by every call in the process on a given device and keeps
// the previous call's contents; each call clears the part it uses first.  Two
// calls whose work overlaps on the GPU (different streams, no ordering) race on
// the array.
#include <mutex>
#include <vector>

#include "sfhk_internal.cuh"

namespace sfhk {
namespace {

// 2^20 doubles (8 MiB): n_blocks * 2 * n_bins partial sums must fit.
constexpr size_t kStaticPartials = (size_t)1 << 20;
__device__ __align__(256) double g_static_partials[kStaticPartials];

std::mutex g_sym_mu;
std::vector<double*> g_sym_addr;   // per device; nullptr until looked up

// Device address of g_static_partials for the current device (looked up once).
sfhk_status static_partials(double** out) {
    int dev;
    sfhk_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    std::lock_guard<std::mutex> lk(g_sym_mu);
    if ((int)g_sym_addr.size() <= dev) g_sym_addr.resize(dev + 1, nullptr);
    if (!g_sym_addr[dev]) {
        void* p = nullptr;
        st = check_cuda(cudaGetSymbolAddress(&p, g_static_partials), "cudaGetSymbolAddress");
        if (st) return st;
        g_sym_addr[dev] = static_cast<double*>(p);
    }
    *out = g_sym_addr[dev];
    return SFHK_OK;
}

}  // namespace
}  // namespace sfhk

using namespace sfhk;

extern "C" sfhk_status sfhk_dipole_static_scratch(const sfhk_field* field, const sfhk_target* target,
                                                  const sfhk_births* b, int64_t n, const sfhk_prop_params* pp,
                                                  double* d_len, double* d_vel, sfhk_stats* stats,
                                                  void* stream) {
    NvtxRange nvtx_range("sfhk_dipole_static_scratch");
    // the checks of sfhk_dipole, in its order
    sfhk_status st = check_handles(field, target);
    if (st) return st;
    st = check_births(b, n, true);
    if (st) return st;
    if (!d_len || !d_vel) return fail(SFHK_EINVAL, "bins are NULL");
    if (n == 0) return SFHK_OK;
    int block, chunk;
    st = check_prop(pp, field->f, &block, &chunk);
    if (st) return st;
    // what this entry cannot do without allocating
    if (pp->precision == 1 && pp->esc_ratio > 0.0)
        return fail(SFHK_EINVAL, "escalation needs per-birth scratch: use sfhk_dipole, or esc_ratio <= 0");
    const int planar = (b->q0x == nullptr && b->q0y == nullptr && pp->geometry == 0) ? 1 : 0;   // as sfhk_dipole
    if (pp->precision == 2 && !planar) return fail(SFHK_EUNSUPPORTED, "precision 2 needs the planar form");
    // the launch shape sfhk_dipole would use (the autotuned one when block = chunk_steps = 0)
    tuned_shape(pp, field->f, target->t.pot, planar, &block, &chunk);
    const int64_t n_blocks = (n + block - 1) / block;
    const size_t need = (size_t)n_blocks * 2 * (size_t)field->f.n_bins;
    if (need > kStaticPartials)
        return fail(SFHK_EINVAL, "n_blocks*2*n_bins = %zu exceeds the static scratch of %zu doubles", need,
                    kStaticPartials);
    double* part = nullptr;
    st = static_partials(&part);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = check_cuda(cudaMemsetAsync(part, 0, need * sizeof(double), s), "clear static scratch");
    if (st) return st;
    TrajArgs a{};
    a.n = n;
    a.n0 = b->n0;
    a.px = b->p0x;
    a.py = b->p0y;
    a.pz = b->p0z;
    a.qx = b->q0x;
    a.qy = b->q0y;
    a.qz = b->q0z;
    a.amp_re = b->amp_re;
    a.amp_im = b->amp_im;
    a.gamma = pp->gamma;
    a.gamma32 = (float)pp->gamma;
    a.qg32 = (float)(0.25 / pp->gamma);
    a.qg64 = 1.0 / (4.0 * pp->gamma);
    a.d_t = pp->d_t;
    a.pw_mask = pp->pw_mask;
    a.pw_radius = pp->pw_radius;
    a.mode = 1;
    a.n_last = field->f.n_steps;
    a.d_len = d_len;
    a.d_vel = d_vel;
    a.part = part;
    a.stats = stats;
    a.block = block;
    a.chunk = chunk;
    a.planar = planar;
    st = check_cuda(launch_traj(field->f, target->t, pp->precision, a, s), "trajectory launch");
    if (st) return st;
    return check_cuda(launch_reduce_partials(part, n_blocks, field->f.n_bins, d_len, d_vel, s), "reduce launch");
}
