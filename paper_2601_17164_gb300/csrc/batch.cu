// Batched configurations in one persistent launch.
//
// A batch plan holds, in device memory, one record per configuration (field,
// target, recombination constants, trajectory arguments) and a work list of
// (configuration, block of 128 births) items ordered longest-first by their
// estimated remaining steps.  The persistent kernel keeps a grid of
// SMs x resident-blocks CTAs busy: each CTA takes the next item from an atomic
// counter, copies that configuration's record to shared memory and runs the
// block exactly as the single-configuration kernel does.  Escalated births of
// the mixed path are then compacted and redone per configuration on side
// streams.  All launches of a run are stream-ordered and allocation-free, so a
// run can be captured in a CUDA graph after the plan exists.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "traj_block.cuh"

namespace sfhk {
namespace {

struct alignas(16) BatchCfg {
    FieldDev f;
    TargetDev t;
    GtoTerms g;
    TrajArgs a;
};

template <typename R, bool PLANAR>
__global__ void __launch_bounds__(128, std::is_same<R, float>::value ? (PLANAR ? 4 : 3) : (PLANAR ? 2 : 1))
    batch_kernel(const BatchCfg* __restrict__ cfgs, const int2* __restrict__ items, int n_items, int* head) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_nmin;
    __shared__ int s_item;
    __shared__ __align__(16) BatchCfg s_cfg;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 w = items[it];
        const int4* src = reinterpret_cast<const int4*>(cfgs + w.x);
        int4* dst = reinterpret_cast<int4*>(&s_cfg);
        for (int u = threadIdx.x; u < (int)(sizeof(BatchCfg) / 16); u += blockDim.x) dst[u] = src[u];
        __syncthreads();
        switch (s_cfg.t.pot) {
            case POT_SOFTCORE: traj_block<R, POT_SOFTCORE, PLANAR>(s_cfg.f, s_cfg.t, s_cfg.g, s_cfg.a, w.y, smem, s_nmin); break;
            case POT_TONGLIN: traj_block<R, POT_TONGLIN, PLANAR>(s_cfg.f, s_cfg.t, s_cfg.g, s_cfg.a, w.y, smem, s_nmin); break;
            case POT_HARMONIC: traj_block<R, POT_HARMONIC, PLANAR>(s_cfg.f, s_cfg.t, s_cfg.g, s_cfg.a, w.y, smem, s_nmin); break;
            default: traj_block<R, POT_ZERO, PLANAR>(s_cfg.f, s_cfg.t, s_cfg.g, s_cfg.a, w.y, smem, s_nmin); break;
        }
    }
}

template <typename R, bool PLANAR>
cudaError_t launch_batch(const BatchCfg* cfgs, const int2* items, int n_items, int* head, int chunk, int max_nbw,
                         cudaStream_t s) {
    const int block = 128, nw = block / 32;
    using RC = typename std::conditional<std::is_same<R, dfloat>::value, float, R>::type;
    const size_t smem = ((size_t)(2 * chunk + 2) * sizeof(R) + 15) / 16 * 16 +
                        (size_t)nw * 2 * max_nbw * sizeof(double) + (size_t)max_nbw * sizeof(Cx<RC>);
    auto kern = batch_kernel<R, PLANAR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev, sms, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem)) != cudaSuccess) return e;
    const int grid = std::max(1, std::min(n_items, sms * std::max(per_sm, 1)));
    kern<<<grid, block, smem, s>>>(cfgs, items, n_items, head);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sfhk

using namespace sfhk;

struct sfhk_batch {
    int device;
    int n_cfg;
    int precision, planar, chunk, max_nbw, n_items;
    double esc_ratio, esc_floor, esc_ratio_big, esc_big;
    int esc_precision;
    std::vector<BatchCfg> host_cfg;
    std::vector<int64_t> n;
    BatchCfg* d_cfg = nullptr;
    int2* d_items = nullptr;
    int* d_head = nullptr;
    // escalation scratch, per configuration slices
    int32_t *d_esc = nullptr, *d_idx = nullptr, *d_kfrom = nullptr, *d_blk = nullptr, *d_count = nullptr;
    double* d_amax2 = nullptr;   // per configuration max |amp|^2 (escalation floor)
    int* d_rctr = nullptr;       // counters and group plan of the four-warp redo, one set per side stream
    size_t rctr_words = 0;       // ints per side stream
    std::vector<int64_t> esc_off, blk_off;
    cudaStream_t side[8] = {};
    cudaEvent_t fork = nullptr, done[8] = {};
};

static void batch_free(sfhk_batch* b) {
    if (!b) return;
    cudaFree(b->d_cfg);
    cudaFree(b->d_items);
    cudaFree(b->d_head);
    cudaFree(b->d_esc);
    cudaFree(b->d_amax2);
    cudaFree(b->d_idx);
    cudaFree(b->d_kfrom);
    cudaFree(b->d_blk);
    cudaFree(b->d_count);
    cudaFree(b->d_rctr);
    for (int i = 0; i < 8; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->done[i]) cudaEventDestroy(b->done[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

extern "C" {

sfhk_status sfhk_batch_create(int32_t n_cfg, const sfhk_field* const* fields, const sfhk_target* const* targets,
                              const sfhk_births* births, const int64_t* n, const sfhk_prop_params* pp,
                              double* const* d_len, double* const* d_vel, sfhk_stats* stats, sfhk_batch** out) {
    NvtxRange nvtx_range("sfhk_batch_create");
    if (!out) return fail(SFHK_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_cfg < 1 || n_cfg > 4096) return fail(SFHK_EINVAL, "n_cfg must be 1..4096");
    if (!fields || !targets || !births || !n || !pp || !d_len || !d_vel) return fail(SFHK_EINVAL, "NULL argument");
    if (pp->precision != 0 && pp->precision != 1) return fail(SFHK_EINVAL, "batch precision must be 0 or 1");
    if (!(pp->gamma > 0) || !(pp->d_t > 1.0) || !isfinite(pp->esc_ratio) || !isfinite(pp->esc_floor) ||
        pp->esc_floor < 0 || !isfinite(pp->esc_ratio_big) || !isfinite(pp->esc_big) || pp->esc_big < 0 || pp->pw_mask < 0 || pp->pw_mask > 15 ||
        (pp->pw_mask && !(pp->pw_radius > 0 && isfinite(pp->pw_radius))))
        return fail(SFHK_EINVAL, "bad params");
    if (pp->block != 0 && pp->block != 128) return fail(SFHK_EINVAL, "batch block must be 0 or 128");
    if (pp->esc_precision < 0 || pp->esc_precision > 2) return fail(SFHK_EINVAL, "esc_precision must be 0, 1 or 2");
    int dev;
    sfhk_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    sfhk_batch* b = new (std::nothrow) sfhk_batch();
    if (!b) return fail(SFHK_ENOMEM, "host allocation");
    b->device = dev;
    b->n_cfg = n_cfg;
    b->precision = pp->precision;
    b->esc_ratio = pp->precision == 1 ? pp->esc_ratio : 0.0;
    b->esc_precision = pp->esc_precision;
    b->esc_floor = pp->esc_floor;
    b->esc_ratio_big = pp->esc_ratio_big;
    b->esc_big = pp->esc_big;
    b->chunk = pp->chunk_steps ? pp->chunk_steps : 1000;
    b->planar = pp->geometry == 0 ? 1 : 0;
    b->max_nbw = 0;
    int64_t total = 0;
    std::vector<std::pair<double, int2>> items;
    for (int c = 0; c < n_cfg; ++c) {
        const sfhk_field* F = fields[c];
        const sfhk_target* T = targets[c];
        const sfhk_births& B = births[c];
        if (!F || !T || F->device != dev || T->device != dev) {
            batch_free(b);
            return fail(SFHK_EINVAL, "configuration %d: bad handle or device", c);
        }
        if (n[c] < 0 || n[c] > B.capacity || n[c] >= ((int64_t)1 << 31)) {
            batch_free(b);
            return fail(SFHK_EINVAL, "configuration %d: bad birth count", c);
        }
        if (n[c] > 0 && (!B.n0 || !B.p0x || !B.p0y || !B.p0z || !B.q0z || !B.amp_re || !B.amp_im || !d_len[c] ||
                         !d_vel[c])) {
            batch_free(b);
            return fail(SFHK_EINVAL, "configuration %d: NULL arrays", c);
        }
        if (B.q0x || B.q0y) b->planar = 0;
        if (b->chunk % F->f.n_out != 0 || b->chunk < 64 || b->chunk > 8192) {
            batch_free(b);
            return fail(SFHK_EINVAL, "chunk_steps %d must be a multiple of every n_out (config %d: %lld)", b->chunk, c,
                        (long long)F->f.n_out);
        }
        b->max_nbw = std::max(b->max_nbw, (int)(b->chunk / F->f.n_out));
        BatchCfg cfg{};
        cfg.f = F->f;
        cfg.t = T->t;
        cfg.g = make_gto_terms(T->t, pp->gamma);
        TrajArgs& a = cfg.a;
        a.n = n[c];
        a.n0 = B.n0;
        a.px = B.p0x;
        a.py = B.p0y;
        a.pz = B.p0z;
        a.qx = B.q0x;
        a.qy = B.q0y;
        a.qz = B.q0z;
        a.amp_re = B.amp_re;
        a.amp_im = B.amp_im;
        a.gamma = pp->gamma;
        a.gamma32 = (float)pp->gamma;
        a.qg32 = (float)(0.25 / pp->gamma);
        a.qg64 = 1.0 / (4.0 * pp->gamma);
        a.d_t = pp->d_t;
        a.pw_mask = pp->pw_mask;
        a.pw_radius = pp->pw_radius;
        a.mode = 1;
        a.n_last = F->f.n_steps;
        a.d_len = d_len[c];
        a.d_vel = d_vel[c];
        a.block = 128;
        a.chunk = b->chunk;
        a.stats = stats;
        b->host_cfg.push_back(cfg);
        b->n.push_back(n[c]);
        b->esc_off.push_back(total);
        total += n[c];
        // items: blocks of 128 births; births sorted by n0 and spread over the
        // pulse, so block k of K has about (1 - k/K) of the grid left
        const int64_t nb = (n[c] + 127) / 128;
        for (int64_t k = 0; k < nb; ++k)
            items.push_back({(double)F->f.n_steps * (1.0 - (double)k / (double)nb), int2{c, (int)k}});
    }
    std::stable_sort(items.begin(), items.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    b->n_items = (int)items.size();
    std::vector<int2> it(items.size());
    for (size_t k = 0; k < items.size(); ++k) it[k] = items[k].second;
    const bool esc = b->esc_ratio > 0.0;
    int64_t blk_total = 0;
    for (int c = 0; c < n_cfg; ++c) {
        b->blk_off.push_back(blk_total);
        blk_total += compact_blocks(b->n[c]) + 1;
    }
    st = check_cuda(cudaMalloc(&b->d_cfg, sizeof(BatchCfg) * n_cfg), "batch alloc");
    if (!st) st = check_cuda(cudaMalloc(&b->d_items, sizeof(int2) * std::max<size_t>(1, it.size())), "batch alloc");
    if (!st) st = check_cuda(cudaMalloc(&b->d_head, sizeof(int)), "batch alloc");
    if (!st && esc) {
        st = check_cuda(cudaMalloc(&b->d_esc, sizeof(int32_t) * std::max<int64_t>(1, total)), "batch alloc");
        if (!st) st = check_cuda(cudaMalloc(&b->d_idx, sizeof(int32_t) * std::max<int64_t>(1, total)), "batch alloc");
        if (!st) st = check_cuda(cudaMalloc(&b->d_kfrom, sizeof(int32_t) * std::max<int64_t>(1, total)), "alloc");
        if (!st) st = check_cuda(cudaMalloc(&b->d_blk, sizeof(int32_t) * std::max<int64_t>(1, blk_total)), "alloc");
        if (!st) st = check_cuda(cudaMalloc(&b->d_count, sizeof(int32_t) * n_cfg), "batch alloc");
        if (!st) st = check_cuda(cudaMalloc(&b->d_amax2, sizeof(double) * n_cfg), "batch alloc");
        int64_t n_max = 0;
        for (int c = 0; c < n_cfg; ++c) n_max = std::max(n_max, b->n[c]);
        b->rctr_words = redo_scratch_words(n_max);
        if (!st) st = check_cuda(cudaMalloc(&b->d_rctr, sizeof(int) * 8 * b->rctr_words), "batch alloc");
        for (int c = 0; c < n_cfg && !st; ++c) {
            b->host_cfg[c].a.esc_bin = b->d_esc + b->esc_off[c];
            b->host_cfg[c].a.esc_ratio = b->esc_ratio;
            b->host_cfg[c].a.esc_l2 = b->esc_ratio > 0.0 ? (float)log2(b->esc_ratio) : 0.f;
            b->host_cfg[c].a.esc_l2_big =
                b->esc_ratio_big > 0.0 ? (float)log2(b->esc_ratio_big) : b->host_cfg[c].a.esc_l2;
            b->host_cfg[c].a.esc_l2_lo =
                b->esc_big > 0.0 ? fminf(b->host_cfg[c].a.esc_l2, b->host_cfg[c].a.esc_l2_big) : b->host_cfg[c].a.esc_l2;
            b->host_cfg[c].a.esc_l2_floor = b->esc_floor > 0.0 ? (float)log2(b->esc_floor * b->esc_floor) : -1e30f;
            b->host_cfg[c].a.esc_l2_bigw = b->esc_big > 0.0 ? (float)log2(b->esc_big * b->esc_big) : 1e30f;
            if (b->esc_floor > 0.0 || b->esc_big > 0.0) {
                b->host_cfg[c].a.esc_amax2 = b->d_amax2 + c;
                b->host_cfg[c].a.esc_floor = b->esc_floor;
                b->host_cfg[c].a.esc_big = b->esc_big;
                b->host_cfg[c].a.esc_ratio_big = b->esc_ratio_big;
            }
        }
        for (int i = 0; i < 8 && !st; ++i) {
            st = check_cuda(cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking), "side stream");
            if (!st) st = check_cuda(cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming), "event");
        }
        if (!st) st = check_cuda(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
    }
    for (auto& cfg : b->host_cfg) cfg.a.planar = b->planar;
    if (!st) st = check_cuda(cudaMemcpy(b->d_cfg, b->host_cfg.data(), sizeof(BatchCfg) * n_cfg,
                                        cudaMemcpyHostToDevice), "batch upload");
    if (!st && !it.empty())
        st = check_cuda(cudaMemcpy(b->d_items, it.data(), sizeof(int2) * it.size(), cudaMemcpyHostToDevice),
                        "batch upload");
    if (st) {
        batch_free(b);
        return st;
    }
    *out = b;
    return SFHK_OK;
}

sfhk_status sfhk_batch_run(sfhk_batch* b, void* stream) {
    NvtxRange nvtx_range("sfhk_batch_run");
    if (!b) return fail(SFHK_EINVAL, "batch is NULL");
    int dev;
    sfhk_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    if (dev != b->device) return fail(SFHK_EINVAL, "batch belongs to device %d", b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const bool esc = b->esc_ratio > 0.0;
    st = check_cuda(cudaMemsetAsync(b->d_head, 0, sizeof(int), s), "queue reset");
    if (st) return st;
    if (esc) {
        int64_t total = b->esc_off.back() + b->n.back();
        st = check_cuda(cudaMemsetAsync(b->d_esc, 0xff, sizeof(int32_t) * std::max<int64_t>(1, total), s), "clear");
        if (st) return st;
        for (int c = 0; c < b->n_cfg && (b->esc_floor > 0.0 || b->esc_big > 0.0); ++c) {
            const TrajArgs& a = b->host_cfg[c].a;
            st = check_cuda(launch_amp_max(a.amp_re, a.amp_im, b->n[c], b->d_amax2 + c, s), "amplitude maximum");
            if (st) return st;
        }
    }
    if (b->n_items > 0) {
        cudaError_t e;
        if (b->precision == 1)
            e = b->planar ? launch_batch<float, true>(b->d_cfg, b->d_items, b->n_items, b->d_head, b->chunk,
                                                      b->max_nbw, s)
                          : launch_batch<float, false>(b->d_cfg, b->d_items, b->n_items, b->d_head, b->chunk,
                                                       b->max_nbw, s);
        else
            e = b->planar ? launch_batch<double, true>(b->d_cfg, b->d_items, b->n_items, b->d_head, b->chunk,
                                                       b->max_nbw, s)
                          : launch_batch<double, false>(b->d_cfg, b->d_items, b->n_items, b->d_head, b->chunk,
                                                        b->max_nbw, s);
        st = check_cuda(e, "batch launch");
        if (st) return st;
    }
    if (!esc) return SFHK_OK;
    // escalated births: per configuration compaction and high-precision pass,
    // spread over the side streams
    st = check_cuda(cudaEventRecord(b->fork, s), "event record");
    if (st) return st;
    for (int i = 0; i < 8; ++i) {
        st = check_cuda(cudaStreamWaitEvent(b->side[i], b->fork, 0), "stream wait");
        if (st) return st;
    }
    for (int c = 0; c < b->n_cfg; ++c) {
        if (b->n[c] == 0) continue;
        cudaStream_t side = b->side[c % 8];
        const BatchCfg& cfg = b->host_cfg[c];
        st = check_cuda(launch_compact(b->d_esc + b->esc_off[c], b->n[c], b->d_blk + b->blk_off[c],
                                       b->d_idx + b->esc_off[c], b->d_kfrom + b->esc_off[c], b->d_count + c, side),
                        "compaction launch");
        if (st) return st;
        TrajArgs e = cfg.a;
        e.esc_bin = nullptr;
        e.esc_ratio = 0.0;
        e.idx = b->d_idx + b->esc_off[c];
        e.k_from = b->d_kfrom + b->esc_off[c];
        e.count = b->d_count + c;
        e.redo_lists = redo_lists();
        e.redo_ctr = b->d_rctr + (size_t)(c % 8) * b->rctr_words;
        st = check_cuda(launch_escalation(cfg.f, cfg.t, b->esc_precision, e, side), "escalation launch");
        if (st) return st;
    }
    for (int i = 0; i < 8; ++i) {
        st = check_cuda(cudaEventRecord(b->done[i], b->side[i]), "event record");
        if (!st) st = check_cuda(cudaStreamWaitEvent(s, b->done[i], 0), "stream wait");
        if (st) return st;
    }
    return SFHK_OK;
}

void sfhk_batch_destroy(sfhk_batch* b) { batch_free(b); }

sfhk_status sfhk_dipole_batch(int32_t n_cfg, const sfhk_field* const* fields, const sfhk_target* const* targets,
                              const sfhk_births* births, const int64_t* n, const sfhk_prop_params* params,
                              double* const* d_len, double* const* d_vel, sfhk_stats* stats, void* stream) {
    NvtxRange nvtx_range("sfhk_dipole_batch");
    sfhk_batch* b = nullptr;
    sfhk_status st = sfhk_batch_create(n_cfg, fields, targets, births, n, params, d_len, d_vel, stats, &b);
    if (st) return st;
    st = sfhk_batch_run(b, stream);
    const sfhk_status ss = check_cuda(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
    batch_free(b);
    return st ? st : ss;
}

}  // extern "C"
