// C ABI of the SFHK library: argument validation, handles, launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "sfhk_internal.cuh"

namespace sfhk {

static thread_local char g_err[512] = "";

sfhk_status fail(sfhk_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

sfhk_status check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SFHK_OK;
    if (e == cudaErrorMemoryAllocation) return fail(SFHK_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(SFHK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

sfhk_status check_launch(const char* what) { return check_cuda(cudaGetLastError(), what); }

namespace {
std::mutex g_mu;
std::vector<unsigned int*> g_status;   // per device
std::vector<double*> g_scratch;        // per device, deterministic partial bins
std::vector<size_t> g_scratch_bytes;

sfhk_status current_device(int* dev) { return check_cuda(cudaGetDevice(dev), "cudaGetDevice"); }

bool is_fin(double x) { return std::isfinite(x); }

// The RK4 step constants in the arithmetic of R (the device step loops read them).
template <typename R>
StepK<R> step_constants(R h) {
    StepK<R> k;
    k.h = h;
    k.hh = R(0.5) * h;
    k.h6 = h * R(1.0 / 6.0);
    k.c2 = h * h * R(1.0 / 6.0);
    k.c3 = h * h * h * R(1.0 / 12.0);
    k.c4 = h * h * h * h * R(1.0 / 24.0);
    return k;
}

// Scratch for deterministic reductions, grown on demand (library-owned).
sfhk_status scratch(size_t bytes, double** out) {
    int dev;
    sfhk_status st = current_device(&dev);
    if (st) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_scratch.size() <= dev) {
        g_scratch.resize(dev + 1, nullptr);
        g_scratch_bytes.resize(dev + 1, 0);
    }
    if (g_scratch_bytes[dev] < bytes) {
        if (g_scratch[dev]) cudaFree(g_scratch[dev]);
        g_scratch[dev] = nullptr;
        g_scratch_bytes[dev] = 0;
        st = check_cuda(cudaMalloc(&g_scratch[dev], bytes), "scratch allocation");
        if (st) return st;
        g_scratch_bytes[dev] = bytes;
    }
    *out = g_scratch[dev];
    return SFHK_OK;
}

// Side streams and events for the overlapped escalation passes (per device).
constexpr int kSide = 8;
struct SidePool {
    cudaStream_t stream[kSide];   // priorities from the highest (0) to the lowest
    cudaEvent_t ready[kSide], done[kSide], fork, join;
    bool ok = false;
};
std::vector<SidePool> g_side;

sfhk_status side_pool(SidePool** out) {
    int dev;
    sfhk_status st = current_device(&dev);
    if (st) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_side.size() <= dev) g_side.resize(dev + 1);
    SidePool& p = g_side[dev];
    if (!p.ok) {
        // side stream i carries the i-th chunk of births in birth order: the
        // earliest births live longest and their escalation redo ends last, so
        // the earlier chunks get the higher priorities
        int least = 0, greatest = 0;
        st = check_cuda(cudaDeviceGetStreamPriorityRange(&least, &greatest), "priority range");
        if (st) return st;
        for (int i = 0; i < kSide; ++i) {
            const int span = least - greatest;   // >= 0; numerically lower = higher priority
            const int prio = greatest + (span * i) / (kSide - 1);
            st = check_cuda(cudaStreamCreateWithPriority(&p.stream[i], cudaStreamNonBlocking, prio), "side stream");
            if (!st) st = check_cuda(cudaEventCreateWithFlags(&p.ready[i], cudaEventDisableTiming), "event");
            if (!st) st = check_cuda(cudaEventCreateWithFlags(&p.done[i], cudaEventDisableTiming), "event");
            if (st) return st;
        }
        st = check_cuda(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming), "event");
        if (!st) st = check_cuda(cudaEventCreateWithFlags(&p.join, cudaEventDisableTiming), "event");
        if (st) return st;
        p.ok = true;
    }
    *out = &p;
    return SFHK_OK;
}

// Phase timing (sfhk_set_phase_timing): four timing events per device, recorded
// by sfhk_dipole on its stream when enabled and the stream is not capturing.
std::atomic<int> g_timing{0};
struct PhaseEvents {
    cudaEvent_t e[4];
    bool ok = false, recorded = false, phases = false;
};
std::vector<PhaseEvents> g_phase;

// The device's event set with the call's start recorded, or null (timing off,
// capturing stream, or no events).
PhaseEvents* phase_begin(cudaStream_t s) {
    if (!g_timing.load()) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_phase.size() <= dev) g_phase.resize(dev + 1);
    PhaseEvents& p = g_phase[dev];
    if (!p.ok) {
        for (int k = 0; k < 4; ++k)
            if (cudaEventCreate(&p.e[k]) != cudaSuccess) return nullptr;
        p.ok = true;
    }
    p.recorded = false;
    if (cudaEventRecord(p.e[0], s) != cudaSuccess) return nullptr;
    return &p;
}
void phase_mark(PhaseEvents* p, int k, cudaStream_t s) {
    if (p) cudaEventRecord(p->e[k], s);
}
// the call's end: events k..3 at this point of the stream
void phase_end(PhaseEvents* p, int k, bool phases, cudaStream_t s) {
    if (!p) return;
    for (int j = k; j < 4; ++j) cudaEventRecord(p->e[j], s);
    std::lock_guard<std::mutex> lk(g_mu);
    p->recorded = true;
    p->phases = phases;
}

}  // namespace

// Argument checks and launch shapes shared with the other dipole entry points.
sfhk_status check_handles(const sfhk_field* f, const sfhk_target* t) {
    if (!f) return fail(SFHK_EINVAL, "field is NULL");
    if (!t) return fail(SFHK_EINVAL, "target is NULL");
    int dev;
    sfhk_status st = current_device(&dev);
    if (st) return st;
    if (f->device != dev || t->device != dev)
        return fail(SFHK_EINVAL, "handle belongs to device %d/%d, current device is %d", f->device, t->device, dev);
    return SFHK_OK;
}

// Launch shapes chosen by sfhk_autotune, per (device, precision, planar, potential).
struct Tuned {
    int dev, precision, planar, pot, block, chunk_bins;
};
std::vector<Tuned> g_tuned;

bool tuned_lookup(int precision, int planar, int pot, int* block, int* chunk_bins) {
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Tuned& t : g_tuned)
        if (t.dev == dev && t.precision == precision && t.planar == planar && t.pot == pot) {
            *block = t.block;
            *chunk_bins = t.chunk_bins;
            return true;
        }
    return false;
}

sfhk_status check_prop(const sfhk_prop_params* pp, const sfhk::FieldDev& f, int* block, int* chunk) {
    if (!pp) return fail(SFHK_EINVAL, "prop params is NULL");
    if (pp->precision < 0 || pp->precision > 2) return fail(SFHK_EINVAL, "precision must be 0, 1 or 2");
    if (pp->deterministic != 0 && pp->deterministic != 1) return fail(SFHK_EINVAL, "deterministic must be 0 or 1");
    if (!is_fin(pp->gamma) || pp->gamma <= 0) return fail(SFHK_EINVAL, "gamma must be finite and > 0");
    if (!is_fin(pp->d_t) || pp->d_t <= 1.0) return fail(SFHK_EINVAL, "d_t must be finite and > 1");
    if (!is_fin(pp->esc_ratio)) return fail(SFHK_EINVAL, "esc_ratio must be finite");
    if (!is_fin(pp->esc_floor) || pp->esc_floor < 0) return fail(SFHK_EINVAL, "esc_floor must be finite and >= 0");
    if (!is_fin(pp->esc_ratio_big) || !is_fin(pp->esc_big) || pp->esc_big < 0)
        return fail(SFHK_EINVAL, "esc_ratio_big must be finite and esc_big finite and >= 0");
    if (pp->precision == 1 && pp->d_t > 1e36) return fail(SFHK_EINVAL, "MIXED needs d_t <= 1e36 (float range)");
    if (pp->geometry != 0 && pp->geometry != 1) return fail(SFHK_EINVAL, "geometry must be 0 or 1");
    if (pp->esc_precision < 0 || pp->esc_precision > 2) return fail(SFHK_EINVAL, "esc_precision must be 0, 1 or 2");
    if (pp->pw_mask < 0 || pp->pw_mask > 15) return fail(SFHK_EINVAL, "pw_mask must be in 0..15");
    if (pp->esc_overlap < 0 || pp->esc_overlap > 2) return fail(SFHK_EINVAL, "esc_overlap must be 0, 1 or 2");
    if (pp->pw_mask && (!is_fin(pp->pw_radius) || pp->pw_radius <= 0))
        return fail(SFHK_EINVAL, "pw_radius must be finite and > 0");
    int b = pp->block ? pp->block : 128;
    if (b != 64 && b != 128) return fail(SFHK_EINVAL, "block must be 0, 64 or 128");
    int n_out = (int)f.n_out;
    int c = pp->chunk_steps;
    if (c == 0) c = n_out * (int)((1000 + n_out - 1) / n_out);
    if (c < 64 || c > 8192 || c % n_out != 0)
        return fail(SFHK_EINVAL, "chunk_steps must be 0 or a multiple of n_out in [64, 8192]");
    *block = b;
    *chunk = c;
    return SFHK_OK;
}

sfhk_status check_births(const sfhk_births* b, int64_t n, bool need_amp) {
    if (!b) return fail(SFHK_EINVAL, "births is NULL");
    if (n < 0) return fail(SFHK_EINVAL, "n must be >= 0");
    if (n > b->capacity) return fail(SFHK_EINVAL, "n=%lld exceeds births capacity %lld", (long long)n,
                                     (long long)b->capacity);
    if (n > ((int64_t)1 << 40)) return fail(SFHK_EINVAL, "n too large");
    if (n == 0) return SFHK_OK;
    if (!b->n0 || !b->p0x || !b->p0y || !b->p0z || !b->q0z) return fail(SFHK_EINVAL, "births arrays are NULL");
    if (need_amp && (!b->amp_re || !b->amp_im)) return fail(SFHK_EINVAL, "birth amplitudes are NULL");
    return SFHK_OK;
}

void tuned_shape(const sfhk_prop_params* pp, const FieldDev& f, int pot, int planar, int* block, int* chunk) {
    if (pp->block != 0 || pp->chunk_steps != 0) return;
    int tb, tc;
    if (tuned_lookup(pp->precision, planar, pot, &tb, &tc)) {
        *block = tb;
        *chunk = tc * (int)f.n_out;
        if (*chunk > 8192) *chunk = (8192 / (int)f.n_out) * (int)f.n_out;
    }
}


unsigned int* device_status() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_status.size() <= dev) g_status.resize(dev + 1, nullptr);
    if (!g_status[dev]) {
        if (cudaMalloc(&g_status[dev], sizeof(unsigned int)) != cudaSuccess) return nullptr;
        if (cudaMemset(g_status[dev], 0, sizeof(unsigned int)) != cudaSuccess) return nullptr;
    }
    return g_status[dev];
}

}  // namespace sfhk

using namespace sfhk;

extern "C" {

const char* sfhk_last_error(void) { return g_err; }

const char* sfhk_version(void) { return "sfhk-gb300 0.1 (sm_103a)"; }

sfhk_status sfhk_sync(void* stream) {
    sfhk_status st = check_cuda(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
    if (st) return st;
    unsigned int* d = device_status();
    if (!d) return fail(SFHK_ECUDA, "device status word unavailable");
    unsigned int h = 0;
    st = check_cuda(cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost), "status read");
    if (st) return st;
    if (h) {
        cudaMemset(d, 0, sizeof(unsigned int));
        return fail(SFHK_ETIMEOUT, "a bounded device wait ran out (code %u)", h);
    }
    return SFHK_OK;
}

sfhk_status sfhk_make_field(const sfhk_pulse* pulse, double dt, double t_out_step, sfhk_field** out) {
    NvtxRange nvtx_range("sfhk_make_field");
    if (!pulse || !out) return fail(SFHK_EINVAL, "NULL argument");
    *out = nullptr;
    if (pulse->envelope != 0) return fail(SFHK_EUNSUPPORTED, "only the sin^2 envelope (0) is supported");
    if (!is_fin(pulse->intensity_wcm2) || pulse->intensity_wcm2 < 0) return fail(SFHK_EINVAL, "bad intensity");
    if (!is_fin(pulse->lambda_nm) || pulse->lambda_nm <= 0) return fail(SFHK_EINVAL, "bad wavelength");
    if (!is_fin(pulse->cycles) || pulse->cycles <= 0) return fail(SFHK_EINVAL, "bad cycle count");
    if (!is_fin(pulse->cep_rad)) return fail(SFHK_EINVAL, "bad CEP");
    if (!is_fin(dt) || dt <= 0) return fail(SFHK_EINVAL, "dt must be finite and > 0");
    if (!is_fin(t_out_step) || t_out_step <= 0) return fail(SFHK_EINVAL, "t_out_step must be finite and > 0");
    FieldDev f{};
    f.E0 = sqrt(pulse->intensity_wcm2 / 3.50944758e16);
    f.omega = 45.5633525 / pulse->lambda_nm;
    f.Tp = pulse->cycles * 2.0 * kPi / f.omega;
    f.cep = pulse->cep_rad;
    f.t_start = -0.5 * f.Tp;
    f.dt = dt;
    f.dt32 = (float)dt;
    f.k32 = step_constants<float>(f.dt32);
    f.k64 = step_constants<double>(dt);
    f.t_out = t_out_step;
    double ns = ceil(f.Tp / dt - 1e-9);
    if (ns < 2 || ns > (double)(1 << 30)) return fail(SFHK_EINVAL, "step count %.0f out of range", ns);
    f.n_steps = (int64_t)ns;
    double no = floor(t_out_step / dt + 0.5);
    if (no < 1 || fabs(no * dt - t_out_step) > 1e-12) return fail(SFHK_EINVAL, "t_out_step/dt must be an integer");
    f.n_out = (int64_t)no;
    f.n_bins = f.n_steps / f.n_out + 1;
    // A(t) = -(E0/w) cos^2(pi t/Tp) sin(w t + cep) as three sinusoids
    const double Om = 2.0 * kPi / f.Tp;
    f.n_modes = 3;
    f.a[0] = -f.E0 / (2.0 * f.omega);
    f.w[0] = f.omega;
    f.a[1] = -f.E0 / (4.0 * f.omega);
    f.w[1] = f.omega + Om;
    f.a[2] = -f.E0 / (4.0 * f.omega);
    f.w[2] = f.omega - Om;
    // half-step E table, E = -dA/dt = -sum a_j w_j cos(w_j t + cep), zero outside the pulse
    const int64_t nt = 2 * f.n_steps + 1;
    const int64_t len = (nt + 64) / 64 * 64;
    std::vector<double> e64(len, 0.0);
    std::vector<float> e32(len, 0.0f);
    for (int64_t j = 0; j < nt; ++j) {
        double t = f.t_start + 0.5 * (double)j * dt;
        double e = 0.0;
        if (fabs(t) <= 0.5 * f.Tp)
            for (int m = 0; m < 3; ++m) e -= f.a[m] * f.w[m] * cos(f.w[m] * t + f.cep);
        e64[j] = e;
        e32[j] = (float)e;
    }
    f.table_len = len;
    int dev;
    sfhk_status st = current_device(&dev);
    if (st) return st;
    sfhk_field* h = new (std::nothrow) sfhk_field();
    if (!h) return fail(SFHK_ENOMEM, "host allocation");
    h->device = dev;
    st = check_cuda(cudaMalloc(&h->d_E64, len * sizeof(double)), "field table");
    if (!st) st = check_cuda(cudaMalloc(&h->d_E32, len * sizeof(float)), "field table");
    if (!st) st = check_cuda(cudaMemcpy(h->d_E64, e64.data(), len * sizeof(double), cudaMemcpyHostToDevice), "copy");
    if (!st) st = check_cuda(cudaMemcpy(h->d_E32, e32.data(), len * sizeof(float), cudaMemcpyHostToDevice), "copy");
    if (st) {
        sfhk_field_destroy(h);
        return st;
    }
    f.E64 = h->d_E64;
    f.E32 = h->d_E32;
    h->f = f;
    *out = h;
    return SFHK_OK;
}

sfhk_status sfhk_field_get_info(const sfhk_field* field, sfhk_field_info* info) {
    if (!field || !info) return fail(SFHK_EINVAL, "NULL argument");
    const FieldDev& f = field->f;
    info->E0 = f.E0;
    info->omega = f.omega;
    info->Tp = f.Tp;
    info->t_start = f.t_start;
    info->dt = f.dt;
    info->t_out = f.t_out;
    info->n_steps = f.n_steps;
    info->n_out = f.n_out;
    info->n_bins = f.n_bins;
    return SFHK_OK;
}

void sfhk_field_destroy(sfhk_field* field) {
    if (!field) return;
    if (field->d_E64) cudaFree(field->d_E64);
    if (field->d_E32) cudaFree(field->d_E32);
    delete field;
}

sfhk_status sfhk_make_target(const sfhk_target_desc* d, sfhk_target** out) {
    NvtxRange nvtx_range("sfhk_make_target");
    if (!d || !out) return fail(SFHK_EINVAL, "NULL argument");
    *out = nullptr;
    if (d->potential < 0 || d->potential > 3) return fail(SFHK_EINVAL, "potential must be 0..3");
    if (d->gto_l != 0 && d->gto_l != 1) return fail(SFHK_EINVAL, "gto_l must be 0 or 1");
    if (d->amp < 0 || d->amp > 2) return fail(SFHK_EINVAL, "amp must be 0, 1 or 2");
    if (d->n_gto < 1 || d->n_gto > kMaxGto) return fail(SFHK_EINVAL, "n_gto must be 1..%d", kMaxGto);
    if (!d->gto_c || !d->gto_alpha) return fail(SFHK_EINVAL, "GTO arrays are NULL");
    if (!is_fin(d->ip) || d->ip <= 0) return fail(SFHK_EINVAL, "ip must be finite and > 0");
    for (int j = 0; j < 8; ++j)
        if (!is_fin(d->pot_param[j])) return fail(SFHK_EINVAL, "pot_param[%d] not finite", j);
    if (d->potential == 1 && d->pot_param[0] <= 0) return fail(SFHK_EINVAL, "softcore a must be > 0");
    if (d->potential == 3 && d->pot_param[0] <= 0) return fail(SFHK_EINVAL, "harmonic w must be > 0");
    sfhk_target* h = new (std::nothrow) sfhk_target();
    if (!h) return fail(SFHK_ENOMEM, "host allocation");
    TargetDev& t = h->t;
    t.pot = d->potential;
    t.gto_l = d->gto_l;
    t.n_gto = d->n_gto;
    t.amp = d->amp;
    for (int j = 0; j < 8; ++j) t.pot_param[j] = d->pot_param[j];
    for (int j = 0; j < 8; ++j) t.pot_param32[j] = (float)d->pot_param[j];
    t.a2_32 = (float)(d->pot_param[0] * d->pot_param[0]);
    t.ip = d->ip;
    for (int j = 0; j < d->n_gto; ++j) {
        if (!is_fin(d->gto_c[j]) || !is_fin(d->gto_alpha[j]) || d->gto_alpha[j] <= 0) {
            delete h;
            return fail(SFHK_EINVAL, "GTO %d invalid", j);
        }
        t.c[j] = d->gto_c[j];
        t.alpha[j] = d->gto_alpha[j];
    }
    int dev;
    sfhk_status st = current_device(&dev);
    if (st) {
        delete h;
        return st;
    }
    h->device = dev;
    *out = h;
    return SFHK_OK;
}

void sfhk_target_destroy(sfhk_target* target) { delete target; }

sfhk_status sfhk_sample_births(const sfhk_field* field, const sfhk_target* target, const sfhk_birth_params* p,
                               const sfhk_births* b, void* stream) {
    NvtxRange nvtx_range("sfhk_sample_births");
    sfhk_status st = check_handles(field, target);
    if (st) return st;
    if (!p || !b) return fail(SFHK_EINVAL, "NULL argument");
    if (p->n < 0) return fail(SFHK_EINVAL, "n must be >= 0");
    if (p->n > ((int64_t)1 << 40)) return fail(SFHK_EINVAL, "n too large");
    if (p->first < 0 || p->first > p->n) return fail(SFHK_EINVAL, "first outside [0, n]");
    const int64_t count = p->count ? p->count : p->n - p->first;
    if (count < 0 || p->first + count > p->n) return fail(SFHK_EINVAL, "first + count exceeds n");
    if (count > b->capacity) return fail(SFHK_EINVAL, "count exceeds births capacity");
    if (p->mode == 0) {
        if (p->n_t <= 0 || p->n_k <= 0 || (int64_t)p->n_t * p->n_k != p->n)
            return fail(SFHK_EINVAL, "grid mode needs n == n_t * n_k > 0");
        if (!is_fin(p->kmax) || p->kmax <= 0) return fail(SFHK_EINVAL, "kmax must be finite and > 0");
    } else if (p->mode == 1) {
        if (!is_fin(p->sigma_k) || p->sigma_k <= 0) return fail(SFHK_EINVAL, "sigma_k must be finite and > 0");
    } else {
        return fail(SFHK_EINVAL, "mode must be 0 or 1");
    }
    if (count == 0) return SFHK_OK;
    if (!b->n0 || !b->t0 || !b->p0x || !b->p0y || !b->p0z || !b->q0z || !b->amp_re || !b->amp_im)
        return fail(SFHK_EINVAL, "births arrays are NULL");
    BirthArgs a{};
    a.n = p->n;
    a.first = p->first;
    a.count = count;
    a.mode = p->mode;
    a.n_t = p->n_t;
    a.n_k = p->n_k;
    a.sigma = p->sigma_k;
    a.kmax = p->kmax;
    a.seed = p->seed;
    a.n0 = b->n0;
    a.t0 = b->t0;
    a.px = b->p0x;
    a.py = b->p0y;
    a.pz = b->p0z;
    a.qz = b->q0z;
    a.amp_re = b->amp_re;
    a.amp_im = b->amp_im;
    return check_cuda(launch_births(field->f, target->t, a, (cudaStream_t)stream), "births launch");
}

sfhk_status sfhk_resample_births(const sfhk_births* pool, int64_t m, int64_t n, uint64_t seed, const sfhk_births* out,
                                 int64_t* n_distinct, void* stream) {
    NvtxRange nvtx_range("sfhk_resample_births");
    if (!pool || !out) return fail(SFHK_EINVAL, "NULL argument");
    if (m < 0 || n < 0) return fail(SFHK_EINVAL, "m and n must be >= 0");
    if (m >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31)) return fail(SFHK_EINVAL, "m and n must be < 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        if (n_distinct) return check_cuda(cudaMemsetAsync(n_distinct, 0, sizeof(int64_t), s), "n_distinct clear");
        return SFHK_OK;
    }
    if (m < 1) return fail(SFHK_EINVAL, "resampling n > 0 births needs a pool of m >= 1");
    if (pool->capacity < m) return fail(SFHK_EINVAL, "pool capacity below m");
    if (out->capacity < n) return fail(SFHK_EINVAL, "out capacity below n");
    const void* pa[8] = {pool->n0, pool->t0, pool->p0x, pool->p0y, pool->p0z, pool->q0z, pool->amp_re, pool->amp_im};
    const void* oa[8] = {out->n0, out->t0, out->p0x, out->p0y, out->p0z, out->q0z, out->amp_re, out->amp_im};
    for (int k = 0; k < 8; ++k) {
        if (!pa[k] || !oa[k]) return fail(SFHK_EINVAL, "births arrays are NULL");
        for (int l = 0; l < 8; ++l)
            if (pa[k] == oa[l]) return fail(SFHK_EINVAL, "pool and out share an array");
    }
    unsigned char* sc = nullptr;
    sfhk_status st = scratch(resample_scratch_bytes(m), reinterpret_cast<double**>(&sc));
    if (st) return st;
    BirthArgs p{}, o{};
    p.n0 = pool->n0;
    p.t0 = pool->t0;
    p.px = pool->p0x;
    p.py = pool->p0y;
    p.pz = pool->p0z;
    p.qz = pool->q0z;
    p.amp_re = pool->amp_re;
    p.amp_im = pool->amp_im;
    o.n0 = out->n0;
    o.t0 = out->t0;
    o.px = out->p0x;
    o.py = out->p0y;
    o.pz = out->p0z;
    o.qz = out->q0z;
    o.amp_re = out->amp_re;
    o.amp_im = out->amp_im;
    return check_cuda(launch_resample(p, m, n, seed, o, sc, n_distinct, s), "resampling launch");
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

static sfhk_status run_traj(const sfhk_field* field, const sfhk_target* target, const sfhk_births* b, int64_t n,
                            const sfhk_prop_params* pp, int mode, int64_t n_last, double* d_len, double* d_vel,
                            const sfhk_endpoints* ep, sfhk_stats* stats, void* stream) {
    int block, chunk;
    sfhk_status st = check_prop(pp, field->f, &block, &chunk);
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
    a.pw_mask = mode == 1 ? pp->pw_mask : 0;
    a.pw_radius = pp->pw_radius;
    a.seg_lo = 0;
    a.seg_hi = n_last;
    a.state = nullptr;
    a.mode = mode;
    a.n_last = n_last;
    a.d_len = d_len;
    a.d_vel = d_vel;
    a.stats = stats;
    a.block = block;
    a.chunk = chunk;
    // planar form: dipole mode, births on the z axis (q0x = q0y = NULL), not forced to 3D
    a.planar = (mode == 1 && b->q0x == nullptr && b->q0y == nullptr && pp->geometry == 0) ? 1 : 0;
    tuned_shape(pp, field->f, target->t.pot, a.planar, &block, &chunk);
    a.block = block;
    a.chunk = chunk;
    if (pp->precision == 2 && !a.planar)
        return fail(SFHK_EUNSUPPORTED, "precision 2 (double-float) needs the planar form: dipole mode, "
                                       "q0x = q0y = NULL, geometry 0");
    if (ep) {
        a.st_out = ep->state;
        a.c_re = ep->c_re;
        a.c_im = ep->c_im;
        a.flags = ep->flags;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_blocks = (n + a.block - 1) / a.block;
    const bool det = mode == 1 && pp->deterministic;
    const bool esc = mode == 1 && pp->precision == 1 && pp->esc_ratio > 0.0;
    if (esc && n >= ((int64_t)1 << 31)) return fail(SFHK_EINVAL, "escalation supports n < 2^31 births");
    // segmented float pass (escalation, not deterministic): kSide time segments
    const bool segmented = esc && !det && pp->esc_overlap == 1;
    const int nseg = segmented ? kSide : 1;
    const int words = segmented ? state_words(a.planar) : 0;
    // library-owned scratch: [partials | esc_bin | idx[nseg] | k_from[nseg] | block counts[nseg] |
    //                         counts + amplitude maximum | saved state]
    const size_t part_b = det ? align256((size_t)n_blocks * 2 * field->f.n_bins * sizeof(double)) : 0;
    const size_t esc_b = esc ? align256((size_t)n * 4) : 0;
    const size_t blk_b = esc ? align256((size_t)(compact_blocks(n) + 16) * 4) : 0;
    const size_t state_b = align256((size_t)words * (size_t)n * 4);
    const size_t rw = redo_scratch_words(n);
    const size_t ctr_b = esc ? (size_t)kSide * rw * 4 : 0;   // redo counters and group plan, per side stream
    const size_t total = part_b + esc_b * (1 + 2 * (size_t)nseg) + blk_b * nseg + (esc ? 256 : 0) + state_b + ctr_b;
    unsigned char* base = nullptr;
    if (total) {
        st = scratch(total, reinterpret_cast<double**>(&base));
        if (st) return st;
    }
    double* part = det ? reinterpret_cast<double*>(base) : nullptr;
    unsigned char* eb = base + part_b;
    int32_t* esc_bin = esc ? reinterpret_cast<int32_t*>(eb) : nullptr;
    int32_t* idx = esc ? reinterpret_cast<int32_t*>(eb + esc_b) : nullptr;                 // + s * n
    int32_t* kfrom = esc ? reinterpret_cast<int32_t*>(eb + esc_b * (1 + nseg)) : nullptr;   // + s * n
    unsigned char* bb = eb + esc_b * (1 + 2 * (size_t)nseg);
    int32_t* blk = esc ? reinterpret_cast<int32_t*>(bb) : nullptr;                         // + s * blk_b
    int32_t* count = esc ? reinterpret_cast<int32_t*>(bb + blk_b * nseg) : nullptr;
    double* amax2 = esc ? reinterpret_cast<double*>(bb + blk_b * nseg + 128) : nullptr;
    uint32_t* state = words ? reinterpret_cast<uint32_t*>(bb + blk_b * nseg + 256) : nullptr;
    int* rctr = esc ? reinterpret_cast<int*>(bb + blk_b * nseg + 256 + state_b) : nullptr;
    a.redo_lists = redo_lists();
    a.esc_l2 = pp->esc_ratio > 0.0 ? (float)log2(pp->esc_ratio) : 0.f;
    a.esc_l2_big = pp->esc_ratio_big > 0.0 ? (float)log2(pp->esc_ratio_big) : a.esc_l2;
    a.esc_l2_lo = pp->esc_big > 0.0 ? fminf(a.esc_l2, a.esc_l2_big) : a.esc_l2;
    a.esc_l2_floor = pp->esc_floor > 0.0 ? (float)log2(pp->esc_floor * pp->esc_floor) : -1e30f;
    a.esc_l2_bigw = pp->esc_big > 0.0 ? (float)log2(pp->esc_big * pp->esc_big) : 1e30f;
    PhaseEvents* pe = phase_begin(s);
    if (esc && (pp->esc_floor > 0.0 || pp->esc_big > 0.0)) {
        // max |amp|^2 over the births, before any float pass reads it
        st = check_cuda(launch_amp_max(b->amp_re, b->amp_im, n, amax2, s), "amplitude maximum");
        if (st) return st;
        a.esc_amax2 = amax2;
        a.esc_floor = pp->esc_floor;
        a.esc_big = pp->esc_big;
        a.esc_ratio_big = pp->esc_ratio_big;
    }
    if (det) {
        st = check_cuda(cudaMemsetAsync(part, 0, part_b, s), "scratch clear");
        if (st) return st;
        a.part = part;
    }
    if (esc && !det && pp->esc_overlap != 2) {
        // Overlapped escalation (esc_overlap): birth chunks, or a time-segmented
        // float pass whose every segment's escalations are redone at once; the
        // caller's stream waits for every redo.
        SidePool* sp = nullptr;
        st = side_pool(&sp);
        if (st) return st;
        st = check_cuda(cudaMemsetAsync(esc_bin, 0xff, (size_t)n * 4, s), "scratch clear");   // -1
        if (st) return st;
        const int epr = pp->esc_precision;
        if (pp->esc_overlap == 0) {
            // Birth chunks: the births are cut into up to kSide chunks (birth order,
            // whole blocks); each chunk runs its float pass, then the compaction and
            // high-precision redo of its escalated births, on its own side stream
            // (earlier chunks at higher priority), so that the chains overlap and
            // fill each other's tails.
            const int64_t per = (n + kSide - 1) / kSide;
            const int64_t csz = std::max<int64_t>((per + block - 1) / block * block, (int64_t)64 * block);
            st = check_cuda(cudaEventRecord(sp->fork, s), "event record");
            if (st) return st;
            int c = 0;
            int64_t blk_off = 0;
            for (int64_t c0 = 0; c0 < n; c0 += csz, ++c) {
                const int64_t cn = std::min(csz, n - c0);
                TrajArgs f = a;
                f.n = cn;
                f.n0 = b->n0 + c0;
                f.px = b->p0x + c0;
                f.py = b->p0y + c0;
                f.pz = b->p0z + c0;
                f.qx = b->q0x ? b->q0x + c0 : nullptr;
                f.qy = b->q0y ? b->q0y + c0 : nullptr;
                f.qz = b->q0z + c0;
                f.amp_re = b->amp_re + c0;
                f.amp_im = b->amp_im + c0;
                f.esc_bin = esc_bin + c0;
                f.esc_ratio = pp->esc_ratio;
                cudaStream_t side = sp->stream[c];
                st = check_cuda(cudaStreamWaitEvent(side, sp->fork, 0), "stream wait");
                if (st) return st;
                st = check_cuda(launch_traj(field->f, target->t, pp->precision, f, side), "trajectory launch");
                if (st) return st;
                st = check_cuda(launch_compact(esc_bin + c0, cn, blk + blk_off, idx + c0, kfrom + c0, count + c, side),
                                "compaction launch");
                blk_off += compact_blocks(cn);
                if (st) return st;
                TrajArgs e = f;
                e.esc_bin = nullptr;
                e.esc_ratio = 0.0;
                e.idx = idx + c0;
                e.k_from = kfrom + c0;
                e.count = count + c;
                e.redo_ctr = rctr + (size_t)c * rw;
                st = check_cuda(launch_escalation(field->f, target->t, epr, e, side), "escalation launch");
                if (st) return st;
                st = check_cuda(cudaEventRecord(sp->done[c], side), "event record");
                if (st) return st;
            }
            for (int j = 0; j < c; ++j) {
                st = check_cuda(cudaStreamWaitEvent(s, sp->done[j], 0), "stream wait");
                if (st) return st;
            }
            phase_end(pe, 1, false, s);
            return SFHK_OK;
        }
        // Time segments (esc_overlap 1): the float pass runs as nseg launches over
        // consecutive time segments (whole field windows), every live trajectory's
        // state saved in device memory between them; after each segment the
        // trajectories it escalated are compacted and their redo (from birth)
        // starts at once on a side stream, overlapping the later segments.
        cudaStream_t fs = s;
        const int64_t n_win = (a.n_last + a.chunk) / a.chunk;      // windows covering grid points 0..n_last
        const int ns = (int)std::min<int64_t>(nseg, n_win);
        const size_t blk_words = blk_b / 4;
        for (int g = 0; g < ns; ++g) {
            const int64_t w_lo = n_win * g / ns, w_hi = n_win * (g + 1) / ns;   // windows [w_lo, w_hi)
            TrajArgs f = a;
            f.seg_lo = w_lo * a.chunk;
            f.seg_hi = (g == ns - 1) ? a.n_last : w_hi * a.chunk - 1;
            f.state = state;
            f.esc_bin = esc_bin;
            f.esc_ratio = pp->esc_ratio;
            st = check_cuda(launch_traj(field->f, target->t, pp->precision, f, fs), "trajectory launch");
            if (st) return st;
            // escalations of this segment: bins k with k n_out in [seg_lo, seg_hi]
            const int64_t no = field->f.n_out;
            const int32_t k_lo = (int32_t)((f.seg_lo + no - 1) / no), k_hi = (int32_t)(f.seg_hi / no);
            int32_t* idx_g = idx + (size_t)g * n;
            int32_t* kf_g = kfrom + (size_t)g * n;
            st = check_cuda(launch_compact(esc_bin, n, blk + (size_t)g * blk_words, idx_g, kf_g, count + g, fs, k_lo,
                                           k_hi),
                            "compaction launch");
            if (st) return st;
            st = check_cuda(cudaEventRecord(sp->ready[g], fs), "event record");
            if (st) return st;
            cudaStream_t side = sp->stream[g];
            st = check_cuda(cudaStreamWaitEvent(side, sp->ready[g], 0), "stream wait");
            if (st) return st;
            TrajArgs e = a;
            e.esc_bin = nullptr;
            e.esc_ratio = 0.0;
            e.idx = idx_g;
            e.k_from = kf_g;
            e.count = count + g;
            e.redo_ctr = rctr + (size_t)g * rw;
            st = check_cuda(launch_escalation(field->f, target->t, epr, e, side), "escalation launch");
            if (st) return st;
            st = check_cuda(cudaEventRecord(sp->done[g], side), "event record");
            if (st) return st;
        }
        if (fs != s) {
            st = check_cuda(cudaEventRecord(sp->join, fs), "event record");
            if (!st) st = check_cuda(cudaStreamWaitEvent(s, sp->join, 0), "stream wait");
            if (st) return st;
        }
        for (int g = 0; g < ns; ++g) {   // the caller's stream waits for every redo
            st = check_cuda(cudaStreamWaitEvent(s, sp->done[g], 0), "stream wait");
            if (st) return st;
        }
        phase_end(pe, 1, false, s);
        return SFHK_OK;
    }
    if (esc) {
        st = check_cuda(cudaMemsetAsync(esc_bin, 0xff, (size_t)n * 4, s), "scratch clear");   // -1
        if (st) return st;
        a.esc_bin = esc_bin;
        a.esc_ratio = pp->esc_ratio;
    }
    st = check_cuda(launch_traj(field->f, target->t, pp->precision, a, s), "trajectory launch");
    if (st) return st;
    if (det) {
        st = check_cuda(launch_reduce_partials(part, n_blocks, field->f.n_bins, d_len, d_vel, s), "reduce launch");
        if (st) return st;
    }
    phase_mark(pe, 1, s);
    if (esc) {
        // one high-precision pass over all escalated births, after the float pass
        // (deterministic mode, or the sequential schedule esc_overlap 2)
        st = check_cuda(launch_compact(esc_bin, n, blk, idx, kfrom, count, s), "compaction launch");
        if (st) return st;
        phase_mark(pe, 2, s);
        TrajArgs e = a;
        e.esc_bin = nullptr;
        e.esc_ratio = 0.0;
        e.idx = idx;
        e.k_from = kfrom;
        e.count = count;
        e.redo_ctr = rctr;
        if (det) {
            st = check_cuda(cudaMemsetAsync(part, 0, part_b, s), "scratch clear");
            if (st) return st;
        }
        st = check_cuda(launch_escalation(field->f, target->t, pp->esc_precision, e, s), "escalation launch");
        if (st) return st;
        if (det)
            st = check_cuda(launch_reduce_partials(part, n_blocks, field->f.n_bins, d_len, d_vel, s), "reduce launch");
        if (st) return st;
    }
    phase_end(pe, esc ? 3 : 2, true, s);
    return st;
}

sfhk_status sfhk_propagate(const sfhk_field* field, const sfhk_target* target, const sfhk_births* births, int64_t n,
                           const sfhk_prop_params* params, const sfhk_endpoints* out, sfhk_stats* stats,
                           void* stream) {
    NvtxRange nvtx_range("sfhk_propagate");
    sfhk_status st = check_handles(field, target);
    if (st) return st;
    st = check_births(births, n, false);
    if (st) return st;
    if (!out) return fail(SFHK_EINVAL, "endpoints is NULL");
    if (n > 0 && (!out->state || !out->c_re || !out->c_im || !out->flags))
        return fail(SFHK_EINVAL, "endpoint arrays are NULL");
    if (out->n_end < 0 || out->n_end > field->f.n_steps)
        return fail(SFHK_EINVAL, "n_end=%lld outside [0, %lld]", (long long)out->n_end, (long long)field->f.n_steps);
    if (n == 0) return SFHK_OK;
    sfhk_prop_params pp = *params;
    pp.deterministic = 0;
    return run_traj(field, target, births, n, &pp, 0, out->n_end, nullptr, nullptr, out, stats, stream);
}

sfhk_status sfhk_dipole(const sfhk_field* field, const sfhk_target* target, const sfhk_births* births, int64_t n,
                        const sfhk_prop_params* params, double* d_len, double* d_vel, sfhk_stats* stats,
                        void* stream) {
    NvtxRange nvtx_range("sfhk_dipole");
    sfhk_status st = check_handles(field, target);
    if (st) return st;
    st = check_births(births, n, true);
    if (st) return st;
    if (!d_len || !d_vel) return fail(SFHK_EINVAL, "bins are NULL");
    if (n == 0) return SFHK_OK;
    return run_traj(field, target, births, n, params, 1, field->f.n_steps, d_len, d_vel, nullptr, stats, stream);
}

sfhk_status sfhk_spectrum(const double* bins, int64_t n_bins, double t0, double dt_out, double tau_h,
                          const double* omega, int64_t n_omega, double* out_re, double* out_im, void* stream) {
    NvtxRange nvtx_range("sfhk_spectrum");
    if (n_bins < 0 || n_omega < 0) return fail(SFHK_EINVAL, "negative size");
    if (!is_fin(t0) || !is_fin(dt_out) || dt_out <= 0 || !is_fin(tau_h) || tau_h <= 0)
        return fail(SFHK_EINVAL, "bad grid parameters");
    if (n_omega == 0) return SFHK_OK;
    if ((n_bins > 0 && !bins) || !omega || !out_re || !out_im) return fail(SFHK_EINVAL, "NULL array");
    return check_cuda(launch_spectrum(bins, n_bins, t0, dt_out, tau_h, omega, n_omega, out_re, out_im,
                                      (cudaStream_t)stream),
                      "spectrum launch");
}

sfhk_status sfhk_gabor(const double* bins, int64_t n_bins, double t0, double dt_out, double sigma,
                       const double* times, int64_t n_times, const double* omega, int64_t n_omega, double* out_re,
                       double* out_im, void* stream) {
    NvtxRange nvtx_range("sfhk_gabor");
    if (n_bins < 0 || n_times < 0 || n_omega < 0) return fail(SFHK_EINVAL, "negative size");
    if (!is_fin(t0) || !is_fin(dt_out) || dt_out <= 0 || !is_fin(sigma) || sigma <= 0)
        return fail(SFHK_EINVAL, "bad grid or window parameters");
    if (n_omega == 0 || n_times == 0) return SFHK_OK;
    if ((n_bins > 0 && !bins) || !times || !omega || !out_re || !out_im) return fail(SFHK_EINVAL, "NULL array");
    return check_cuda(launch_gabor(bins, n_bins, t0, dt_out, sigma, times, n_times, omega, n_omega, out_re, out_im,
                                   (cudaStream_t)stream),
                      "gabor launch");
}

sfhk_status sfhk_emission_time(const double* g_re, const double* g_im, int64_t n_times, int64_t n_omega,
                               const double* times, double t_a, double t_b, double* centroid, double* peak,
                               void* stream) {
    NvtxRange nvtx_range("sfhk_emission_time");
    if (n_times < 0 || n_omega < 0) return fail(SFHK_EINVAL, "negative size");
    if (std::isnan(t_a) || std::isnan(t_b)) return fail(SFHK_EINVAL, "window bound is NaN");
    if (n_omega == 0) return SFHK_OK;
    if ((n_times > 0 && (!g_re || !g_im || !times)) || !centroid || !peak) return fail(SFHK_EINVAL, "NULL array");
    return check_cuda(launch_emission_time(g_re, g_im, n_times, n_omega, times, t_a, t_b, centroid, peak,
                                           (cudaStream_t)stream),
                      "emission time launch");
}

sfhk_status sfhk_set_phase_timing(int32_t on) {
    if (on != 0 && on != 1) return fail(SFHK_EINVAL, "on must be 0 or 1");
    g_timing.store(on);
    return SFHK_OK;
}

sfhk_status sfhk_get_phase_times(sfhk_phase_times* out) {
    if (!out) return fail(SFHK_EINVAL, "out is NULL");
    int dev;
    sfhk_status st = current_device(&dev);
    if (st) return st;
    PhaseEvents* p = nullptr;
    bool phases = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if ((int)g_phase.size() > dev && g_phase[dev].ok && g_phase[dev].recorded) {
            p = &g_phase[dev];
            phases = p->phases;
        }
    }
    if (!p) return fail(SFHK_EINVAL, "no timed call on this device (enable sfhk_set_phase_timing first)");
    st = check_cuda(cudaEventSynchronize(p->e[3]), "phase event wait");
    if (st) return st;
    float ms[3] = {0.f, 0.f, 0.f}, tot = 0.f;
    for (int k = 0; k < 3 && !st; ++k) st = check_cuda(cudaEventElapsedTime(&ms[k], p->e[k], p->e[k + 1]), "elapsed");
    if (!st) st = check_cuda(cudaEventElapsedTime(&tot, p->e[0], p->e[3]), "elapsed");
    if (st) return st;
    out->traj_ms = phases ? ms[0] : 0.f;
    out->compact_ms = phases ? ms[1] : 0.f;
    out->redo_ms = phases ? ms[2] : 0.f;
    out->total_ms = tot;
    out->phases = phases ? 1 : 0;
    out->reserved = 0;
    return SFHK_OK;
}

sfhk_status sfhk_autotune(const sfhk_field* field, const sfhk_target* target, const sfhk_births* births,
                          int64_t n_sample, const sfhk_prop_params* params, int32_t* best_block, int32_t* best_chunk,
                          double* best_ms, void* stream) {
    NvtxRange nvtx_range("sfhk_autotune");
    sfhk_status st = check_handles(field, target);
    if (st) return st;
    st = check_births(births, n_sample, true);
    if (st) return st;
    if (!params || n_sample < 1) return fail(SFHK_EINVAL, "params NULL or empty sample");
    const int n_out = (int)field->f.n_out;
    double* bins = nullptr;
    const size_t nb = (size_t)field->f.n_bins;
    st = check_cuda(cudaMalloc(&bins, 2 * nb * sizeof(double)), "autotune bins");
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks[2] = {64, 128};
    const int chunk_bins[5] = {25, 50, 100, 200, 400};
    float best = 1e30f;
    int bb = 128, bc = 100;
    for (int ib = 0; ib < 2 && !st; ++ib)
        for (int ic = 0; ic < 5 && !st; ++ic) {
            sfhk_prop_params pp = *params;
            pp.block = blocks[ib];
            pp.chunk_steps = chunk_bins[ic] * n_out;
            pp.esc_ratio = 0.0;
            pp.deterministic = 0;
            if (pp.chunk_steps < 64 || pp.chunk_steps > 8192) continue;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && !st; ++rep) {   // warm-up, then timed
                cudaEventRecord(e0, s);
                st = sfhk_dipole(field, target, births, n_sample, &pp, bins, bins + nb, nullptr, stream);
                cudaEventRecord(e1, s);
                if (!st) st = check_cuda(cudaEventSynchronize(e1), "autotune sync");
                if (!st) cudaEventElapsedTime(&ms, e0, e1);
            }
            if (!st && ms < best) {
                best = ms;
                bb = blocks[ib];
                bc = chunk_bins[ic];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(bins);
    if (st) return st;
    int dev;
    cudaGetDevice(&dev);
    const int planar = (births->q0x == nullptr && births->q0y == nullptr && params->geometry == 0) ? 1 : 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        bool found = false;
        for (Tuned& t : g_tuned)
            if (t.dev == dev && t.precision == params->precision && t.planar == planar && t.pot == target->t.pot) {
                t.block = bb;
                t.chunk_bins = bc;
                found = true;
            }
        if (!found) g_tuned.push_back(Tuned{dev, params->precision, planar, target->t.pot, bb, bc});
    }
    if (best_block) *best_block = bb;
    if (best_chunk) *best_chunk = bc * n_out;
    if (best_ms) *best_ms = best;
    return SFHK_OK;
}

}  // extern "C"
