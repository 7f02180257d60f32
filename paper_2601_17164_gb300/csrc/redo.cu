// FP64 redo of the escalated births of a mixed-precision pass, planar form,
// with the work of one trajectory-step split across four warps.
//
// Same arithmetic as the FP64 planar trajectory block (traj_block.cuh: App. A
// propagation, Eq. C_HK prefactor with per-step branch tracking, Sec. III.A
// removal, App. C recombination terms), reorganised for latency: an escalation
// list is short (a few per cent of the births) and its longest members run
// the whole pulse, so the redo is bound by the chain of dependent FP64
// operations of one trajectory, not by the number of trajectories (one warp's
// FP64 instruction occupies its sub-partition's FP64 unit for 64 cycles).  A
// block of 128 threads holds 32 trajectories (one per lane) and gives each of
// its four warps about a quarter of the FP64 work of every step:
//   dynamics  RK4 stages of (q, p) and the stage Hessian data,
//   matrix    the step matrix [[A, B], [C, D]] (and its out-of-plane analogue),
//   columns   the stability columns advanced by the step matrix, and the action
//             increment (moved here from the matrix role, the one with the most
//             FP64 work: a group alone on its SM then keeps 0.68 of the FP64
//             units busy instead of 0.65),
//   bins      det Z of the new columns and the branch of sqrt det Z, the
//             partial-wave labels, removal and the prefactor at the bins, and
//             the GTO recombination sums, spread over the steps between bins,
//             with the warp reduction and the atomic bin update.
// The warps form a pipeline one grid point apart, handing data on through
// double-buffered shared-memory slots with one CTA barrier per grid point.
// The roles rotate with the block index so that the heavier roles of the
// blocks resident on one SM spread over its four sub-partitions.  Removal is
// decided by the bins warp; the warps ahead of it learn of it a few grid
// points late and only skip work that no longer counts.
//
// Each part runs the same device functions as the one-thread-per-trajectory
// kernel (TrajP::stages_qp / action_term / action_sum, TrajP::step_matrix,
// TrajP::apply_step_matrix, TrajP::detc, follow_branch, gto_terms,
// contribution_final), so trajectories, branches, labels and removals are the
// same; only the order of the final bin sums (one warp per block instead of
// four) differs.
#include <algorithm>

#include "sfhk_internal.cuh"
#include "traj_block.cuh"

namespace sfhk {
namespace {

constexpr int kW = 32;            // trajectories per block
constexpr int kThreads = 128;     // four warps
// dynamics -> matrix: stage positions (8), g (4), h (4), stage momenta 2..4 (6), stage
// potentials (4), three unused words, state (q0, q2, p0, p2)
constexpr int kS01 = 33;
// matrix -> columns: 19 matrix entries, state (q0, q2, p0, p2), then the action
// increment's inputs: stage z of stages 2..4 (3), stage momenta of stages 2..4 (6),
// stage potentials (4); the columns warp reads E itself (static shared memory stays
// within 48 KB per block)
constexpr int kS12 = 36;
constexpr int kS23 = 25;          // columns -> bins: columns after the step (16 in-plane, 4 out-of-plane), state

// read-only view of the planar state for the recombination terms (q_y = p_y = 0)
struct PView {
    double q[3], p[3];
    struct {
        double s;
        __device__ double reduced() const { return s; }
    } S;
    __device__ PView(double q0, double q2, double p0, double p2, double s) : q{q0, 0.0, q2}, p{p0, 0.0, p2}, S{s} {}
};

// Two-slot hand-offs between consecutive roles on named barriers (0 is left to
// __syncthreads): hand-off h in {0, 1, 2}, slot d in {0, 1}; "full" is arrived at by
// the producer and waited on by the consumer, "empty" the other way round, 64
// threads each (the two warps).  A role runs ahead of the next by at most two
// grid points, so uneven work per grid point evens out across the pipeline.
__device__ __forceinline__ void bar_sync64(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }
__device__ __forceinline__ void bar_arrive64(int id) { asm volatile("bar.arrive %0, 64;" ::"r"(id) : "memory"); }
struct Producer {
    int h;
    int64_t k;
    __device__ explicit Producer(int h_) : h(h_), k(0) {}
    __device__ int acquire() {                     // slot for item k, once its item k - 2 is consumed
        const int d = (int)(k & 1);
        if (k >= 2) bar_sync64(3 + 4 * h + d);
        return d;
    }
    __device__ void publish(int d) {
        bar_arrive64(1 + 4 * h + d);
        ++k;
    }
    __device__ void drain() {                      // the consumer's releases of the last items
        for (int64_t j = (k >= 2 ? k - 2 : 0); j < k; ++j) bar_sync64(3 + 4 * h + (int)(j & 1));
    }
};
struct Consumer {
    int h;
    int64_t k;
    __device__ explicit Consumer(int h_) : h(h_), k(0) {}
    __device__ int wait() {
        const int d = (int)(k & 1);
        bar_sync64(1 + 4 * h + d);
        return d;
    }
    __device__ void release(int d) {
        bar_arrive64(3 + 4 * h + d);
        ++k;
    }
};

struct Shared {
    double s01[2][kS01][kW];
    double s12[2][kS12][kW];
    double s23[2][kS23][kW];
    int alive[kW];   // written by the bins warp, read late and without order by the warps ahead
};

struct Common {
    int64_t n_first, n_last;   // first and last grid point of the block
    int n_out;
    bool have;
    int64_t i, n0, k_cnt;
    bool alive0;
};

// dynamics: the state at grid point n and the stages of the step n -> n + 1
template <int POT>
__device__ void run_dynamics(const FieldDev& f, const TargetDev& tg, const TrajArgs& a, const Common& c, Shared& sm,
                             int lane) {
    PotConst<double> pc;
    if (POT == POT_SOFTCORE || POT == POT_HARMONIC) pc.a2 = tg.pot_param[0] * tg.pot_param[0];
    pc.Zc = tg.pot_param[0]; pc.a1 = tg.pot_param[1]; pc.a2t = tg.pot_param[2];
    pc.a3 = tg.pot_param[3]; pc.a4 = tg.pot_param[4]; pc.a5 = tg.pot_param[5];
    pc.a6 = tg.pot_param[6];
    TrajP<double, POT> T;
    T.init(0.0, 0.0, c.have ? a.qz[c.i] : 0.0, c.have ? a.px[c.i] : 0.0, c.have ? a.py[c.i] : 0.0,
           c.have ? a.pz[c.i] : 0.0);
    const StepK<double> hk = f.k64;
    const double* E = f.E64;
    auto e_at = [&](int64_t j) { return j < f.table_len ? __ldg(E + j) : 0.0; };
    double e0 = e_at(2 * c.n_first), e1 = e_at(2 * c.n_first + 1), e2 = e_at(2 * c.n_first + 2);
    const volatile int* alive = sm.alive;
    Producer out(0);
    for (int64_t n = c.n_first; n <= c.n_last; ++n) {
        {
            const int d = out.acquire();
            double* o = &sm.s01[d][0][lane];
            o[29 * kW] = T.q[0];
            o[30 * kW] = T.q[2];
            o[31 * kW] = T.p[0];
            o[32 * kW] = T.p[2];
            // the E values of the next step, loaded one step ahead
            const double f0 = e_at(2 * n + 2), f1 = e_at(2 * n + 3), f2 = e_at(2 * n + 4);
            const bool step = c.have && n >= c.n0 && n < c.n_last && alive[lane];
            if (step) {
                double qs[4][2], gs[4], hs[4], ps[4][2], Vs[4];
                T.stages_qp(e0, e1, e2, hk, pc, qs, gs, hs, ps, Vs);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    o[(2 * k) * kW] = qs[k][0];
                    o[(2 * k + 1) * kW] = qs[k][1];
                    o[(8 + k) * kW] = gs[k];
                    o[(12 + k) * kW] = hs[k];
                    o[(22 + k) * kW] = Vs[k];
                }
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    o[(14 + 2 * k) * kW] = ps[k][0];
                    o[(15 + 2 * k) * kW] = ps[k][1];
                }
            }
            out.publish(d);
            e0 = f0;
            e1 = f1;
            e2 = f2;
        }
    }
    out.drain();
}

// matrix: the step matrix of grid point n (one iteration behind the dynamics); the
// action increment's inputs go on to the columns warp
template <int POT>
__device__ void run_matrix(const FieldDev& f, const Common& c, Shared& sm, int lane) {
    const StepK<double> hk = f.k64;
    Consumer in_q(0);
    Producer out(1);
    for (int64_t n = c.n_first; n <= c.n_last; ++n) {
        {
            const int di = in_q.wait();
            const int dq = out.acquire();
            const double* in = &sm.s01[di][0][lane];
            double* o = &sm.s12[dq][0][lane];
#pragma unroll
            for (int k = 0; k < 4; ++k) o[(19 + k) * kW] = in[(29 + k) * kW];
            if (c.have && n >= c.n0 && n < c.n_last) {
                double qs[4][2], gs[4], hs[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    qs[k][0] = in[(2 * k) * kW];
                    qs[k][1] = in[(2 * k + 1) * kW];
                    gs[k] = in[(8 + k) * kW];
                    hs[k] = in[(12 + k) * kW];
                }
                const StepMat<double> M = TrajP<double, POT>::step_matrix(qs, gs, hs, hk);
#pragma unroll
                for (int k = 0; k < 19; ++k) o[k * kW] = M.m[k];
                // the action increment's inputs
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    o[(22 + k) * kW] = qs[k][1];
                    o[(24 + 2 * k) * kW] = in[(14 + 2 * k) * kW];
                    o[(25 + 2 * k) * kW] = in[(15 + 2 * k) * kW];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) o[(32 + k) * kW] = in[(22 + k) * kW];
            }
            in_q.release(di);
            out.publish(dq);
        }
    }
    out.drain();
}

// columns: the stability columns advanced by the step matrix of grid point n, and
// the action S (its increment from the stage data the matrix warp hands on)
template <int POT>
__device__ void run_columns(const FieldDev& f, const Common& c, Shared& sm, int lane) {
    TrajP<double, POT> T;
    T.init(0.0, 0.0, 0.0, 0.0, 0.0, 0.0);   // columns: identity (the state is read from the slots)
    const double h6 = f.k64.h6;
    Action<double> S;
    S.init();
    const volatile int* alive = sm.alive;
    Consumer in_q(1);
    Producer out(2);
    for (int64_t n = c.n_first; n <= c.n_last; ++n) {
        {
            const int di = in_q.wait();
            const int dq = out.acquire();
            const double* in = &sm.s12[di][0][lane];
            double* o = &sm.s23[dq][0][lane];
            const double s_n = S.value();   // the action at grid point n
            if (c.have && n >= c.n0 && n < c.n_last && alive[lane]) {
                StepMat<double> M;
#pragma unroll
                for (int k = 0; k < 19; ++k) M.m[k] = in[k * kW];
                T.apply_step_matrix(M);
            }
            if (c.have && n >= c.n0 && n < c.n_last) {
                double qs[4][2], ps[4][2], Vs[4];
                qs[0][1] = in[20 * kW];   // the state at n: q_z, p_x', p_z
                ps[0][0] = in[21 * kW];
                ps[0][1] = in[22 * kW];
#pragma unroll
                for (int k = 1; k < 4; ++k) {
                    qs[k][1] = in[(22 + k) * kW];
                    ps[k][0] = in[(24 + 2 * k) * kW];
                    ps[k][1] = in[(25 + 2 * k) * kW];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    qs[k][0] = 0.0;   // not read by the action terms
                    Vs[k] = in[(32 + k) * kW];
                }
                auto e_at = [&](int64_t j) { return j < f.table_len ? __ldg(f.E64 + j) : 0.0; };
                S.add(TrajP<double, POT>::action_increment(ps, qs, Vs, e_at(2 * n), e_at(2 * n + 1), e_at(2 * n + 2),
                                                           h6));
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                o[(4 * k) * kW] = T.X[k][0];
                o[(4 * k + 1) * kW] = T.X[k][1];
                o[(4 * k + 2) * kW] = T.Y[k][0];
                o[(4 * k + 3) * kW] = T.Y[k][1];
            }
            o[16 * kW] = T.aq;
            o[17 * kW] = T.ap;
            o[18 * kW] = T.bq;
            o[19 * kW] = T.bp;
#pragma unroll
            for (int k = 0; k < 4; ++k) o[(20 + k) * kW] = in[(19 + k) * kW];
            o[24 * kW] = s_n;
            in_q.release(di);
            out.publish(dq);
        }
    }
    out.drain();
}

// bins: det Z and its branch, labels, removal, prefactor and the recombination
// sums of the bins, a few GTO terms per grid point
template <int POT>
__device__ void run_bins(const FieldDev& f, const TargetDev& tg, const GtoTerms& gt, const TrajArgs& a,
                         const Common& c, Shared& sm, int lane) {
    const Cx<double> amp{c.have ? a.amp_re[c.i] : 0.0, c.have ? a.amp_im[c.i] : 0.0};
    const bool fbins = a.float_bins != 0;   // recombination terms in float (as the float pass forms them)
    const float gamf = (float)a.gamma;
    const int tps = (gt.n + c.n_out - 1) / c.n_out > 0 ? (gt.n + c.n_out - 1) / c.n_out : 1;
    TrajP<double, POT> T;                    // holds the columns read from the slots for detc
    T.init(0.0, 0.0, 0.0, 0.0, 0.0, 0.0);
    bool alive = c.alive0;
    unsigned flags = (c.have && !alive) ? 8u : 0u;
    Cx2<double> Dp{1.0, 0.0};
    double sgn = 1.0;
    const double rg = a.gamma;
    const bool pw = a.pw_mask != 0;
    const double pw_r2 = a.pw_radius * a.pw_radius;
    int pw_cls = -1;
    bool pw_in = false;
    unsigned long long all_steps = 0, steps = 0;
    // the bin in progress
    bool pending = false, valid = false;
    int64_t k_bin = 0;
    int j_next = 0;
    double bq0 = 0, bq2 = 0, bp0 = 0, bp2 = 0, bS = 0, p2s = 0, q2s = 0, pqs = 0;
    float p2f = 0.f, q2f = 0.f, pqf = 0.f;
    Cx<double> C{0.0, 0.0};
    GtoSums<double> acc{};
    GtoSums<float> accf{};
    auto terms = [&](int j0, int j1) {
        if (fbins) gto_terms<float>(gt, p2f, q2f, pqf, j0, j1, accf);
        else gto_terms<double>(gt, p2s, q2s, pqs, j0, j1, acc);
    };
    auto finish = [&]() {
        double cl = 0.0, cv = 0.0;
        if (valid) {
            terms(j_next, gt.n);
            const int64_t nb = k_bin * c.n_out;
            const double tk = f.t_start + (double)nb * f.dt;
            double sn, cs;
            sincos(fmod(tg.ip * tk, 2.0 * kPi), &sn, &cs);
            if (fbins) {
                float fl, fv;
                contribution_final<float>(FloatState(bq0, 0.0, bq2, bp0, 0.0, bp2, bS), gt, gamf,
                                          Cx<float>{(float)C.re, (float)C.im}, Cx<float>{(float)amp.re, (float)amp.im},
                                          Cx<float>{(float)cs, (float)(-sn)}, accf, fl, fv);
                cl = (double)fl;
                cv = (double)fv;
            } else {
                contribution_final<double>(PView(bq0, bq2, bp0, bp2, bS), gt, a.gamma, C, amp, Cx<double>{cs, -sn},
                                           acc, cl, cv);
            }
        }
        if (__any_sync(0xffffffffu, cl != 0.0 || cv != 0.0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                cl += __shfl_xor_sync(0xffffffffu, cl, o);
                cv += __shfl_xor_sync(0xffffffffu, cv, o);
            }
            const double sl = 0.0 + cl, sv = 0.0 + cv;
            if (lane == 0 && k_bin < f.n_bins && (sl != 0.0 || sv != 0.0)) {
                atomicAdd(&a.d_len[k_bin], sl);
                atomicAdd(&a.d_vel[k_bin], sv);
            }
        }
        pending = false;
    };
    int rem = (int)(c.n_first % c.n_out);
    int64_t k_next = (c.n_first + c.n_out - 1) / c.n_out;   // bin index of the next output point
    volatile int* alive_out = sm.alive;
    Consumer in_q(2);
    for (int64_t n = c.n_first; n <= c.n_last; ++n) {
        {
            const int di = in_q.wait();
            const double* in = &sm.s23[di][0][lane];
            const double q0 = in[20 * kW], q2 = in[21 * kW], p0 = in[22 * kW], p2 = in[23 * kW], S = in[24 * kW];
            const bool on_bin = rem == 0;
            // partial waves (Sec. III.A-B): class at each entry into r < R, labels at
            // every grid point from birth on while the trajectory is integrated
            if (pw && alive && n >= c.n0) {
                const double qx = q0, qy = 0.0, qz = q2;
                const bool inside = qx * qx + qy * qy + qz * qz < pw_r2;
                if (inside && !pw_in) {
                    const double px = p0, py = 0.0, pz = p2;
                    const double lx = qy * pz - qz * py, ly = qz * px - qx * pz, lz = qx * py - qy * px;
                    const double L2 = lx * lx + ly * ly + lz * lz;
                    pw_cls = L2 < 0.25 ? 0 : (L2 < 2.25 ? 1 : (L2 < 6.25 ? 2 : 3));
                }
                pw_in = inside;
            }
            const bool pw_ok = !pw || (pw_cls >= 0 && ((a.pw_mask >> pw_cls) & 1));
            if (on_bin) {
                if (pending) finish();
                valid = false;
                if (alive && n >= c.n0) {
                    const double fs = q0 + q2 + p0 + p2;
                    const bool ok = isfinite(fs) && isfinite(S);
                    const cd D{Dp.re, Dp.im};
                    const double m2 = D.re * D.re + D.im * D.im;
                    if (!ok || !(m2 <= a.d_t * a.d_t)) {
                        alive = false;
                        flags |= 1u;
                        if (!ok || !isfinite(m2)) flags |= 2u;
                    } else if (n >= c.k_cnt && pw_ok) {
                        cd Cz = c_sqrt(D);
                        if (sgn < 0.0) Cz = -Cz;
                        C = Cx<double>{Cz.re, Cz.im};
                        valid = true;
                        bq0 = q0;
                        bq2 = q2;
                        bp0 = p0;
                        bp2 = p2;
                        bS = S;
                        if (fbins)
                            recomb_invariants<float>(FloatState(bq0, 0.0, bq2, bp0, 0.0, bp2, bS), p2f, q2f, pqf);
                        else
                            recomb_invariants<double>(PView(bq0, bq2, bp0, bp2, bS), p2s, q2s, pqs);
                    }
                }
                k_bin = k_next++;
                pending = true;
                j_next = 0;
                acc = GtoSums<double>{};
                accf = GtoSums<float>{};
            }
            // the step n -> n + 1: det Z of the advanced columns and its branch
            if (alive && n >= c.n0 && n < c.n_last) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    T.X[k][0] = in[(4 * k) * kW];
                    T.X[k][1] = in[(4 * k + 1) * kW];
                    T.Y[k][0] = in[(4 * k + 2) * kW];
                    T.Y[k][1] = in[(4 * k + 3) * kW];
                }
                T.aq = in[16 * kW];
                T.ap = in[17 * kW];
                T.bq = in[18 * kW];
                T.bp = in[19 * kW];
                const Cx2<double> D = T.detc(0.5, -rg, a.qg64);
                follow_branch<double>(Dp, D, sgn, flags);
                ++all_steps;
                if (n >= c.k_cnt) ++steps;
            }
            in_q.release(di);
            alive_out[lane] = alive ? 1 : 0;
            rem = (rem + 1 == c.n_out) ? 0 : rem + 1;
        }
        if (pending) {
            const int j_end = j_next + tps < gt.n ? j_next + tps : gt.n;
            if (valid) terms(j_next, j_end);
            j_next = j_end;
            if (j_next >= gt.n) finish();
        }
    }
    if (pending) finish();
    if (a.stats) {
        unsigned rm = __reduce_add_sync(0xffffffffu, (flags & 1u) ? 1u : 0u);
        unsigned nf = __reduce_add_sync(0xffffffffu, (flags & 2u) ? 1u : 0u);
        unsigned bg = __reduce_add_sync(0xffffffffu, (flags & 4u) ? 1u : 0u);
        unsigned sk = __reduce_add_sync(0xffffffffu, (flags & 8u) ? 1u : 0u);
        unsigned long long st = steps, ast = all_steps;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st += __shfl_xor_sync(0xffffffffu, st, o);
            ast += __shfl_xor_sync(0xffffffffu, ast, o);
        }
        if (lane == 0) {
            if (rm) atomicAdd(&a.stats->removed, (unsigned long long)rm);
            if (nf) atomicAdd(&a.stats->nonfinite, (unsigned long long)nf);
            if (bg) atomicAdd(&a.stats->branch_guard, (unsigned long long)bg);
            if (sk) atomicAdd(&a.stats->skipped, (unsigned long long)sk);
            if (ast) atomicAdd(&a.stats->esc_steps, ast);
            if (ast > st) atomicAdd(&a.stats->esc_steps_pre, ast - st);
            if (st) atomicAdd(&a.stats->traj_steps, st);
        }
    }
}

// One group of 32 list entries (list positions 32 g .. 32 g + 31).
template <int POT>
__device__ void redo_group(const FieldDev& f, const TargetDev& tg, const GtoTerms& gt, const TrajArgs& a,
                           int64_t g, int64_t n_list, Shared& sm, int lane, int warp) {
    Common c;
    c.n_out = (int)f.n_out;
    c.n_last = a.n_last;
    const int64_t j = g * kW + lane;
    c.have = j < n_list;
    c.i = c.have ? (int64_t)a.idx[j] : 0;
    const int64_t k_min = c.have ? (int64_t)a.k_from[j] : 0;
    c.k_cnt = k_min * c.n_out;
    c.n0 = c.have ? (int64_t)a.n0[c.i] : 0;
    const double ar = c.have ? a.amp_re[c.i] : 0.0, ai = c.have ? a.amp_im[c.i] : 0.0;
    c.alive0 = c.have && c.n0 <= a.n_last && c.n0 >= 0 && (ar != 0.0 || ai != 0.0);
    // first grid point of the block: the earliest birth among its live trajectories
    long long m = c.alive0 ? (long long)c.n0 : LLONG_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t < m ? t : m;
    }
    if (m == LLONG_MAX) {
        // nothing to integrate; one warp still reports skipped births
        if (a.stats && warp == 0) {
            const unsigned sk = __reduce_add_sync(0xffffffffu, c.have ? 1u : 0u);
            if (lane == 0 && sk) atomicAdd(&a.stats->skipped, (unsigned long long)sk);
        }
        return;
    }
    c.n_first = m;
    if (warp == 0) sm.alive[lane] = c.alive0 ? 1 : 0;
    __syncthreads();
    const int role = (warp + (int)(g & 3)) & 3;
    if (role == 0) run_dynamics<POT>(f, tg, a, c, sm, lane);
    else if (role == 1) run_matrix<POT>(f, c, sm, lane);
    else if (role == 2) run_columns<POT>(f, c, sm, lane);
    else run_bins<POT>(f, tg, gt, a, c, sm, lane);
}

__device__ __forceinline__ unsigned sm_id() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Groups to SMs.  The list is in birth order, so group g's length (grid points from
// its earliest birth to the end) falls with g.  One warp plans the launch: it takes
// the groups longest first and gives each to the list (one per SM) with the least
// length so far (longest-processing-time-first), then lays the lists out in the
// scratch (plan: [0, L) counters, [K, K + L) list lengths, [2K, 2K + L) list starts,
// [3K, 3K + G) the groups list by list, longest first, then the assignment of each
// group; K = kRedoLists).  A block takes the groups of its own SM's list (one atomic
// counter per list), longest first, and then those left on the other lists, so
// every group is taken exactly once whatever the SMs' numbering and the blocks'
// placement.
__global__ void redo_plan_kernel(const int32_t* __restrict__ idx, const int32_t* __restrict__ n0,
                                 const int32_t* __restrict__ count, int64_t n_last, int L, int64_t g_max, int* plan) {
    __shared__ long long load[kRedoLists];
    __shared__ int cursor[kRedoLists];
    const int lane = threadIdx.x;   // one warp
    int* const len = plan + kRedoLists;
    int* const start = plan + 2 * kRedoLists;
    int* const grp = plan + 3 * kRedoLists;
    int* const asg = grp + g_max;
    const int64_t n_list = *count;
    const int64_t G = min((n_list + kW - 1) / kW, g_max);
    for (int l = lane; l < L; l += 32) {
        load[l] = 0;
        cursor[l] = 0;
    }
    __syncwarp();
    for (int64_t g = 0; g < G; ++g) {
        // the group's length: from its earliest birth in range to the end
        const int64_t j = g * kW + lane;
        long long m = LLONG_MAX;
        if (j < n_list) {
            const long long b = n0[idx[j]];
            if (b >= 0 && b <= n_last) m = b;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = min(m, (long long)__shfl_xor_sync(0xffffffffu, m, o));
        const long long lg = m == LLONG_MAX ? 1 : n_last - m + 1;
        // the least loaded list (ties: the lowest index)
        long long bv = LLONG_MAX;
        int bl = 0;
        for (int l = lane; l < L; l += 32)
            if (load[l] < bv) {
                bv = load[l];
                bl = l;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (ov < bv || (ov == bv && ol < bl)) {
                bv = ov;
                bl = ol;
            }
        }
        if (lane == 0) {
            load[bl] += lg;
            ++cursor[bl];
            asg[g] = bl;
        }
        __syncwarp();
    }
    // list starts: exclusive prefix of the list lengths
    if (lane == 0) {
        int acc = 0;
        for (int l = 0; l < L; ++l) {
            len[l] = cursor[l];
            start[l] = acc;
            acc += cursor[l];
            cursor[l] = 0;
        }
        // the groups list by list, in order of g (longest first)
        for (int64_t g = 0; g < G; ++g) {
            const int l = asg[g];
            grp[start[l] + cursor[l]++] = (int)g;
        }
    }
}

template <int POT>
__global__ void __launch_bounds__(kThreads, 4) redo_kernel(FieldDev f, TargetDev tg, GtoTerms gt, TrajArgs a) {
    __shared__ Shared sm;
    __shared__ long long s_g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_list = (int64_t)*a.count;
    const int L = a.redo_lists;
    const int* const len = a.redo_ctr + kRedoLists;
    const int* const start = a.redo_ctr + 2 * kRedoLists;
    const int* const grp = a.redo_ctr + 3 * kRedoLists;
    const int home = (int)(sm_id() % (unsigned)L);
    for (int probe = 0; probe < L; ++probe) {
        const int l = (home + probe) % L;
        for (;;) {
            if (threadIdx.x == 0) {
                const int k = atomicAdd(&a.redo_ctr[l], 1);
                s_g = k < len[l] ? (long long)grp[start[l] + k] : -1;
            }
            __syncthreads();
            const long long g = s_g;
            __syncthreads();   // every thread has read s_g before thread 0 writes the next
            if (g < 0) break;
            redo_group<POT>(f, tg, gt, a, (int64_t)g, n_list, sm, lane, warp);
            __syncthreads();   // every role has drained its hand-offs before the next group
        }
    }
}

template <int POT>
cudaError_t launch_pot(const FieldDev& f, const TargetDev& t, const GtoTerms& gt, const TrajArgs& a, cudaStream_t s) {
    // persistent: as many blocks as fit (4 per SM), each looping over groups
    const int64_t need = (a.n + kW - 1) / kW;   // an upper bound on the groups (the count is on the device)
    const int64_t blocks = std::min<int64_t>(need, (int64_t)a.redo_lists * 4);
    redo_kernel<POT><<<(unsigned)blocks, kThreads, 0, s>>>(f, t, gt, a);
    return cudaGetLastError();
}

}  // namespace

int64_t redo_blocks(int64_t n) { return (n + kW - 1) / kW; }

int redo_lists() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return std::max(1, std::min(sms, kRedoLists));
}

cudaError_t launch_redo(const FieldDev& f, const TargetDev& t, const TrajArgs& a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.redo_lists < 1 || a.redo_ctr == nullptr) return cudaErrorInvalidValue;
    if (a.redo_lists > kRedoLists) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(a.redo_ctr, 0, (size_t)a.redo_lists * sizeof(int), s);
    if (e != cudaSuccess) return e;
    redo_plan_kernel<<<1, 32, 0, s>>>(a.idx, a.n0, a.count, a.n_last, a.redo_lists, (int64_t)((a.n + kW - 1) / kW + 1),
                                      a.redo_ctr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const GtoTerms gt = make_gto_terms(t, a.gamma);
    switch (t.pot) {
        case POT_SOFTCORE: return launch_pot<POT_SOFTCORE>(f, t, gt, a, s);
        case POT_TONGLIN: return launch_pot<POT_TONGLIN>(f, t, gt, a, s);
        case POT_HARMONIC: return launch_pot<POT_HARMONIC>(f, t, gt, a, s);
        default: return launch_pot<POT_ZERO>(f, t, gt, a, s);
    }
}

}  // namespace sfhk
