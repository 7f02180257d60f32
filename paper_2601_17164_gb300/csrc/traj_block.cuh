// Trajectory block: classical propagation with stability blocks and action,
// Herman-Kluk prefactor with branch tracking and removal, and the fused
// recombination-dipole reduction.
//
//   App. A (after Eq. HKpropa): qdot = p, pdot = -grad V - E(t) z,
//     d/dt dq/dz = dp/dz, d/dt dp/dz = -Hess V dq/dz  (z = q0 or p0),
//     S = int (p.qdot - H) dt, H = p^2/2 + V(q) + z E(t).
//   Eq. C_HK: C = sqrt(det Z), Z = (Mpp + Mqq - 2 i gamma Mqp - Mpq/(2 i gamma))/2.
//   Sec. III.A: a trajectory with |C|^2 > D_t is removed (Kay).
//   App. C, Eq. D_t / Eq. V_t: recombination terms and their -2 Re sums.
//
// One trajectory per thread.  Classical RK4 with the grid step.  The four
// stage positions of (q, p, S) are integrated first and their Hessian data
// (g, h: Hess V = g I + h q q^T for a central potential) kept; the stability
// columns are then advanced with those stage Hessians, which is the same RK4
// on the 43-component state with far fewer live registers: in the 3D form the
// six columns of the 6x6 monodromy matrix one by one through the stages, in
// the planar form (25 components) all columns at once by the RK4 step written
// as one matrix [[A, B], [C, D]] (TrajP::step_matrix).  The float path packs
// its paired updates into FFMA2/FADD2/FMUL2 instructions.  The block walks the
// grid in lockstep; E(t) at the half steps is staged into shared memory per
// window of `chunk` steps; the per-bin contributions are warp-reduced into
// per-warp shared bins and flushed to global memory once per window.
//
// Shared by the single-configuration kernel (traj.cu) and the batched
// persistent kernel (batch.cu).
#pragma once

#include <type_traits>

#include "dfloat.cuh"
#include "sfhk_device.cuh"

namespace sfhk {
namespace {


constexpr int POT_ZERO = 0, POT_SOFTCORE = 1, POT_TONGLIN = 2, POT_HARMONIC = 3;

template <typename R>
struct Cx2 {
    R re, im;
};

template <typename R>
struct PotConst {
    R a2;                          // softcore a^2 ; harmonic w^2
    R Zc, a1, a2t, a3, a4, a5, a6; // Tong-Lin
};

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float ex(float x) { return expf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }

// V, and g, h with grad V = g q, Hess V = g I + h q q^T.
template <typename R, int POT>
__device__ __forceinline__ void potential(R x, R y, R z, const PotConst<R>& c, R& V, R& g, R& h) {
    if constexpr (POT == POT_SOFTCORE) {
        R r2 = fma(x, x, fma(y, y, fma(z, z, c.a2)));
        R s = rsq(r2);
        R s2 = s * s, s3 = s2 * s;
        V = -s;
        g = s3;
        h = R(-3) * s3 * s2;
    } else if constexpr (POT == POT_TONGLIN) {
        R r2 = fma(x, x, fma(y, y, z * z));
        R ir = rsq(r2);
        R r = r2 * ir;
        R e2 = ex(-c.a2t * r), e4 = ex(-c.a4 * r), e6 = ex(-c.a6 * r);
        R Y = c.Zc + c.a1 * e2 + c.a3 * r * e4 + c.a5 * e6;
        R Y1 = -c.a1 * c.a2t * e2 + c.a3 * (R(1) - c.a4 * r) * e4 - c.a5 * c.a6 * e6;
        R Y2 = c.a1 * c.a2t * c.a2t * e2 + c.a3 * (c.a4 * c.a4 * r - R(2) * c.a4) * e4 + c.a5 * c.a6 * c.a6 * e6;
        R ir2 = ir * ir;
        V = -Y * ir;
        g = (Y * ir - Y1) * ir2;
        h = (R(-3) * Y * ir2 + R(3) * Y1 * ir - Y2) * ir2 * ir;
    } else if constexpr (POT == POT_HARMONIC) {
        V = R(0.5) * c.a2 * fma(x, x, fma(y, y, z * z));
        g = c.a2;
        h = R(0);
    } else {
        V = R(0);
        g = R(0);
        h = R(0);
    }
}

// The same in the plane y = 0 of the planar form (the y terms, exactly zero there, dropped).
template <typename R, int POT>
__device__ __forceinline__ void potential_xz(R x, R z, const PotConst<R>& c, R& V, R& g, R& h) {
    if constexpr (POT == POT_SOFTCORE) {
        R r2 = fma(x, x, fma(z, z, c.a2));
        R s = rsq(r2);
        R s2 = s * s, s3 = s2 * s;
        V = -s;
        g = s3;
        h = R(-3) * s3 * s2;
    } else if constexpr (POT == POT_TONGLIN) {
        R r2 = fma(x, x, z * z);
        R ir = rsq(r2);
        R r = r2 * ir;
        R e2 = ex(-c.a2t * r), e4 = ex(-c.a4 * r), e6 = ex(-c.a6 * r);
        R Y = c.Zc + c.a1 * e2 + c.a3 * r * e4 + c.a5 * e6;
        R Y1 = -c.a1 * c.a2t * e2 + c.a3 * (R(1) - c.a4 * r) * e4 - c.a5 * c.a6 * e6;
        R Y2 = c.a1 * c.a2t * c.a2t * e2 + c.a3 * (c.a4 * c.a4 * r - R(2) * c.a4) * e4 + c.a5 * c.a6 * c.a6 * e6;
        R ir2 = ir * ir;
        V = -Y * ir;
        g = (Y * ir - Y1) * ir2;
        h = (R(-3) * Y * ir2 + R(3) * Y1 * ir - Y2) * ir2 * ir;
    } else {
        potential<R, POT>(x, R(0), z, c, V, g, h);
    }
}

// Action accumulator: plain in double; two-float reduced mod 2 pi in float.
template <typename R>
struct Action;
template <>
struct Action<double> {
    double s;
    __device__ void init() { s = 0.0; }
    __device__ void add(double d) { s += d; }
    __device__ double value() const { return s; }
    __device__ double reduced() const { return s; }
    __device__ bool finite() const { return isfinite(s); }
};
template <>
struct Action<float> {
    float hi, lo;
    int wraps;
    __device__ void init() {
        hi = 0.f;
        lo = 0.f;
        wraps = 0;
    }
    __device__ void add(float d) {
        // TwoSum (Knuth): hi + d = s + e exactly
        float s = hi + d;
        float bb = s - hi;
        float e = (hi - (s - bb)) + (d - bb);
        lo += e;
        hi = s;
        if (fabsf(hi) > 3.14159265f) {
            const float TWO_PI_HI = 6.28318548f, TWO_PI_LO = -1.7484555e-07f;  // 2 pi = HI + LO
            const bool pos = hi > 0.f;
            const float sg = pos ? 1.f : -1.f;
            hi -= sg * TWO_PI_HI;   // exact (Sterbenz)
            lo -= sg * TWO_PI_LO;
            wraps += pos ? 1 : -1;  // integer select: no float-to-int conversion on the step path
        }
    }
    // planar float pass: each step's increment a b joins lo in one FMA, and fold()
    // moves lo into hi (TwoSum, reduction) every fifth step and before every read
    // of the state; value() holds at any point
    __device__ void add_lazy(float a, float b) { lo = fmaf(a, b, lo); }
    __device__ void fold() {
        const float l = lo;
        lo = 0.f;
        add(l);
    }
    __device__ double value() const { return (double)wraps * 6.283185307179586 + (double)hi + (double)lo; }
    __device__ float reduced() const { return hi + lo; }
    __device__ bool finite() const { return isfinite(hi) && isfinite(lo); }   // value() finite, in float
    template <class F>
    __device__ __forceinline__ void visit(F&& f) {
        f(hi);
        f(lo);
        f(wraps);
    }
};

template <>
struct Action<dfloat> {
    dfloat s;
    __device__ void init() { s = dfloat(0.f); }
    __device__ void add(dfloat d) { s += d; }
    __device__ double value() const { return (double)s; }
    __device__ float reduced() const { return (float)fmod((double)s, 6.283185307179586); }
    __device__ bool finite() const { return isfinite((double)s); }
};

// Packed pairs of float operations (one FFMA2 / FADD2 / FMUL2 instruction does two
// independent correctly rounded operations): the float path issues half the
// instructions for its paired updates, with results identical to the scalar ones.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }  // a - b

// Compensated increment y += d (float); plain add for double and double-float.
template <typename R>
__device__ __forceinline__ void cadd(R& y, R& c, R d) {
    if constexpr (std::is_same<R, float>::value) {
        R dd = d + c;
        R t = y + dd;
        c = dd - (t - y);
        y = t;
    } else {
        y += d;
    }
}
// Compensated increment y += a b: in float the carry enters as the addend of the
// product's FMA (one rounding, one instruction less than cadd of a rounded product).
template <typename R>
__device__ __forceinline__ void caddm(R& y, R& c, R a, R b) {
    if constexpr (std::is_same<R, float>::value) {
        const R dd = fmaf(a, b, c);
        const R t = y + dd;
        c = dd - (t - y);
        y = t;
    } else {
        cadd<R>(y, c, a * b);
    }
}

// The step constants in the working arithmetic (double-float; float and FP64 read
// the host-made copies of the field record).
template <typename R>
__device__ __forceinline__ StepK<R> step_constants_dev(R h) {
    return StepK<R>{h, R(0.5) * h, h * R(1.0 / 6.0), h * h * R(1.0 / 6.0), h * h * h * R(1.0 / 12.0),
                    h * h * h * h * R(1.0 / 24.0)};
}

template <typename R, int POT>
struct Traj {
    R q[3], p[3], cq[3], cp[3];
    R cX[6][3], cY[6][3];  // compensation terms of the float monodromy columns
    R X[6][3], Y[6][3];   // columns of the monodromy matrix: X = dq/dz_c, Y = dp/dz_c
    Action<R> S;

    __device__ void init(R qx, R qy, R qz, R px, R py, R pz) {
        q[0] = qx; q[1] = qy; q[2] = qz;
        p[0] = px; p[1] = py; p[2] = pz;
#pragma unroll
        for (int i = 0; i < 3; ++i) { cq[i] = R(0); cp[i] = R(0); }
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int i = 0; i < 3; ++i) { cX[c][i] = R(0); cY[c][i] = R(0); }
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                X[c][i] = (c == i) ? R(1) : R(0);
                Y[c][i] = (c == i + 3) ? R(1) : R(0);
            }
        S.init();
    }

    // every member, in a fixed order (state saved between launches of a segmented pass)
    template <class F>
    __device__ __forceinline__ void visit(F&& f) {
#pragma unroll
        for (int i = 0; i < 3; ++i) { f(q[i]); f(p[i]); f(cq[i]); f(cp[i]); }
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int i = 0; i < 3; ++i) { f(X[c][i]); f(Y[c][i]); f(cX[c][i]); f(cY[c][i]); }
        S.visit(f);
    }

    // One classical RK4 step of length h with E at t, t + h/2, t + h.
    __device__ __forceinline__ void step(R Ea, R Eb, R Ec, const StepK<R>& k, const PotConst<R>& pc) {
        const R h = k.h, hh = k.hh, h6 = k.h6;
        R qs[4][3], gs[4], hs[4];
        R V, g, hc;
        // stage 1
        potential<R, POT>(q[0], q[1], q[2], pc, V, g, hc);
        R kp1[3] = {-g * q[0], -g * q[1], -fma(g, q[2], Ea)};
        R kS1 = fma(R(0.5), fma(p[0], p[0], fma(p[1], p[1], p[2] * p[2])), -fma(q[2], Ea, V));
#pragma unroll
        for (int i = 0; i < 3; ++i) qs[0][i] = q[i];
        gs[0] = g; hs[0] = hc;
        // stage 2
        R p2[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) { qs[1][i] = fma(hh, p[i], q[i]); p2[i] = fma(hh, kp1[i], p[i]); }
        potential<R, POT>(qs[1][0], qs[1][1], qs[1][2], pc, V, g, hc);
        gs[1] = g; hs[1] = hc;
        R kp2[3] = {-g * qs[1][0], -g * qs[1][1], -fma(g, qs[1][2], Eb)};
        R kS2 = fma(R(0.5), fma(p2[0], p2[0], fma(p2[1], p2[1], p2[2] * p2[2])), -fma(qs[1][2], Eb, V));
        // stage 3
        R p3[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) { qs[2][i] = fma(hh, p2[i], q[i]); p3[i] = fma(hh, kp2[i], p[i]); }
        potential<R, POT>(qs[2][0], qs[2][1], qs[2][2], pc, V, g, hc);
        gs[2] = g; hs[2] = hc;
        R kp3[3] = {-g * qs[2][0], -g * qs[2][1], -fma(g, qs[2][2], Eb)};
        R kS3 = fma(R(0.5), fma(p3[0], p3[0], fma(p3[1], p3[1], p3[2] * p3[2])), -fma(qs[2][2], Eb, V));
        // stage 4
        R p4[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) { qs[3][i] = fma(h, p3[i], q[i]); p4[i] = fma(h, kp3[i], p[i]); }
        potential<R, POT>(qs[3][0], qs[3][1], qs[3][2], pc, V, g, hc);
        gs[3] = g; hs[3] = hc;
        R kp4[3] = {-g * qs[3][0], -g * qs[3][1], -fma(g, qs[3][2], Ec)};
        R kS4 = fma(R(0.5), fma(p4[0], p4[0], fma(p4[1], p4[1], p4[2] * p4[2])), -fma(qs[3][2], Ec, V));
        // combine (weights 1/6, 1/3, 1/3, 1/6)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const R sq = fma(R(2), p2[i] + p3[i], p[i]) + p4[i];
            const R sp = fma(R(2), kp2[i] + kp3[i], kp1[i]) + kp4[i];
            caddm<R>(q[i], cq[i], h6, sq);
            caddm<R>(p[i], cp[i], h6, sp);
        }
        S.add(h6 * (fma(R(2), kS2 + kS3, kS1) + kS4));
        // monodromy columns with the stage Hessians H_s v = g_s v + h_s q_s (q_s.v)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            R x[3], y[3], xs[3], ys[3], ky[3], ay[3], ax[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) { x[i] = X[c][i]; y[i] = Y[c][i]; }
            // stage 1: kx = y, ky = -H1 x
            R d = fma(qs[0][0], x[0], fma(qs[0][1], x[1], qs[0][2] * x[2])) * hs[0];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                ky[i] = -fma(gs[0], x[i], d * qs[0][i]);
                ax[i] = y[i];
                ay[i] = ky[i];
                xs[i] = fma(hh, y[i], x[i]);
                ys[i] = fma(hh, ky[i], y[i]);
            }
            // stage 2: kx = ys, ky = -H2 xs
            d = fma(qs[1][0], xs[0], fma(qs[1][1], xs[1], qs[1][2] * xs[2])) * hs[1];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                ky[i] = -fma(gs[1], xs[i], d * qs[1][i]);
                ax[i] = fma(R(2), ys[i], ax[i]);
                ay[i] = fma(R(2), ky[i], ay[i]);
                xs[i] = fma(hh, ys[i], x[i]);
                ys[i] = fma(hh, ky[i], y[i]);
            }
            // stage 3
            d = fma(qs[2][0], xs[0], fma(qs[2][1], xs[1], qs[2][2] * xs[2])) * hs[2];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                ky[i] = -fma(gs[2], xs[i], d * qs[2][i]);
                ax[i] = fma(R(2), ys[i], ax[i]);
                ay[i] = fma(R(2), ky[i], ay[i]);
                xs[i] = fma(h, ys[i], x[i]);
                ys[i] = fma(h, ky[i], y[i]);
            }
            // stage 4
            d = fma(qs[3][0], xs[0], fma(qs[3][1], xs[1], qs[3][2] * xs[2])) * hs[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                ky[i] = -fma(gs[3], xs[i], d * qs[3][i]);
                ax[i] += ys[i];
                ay[i] += ky[i];
                caddm<R>(X[c][i], cX[c][i], h6, ax[i]);
                caddm<R>(Y[c][i], cY[c][i], h6, ay[i]);
            }
        }
    }

    __device__ bool finite_state() const {
        R s = q[0] + q[1] + q[2] + p[0] + p[1] + p[2];
        return isfinite(s) && S.finite();
    }

    __device__ __forceinline__ cd det64(double gam) const;
    __device__ __forceinline__ Cx2<R> detc(R hz, R gz, R qz) const;
};

// Planar form of the same state.  With the field along z, a central potential
// and a birth at q0 = (0, 0, qz), the motion stays in the plane spanned by z and
// the initial transverse momentum.  In coordinates rotated about z so that this
// momentum lies along x', the monodromy matrix splits into an in-plane block
// (x', z; four columns of four) and the out-of-plane y block (two columns of
// two, Hess V_yy = g): 25 reals instead of 43, the same RK4 arithmetic, and
// det Z = det(Z_in-plane) * Z_yy (Z in the rotated frame is R Z R^T).
// q[1] = p[1] = 0 throughout; the recombination terms need only p^2, q^2, p.q,
// p_z and q_z, which the rotation leaves unchanged.
// Compensated increment of a pair (y0, y1) += d, the carries (c0, c1): the float
// cadd below, two at a time, with d + c formed by the caller (the carries as the
// innermost addends of the increments' FMA chains: one rounding, no separate add).
__device__ __forceinline__ void cadd2(float& y0, float& y1, float& c0, float& c1, float2 dd) {
    const float2 y = f2(y0, y1);
    const float2 t = add2(y, dd);
    const float2 c = sub2(dd, sub2(t, y));
    y0 = t.x;
    y1 = t.y;
    c0 = c.x;
    c1 = c.y;
}

// One RK4 step of the planar stability equations as a matrix: A (4), B (3, symmetric),
// C (4), D (4) in-plane, then the out-of-plane a, b, c, d.
template <typename R>
struct StepMat {
    R m[19];
};

template <typename R, int POT>
struct TrajP {
    R q[3], p[3], cq[3], cp[3];
    R X[4][2], Y[4][2], cX[4][2], cY[4][2];   // in-plane columns (z_c = x0', z0, px0', pz0), compensation
    R aq, ap, bq, bp, caq, cap, cbq, cbp;     // out-of-plane: (dy, dpy)/dy0 and (dy, dpy)/dpy0, compensation
    Action<R> S;

    __device__ void init(R qx, R qy, R qz, R px, R py, R pz) {
        (void)qx;
        (void)qy;   // zero by the planar precondition
        q[0] = R(0); q[1] = R(0); q[2] = qz;
        p[0] = sqrt(px * px + py * py); p[1] = R(0); p[2] = pz;
#pragma unroll
        for (int i = 0; i < 3; ++i) { cq[i] = R(0); cp[i] = R(0); }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                X[c][i] = (c == i) ? R(1) : R(0);
                Y[c][i] = (c == i + 2) ? R(1) : R(0);
                cX[c][i] = R(0);
                cY[c][i] = R(0);
            }
        aq = R(1); ap = R(0); bq = R(0); bp = R(1);
        caq = cap = cbq = cbp = R(0);
        S.init();
    }

    template <class F>
    __device__ __forceinline__ void visit(F&& f) {
#pragma unroll
        for (int i = 0; i < 3; ++i) { f(q[i]); f(p[i]); f(cq[i]); f(cp[i]); }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int i = 0; i < 2; ++i) { f(X[c][i]); f(Y[c][i]); f(cX[c][i]); f(cY[c][i]); }
        f(aq); f(ap); f(bq); f(bp); f(caq); f(cap); f(cbq); f(cbp);
        S.visit(f);
    }

    __device__ __forceinline__ void step(R Ea, R Eb, R Ec, const StepK<R>& k, const PotConst<R>& pc) {
        R qs[4][2], gs[4], hs[4];
        stages(Ea, Eb, Ec, k, pc, qs, gs, hs);
        // The RK4 step of the linear stability equations written once as a matrix,
        // d[x; p] = [[A, B], [C, D]] [x; p], from the stage Hessians H_s (2x2
        // symmetric a, b, c; exact algebra of the four RK4 stages):
        //   A = -h^2/6 (H1+H2+H3) + h^4/24 H3 H1      B = h I - h^3/12 (H2+H3)
        //   C = -h/6 (H1+2H2+2H3+H4) + h^3/12 (H3 H1 + H4 H2)
        //   D = -h^2/6 (H2+H3+H4) + h^4/24 H4 H2
        // then applied to the four in-plane columns (and, with H_s = g_s, to the
        // two out-of-plane ones); in float the increments are added compensated
        apply_step_matrix(step_matrix(qs, gs, hs, k));
    }

    // RK4 step of (q, p, S); returns the stage positions and the Hessian data (g, h) there
    __device__ __forceinline__ void stages(R Ea, R Eb, R Ec, const StepK<R>& k, const PotConst<R>& pc, R qs[4][2],
                                           R gs[4], R hs[4]) {
        stages_impl<true>(Ea, Eb, Ec, k, pc, qs, gs, hs, nullptr, nullptr);
    }
    // the same step of (q, p) alone; the stage momenta ps and potentials Vs that the
    // action increment needs are returned instead (action_increment gives it)
    __device__ __forceinline__ void stages_qp(R Ea, R Eb, R Ec, const StepK<R>& k, const PotConst<R>& pc,
                                              R qs[4][2], R gs[4], R hs[4], R ps[4][2], R Vs[4]) {
        stages_impl<false>(Ea, Eb, Ec, k, pc, qs, gs, hs, ps, Vs);
    }
    // integrand p^2/2 - (V + z E) of the action at one stage, and the RK4 sum
    __device__ __forceinline__ static R action_term(R p0, R p2, R qz, R E, R V) {
        return fma(R(0.5), fma(p0, p0, p2 * p2), -fma(qz, E, V));
    }
    __device__ __forceinline__ static R action_sum(R kS1, R kS2, R kS3, R kS4, R h6) {
        return h6 * (fma(R(2), kS2 + kS3, kS1) + kS4);
    }
    __device__ __forceinline__ static R action_increment(const R ps[4][2], const R qs[4][2], const R Vs[4], R Ea, R Eb,
                                                         R Ec, R h6) {
        return action_sum(action_term(ps[0][0], ps[0][1], qs[0][1], Ea, Vs[0]),
                          action_term(ps[1][0], ps[1][1], qs[1][1], Eb, Vs[1]),
                          action_term(ps[2][0], ps[2][1], qs[2][1], Eb, Vs[2]),
                          action_term(ps[3][0], ps[3][1], qs[3][1], Ec, Vs[3]), h6);
    }

    template <bool ACTION>
    __device__ __forceinline__ void stages_impl(R Ea, R Eb, R Ec, const StepK<R>& k, const PotConst<R>& pc,
                                                R qs[4][2], R gs[4], R hs[4], R (*ps)[2], R* Vs) {
        if constexpr (std::is_same<R, float>::value) {
            stages_packed<ACTION>(Ea, Eb, Ec, k, pc, qs, gs, hs, ps, Vs);
            return;
        }
        const R h = k.h, hh = k.hh, h6 = k.h6;
        R V, g, hc;
        R kS1 = R(0), kS2 = R(0), kS3 = R(0), kS4 = R(0);
        // stage 1 (in-plane components: [0] = x', [1] = z)
        potential_xz<R, POT>(q[0], q[2], pc, V, g, hc);
        const R kp1[2] = {-g * q[0], -fma(g, q[2], Ea)};
        if constexpr (ACTION) kS1 = action_term(p[0], p[2], q[2], Ea, V);
        else { ps[0][0] = p[0]; ps[0][1] = p[2]; Vs[0] = V; }
        qs[0][0] = q[0]; qs[0][1] = q[2]; gs[0] = g; hs[0] = hc;
        // stage 2
        const R p2[2] = {fma(hh, kp1[0], p[0]), fma(hh, kp1[1], p[2])};
        qs[1][0] = fma(hh, p[0], q[0]); qs[1][1] = fma(hh, p[2], q[2]);
        potential_xz<R, POT>(qs[1][0], qs[1][1], pc, V, g, hc);
        gs[1] = g; hs[1] = hc;
        const R kp2[2] = {-g * qs[1][0], -fma(g, qs[1][1], Eb)};
        if constexpr (ACTION) kS2 = action_term(p2[0], p2[1], qs[1][1], Eb, V);
        else { ps[1][0] = p2[0]; ps[1][1] = p2[1]; Vs[1] = V; }
        // stage 3
        const R p3[2] = {fma(hh, kp2[0], p[0]), fma(hh, kp2[1], p[2])};
        qs[2][0] = fma(hh, p2[0], q[0]); qs[2][1] = fma(hh, p2[1], q[2]);
        potential_xz<R, POT>(qs[2][0], qs[2][1], pc, V, g, hc);
        gs[2] = g; hs[2] = hc;
        const R kp3[2] = {-g * qs[2][0], -fma(g, qs[2][1], Eb)};
        if constexpr (ACTION) kS3 = action_term(p3[0], p3[1], qs[2][1], Eb, V);
        else { ps[2][0] = p3[0]; ps[2][1] = p3[1]; Vs[2] = V; }
        // stage 4
        const R p4[2] = {fma(h, kp3[0], p[0]), fma(h, kp3[1], p[2])};
        qs[3][0] = fma(h, p3[0], q[0]); qs[3][1] = fma(h, p3[1], q[2]);
        potential_xz<R, POT>(qs[3][0], qs[3][1], pc, V, g, hc);
        gs[3] = g; hs[3] = hc;
        const R kp4[2] = {-g * qs[3][0], -fma(g, qs[3][1], Ec)};
        if constexpr (ACTION) kS4 = action_term(p4[0], p4[1], qs[3][1], Ec, V);
        else { ps[3][0] = p4[0]; ps[3][1] = p4[1]; Vs[3] = V; }
        // combine
        const R pp0 = p[0], pp2 = p[2];
        cadd<R>(q[0], cq[0], h6 * (fma(R(2), p2[0] + p3[0], pp0) + p4[0]));
        cadd<R>(q[2], cq[2], h6 * (fma(R(2), p2[1] + p3[1], pp2) + p4[1]));
        cadd<R>(p[0], cp[0], h6 * (fma(R(2), kp2[0] + kp3[0], kp1[0]) + kp4[0]));
        cadd<R>(p[2], cp[2], h6 * (fma(R(2), kp2[1] + kp3[1], kp1[1]) + kp4[1]));
        if constexpr (ACTION) S.add(action_sum(kS1, kS2, kS3, kS4, h6));
    }

    // the float stages with the (x', z) pairs of positions and momenta in packed
    // instructions; every component is the same operation as in the scalar form
    template <bool ACTION>
    __device__ __forceinline__ void stages_packed(float Ea, float Eb, float Ec, const StepK<float>& k,
                                                  const PotConst<float>& pc, float qs[4][2], float gs[4], float hs[4],
                                                  float (*ps)[2], float* Vs) {
        const float h = k.h, hh = k.hh, h6 = k.h6;
        const float2 hh2 = f2(hh, hh), h2 = f2(h, h), h62 = f2(h6, h6), two2 = f2(2.f, 2.f);
        const float2 Q = f2(q[0], q[2]), P = f2(p[0], p[2]);
        float V, g, hc;
        float kS1 = 0.f, kS2 = 0.f, kS3 = 0.f, kS4 = 0.f;
        // stage 1
        potential_xz<float, POT>(Q.x, Q.y, pc, V, g, hc);
        const float2 kp1 = fma2(f2(-g, -g), Q, f2(0.f, -Ea));       // (-g x', -(g z + E))
        if constexpr (ACTION) kS1 = action_term(P.x, P.y, Q.y, Ea, V);
        else { ps[0][0] = P.x; ps[0][1] = P.y; Vs[0] = V; }
        qs[0][0] = Q.x; qs[0][1] = Q.y; gs[0] = g; hs[0] = hc;
        // stage 2
        const float2 P2 = fma2(hh2, kp1, P), Q2 = fma2(hh2, P, Q);
        potential_xz<float, POT>(Q2.x, Q2.y, pc, V, g, hc);
        gs[1] = g; hs[1] = hc; qs[1][0] = Q2.x; qs[1][1] = Q2.y;
        const float2 kp2 = fma2(f2(-g, -g), Q2, f2(0.f, -Eb));
        if constexpr (ACTION) kS2 = action_term(P2.x, P2.y, Q2.y, Eb, V);
        else { ps[1][0] = P2.x; ps[1][1] = P2.y; Vs[1] = V; }
        // stage 3
        const float2 P3 = fma2(hh2, kp2, P), Q3 = fma2(hh2, P2, Q);
        potential_xz<float, POT>(Q3.x, Q3.y, pc, V, g, hc);
        gs[2] = g; hs[2] = hc; qs[2][0] = Q3.x; qs[2][1] = Q3.y;
        const float2 kp3 = fma2(f2(-g, -g), Q3, f2(0.f, -Eb));
        if constexpr (ACTION) kS3 = action_term(P3.x, P3.y, Q3.y, Eb, V);
        else { ps[2][0] = P3.x; ps[2][1] = P3.y; Vs[2] = V; }
        // stage 4
        const float2 P4 = fma2(h2, kp3, P), Q4 = fma2(h2, P3, Q);
        potential_xz<float, POT>(Q4.x, Q4.y, pc, V, g, hc);
        gs[3] = g; hs[3] = hc; qs[3][0] = Q4.x; qs[3][1] = Q4.y;
        const float2 kp4 = fma2(f2(-g, -g), Q4, f2(0.f, -Ec));
        if constexpr (ACTION) kS4 = action_term(P4.x, P4.y, Q4.y, Ec, V);
        else { ps[3][0] = P4.x; ps[3][1] = P4.y; Vs[3] = V; }
        // combine
        cadd2(q[0], q[2], cq[0], cq[2], fma2(h62, add2(fma2(two2, add2(P2, P3), P), P4), f2(cq[0], cq[2])));
        cadd2(p[0], p[2], cp[0], cp[2], fma2(h62, add2(fma2(two2, add2(kp2, kp3), kp1), kp4), f2(cp[0], cp[2])));
        if constexpr (ACTION) S.add_lazy(h6, fmaf(2.f, kS2 + kS3, kS1) + kS4);
    }

    // the step matrix [[A, B], [C, D]] (in-plane) and its out-of-plane 2x2 analogue
    __device__ __forceinline__ static StepMat<R> step_matrix(const R qs[4][2], const R gs[4], const R hs[4],
                                                             const StepK<R>& k) {
        R Ha[4], Hb[4], Hc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const R hx = hs[k] * qs[k][0];
            Ha[k] = fma(hx, qs[k][0], gs[k]);
            Hb[k] = hx * qs[k][1];
            Hc[k] = fma(hs[k] * qs[k][1], qs[k][1], gs[k]);
        }
        const R h = k.h, c2 = k.c2, c4 = k.c4, c3 = k.c3, c1 = k.h6;
        // S23 = H2 + H3, S123, S234, W = H1 + 2 S23 + H4
        const R s23a = Ha[1] + Ha[2], s23b = Hb[1] + Hb[2], s23c = Hc[1] + Hc[2];
        // P31 = H3 H1, P42 = H4 H2 (products of symmetric 2x2, general)
        const R p31aa = fma(Ha[2], Ha[0], Hb[2] * Hb[0]), p31ab = fma(Ha[2], Hb[0], Hb[2] * Hc[0]);
        const R p31ba = fma(Hb[2], Ha[0], Hc[2] * Hb[0]), p31bb = fma(Hb[2], Hb[0], Hc[2] * Hc[0]);
        const R p42aa = fma(Ha[3], Ha[1], Hb[3] * Hb[1]), p42ab = fma(Ha[3], Hb[1], Hb[3] * Hc[1]);
        const R p42ba = fma(Hb[3], Ha[1], Hc[3] * Hb[1]), p42bb = fma(Hb[3], Hb[1], Hc[3] * Hc[1]);
        const R Aaa = fma(c4, p31aa, -c2 * (s23a + Ha[0])), Aab = fma(c4, p31ab, -c2 * (s23b + Hb[0]));
        const R Aba = fma(c4, p31ba, -c2 * (s23b + Hb[0])), Abb = fma(c4, p31bb, -c2 * (s23c + Hc[0]));
        const R Baa = fma(-c3, s23a, h), Bab = -c3 * s23b, Bbb = fma(-c3, s23c, h);
        const R Caa = fma(c3, p31aa + p42aa, -c1 * (fma(R(2), s23a, Ha[0]) + Ha[3]));
        const R Cab = fma(c3, p31ab + p42ab, -c1 * (fma(R(2), s23b, Hb[0]) + Hb[3]));
        const R Cba = fma(c3, p31ba + p42ba, -c1 * (fma(R(2), s23b, Hb[0]) + Hb[3]));
        const R Cbb = fma(c3, p31bb + p42bb, -c1 * (fma(R(2), s23c, Hc[0]) + Hc[3]));
        const R Daa = fma(c4, p42aa, -c2 * (s23a + Ha[3])), Dab = fma(c4, p42ab, -c2 * (s23b + Hb[3]));
        const R Dba = fma(c4, p42ba, -c2 * (s23b + Hb[3])), Dbb = fma(c4, p42bb, -c2 * (s23c + Hc[3]));
        // out-of-plane: H_s = g_s
        const R g23 = gs[1] + gs[2];
        const R oa = fma(c4, gs[2] * gs[0], -c2 * (g23 + gs[0]));
        const R ob = fma(-c3, g23, h);
        const R oc = fma(c3, fma(gs[2], gs[0], gs[3] * gs[1]), -c1 * (fma(R(2), g23, gs[0]) + gs[3]));
        const R od = fma(c4, gs[3] * gs[1], -c2 * (g23 + gs[3]));
        return StepMat<R>{{Aaa, Aab, Aba, Abb, Baa, Bab, Bbb, Caa, Cab, Cba, Cbb, Daa, Dab, Dba, Dbb, oa, ob, oc, od}};
    }

    // columns += M columns (compensated in float)
    __device__ __forceinline__ void apply_step_matrix(const StepMat<R>& M) {
        const R Aaa = M.m[0], Aab = M.m[1], Aba = M.m[2], Abb = M.m[3], Baa = M.m[4], Bab = M.m[5], Bbb = M.m[6];
        const R Caa = M.m[7], Cab = M.m[8], Cba = M.m[9], Cbb = M.m[10], Daa = M.m[11], Dab = M.m[12];
        const R Dba = M.m[13], Dbb = M.m[14], oa = M.m[15], ob = M.m[16], oc = M.m[17], od = M.m[18];
        if constexpr (std::is_same<R, float>::value) {
            // rows in pairs: (dx0, dx1) and (dy0, dy1) of each column in packed instructions,
            // each increment added with Kahan's compensation (with one rounded add instead
            // the float pass is 13 % faster, but the plateau yields of 1e6-birth H samples
            // move up to 4.3e-4 from FP64 instead of 9e-5, Ar 1600 nm 1.7e-4 instead of 1.1e-5)
            const float2 A0 = f2(Aaa, Aba), A1 = f2(Aab, Abb), B0 = f2(Baa, Bab), B1 = f2(Bab, Bbb);
            const float2 C0 = f2(Caa, Cba), C1 = f2(Cab, Cbb), D0 = f2(Daa, Dba), D1 = f2(Dab, Dbb);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float2 X0 = f2(X[c][0], X[c][0]), X1 = f2(X[c][1], X[c][1]);
                const float2 Y0 = f2(Y[c][0], Y[c][0]), Y1 = f2(Y[c][1], Y[c][1]);
                const float2 dx = fma2(A0, X0, fma2(A1, X1, fma2(B0, Y0, fma2(B1, Y1, f2(cX[c][0], cX[c][1])))));
                const float2 dy = fma2(C0, X0, fma2(C1, X1, fma2(D0, Y0, fma2(D1, Y1, f2(cY[c][0], cY[c][1])))));
                cadd2(X[c][0], X[c][1], cX[c][0], cX[c][1], dx);
                cadd2(Y[c][0], Y[c][1], cY[c][0], cY[c][1], dy);
            }
            const float2 O0 = f2(oa, oc), O1 = f2(ob, od);
            cadd2(aq, ap, caq, cap, fma2(O0, f2(aq, aq), fma2(O1, f2(ap, ap), f2(caq, cap))));
            cadd2(bq, bp, cbq, cbp, fma2(O0, f2(bq, bq), fma2(O1, f2(bp, bp), f2(cbq, cbp))));
            return;
        }
        if constexpr (std::is_same<R, double>::value) {
            // FP64: each entry's old value is the innermost addend of its FMA chain,
            // x + (a x0 + b x1 + c y0 + d y1) as four FMAs instead of three, a
            // multiply and an add (the FP64 units are the bound of the FP64 kernels)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const R x0 = X[c][0], x1 = X[c][1], y0 = Y[c][0], y1 = Y[c][1];
                X[c][0] = fma(Aaa, x0, fma(Aab, x1, fma(Baa, y0, fma(Bab, y1, x0))));
                X[c][1] = fma(Aba, x0, fma(Abb, x1, fma(Bab, y0, fma(Bbb, y1, x1))));
                Y[c][0] = fma(Caa, x0, fma(Cab, x1, fma(Daa, y0, fma(Dab, y1, y0))));
                Y[c][1] = fma(Cba, x0, fma(Cbb, x1, fma(Dba, y0, fma(Dbb, y1, y1))));
            }
            const R aq0 = aq, ap0 = ap, bq0 = bq, bp0 = bp;
            aq = fma(oa, aq0, fma(ob, ap0, aq0));
            ap = fma(oc, aq0, fma(od, ap0, ap0));
            bq = fma(oa, bq0, fma(ob, bp0, bq0));
            bp = fma(oc, bq0, fma(od, bp0, bp0));
            return;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const R x0 = X[c][0], x1 = X[c][1], y0 = Y[c][0], y1 = Y[c][1];
            const R dx0 = fma(Aaa, x0, fma(Aab, x1, fma(Baa, y0, Bab * y1)));
            const R dx1 = fma(Aba, x0, fma(Abb, x1, fma(Bab, y0, Bbb * y1)));
            const R dy0 = fma(Caa, x0, fma(Cab, x1, fma(Daa, y0, Dab * y1)));
            const R dy1 = fma(Cba, x0, fma(Cbb, x1, fma(Dba, y0, Dbb * y1)));
            X[c][0] += dx0;
            X[c][1] += dx1;
            Y[c][0] += dy0;
            Y[c][1] += dy1;
        }
        const R daq = fma(oa, aq, ob * ap), dap = fma(oc, aq, od * ap);
        const R dbq = fma(oa, bq, ob * bp), dbp = fma(oc, bq, od * bp);
        aq += daq;
        ap += dap;
        bq += dbq;
        bp += dbp;
    }

    __device__ bool finite_state() const {
        R s = q[0] + q[2] + p[0] + p[2];
        return isfinite(s) && S.finite();
    }

    // det Z in FP64: det of the in-plane 2x2 block times Z_yy
    __device__ __forceinline__ cd det64(double gam) const {
        const double qg = 0.25 / gam;
        double zr[2][2], zi[2][2], yr, yi;
        if constexpr (std::is_same<R, float>::value) {
            // float blocks: Z's entries formed in float (their rounding is below the
            // blocks' own float error), the determinant in FP64
            const float g = (float)gam, q = (float)qg;
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    zr[i][j] = (double)(0.5f * (Y[2 + j][i] + X[j][i]));
                    zi[i][j] = (double)fmaf(-g, X[2 + j][i], q * Y[j][i]);
                }
            yr = (double)(0.5f * (bp + aq));
            yi = (double)fmaf(-g, bq, q * ap);
        } else {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    zr[i][j] = 0.5 * ((double)Y[2 + j][i] + (double)X[j][i]);
                    zi[i][j] = fma(-gam, (double)X[2 + j][i], qg * (double)Y[j][i]);
                }
            yr = 0.5 * ((double)bp + (double)aq);
            yi = fma(-gam, (double)bq, qg * (double)ap);
        }
        const double ar = fma(zr[0][0], zr[1][1], -zi[0][0] * zi[1][1]) - fma(zr[0][1], zr[1][0], -zi[0][1] * zi[1][0]);
        const double ai = fma(zr[0][0], zi[1][1], zi[0][0] * zr[1][1]) - fma(zr[0][1], zi[1][0], zi[0][1] * zr[1][0]);
        return cd{fma(ar, yr, -ai * yi), fma(ar, yi, ai * yr)};
    }

    // float: the action's pending increments moved into its two-float value
    __device__ __forceinline__ void settle() {
        if constexpr (std::is_same<R, float>::value) S.fold();
    }

    // det(c Z) in the working precision (argument only)
    __device__ __forceinline__ Cx2<R> detc(R hz, R gz, R qz) const {
        R zr[2][2], zi[2][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                zr[i][j] = hz * (Y[2 + j][i] + X[j][i]);
                zi[i][j] = fma(gz, X[2 + j][i], qz * Y[j][i]);
            }
        const R ar = fma(zr[0][0], zr[1][1], -zi[0][0] * zi[1][1]) - fma(zr[0][1], zr[1][0], -zi[0][1] * zi[1][0]);
        const R ai = fma(zr[0][0], zi[1][1], zi[0][0] * zr[1][1]) - fma(zr[0][1], zi[1][0], zi[0][1] * zr[1][0]);
        const R yr = hz * (bp + aq);
        const R yi = fma(gz, bq, qz * ap);
        return Cx2<R>{fma(ar, yr, -ai * yi), fma(ar, yi, ai * yr)};
    }
};

// det Z in FP64 from the monodromy columns.
template <typename R, int POT>
__device__ __forceinline__ cd det_Z(const Traj<R, POT>& T, double gam) {
    double zr[3][3], zi[3][3];
    const double qg = 0.25 / gam;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            // Mqq[i][j] = X[j][i], Mqp[i][j] = X[3+j][i], Mpq[i][j] = Y[j][i], Mpp[i][j] = Y[3+j][i]
            zr[i][j] = 0.5 * ((double)T.Y[3 + j][i] + (double)T.X[j][i]);
            zi[i][j] = fma(-gam, (double)T.X[3 + j][i], qg * (double)T.Y[j][i]);
        }
    auto mul = [](double ar, double ai, double br, double bi, double& cr, double& ci) {
        cr = fma(ar, br, -ai * bi);
        ci = fma(ar, bi, ai * br);
    };
    double m0r, m0i, m1r, m1i, m2r, m2i, tr, ti;
    mul(zr[1][1], zi[1][1], zr[2][2], zi[2][2], m0r, m0i);
    mul(zr[1][2], zi[1][2], zr[2][1], zi[2][1], tr, ti);
    m0r -= tr; m0i -= ti;
    mul(zr[1][0], zi[1][0], zr[2][2], zi[2][2], m1r, m1i);
    mul(zr[1][2], zi[1][2], zr[2][0], zi[2][0], tr, ti);
    m1r -= tr; m1i -= ti;
    mul(zr[1][0], zi[1][0], zr[2][1], zi[2][1], m2r, m2i);
    mul(zr[1][1], zi[1][1], zr[2][0], zi[2][0], tr, ti);
    m2r -= tr; m2i -= ti;
    double dr, di, ar, ai;
    mul(zr[0][0], zi[0][0], m0r, m0i, dr, di);
    mul(zr[0][1], zi[0][1], m1r, m1i, ar, ai);
    dr -= ar; di -= ai;
    mul(zr[0][2], zi[0][2], m2r, m2i, ar, ai);
    dr += ar; di += ai;
    return cd{dr, di};
}

// det(c Z) in the working precision R (c > 0 real: only its argument is used,
// to follow the branch of sqrt(det Z) between output bins).
// hz = c/2, gz = -gamma c, qz = c/(4 gamma).
template <typename R, int POT>
__device__ __forceinline__ Cx2<R> det_Z_scaled(const Traj<R, POT>& T, R hz, R gz, R qz) {
    R zr[3][3], zi[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            zr[i][j] = hz * (T.Y[3 + j][i] + T.X[j][i]);
            zi[i][j] = fma(gz, T.X[3 + j][i], qz * T.Y[j][i]);
        }
    auto mul = [](R ar, R ai, R br, R bi, R& cr, R& ci) {
        cr = fma(ar, br, -ai * bi);
        ci = fma(ar, bi, ai * br);
    };
    R m0r, m0i, m1r, m1i, m2r, m2i, tr, ti;
    mul(zr[1][1], zi[1][1], zr[2][2], zi[2][2], m0r, m0i);
    mul(zr[1][2], zi[1][2], zr[2][1], zi[2][1], tr, ti);
    m0r -= tr; m0i -= ti;
    mul(zr[1][0], zi[1][0], zr[2][2], zi[2][2], m1r, m1i);
    mul(zr[1][2], zi[1][2], zr[2][0], zi[2][0], tr, ti);
    m1r -= tr; m1i -= ti;
    mul(zr[1][0], zi[1][0], zr[2][1], zi[2][1], m2r, m2i);
    mul(zr[1][1], zi[1][1], zr[2][0], zi[2][0], tr, ti);
    m2r -= tr; m2i -= ti;
    R dr, di, ar, ai;
    mul(zr[0][0], zi[0][0], m0r, m0i, dr, di);
    mul(zr[0][1], zi[0][1], m1r, m1i, ar, ai);
    dr -= ar; di -= ai;
    mul(zr[0][2], zi[0][2], m2r, m2i, ar, ai);
    dr += ar; di += ai;
    return Cx2<R>{dr, di};
}

template <typename R, int POT>
__device__ __forceinline__ cd Traj<R, POT>::det64(double gam) const {
    return det_Z<R, POT>(*this, gam);
}
template <typename R, int POT>
__device__ __forceinline__ Cx2<R> Traj<R, POT>::detc(R hz, R gz, R qz) const {
    return det_Z_scaled<R, POT>(*this, hz, gz, qz);
}

// Continuous branch of C = sqrt(det Z): C = sgn * principal sqrt(det Z), and
// sgn flips whenever det Z crosses the negative real axis between two grid
// points (the cut of the principal root); this equals choosing, at every grid
// point, the root closest to the previous C while |d arg det Z| < pi per step.
template <typename R>
__device__ __forceinline__ void follow_branch(Cx2<R>& Dp, Cx2<R> D, R& sgn, unsigned& flags) {
    const R cr = Dp.re * D.im - Dp.im * D.re;
    if (Dp.im * D.im < R(0) && ((cr > R(0)) == (Dp.im > R(0)))) sgn = -sgn;
    if (Dp.re * D.re + Dp.im * D.im < R(0)) flags |= 4u;    // more than pi/2 in one step
    Dp = D;
}

// range reduction to [-pi, pi] for the fast float sincos
__device__ __forceinline__ float reduce_2pi(float x) {
    float k = rintf(x * 0.15915494309189535f);
    x = fmaf(-k, 6.28318548f, x);
    return fmaf(-k, -1.7484555e-07f, x);
}

template <typename R>
struct Cx {
    R re, im;
};
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return Cx<R>{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ void sc(float x, float* s, float* c) { __sincosf(reduce_2pi(x), s, c); }
__device__ __forceinline__ void sc(double x, double* s, double* c) { sincos(x, s, c); }

struct GtoR {
    int n, l;
};

// GTO constants in the working precision (float copies for the float path)
template <typename R>
__device__ __forceinline__ R gtv(const double* d, const float* f, int j) {
    if constexpr (std::is_same<R, float>::value) return f[j];
    else return (R)d[j];
}

// Recombination terms at one output bin: returns (-2 Re c_len, -2 Re c_vel).
// In three parts so that a caller can spread the GTO sum over several steps:
// the invariants p^2, q^2, p.q; the sum over GTO terms j0..j1-1 (in order); the
// closing products with C, e^{iS}, e^{-i Ip t} and the amplitude.
template <typename R>
struct GtoSums {
    Cx<R> s0, s1, s2, s3;
};
template <typename R, typename TT>
__device__ __forceinline__ void recomb_invariants(const TT& T, R& p2, R& q2, R& pq) {
    p2 = fma(T.p[0], T.p[0], fma(T.p[1], T.p[1], T.p[2] * T.p[2]));
    q2 = fma(T.q[0], T.q[0], fma(T.q[1], T.q[1], T.q[2] * T.q[2]));
    pq = fma(T.p[0], T.q[0], fma(T.p[1], T.q[1], T.p[2] * T.q[2]));
}
template <typename R>
__device__ __forceinline__ void gto_terms(const GtoTerms& gt, R p2, R q2, R pq, int j0, int j1, GtoSums<R>& a) {
    const R lim = std::is_same<R, float>::value ? R(-87) : R(-745);
    for (int j = j0; j < j1; ++j) {
        R xr = fma(gtv<R>(gt.kp, gt.kpf, j), p2, gtv<R>(gt.kq, gt.kqf, j) * q2);
        if (xr < lim) continue;                      // exp underflows: exact skip
        R xi = gtv<R>(gt.kx, gt.kxf, j) * pq;
        R e = ex(xr), sn, cs;
        sc(xi, &sn, &cs);
        Cx<R> z{e * cs, e * sn};
        const R w0 = gtv<R>(gt.w0, gt.w0f, j), w1 = gtv<R>(gt.w1, gt.w1f, j);
        a.s0.re = fma(w0, z.re, a.s0.re); a.s0.im = fma(w0, z.im, a.s0.im);
        a.s1.re = fma(w1, z.re, a.s1.re); a.s1.im = fma(w1, z.im, a.s1.im);
        if (gt.l == 1) {
            const R w2 = gtv<R>(gt.w2, gt.w2f, j), w3 = gtv<R>(gt.w3, gt.w3f, j);
            a.s2.re = fma(w2, z.re, a.s2.re); a.s2.im = fma(w2, z.im, a.s2.im);
            a.s3.re = fma(w3, z.re, a.s3.re); a.s3.im = fma(w3, z.im, a.s3.im);
        }
    }
}
template <typename R, typename TT>
__device__ __forceinline__ void contribution_final(const TT& T, const GtoTerms& gt, R gam, Cx<R> C, Cx<R> amp,
                                                   Cx<R> eIp, const GtoSums<R>& a, R& out_l, R& out_v) {
    const Cx<R> s0 = a.s0, s1 = a.s1, s2 = a.s2, s3 = a.s3;
    const R g = gam;
    const Cx<R> bz{R(2) * g * T.q[2], T.p[2]};          // 2 gamma q_z + i p_z
    const Cx<R> uz{T.p[2], R(-2) * g * T.q[2]};         // p_z - 2 i gamma q_z
    Cx<R> dl, dv;
    if (gt.l == 0) {
        dl = cmul(bz, s0);
        dv = cmul(uz, s1);
    } else {
        Cx<R> b2 = cmul(bz, bz), u2 = cmul(uz, uz);
        Cx<R> t0 = cmul(b2, s0);
        dl = Cx<R>{t0.re + s1.re, t0.im + s1.im};         // (b_z^2 + 2 beta) terms
        Cx<R> t2 = cmul(u2, s2);
        R ig = R(0.5) / g;
        Cx<R> sv{fma(ig, t2.re, s3.re), fma(ig, t2.im, s3.im)};
        dv = Cx<R>{-g * sv.im, g * sv.re};                 // i gamma * sv
    }
    // e^{i S} e^{-i Ip t_k} C amp
    R ss, cc;
    sc(T.S.reduced(), &ss, &cc);
    Cx<R> P = cmul(cmul(Cx<R>{cc, ss}, eIp), cmul(C, amp));
    Cx<R> cl = cmul(dl, P), cv = cmul(dv, P);
    if constexpr (std::is_same<R, float>::value) {
        out_l = -2.f * gt.nlf * cl.re;
        out_v = -2.f * gt.nvf * cv.re;
    } else {
        out_l = R(-2.0 * gt.nl) * cl.re;
        out_v = R(-2.0 * gt.nv) * cv.re;
    }
}
template <typename R, typename TT>
__device__ __forceinline__ void contribution(const TT& T, const GtoTerms& gt, R gam, Cx<R> C,
                                             Cx<R> amp, Cx<R> eIp, R& out_l, R& out_v) {
    R p2, q2, pq;
    recomb_invariants<R>(T, p2, q2, pq);
    GtoSums<R> a{};
    gto_terms<R>(gt, p2, q2, pq, 0, gt.n, a);
    contribution_final<R>(T, gt, gam, C, amp, eIp, a, out_l, out_v);
}

template <typename R>
__device__ __forceinline__ const R* etable(const FieldDev& f);
template <>
__device__ __forceinline__ const double* etable<double>(const FieldDev& f) { return f.E64; }
template <>
__device__ __forceinline__ const float* etable<float>(const FieldDev& f) { return f.E32; }
__device__ __forceinline__ const double* etable_df(const FieldDev& f) { return f.E64; }

// float view of an FP64 state for float recombination terms: coordinates rounded to
// float, the action reduced mod 2 pi in FP64 and then rounded
struct FloatState {
    float q[3], p[3];
    struct {
        float r;
        __device__ float reduced() const { return r; }
    } S;
    __device__ FloatState(double q0, double q1, double q2, double p0, double p1, double p2, double s)
        : q{(float)q0, (float)q1, (float)q2}, p{(float)p0, (float)p1, (float)p2}, S{(float)fmod(s, 2.0 * kPi)} {}
};

// float view of a double-float trajectory for the recombination terms
template <typename TT>
struct FloatView {
    float q[3], p[3];
    struct {
        float r;
        __device__ float reduced() const { return r; }
    } S;
    __device__ explicit FloatView(const TT& T) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            q[i] = (float)T.q[i];
            p[i] = (float)T.p[i];
        }
        S.r = T.S.reduced();
    }
};

template <typename R>
constexpr bool kEsc = std::is_same<R, float>::value;

// Mixed path: the FP64 det Z (formed exactly from the float blocks) scaled by
// an exact power of two, D = (re + i im) 2^(2e) with |re + i im| in [1/4, 4),
// so that the rest of the bin work runs in float.
struct ScaledDet {
    float re, im;
    int e;
};
__device__ __forceinline__ ScaledDet scale_det(cd D) {
    const double m = fmax(fabs(D.re), fabs(D.im));
    const int k = ((__double2hiint(m) >> 20) & 0x7ff) - 1023;   // binary exponent of m
    const int e = k >> 1;
    const double s = __hiloint2double((1023 - 2 * e) << 20, 0);  // 2^(-2e), exact
    return ScaledDet{(float)(D.re * s), (float)(D.im * s), e};
}
// the same scaling from a float pair (|det Z| <= D_t < 2^126 holds)
__device__ __forceinline__ ScaledDet scale_detf(float dr, float di) {
    const float m = fmaxf(fabsf(dr), fabsf(di));
    const int k = m > 0.f ? ((__float_as_int(m) >> 23) & 0xff) - 127 : 0;   // binary exponent of m
    const int e = k >> 1;
    const float s = __int_as_float((127 - 2 * e) << 23);                  // 2^(-2e), exact
    return ScaledDet{dr * s, di * s, e};
}
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// binary exponent of a finite non-zero float (0 for zero)
__device__ __forceinline__ int fexp(float m) { return m > 0.f ? ((__float_as_int(m) >> 23) & 0xff) - 127 : 0; }
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }   // 2^k, |k| <= 126

// Compensated dot product of four float products (error-free TwoProd by FMA
// and TwoSum, Ogita-Rump-Oishi "Dot2"): as accurate as the sum evaluated in
// twice the working precision, then rounded.
__device__ __forceinline__ float dot2_4(float a0, float b0, float a1, float b1, float a2, float b2, float a3, float b3) {
    float s = a0 * b0, c = fmaf(a0, b0, -s);
    const float a[3] = {a1, a2, a3}, b[3] = {b1, b2, b3};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float p = a[k] * b[k], ep = fmaf(a[k], b[k], -p);
        float t, et;
        two_sum_f(s, p, t, et);
        s = t;
        c += ep + et;
    }
    return s + c;
}

// det Z of the planar form from float entries, without FP64: the in-plane
// block is scaled by a power of two (exact), its determinant taken with
// compensated products (no cancellation loss), multiplied by Z_yy, and
// returned as a scaled pair, det Z = (re + i im) 2^(2e).  Non-finite entries
// give a non-finite result.
__device__ __forceinline__ ScaledDet det_planar_comp(const float zr[2][2], const float zi[2][2], float yr, float yi) {
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) m = fmaxf(m, fmaxf(fabsf(zr[i][j]), fabsf(zi[i][j])));
    const float my = fmaxf(fabsf(yr), fabsf(yi));
    if (!(m < 1.0e38f) || !(my < 1.0e38f)) return ScaledDet{__int_as_float(0x7fc00000), 0.f, 0};
    const int k1 = fexp(m), k2 = fexp(my);
    const float s1 = pow2f(-k1), s2 = pow2f(-k2);
    float r[2][2], q[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) { r[i][j] = zr[i][j] * s1; q[i][j] = zi[i][j] * s1; }
    // A = z00 z11 - z01 z10 (complex), entries scaled by 2^-k1
    const float ar = dot2_4(r[0][0], r[1][1], -q[0][0], q[1][1], -r[0][1], r[1][0], q[0][1], q[1][0]);
    const float ai = dot2_4(r[0][0], q[1][1], q[0][0], r[1][1], -r[0][1], q[1][0], -q[0][1], r[1][0]);
    const float ur = yr * s2, ui = yi * s2;
    const float pr = fmaf(ar, ur, -ai * ui), pi = fmaf(ar, ui, ai * ur);
    // det Z = (pr + i pi) 2^(2 k1 + k2); renormalise to the 2^(2e) form
    const float mp = fmaxf(fabsf(pr), fabsf(pi));
    if (!(mp >= 0x1p-100f)) return ScaledDet{0.f, 0.f, 0};   // zero (Z is invertible: not reached)
    const int kp = fexp(mp);
    const int E = 2 * k1 + k2 + kp;
    const int e = E >> 1;
    const float sc = pow2f((E - 2 * e) - kp);
    return ScaledDet{pr * sc, pi * sc, e};
}

// det Z of a float trajectory at an output bin, scaled.  Planar form: Z's
// entries formed in float (as det64 forms them) and the determinant taken with
// compensated float products; 3D form: FP64 determinant of the float blocks.
template <int POT>
__device__ __forceinline__ ScaledDet det_scaled_f(const TrajP<float, POT>& T, double gam, float g, float q) {
    (void)gam;
    float zr[2][2], zi[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            zr[i][j] = 0.5f * (T.Y[2 + j][i] + T.X[j][i]);
            zi[i][j] = fmaf(-g, T.X[2 + j][i], q * T.Y[j][i]);
        }
    return det_planar_comp(zr, zi, 0.5f * (T.bp + T.aq), fmaf(-g, T.bq, q * T.ap));
}
template <int POT>
__device__ __forceinline__ ScaledDet det_scaled_f(const Traj<float, POT>& T, double gam, float g, float q) {
    (void)g;
    (void)q;
    const cd D = T.det64(gam);
    return scale_detf((float)D.re, (float)D.im);
}

// principal sqrt of the scaled determinant, times 2^e
__device__ __forceinline__ Cx2<float> sqrt_scaled(const ScaledDet& d) {
    const float r = sqrtf(fmaf(d.re, d.re, d.im * d.im));
    float cr, ci;
    if (d.re >= 0.f) {
        const float t = sqrtf(0.5f * (r + d.re));
        cr = t;
        ci = d.im / (2.f * t);
    } else {
        const float t = sqrtf(0.5f * (r - d.re));
        cr = fabsf(d.im) / (2.f * t);
        ci = copysignf(t, d.im);
    }
    const float sc = __int_as_float((127 + d.e) << 23);          // 2^e, exact
    return Cx2<float>{cr * sc, ci * sc};
}

// Escalation test of the mixed path at an output bin (d = scaled FP64 det Z,
// Dp = float per-step det(zc Z), tau = t - t0), all in float:
//  * growth: |det Z| > esc_ratio (1 + gamma^2 tau^2)^{3/2}, i.e. the prefactor
//    grew beyond free-particle spreading by more than esc_ratio (sensitive,
//    chaotic dynamics where float rounding is amplified);
//  * the float per-step determinant disagrees with the FP64 one by > 10%
//    (its branch tracking is no longer reliable);
//  * a branch-guard event (arg det Z moved by more than pi/2 in one step).
__device__ __forceinline__ bool esc_needed(const ScaledDet& d, Cx2<float> Dp, float zc, unsigned flags, float tau,
                                           float gam, float log2_esc) {
    if (flags & 4u) return true;
    const float a2 = fmaf(d.re, d.re, d.im * d.im);
    const float x = fmaf(gam * gam * tau, tau, 1.0f);
    if (__log2f(a2) + 4.0f * (float)d.e > 2.0f * log2_esc + 3.0f * __log2f(x)) return true;
    const float s = __int_as_float((127 - 2 * d.e) << 23) / (zc * zc * zc);   // 2^(-2e) / zc^3
    const float er = fmaf(Dp.re, s, -d.re), ei = fmaf(Dp.im, s, -d.im);
    return fmaf(er, er, ei * ei) > 0.01f * a2;
}

// The second half of the escalation decision at an output bin, taken only once the
// tests of esc_needed hold at the smaller of the two growth ratios (log2 esc_l2_lo):
// with G = log2 |det Z|^2 (from d) and l_amp = log2(|amp|^2 / max|amp|^2) the trajectory's
// weight w = |amp|^2 |C|^2 / max|amp|^2 has log2 w = G/2 + l_amp; escalate only while
// w >= esc_floor^2, at growth ratio esc_ratio_big where w >= esc_big^2 and esc_ratio
// otherwise (each test of esc_needed repeated at that ratio when it is not the
// smaller one).  The log2 thresholds are host-made kernel parameters.
__device__ __forceinline__ bool esc_weighed(const ScaledDet& d, Cx2<float> Dp, float zc, unsigned flags, float tau,
                                         float gam, float l_amp, const TrajArgs& a) {
    const float G = __log2f(fmaf(d.re, d.re, d.im * d.im)) + 4.0f * (float)d.e;
    const float lw = fmaf(0.5f, G, l_amp);
    if (!(lw >= a.esc_l2_floor)) return false;
    const float l = lw >= a.esc_l2_bigw ? a.esc_l2_big : a.esc_l2;
    return l == a.esc_l2_lo || esc_needed(d, Dp, zc, flags, tau, gam, l);
}

// One block of trajectories: block `bid` of the births (or of an escalation list).
template <typename R, int POT, bool PLANAR>
__device__ __forceinline__ void traj_block(const FieldDev& f, const TargetDev& tg, const GtoTerms& gt,
                                           const TrajArgs& a, const int64_t bid, unsigned char* smem,
                                           long long& s_nmin) {
    using TT = typename std::conditional<PLANAR, TrajP<R, POT>, Traj<R, POT>>::type;
    constexpr bool kDF = std::is_same<R, dfloat>::value;
    using RC = typename std::conditional<kDF, float, R>::type;   // precision of the recombination terms
    const int CH = a.chunk;
    const int n_out = (int)f.n_out;
    const int nbw = CH / n_out;                 // bins per window
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    R* sE = reinterpret_cast<R*>(smem);
    const int e_len = 2 * CH + 2;
    double* sB = reinterpret_cast<double*>(smem + ((e_len * sizeof(R) + 15) / 16) * 16);
    using RCp = typename std::conditional<std::is_same<R, dfloat>::value, float, R>::type;
    Cx<RCp>* sPh = reinterpret_cast<Cx<RCp>*>(sB + (size_t)nw * 2 * nbw);

    const bool dipole = a.mode == 1;
    // list position j -> birth index i (identity unless an escalation list is given)
    const int64_t n_list = a.count ? (int64_t)*a.count : a.n;
    if (bid * blockDim.x >= n_list) return;     // whole block past the list
    const int64_t j = bid * blockDim.x + threadIdx.x;
    const bool have = j < n_list;
    const int64_t i = have ? (a.idx ? (int64_t)a.idx[j] : j) : 0;
    const int64_t k_min = (have && a.k_from) ? (int64_t)a.k_from[j] : 0;   // first bin to contribute
    const bool escalate = kEsc<R> && a.esc_bin != nullptr && a.esc_ratio > 0.0;
    int64_t n0 = have ? (int64_t)a.n0[i] : 0;
    double amp_r = have ? a.amp_re[i] : 0.0, amp_i = have ? a.amp_im[i] : 0.0;
    Cx<RC> amp{(RC)amp_r, (RC)amp_i};
    // dipole mode integrates births whose amplitude is non-zero in the working
    // precision; endpoint mode integrates every birth in range
    bool alive = have && n0 <= a.n_last && n0 >= 0 && (!dipole || amp.re != RC(0) || amp.im != RC(0));
    unsigned flags = (have && !alive) ? 8u : 0u;

    PotConst<R> pc;
    if constexpr (std::is_same<R, float>::value) {
        // the float copies made on the host, read from the kernel parameters: under
        // register pressure the compiler re-reads them there instead of converting
        // the FP64 parameters again on the FP64 units inside the step loop
        pc.a2 = tg.a2_32;
        pc.Zc = tg.pot_param32[0]; pc.a1 = tg.pot_param32[1]; pc.a2t = tg.pot_param32[2];
        pc.a3 = tg.pot_param32[3]; pc.a4 = tg.pot_param32[4]; pc.a5 = tg.pot_param32[5];
        pc.a6 = tg.pot_param32[6];
    } else {
        if (POT == POT_SOFTCORE) pc.a2 = (R)(tg.pot_param[0] * tg.pot_param[0]);
        if (POT == POT_HARMONIC) pc.a2 = (R)(tg.pot_param[0] * tg.pot_param[0]);
        pc.Zc = (R)tg.pot_param[0]; pc.a1 = (R)tg.pot_param[1]; pc.a2t = (R)tg.pot_param[2];
        pc.a3 = (R)tg.pot_param[3]; pc.a4 = (R)tg.pot_param[4]; pc.a5 = (R)tg.pot_param[5];
        pc.a6 = (R)tg.pot_param[6];
    }

    TT T;
    {
        R qx = (have && a.qx) ? (R)a.qx[i] : R(0);
        R qy = (have && a.qy) ? (R)a.qy[i] : R(0);
        R qz = have ? (R)a.qz[i] : R(0);
        R px = have ? (R)a.px[i] : R(0), py = have ? (R)a.py[i] : R(0), pz = have ? (R)a.pz[i] : R(0);
        T.init(qx, qy, qz, px, py, pz);
    }
    constexpr bool kF32 = std::is_same<R, float>::value;
    constexpr bool kScaled = !std::is_same<R, double>::value;   // float exponent range: rescale det
    cd Cacc{1.0, 0.0};                  // C at the last accepted evaluation
    Cx2<R> Dp{R(1), R(0)};              // det(c Z) at the current grid point (M = I at birth)
    R sgn = R(1);                       // branch: C = sgn * principal sqrt(det Z)
    R zc = R(1);                        // scale c of the per-step determinant
    const R rg = [&] {
        if constexpr (kF32) return a.gamma32;
        else return (R)a.gamma;
    }();

    const float log2_dt2 = (float)(2.0 * log2(a.d_t));   // removal: log2 |det Z|^2 > log2 D_t^2
    // escalation weight of this trajectory: log2(|amp|^2 / max |amp|^2) (0 without a maximum)
    float l_amp = 0.f;
    if (escalate && a.esc_amax2 != nullptr) {
        const double m2 = *a.esc_amax2, x2 = amp_r * amp_r + amp_i * amp_i;
        l_amp = (m2 > 0.0 && x2 > 0.0) ? (float)(log2(x2) - log2(m2)) : -1e30f;
    }
    const float dtf = f.dt32;
    const float gamf = a.gamma32;
    const float qgf = a.qg32;   // 1/(4 gamma) for Z's entries in float
    const int64_t k_cnt = k_min * n_out;        // steps before the escalation bin were counted in the float pass
    // partial-wave filter: class at the latest entry into the near-core sphere (-1: none yet)
    using RP = typename std::conditional<std::is_same<R, double>::value, double, float>::type;
    const bool pw = dipole && a.pw_mask != 0;
    const RP pw_r2 = (RP)(a.pw_radius * a.pw_radius);
    int pw_cls = -1;
    bool pw_in = false;
    unsigned long long all_steps = 0;
    unsigned long long steps = 0;

    // segmented float pass: a trajectory born before this segment resumes from its
    // saved state (kernel scalars first, then the members of T)
    const bool seg = kF32 && a.state != nullptr;
    const int64_t n_end = (seg && a.seg_hi < a.n_last) ? a.seg_hi : a.n_last;   // last grid point of this launch
    unsigned flags_in = 0;
    if constexpr (kF32) {
        if (seg && have && a.seg_lo > 0 && n0 < a.seg_lo) {
            const uint32_t* st = a.state;
            const size_t sn = (size_t)a.n;
            const uint32_t w0 = st[i];
            alive = (w0 & 0x80000000u) != 0;
            flags = w0 & 0xffu;
            pw_in = (w0 & 0x100u) != 0;
            pw_cls = (int)((w0 >> 9) & 7u) - 1;
            if (alive) {
                Dp.re = __uint_as_float(st[sn + i]);
                Dp.im = __uint_as_float(st[2 * sn + i]);
                sgn = __uint_as_float(st[3 * sn + i]);
                zc = __uint_as_float(st[4 * sn + i]);
                size_t k = 5;
                T.visit([&](auto& v) {
                    const uint32_t u = st[k * sn + i];
                    ++k;
                    if constexpr (std::is_same<std::remove_reference_t<decltype(v)>, float>::value) v = __uint_as_float(u);
                    else v = (int)u;
                });
            }
            flags_in = flags;
        }
        // a birth after this segment is counted by the segment that holds it
        if (seg && have && n0 > n_end) flags_in = flags;
    }

    if (threadIdx.x == 0) s_nmin = LLONG_MAX;
    __syncthreads();
    if (alive) atomicMin(&s_nmin, (long long)n0);
    __syncthreads();
    const int64_t n_first = (seg && s_nmin != LLONG_MAX && s_nmin < a.seg_lo) ? a.seg_lo : s_nmin;
    const int64_t n_last = n_end;
    const auto* table = [&] {
        if constexpr (std::is_same<R, dfloat>::value) return etable_df(f);
        else return etable<R>(f);
    }();
    // step constants: host-made for float and FP64, derived here for double-float
    const StepK<R> hk = [&] {
        if constexpr (kF32) return f.k32;
        else if constexpr (std::is_same<R, double>::value) return f.k64;
        else return step_constants_dev<R>((R)f.dt);
    }();

    if (n_first != LLONG_MAX) {
        for (int64_t ws = (n_first / CH) * CH; ws <= n_last; ws += CH) {
            __syncthreads();
            for (int u = threadIdx.x; u < e_len; u += blockDim.x) {
                int64_t j = 2 * ws + u;
                sE[u] = (j < f.table_len) ? table[j] : R(0);
            }
            if (dipole) {
                for (int u = threadIdx.x; u < nw * 2 * nbw; u += blockDim.x) sB[u] = 0.0;
                for (int b = threadIdx.x; b < nbw; b += blockDim.x) {
                    int64_t k = ws / n_out + b;
                    double tk = f.t_start + (double)(k * n_out) * f.dt;
                    double ph = fmod(tg.ip * tk, 2.0 * kPi);
                    double sn, cs;
                    sincos(ph, &sn, &cs);
                    sPh[b] = Cx<RC>{(RC)cs, (RC)(-sn)};    // e^{-i Ip t_k}
                }
            }
            __syncthreads();
            const int64_t n_lo = ws > n_first ? ws : n_first;
            const int64_t n_hi = (ws + CH - 1 < n_last) ? ws + CH - 1 : n_last;
            // partial waves (Sec. III.A-B): label by L = |q x p| at each entry into r < R
            auto pw_update = [&]() {
                const RP qx = (RP)T.q[0], qy = (RP)T.q[1], qz = (RP)T.q[2];
                const bool in = qx * qx + qy * qy + qz * qz < pw_r2;
                if (in && !pw_in) {
                    const RP px = (RP)T.p[0], py = (RP)T.p[1], pz = (RP)T.p[2];
                    const RP lx = qy * pz - qz * py, ly = qz * px - qx * pz, lz = qx * py - qy * px;
                    const RP L2 = lx * lx + ly * ly + lz * lz;
                    pw_cls = L2 < RP(0.25) ? 0 : (L2 < RP(2.25) ? 1 : (L2 < RP(6.25) ? 2 : 3));
                }
                pw_in = in;
            };
            // birth grid point relative to the window (clamped to int range)
            const int un0 = (int)(n0 - ws < -1 ? -1 : (n0 - ws > CH + 1 ? CH + 1 : n0 - ws));
            // windows start on multiples of the chunk, itself a multiple of n_out, so grid
            // indices are reduced modulo n_out by their 32-bit offset in the window
            int rem = (int)(n_lo - ws) % n_out;       // steps past the last output index
            int bw = ((int)(n_lo - ws) + n_out - 1) / n_out;   // window bin of the next output index
            // grid points in groups: the work of a group's first point (labels, output
            // bin), then the steps up to the next output index; removal and escalation
            // happen only at output indices, so `alive` is constant over a group's steps
            for (int64_t n = n_lo; n <= n_hi;) {
                const bool on_bin = rem == 0;
                const bool live = alive && n >= n0;
                if (pw && live) pw_update();
                const bool pw_ok = !pw || (pw_cls >= 0 && ((a.pw_mask >> pw_cls) & 1));
                if (on_bin || (!dipole && n == n_last)) {
                    RC cl = RC(0), cv = RC(0);
                    if (live) {
                        const bool ok = T.finite_state();
                        if constexpr (kF32) {
                            // accurate determinant from the float blocks (planar: compensated
                            // float; 3D: FP64), scaled by a power of two; the rest of the bin
                            // work runs in float
                            const ScaledDet sd = det_scaled_f(T, a.gamma, gamf, qgf);
                            const float a2 = fmaf(sd.re, sd.re, sd.im * sd.im);
                            const bool fin = ::isfinite(a2);
                            if (!ok || !fin || __log2f(a2) + 4.0f * (float)sd.e > log2_dt2) {
                                alive = false;
                                flags |= 1u;
                                if (!ok || !fin) flags |= 2u;
                            } else if (escalate &&
                                       esc_needed(sd, Cx2<float>{(float)Dp.re, (float)Dp.im}, (float)zc, flags,
                                                  (float)(int)(n - n0) * dtf, gamf, a.esc_l2_lo) &&
                                       esc_weighed(sd, Cx2<float>{(float)Dp.re, (float)Dp.im}, (float)zc, flags,
                                                   (float)(int)(n - n0) * dtf, gamf, l_amp, a)) {
                                // the float trajectory no longer follows the FP64 one closely
                                // enough: stop here, the high-precision pass redoes it from this bin on
                                alive = false;
                                flags |= 16u;
                                a.esc_bin[i] = (int32_t)(n / n_out);
                            } else {
                                Cx2<float> c = sqrt_scaled(sd);
                                // branch sign; flip also if the float per-step and the FP64
                                // determinants lie on opposite sides of the cut
                                bool neg = sgn < R(0);
                                if (sd.re < 0.f && sd.im * (float)Dp.im < 0.f) neg = !neg;
                                if (neg) c = Cx2<float>{-c.re, -c.im};
                                if (!dipole) Cacc = cd{(double)c.re, (double)c.im};
                                // rescale the per-step float determinant to magnitude ~1
                                const float m = fabsf((float)Dp.re) + fabsf((float)Dp.im);
                                if (m > 0.f && ::isfinite(m)) zc = zc * exp2f(-__log2f(m) * (1.0f / 3.0f));
                                if (dipole && on_bin && n >= k_cnt && pw_ok)
                                    contribution<float>(T, gt, gamf, Cx<float>{c.re, c.im}, amp, sPh[bw], cl, cv);
                            }
                        } else {
                            // FP64 / double-float: the determinant of this grid point
                            const cd D = kScaled ? T.det64(a.gamma) : cd{(double)Dp.re, (double)Dp.im};
                            const double m2 = D.re * D.re + D.im * D.im;
                            if (!ok || !(m2 <= a.d_t * a.d_t)) {
                                alive = false;
                                flags |= 1u;
                                if (!ok || !isfinite(m2)) flags |= 2u;
                            } else {
                                cd C = c_sqrt(D);
                                bool neg = sgn < R(0);
                                if constexpr (kDF) {
                                    if (D.re < 0.0 && D.im * (double)Dp.im < 0.0) neg = !neg;
                                    const float m = fabsf(Dp.re.hi) + fabsf(Dp.im.hi);
                                    if (m > 0.f && ::isfinite(m)) zc = zc * R(exp2f(-__log2f(m) * (1.0f / 3.0f)));
                                }
                                if (neg) C = -C;
                                Cacc = C;
                                if (dipole && on_bin && n >= k_cnt && pw_ok) {
                                    if constexpr (kDF)
                                        contribution<float>(FloatView<TT>(T), gt, gamf,
                                                            Cx<float>{(float)C.re, (float)C.im}, amp,
                                                            sPh[bw], cl, cv);
                                    else if (a.float_bins) {
                                        float fl, fv;
                                        contribution<float>(
                                            FloatState((double)T.q[0], (double)T.q[1], (double)T.q[2], (double)T.p[0],
                                                       (double)T.p[1], (double)T.p[2], (double)T.S.value()),
                                            gt, gamf, Cx<float>{(float)C.re, (float)C.im},
                                            Cx<float>{(float)amp.re, (float)amp.im},
                                            Cx<float>{(float)sPh[bw].re, (float)sPh[bw].im}, fl, fv);
                                        cl = (RC)fl;
                                        cv = (RC)fv;
                                    } else
                                        contribution<R>(T, gt, (R)a.gamma, Cx<R>{(R)C.re, (R)C.im}, amp,
                                                        sPh[bw], cl, cv);
                                }
                            }
                        }
                    }
                    if (dipole && on_bin) {
                        if (__any_sync(0xffffffffu, cl != RC(0) || cv != RC(0))) {
                            double sl, sv;
                            if constexpr (std::is_same<RC, float>::value) {
                                // compensated float reduction: pairwise TwoSum, errors carried
                                float el = 0.f, ev = 0.f;
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) {
                                    const float tl = __shfl_xor_sync(0xffffffffu, cl, o);
                                    const float tel = __shfl_xor_sync(0xffffffffu, el, o);
                                    const float tv = __shfl_xor_sync(0xffffffffu, cv, o);
                                    const float tev = __shfl_xor_sync(0xffffffffu, ev, o);
                                    float s1, e1, s2, e2;
                                    two_sum_f(cl, tl, s1, e1);
                                    two_sum_f(cv, tv, s2, e2);
                                    cl = s1;
                                    cv = s2;
                                    el = el + tel + e1;
                                    ev = ev + tev + e2;
                                }
                                sl = (double)cl + (double)el;
                                sv = (double)cv + (double)ev;
                            } else {
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) {
                                    cl += __shfl_xor_sync(0xffffffffu, cl, o);
                                    cv += __shfl_xor_sync(0xffffffffu, cv, o);
                                }
                                sl = (double)cl;
                                sv = (double)cv;
                            }
                            if (lane == 0) {
                                sB[(warp * 2) * nbw + bw] = sl;
                                sB[(warp * 2 + 1) * nbw + bw] = sv;
                            }
                        }
                    }
                }
                // steps n -> n + 1 up to the next output index (or the window's end)
                int64_t n_stop = (n + (n_out - rem) < n_hi + 1) ? n + (n_out - rem) : n_hi + 1;
                if (!dipole && n < n_last && n_last < n_stop) n_stop = n_last;   // the end point is evaluated
                const int u_start = (int)(n - ws);
                const int u_end = (int)((n_stop < a.n_last ? n_stop : a.n_last) - ws);
                if (alive) {
                    const int u_first = u_start > un0 ? u_start : un0;
                    if (u_end > u_first) {
                        const unsigned long long m = (unsigned long long)(u_end - u_first);
                        all_steps += m;
                        if (n >= k_cnt) steps += m;
                    }
                    // scale factors of the per-step det(zc Z): zc is constant over a group
                    const R zh = R(0.5) * zc, zg = -rg * zc, zq = zc / (R(4) * rg);
                    // the steps from the group's start or the birth, whichever is later
                    const int u_lo = u_start > un0 ? u_start : un0;
                    if (pw && u_lo == un0 && un0 != u_start && u_lo < u_end) pw_update();   // birth inside a group
                    const int u_inner = (int)(n_stop - ws);
                    int k5 = (u_lo - u_start) % 5;   // steps since the group's start, mod 5
                    for (int u = u_lo; u < u_end; ++u) {
                        T.step(sE[2 * u], sE[2 * u + 1], sE[2 * u + 2], hk, pc);
                        // the float pass follows the branch every fifth step (and at the
                        // group's last step); a turn of det Z by more than pi/2 between two
                        // evaluations flags the trajectory, which then leaves float at the bin;
                        // the planar float action is folded at the same points
                        if (!kF32 || k5 == 4 || u + 1 == u_end) {
                            const Cx2<R> D = T.detc(zh, zg, zq);
                            follow_branch<R>(Dp, D, sgn, flags);
                            if constexpr (kF32 && PLANAR) T.settle();
                        }
                        k5 = k5 == 4 ? 0 : k5 + 1;
                        if (pw && u + 1 < u_inner) pw_update();   // labels at the inner points
                    }
                }
                if (on_bin) ++bw;
                // the next group starts on an output index unless it is the end point
                rem = (n_stop == n + (n_out - rem) || n_stop == n_hi + 1) ? 0 : (int)(n_stop - ws) % n_out;
                n = n_stop;
            }
            __syncthreads();
            if (dipole) {
                for (int b = threadIdx.x; b < nbw; b += blockDim.x) {
                    int64_t k = ws / n_out + b;
                    if (k >= f.n_bins) continue;
                    double sl = 0.0, sv = 0.0;
                    for (int w = 0; w < nw; ++w) {
                        sl += sB[(w * 2) * nbw + b];
                        sv += sB[(w * 2 + 1) * nbw + b];
                    }
                    if (a.part) {
                        a.part[((size_t)bid * 2) * f.n_bins + k] = sl;
                        a.part[((size_t)bid * 2 + 1) * f.n_bins + k] = sv;
                    } else if (sl != 0.0 || sv != 0.0) {
                        atomicAdd(&a.d_len[k], sl);
                        atomicAdd(&a.d_vel[k], sv);
                    }
                }
            }
        }
    }

    if constexpr (kF32) {
        // segmented pass: save the state at seg_hi + 1 for the next segment
        if (seg && have && n0 <= n_end && a.seg_hi < a.n_last) {
            uint32_t* st = a.state;
            const size_t sn = (size_t)a.n;
            st[i] = (alive ? 0x80000000u : 0u) | (flags & 0xffu) | (pw_in ? 0x100u : 0u) |
                    ((unsigned)(pw_cls + 1) << 9);
            if (alive) {
                st[sn + i] = __float_as_uint(Dp.re);
                st[2 * sn + i] = __float_as_uint(Dp.im);
                st[3 * sn + i] = __float_as_uint(sgn);
                st[4 * sn + i] = __float_as_uint(zc);
                size_t k = 5;
                T.visit([&](auto& v) {
                    uint32_t u;
                    if constexpr (std::is_same<std::remove_reference_t<decltype(v)>, float>::value) u = __float_as_uint(v);
                    else u = (uint32_t)v;
                    st[k * sn + i] = u;
                    ++k;
                });
            }
        }
    }

    if constexpr (!PLANAR) {
    if (!dipole && have) {
        const int64_t n = a.n;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.st_out[(size_t)c * n + i] = (double)T.q[c];
            a.st_out[(size_t)(3 + c) * n + i] = (double)T.p[c];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a.st_out[(size_t)(6 + 3 * r + c) * n + i] = (double)T.X[c][r];        // Mqq
                a.st_out[(size_t)(15 + 3 * r + c) * n + i] = (double)T.X[3 + c][r];   // Mqp
                a.st_out[(size_t)(24 + 3 * r + c) * n + i] = (double)T.Y[c][r];       // Mpq
                a.st_out[(size_t)(33 + 3 * r + c) * n + i] = (double)T.Y[3 + c][r];   // Mpp
            }
        a.st_out[(size_t)42 * n + i] = T.S.value();
        a.c_re[i] = Cacc.re;
        a.c_im[i] = Cacc.im;
        a.flags[i] = (uint8_t)flags;
    }
    }
    if (a.stats) {
        const unsigned fn = flags & ~flags_in;  // events of this launch (a resumed trajectory brings its earlier flags)
        unsigned rem = __reduce_add_sync(0xffffffffu, (fn & 1u) ? 1u : 0u);
        unsigned nf = __reduce_add_sync(0xffffffffu, (fn & 2u) ? 1u : 0u);
        unsigned bg = __reduce_add_sync(0xffffffffu, (fn & 4u) ? 1u : 0u);
        unsigned sk = __reduce_add_sync(0xffffffffu, (fn & 8u) ? 1u : 0u);
        unsigned es = __reduce_add_sync(0xffffffffu, (fn & 16u) ? 1u : 0u);
        unsigned long long st = steps, ast = all_steps;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st += __shfl_xor_sync(0xffffffffu, st, o);
            ast += __shfl_xor_sync(0xffffffffu, ast, o);
        }
        if (lane == 0) {
            if (rem) atomicAdd(&a.stats->removed, (unsigned long long)rem);
            if (nf) atomicAdd(&a.stats->nonfinite, (unsigned long long)nf);
            if (bg) atomicAdd(&a.stats->branch_guard, (unsigned long long)bg);
            if (sk) atomicAdd(&a.stats->skipped, (unsigned long long)sk);
            if (es) atomicAdd(&a.stats->escalated, (unsigned long long)es);
            if (a.idx && ast) atomicAdd(&a.stats->esc_steps, ast);
            if (a.idx && ast > st) atomicAdd(&a.stats->esc_steps_pre, ast - st);
            if (st) atomicAdd(&a.stats->traj_steps, st);
        }
    }
}

}  // namespace
}  // namespace sfhk
