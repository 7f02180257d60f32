// Device helpers of the SFHK library: complex double arithmetic, the
// Philox4x64-10 counter-based generator, and the analytic laser field for
// complex times.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sfhk_internal.cuh"

namespace sfhk {

struct cd {
    double re, im;
};
__device__ __forceinline__ cd mk(double r, double i) { return cd{r, i}; }
__device__ __forceinline__ cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd operator-(cd a) { return cd{-a.re, -a.im}; }
__device__ __forceinline__ cd operator*(cd a, cd b) {
    return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
    double d = b.re * b.re + b.im * b.im;
    return cd{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ cd c_exp(cd z) {
    double s, c;
    sincos(z.im, &s, &c);
    double e = exp(z.re);
    return cd{e * c, e * s};
}
// sin(x + i y) = sin x cosh y + i cos x sinh y
__device__ __forceinline__ cd c_sin(cd z) {
    double s, c;
    sincos(z.re, &s, &c);
    return cd{s * cosh(z.im), c * sinh(z.im)};
}
// cos(x + i y) = cos x cosh y - i sin x sinh y
__device__ __forceinline__ cd c_cos(cd z) {
    double s, c;
    sincos(z.re, &s, &c);
    return cd{c * cosh(z.im), -s * sinh(z.im)};
}
// principal square root
__device__ __forceinline__ cd c_sqrt(cd z) {
    double r = hypot(z.re, z.im);
    if (r == 0.0) return cd{0.0, 0.0};
    if (z.re >= 0.0) {
        double t = sqrt(0.5 * (r + z.re));
        return cd{t, z.im / (2.0 * t)};
    }
    double t = sqrt(0.5 * (r - z.re));
    return cd{fabs(z.im) / (2.0 * t), copysign(t, z.im)};
}

// ---- Philox4x64-10 (Salmon et al., SC'11) ----------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
        uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

// ---- analytic field on complex time ----------------------------------------
// A(t) = sum_j a_j sin(w_j t + cep), E = -dA/dt, F = int_0^t A, G = int_0^t A^2.
__device__ __forceinline__ cd field_A(const FieldDev& f, cd t) {
    cd s = mk(0, 0);
    for (int j = 0; j < f.n_modes; ++j) s = s + f.a[j] * c_sin(mk(f.w[j] * t.re + f.cep, f.w[j] * t.im));
    return s;
}
__device__ __forceinline__ cd field_E(const FieldDev& f, cd t) {
    cd s = mk(0, 0);
    for (int j = 0; j < f.n_modes; ++j)
        s = s + (-f.a[j] * f.w[j]) * c_cos(mk(f.w[j] * t.re + f.cep, f.w[j] * t.im));
    return s;
}
// int_0^t cos(w s + th) ds for complex t
__device__ __forceinline__ cd int_cos(double w, double th, cd t) {
    if (fabs(w) < 1e-14) return cos(th) * t;
    cd v = c_sin(mk(w * t.re + th, w * t.im));
    return (1.0 / w) * (v - mk(sin(th), 0.0));
}
__device__ __forceinline__ cd field_F(const FieldDev& f, cd t) {
    cd s = mk(0, 0);
    for (int j = 0; j < f.n_modes; ++j) {
        double w = f.w[j];
        if (fabs(w) < 1e-14) {
            s = s + (f.a[j] * sin(f.cep)) * t;
        } else {
            cd v = c_cos(mk(w * t.re + f.cep, w * t.im));
            s = s + (f.a[j] / w) * (mk(cos(f.cep), 0.0) - v);
        }
    }
    return s;
}
__device__ __forceinline__ cd field_G(const FieldDev& f, cd t) {
    cd s = mk(0, 0);
    for (int j = 0; j < f.n_modes; ++j)
        for (int k = 0; k < f.n_modes; ++k) {
            double c = 0.5 * f.a[j] * f.a[k];
            s = s + c * (int_cos(f.w[j] - f.w[k], 0.0, t) - int_cos(f.w[j] + f.w[k], 2.0 * f.cep, t));
        }
    return s;
}

// The same four functions at one time from the sines and cosines of the mode phases
// a_j = w_j t + cep, each computed once: A and E are sums over them, F a sum over
// the cosines, and G's terms sin((w_j -+ w_k) t + ...) = sin(a_j -+ a_k) follow by
// the angle-sum identities (no further transcendental calls).  At a real time the
// hyperbolic factors (1 and 0) are left out.
struct FieldAt {
    cd A, E, F, G;
};
__device__ __forceinline__ FieldAt field_at(const FieldDev& f, cd t) {
    cd s[3], c[3];
    const int nm = f.n_modes < 3 ? f.n_modes : 3;
    for (int j = 0; j < nm; ++j) {
        double sn, cs;
        sincos(f.w[j] * t.re + f.cep, &sn, &cs);
        if (t.im == 0.0) {
            s[j] = mk(sn, 0.0);
            c[j] = mk(cs, 0.0);
        } else {
            const double y = f.w[j] * t.im, ch = cosh(y), sh = sinh(y);
            s[j] = mk(sn * ch, cs * sh);     // sin(x + i y)
            c[j] = mk(cs * ch, -sn * sh);    // cos(x + i y)
        }
    }
    double s_cep, c_cep, s_2cep, c_2cep;
    sincos(f.cep, &s_cep, &c_cep);
    sincos(2.0 * f.cep, &s_2cep, &c_2cep);
    FieldAt r{mk(0, 0), mk(0, 0), mk(0, 0), mk(0, 0)};
    for (int j = 0; j < nm; ++j) {
        const double a = f.a[j], w = f.w[j];
        r.A = r.A + a * s[j];
        r.E = r.E + (-a * w) * c[j];
        if (fabs(w) < 1e-14) r.F = r.F + (a * s_cep) * t;
        else r.F = r.F + (a / w) * (mk(c_cep, 0.0) - c[j]);
    }
    for (int j = 0; j < nm; ++j)
        for (int k = 0; k < nm; ++k) {
            const double cf = 0.5 * f.a[j] * f.a[k];
            const cd sc = s[j] * c[k], cs = c[j] * s[k];
            const double wm = f.w[j] - f.w[k], wp = f.w[j] + f.w[k];
            const cd im = fabs(wm) < 1e-14 ? t : (1.0 / wm) * (sc - cs);                           // int cos(wm s) ds
            const cd ip = fabs(wp) < 1e-14 ? c_2cep * t : (1.0 / wp) * ((sc + cs) - mk(s_2cep, 0.0));  // int cos(wp s + 2 cep)
            r.G = r.G + cf * (im - ip);
        }
    return r;
}

}  // namespace sfhk
