// Double values as unevaluated sums of two floats, and compensated FP32 arithmetic on them: the
// mixed solver forms the right-hand side of its steps, the residual apply, the gradient products
// of Eq. grad-int and the state update of the implicit midpoint rule with these instead of FP64
// multiply-adds.  On this GPU a warp's FP64 instruction occupies the issuing warp for ~60 cycles
// and the SM retires ~2 FP64 lanes a cycle, against 128 FP32 lanes.  Every function here runs on
// the host too (the CPU tests pin them);
// the host side must be compiled without floating-point contraction (-ffp-contract=off), the
// device side uses the _rn intrinsics, which the compiler never fuses.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace msqoc {

// ------------------------------------------------------------------ bit casts (host and device)
__host__ __device__ __forceinline__ uint64_t bits_of(double x) {
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return u;
}
__host__ __device__ __forceinline__ double double_of(uint64_t u) {
    double x;
    memcpy(&x, &u, sizeof x);
    return x;
}
__host__ __device__ __forceinline__ uint32_t bits_of(float x) {
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    return u;
}
__host__ __device__ __forceinline__ float float_of(uint32_t u) {
    float x;
    memcpy(&x, &u, sizeof x);
    return x;
}

// ------------------------------------------------------------------ FP32 operations, never fused
#ifdef __CUDA_ARCH__
__device__ __forceinline__ float fmul_n(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd_n(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub_n(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ffma_n(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float fmul_n(float a, float b) { return a * b; }
inline float fadd_n(float a, float b) { return a + b; }
inline float fsub_n(float a, float b) { return a - b; }
inline float ffma_n(float a, float b, float c) { return __builtin_fmaf(a, b, c); }
#endif

// ------------------------------------------------------------------ the split
// x 2^-sh = hi + lo + err with hi = x 2^-sh rounded to 24 bits (ties away from zero, as the
// mixed solver's f64 -> f32 conversion), lo = the remainder rounded to nearest, |err| <= 2^-48
// |x 2^-sh|.  Range (of the scaled value x'): |x'| < 2^-126 and FP64 zeros and subnormals give
// hi = lo = signed zero; for 2^-126 <= |x'| < 2^-74 lo is zero (|err| <= 2^-24 |x'|); |x'| must
// stay below 2^127 (the mixed solver's column scale keeps it below 1).  Integer and FP32
// operations only: hi is the top 24 bits of the scaled double, lo is the dropped 29-bit
// remainder k (a signed count of units 2^(e - 1075) of the scaled exponent field e) converted
// in two exact halves and scaled by a power of two.
// The arithmetic is on the two 32-bit words of the double: with 64-bit integer arithmetic on the
// double's bits the device executed one FP64 add per split (ncu), an FP64-pipe instruction
// that the step's split of its state paid six times a fiber.
__host__ __device__ __forceinline__ float2 split_scaled(double x, int sh) {
#ifdef __CUDA_ARCH__
    const uint32_t whi = static_cast<uint32_t>(__double2hiint(x)), wlo = static_cast<uint32_t>(__double2loint(x));
#else
    const uint64_t u = bits_of(x);
    const uint32_t whi = static_cast<uint32_t>(u >> 32), wlo = static_cast<uint32_t>(u);
#endif
    const uint32_t sgn = whi & 0x80000000u;
    const uint32_t ahi = whi & 0x7fffffffu;
    const int ex = static_cast<int>(ahi >> 20);
    const int e = ex - sh;   // exponent field of x 2^-sh
    if (ex == 0 || e < 897) return make_float2(float_of(sgn), float_of(sgn));
    // r = |x| 2^-sh (exponent field lowered by sh) + 2^28, as words (rhi, rlo)
    const uint32_t rlo = wlo + (1u << 28);
    const uint32_t rhi = ahi - (static_cast<uint32_t>(sh) << 20) + (rlo < wlo ? 1u : 0u);
    const float hi = float_of((((rhi << 3) | (rlo >> 29)) - (896u << 23)) | sgn);   // r >> 29
    const int k = static_cast<int>(rlo & 0x1fffffffu) - (1 << 28);
    // float(k), rounded once: k = kh 2^14 + kl with both halves exact through the 1.5 2^23 trick
    const float fkh = fsub_n(float_of(0x4b400000u + static_cast<uint32_t>(k >> 14)), 12582912.f);
    const float fkl = fsub_n(float_of(0x4b400000u + static_cast<uint32_t>(k & 0x3fff)), 12582912.f);
    const float kf = ffma_n(fkh, 16384.f, fkl);
    const float unit = float_of((static_cast<uint32_t>(e - 948) << 23) | sgn);   // +-2^(e - 1075)
    const float lo = e < 949 ? float_of(sgn) : fmul_n(kf, unit);
    return make_float2(hi, lo);
}
// a complex entry: (hi.x, hi.y, lo.x, lo.y)
__host__ __device__ __forceinline__ float4 split_scaled(double2 v, int sh) {
    const float2 x = split_scaled(v.x, sh), y = split_scaled(v.y, sh);
    return make_float4(x.x, y.x, x.y, y.y);
}

// ------------------------------------------------------------------ compensated accumulation
// A sum kept as s + c (floats): s the running FP32 sum, c the accumulated rounding errors and
// low-order terms.
struct DF {
    float s, c;
};
// a += x y for x = xh + xl, y = yh + yl: xh yh = p + e exactly (FMA), p added to s with an exact
// two-sum, e, the two-sum's error and the cross terms xh yl + xl yh added to c; xl yl
// (<= 2^-48 |x y|) is dropped.  Error of the finished sum: about 2^-47 times the sum of the
// magnitudes of its terms and partial sums.
__host__ __device__ __forceinline__ void df_mac(DF& a, float xh, float xl, float yh, float yl) {
    const float p = fmul_n(xh, yh);
    const float e = ffma_n(xh, yh, -p);
    const float s = fadd_n(a.s, p);
    const float bp = fsub_n(s, a.s);
    const float t = fadd_n(fsub_n(a.s, fsub_n(s, bp)), fsub_n(p, bp));
    a.s = s;
    a.c = fadd_n(a.c, fadd_n(t, ffma_n(xh, yl, ffma_n(xl, yh, e))));
}
// a + b (exact two-sum of the leading parts)
__host__ __device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = fadd_n(a.s, b.s);
    const float bp = fsub_n(s, a.s);
    const float t = fadd_n(fsub_n(a.s, fsub_n(s, bp)), fsub_n(b.s, bp));
    return DF{s, fadd_n(fadd_n(a.c, b.c), t)};
}
// a + b as s + c with s = RN(a + b) and c its exact error (two-sum)
__host__ __device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = fadd_n(a, b);
    const float bp = fsub_n(s, a);
    return DF{s, fadd_n(fsub_n(a, fsub_n(s, bp)), fsub_n(b, bp))};
}
// a + b as s + c for |a| >= |b| (or a = 0): s = RN(a + b), c its exact error
__host__ __device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = fadd_n(a, b);
    return DF{s, fsub_n(b, fsub_n(s, a))};
}
// one real part of a complex product, x1 y1 + x2 y2 for split factors (h, l): the two leading
// products exact (FMA) and added with an exact two-sum, their errors and the four cross terms
// in the low part; the l l terms (<= 2^-48 of each product) are dropped
__host__ __device__ __forceinline__ DF dot2_df(float x1h, float x1l, float y1h, float y1l, float x2h, float x2l,
                                               float y2h, float y2l) {
    const float p1 = fmul_n(x1h, y1h), e1 = ffma_n(x1h, y1h, -p1);
    const float p2 = fmul_n(x2h, y2h), e2 = ffma_n(x2h, y2h, -p2);
    const DF s = two_sum(p1, p2);
    float c = ffma_n(x1h, y1l, e1);
    c = ffma_n(x1l, y1h, c);
    c = ffma_n(x2h, y2l, c);
    c = ffma_n(x2l, y2h, c);
    return DF{s.s, fadd_n(fadd_n(c, e2), s.c)};
}
// x y for split complex x = (hi.x, hi.y, lo.x, lo.y) and y split the same way
__host__ __device__ __forceinline__ void cmul_df(const float4& x, const float4& y, DF& re, DF& im) {
    re = dot2_df(x.x, x.z, y.x, y.z, -x.y, -x.w, y.y, y.w);
    im = dot2_df(x.x, x.z, y.y, y.w, x.y, x.w, y.x, y.z);
}
// a w for w = wh + wl (a constant split the same way)
__host__ __device__ __forceinline__ DF df_scale(DF a, float wh, float wl) {
    const float p = fmul_n(a.s, wh);
    const float e = ffma_n(a.s, wh, -p);
    return DF{p, ffma_n(a.c, wh, ffma_n(a.s, wl, e))};
}
__host__ __device__ __forceinline__ DF df_neg(DF a) { return DF{-a.s, -a.c}; }

// sqrt(j) for a ladder weight (j >= 1) as hi + lo floats (compile-time constants)
__host__ __device__ constexpr float sqrt_hi(int j) {
    return static_cast<float>(j == 1 ? 1.0 : j == 2 ? 1.4142135623730951 : j == 3 ? 1.7320508075688772 : 2.0);
}
__host__ __device__ constexpr float sqrt_lo(int j) {
    return static_cast<float>((j == 1 ? 1.0 : j == 2 ? 1.4142135623730951 : j == 3 ? 1.7320508075688772 : 2.0) -
                              static_cast<double>(sqrt_hi(j)));
}
// a sqrt(j), the identity for j = 1
__host__ __device__ __forceinline__ DF df_scale_sqrt(DF a, int j) {
    if (j == 1) return a;
    return df_scale(a, j == 2 ? sqrt_hi(2) : j == 3 ? sqrt_hi(3) : sqrt_hi(4),
                    j == 2 ? sqrt_lo(2) : j == 3 ? sqrt_lo(3) : sqrt_lo(4));
}

// f 2^sh as a double: exact where the result is a normal double, rounded to nearest (ties up)
// among the double subnormals below that range, infinity above it; zero and FP32 subnormals
// give signed zero.  Integer operations only.
__host__ __device__ __forceinline__ double f64_of_float_scaled(float f, int sh) {
    const uint32_t b = bits_of(f);
    const uint64_t sgn = static_cast<uint64_t>(b & 0x80000000u) << 32;
    const uint32_t a = b & 0x7fffffffu;
    const int e = static_cast<int>(a >> 23) + 896 + sh;   // biased double exponent
    uint64_t mag = 0;
    if (a >= 0x00800000u) {
        if (e >= 2047) {
            mag = uint64_t(0x7ff) << 52;
        } else if (e > 0) {
            mag = static_cast<uint64_t>(e) << 52 | static_cast<uint64_t>(a & 0x7fffffu) << 29;
        } else {
            // subnormal: the 24-bit significand in units of 2^-1074 is m 2^(e + 28)
            const uint64_t m = (a & 0x7fffffu) | 0x800000u;
            const int s = e + 28;
            mag = s >= 0 ? m << s : (s > -25 ? (m + (uint64_t(1) << (-s - 1))) >> -s : 0);
        }
    }
    return double_of(sgn | mag);
}
// f 2^sh as a double for |sh| <= 896, where every normal float gives a normal double: the
// exponent moved by 896 + sh, the significand widened; zero and FP32 subnormals give signed
// zero (the mixed solver's column scale keeps its values' scaled magnitudes in that range).
// Integer operations on the two 32-bit words only.
__host__ __device__ __forceinline__ double f64_of_float_scaled_normal(float f, int sh) {
    const uint32_t b = bits_of(f);
    const uint32_t sgn = b & 0x80000000u, a = b & 0x7fffffffu;
    const uint32_t hi = a < 0x00800000u ? sgn : (sgn | ((a >> 3) + (static_cast<uint32_t>(896 + sh) << 20)));
    const uint32_t lo = a < 0x00800000u ? 0u : a << 29;
#ifdef __CUDA_ARCH__
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
#else
    return double_of(static_cast<uint64_t>(hi) << 32 | lo);
#endif
}
// the finished sum s + c times 2^sh, as one double (one FP64 add)
__host__ __device__ __forceinline__ double df_to_f64_scaled(DF a, int sh) {
    return f64_of_float_scaled(a.s, sh) + f64_of_float_scaled(a.c, sh);
}

// ------------------------------------------------------------------ the compensated state update
// The mixed solver's implicit-midpoint state update U_{n+1} = 2 Ubar - U_n = R U_n + 2 d, with
// R = 2P - 1, P = 1 / (1 + i kappa) the diagonal preconditioner entry (kappa = (h/2) D real) and d
// the step's correction (Ubar = P U_n + d).  Since R - 1 = -2 i kappa P, where |2 kappa| <= 2^-4.5
// the state is kept as an FP64 part u and an FP32 carry (units 2^-sh) and
//   u' + carry' = u + carry + 2 kappa (Im b, -Re b) + 2 d,   b = P (u + carry),
// the increment formed as a two-float sum s + c and renormalised: u' = u + s (one FP64 add; s is
// exact as a double), carry' = c.  b is the step's right-hand side (carry_rhs); its compensated
// error (about 2^-47 |b|) enters times |2 kappa|, of the order of the FP64 rounding of u.
constexpr double CARRY_UPDATE_K2 = 0.001953125;   // (2 kappa)^2 <= 2^-9

// The constants P and 2 kappa enter every step, so their splits are made exact with a third part
// (x - hi - lo, at most 5 bits: exact as a float): otherwise the 2^-48 remainders of the splits
// would act as a constant error of P and kappa and add up over the steps.
__host__ __device__ __forceinline__ float split_third(double x, float2 s) {
    return static_cast<float>((x - static_cast<double>(s.x)) - static_cast<double>(s.y));
}
// b = P (u + carry) from the split u (units 2^-sh), the split P and its third parts P3; the
// carry (at most half an FP32 unit of the last increment) goes into the low parts
__host__ __device__ __forceinline__ void carry_rhs(const float4& us, const float4& P, float2 P3, float2 car, DF& bre,
                                                   DF& bim) {
    cmul_df(us, P, bre, bim);
    const float cr = ffma_n(P.x, car.x, ffma_n(-P.y, car.y, ffma_n(P3.x, us.x, fmul_n(-P3.y, us.y))));
    const float ci = ffma_n(P.x, car.y, ffma_n(P.y, car.x, ffma_n(P3.x, us.y, fmul_n(P3.y, us.x))));
    bre.c = fadd_n(bre.c, cr);
    bim.c = fadd_n(bim.c, ci);
}
// u' (returned) and carry' from u, b = (bre, bim), the split 2 kappa (k2) and its third part k3,
// and d = (dre, dim)
__host__ __device__ __forceinline__ double2 carry_update(double2 u, DF bre, DF bim, float2 k2, float k3, DF dre, DF dim,
                                                         int sh, float2& car) {
    DF qr = df_scale(bim, k2.x, k2.y), qi = df_neg(df_scale(bre, k2.x, k2.y));
    qr.c = fadd_n(qr.c, ffma_n(k3, bim.s, car.x));
    qi.c = fadd_n(qi.c, ffma_n(-k3, bre.s, car.y));
    const DF ar = df_add(qr, DF{fadd_n(dre.s, dre.s), fadd_n(dre.c, dre.c)});
    const DF ai = df_add(qi, DF{fadd_n(dim.s, dim.s), fadd_n(dim.c, dim.c)});
    // renormalised, so that u takes all but the last rounding of the increment and the carry
    // stays within half an FP32 unit of it (else it would gather the low parts of every step)
    // (a fast two-sum: |ar.c| is below |ar.s| but where ar.s cancels to nothing, and there the
    // carry's error is of the order of the cancelled parts' rounding)
    const DF xr = fast_two_sum(ar.s, ar.c), xi = fast_two_sum(ai.s, ai.c);
    car = make_float2(xr.c, xi.c);
    return make_double2(u.x + f64_of_float_scaled_normal(xr.s, sh), u.y + f64_of_float_scaled_normal(xi.s, sh));
}
// the state u + carry as one double (one FP64 add a component)
__host__ __device__ __forceinline__ double2 carry_finish(double2 u, float2 car, int sh) {
    return make_double2(u.x + f64_of_float_scaled_normal(car.x, sh), u.y + f64_of_float_scaled_normal(car.y, sh));
}

}  // namespace msqoc
