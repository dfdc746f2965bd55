// df.cuh -- double-float arithmetic for the split-precision (fp64-accurate) path.
//
// A df value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2 after
// normalisation, about 48 significant bits.  Products use FMA to obtain the exact
// low part of h_a h_b (Dekker/Kahan two-product); sums use Knuth's TwoSum and
// Fast2Sum.  On GB300 these FP32 sequences run far faster than the FP64 pipe
// (2 FP64 FMA/clk/SM against 128 FP32 FMA/clk/SM).  A complex value (cdf) is
// stored as float4 (re.h, re.l, im.h, im.l), the same 16 bytes as a complex128.
#pragma once

#include <cuda_runtime.h>

namespace nnfft {
namespace dfa {

struct df {
    float h, l;
};
struct cdf {
    df re, im;
};

__device__ __forceinline__ df mk(float h, float l = 0.0f) {
    df r;
    r.h = h;
    r.l = l;
    return r;
}

// Fast2Sum: requires |a| >= |b| (or a == 0); returns the normalised pair
__device__ __forceinline__ df fast2sum(float a, float b) {
    df r;
    r.h = a + b;
    r.l = b - (r.h - a);
    return r;
}

__device__ __forceinline__ df norm(df a) { return fast2sum(a.h, a.l); }

// accurate sum of two df values
__device__ __forceinline__ df add(df a, df b) {
    const float s = a.h + b.h;
    const float bp = s - a.h;
    const float e = (a.h - (s - bp)) + (b.h - bp);
    return fast2sum(s, e + (a.l + b.l));
}

// a + b with TwoSum on the high parts and the low parts added, not renormalised (for the
// exchanges of partial sums, which are renormalised once at the end with norm_any)
__device__ __forceinline__ df add_lazy(df a, df b) {
    const float s = a.h + b.h;
    const float bp = s - a.h;
    const float e = (a.h - (s - bp)) + (b.h - bp);
    return mk(s, (a.l + b.l) + e);
}

// normalise with TwoSum: no ordering requirement on |h| and |l|
__device__ __forceinline__ df norm_any(df a) {
    const float s = a.h + a.l;
    const float bp = s - a.h;
    return mk(s, (a.h - (s - bp)) + (a.l - bp));
}

__device__ __forceinline__ df neg(df a) { return mk(-a.h, -a.l); }
__device__ __forceinline__ df sub(df a, df b) { return add(a, neg(b)); }

// product, low parts of the low x low term dropped (below 2^-48 relative); unnormalised
__device__ __forceinline__ df mul_u(df a, df b) {
    df r;
    r.h = a.h * b.h;
    float e = fmaf(a.h, b.h, -r.h);
    e = fmaf(a.h, b.l, e);
    r.l = fmaf(a.l, b.h, e);
    return r;
}
__device__ __forceinline__ df mul(df a, df b) { return norm(mul_u(a, b)); }

// s += p with TwoSum on the high parts; low parts accumulate (normalise at the end)
__device__ __forceinline__ void acc(df &s, df p) {
    const float t = s.h + p.h;
    const float bp = t - s.h;
    const float e = (s.h - (t - bp)) + (p.h - bp);
    s.l = s.l + (e + p.l);
    s.h = t;
}

__device__ __forceinline__ cdf cadd(cdf a, cdf b) {
    cdf r;
    r.re = add(a.re, b.re);
    r.im = add(a.im, b.im);
    return r;
}
__device__ __forceinline__ cdf csub(cdf a, cdf b) {
    cdf r;
    r.re = sub(a.re, b.re);
    r.im = sub(a.im, b.im);
    return r;
}
// a * w
__device__ __forceinline__ cdf cmul(cdf a, cdf w) {
    cdf r;
    r.re = sub(mul_u(a.re, w.re), mul_u(a.im, w.im));
    r.im = add(mul_u(a.re, w.im), mul_u(a.im, w.re));
    return r;
}
// a * (i * sign), sign = +-1
__device__ __forceinline__ cdf cmul_isign(cdf a, int sign) {
    cdf r;
    if (sign > 0) {
        r.re = neg(a.im);
        r.im = a.re;
    } else {
        r.re = a.im;
        r.im = neg(a.re);
    }
    return r;
}
// a * s for a df scalar s
__device__ __forceinline__ cdf cscale(cdf a, df s) {
    cdf r;
    r.re = mul(a.re, s);
    r.im = mul(a.im, s);
    return r;
}
__device__ __forceinline__ cdf conj_if(cdf a, bool c) {
    if (c) a.im = neg(a.im);
    return a;
}

__device__ __forceinline__ cdf ld(const float4 *p) {
    const float4 v = *p;
    cdf r;
    r.re = mk(v.x, v.y);
    r.im = mk(v.z, v.w);
    return r;
}
__device__ __forceinline__ void st(float4 *p, cdf a) {
    *p = make_float4(a.re.h, a.re.l, a.im.h, a.im.l);
}
__device__ __forceinline__ cdf czero() {
    cdf r;
    r.re = mk(0.f);
    r.im = mk(0.f);
    return r;
}

// double -> (hi, lo) floats with integer operations only: hi keeps the top 24
// significant bits (truncated), lo the next 24 (rounded), so hi + lo = x to 2^-48.
// |x| outside [2^-75, 2^127) loses the lo part (or both parts below 2^-100).
__device__ __forceinline__ df split_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int ex = (int)((hi >> 20) & 0x7ffu);
    const unsigned mh = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const bool ok = ex > 1023 - 100 && ex < 1023 + 127;
    df r;
    r.h = ok ? __uint_as_float(sign | ((unsigned)(ex - 896) << 23) | mh) : 0.0f;
    const float rem = __uint2float_rn(lo & 0x1fffffffu);
    const int se = ex - 1075 + 127;
    const float scale = se > 0 ? __uint_as_float((unsigned)se << 23) : 0.0f;
    const float lv = rem * scale;
    r.l = ok ? (sign ? -lv : lv) : 0.0f;
    return r;
}

// float -> double with integer operations (exact; zero and subnormals -> signed 0)
__device__ __forceinline__ double float_to_double_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned ex = (u >> 23) & 0xffu;
    const unsigned man = u & 0x7fffffu;
    const unsigned hi = ex ? (sign | ((ex + 896u) << 20) | (man >> 3)) : sign;
    const unsigned lo = ex ? ((man & 7u) << 29) : 0u;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

__device__ __forceinline__ double to_double(df a) {
    return float_to_double_bits(a.h) + float_to_double_bits(a.l);
}

}  // namespace dfa
}  // namespace nnfft
