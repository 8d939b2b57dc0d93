// Device-side storage formats of spinor and link fields, and complex helpers.
//
// Spinor formats (one parity, one right-hand side; site index i = lex/2):
//   SpF64  [12][vh] double2   planar complex128 (the canonical FP64 layout)
//   SpF32  [12][vh] float2    planar complex64  (the canonical FP32 layout)
//   SpH16  [3][vh] uint4 + [vh] float   16-bit values scaled by a per-site norm:
//          uint4 plane q holds spin-colour components 4q..4q+3 as half2 (re, im);
//          norm[i] = max |real or imaginary part| over the site's 24 reals
//   SpB16  like SpH16 with bfloat16 values
// Link formats (one direction mu, one base-site parity; 3x3 complex per site):
//   LkF64_18 [9][vh] double2            row-major U_ab
//   LkF64_12 [6][vh] double2            rows 0, 1; row 2 = conj(row0 x row1)
//   LkF32_18 [4][vh] float4 + [vh] float2
//   LkF32_12 [3][vh] float4
//   LkH16_18 [2][vh] uint4 + [vh] uint32 (half2 per complex)
//   LkH16_12 [vh] uint4 + [vh] uint2
//   LkB16_*  like LkH16_* with bfloat16
// Every plane starts on a 16-byte boundary because vh = V/2 is a multiple of 8.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace weo {

template <typename T>
struct cx {
    T r, i;
};

// ---------------------------------------------------------- float-float --
// A float-float number hi + lo (|lo| <= half an ulp of hi) carries about 48
// significant bits, enough for FP64-class accuracy, with FP32 arithmetic only:
// Knuth's error-free two-sum, the FMA-based exact product of two floats
// (Dekker's product without splitting) and the usual renormalisation
// (double-float arithmetic as in Dekker 1971 and the QD / DSFUN libraries).
// On GB300 the FP32 pipes issue 64 times as many operations per cycle as the
// FP64 pipe, so a stencil in this arithmetic outruns native FP64 several-fold.
// The _rn intrinsics keep the compiler from contracting the error-free steps
// into fused multiply-adds, which would change what they compute.
struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr ff(int v) : hi(float(v)), lo(0.f) {}
    __host__ __device__ constexpr ff(float v) : hi(v), lo(0.f) {}
    __device__ ff(double v) : hi(float(v)), lo(float(v - double(float(v)))) {}
};

// s + e = a + b exactly
__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ void ff_fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator+(ff a, ff b)
{
    float s, e;
    ff_two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    ff_fast_two_sum(s, e, s, e);
    return ff(s, e);
}
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
// a * b + (cross terms): exact product of the high parts as (p, e), with the
// two cross products folded into e (|e| ~ 2^-24 |p|; the sloppy addition
// below accepts such an unnormalised pair)
__device__ __forceinline__ ff ff_prod(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff(p, e);
}

// the float and double fma stay visible next to the float-float one
using ::fma;

// c + a * b: exact product of the high parts, cross terms in FP32, one
// renormalised sum
__device__ __forceinline__ ff fma(ff a, ff b, ff c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    ff_two_sum(p, c.hi, s, t);
    t = __fadd_rn(t, __fadd_rn(e, c.lo));
    ff_fast_two_sum(s, t, s, t);
    return ff(s, t);
}

template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.r - b.r, a.i - b.i}; }
// i * a
template <typename T>
__device__ __forceinline__ cx<T> cmuli(cx<T> a) { return {-a.i, a.r}; }
template <typename T>
__device__ __forceinline__ cx<T> cneg(cx<T> a) { return {-a.r, -a.i}; }
// acc + a * b
template <typename T>
__device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> acc)
{
    acc.r = fma(a.r, b.r, acc.r);
    acc.r = fma(-a.i, b.i, acc.r);
    acc.i = fma(a.r, b.i, acc.i);
    acc.i = fma(a.i, b.r, acc.i);
    return acc;
}
// acc + conj(a) * b
template <typename T>
__device__ __forceinline__ cx<T> cfmaconj(cx<T> a, cx<T> b, cx<T> acc)
{
    acc.r = fma(a.r, b.r, acc.r);
    acc.r = fma(a.i, b.i, acc.r);
    acc.i = fma(a.r, b.i, acc.i);
    acc.i = fma(-a.i, b.r, acc.i);
    return acc;
}
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) { return cfma(a, b, cx<T>{0, 0}); }
template <typename T>
__device__ __forceinline__ cx<T> cconj(cx<T> a) { return {a.r, -a.i}; }
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.r * s, a.i * s}; }

// ------------------------------------------------------------ loads/stores --
// Spinor neighbour reads are re-used by up to eight output sites: plain cached
// loads. Links are used once per pass: streaming loads (evict-first) so they do
// not push the spinor working set out of L2.

template <typename T>
__device__ __forceinline__ T ld_keep(const T *p) { return __ldg(p); }
template <typename T>
__device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }


// Load policies of the link fields. LdStream: the links are read once per pass
// (evict first). LdL2: another CTA reads the same links again shortly (the
// second hop of the fused M_eo): keep them in L2 at normal priority and skip L1.
struct LdStream {
    template <typename T>
    __device__ static __forceinline__ T ld(const T *p) { return __ldcs(p); }
};
struct LdL2 {
    template <typename T>
    __device__ static __forceinline__ T ld(const T *p) { return __ldcg(p); }
};

// ---------------------------------------------------------------- spinors --

struct SpF64 {
    using real = double;
    static constexpr int kBytesPerSite = 192;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> v[12])
    {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 d = ld_keep(p + k * vh + i);
            v[k] = {R(d.x), R(d.y)};
        }
    }
    template <typename R>
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<R> v[12])
    {
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k * vh + i] = make_double2(double(v[k].r), double(v[k].i));
    }
};

struct SpF32 {
    using real = float;
    static constexpr int kBytesPerSite = 96;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> v[12])
    {
        const float2 *p = static_cast<const float2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float2 d = ld_keep(p + k * vh + i);
            v[k] = {R(d.x), R(d.y)};
        }
    }
    template <typename R>
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<R> v[12])
    {
        float2 *p = static_cast<float2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k * vh + i] = make_float2(float(v[k].r), float(v[k].i));
    }
};

// FP64-class spinor in float-float: 12 planes of the high parts, then 12 of
// the low parts (192 bytes per site, as FP64).
struct SpFF {
    using real = ff;
    static constexpr int kBytesPerSite = 192;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> v[12])
    {
        const float2 *p = static_cast<const float2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float2 h = ld_keep(p + k * vh + i), l = ld_keep(p + (12 + k) * vh + i);
            v[k] = {ff(h.x, l.x), ff(h.y, l.y)};
        }
    }
    __device__ static __forceinline__ void store(void *base, long long vh, long long i, const cx<ff> v[12])
    {
        float2 *p = static_cast<float2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            p[k * vh + i] = make_float2(v[k].r.hi, v[k].i.hi);
            p[(12 + k) * vh + i] = make_float2(v[k].r.lo, v[k].i.lo);
        }
    }
};

struct H16Traits {
    using scalar2 = __half2;
    __device__ static __forceinline__ float2 to_f2(uint32_t u)
    {
        __half2 h = *reinterpret_cast<__half2 *>(&u);
        return __half22float2(h);
    }
    __device__ static __forceinline__ uint32_t from_f2(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};

struct B16Traits {
    using scalar2 = __nv_bfloat162;
    __device__ static __forceinline__ float2 to_f2(uint32_t u)
    {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
        return __bfloat1622float2(h);
    }
    __device__ static __forceinline__ uint32_t from_f2(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
};

// 16-bit spinor with per-site FP32 norm; Tr = H16Traits or B16Traits.
template <class Tr>
struct Sp16 {
    using real = float;
    static constexpr int kBytesPerSite = 52;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> v[12])
    {
        const uint4 *p = static_cast<const uint4 *>(base);
        const float *nrm = reinterpret_cast<const float *>(p + 3 * vh);
        const float n = ld_keep(nrm + i);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            uint4 w = ld_keep(p + q * vh + i);
            float2 a = Tr::to_f2(w.x), b = Tr::to_f2(w.y), c = Tr::to_f2(w.z), d = Tr::to_f2(w.w);
            v[4 * q + 0] = {R(a.x * n), R(a.y * n)};
            v[4 * q + 1] = {R(b.x * n), R(b.y * n)};
            v[4 * q + 2] = {R(c.x * n), R(c.y * n)};
            v[4 * q + 3] = {R(d.x * n), R(d.y * n)};
        }
    }
    template <typename R>
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<R> v[12])
    {
        uint4 *p = static_cast<uint4 *>(base);
        float *nrm = reinterpret_cast<float *>(p + 3 * vh);
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(float(v[k].r)), fabsf(float(v[k].i))));
        const float s = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            uint4 w;
            w.x = Tr::from_f2(float(v[4 * q + 0].r) * s, float(v[4 * q + 0].i) * s);
            w.y = Tr::from_f2(float(v[4 * q + 1].r) * s, float(v[4 * q + 1].i) * s);
            w.z = Tr::from_f2(float(v[4 * q + 2].r) * s, float(v[4 * q + 2].i) * s);
            w.w = Tr::from_f2(float(v[4 * q + 3].r) * s, float(v[4 * q + 3].i) * s);
            p[q * vh + i] = w;
        }
        nrm[i] = m;
    }
};
using SpH16 = Sp16<H16Traits>;
using SpB16 = Sp16<B16Traits>;

// ------------------------------------------------------------------ links --

template <typename R>
__device__ __forceinline__ void reconstruct_row2(cx<R> U[3][3])
{
    // row2 = conj(row0 x row1), exact for SU(3)
    U[2][0] = cconj(csub(cmul(U[0][1], U[1][2]), cmul(U[0][2], U[1][1])));
    U[2][1] = cconj(csub(cmul(U[0][2], U[1][0]), cmul(U[0][0], U[1][2])));
    U[2][2] = cconj(csub(cmul(U[0][0], U[1][1]), cmul(U[0][1], U[1][0])));
}

struct LkF64_18 {
    static constexpr int kBytesPerSite = 144;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> U[3][3])
    {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 d = ld_stream(p + k * vh + i);
            U[k / 3][k % 3] = {R(d.x), R(d.y)};
        }
    }
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<double> U[3][3])
    {
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int k = 0; k < 9; ++k) p[k * vh + i] = make_double2(U[k / 3][k % 3].r, U[k / 3][k % 3].i);
    }
};

struct LkF64_12 {
    static constexpr int kBytesPerSite = 96;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> U[3][3])
    {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            double2 d = ld_stream(p + k * vh + i);
            U[k / 3][k % 3] = {R(d.x), R(d.y)};
        }
        reconstruct_row2(U);
    }
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<double> U[3][3])
    {
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k * vh + i] = make_double2(U[k / 3][k % 3].r, U[k / 3][k % 3].i);
    }
};

template <class Ld = LdStream>
struct LkF32_18T {
    static constexpr int kBytesPerSite = 72;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> U[3][3])
    {
        const float4 *p = static_cast<const float4 *>(base);
        float4 a = Ld::ld(p + i), b = Ld::ld(p + vh + i), c = Ld::ld(p + 2 * vh + i),
               d = Ld::ld(p + 3 * vh + i);
        float2 e = Ld::ld(reinterpret_cast<const float2 *>(p + 4 * vh) + i);
        U[0][0] = {R(a.x), R(a.y)};
        U[0][1] = {R(a.z), R(a.w)};
        U[0][2] = {R(b.x), R(b.y)};
        U[1][0] = {R(b.z), R(b.w)};
        U[1][1] = {R(c.x), R(c.y)};
        U[1][2] = {R(c.z), R(c.w)};
        U[2][0] = {R(d.x), R(d.y)};
        U[2][1] = {R(d.z), R(d.w)};
        U[2][2] = {R(e.x), R(e.y)};
    }
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<double> U[3][3])
    {
        float4 *p = static_cast<float4 *>(base);
        p[i] = make_float4(U[0][0].r, U[0][0].i, U[0][1].r, U[0][1].i);
        p[vh + i] = make_float4(U[0][2].r, U[0][2].i, U[1][0].r, U[1][0].i);
        p[2 * vh + i] = make_float4(U[1][1].r, U[1][1].i, U[1][2].r, U[1][2].i);
        p[3 * vh + i] = make_float4(U[2][0].r, U[2][0].i, U[2][1].r, U[2][1].i);
        reinterpret_cast<float2 *>(p + 4 * vh)[i] = make_float2(U[2][2].r, U[2][2].i);
    }
};

template <class Ld = LdStream>
struct LkF32_12T {
    static constexpr int kBytesPerSite = 48;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> U[3][3])
    {
        const float4 *p = static_cast<const float4 *>(base);
        float4 a = Ld::ld(p + i), b = Ld::ld(p + vh + i), c = Ld::ld(p + 2 * vh + i);
        U[0][0] = {R(a.x), R(a.y)};
        U[0][1] = {R(a.z), R(a.w)};
        U[0][2] = {R(b.x), R(b.y)};
        U[1][0] = {R(b.z), R(b.w)};
        U[1][1] = {R(c.x), R(c.y)};
        U[1][2] = {R(c.z), R(c.w)};
        reconstruct_row2(U);
    }
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<double> U[3][3])
    {
        float4 *p = static_cast<float4 *>(base);
        p[i] = make_float4(U[0][0].r, U[0][0].i, U[0][1].r, U[0][1].i);
        p[vh + i] = make_float4(U[0][2].r, U[0][2].i, U[1][0].r, U[1][0].i);
        p[2 * vh + i] = make_float4(U[1][1].r, U[1][1].i, U[1][2].r, U[1][2].i);
    }
};

template <class Tr, class Ld = LdStream>
struct Lk16_18 {
    static constexpr int kBytesPerSite = 36;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> U[3][3])
    {
        const uint4 *p = static_cast<const uint4 *>(base);
        uint4 a = Ld::ld(p + i), b = Ld::ld(p + vh + i);
        uint32_t e = Ld::ld(reinterpret_cast<const unsigned int *>(p + 2 * vh) + i);
        const uint32_t w[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, e};
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float2 f = Tr::to_f2(w[k]);
            U[k / 3][k % 3] = {R(f.x), R(f.y)};
        }
    }
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<double> U[3][3])
    {
        uint32_t w[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) w[k] = Tr::from_f2(float(U[k / 3][k % 3].r), float(U[k / 3][k % 3].i));
        uint4 *p = static_cast<uint4 *>(base);
        p[i] = make_uint4(w[0], w[1], w[2], w[3]);
        p[vh + i] = make_uint4(w[4], w[5], w[6], w[7]);
        reinterpret_cast<unsigned int *>(p + 2 * vh)[i] = w[8];
    }
};

template <class Tr, class Ld = LdStream>
struct Lk16_12 {
    static constexpr int kBytesPerSite = 24;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> U[3][3])
    {
        const uint4 *p = static_cast<const uint4 *>(base);
        uint4 a = Ld::ld(p + i);
        uint2 b = Ld::ld(reinterpret_cast<const uint2 *>(p + vh) + i);
        const uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float2 f = Tr::to_f2(w[k]);
            U[k / 3][k % 3] = {R(f.x), R(f.y)};
        }
        reconstruct_row2(U);
    }
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<double> U[3][3])
    {
        uint32_t w[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = Tr::from_f2(float(U[k / 3][k % 3].r), float(U[k / 3][k % 3].i));
        uint4 *p = static_cast<uint4 *>(base);
        p[i] = make_uint4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<uint2 *>(p + vh)[i] = make_uint2(w[4], w[5]);
    }
};

// FP64-class links in float-float: the high parts in the LkF32_18 layout,
// then the low parts in the same layout (144 bytes per site, as FP64).
struct LkFF18 {
    static constexpr int kBytesPerSite = 144;
    template <typename R>
    __device__ static __forceinline__ void load(const void *base, long long vh, long long i,
                                                cx<R> U[3][3])
    {
        cx<float> H[3][3], L[3][3];
        LkF32_18T<>::load(base, vh, i, H);
        LkF32_18T<>::load(static_cast<const char *>(base) + 72 * vh, vh, i, L);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) U[a][b] = {ff(H[a][b].r, L[a][b].r), ff(H[a][b].i, L[a][b].i)};
    }
    __device__ static __forceinline__ void store(void *base, long long vh, long long i,
                                                 const cx<double> U[3][3])
    {
        cx<double> H[3][3], L[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const ff r(U[a][b].r), m(U[a][b].i);
                H[a][b] = {double(r.hi), double(m.hi)};
                L[a][b] = {double(r.lo), double(m.lo)};
            }
        LkF32_18T<>::store(base, vh, i, H);
        LkF32_18T<>::store(static_cast<char *>(base) + 72 * vh, vh, i, L);
    }
};

using LkF32_18 = LkF32_18T<>;
using LkF32_12 = LkF32_12T<>;
using LkH16_18 = Lk16_18<H16Traits>;
using LkH16_12 = Lk16_12<H16Traits>;
using LkB16_18 = Lk16_18<B16Traits>;
using LkB16_12 = Lk16_12<B16Traits>;

}  // namespace weo
