// Device-side building blocks shared by every kernel of the library:
// complex arithmetic, packed loads/stores of the even-odd spinor layout in
// FP64 / FP32 / BF16 storage, lattice geometry and block reductions.
//
// Internal field layout ("EO tile"): a half-lattice field of parity p holds
// complex values at [cb][c][r] with cb the checkerboard site index
// (lexicographic index >> 1), c = 3*spin + colour (12 components) and r the
// right-hand side (N of them, contiguous).  Threads of one site read the N
// right-hand sides of a component as one contiguous run, so every load of a
// warp is a handful of full 128-byte lines.
//
// Gauge layout: [parity][cb][mu][9 complex] (row-major 3x3 U_mu(x)).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace dl {

typedef __nv_bfloat16 bf16;

// ----------------------------------------------------------------------------
// complex numbers
// ----------------------------------------------------------------------------
template <typename T>
struct cx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T r, T i) { cx<T> z; z.re = r; z.im = i; return z; }
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a) { return mk(-a.re, -a.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// i*a and -i*a
template <typename T>
__device__ __forceinline__ cx<T> ti(cx<T> a) { return mk(-a.im, a.re); }
template <typename T>
__device__ __forceinline__ cx<T> tmi(cx<T> a) { return mk(a.im, -a.re); }
template <typename T>
__device__ __forceinline__ cx<T> cj(cx<T> a) { return mk(a.re, -a.im); }
// acc += a*b ; acc += conj(a)*b
template <typename T>
__device__ __forceinline__ void cmac(cx<T> &acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
template <typename T>
__device__ __forceinline__ void cjmac(cx<T> &acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}
template <typename T>
__device__ __forceinline__ cx<T> zero() { return mk<T>(T(0), T(0)); }

// ----------------------------------------------------------------------------
// float-float ("double-float") reals: the unevaluated sum hi + lo of two
// floats, about 48 significant bits.  Sums use Knuth's error-free two-sum and
// products the FMA-based exact product (Dekker), each followed by a
// renormalisation.  GB300 issues FP64 at about 1/60 of the FP32 rate, so FP64
// work whose rounding needs more than FP32 but not all 53 bits runs faster in
// this form on the FP32 pipes.
// ----------------------------------------------------------------------------
struct dfloat {
    float hi, lo;
    __device__ __forceinline__ dfloat() {}
    __device__ __forceinline__ explicit dfloat(float h) : hi(h), lo(0.f) {}
    __device__ __forceinline__ dfloat(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return dfloat(h, e - (h - s));
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return dfloat(h, e - (h - p));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df_add(a, -b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df_mul(a, b); }
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = df_add(a, b); }
// a * b + c with one renormalisation: the exact product's error terms and the
// two-sum error of p + c.hi are gathered into one low word.
__device__ __forceinline__ dfloat df_fma(dfloat a, dfloat b, dfloat c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = p + c.hi;
    const float bb = s - p;
    e += ((p - (s - bb)) + (c.hi - bb)) + c.lo;
    const float h = s + e;
    return dfloat(h, e - (h - s));
}
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return df_fma(a, b, c); }
// a + b as an unnormalised pair: the two-sum of the high parts with the low
// parts added to its error, without the final renormalisation (8 instructions
// instead of 11).  Used for operands of products, where a low part up to a few
// units of the high part's last place costs no accuracy: the error stays below
// 2^-47 of |a| + |b|.
__device__ __forceinline__ dfloat df_add_lazy(dfloat a, dfloat b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return dfloat(s, e + (a.lo + b.lo));
}

// Unnormalised float-float accumulator: the value is s + e, where s is the
// running float sum of the high parts and e gathers the two-sum errors of
// those additions and the low parts of the terms.  One addition costs 8
// instructions and a product-accumulate 12 (against 11 and 15 with a
// renormalisation each time); da_norm renormalises once at the end.  Over K
// terms the error stays below about K 2^-48 of the sum of their magnitudes.
struct dacc {
    float s, e;
};
__device__ __forceinline__ void da_add(dacc &a, float hi, float lo) {
    const float t = a.s + hi;
    const float bb = t - a.s;
    const float err = (a.s - (t - bb)) + (hi - bb);
    a.s = t;
    a.e += err + lo;
}
// a += x * y (the exact product of the high parts, the two cross terms; x.lo y.lo dropped)
__device__ __forceinline__ void da_mac(dacc &a, dfloat x, dfloat y) {
    const float p = x.hi * y.hi;
    float pe = fmaf(x.hi, y.hi, -p);
    pe = fmaf(x.hi, y.lo, pe);
    pe = fmaf(x.lo, y.hi, pe);
    da_add(a, p, pe);
}
__device__ __forceinline__ dfloat da_norm(dacc a) {
    const float h = a.s + a.e;
    return dfloat(h, a.e - (h - a.s));
}
// Complex lazy accumulator and its updates.
struct cdacc {
    dacc re, im;
};
__device__ __forceinline__ cdacc cda_zero() {
    cdacc z;
    z.re.s = z.re.e = z.im.s = z.im.e = 0.f;
    return z;
}
// w += u h (DAG: conj(u) h)
template <bool DAG>
__device__ __forceinline__ void cda_mac(cdacc &w, cx<dfloat> u, cx<dfloat> h) {
    const dfloat ui = DAG ? -u.im : u.im;
    da_mac(w.re, u.re, h.re);
    da_mac(w.re, -ui, h.im);
    da_mac(w.im, u.re, h.im);
    da_mac(w.im, ui, h.re);
}
// acc += r w with r = 1, i, -1, -i for ROT = 0, 1, 2, 3
template <int ROT>
__device__ __forceinline__ void cda_add(cdacc &acc, const cdacc &w) {
    if (ROT == 0) {
        da_add(acc.re, w.re.s, w.re.e);
        da_add(acc.im, w.im.s, w.im.e);
    } else if (ROT == 1) {
        da_add(acc.re, -w.im.s, -w.im.e);
        da_add(acc.im, w.re.s, w.re.e);
    } else if (ROT == 2) {
        da_add(acc.re, -w.re.s, -w.re.e);
        da_add(acc.im, -w.im.s, -w.im.e);
    } else {
        da_add(acc.re, w.im.s, w.im.e);
        da_add(acc.im, -w.re.s, -w.re.e);
    }
}
// double -> float-float with FP64 arithmetic (exact for normal floats).
__device__ __forceinline__ dfloat df_from_double(double x) {
    const float h = (float)x;
    return dfloat(h, (float)(x - (double)h));
}
// double -> float-float from its bit pattern with integer operations only
// (no FP64 instruction).  hi keeps the leading 24 significant bits
// (truncated); lo is the remaining 29 bits rounded to a float, so hi + lo
// agrees with x to about 2^-48 relative.  |x| below 2^-126 becomes 0, the lo
// part of |x| below 2^-74 is dropped, and infinities and NaN propagate in hi.
__device__ __forceinline__ dfloat df_from_bits(uint32_t w0, uint32_t w1) {
    const uint32_t sign = w1 & 0x80000000u;
    const int e = (int)((w1 >> 20) & 0x7ffu);
    if (e == 0x7ff) {
        const bool nan = ((w1 & 0xfffffu) | w0) != 0u;
        return dfloat(__uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.f);
    }
    const int eb = e - 1023 + 127;  // float exponent field of hi
    if (eb <= 0) return dfloat(0.f, 0.f);
    if (eb >= 255) return dfloat(__uint_as_float(sign | 0x7f800000u), 0.f);
    const float hi = __uint_as_float(sign | ((uint32_t)eb << 23) | ((w1 & 0xfffffu) << 3) | (w0 >> 29));
    const int es = e - 1075 + 127;  // float exponent field of 2^(e - 1075), the weight of mantissa bit 0
    float lo = es > 0 ? __uint2float_rn(w0 & 0x1fffffffu) * __uint_as_float((uint32_t)es << 23) : 0.f;
    return dfloat(hi, sign ? -lo : lo);
}
// float-float -> double with integer operations only.  hi is widened exactly to
// a 53-bit significand and lo, which lies at least 24 binary places below it
// once renormalised, is added on that integer significand; bits of lo below its
// last place are truncated (error below 2^-52 relative).  A zero or subnormal
// hi gives a signed zero, an infinite or NaN hi propagates, and an
// unnormalised pair (lo within 24 places of hi) takes the FP64 sum.
__device__ __forceinline__ double df_to_f64(dfloat x) {
    const uint32_t hb = __float_as_uint(x.hi), lb = __float_as_uint(x.lo);
    const int he = (int)((hb >> 23) & 0xffu), le = (int)((lb >> 23) & 0xffu);
    const uint64_t sign = (uint64_t)(hb >> 31) << 63;
    if (he == 0) return __longlong_as_double((long long)sign);
    if (he == 0xff)
        return __longlong_as_double((long long)(sign | (0x7ffull << 52) | ((hb & 0x7fffffu) ? (1ull << 51) : 0ull)));
    const uint32_t lsig = le ? ((lb & 0x7fffffu) | 0x800000u) : (lb & 0x7fffffu);  // subnormal lo: no hidden bit
    const int sh = he - (le ? le : 1);
    if (lsig != 0 && sh < 24) return (double)x.hi + (double)x.lo;
    uint64_t m = (uint64_t)((hb & 0x7fffffu) | 0x800000u) << 29;  // hi on 53 bits
    int e = he;
    if (lsig != 0 && sh < 53) {
        const uint64_t l = lsig;
        const uint64_t lm = sh <= 29 ? (l << (29 - sh)) : (l >> (sh - 29));  // lo in units of m's last place
        if ((hb ^ lb) >> 31) {
            m -= lm;
            if (!(m >> 52)) {
                m <<= 1;
                --e;
            }
        } else {
            m += lm;
            if (m >> 53) {
                m >>= 1;
                ++e;
            }
        }
    }
    return __longlong_as_double((long long)(sign | ((uint64_t)(e - 127 + 1023) << 52) | (m & ((1ull << 52) - 1))));
}

// Shuffle of a real across a warp (float-float: both halves).
template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
template <>
__device__ __forceinline__ dfloat shfl_xor<dfloat>(dfloat v, int off) {
    return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

// A host-side double coefficient in the arithmetic type T.
template <typename T> __device__ __forceinline__ T from_double(double x) { return (T)x; }
template <> __device__ __forceinline__ dfloat from_double<dfloat>(double x) { return df_from_double(x); }

// ----------------------------------------------------------------------------
// storage traits: S is the element type in memory (re and im interleaved);
// arithmetic happens in Real<S> (double for FP64 storage, float otherwise).
// ----------------------------------------------------------------------------
template <typename S> struct Real;
template <> struct Real<double> { typedef double type; };
template <> struct Real<float> { typedef float type; };
template <> struct Real<bf16> { typedef float type; };

// FP32 storage with the right-hand sides of a field interleaved in pairs: each
// 16-byte group holds (re_r, re_r+1, im_r, im_r+1) for the two right-hand
// sides r = 2k, 2k+1 of one field element (N even).  An element's address is
// the one it has in the plain FP32 layout (re, im pairs of floats), so the
// kernels' offsets do not change: only the order inside each group does.
// Groups start on 16-byte boundaries (field bases are), so bit 3 of an
// element's address tells which member of its pair it is.  One 16-byte load
// gives the real parts of two right-hand sides as one FP32 pair and their
// imaginary parts as another: the operands of the packed FP32 instructions.
struct f32p {
    float v;
};
template <> struct Real<f32p> { typedef float type; };
template <typename S> struct IsPaired { static constexpr bool v = false; };
template <> struct IsPaired<f32p> { static constexpr bool v = true; };

template <typename S>
__host__ __device__ constexpr int cbytes() { return 2 * (int)sizeof(S); }

// raw loads of NB bytes (NB in 4, 8, 16, 32, 64), read-only path (NC) or plain.
template <int NB, bool NC>
struct RawLd;
template <bool NC> struct RawLd<4, NC> {
    __device__ __forceinline__ static void ld(const void *p, uint32_t *w) {
        w[0] = NC ? __ldg((const unsigned int *)p) : *(const unsigned int *)p;
    }
};
template <bool NC> struct RawLd<8, NC> {
    __device__ __forceinline__ static void ld(const void *p, uint32_t *w) {
        uint2 v = NC ? __ldg((const uint2 *)p) : *(const uint2 *)p;
        w[0] = v.x; w[1] = v.y;
    }
};
template <bool NC> struct RawLd<16, NC> {
    __device__ __forceinline__ static void ld(const void *p, uint32_t *w) {
        uint4 v = NC ? __ldg((const uint4 *)p) : *(const uint4 *)p;
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
};
template <bool NC> struct RawLd<32, NC> {
    __device__ __forceinline__ static void ld(const void *p, uint32_t *w) {
        RawLd<16, NC>::ld(p, w);
        RawLd<16, NC>::ld((const char *)p + 16, w + 4);
    }
};
template <bool NC> struct RawLd<64, NC> {
    __device__ __forceinline__ static void ld(const void *p, uint32_t *w) {
        RawLd<32, NC>::ld(p, w);
        RawLd<32, NC>::ld((const char *)p + 32, w + 8);
    }
};

template <int NB>
struct RawSt;
template <> struct RawSt<4> {
    __device__ __forceinline__ static void st(void *p, const uint32_t *w) { *(unsigned int *)p = w[0]; }
};
template <> struct RawSt<8> {
    __device__ __forceinline__ static void st(void *p, const uint32_t *w) { *(uint2 *)p = make_uint2(w[0], w[1]); }
};
template <> struct RawSt<16> {
    __device__ __forceinline__ static void st(void *p, const uint32_t *w) {
        *(uint4 *)p = make_uint4(w[0], w[1], w[2], w[3]);
    }
};
template <> struct RawSt<32> {
    __device__ __forceinline__ static void st(void *p, const uint32_t *w) {
        RawSt<16>::st(p, w);
        RawSt<16>::st((char *)p + 16, w + 4);
    }
};
template <> struct RawSt<64> {
    __device__ __forceinline__ static void st(void *p, const uint32_t *w) {
        RawSt<32>::st(p, w);
        RawSt<32>::st((char *)p + 32, w + 8);
    }
};

// word <-> complex conversion
template <typename S> struct Conv;
template <> struct Conv<double> {
    static constexpr int W = 4;  // 32-bit words per complex
    __device__ __forceinline__ static cx<double> get(const uint32_t *w) {
        double r = __hiloint2double((int)w[1], (int)w[0]);
        double i = __hiloint2double((int)w[3], (int)w[2]);
        return mk(r, i);
    }
    __device__ __forceinline__ static void put(cx<double> z, uint32_t *w) {
        w[0] = (uint32_t)__double2loint(z.re); w[1] = (uint32_t)__double2hiint(z.re);
        w[2] = (uint32_t)__double2loint(z.im); w[3] = (uint32_t)__double2hiint(z.im);
    }
};
template <> struct Conv<float> {
    static constexpr int W = 2;
    __device__ __forceinline__ static cx<float> get(const uint32_t *w) {
        return mk(__uint_as_float(w[0]), __uint_as_float(w[1]));
    }
    __device__ __forceinline__ static void put(cx<float> z, uint32_t *w) {
        w[0] = __float_as_uint(z.re); w[1] = __float_as_uint(z.im);
    }
};
template <> struct Conv<f32p> : Conv<float> {};  // unpaired data (links) in f32p-typed buffers
template <> struct Conv<bf16> {
    static constexpr int W = 1;
    __device__ __forceinline__ static cx<float> get(const uint32_t *w) {
        __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(w);
        float2 f = __bfloat1622float2(b);
        return mk(f.x, f.y);
    }
    __device__ __forceinline__ static void put(cx<float> z, uint32_t *w) {
        __nv_bfloat162 b = __floats2bfloat162_rn(z.re, z.im);
        *reinterpret_cast<__nv_bfloat162 *>(w) = b;
    }
};

// Paired FP32 layout (f32p): R = 1 reads or writes its own member of a group
// (two 4-byte accesses), even R whole groups (16-byte accesses; the first
// right-hand side must be even).
template <int R, bool NC>
__device__ __forceinline__ void ld_paired(const float *p, cx<float> (&v)[R]) {
    if constexpr (R == 1) {
        const int m = (int)((reinterpret_cast<uintptr_t>(p) >> 3) & 1);
        const float *g = p - 2 * m;
        v[0] = NC ? mk(__ldg(g + m), __ldg(g + 2 + m)) : mk(g[m], g[2 + m]);
    } else {
        static_assert(R % 2 == 0, "paired layout: R = 1 or even");
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const float4 q = NC ? __ldg(reinterpret_cast<const float4 *>(p) + k) : reinterpret_cast<const float4 *>(p)[k];
            v[2 * k] = mk(q.x, q.z);
            v[2 * k + 1] = mk(q.y, q.w);
        }
    }
}
template <int R>
__device__ __forceinline__ void st_paired(float *p, const cx<float> (&v)[R]) {
    if constexpr (R == 1) {
        const int m = (int)((reinterpret_cast<uintptr_t>(p) >> 3) & 1);
        float *g = p - 2 * m;
        g[m] = v[0].re;
        g[2 + m] = v[0].im;
    } else {
        static_assert(R % 2 == 0, "paired layout: R = 1 or even");
#pragma unroll
        for (int k = 0; k < R / 2; ++k)
            reinterpret_cast<float4 *>(p)[k] = make_float4(v[2 * k].re, v[2 * k + 1].re, v[2 * k].im, v[2 * k + 1].im);
    }
}

// Load / store R consecutive complex values of storage type S.
template <typename S, int R, bool NC>
__device__ __forceinline__ void ld_pack(const S *p, cx<typename Real<S>::type> (&v)[R]) {
    if constexpr (IsPaired<S>::v) {
        ld_paired<R, NC>(reinterpret_cast<const float *>(p), v);
        return;
    }
    constexpr int NB = R * cbytes<S>();
    uint32_t w[NB / 4];
    RawLd<NB, NC>::ld(p, w);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = Conv<S>::get(w + r * Conv<S>::W);
}
template <typename S, int R>
__device__ __forceinline__ void st_pack(S *p, const cx<typename Real<S>::type> (&v)[R]) {
    if constexpr (IsPaired<S>::v) {
        st_paired<R>(reinterpret_cast<float *>(p), v);
        return;
    }
    constexpr int NB = R * cbytes<S>();
    uint32_t w[NB / 4];
#pragma unroll
    for (int r = 0; r < R; ++r) Conv<S>::put(v[r], w + r * Conv<S>::W);
    RawSt<NB>::st(p, w);
}

// One complex of a link (read-only path).
template <typename S>
__device__ __forceinline__ cx<typename Real<S>::type> ld_link(const S *p) {
    uint32_t w[cbytes<S>() / 4];
    RawLd<cbytes<S>(), true>::ld(p, w);
    return Conv<S>::get(w);
}

// ----------------------------------------------------------------------------
// geometry
// ----------------------------------------------------------------------------
struct Geom {
    int L[4];       // Lx, Ly, Lz, T
    int stride[4];  // 1, Lx, Lx*Ly, Lx*Ly*Lz
    int Vh;         // sites per parity
    int V3h;        // sites per parity per timeslice
    int t_bc;       // +1 or -1
};

struct Site {
    int c[4];
    int i;  // lexicographic index
};

__device__ __forceinline__ Site decode(uint32_t packed, const Geom &g) {
    Site s;
    s.c[0] = packed & 0xff;
    s.c[1] = (packed >> 8) & 0xff;
    s.c[2] = (packed >> 16) & 0xff;
    s.c[3] = (packed >> 24) & 0xff;
    s.i = s.c[0] + g.stride[1] * s.c[1] + g.stride[2] * s.c[2] + g.stride[3] * s.c[3];
    return s;
}

// checkerboard index of the neighbour x + mu (fwd) or x - mu
__device__ __forceinline__ int nbr_fwd(const Site &s, const Geom &g, int mu) {
    int i = s.i + g.stride[mu];
    if (s.c[mu] == g.L[mu] - 1) i -= g.L[mu] * g.stride[mu];
    return i >> 1;
}
__device__ __forceinline__ int nbr_bwd(const Site &s, const Geom &g, int mu) {
    int i = s.i - g.stride[mu];
    if (s.c[mu] == 0) i += g.L[mu] * g.stride[mu];
    return i >> 1;
}

// ----------------------------------------------------------------------------
// block reduction of per-thread values v[R][NV] over threads with the same
// right-hand-side group g = (global thread index) mod G, G a power of two that
// divides blockDim.x (so g = threadIdx.x mod G).  Writes
// partials[blockIdx.x][g*R + rr][v] as double2, in a fixed order.
// G <= 32: lanes l and l ^ off (off >= G) share g, reduce with shuffles first.
// G  > 32: every lane of a warp has its own g; warps are combined in shared memory.
// smem must hold (blockDim.x/32) * min(G, 32) * R * NV cx<T>.
// ----------------------------------------------------------------------------
template <int R, int NV, typename T>
__device__ __forceinline__ void block_reduce(cx<T> (&v)[R][NV], int G, int N, double2 *partials, void *smem_raw) {
    cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    const int GW = G < 32 ? G : 32;  // distinct groups per warp
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        if (off < G) break;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                v[r][k].re += shfl_xor(v[r][k].re, off);
                v[r][k].im += shfl_xor(v[r][k].im, off);
            }
    }
    if (lane < GW) {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k = 0; k < NV; ++k) sm[((warp * GW + lane) * R + r) * NV + k] = v[r][k];
    }
    __syncthreads();
    const int nout = G * R * NV;  // == N * NV
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const int k = o % NV;
        const int rr = (o / NV) % R;
        const int gg = o / (NV * R);
        const int l = gg % GW;  // lane holding group gg
        double re = 0.0, im = 0.0;
        for (int w = 0; w < nwarp; ++w) {
            if (((w * 32) % G) != gg - l) continue;  // warp w's lanes hold groups (32w .. 32w+31) mod G
            cx<T> z = sm[((w * GW + l) * R + rr) * NV + k];
            re += (double)z.re;
            im += (double)z.im;
        }
        partials[((size_t)blockIdx.x * N + gg * R + rr) * NV + k] = make_double2(re, im);
    }
}

}  // namespace dl
