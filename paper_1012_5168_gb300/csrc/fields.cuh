// Field-level kernels around the solver: layout conversion, gauge reordering,
// complex Z2 / point sources, Gaussian smearing, loop contraction and the
// per-timeslice Gamma-weighted spin matrices of the loop gradients.
#pragma once

#include "common.cuh"

namespace dl {

// ---------------------------------------------------------------------------
// canonical [rhs][V][12] complex128  <->  EO tile [2][Vh][12][N] complex128
// thread = (parity, cb, j); cb restricted to [cb0, cb1) in both parities.
// ---------------------------------------------------------------------------
struct ConvArgs {
    const uint32_t *coords;
    Geom g;
    int cb0, cb1;
    int n;       // right-hand sides converted (j < n)
    int N;       // layout width
    int gamma5;  // negate spins 2, 3
    const int *tcol;  // if set: column j covers timeslice tcol[j] only (cb range [cb0, cb1) inside it)
};
__device__ __forceinline__ int col_offset(const int *tcol, int j, int n, const Geom &g) {
    return (tcol && j < n) ? tcol[j] * g.V3h : 0;
}

static __global__ void canon_to_eo_kernel(ConvArgs a, const double *canon, double *eo) {
    const int nsite = a.cb1 - a.cb0;
    const long total = 2L * nsite * a.N;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % a.N);
        const long sp = idx / a.N;
        const int p = (int)(sp / nsite);
        const int cb = a.cb0 + (int)(sp % nsite) + col_offset(a.tcol, j, a.n, a.g);
        const Site st = decode(a.coords[(size_t)p * a.g.Vh + cb], a.g);
        double *dst = eo + ((size_t)p * a.g.Vh + cb) * 12 * a.N * 2 + (size_t)j * 2;
        if (j >= a.n) {
            for (int c = 0; c < 12; ++c) *(double2 *)(dst + (size_t)c * a.N * 2) = make_double2(0.0, 0.0);
            continue;
        }
        const double2 *src = (const double2 *)(canon + ((size_t)j * 2 * a.g.Vh + st.i) * 24);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 v = src[c];
            if (a.gamma5 && c >= 6) { v.x = -v.x; v.y = -v.y; }
            *(double2 *)(dst + (size_t)c * a.N * 2) = v;
        }
    }
}

static __global__ void eo_to_canon_kernel(ConvArgs a, const double *eo, double *canon) {
    const int nsite = a.cb1 - a.cb0;
    const long total = 2L * nsite * a.n;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % a.n);
        const long sp = idx / a.n;
        const int p = (int)(sp / nsite);
        const int cb = a.cb0 + (int)(sp % nsite) + col_offset(a.tcol, j, a.n, a.g);
        const Site st = decode(a.coords[(size_t)p * a.g.Vh + cb], a.g);
        const double *src = eo + ((size_t)p * a.g.Vh + cb) * 12 * a.N * 2 + (size_t)j * 2;
        double2 *dst = (double2 *)(canon + ((size_t)j * 2 * a.g.Vh + st.i) * 24);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 v = *(const double2 *)(src + (size_t)c * a.N * 2);
            if (a.gamma5 && c >= 6) { v.x = -v.x; v.y = -v.y; }
            dst[c] = v;
        }
    }
}

// Tiled conversions for whole-lattice batches (cb range [0, Vh), no per-column
// timeslices) of width N >= 16.  A block moves one tile: the cb range
// [cb0, cb0 + TS) of both parities, TS = 64 / N, which holds exactly the
// lexicographic sites [2 cb0, 2 cb0 + 2 TS).  The EO side of a tile is one
// contiguous run [TS][12][N] per parity and the canonical side one contiguous
// run [2 TS][12] per right-hand side, so both sides are read and written in
// coalesced runs, through shared memory [2][TS][12][N + 1] complex (the pad
// keeps the column reads apart in the banks).  Site i = 2 cb0 + o has the
// parity of o + y + z + t, since its x has the parity of i (L_x even).
constexpr int CONV_TILE = 64;  // TS N
__device__ __forceinline__ int lex_parity(int i, const Geom &g) {
    const int R = i / g.L[0];                   // x-row: y + Ly (z + Lz t)
    const int R2 = R / g.L[1], R3 = R2 / g.L[2];  // z + Lz t, t
    return (i + R + R2 + R3) & 1;                 // x + y + z + t mod 2 (the extents are even)
}
static __global__ void __launch_bounds__(256) eo_to_canon_tiled(ConvArgs a, const double *eo, double *canon) {
    extern __shared__ double2 cvt[];
    const int N = a.N, TS = CONV_TILE / N, NP = N + 1, run = TS * 12 * N, per = 2 * TS * 12;
    const int V = 2 * a.g.Vh;
    for (int tile = blockIdx.x; tile < a.g.Vh / TS; tile += gridDim.x) {
        const int cb0 = tile * TS;
        for (int k = threadIdx.x; k < 2 * run; k += blockDim.x) {
            const int p = k / run, r = k - p * run;  // r = (s 12 + c) N + j
            cvt[(p * TS * 12 + r / N) * NP + r % N] =
                reinterpret_cast<const double2 *>(eo)[((size_t)p * a.g.Vh + cb0) * 12 * N + r];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < a.n * per; k += blockDim.x) {
            const int j = k / per, q = k - j * per, o = q / 12, c = q - o * 12;
            const int i = 2 * cb0 + o, p = lex_parity(i, a.g);
            double2 v = cvt[(p * TS * 12 + (o >> 1) * 12 + c) * NP + j];
            if (a.gamma5 && c >= 6) { v.x = -v.x; v.y = -v.y; }
            reinterpret_cast<double2 *>(canon)[((size_t)j * V + i) * 12 + c] = v;
        }
        __syncthreads();
    }
}
static __global__ void __launch_bounds__(256) canon_to_eo_tiled(ConvArgs a, const double *canon, double *eo) {
    extern __shared__ double2 cvt[];
    const int N = a.N, TS = CONV_TILE / N, NP = N + 1, run = TS * 12 * N, per = 2 * TS * 12;
    const int V = 2 * a.g.Vh;
    for (int tile = blockIdx.x; tile < a.g.Vh / TS; tile += gridDim.x) {
        const int cb0 = tile * TS;
        for (int k = threadIdx.x; k < N * per; k += blockDim.x) {
            const int j = k / per, q = k - j * per, o = q / 12, c = q - o * 12;
            const int i = 2 * cb0 + o, p = lex_parity(i, a.g);
            double2 v = make_double2(0.0, 0.0);  // columns j >= n are zero
            if (j < a.n) {
                v = reinterpret_cast<const double2 *>(canon)[((size_t)j * V + i) * 12 + c];
                if (a.gamma5 && c >= 6) { v.x = -v.x; v.y = -v.y; }
            }
            cvt[(p * TS * 12 + (o >> 1) * 12 + c) * NP + j] = v;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * run; k += blockDim.x) {
            const int p = k / run, r = k - p * run;
            reinterpret_cast<double2 *>(eo)[((size_t)p * a.g.Vh + cb0) * 12 * N + r] =
                cvt[(p * TS * 12 + r / N) * NP + r % N];
        }
        __syncthreads();
    }
}

// gauge: canonical [V][4][3][3] complex128 -> EO [2][Vh][4][9] complex in S
template <typename S>
static __global__ void gauge_reorder_kernel(const uint32_t *coords, Geom g, const double *canon, S *eo) {
    typedef typename Real<S>::type T;
    const int total = 2 * g.Vh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const Site st = decode(coords[idx], g);
        const double2 *src = (const double2 *)(canon + (size_t)st.i * 72);
        S *dst = eo + (size_t)idx * 72;
        for (int k = 0; k < 36; ++k) {
            const double2 v = src[k];
            cx<T> z[1];
            z[0] = mk((T)v.x, (T)v.y);
            st_pack<S, 1>(dst + 2 * k, z);
        }
    }
}

// The packed-arithmetic hop's links: per output site the eight links of its
// hop directions (d = 2 mu: U_mu(x); d = 2 mu + 1: V = U_mu(x - mu)^dag, the
// conjugate transpose taken here), each element V[a][b] stored as the FP32
// quad (Re V, Re V, -Im V, Im V), with the time boundary factor t_bc folded
// into the links of the hops that cross t = T-1 <-> 0.
static __global__ void gauge8q_kernel(const uint32_t *coords, Geom g, const double *canon, float4 *out) {
    const int total = 2 * g.Vh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const Site st = decode(coords[idx], g);
        for (int d = 0; d < 8; ++d) {
            const int mu = d >> 1;
            int src = st.i;
            if (d & 1) {
                src = st.i - g.stride[mu];
                if (st.c[mu] == 0) src += g.L[mu] * g.stride[mu];
            }
            const double2 *u = (const double2 *)(canon + ((size_t)src * 4 + mu) * 18);
            float4 *dst = out + ((size_t)idx * 8 + d) * 9;
            const double sg = (mu == 3 && g.t_bc < 0 && st.c[3] == ((d & 1) ? 0 : g.L[3] - 1)) ? -1.0 : 1.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const double2 z = (d & 1) ? make_double2(u[b * 3 + a].x, -u[b * 3 + a].y) : u[a * 3 + b];
                    const float re = (float)(sg * z.x), im = (float)(sg * z.y);
                    dst[a * 3 + b] = make_float4(re, re, -im, im);
                }
        }
    }
}

// gauge, site-major with all eight links of a site in one row: for site x of
// parity p, row d = 2 mu holds U_mu(x) and row d = 2 mu + 1 holds U_mu(x - mu)
// (not conjugated), the time boundary factor t_bc folded into the links of
// the hops that cross t = T-1 <-> 0.  Out: [2][Vh][8][9] complex in S.
template <typename S>
__global__ void gauge8_kernel(const uint32_t *coords, Geom g, const double *canon, S *out) {
    typedef typename Real<S>::type T;
    const int total = 2 * g.Vh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const Site st = decode(coords[idx], g);
        for (int d = 0; d < 8; ++d) {
            const int mu = d >> 1;
            int src = st.i;
            if (d & 1) {
                src = st.i - g.stride[mu];
                if (st.c[mu] == 0) src += g.L[mu] * g.stride[mu];
            }
            const double2 *u = (const double2 *)(canon + ((size_t)src * 4 + mu) * 18);
            S *dst = out + ((size_t)idx * 8 + d) * 18;
            // the time boundary factor of the quark fields rides on the link of the hop that crosses it
            const double sg = (mu == 3 && g.t_bc < 0 && st.c[3] == ((d & 1) ? 0 : g.L[3] - 1)) ? -1.0 : 1.0;
            for (int k = 0; k < 9; ++k) {
                cx<T> z[1];
                z[0] = mk((T)(sg * u[k].x), (T)(sg * u[k].y));
                st_pack<S, 1>(dst + 2 * k, z);
            }
        }
    }
}

// The paired-layout hop's links (kind 7): the site-major rows of gauge8_kernel
// (U_mu(x) for d = 2 mu, U_mu(x - mu) for d = 2 mu + 1, time boundary factor
// folded in) with every FP32 element stored as the quad (Re U, Re U, Im U, Im U),
// so that each half is an FP32 pair operand for two right-hand sides at once.
static __global__ void gauge8d_kernel(const uint32_t *coords, Geom g, const double *canon, float4 *out) {
    const int total = 2 * g.Vh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const Site st = decode(coords[idx], g);
        for (int d = 0; d < 8; ++d) {
            const int mu = d >> 1;
            int src = st.i;
            if (d & 1) {
                src = st.i - g.stride[mu];
                if (st.c[mu] == 0) src += g.L[mu] * g.stride[mu];
            }
            const double2 *u = (const double2 *)(canon + ((size_t)src * 4 + mu) * 18);
            float4 *dst = out + ((size_t)idx * 8 + d) * 9;
            const double sg = (mu == 3 && g.t_bc < 0 && st.c[3] == ((d & 1) ? 0 : g.L[3] - 1)) ? -1.0 : 1.0;
            for (int k = 0; k < 9; ++k) {
                const float re = (float)(sg * u[k].x), im = (float)(sg * u[k].y);
                dst[k] = make_float4(re, re, im, im);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11) and complex Z2 sources
// ---------------------------------------------------------------------------
struct PhiloxOut {
    uint64_t v[4];
};

__device__ __forceinline__ PhiloxOut philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                                   uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    PhiloxOut o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

struct SourceArgs {
    const uint32_t *coords;
    Geom g;
    uint64_t seed;
    int64_t noise_first;
    int n_noise;
    int dil_spin, dil_colour, dil_eo, dil_cubic, dil_time;  // class counts (1 if absent); time flag
    int t0;
    int k_first, k_count;  // classes k_first .. k_first+k_count-1 of each noise vector are written
};

// thread = (rhs, p, cb): one site of one diluted source, canonical output
// One complex value of a canonical field in output storage O (double2: complex128,
// float2: complex64, bf16 pairs); the value is rounded from FP64 (to float first
// for BF16, the way the solver rounds its fields).
template <typename O> __device__ __forceinline__ void put_cx(O *dst, double re, double im);
template <> __device__ __forceinline__ void put_cx<double2>(double2 *dst, double re, double im) {
    *dst = make_double2(re, im);
}
template <> __device__ __forceinline__ void put_cx<float2>(float2 *dst, double re, double im) {
    *dst = make_float2((float)re, (float)im);
}
template <> __device__ __forceinline__ void put_cx<__nv_bfloat162>(__nv_bfloat162 *dst, double re, double im) {
    *dst = __floats2bfloat162_rn((float)re, (float)im);
}

template <typename O>
static __global__ void z2_source_kernel(SourceArgs a, O *out) {
    const long nsite = 2L * a.g.Vh;
    const long total = (long)a.n_noise * a.k_count * nsite;
    const double s2 = sqrt(0.5);  // 1/sqrt(2), rounded once
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const long rhs = idx / nsite;
        const int sp = (int)(idx % nsite);
        const int j = (int)(rhs / a.k_count);
        const int k = a.k_first + (int)(rhs % a.k_count);
        const int64_t n = a.noise_first + j;
        const Site st = decode(a.coords[sp], a.g);
        const PhiloxOut b = philox4x64_10((uint64_t)(st.i >> 2), (uint64_t)n, 0, 0, a.seed, 0);
        const uint64_t w = b.v[st.i & 3];
        // class index digits, k = ((ks*C + kc)*E + ke)*Q + kq
        const int kq = k % a.dil_cubic;
        const int ke = (k / a.dil_cubic) % a.dil_eo;
        const int kc = (k / (a.dil_cubic * a.dil_eo)) % a.dil_colour;
        const int ks = k / (a.dil_cubic * a.dil_eo * a.dil_colour);
        bool site_on = true;
        if (a.dil_eo > 1) site_on &= (((st.c[0] + st.c[1] + st.c[2] + st.c[3]) & 1) == ke);
        if (a.dil_cubic > 1) site_on &= (((st.c[0] & 1) + 2 * (st.c[1] & 1) + 4 * (st.c[2] & 1)) == kq);
        if (a.dil_time) {
            const int tn = a.t0 >= 0 ? a.t0 : (int)(n % a.g.L[3]);
            site_on &= (st.c[3] == tn);
        }
        O *dst = out + ((size_t)rhs * 2 * a.g.Vh + st.i) * 12;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const int alpha = c / 3, col = c % 3;
            const bool on = site_on && (a.dil_spin == 1 || alpha == ks) && (a.dil_colour == 1 || col == kc);
            double re = 0.0, im = 0.0;
            if (on) {
                re = ((w >> (2 * c)) & 1) ? -s2 : s2;
                im = ((w >> (2 * c + 1)) & 1) ? -s2 : s2;
            }
            put_cx<O>(dst + c, re, im);
        }
    }
}

// point sources e_s, s = first + j, s = 12 i + c: canonical output, n fields
template <typename O>
static __global__ void point_source_kernel(int64_t first, int n, long V, O *out) {
    const long total = (long)n * V * 12;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const long j = idx / (V * 12);
        const long e = idx % (V * 12);
        put_cx<O>(out + idx, e == first + j ? 1.0 : 0.0, 0.0);
    }
}

// ---------------------------------------------------------------------------
// Gaussian smearing step on EO tile fields, both parities in one launch:
//   out_p = a * in_p + c * H_{p,1-p} in_{1-p},
//   (H psi)(x) = sum_{j=x,y,z} [U_j(x) psi(x+j) + U_j(x-j)^dag psi(x-j)]
// thread = (p, cb, rhs) with cb in [cb0, cb1).
// ---------------------------------------------------------------------------
struct SmearArgs {
    const double *in;   // [2][Vh][12][N]
    double *out;
    const double *in2;  // optional second field smeared in the same launch by blockIdx.y = 1
    double *out2;       // (float-float kernel); null: one field
    const double *gauge;  // [2][Vh][4][9] complex128
    const uint32_t *coords;
    Geom g;
    int cb0, cb1, N;
    int n;  // right-hand sides in use (columns j >= n are left untouched)
    double a, c;
    const int *tcol;  // if set: column j is smeared on timeslice tcol[j] only
};

static __global__ void __launch_bounds__(256) smear_kernel(SmearArgs A) {
    const int nsite = A.cb1 - A.cb0;
    const long total = 2L * nsite * A.n;  // only the columns in use
    const size_t half = (size_t)A.g.Vh * 12 * A.N * 2;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % A.n);
        const int sp = (int)(idx / A.n);
        const int p = sp / nsite;
        const int cb = A.cb0 + sp % nsite + col_offset(A.tcol, j, A.n, A.g);
        const Site st = decode(__ldg(A.coords + (size_t)p * A.g.Vh + cb), A.g);
        const double *inn = A.in + (size_t)(1 - p) * half;
        cx<double> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = zero<double>();
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            for (int dir = 0; dir < 2; ++dir) {
                const int nb = dir == 0 ? nbr_fwd(st, A.g, mu) : nbr_bwd(st, A.g, mu);
                const double *up = dir == 0 ? A.gauge + (((size_t)p * A.g.Vh + cb) * 4 + mu) * 18
                                            : A.gauge + (((size_t)(1 - p) * A.g.Vh + nb) * 4 + mu) * 18;
                cx<double> u[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) u[k] = ld_link<double>(up + 2 * k);
                const double *src = inn + (size_t)nb * 12 * A.N * 2 + (size_t)j * 2;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    cx<double> v[3];
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const double2 q = __ldg((const double2 *)(src + (size_t)(3 * s + b) * A.N * 2));
                        v[b] = mk(q.x, q.y);
                    }
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            if (dir == 0) cmac(acc[3 * s + aa], u[aa * 3 + b], v[b]);
                            else cjmac(acc[3 * s + aa], u[b * 3 + aa], v[b]);
                        }
                }
            }
        }
        const double *y = A.in + (size_t)p * half + (size_t)cb * 12 * A.N * 2 + (size_t)j * 2;
        double *o = A.out + (size_t)p * half + (size_t)cb * 12 * A.N * 2 + (size_t)j * 2;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 q = __ldg((const double2 *)(y + (size_t)k * A.N * 2));
            *(double2 *)(o + (size_t)k * A.N * 2) =
                make_double2(A.a * q.x + A.c * acc[k].re, A.a * q.y + A.c * acc[k].im);
        }
    }
}

// ---------------------------------------------------------------------------
// Gaussian smearing in float-float arithmetic (dfloat, common.cuh).  The
// smearing runs on the FP32 pipes, which on GB300 issue about 60 times as fast
// as FP64, while its rounding (~1e-14 relative per step) stays far below the
// tolerance of the loops.  Fields in this format occupy the same 8 bytes per
// real as FP64 and are converted in place before and after the iterations.
// ---------------------------------------------------------------------------
typedef dfloat ff;
struct ffc {
    ff re, im;
};
__device__ __forceinline__ ffc ld_ffc(const double *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    ffc z;
    z.re.hi = v.x;
    z.re.lo = v.y;
    z.im.hi = v.z;
    z.im.lo = v.w;
    return z;
}

// In-place conversion of an EO tile field (both parities, cb range, n of N
// columns) between FP64 and float-float.  to_ff = 1: double -> ff; 0: back.
static __global__ void ff_convert_kernel(double *f, int Vh, int cb0, int cb1, int N, int n, int to_ff,
                                         const int *tcol, int V3h) {
    const long nsite = cb1 - cb0;
    const long total = 2 * nsite * 12 * n;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % n);
        const long q = idx / n;
        const int c = (int)(q % 12);
        const long sp = q / 12;
        const int p = (int)(sp / nsite);
        const int cb = cb0 + (int)(sp % nsite) + (tcol ? tcol[j] * V3h : 0);
        double *e = f + (((size_t)p * Vh + cb) * 12 * N + (size_t)c * N + j) * 2;
        if (to_ff) {
            const ff a = df_from_double(e[0]), b = df_from_double(e[1]);
            *reinterpret_cast<float4 *>(e) = make_float4(a.hi, a.lo, b.hi, b.lo);
        } else {
            const float4 v = *reinterpret_cast<const float4 *>(e);
            ff a, b;
            a.hi = v.x; a.lo = v.y; b.hi = v.z; b.lo = v.w;
            e[0] = (double)a;
            e[1] = (double)b;
        }
    }
}

// Links in float-float: [2][Vh][4][9] complex as (re.hi, re.lo, im.hi, im.lo).
static __global__ void gauge_ff_kernel(const double *g64, float *out, long n_complex) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_complex; i += (long)gridDim.x * blockDim.x) {
        const ff a = df_from_double(g64[2 * i]), b = df_from_double(g64[2 * i + 1]);
        reinterpret_cast<float4 *>(out)[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
}

// One smearing step in float-float (same contract as smear_kernel, fields
// and links in float-float format), with the three colour rows of a site on
// three threads: thread (site, a, j) produces the four spin components of
// colour a.  It holds one link row and one colour vector at a time instead of
// the whole link and the 12-component accumulator, so it needs far fewer
// registers and more warps stay resident; the three threads of a site read the
// same neighbour spinors, which then come from L1.  Two resident blocks per SM
// (up to 128 registers a thread) measured 9% faster than three (85): 0.198
// against 0.217 ms per iteration for 96 fields on one 16^3 timeslice.
static __global__ void __launch_bounds__(256, 2) smear_ff_rows_kernel(SmearArgs A, const float *gauge_ff) {
    const int nsite = A.cb1 - A.cb0;
    const long total = 2L * nsite * 3 * A.n;  // only the columns in use
    const size_t half = (size_t)A.g.Vh * 12 * A.N * 2;
    const ff fa = df_from_double(A.a), fc = df_from_double(A.c);
    const double *__restrict__ fin = blockIdx.y ? A.in2 : A.in;  // the field of this grid row
    double *__restrict__ fout = blockIdx.y ? A.out2 : A.out;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % A.n);
        const long rest = idx / A.n;
        const int a = (int)(rest % 3);
        const int sp = (int)(rest / 3);
        const int p = sp / nsite;
        const int cb = A.cb0 + sp % nsite + col_offset(A.tcol, j, A.n, A.g);
        const Site st = decode(__ldg(A.coords + (size_t)p * A.g.Vh + cb), A.g);
        const double *inn = fin + (size_t)(1 - p) * half;
        cdacc acc[4];  // unnormalised sums (common.cuh), renormalised once at the end
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = cda_zero();
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
#pragma unroll
            for (int dir = 0; dir < 2; ++dir) {
                const int nb = dir == 0 ? nbr_fwd(st, A.g, mu) : nbr_bwd(st, A.g, mu);
                const double *up = reinterpret_cast<const double *>(
                    gauge_ff + (dir == 0 ? (((size_t)p * A.g.Vh + cb) * 4 + mu) * 36
                                         : (((size_t)(1 - p) * A.g.Vh + nb) * 4 + mu) * 36));
                // forward: row a of U; backward: column a of U, conjugated in the product
                cx<ff> u[3];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const ffc w = ld_ffc(up + 2 * (dir == 0 ? a * 3 + b : b * 3 + a));
                    u[b] = mk(w.re, w.im);
                }
                const double *src = inn + (size_t)nb * 12 * A.N * 2 + (size_t)j * 2;
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const ffc v = ld_ffc(src + (size_t)(3 * s + b) * A.N * 2);
                        if (dir == 0) cda_mac<false>(acc[s], u[b], mk(v.re, v.im));
                        else cda_mac<true>(acc[s], u[b], mk(v.re, v.im));
                    }
            }
        }
        const double *y = fin + (size_t)p * half + (size_t)cb * 12 * A.N * 2 + (size_t)j * 2;
        double *o = fout + (size_t)p * half + (size_t)cb * 12 * A.N * 2 + (size_t)j * 2;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int k = 3 * s + a;
            const ffc q = ld_ffc(y + (size_t)k * A.N * 2);
            ffc r;
            r.re = df_add(df_mul(fa, q.re), df_mul(fc, da_norm(acc[s].re)));
            r.im = df_add(df_mul(fa, q.im), df_mul(fc, da_norm(acc[s].im)));
            *reinterpret_cast<float4 *>(o + (size_t)k * A.N * 2) = make_float4(r.re.hi, r.re.lo, r.im.hi, r.im.lo);
        }
    }
}

// ---------------------------------------------------------------------------
// loop contraction: per timeslice t and right-hand side j,
//   S(t)_{beta alpha} = sum_{x in t} sum_a phi_{beta a}(x) conj(eta_{alpha a}(x)),
// grid = (bx, timeslice offset, parity); partials [(tt*2 + p)*nbx + bx][N][16]
// ---------------------------------------------------------------------------
struct ContractArgs {
    const double *eta;  // EO tile [2][Vh][12][N]
    const double *phi;
    Geom g;
    int t_lo;
    int N;
    double2 *partials;
    const int *tcol;  // if set (R = 1, one timeslice slot): column j is contracted on tcol[j]
    int n;
};

template <int R>
static __global__ void __launch_bounds__(128) contract_kernel(ContractArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int p = blockIdx.z;
    const int t = A.t_lo + blockIdx.y;
    const int G = A.N / R;
    const int lgG = __ffs(G) - 1;
    const int cb0 = t * A.g.V3h;
    const int total = A.g.V3h << lgG;
    const size_t half = (size_t)A.g.Vh * 12 * A.N * 2;
    cx<double> acc[R][16];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[r][k] = zero<double>();
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int r0 = (idx & (G - 1)) * R;
        const int cb = cb0 + (idx >> lgG) + (A.tcol ? col_offset(A.tcol, r0, A.n, A.g) - t * A.g.V3h : 0);
        const size_t base = (size_t)p * half + (size_t)cb * 12 * A.N * 2 + (size_t)r0 * 2;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<double> e[R][4], f[R][4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                cx<double> ev[R], fv[R];
                ld_pack<double, R, true>(A.eta + base + (size_t)(3 * s + a) * A.N * 2, ev);
                ld_pack<double, R, true>(A.phi + base + (size_t)(3 * s + a) * A.N * 2, fv);
#pragma unroll
                for (int r = 0; r < R; ++r) { e[r][s] = ev[r]; f[r][s] = fv[r]; }
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int be = 0; be < 4; ++be)
#pragma unroll
                    for (int al = 0; al < 4; ++al) cjmac(acc[r][be * 4 + al], e[r][al], f[r][be]);
        }
    }
    double2 *part = A.partials + ((size_t)(blockIdx.y * 2 + p) * gridDim.x) * A.N * 16;
    // block_reduce writes partials[blockIdx.x][N][16] relative to `part`
    block_reduce<R, 16, double>(acc, G, A.N, part, smem);
}

// final: sum partials over (parity, bx) in fixed order, then L_Gamma(t) =
// sum_{alpha beta} Gamma_{alpha beta} S_{beta alpha}.  out[j][16][T] double2.
// grid = (n_t, n), block = 32.
static __global__ void contract_final_kernel(const double2 *partials, int nbx, int N, int t_lo, int T,
                                      const double2 *gammas /* [16][4][4] */, double2 *out, const int *tcol) {
    const int tt = blockIdx.x;
    const int j = blockIdx.y;
    __shared__ double2 S[16];
    const int lane = threadIdx.x;
    if (lane < 16) {
        double re = 0.0, im = 0.0;
        for (int p = 0; p < 2; ++p)
            for (int b = 0; b < nbx; ++b) {
                const double2 v = partials[(((size_t)(tt * 2 + p) * nbx + b) * N + j) * 16 + lane];
                re += v.x;
                im += v.y;
            }
        S[lane] = make_double2(re, im);  // S[beta*4 + alpha]
    }
    __syncthreads();
    if (lane < 16) {
        double re = 0.0, im = 0.0;
        for (int al = 0; al < 4; ++al)
            for (int be = 0; be < 4; ++be) {
                const double2 gm = gammas[(lane * 4 + al) * 4 + be];
                const double2 s = S[be * 4 + al];
                re += gm.x * s.x - gm.y * s.y;
                im += gm.x * s.y + gm.y * s.x;
            }
        out[((size_t)j * 16 + lane) * T + (tcol ? tcol[j] : t_lo + tt)] = make_double2(re, im);
    }
}

// ---------------------------------------------------------------------------
// Gamma-weighted spin matrices for the loop gradients
//   mode 0: W_{j,t} = sum_G w[j][G][t] G^dag ;  mode 1: W_{j,t} = sum_G conj(w[j][G][t]) G
// then out(x) (+)= W_{j,t(x)} in(x) on canonical fields.
// ---------------------------------------------------------------------------
static __global__ void gamma_weights_kernel(const double2 *w, int n, int T, int mode, const double2 *gammas,
                                     double2 *W /* [n][T][4][4] */) {
    const int total = n * T * 16;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int e = idx % 16;  // row*4 + col of W
        const int t = (idx / 16) % T;
        const int j = idx / (16 * T);
        const int row = e / 4, col = e % 4;
        double re = 0.0, im = 0.0;
        for (int G = 0; G < 16; ++G) {
            const double2 c = w[((size_t)j * 16 + G) * T + t];
            double2 m;
            if (mode == 0) {  // (G^dag)_{row col} = conj(G_{col row})
                const double2 g = gammas[(G * 4 + col) * 4 + row];
                m = make_double2(g.x, -g.y);
                re += c.x * m.x - c.y * m.y;
                im += c.x * m.y + c.y * m.x;
            } else {          // conj(c) G_{row col}
                m = gammas[(G * 4 + row) * 4 + col];
                re += c.x * m.x + c.y * m.y;
                im += c.x * m.y - c.y * m.x;
            }
        }
        W[idx] = make_double2(re, im);
    }
}

static __global__ void apply_spin_matrix_kernel(const double *in, double *out, const double2 *W, int n, long V, int V3,
                                         int T, int accumulate) {
    const long total = (long)n * V * 3;  // thread = (j, site, colour)
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int a = (int)(idx % 3);
        const long js = idx / 3;
        const long i = js % V;
        const long j = js / V;
        const int t = (int)(i / V3);
        const double2 *src = (const double2 *)in + js * 12;
        double2 *dst = (double2 *)out + js * 12;
        const double2 *m = W + ((size_t)j * T + t) * 16;
        double2 v[4];
        for (int s = 0; s < 4; ++s) v[s] = src[3 * s + a];
        for (int r = 0; r < 4; ++r) {
            double re = 0.0, im = 0.0;
            for (int s = 0; s < 4; ++s) {
                const double2 g = m[r * 4 + s];
                re += g.x * v[s].x - g.y * v[s].y;
                im += g.x * v[s].y + g.y * v[s].x;
            }
            if (accumulate) {
                const double2 o = dst[3 * r + a];
                re += o.x;
                im += o.y;
            }
            dst[3 * r + a] = make_double2(re, im);
        }
    }
}

// ---------------------------------------------------------------------------
// exact loops from point-source solutions (EO tile layout): for right-hand
// side j solving e_s (s = first + j = 12 i + 3 alpha + a), add phi_{beta a}(i)
// to S(t_i)_{beta alpha}.  One thread, fixed order (deterministic).
// acc: [T][4][4] double2 (beta*4 + alpha)
// ---------------------------------------------------------------------------
static __global__ void point_diag_kernel(const double *phi_eo, const uint32_t *coords, Geom g, int64_t first, int n, int N,
                                  double2 *acc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    (void)coords;
    const int V3 = 2 * g.V3h;
    for (int j = 0; j < n; ++j) {
        const int64_t s = first + j;
        const int i = (int)(s / 12);
        const int c = (int)(s % 12);
        const int alpha = c / 3, a = c % 3;
        // parity and cb of lexicographic site i
        int rem = i;
        const int x = rem % g.L[0]; rem /= g.L[0];
        const int y = rem % g.L[1]; rem /= g.L[1];
        const int z = rem % g.L[2]; rem /= g.L[2];
        const int t = rem;
        const int p = (x + y + z + t) & 1;
        const int cb = i >> 1;
        const double *site = phi_eo + ((size_t)p * g.Vh + cb) * 12 * N * 2 + (size_t)j * 2;
        for (int beta = 0; beta < 4; ++beta) {
            const double2 v = *(const double2 *)(site + (size_t)(3 * beta + a) * N * 2);
            double2 &o = acc[((size_t)t * 4 + beta) * 4 + alpha];
            o.x += v.x;
            o.y += v.y;
        }
        (void)V3;
    }
}

}  // namespace dl
