// Wilson hop on the paired FP32 layout (f32p) with packed FP32 arithmetic
// (kernel kind 7).
//
// A thread owns one output site and two right-hand sides r0, r0 + 1.  In the
// paired layout one 16-byte load of a field component gives the real parts of
// both right-hand sides as one FP32 pair and their imaginary parts as another,
// so every step of the hop is the same operation on both members of a pair:
// one FFMA2 / FADD2 instruction does the work of two FFMA / FADD, with no
// register moves (multiplying by i only exchanges which pair plays the real
// part).  The links come as quads (Re U, Re U, Im U, Im U) (gauge8d_kernel), a
// pair operand each.  The spin projection, SU(3) product and reconstruction
// follow the scalar kernel (load_project, su3_mul, reconstruct in hop.cuh)
// operation by operation; a subtraction a - b is the FFMA2 b * (-1) + a, which
// rounds the same way.
#pragma once

#include "hop.cuh"

namespace dl {

struct P2 {  // two right-hand sides of one complex component
    float2 re, im;
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <bool NC>
__device__ __forceinline__ P2 ld_p2(const float *p) {
    const float4 q = NC ? __ldg(reinterpret_cast<const float4 *>(p)) : *reinterpret_cast<const float4 *>(p);
    P2 v;
    v.re = make_float2(q.x, q.y);
    v.im = make_float2(q.z, q.w);
    return v;
}
__device__ __forceinline__ void st_p2(float *p, const P2 &v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
}
// a + s i b and a - s i b as pairs, s = +1:  i b = (-b.im, b.re)
__device__ __forceinline__ P2 p2_add(const P2 &a, const P2 &b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ P2 p2_sub(const P2 &a, const P2 &b) { return {sub2(a.re, b.re), sub2(a.im, b.im)}; }
__device__ __forceinline__ P2 p2_add_i(const P2 &a, const P2 &b) { return {sub2(a.re, b.im), add2(a.im, b.re)}; }
__device__ __forceinline__ P2 p2_sub_i(const P2 &a, const P2 &b) { return {add2(a.re, b.im), sub2(a.im, b.re)}; }

// One hop direction: acc += (1 + SG gamma_mu-part) V h, V = U (DAG false) or U^dag.
// GL: src and lk are global memory (read-only path); else shared memory.
template <int MU, int SG, bool DAG, bool GL = true>
__device__ __forceinline__ void hop_dir_pair(const float *src, size_t N, const float4 *lk, P2 (&acc)[12]) {
    // ---- load and project (load_project): h[a] spin 0, h[3 + a] spin 1
    P2 h[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const P2 p0 = ld_p2<GL>(src + (size_t)a * N * 2), p1 = ld_p2<GL>(src + (size_t)(3 + a) * N * 2);
        const P2 p2 = ld_p2<GL>(src + (size_t)(6 + a) * N * 2), p3 = ld_p2<GL>(src + (size_t)(9 + a) * N * 2);
        if (MU == 0) {
            h[a] = SG > 0 ? p2_add_i(p0, p3) : p2_sub_i(p0, p3);
            h[3 + a] = SG > 0 ? p2_add_i(p1, p2) : p2_sub_i(p1, p2);
        } else if (MU == 1) {
            h[a] = SG > 0 ? p2_sub(p0, p3) : p2_add(p0, p3);
            h[3 + a] = SG > 0 ? p2_add(p1, p2) : p2_sub(p1, p2);
        } else if (MU == 2) {
            h[a] = SG > 0 ? p2_add_i(p0, p2) : p2_sub_i(p0, p2);
            h[3 + a] = SG > 0 ? p2_sub_i(p1, p3) : p2_add_i(p1, p3);
        } else {
            h[a] = SG > 0 ? p2_add(p0, p2) : p2_sub(p0, p2);
            h[3 + a] = SG > 0 ? p2_add(p1, p3) : p2_sub(p1, p3);
        }
    }
    // ---- the negated part each product needs: -Im h (U h) or -Re h (U^dag h)
    float2 hn[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) hn[k] = neg2(DAG ? h[k].re : h[k].im);
    // ---- w = V h per output colour a (su3_mul), reconstructed at once (reconstruct)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P2 w[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            float2 wr = make_float2(0.f, 0.f), wi = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float4 q = GL ? __ldg(lk + (DAG ? b * 3 + a : a * 3 + b)) : lk[DAG ? b * 3 + a : a * 3 + b];
                const float2 ur = make_float2(q.x, q.y), ui = make_float2(q.z, q.w);
                const P2 &hb = h[3 * s + b];
                if (!DAG) {  // cmac: re += Re u Re h - Im u Im h, im += Re u Im h + Im u Re h
                    wr = fma2(ur, hb.re, wr);
                    wr = fma2(ui, hn[3 * s + b], wr);
                    wi = fma2(ur, hb.im, wi);
                    wi = fma2(ui, hb.re, wi);
                } else {     // cjmac: re += Re u Re h + Im u Im h, im += Re u Im h - Im u Re h
                    wr = fma2(ur, hb.re, wr);
                    wr = fma2(ui, hb.im, wr);
                    wi = fma2(ur, hb.im, wi);
                    wi = fma2(ui, hn[3 * s + b], wi);
                }
            }
            w[s].re = wr;
            w[s].im = wi;
        }
        const P2 &w0 = w[0], &w1 = w[1];
        acc[a] = p2_add(acc[a], w0);
        acc[3 + a] = p2_add(acc[3 + a], w1);
        // lower spins = SG X^dag w; -i w = (w.im, -w.re), i w = (-w.im, w.re)
        if (MU == 0) {  // (-i w1, -i w0)
            acc[6 + a] = SG > 0 ? p2_sub_i(acc[6 + a], w1) : p2_add_i(acc[6 + a], w1);
            acc[9 + a] = SG > 0 ? p2_sub_i(acc[9 + a], w0) : p2_add_i(acc[9 + a], w0);
        } else if (MU == 1) {  // (w1, -w0)
            acc[6 + a] = SG > 0 ? p2_add(acc[6 + a], w1) : p2_sub(acc[6 + a], w1);
            acc[9 + a] = SG > 0 ? p2_sub(acc[9 + a], w0) : p2_add(acc[9 + a], w0);
        } else if (MU == 2) {  // (-i w0, i w1)
            acc[6 + a] = SG > 0 ? p2_sub_i(acc[6 + a], w0) : p2_add_i(acc[6 + a], w0);
            acc[9 + a] = SG > 0 ? p2_add_i(acc[9 + a], w1) : p2_sub_i(acc[9 + a], w1);
        } else {  // (w0, w1)
            acc[6 + a] = SG > 0 ? p2_add(acc[6 + a], w0) : p2_sub(acc[6 + a], w0);
            acc[9 + a] = SG > 0 ? p2_add(acc[9 + a], w1) : p2_sub(acc[9 + a], w1);
        }
    }
}

template <int MU>
__device__ __forceinline__ void hop_mu_pair(const HopArgs &A, const Site &st, int cb, int r0, size_t N,
                                            P2 (&acc)[12]) {
    const float *in = reinterpret_cast<const float *>(A.in);
    const float4 *lk = A.gauge8d + (((size_t)A.p * A.g.Vh + cb) * 8 + 2 * MU) * 9;
    // forward: (1 - g_mu) U_mu(x) psi(x + mu); backward: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)
    hop_dir_pair<MU, -1, false>(in + ((size_t)nbr_fwd(st, A.g, MU) * 12 * N + r0) * 2, N, lk, acc);
    hop_dir_pair<MU, +1, true>(in + ((size_t)nbr_bwd(st, A.g, MU) * 12 * N + r0) * 2, N, lk + 9, acc);
}

// conj(a) b accumulated as cjmac does, on pairs; an = -a.im
__device__ __forceinline__ void cj_pair(float2 &dr, float2 &di, const P2 &a, float2 an, const P2 &b) {
    dr = fma2(a.re, b.re, dr);
    dr = fma2(a.im, b.im, dr);
    di = fma2(a.re, b.im, di);
    di = fma2(an, b.re, di);
}

template <int RED> struct PairNV {
    static constexpr int n = RedCount<RED>::n > 0 ? RedCount<RED>::n : 1;
};

// out = c D in (PLAIN) or y + c D in (XPAY) at site cb for the two right-hand
// sides r0, r0 + 1, with the reductions of hop_body accumulated on pairs.
template <int MODE, int RED>
__device__ __forceinline__ void epilogue_pair(const HopArgs &A, int cb, int r0, size_t N, float2 c2,
                                              const P2 (&acc)[12], float2 (&dr)[PairNV<RED>::n],
                                              float2 (&di)[PairNV<RED>::n]) {
    const size_t base = ((size_t)cb * 12 * N + r0) * 2;
    float *out = reinterpret_cast<float *>(A.out);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const size_t off = base + (size_t)c * N * 2;
        P2 o, yv;
        if (MODE == MODE_XPAY || RED == RED_BICG) yv = ld_p2<true>(reinterpret_cast<const float *>(A.y) + off);
        if (MODE == MODE_PLAIN) {
            o.re = __fmul2_rn(c2, acc[c].re);
            o.im = __fmul2_rn(c2, acc[c].im);
        } else {  // MODE_XPAY: y + c D in
            o.re = fma2(c2, acc[c].re, yv.re);
            o.im = fma2(c2, acc[c].im, yv.im);
        }
        st_p2(out + off, o);
        if (RED == RED_R0DOT || RED == RED_BICG) {
            const P2 rh = ld_p2<true>(reinterpret_cast<const float *>(A.rhat) + off);
            const float2 rhn = neg2(rh.im);
            if (RED == RED_R0DOT) {
                cj_pair(dr[0], di[0], rh, rhn, o);
            } else {
                const float2 on = neg2(o.im), yn = neg2(yv.im);
                cj_pair(dr[0], di[0], o, on, yv);   // <t, s>
                cj_pair(dr[1], di[1], o, on, o);    // <t, t>
                cj_pair(dr[2], di[2], rh, rhn, yv); // <rhat, s>
                cj_pair(dr[3], di[3], rh, rhn, o);  // <rhat, t>
                cj_pair(dr[4], di[4], yv, yn, yv);  // <s, s>
            }
        } else if (RED == RED_NORM) {
            cj_pair(dr[0], di[0], o, neg2(o.im), o);
        }
    }
}

// The per-right-hand-side sums of the block into the partials (block_reduce).
template <int NV>
__device__ __forceinline__ void reduce_pair(const HopArgs &A, int G, int N, const float2 (&dr)[NV],
                                            const float2 (&di)[NV], void *scratch) {
    cx<float> red[2][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        red[0][k] = mk(dr[k].x, di[k].x);
        red[1][k] = mk(dr[k].y, di[k].y);
    }
    block_reduce<2, NV, float>(red, G, N, A.partials, scratch);
}

// The paired-layout hop with the epilogues of hop_body (PLAIN, XPAY; reductions
// R0DOT, BICG, NORM).  A.N even; A.gauge8d holds the link quads.
template <int MODE, int RED, int NC>
__device__ __forceinline__ void hop_body_pair(const HopArgs &A) {
    constexpr int NV = PairNV<RED>::n;
    extern __shared__ __align__(128) unsigned char smem[];
    const int NN = NC ? NC : A.N;
    const int G = NN / 2;  // threads per site: a power of two dividing 32
    const int lgG = __ffs(G) - 1;
    const size_t N = (size_t)NN;
    const int total = (A.cb_end - A.cb_begin) << lgG;
    const float cD = (float)A.c;
    const float2 c2 = make_float2(cD, cD);
    float2 dr[NV], di[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) dr[k] = di[k] = make_float2(0.f, 0.f);
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (A.act && idx < total) {  // the thread's two right-hand sides are the same at every site
        const int r0 = (idx & (G - 1)) * 2;
        if (__ldg(A.act + (size_t)r0 * A.act_stride) == 0 && __ldg(A.act + (size_t)(r0 + 1) * A.act_stride) == 0)
            idx = total;  // both have stopped
    }
    for (; idx < total; idx += gridDim.x * blockDim.x) {
        const int cb = A.cb_begin + (idx >> lgG);
        const int r0 = (idx & (G - 1)) * 2;
        const Site st = decode(__ldg(A.coords + (size_t)A.p * A.g.Vh + cb), A.g);
        P2 acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c].re = acc[c].im = make_float2(0.f, 0.f);
        hop_mu_pair<0>(A, st, cb, r0, N, acc);
        hop_mu_pair<1>(A, st, cb, r0, N, acc);
        hop_mu_pair<2>(A, st, cb, r0, N, acc);
        hop_mu_pair<3>(A, st, cb, r0, N, acc);
        epilogue_pair<MODE, RED>(A, cb, r0, N, c2, acc, dr, di);
    }
    if (RED != RED_NONE) reduce_pair<NV>(A, G, NN, dr, di, smem);
}

template <int MODE, int RED, int NC = 0>
__global__ void __launch_bounds__(256) hop_kernel_pair(HopArgs A) {
    hop_body_pair<MODE, RED, NC>(A);
}
// Kind 8: the same with at most 128 registers per thread (four 128-thread
// blocks per SM instead of three), a few spilled values.
template <int MODE, int RED, int NC = 0>
__global__ void __maxnreg__(128) hop_kernel_pair_cap(HopArgs A) {
    hop_body_pair<MODE, RED, NC>(A);
}

}  // namespace dl
