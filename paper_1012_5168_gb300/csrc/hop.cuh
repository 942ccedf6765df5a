// Even-odd Wilson hopping term for N right-hand sides.
//
//   (D_{p,1-p} psi)(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x + mu)
//                               + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu) ]
//
// for x of parity p (Sec. 2: the N_f = 2 Wilson matrix M = 1 - kappa D; the
// even-odd split of D is the Schur-complement preconditioning of the solver).
//
// Spin structure.  In the chiral (DeGrand-Rossi) basis every g_mu has the block
// form [[0, X_mu], [X_mu^dag, 0]] with X_1 = i sigma_x, X_2 = -i sigma_y,
// X_3 = i sigma_z, X_4 = 1 (all unitary).  Hence for sign s = -1 (forward,
// 1 - g_mu) or s = +1 (backward, 1 + g_mu):
//
//   (1 + s g_mu) psi = [ h ; s X_mu^dag h ],   h = psi_up + s X_mu psi_down,
//
// so one hop needs the two-spinor h (6 complex), two SU(3) products (U or
// U^dag on h) and a reconstruction of the lower two spins with entries of X
// that are 0, +-1, +-i.  This halves the colour work of a naive 4x4 spin
// product.  Each thread handles one site and R right-hand sides, loading each
// link once and reusing it for its R right-hand sides; the N right-hand sides
// of a site are spread over N/R neighbouring threads, so the link load of a
// warp is a broadcast.
//
// Epilogues (MODE): out = c*D in (PLAIN), out = y + c*D in (XPAY),
// out = z - y - c*D in (RESID).  Reductions (RED), per right-hand side, in the
// arithmetic precision and then FP64 across warps and blocks:
//   R0DOT: <rhat, out>;  BICG: <out, y>, <out, out>, <rhat, y>, <rhat, out>, <y, y>;
//   NORM: <out, out>   (<a, b> = sum conj(a) b).
#pragma once

#include "clover.cuh"
#include "common.cuh"

namespace dl {

enum { MODE_PLAIN = 0, MODE_XPAY = 1, MODE_RESID = 2 };
enum { RED_NONE = 0, RED_R0DOT = 1, RED_BICG = 2, RED_NORM = 3 };

template <int RED> struct RedCount { static constexpr int n = 0; };
template <> struct RedCount<RED_R0DOT> { static constexpr int n = 1; };
template <> struct RedCount<RED_BICG> { static constexpr int n = 5; };
template <> struct RedCount<RED_NORM> { static constexpr int n = 1; };

struct HopArgs {
    void *out;              // parity p half field  [Vh][12][N]
    const void *in;         // parity 1-p half field
    const void *y;          // parity p (XPAY / RESID)
    const void *z;          // parity p (RESID)
    const void *rhat;       // parity p (R0DOT / BICG)
    const void *gauge;      // [2][Vh][4][9] complex
    const uint32_t *coords; // [2][Vh] packed x | y<<8 | z<<16 | t<<24
    double2 *partials;      // [gridDim.x][N][NV]
    int p;                  // output parity
    int N;                  // right-hand sides in the layout
    int cb_begin, cb_end;   // output sites processed
    double c;               // coefficient of D
    Geom g;
    const void *gauge8;     // [2][Vh][8][9] complex, site-major links (staged kernel)
    int *err;               // [2]: the staged kernel sets [0] when a bounded wait runs out, [1] when a drain wait does too
    int blocked;            // direct kernel: 0 cyclic site mapping, 1 one contiguous range per block
    const float4 *gauge8q;  // [2][Vh][8][9] FP32 quads (Re V, Re V, -Im V, Im V), V = U (forward) or U^dag
                            // (backward, already conjugated): the packed-arithmetic kernel's links
    const int *act;         // per right-hand side r: act[r * act_stride] != 0 if it takes part in this
    int act_stride;         // iteration; NULL: all do.  The direct kernels skip the others' loads and stores.
    const float4 *gauge8d;  // [2][Vh][8][9] FP32 quads (Re U, Re U, Im U, Im U) of the site-major rows:
                            // the paired-layout kernel's links
    const void *clovinv;    // clover: A^-1 of the output sites in the storage type ([2][Vh][2][6][6]
                            // complex), applied to D in before the epilogue; NULL: no clover term
};

// Load the 12 components of R right-hand sides at one neighbour site and
// project them to the two-spinor h = psi_up + s X_mu psi_down (s = SG).
template <typename S, int R, int MU, int SG>
__device__ __forceinline__ void load_project(const S *src, size_t N, cx<typename Real<S>::type> (&h)[R][6]) {
    typedef typename Real<S>::type T;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<T> q0[R], q1[R], q2[R], q3[R];
        ld_pack<S, R, true>(src + (size_t)a * N * 2, q0);
        ld_pack<S, R, true>(src + (size_t)(3 + a) * N * 2, q1);
        ld_pack<S, R, true>(src + (size_t)(6 + a) * N * 2, q2);
        ld_pack<S, R, true>(src + (size_t)(9 + a) * N * 2, q3);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const cx<T> p0 = q0[r], p1 = q1[r], p2 = q2[r], p3 = q3[r];
            if (MU == 0) {        // X = i sigma_x : X psi_d = (i p3, i p2)
                h[r][a] = SG > 0 ? p0 + ti(p3) : p0 - ti(p3);
                h[r][3 + a] = SG > 0 ? p1 + ti(p2) : p1 - ti(p2);
            } else if (MU == 1) { // X = -i sigma_y = [[0,-1],[1,0]] : X psi_d = (-p3, p2)
                h[r][a] = SG > 0 ? p0 - p3 : p0 + p3;
                h[r][3 + a] = SG > 0 ? p1 + p2 : p1 - p2;
            } else if (MU == 2) { // X = i sigma_z : X psi_d = (i p2, -i p3)
                h[r][a] = SG > 0 ? p0 + ti(p2) : p0 - ti(p2);
                h[r][3 + a] = SG > 0 ? p1 - ti(p3) : p1 + ti(p3);
            } else {              // X = 1
                h[r][a] = SG > 0 ? p0 + p2 : p0 - p2;
                h[r][3 + a] = SG > 0 ? p1 + p3 : p1 - p3;
            }
        }
    }
}

// acc += [ w ; s X_mu^dag w ] (the reconstructed lower spins), s = S.
template <typename T, int MU, int S>
__device__ __forceinline__ void reconstruct(const cx<T> (&w)[6], cx<T> (&acc)[12]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const cx<T> w0 = w[a], w1 = w[3 + a];
        acc[a] = acc[a] + w0;
        acc[3 + a] = acc[3 + a] + w1;
        // lower = s X^dag w
        if (MU == 0) {        // X^dag w = (-i w1, -i w0)
            acc[6 + a] = S > 0 ? acc[6 + a] + tmi(w1) : acc[6 + a] - tmi(w1);
            acc[9 + a] = S > 0 ? acc[9 + a] + tmi(w0) : acc[9 + a] - tmi(w0);
        } else if (MU == 1) { // X^dag w = (w1, -w0)
            acc[6 + a] = S > 0 ? acc[6 + a] + w1 : acc[6 + a] - w1;
            acc[9 + a] = S > 0 ? acc[9 + a] - w0 : acc[9 + a] + w0;
        } else if (MU == 2) { // X^dag w = (-i w0, i w1)
            acc[6 + a] = S > 0 ? acc[6 + a] + tmi(w0) : acc[6 + a] - tmi(w0);
            acc[9 + a] = S > 0 ? acc[9 + a] + ti(w1) : acc[9 + a] - ti(w1);
        } else {              // X^dag w = (w0, w1)
            acc[6 + a] = S > 0 ? acc[6 + a] + w0 : acc[6 + a] - w0;
            acc[9 + a] = S > 0 ? acc[9 + a] + w1 : acc[9 + a] - w1;
        }
    }
}

// w = U h (DAG = false) or U^dag h (DAG = true) on both spin components of h.
template <typename T, bool DAG>
__device__ __forceinline__ void su3_mul(const cx<T> (&u)[9], const cx<T> (&h)[6], cx<T> (&w)[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<T> acc = zero<T>();
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (DAG) cjmac(acc, u[b * 3 + a], h[3 * s + b]);
                else cmac(acc, u[a * 3 + b], h[3 * s + b]);
            }
            w[3 * s + a] = acc;
        }
}

template <typename S, int R, int MU, int NC>
__device__ __forceinline__ void hop_dir(const HopArgs &A, const Site &st, int cb, int r0,
                                        cx<typename Real<S>::type> (&acc)[R][12]) {
    typedef typename Real<S>::type T;
    constexpr bool G8 = sizeof(S) < sizeof(double);  // FP32 / BF16 read the site-major link rows
    const S *in = reinterpret_cast<const S *>(A.in);
    const S *gauge = reinterpret_cast<const S *>(A.gauge);
    const size_t N = NC ? (size_t)NC : (size_t)A.N;
    // ---- forward: (1 - g_mu) U_mu(x) psi(x + mu)
    {
        const int nb = nbr_fwd(st, A.g, MU);
        // the low-precision link rows carry the time boundary factor already
        const bool flip = !G8 && (MU == 3) && (A.g.t_bc < 0) && (st.c[3] == A.g.L[3] - 1);
        cx<T> u[9];
        // low precision: site-major rows (all eight links of the output site together)
        const S *up = G8 ? reinterpret_cast<const S *>(A.gauge8) + (((size_t)A.p * A.g.Vh + cb) * 8 + 2 * MU) * 18
                         : gauge + (((size_t)A.p * A.g.Vh + cb) * 4 + MU) * 18;
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k] = ld_link<S>(up + 2 * k);
        const S *src = in + (size_t)nb * 12 * N * 2 + (size_t)r0 * 2;
        cx<T> hh[R][6];
        load_project<S, R, MU, -1>(src, N, hh);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cx<T> w[6];
            cx<T> (&h)[6] = hh[r];
            if (flip) {
#pragma unroll
                for (int k = 0; k < 6; ++k) h[k] = -h[k];
            }
            su3_mul<T, false>(u, h, w);
            reconstruct<T, MU, -1>(w, acc[r]);
        }
    }
    // ---- backward: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)
    {
        const int nb = nbr_bwd(st, A.g, MU);
        const bool flip = !G8 && (MU == 3) && (A.g.t_bc < 0) && (st.c[3] == 0);
        cx<T> u[9];
        const S *up = G8 ? reinterpret_cast<const S *>(A.gauge8) + (((size_t)A.p * A.g.Vh + cb) * 8 + 2 * MU + 1) * 18
                         : gauge + (((size_t)(1 - A.p) * A.g.Vh + nb) * 4 + MU) * 18;
#pragma unroll
        for (int k = 0; k < 9; ++k) u[k] = ld_link<S>(up + 2 * k);
        const S *src = in + (size_t)nb * 12 * N * 2 + (size_t)r0 * 2;
        cx<T> hh[R][6];
        load_project<S, R, MU, +1>(src, N, hh);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cx<T> w[6];
            cx<T> (&h)[6] = hh[r];
            if (flip) {
#pragma unroll
                for (int k = 0; k < 6; ++k) h[k] = -h[k];
            }
            su3_mul<T, true>(u, h, w);
            reconstruct<T, MU, +1>(w, acc[r]);
        }
    }
}

// ---------------------------------------------------------------------------
// Packed FP32 arithmetic (sm_100 and later: one FFMA2 / FADD2 instruction does
// two FP32 operations).  A complex value is an FP32 pair (re, im); with the
// link element stored as the quads (Re V, Re V) and (-Im V, Im V),
//   w += V h  is  w = ffma2((Re V, Re V), (Re h, Im h), w)
//                 w = ffma2((-Im V, Im V), (Im h, Re h), w),
// the same four FMAs in the same order as cmac/cjmac of the scalar kernel, so
// the results agree bit for bit; the instruction count of the SU(3) products
// and of the real-valued reconstructions halves.  Backward links are stored
// already conjugated, so every direction is a plain product.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }

// acc += [ w ; s X_mu^dag w ] on FP32 pairs (s = S); the i-rotations stay scalar.
template <int MU, int S>
__device__ __forceinline__ void reconstruct_x2(const float2 (&w)[6], float2 (&acc)[12]) {
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 w0 = w[a], w1 = w[3 + a];
        acc[a] = __fadd2_rn(acc[a], w0);
        acc[3 + a] = __fadd2_rn(acc[3 + a], w1);
        float2 &l6 = acc[6 + a], &l9 = acc[9 + a];
        if (MU == 0) {        // X^dag w = (-i w1, -i w0); -i z = (z.im, -z.re)
            l6 = S > 0 ? make_float2(l6.x + w1.y, l6.y - w1.x) : make_float2(l6.x - w1.y, l6.y + w1.x);
            l9 = S > 0 ? make_float2(l9.x + w0.y, l9.y - w0.x) : make_float2(l9.x - w0.y, l9.y + w0.x);
        } else if (MU == 1) { // X^dag w = (w1, -w0)
            l6 = S > 0 ? __fadd2_rn(l6, w1) : __ffma2_rn(m1, w1, l6);
            l9 = S > 0 ? __ffma2_rn(m1, w0, l9) : __fadd2_rn(l9, w0);
        } else if (MU == 2) { // X^dag w = (-i w0, i w1); i z = (-z.im, z.re)
            l6 = S > 0 ? make_float2(l6.x + w0.y, l6.y - w0.x) : make_float2(l6.x - w0.y, l6.y + w0.x);
            l9 = S > 0 ? make_float2(l9.x - w1.y, l9.y + w1.x) : make_float2(l9.x + w1.y, l9.y - w1.x);
        } else {              // X^dag w = (w0, w1)
            l6 = S > 0 ? __fadd2_rn(l6, w0) : __ffma2_rn(m1, w0, l6);
            l9 = S > 0 ? __fadd2_rn(l9, w1) : __ffma2_rn(m1, w1, l9);
        }
    }
}

// One hop direction D = 2 MU (+1 backward) of the packed kernel.
template <int MU, int SG, int NC>
__device__ __forceinline__ void hop_dir_x2(const HopArgs &A, const Site &st, int cb, int r0, float2 (&acc)[12]) {
    const float *in = reinterpret_cast<const float *>(A.in);
    const size_t N = NC ? (size_t)NC : (size_t)A.N;
    constexpr int D = 2 * MU + (SG > 0 ? 1 : 0);
    const int nb = SG < 0 ? nbr_fwd(st, A.g, MU) : nbr_bwd(st, A.g, MU);
    const float *src = in + (size_t)nb * 12 * N * 2 + (size_t)r0 * 2;
    cx<float> hh[1][6];
    load_project<float, 1, MU, SG>(src, N, hh);
    float2 h[6];  // (the link quads carry the time boundary factor)
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = make_float2(hh[0][k].re, hh[0][k].im);
    const float4 *q = A.gauge8q + (((size_t)A.p * A.g.Vh + cb) * 8 + D) * 9;
    float2 w[6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float4 v[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) v[b] = __ldg(q + a * 3 + b);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
            float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float2 hb = h[3 * sp + b];
                acc2 = __ffma2_rn(make_float2(v[b].x, v[b].y), hb, acc2);
                acc2 = __ffma2_rn(make_float2(v[b].z, v[b].w), swap2(hb), acc2);
            }
            w[3 * sp + a] = acc2;
        }
    }
    reconstruct_x2<MU, SG>(w, acc);
}

// NC > 0: the number of right-hand sides in the layout is the compile-time
// constant NC (= A.N), so component offsets fold into the load and store
// instructions; NC = 0 reads it from A.N.
template <typename S, int R, int MODE, int RED, int NC = 0, int X2 = 0, int CLOV = 0>
__device__ __forceinline__ void hop_body(const HopArgs &A) {
    typedef typename Real<S>::type T;
    constexpr int NV = RedCount<RED>::n > 0 ? RedCount<RED>::n : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    const int NN = NC ? NC : A.N;
    const int G = NN / R;  // a power of two dividing 32 (checked by the host)
    const int lgG = __ffs(G) - 1;
    const size_t N = (size_t)NN;
    const int total = (A.cb_end - A.cb_begin) << lgG;  // < 2^31 (checked by the host)
    const T cD = from_double<T>(A.c);
    cx<T> red[R][NV];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[r][k] = zero<T>();

    // Cyclic mapping: consecutive blocks take consecutive sites and the grid strides
    // over the lattice.  Blocked mapping: each (large) block walks its own contiguous
    // range of sites, so the neighbours loaded for one step (the same and the adjacent
    // x-rows of the other parity) are still in L1 for the next steps.
    int idx = blockIdx.x * blockDim.x + threadIdx.x, idx_end = total, stride = gridDim.x * blockDim.x;
    if (A.blocked) {
        const int per = ((total + (int)gridDim.x - 1) / (int)gridDim.x + (int)blockDim.x - 1) / (int)blockDim.x *
                        (int)blockDim.x;
        idx = blockIdx.x * per + threadIdx.x;
        idx_end = min(total, (int)(blockIdx.x + 1) * per);
        stride = blockDim.x;
    }
    // A thread keeps its right-hand sides for the whole launch (the stride is a
    // multiple of G), so those that have converged (or stopped) are read once:
    // such a thread loads and stores nothing.
    if (A.act && idx < idx_end) {
        const int r0 = (idx & (G - 1)) * R;
        bool any = false;
#pragma unroll
        for (int r = 0; r < R; ++r) any |= __ldg(A.act + (size_t)(r0 + r) * A.act_stride) != 0;
        if (!any) idx = idx_end;
    }
    for (; idx < idx_end; idx += stride) {
        const int cb = A.cb_begin + (idx >> lgG);
        const int r0 = (idx & (G - 1)) * R;
        const Site st = decode(__ldg(A.coords + (size_t)A.p * A.g.Vh + cb), A.g);
        cx<T> acc[R][12];
        if constexpr (X2 != 0 && sizeof(S) == 4 && R == 1) {
            float2 a2[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) a2[c] = make_float2(0.f, 0.f);
            hop_dir_x2<0, -1, NC>(A, st, cb, r0, a2);
            hop_dir_x2<0, +1, NC>(A, st, cb, r0, a2);
            hop_dir_x2<1, -1, NC>(A, st, cb, r0, a2);
            hop_dir_x2<1, +1, NC>(A, st, cb, r0, a2);
            hop_dir_x2<2, -1, NC>(A, st, cb, r0, a2);
            hop_dir_x2<2, +1, NC>(A, st, cb, r0, a2);
            hop_dir_x2<3, -1, NC>(A, st, cb, r0, a2);
            hop_dir_x2<3, +1, NC>(A, st, cb, r0, a2);
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[0][c] = mk((T)a2[c].x, (T)a2[c].y);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < 12; ++c) acc[r][c] = zero<T>();
            hop_dir<S, R, 0, NC>(A, st, cb, r0, acc);
            hop_dir<S, R, 1, NC>(A, st, cb, r0, acc);
            hop_dir<S, R, 2, NC>(A, st, cb, r0, acc);
            hop_dir<S, R, 3, NC>(A, st, cb, r0, acc);
            if constexpr (CLOV != 0 && R == 1)  // clover: A^-1 of the output site on D in
                clover_inv_apply<S, T>(reinterpret_cast<const S *>(A.clovinv) + ((size_t)A.p * A.g.Vh + cb) * 72 * 2,
                                       acc[0]);
        }

        const size_t base = (size_t)cb * 12 * N * 2 + (size_t)r0 * 2;
        S *out = reinterpret_cast<S *>(A.out);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t off = base + (size_t)c * N * 2;
            cx<T> o[R];
            if (MODE == MODE_PLAIN) {
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = cD * acc[r][c];
            }
            cx<T> yv[R];
            if (MODE == MODE_XPAY || MODE == MODE_RESID || RED == RED_BICG) {
                ld_pack<S, R, true>(reinterpret_cast<const S *>(A.y) + off, yv);
            }
            if (MODE == MODE_XPAY) {
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = yv[r] + cD * acc[r][c];
            } else if (MODE == MODE_RESID) {
                cx<T> zv[R];
                ld_pack<S, R, true>(reinterpret_cast<const S *>(A.z) + off, zv);
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = zv[r] - yv[r] - cD * acc[r][c];
            }
            st_pack<S, R>(out + off, o);
            if (RED == RED_R0DOT || RED == RED_BICG) {
                cx<T> rh[R];
                ld_pack<S, R, true>(reinterpret_cast<const S *>(A.rhat) + off, rh);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (RED == RED_R0DOT) {
                        cjmac(red[r][0], rh[r], o[r]);
                    } else {
                        cjmac(red[r][0], o[r], yv[r]);   // <t, s>
                        cjmac(red[r][1], o[r], o[r]);    // <t, t>
                        cjmac(red[r][2], rh[r], yv[r]);  // <rhat, s>
                        cjmac(red[r][3], rh[r], o[r]);   // <rhat, t>
                        cjmac(red[r][4], yv[r], yv[r]);  // <s, s>
                    }
                }
            } else if (RED == RED_NORM) {
#pragma unroll
                for (int r = 0; r < R; ++r) cjmac(red[r][0], o[r], o[r]);
            }
        }
    }
    if (RED != RED_NONE) block_reduce<R, NV, T>(red, G, NN, A.partials, smem);
}

// Register caps of the direct hop (0: the compiler's choice under a 256-thread
// launch bound).  The kernel is bound by memory latency: fewer registers per
// thread let more warps, and so more loads, be in flight per SM.  Measured on
// GB300 with FP32 storage, one right-hand side per thread and 32 right-hand
// sides (bench.py --hop-profile), against the compiler's choice:
//   plain hop            80 -> 64 registers: 0.142 -> 0.133 ms
//   XPAY + <rhat, v>     80 -> 72 registers: 0.185 -> 0.170 ms
//   XPAY + 5 reductions 110 -> 72 registers: 0.216 -> 0.182 ms
// R > 1 spills and runs 3-4x slower under such caps.  BF16 at R = 1 gained
// nothing from them and its tuner picks R = 2 or 4.  FP64 is bound by FP64
// issue.  So all of these stay uncapped.
template <typename S, int R, int MODE, int RED> struct HopRegCap {
    static constexpr bool f32r1 = sizeof(S) == 4 && R == 1;
    static constexpr int n = !f32r1 ? 0 : (MODE == MODE_PLAIN ? 64 : 72);
};

template <typename S, int R, int MODE, int RED>
__global__ void __launch_bounds__(256) hop_kernel(HopArgs A) {
    hop_body<S, R, MODE, RED>(A);
}

template <typename S, int R, int MODE, int RED, int CAP, int NC = 0>
__global__ void __maxnreg__(CAP) hop_kernel_cap(HopArgs A) {
    hop_body<S, R, MODE, RED, NC>(A);
}

// Clover direct kernel (one right-hand side per thread): the inner hops of the
// clover operator's asymmetric Schur system, A^-1 D.
template <typename S, int MODE, int RED>
__global__ void __launch_bounds__(256) hop_kernel_clov(HopArgs A) {
    hop_body<S, 1, MODE, RED, 0, 0, 1>(A);
}
// The same under the direct FP32 kernels' register caps, with the width a
// compile-time constant.
template <typename S, int MODE, int RED, int CAP, int NC>
__global__ void __maxnreg__(CAP) hop_kernel_clov_cap(HopArgs A) {
    hop_body<S, 1, MODE, RED, NC, 0, 1>(A);
}

// Packed-arithmetic direct kernel (FP32 storage, one right-hand side per thread).
template <int MODE, int RED, int CAP, int NC = 0>
__global__ void __maxnreg__(CAP) hop_kernel_x2(HopArgs A) {
    hop_body<float, 1, MODE, RED, NC, 1>(A);
}




// ---------------------------------------------------------------------------
// Prefetching variant.  Each thread streams its neighbour spinors and links
// through a private two-stage shared-memory ring with cp.async: the data of
// the next hop direction (or of the first direction of its next site) are in
// flight while the current direction is computed, so the memory pipeline stays
// full without holding the loads in registers.  Shared layout
// [stage][item][thread] keeps every warp access conflict-free.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void *src) {
    if (BYTES == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
    else if (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N_PENDING>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N_PENDING)); }

template <typename S, int R>
struct PfLayout {
    static constexpr int PB = R * cbytes<S>();            // bytes of one packed component
    static constexpr int CH = PB > 16 ? 16 : PB;          // bytes per cp.async
    static constexpr int NCH = PB / CH;                   // copies per component
    static constexpr int LB = cbytes<S>();                // bytes of one link entry
    static constexpr int STAGE = 12 * PB + 9 * LB;        // bytes per thread per stage
};

// Issue the copies of direction D (MU = D/2, forward if D even) of site `st`.
template <typename S, int R, int D>
__device__ __forceinline__ void pf_issue(const HopArgs &A, const Site &st, int cb, int r0, unsigned char *stage_base,
                                         int nthreads) {
    typedef PfLayout<S, R> L;
    constexpr int MU = D / 2;
    const S *in = reinterpret_cast<const S *>(A.in);
    const S *gauge = reinterpret_cast<const S *>(A.gauge);
    const int nb = (D % 2 == 0) ? nbr_fwd(st, A.g, MU) : nbr_bwd(st, A.g, MU);
    const S *src = in + (size_t)nb * 12 * A.N * 2 + (size_t)r0 * 2;
    const S *up = (D % 2 == 0) ? gauge + (((size_t)A.p * A.g.Vh + cb) * 4 + MU) * 18
                               : gauge + (((size_t)(1 - A.p) * A.g.Vh + nb) * 4 + MU) * 18;
    const uint32_t base = smem_addr(stage_base) + threadIdx.x * L::CH;
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int h = 0; h < L::NCH; ++h)
            cp_async<L::CH>(base + (uint32_t)((c * L::NCH + h) * nthreads * L::CH),
                            reinterpret_cast<const unsigned char *>(src + (size_t)c * A.N * 2) + h * L::CH);
    const uint32_t lbase = smem_addr(stage_base + 12 * L::PB * nthreads) + threadIdx.x * L::LB;
#pragma unroll
    for (int k = 0; k < 9; ++k) cp_async<L::LB>(lbase + (uint32_t)(k * nthreads * L::LB), up + 2 * k);
}

// Compute direction D of the current site from a landed stage.
template <typename S, int R, int D>
__device__ __forceinline__ void pf_compute(const HopArgs &A, const Site &st, const unsigned char *stage_base,
                                           int nthreads, cx<typename Real<S>::type> (&acc)[R][12]) {
    typedef typename Real<S>::type T;
    typedef PfLayout<S, R> L;
    constexpr int MU = D / 2;
    constexpr int SG = (D % 2 == 0) ? -1 : +1;
    cx<T> hh[R][6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<T> q[4][R];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            const int c = 3 * sp + a;
            uint32_t w[L::PB / 4];
#pragma unroll
            for (int h = 0; h < L::NCH; ++h) {
                const unsigned char *p = stage_base + ((c * L::NCH + h) * nthreads + threadIdx.x) * L::CH;
#pragma unroll
                for (int k = 0; k < L::CH / 4; ++k) w[h * (L::CH / 4) + k] = reinterpret_cast<const uint32_t *>(p)[k];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) q[sp][r] = Conv<S>::get(w + r * Conv<S>::W);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const cx<T> p0 = q[0][r], p1 = q[1][r], p2 = q[2][r], p3 = q[3][r];
            if (MU == 0) {
                hh[r][a] = SG > 0 ? p0 + ti(p3) : p0 - ti(p3);
                hh[r][3 + a] = SG > 0 ? p1 + ti(p2) : p1 - ti(p2);
            } else if (MU == 1) {
                hh[r][a] = SG > 0 ? p0 - p3 : p0 + p3;
                hh[r][3 + a] = SG > 0 ? p1 + p2 : p1 - p2;
            } else if (MU == 2) {
                hh[r][a] = SG > 0 ? p0 + ti(p2) : p0 - ti(p2);
                hh[r][3 + a] = SG > 0 ? p1 - ti(p3) : p1 + ti(p3);
            } else {
                hh[r][a] = SG > 0 ? p0 + p2 : p0 - p2;
                hh[r][3 + a] = SG > 0 ? p1 + p3 : p1 - p3;
            }
        }
    }
    cx<T> u[9];
    const unsigned char *lb = stage_base + 12 * L::PB * nthreads;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        uint32_t w[L::LB / 4];
#pragma unroll
        for (int j = 0; j < L::LB / 4; ++j)
            w[j] = reinterpret_cast<const uint32_t *>(lb + (k * nthreads + threadIdx.x) * L::LB)[j];
        u[k] = Conv<S>::get(w);
    }
    const bool flip = (MU == 3) && (A.g.t_bc < 0) && (st.c[3] == ((D % 2 == 0) ? A.g.L[3] - 1 : 0));
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cx<T> w[6];
        cx<T>(&h)[6] = hh[r];
        if (flip) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = -h[k];
        }
        su3_mul<T, (D % 2 == 1)>(u, h, w);
        reconstruct<T, MU, SG>(w, acc[r]);
    }
}

template <typename S, int R, int MODE, int RED>
__global__ void __launch_bounds__(256) hop_kernel_pf(HopArgs A) {
    typedef typename Real<S>::type T;
    typedef PfLayout<S, R> L;
    constexpr int NV = RedCount<RED>::n > 0 ? RedCount<RED>::n : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    const int nthreads = blockDim.x;
    unsigned char *stage[2] = {smem, smem + (size_t)L::STAGE * nthreads};
    const int G = A.N / R;
    const int lgG = __ffs(G) - 1;
    const size_t N = (size_t)A.N;
    const int total = (A.cb_end - A.cb_begin) << lgG;
    const int stride = gridDim.x * blockDim.x;
    const T cD = from_double<T>(A.c);
    cx<T> red[R][NV];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[r][k] = zero<T>();

    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int cb = 0, r0 = 0;
    Site st;
    if (idx < total) {
        cb = A.cb_begin + (idx >> lgG);
        r0 = (idx & (G - 1)) * R;
        st = decode(__ldg(A.coords + (size_t)A.p * A.g.Vh + cb), A.g);
        pf_issue<S, R, 0>(A, st, cb, r0, stage[0], nthreads);
    }
    cp_commit();
    for (; idx < total; idx += stride) {
        cx<T> acc[R][12];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[r][c] = zero<T>();
        // next site (for the prefetch issued during direction 7)
        const int nidx = idx + stride;
        int ncb = 0, nr0 = 0;
        Site nst = st;
        if (nidx < total) {
            ncb = A.cb_begin + (nidx >> lgG);
            nr0 = (nidx & (G - 1)) * R;
            nst = decode(__ldg(A.coords + (size_t)A.p * A.g.Vh + ncb), A.g);
        }
#define DL_PF_STEP(D)                                                                  \
        {                                                                              \
            if (D < 7) pf_issue<S, R, (D + 1) % 8>(A, st, cb, r0, stage[(D + 1) & 1], nthreads); \
            else if (nidx < total) pf_issue<S, R, 0>(A, nst, ncb, nr0, stage[0], nthreads);     \
            cp_commit();                                                               \
            cp_wait<1>();                                                              \
            pf_compute<S, R, D>(A, st, stage[D & 1], nthreads, acc);                   \
        }
        DL_PF_STEP(0) DL_PF_STEP(1) DL_PF_STEP(2) DL_PF_STEP(3)
        DL_PF_STEP(4) DL_PF_STEP(5) DL_PF_STEP(6) DL_PF_STEP(7)
#undef DL_PF_STEP

        const size_t base = (size_t)cb * 12 * N * 2 + (size_t)r0 * 2;
        S *out = reinterpret_cast<S *>(A.out);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t off = base + (size_t)c * N * 2;
            cx<T> o[R];
            if (MODE == MODE_PLAIN) {
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = cD * acc[r][c];
            }
            cx<T> yv[R];
            if (MODE == MODE_XPAY || MODE == MODE_RESID || RED == RED_BICG) {
                ld_pack<S, R, true>(reinterpret_cast<const S *>(A.y) + off, yv);
            }
            if (MODE == MODE_XPAY) {
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = yv[r] + cD * acc[r][c];
            } else if (MODE == MODE_RESID) {
                cx<T> zv[R];
                ld_pack<S, R, true>(reinterpret_cast<const S *>(A.z) + off, zv);
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = zv[r] - yv[r] - cD * acc[r][c];
            }
            st_pack<S, R>(out + off, o);
            if (RED == RED_R0DOT || RED == RED_BICG) {
                cx<T> rh[R];
                ld_pack<S, R, true>(reinterpret_cast<const S *>(A.rhat) + off, rh);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (RED == RED_R0DOT) {
                        cjmac(red[r][0], rh[r], o[r]);
                    } else {
                        cjmac(red[r][0], o[r], yv[r]);
                        cjmac(red[r][1], o[r], o[r]);
                        cjmac(red[r][2], rh[r], yv[r]);
                        cjmac(red[r][3], rh[r], o[r]);
                        cjmac(red[r][4], yv[r], yv[r]);
                    }
                }
            } else if (RED == RED_NORM) {
#pragma unroll
                for (int r = 0; r < R; ++r) cjmac(red[r][0], o[r], o[r]);
            }
        }
        st = nst;
        cb = ncb;
        r0 = nr0;
    }
    cp_wait<0>();
    if (RED != RED_NONE) {
        __syncthreads();  // the reduction reuses the staging buffer
        block_reduce<R, NV, T>(red, G, A.N, A.partials, smem);
    }
}
}  // namespace dl
