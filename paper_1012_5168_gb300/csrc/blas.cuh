// BiCGStab vector updates, scalar recurrences and the FP64 defect-correction
// steps, for N right-hand sides in the even-odd tile layout (see common.cuh).
//
// The Krylov solver is BiCGStab (van der Vorst 1992; Sec. 2 of the paper uses
// QUDA's mixed-precision CG/BiCGStab) on the even-site Schur complement
// Mhat = 1 - kappa^2 D_eo D_oe.  One iteration, per right-hand side:
//
//   v = Mhat p                 (two hops; <rhat, v> fused in the second)
//   alpha = rho / <rhat, v>
//   s = r - alpha v
//   t = Mhat s                 (two hops; <t,s>, <t,t>, <rhat,s>, <rhat,t>, <s,s> fused)
//   omega = <t,s> / <t,t>
//   rho'  = <rhat, s - omega t> = <rhat,s> - omega <rhat,t>
//   beta  = (rho'/rho) (alpha/omega)
//   |r'|^2 = <s,s> - |<t,s>|^2/<t,t>      (r' = s - omega t)
//   x += alpha p + omega s ;  r = s - omega t ;  p = r + beta (p - omega v)
//
// Knowing rho' and beta before the vector update lets one kernel do all three
// updates (5 reads, 3 writes per element).  Per-right-hand-side scalars live in
// device memory (RhsState) so whole iterations can be captured in CUDA graphs;
// every right-hand side carries its own active flag and stops independently.
#pragma once

#include "common.cuh"

namespace dl {

enum { ST_OK = 0, ST_BREAKDOWN = 5, ST_NAN = 6 };

struct RhsState {
    double2 rho, alpha, omega, beta;
    double r2;       // recursive residual norm^2 of the inner iteration
    double r2_0;     // at the start of the inner cycle
    double target2;  // stop the inner cycle when r2 <= target2
    int active;      // takes part in the current iteration
    int next_active; // takes part in the next iteration
    int iters;       // inner iterations in this cycle
    int status;      // ST_OK / ST_BREAKDOWN / ST_NAN (inner cycle)
    int max_iters;   // cap on iterations in this cycle
    int fixed;       // 1: run exactly max_iters iterations
};

struct OuterState {
    double b2;        // |bhat|^2 (even-site Schur system)
    double r2;        // |bhat - Mhat x|^2 (FP64 true residual of the Schur system)
    double full_b2;   // |b|^2 (full lattice)
    double full_r2;   // |b - M x|^2 (full lattice)
    double tol2;      // tol^2
    int active;       // not yet converged
    int status;
    int outer;        // defect-correction cycles done
    int iters;        // inner iterations summed over cycles
    double sigma;     // |r64| that scaled the current inner phase (0 before the first)
    int scale_exp;    // the batch's fields carry the exact factor 2^scale_exp (float-float outer loop)
};

__device__ __forceinline__ bool finite2(double2 z) { return isfinite(z.x) && isfinite(z.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Sum partials[b][rhs][k] over blocks b for one right-hand side, by the whole
// thread block (a multiple of 32 threads), in a fixed order: strided per-thread
// sums, then warp shuffles, then the warps in index order.  Every thread gets
// the total.
__device__ __forceinline__ double2 sum_partials(const double2 *partials, int nblocks, int N, int NV, int rhs, int k) {
    __shared__ double2 wsum[32];
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double2 v = partials[((size_t)b * N + rhs) * NV + k];
        re += v.x;
        im += v.y;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, off);
        im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    const int nw = blockDim.x >> 5;
    if (nw == 1) return make_double2(re, im);
    __syncthreads();  // an earlier call may still be reading wsum
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = make_double2(re, im);
    __syncthreads();
    re = 0.0;
    im = 0.0;
    for (int w = 0; w < nw; ++w) {
        re += wsum[w].x;
        im += wsum[w].y;
    }
    return make_double2(re, im);
}

// All NV values of right-hand side `rhs` at once, each summed in exactly the
// order of sum_partials (so the results are bitwise the same), in one pass over
// the blocks: a thread reads the NV contiguous values of each of its blocks.
template <int NV>
__device__ __forceinline__ void sum_partials_all(const double2 *partials, int nblocks, int N, int rhs,
                                                 double2 (&out)[NV]) {
    __shared__ double2 wsum[32][NV];
    double re[NV], im[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) re[k] = im[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const double2 *p = partials + ((size_t)b * N + rhs) * NV;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double2 v = p[k];
            re[k] += v.x;
            im[k] += v.y;
        }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            re[k] += __shfl_xor_sync(0xffffffffu, re[k], off);
            im[k] += __shfl_xor_sync(0xffffffffu, im[k], off);
        }
    const int nw = blockDim.x >> 5;
    if (nw == 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = make_double2(re[k], im[k]);
        return;
    }
    __syncthreads();  // an earlier call may still be reading wsum
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) wsum[threadIdx.x >> 5][k] = make_double2(re[k], im[k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double sr = 0.0, si = 0.0;
        for (int w = 0; w < nw; ++w) {
            sr += wsum[w][k].x;
            si += wsum[w][k].y;
        }
        out[k] = make_double2(sr, si);
    }
}

// Threads per block of the per-right-hand-side scalar kernels (grid = N blocks).
constexpr int kScalarThreads = 256;

// Relative reduction the inner phase aims for: delta, or less when less suffices
// for the outer test |r| <= 0.5 tol min(|bhat|, |b|) (outer_update_kernel), with
// a further factor of 2 for the drift of the low-precision recursive residual.
__device__ __forceinline__ double inner_reduction(const OuterState &o, double delta) {
    if (!(o.r2 > 0.0)) return delta;
    const double need = 0.25 * sqrt(o.tol2 * fmin(o.b2, o.full_b2) / o.r2);
    return fmax(delta, need);
}

// ---------------------------------------------------------------------------
// scalar kernels: grid = N blocks of kScalarThreads (one block per right-hand side)
// ---------------------------------------------------------------------------

// Start an inner phase: rho = <rhat, r_l>, r2 = |r_l|^2 (from the partials of
// inner_init_kernel), target and caps; records the scale sigma = |r64| of the
// phase.  max_iters caps this phase; max_total the iterations over all phases.
static __global__ void inner_start_kernel(RhsState *st, OuterState *os, const double2 *partials,
                                   int nblocks, int N, double delta, int max_iters, int max_total, int fixed) {
    const int r = blockIdx.x;
    double2 v[2];
    sum_partials_all<2>(partials, nblocks, N, r, v);
    const double2 rho = v[0], n2 = v[1];
    if (threadIdx.x != 0) return;
    os[r].sigma = os[r].active ? sqrt(os[r].r2) : 0.0;
    RhsState s;
    s.rho = rho;
    s.alpha = make_double2(1.0, 0.0);
    s.omega = make_double2(1.0, 0.0);
    s.beta = make_double2(0.0, 0.0);
    s.r2 = n2.x;
    s.r2_0 = n2.x;
    const double red = inner_reduction(os[r], delta);
    s.target2 = red * red * n2.x;
    s.iters = 0;
    s.status = ST_OK;
    const int left = max_total - os[r].iters;
    s.max_iters = fixed ? max_iters : (max_iters < left ? max_iters : left);
    s.fixed = fixed;
    const bool on = os[r].active && n2.x > 0.0 && isfinite(n2.x) && (rho.x != 0.0 || rho.y != 0.0) &&
                    s.max_iters > 0;
    s.active = on;
    s.next_active = on;
    st[r] = s;
}

// After v = Mhat p: alpha = rho / <rhat, v>.
static __global__ void scalar_alpha_kernel(RhsState *st, const double2 *partials, int nblocks, int N) {
    const int r = blockIdx.x;
    const double2 d = sum_partials(partials, nblocks, N, 1, r, 0);
    if (threadIdx.x != 0) return;
    RhsState &s = st[r];
    s.active = s.next_active;
    if (!s.active) return;
    const double2 a = cdiv(s.rho, d);
    if (!(d.x * d.x + d.y * d.y > 0.0) || !finite2(a)) {
        s.status = finite2(d) ? ST_BREAKDOWN : ST_NAN;
        s.active = 0;
        s.next_active = 0;
        return;
    }
    s.alpha = a;
}

// After t = Mhat s: omega, rho', beta, |r'|^2 and the stopping test.
static __global__ void scalar_omega_kernel(RhsState *st, const double2 *partials, int nblocks, int N) {
    const int r = blockIdx.x;
    double2 v[5];
    sum_partials_all<5>(partials, nblocks, N, r, v);
    if (threadIdx.x != 0) return;
    RhsState &s = st[r];
    if (!s.active) return;
    const double2 ts = v[0];
    const double tt = v[1].x;
    const double2 r0s = v[2], r0t = v[3];
    const double ss = v[4].x;
    s.iters += 1;
    bool stop = false;
    if (!(isfinite(tt) && isfinite(ss) && finite2(ts) && finite2(r0s) && finite2(r0t))) {
        s.status = ST_NAN;
        s.omega = make_double2(0.0, 0.0);
        s.active = 0;  // the vector update is skipped
        s.next_active = 0;
        return;
    }
    if (!(tt > 0.0)) {
        // t = 0: s is already the solution's residual (zero) or the iteration broke down
        s.omega = make_double2(0.0, 0.0);
        s.r2 = ss;
        s.beta = make_double2(0.0, 0.0);
        if (ss > s.target2) s.status = ST_BREAKDOWN;
        stop = true;
    } else {
        const double2 om = make_double2(ts.x / tt, ts.y / tt);
        const double2 rho_new = make_double2(r0s.x - (om.x * r0t.x - om.y * r0t.y),
                                             r0s.y - (om.x * r0t.y + om.y * r0t.x));
        double r2 = ss - (ts.x * ts.x + ts.y * ts.y) / tt;
        if (r2 < 0.0) r2 = 0.0;
        s.omega = om;
        s.r2 = r2;
        const double2 beta = cmul2(cdiv(rho_new, s.rho), cdiv(s.alpha, om));
        if (!finite2(beta) || !(rho_new.x * rho_new.x + rho_new.y * rho_new.y > 0.0)) {
            s.beta = make_double2(0.0, 0.0);
            if (r2 > s.target2) s.status = ST_BREAKDOWN;
            stop = true;
        } else {
            s.beta = beta;
        }
        s.rho = rho_new;
    }
    const bool done = s.fixed ? (s.iters >= s.max_iters)
                              : (s.r2 <= s.target2 || s.iters >= s.max_iters);
    s.next_active = !(stop || done);
}

static __global__ void count_active_kernel(const RhsState *st, int N, int *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int n = 0;
        for (int r = 0; r < N; ++r) n += st[r].next_active;
        *out = n;
    }
}

// ---------------------------------------------------------------------------
// vector kernels (even half field, [Vh][12][N]; thread = (element, RHS group))
// ---------------------------------------------------------------------------
struct VecArgs {
    int n_elem;   // Vh * 12
    int N;        // right-hand sides in the layout
};

// s = r - alpha v
template <typename S, int R>
static __global__ void __launch_bounds__(256) axpy_s_kernel(VecArgs a, const RhsState *st, const S *r_, const S *v_, S *s_) {
    typedef typename Real<S>::type T;
    const int G = a.N / R, lgG = __ffs(G) - 1;
    const long total = (long)a.n_elem << lgG;  // elements x groups: may exceed 2^31
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int e = (int)(idx >> lgG), r0 = (int)(idx & (G - 1)) * R;
        bool any = false;
        cx<T> al[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const RhsState &q = st[r0 + k];
            any |= (q.active != 0);
            al[k] = mk((T)q.alpha.x, (T)q.alpha.y);
        }
        if (!any) continue;
        const size_t off = ((size_t)e * a.N + r0) * 2;
        cx<T> rv[R], vv[R], sv[R];
        ld_pack<S, R, true>(r_ + off, rv);
        ld_pack<S, R, true>(v_ + off, vv);
#pragma unroll
        for (int k = 0; k < R; ++k) sv[k] = rv[k] - al[k] * vv[k];
        st_pack<S, R>(s_ + off, sv);
    }
}

// x += alpha p + omega s ; r = s - omega t ; p = r + beta (p - omega v)
// (5 reads, 3 writes per element while every right-hand side is active)
template <typename S, int R>
static __global__ void __launch_bounds__(256) update_kernel(VecArgs a, const RhsState *st, S *x_, S *r_, S *p_,
                                                    const S *s_, const S *t_, const S *v_) {
    typedef typename Real<S>::type T;
    const int G = a.N / R, lgG = __ffs(G) - 1;
    const long total = (long)a.n_elem << lgG;  // elements x groups: may exceed 2^31
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int e = (int)(idx >> lgG), r0 = (int)(idx & (G - 1)) * R;
        bool any = false;
        bool on[R];
        cx<T> al[R], om[R], be[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const RhsState &q = st[r0 + k];
            on[k] = q.active != 0;
            any |= on[k];
            al[k] = mk((T)q.alpha.x, (T)q.alpha.y);
            om[k] = mk((T)q.omega.x, (T)q.omega.y);
            be[k] = mk((T)q.beta.x, (T)q.beta.y);
        }
        if (!any) continue;
        bool all = true;
#pragma unroll
        for (int k = 0; k < R; ++k) all &= on[k];
        const size_t off = ((size_t)e * a.N + r0) * 2;
        cx<T> xv[R], pv[R], sv[R], tv[R], vv[R], rv[R];
        ld_pack<S, R, false>(x_ + off, xv);
        ld_pack<S, R, false>(p_ + off, pv);
        ld_pack<S, R, true>(s_ + off, sv);
        ld_pack<S, R, true>(t_ + off, tv);
        ld_pack<S, R, true>(v_ + off, vv);
        // the old residual is only needed to keep the entries of inactive right-hand sides
        if (!all) ld_pack<S, R, false>(r_ + off, rv);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (!on[k]) continue;
            xv[k] = xv[k] + al[k] * pv[k] + om[k] * sv[k];
            rv[k] = sv[k] - om[k] * tv[k];
            pv[k] = rv[k] + be[k] * (pv[k] - om[k] * vv[k]);
        }
        st_pack<S, R>(x_ + off, xv);
        st_pack<S, R>(r_ + off, rv);
        st_pack<S, R>(p_ + off, pv);
    }
}

// Inner-phase set-up from the FP64 residual r64 (one of two modes per
// right-hand side):
//  restart:   r_l = r64/|r64| rounded to S; rhat = p = r_l; x_l = 0.
//  continue:  r_l = r64/|r64|; p *= sigma_prev/|r64| (the search direction of the
//             previous phase, rescaled to the new unit); rhat kept; x_l = 0.
//             This is a reliable update (Sleijpen & van der Vorst 1996): the
//             Krylov recurrence carries on and only the residual is replaced by
//             the true one.
// A right-hand side restarts on the first phase, after a breakdown or NaN, or
// when `restart` is set.  Partials: [0] <rhat, r_l> (rho), [1] |r_l|^2, both
// of the rounded values.  Right-hand sides no longer active in the outer loop
// get zero vectors.
template <typename S, int R>
__global__ void __launch_bounds__(256) inner_init_kernel(VecArgs a, const OuterState *os, const RhsState *st,
                                                        const double *r64, S *x_, S *r_, S *rhat_, S *p_,
                                                        double2 *partials, int restart) {
    typedef typename Real<S>::type T;
    extern __shared__ __align__(128) unsigned char smem[];
    const int G = a.N / R, lgG = __ffs(G) - 1;
    const long total = (long)a.n_elem << lgG;  // elements x groups: may exceed 2^31
    cx<T> red[R][2];
#pragma unroll
    for (int k = 0; k < R; ++k) red[k][0] = red[k][1] = zero<T>();
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int e = (int)(idx >> lgG), r0 = (int)(idx & (G - 1)) * R;
        const size_t off = ((size_t)e * a.N + r0) * 2;
        cx<double> src[R];
        ld_pack<double, R, true>(r64 + off, src);
        cx<T> lo[R], zr[R], pv[R], rh[R];
        bool cont[R];
        bool any_cont = false;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const OuterState &o = os[r0 + k];
            const bool on = o.active && o.r2 > 0.0;
            const double sc = on ? 1.0 / sqrt(o.r2) : 0.0;
            lo[k] = mk((T)(src[k].re * sc), (T)(src[k].im * sc));
            zr[k] = zero<T>();
            cont[k] = on && !restart && o.sigma > 0.0 && st[r0 + k].status == ST_OK;
            any_cont |= cont[k];
        }
        st_pack<S, R>(r_ + off, lo);
        ld_pack<S, R, false>(r_ + off, lo);  // the rounded value, for a consistent rho
        if (any_cont) {
            ld_pack<S, R, false>(p_ + off, pv);
            ld_pack<S, R, false>(rhat_ + off, rh);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (cont[k]) {
                const OuterState &o = os[r0 + k];
                const T f = (T)(o.sigma / sqrt(o.r2));
                pv[k] = f * pv[k];
            } else {
                pv[k] = lo[k];
                rh[k] = lo[k];
            }
        }
        st_pack<S, R>(p_ + off, pv);
        st_pack<S, R>(rhat_ + off, rh);
        ld_pack<S, R, false>(rhat_ + off, rh);
        st_pack<S, R>(x_ + off, zr);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            cjmac(red[k][0], rh[k], lo[k]);
            cjmac(red[k][1], lo[k], lo[k]);
        }
    }
    block_reduce<R, 2, T>(red, G, a.N, partials, smem);
}

// ---------------------------------------------------------------------------
// CG on the normal equations (CGNR: Hestenes-Stiefel CG applied to
// Mhat^dag Mhat e = Mhat^dag r_l), the single-precision solver Sec. 2 uses for
// the low-precision inversions of the truncated solver method.  Mhat is
// gamma5-hermitian (g5 Mhat g5 = Mhat^dag), so Mhat^dag costs the same two
// hops as Mhat.  Per right-hand side and iteration:
//
//   w = Mhat p                       (two hops; |w|^2 fused in the second)
//   alpha = |z|^2 / |w|^2
//   x += alpha p ;  r -= alpha w     (r stored as g5 r; |r|^2 fused)
//   u = Mhat (g5 r)                  (two hops; |u|^2 fused), z' = g5 u = Mhat^dag r
//   beta = |z'|^2 / |z|^2 ;  p = g5 u + beta p
//
// r is the residual of Mhat e = r_l itself, so the inner stopping test
// |r| <= delta |r_l| is the one BiCGStab uses.  RhsState.rho.x holds |z|^2.
// ---------------------------------------------------------------------------

// gamma5 = diag(1, 1, -1, -1) in spin: components 6..11 of a site are negated.
__device__ __forceinline__ bool g5_negates(int e) { return (e % 12) >= 6; }

// Phase set-up: g5 r_l with r_l = r64/|r64| rounded to S; x_l = 0.
// Partials [0] = |r_l|^2 of the rounded value.  Right-hand sides no longer
// active in the outer loop get zero vectors.
template <typename S, int R>
__global__ void __launch_bounds__(256) cg_init_kernel(VecArgs a, const OuterState *os, const double *r64, S *x_,
                                                     S *r5_, double2 *partials) {
    typedef typename Real<S>::type T;
    extern __shared__ __align__(128) unsigned char smem[];
    const int G = a.N / R, lgG = __ffs(G) - 1;
    const long total = (long)a.n_elem << lgG;  // elements x groups: may exceed 2^31
    cx<T> red[R][1];
#pragma unroll
    for (int k = 0; k < R; ++k) red[k][0] = zero<T>();
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int e = (int)(idx >> lgG), r0 = (int)(idx & (G - 1)) * R;
        const size_t off = ((size_t)e * a.N + r0) * 2;
        const double sg = g5_negates(e) ? -1.0 : 1.0;
        cx<double> src[R];
        ld_pack<double, R, true>(r64 + off, src);
        cx<T> lo[R], zr[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const OuterState &o = os[r0 + k];
            const double sc = (o.active && o.r2 > 0.0) ? sg / sqrt(o.r2) : 0.0;
            lo[k] = mk((T)(src[k].re * sc), (T)(src[k].im * sc));
            zr[k] = zero<T>();
        }
        st_pack<S, R>(r5_ + off, lo);
        ld_pack<S, R, false>(r5_ + off, lo);  // the rounded value
        st_pack<S, R>(x_ + off, zr);
#pragma unroll
        for (int k = 0; k < R; ++k) cjmac(red[k][0], lo[k], lo[k]);
    }
    block_reduce<R, 1, T>(red, G, a.N, partials, smem);
}

// x += alpha p ;  g5 r -= alpha g5 w  for active right-hand sides; partials [0] = |r|^2.
template <typename S, int R>
__global__ void __launch_bounds__(256) cg_update_kernel(VecArgs a, const RhsState *st, S *x_, S *r5_, const S *p_,
                                                       const S *w_, double2 *partials) {
    typedef typename Real<S>::type T;
    extern __shared__ __align__(128) unsigned char smem[];
    const int G = a.N / R, lgG = __ffs(G) - 1;
    const long total = (long)a.n_elem << lgG;  // elements x groups: may exceed 2^31
    cx<T> red[R][1];
#pragma unroll
    for (int k = 0; k < R; ++k) red[k][0] = zero<T>();
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int e = (int)(idx >> lgG), r0 = (int)(idx & (G - 1)) * R;
        bool on[R];
        bool any = false;
        T al[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const RhsState &q = st[r0 + k];
            on[k] = q.active != 0;
            any |= on[k];
            al[k] = (T)q.alpha.x;
        }
        if (!any) continue;
        const T sg = g5_negates(e) ? (T)-1 : (T)1;
        const size_t off = ((size_t)e * a.N + r0) * 2;
        cx<T> xv[R], rv[R], pv[R], wv[R];
        ld_pack<S, R, false>(x_ + off, xv);
        ld_pack<S, R, false>(r5_ + off, rv);
        ld_pack<S, R, true>(p_ + off, pv);
        ld_pack<S, R, true>(w_ + off, wv);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (!on[k]) continue;
            xv[k] = xv[k] + al[k] * pv[k];
            rv[k] = rv[k] - (sg * al[k]) * wv[k];
        }
        st_pack<S, R>(x_ + off, xv);
        st_pack<S, R>(r5_ + off, rv);
        ld_pack<S, R, false>(r5_ + off, rv);  // the rounded value
#pragma unroll
        for (int k = 0; k < R; ++k) cjmac(red[k][0], rv[k], rv[k]);
    }
    block_reduce<R, 1, T>(red, G, a.N, partials, smem);
}

// p = g5 u + beta p for active right-hand sides, or p = g5 u everywhere (init).
template <typename S, int R>
__global__ void __launch_bounds__(256) cg_p_kernel(VecArgs a, const RhsState *st, const S *u_, S *p_, int init) {
    typedef typename Real<S>::type T;
    const int G = a.N / R, lgG = __ffs(G) - 1;
    const long total = (long)a.n_elem << lgG;  // elements x groups: may exceed 2^31
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int e = (int)(idx >> lgG), r0 = (int)(idx & (G - 1)) * R;
        bool on[R];
        bool any = false;
        T be[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const RhsState &q = st[r0 + k];
            on[k] = init || q.active != 0;
            any |= on[k];
            be[k] = init ? (T)0 : (T)q.beta.x;
        }
        if (!any) continue;
        const T sg = g5_negates(e) ? (T)-1 : (T)1;
        const size_t off = ((size_t)e * a.N + r0) * 2;
        cx<T> uv[R], pv[R];
        ld_pack<S, R, true>(u_ + off, uv);
        if (init) {
#pragma unroll
            for (int k = 0; k < R; ++k) pv[k] = sg * uv[k];
        } else {
            ld_pack<S, R, false>(p_ + off, pv);
#pragma unroll
            for (int k = 0; k < R; ++k)
                if (on[k]) pv[k] = sg * uv[k] + be[k] * pv[k];
        }
        st_pack<S, R>(p_ + off, pv);
    }
}

// CG phase start: |r_l|^2 from cg_init_kernel's partials (pr), |z|^2 = |u|^2
// from the second hop of u = Mhat g5 r_l (pu); target, caps and sigma as in
// inner_start_kernel.
static __global__ void cg_start_kernel(RhsState *st, OuterState *os, const double2 *pr, int nr, const double2 *pu,
                                       int nu, int N, double delta, int max_iters, int max_total, int fixed) {
    const int r = blockIdx.x;
    const double2 n2 = sum_partials(pr, nr, N, 1, r, 0);
    const double2 zz = sum_partials(pu, nu, N, 1, r, 0);
    if (threadIdx.x != 0) return;
    os[r].sigma = os[r].active ? sqrt(os[r].r2) : 0.0;
    RhsState s;
    s.rho = make_double2(zz.x, 0.0);
    s.alpha = make_double2(0.0, 0.0);
    s.omega = make_double2(0.0, 0.0);
    s.beta = make_double2(0.0, 0.0);
    s.r2 = n2.x;
    s.r2_0 = n2.x;
    const double red = inner_reduction(os[r], delta);
    s.target2 = red * red * n2.x;
    s.iters = 0;
    s.status = ST_OK;
    const int left = max_total - os[r].iters;
    s.max_iters = fixed ? max_iters : (max_iters < left ? max_iters : left);
    s.fixed = fixed;
    const bool on = os[r].active && n2.x > 0.0 && isfinite(n2.x) && zz.x > 0.0 && isfinite(zz.x) &&
                    s.max_iters > 0;
    s.active = on;
    s.next_active = on;
    st[r] = s;
}

// After w = Mhat p: alpha = |z|^2 / |w|^2.
static __global__ void cg_alpha_kernel(RhsState *st, const double2 *partials, int nblocks, int N) {
    const int r = blockIdx.x;
    const double2 ww = sum_partials(partials, nblocks, N, 1, r, 0);
    if (threadIdx.x != 0) return;
    RhsState &s = st[r];
    s.active = s.next_active;
    if (!s.active) return;
    const double a = s.rho.x / ww.x;
    if (!(ww.x > 0.0) || !isfinite(a)) {
        s.status = isfinite(ww.x) ? ST_BREAKDOWN : ST_NAN;
        s.active = 0;
        s.next_active = 0;
        return;
    }
    s.alpha = make_double2(a, 0.0);
}

// After the update (pr: |r|^2) and u = Mhat g5 r (pu: |u|^2): beta, stopping test.
static __global__ void cg_beta_kernel(RhsState *st, const double2 *pr, int nr, const double2 *pu, int nu, int N) {
    const int r = blockIdx.x;
    const double2 n2 = sum_partials(pr, nr, N, 1, r, 0);
    const double2 zz = sum_partials(pu, nu, N, 1, r, 0);
    if (threadIdx.x != 0) return;
    RhsState &s = st[r];
    if (!s.active) return;
    s.iters += 1;
    if (!isfinite(n2.x) || !isfinite(zz.x)) {
        s.status = ST_NAN;
        s.active = 0;  // the p update is skipped
        s.next_active = 0;
        return;
    }
    s.r2 = n2.x;
    bool stop = false;
    if (!(zz.x > 0.0)) {
        s.beta = make_double2(0.0, 0.0);
        if (n2.x > s.target2) s.status = ST_BREAKDOWN;
        stop = true;
    } else {
        s.beta = make_double2(zz.x / s.rho.x, 0.0);
        s.rho = make_double2(zz.x, 0.0);
    }
    const bool done = s.fixed ? (s.iters >= s.max_iters) : (s.r2 <= s.target2 || s.iters >= s.max_iters);
    s.next_active = !(stop || done);
}

// x64 += |r64| * x_l for right-hand sides active in the outer loop.
template <typename S, int R>
static __global__ void __launch_bounds__(256) accumulate_kernel(VecArgs a, const OuterState *os, const S *x_, double *x64) {
    typedef typename Real<S>::type T;
    const int G = a.N / R, lgG = __ffs(G) - 1;
    const long total = (long)a.n_elem << lgG;  // elements x groups: may exceed 2^31
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int e = (int)(idx >> lgG), r0 = (int)(idx & (G - 1)) * R;
        const size_t off = ((size_t)e * a.N + r0) * 2;
        cx<T> xl[R];
        ld_pack<S, R, true>(x_ + off, xl);
        cx<double> acc[R];
        ld_pack<double, R, false>(x64 + off, acc);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const OuterState &o = os[r0 + k];
            if (o.active) {
                const double sc = sqrt(o.r2);
                acc[k].re += sc * (double)xl[k].re;
                acc[k].im += sc * (double)xl[k].im;
            }
        }
        st_pack<double, R>(x64 + off, acc);
    }
}

// ---------------------------------------------------------------------------
// outer (FP64) bookkeeping: grid = N blocks of kScalarThreads
// ---------------------------------------------------------------------------
// mode 0: initialise (b2 = |bhat|^2 from partials, r2 = b2, active = b2 > 0)
// mode 1: after the true residual r (partials: |r|^2, which is also the
//         full-lattice residual): r2, full_r2, convergence test, cycle count
// mode 2: after a fixed-iteration phase and its residual: full_r2 and the
//         cycle and iteration counts only
static __global__ void outer_update_kernel(OuterState *os, const RhsState *st, const double2 *partials, int nblocks,
                                    int N, int mode, double tol, int max_outer, int max_iter) {
    const int r = blockIdx.x;
    const double2 n2 = sum_partials(partials, nblocks, N, 1, r, 0);
    if (threadIdx.x != 0) return;
    OuterState &o = os[r];
    if (mode == 0) {
        o.b2 = n2.x;
        o.r2 = n2.x;
        o.tol2 = tol * tol;
        o.outer = 0;
        o.iters = 0;
        o.sigma = 0.0;
        o.status = ST_OK;
        o.active = (n2.x > 0.0) ? 1 : 0;
        if (!isfinite(n2.x)) { o.status = ST_NAN; o.active = 0; }
        return;
    }
    o.full_r2 = n2.x;  // every right-hand side: an inactive one's x is unchanged
    if (!o.active) return;
    o.outer += 1;
    o.iters += st[r].iters;
    if (st[r].status == ST_NAN) o.status = ST_NAN;
    if (mode == 2) return;
    o.r2 = n2.x;
    if (!isfinite(n2.x)) {
        o.status = ST_NAN;
        o.active = 0;
    } else if (n2.x <= 0.25 * o.tol2 * fmin(o.b2, o.full_b2)) {
        // half the tolerance on the Schur system, measured against the smaller of
        // |bhat| and |b|, so that the full-lattice residual |b - M x|/|b| meets tol
        o.active = 0;
    } else if (o.outer >= max_outer || o.iters >= max_iter) {
        o.active = 0;  // reported as not converged by the host
    }
}

static __global__ void outer_count_kernel(const OuterState *os, int N, int *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int n = 0;
        for (int r = 0; r < N; ++r) n += os[r].active;
        *out = n;
    }
}

// Exact power-of-two scale of each right-hand side for the float-float outer
// loop, whose numbers keep only the float exponent range (about 1e-38 to 3e38,
// and their low words lose bits below about 1e-31 of that range): k_r =
// -ilogb(|b_r|), so the scaled source has a norm in [1, 2).  A zero or
// non-finite norm keeps k_r = 0.  One thread per right-hand side.
static __global__ void pow2_pick_kernel(OuterState *os, int N) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double b2 = os[r].full_b2;
    os[r].scale_exp = (b2 > 0.0 && isfinite(b2)) ? -ilogb(sqrt(b2)) : 0;
}

// 2^e as a double for e in [-1022, 1023] (built from its bits, exact).
__device__ __forceinline__ double pow2_exact(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// f[e][r] *= 2^(sign * k_r) on a field of n_rows rows of N complex doubles (N a
// power of two dividing the block size, so a thread always meets the same
// right-hand side r = index mod N).  2^k is applied as two factors 2^(k/2) and
// 2^(k - k/2), each a normal double for |k| <= 2046; the products are exact
// unless a value under- or overflows.
static __global__ void pow2_scale_kernel(double *f, size_t n_rows, int N, const OuterState *os, int sign) {
    const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    const int k = sign * os[first & (size_t)(N - 1)].scale_exp;
    if (k == 0) return;
    const double f1 = pow2_exact(k / 2), f2 = pow2_exact(k - k / 2);
    double2 *z = reinterpret_cast<double2 *>(f);
    const size_t total = n_rows * (size_t)N;
    for (size_t i = first; i < total; i += stride) {
        double2 v = z[i];
        v.x = v.x * f1 * f2;
        v.y = v.y * f1 * f2;
        z[i] = v;
    }
}

// full-system norms: mode 0 -> full_b2 (sum of two partial sets), mode 1 -> full_r2
static __global__ void full_norm_kernel(OuterState *os, const double2 *pa, int na, const double2 *pb, int nb, int N,
                                 int mode) {
    const int r = blockIdx.x;
    const double2 a = sum_partials(pa, na, N, 1, r, 0);
    const double2 b = sum_partials(pb, nb, N, 1, r, 0);
    if (threadIdx.x != 0) return;
    if (mode == 0) os[r].full_b2 = a.x + b.x;
    else os[r].full_r2 = a.x + b.x;
}

}  // namespace dl

namespace dl {
// |v|^2 per right-hand side of a half field -> partials
template <typename S, int R>
static __global__ void __launch_bounds__(256) norm2_kernel(VecArgs a, const S *v_, double2 *partials) {
    typedef typename Real<S>::type T;
    extern __shared__ __align__(128) unsigned char smem[];
    const int G = a.N / R, lgG = __ffs(G) - 1;
    const long total = (long)a.n_elem << lgG;  // elements x groups: may exceed 2^31
    cx<T> red[R][1];
#pragma unroll
    for (int k = 0; k < R; ++k) red[k][0] = zero<T>();
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int e = (int)(idx >> lgG), r0 = (int)(idx & (G - 1)) * R;
        cx<T> v[R];
        ld_pack<S, R, true>(v_ + ((size_t)e * a.N + r0) * 2, v);
#pragma unroll
        for (int k = 0; k < R; ++k) cjmac(red[k][0], v[k], v[k]);
    }
    block_reduce<R, 1, T>(red, G, a.N, partials, smem);
}

// FP64 <-> storage type S over n_complex values: to_lo = 1 rounds FP64 to S the
// way the solver's inner phase does (to float, then to S), to_lo = 0 widens S to
// FP64 exactly.
template <typename S>
static __global__ void cast_kernel(double *f64, S *lo, size_t n_complex, int to_lo) {
    typedef typename Real<S>::type T;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_complex; i += (size_t)gridDim.x * blockDim.x) {
        if (to_lo) {
            const double2 v = reinterpret_cast<const double2 *>(f64)[i];
            cx<T> z[1] = {mk((T)v.x, (T)v.y)};
            st_pack<S, 1>(lo + 2 * i, z);
        } else {
            cx<T> z[1];
            ld_pack<S, 1, false>(lo + 2 * i, z);
            reinterpret_cast<double2 *>(f64)[i] = make_double2((double)z[0].re, (double)z[0].im);
        }
    }
}

// deterministic pseudo-random fill (for timing runs only)
template <typename S>
static __global__ void fill_kernel(S *v, size_t n_complex, uint32_t seed) {
    typedef typename Real<S>::type T;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_complex; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u ^ seed;
        h ^= h >> 15; h *= 2246822519u; h ^= h >> 13;
        cx<T> z[1];
        z[0] = mk((T)((h & 0xffff) / 65536.0 - 0.5), (T)((h >> 16) / 65536.0 - 0.5));
        st_pack<S, 1>(v + 2 * i, z);
    }
}
}  // namespace dl
