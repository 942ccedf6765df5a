// The Wilson hop of hop.cuh in float-float arithmetic, with the three colour
// rows of an output site on three threads.  It serves the defect-correction
// steps of mixed-precision solves (the source b_hat = b_e + kappa D_eo b_o, the
// reconstruction x_o = b_o + kappa D_oe x_e and the residual
// r = b_e - x_e + kappa D_eo x_o), whose rounding must stay far below the
// solver tolerance while GB300 issues FP64 at about 1/60 of the FP32 rate.
//
// Thread (site x, colour row a, right-hand side j) accumulates the four spin
// components of colour a of (D psi)(x).  Per direction it loads the full
// neighbour spinor, forms the two-spinor projection h(b) for each colour b
// (recomputed by the three threads of a site, which share the neighbour
// through L1), multiplies with row a of U (or column a of U^dag) and rebuilds
// the lower spins, exactly as the per-site kernel does for all rows at once.
// Holding one link row, one colour of the neighbour and a four-component
// accumulator keeps the register count at 80 (four 192-thread blocks per SM),
// where a whole-site float-float thread needed 186.  Sums are accumulated
// unnormalised (dacc: two-sum errors and low parts gathered in one float) and
// renormalised once per output component, which cut the instruction count
// and the hop time by a fifth (1.76 -> 1.40 ms at 32 right-hand sides).
//
// Formats.  The gathered field `in` is float-float: each complex occupies the
// 16 bytes of an FP64 complex as (re.hi, re.lo, im.hi, im.lo), written by
// ff_cast_kernel.  y is float-float (YFF) or FP64, z is FP64, and out is
// float-float (OFF) or FP64 (converted with integer operations only, so the
// kernel issues no FP64 arithmetic in its main loop).  Links are the
// float-float copy [2][Vh][4][9] of the FP64 field.
#pragma once

#include "hop.cuh"

namespace dl {

typedef cx<dfloat> cff;

__device__ __forceinline__ cff ld_ff(const double *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return mk(dfloat(v.x, v.y), dfloat(v.z, v.w));
}
__device__ __forceinline__ cff ld_f64_as_ff(const double *p) {
    const double2 v = *reinterpret_cast<const double2 *>(p);
    return mk(df_from_bits((uint32_t)__double2loint(v.x), (uint32_t)__double2hiint(v.x)),
              df_from_bits((uint32_t)__double2loint(v.y), (uint32_t)__double2hiint(v.y)));
}

__device__ __forceinline__ cff cadd_lazy(cff a, cff b) { return mk(df_add_lazy(a.re, b.re), df_add_lazy(a.im, b.im)); }

// Projection h = psi_up + s X_mu psi_down of colour b (s = SG), as in
// load_project: h0 is spin row 0, h1 spin row 1 (unnormalised pairs).
template <int MU, int SG>
__device__ __forceinline__ void ff_project(cff p0, cff p1, cff p2, cff p3, cff &h0, cff &h1) {
    if (MU == 0) {
        h0 = cadd_lazy(p0, SG > 0 ? ti(p3) : tmi(p3));
        h1 = cadd_lazy(p1, SG > 0 ? ti(p2) : tmi(p2));
    } else if (MU == 1) {
        h0 = cadd_lazy(p0, SG > 0 ? -p3 : p3);
        h1 = cadd_lazy(p1, SG > 0 ? p2 : -p2);
    } else if (MU == 2) {
        h0 = cadd_lazy(p0, SG > 0 ? ti(p2) : tmi(p2));
        h1 = cadd_lazy(p1, SG > 0 ? tmi(p3) : ti(p3));
    } else {
        h0 = cadd_lazy(p0, SG > 0 ? p2 : -p2);
        h1 = cadd_lazy(p1, SG > 0 ? p3 : -p3);
    }
}

// acc += [w0; w1; s X_mu^dag (w0, w1)] for one colour row (s = S), as in
// reconstruct: X^dag (w0, w1) is (-i w1, -i w0), (w1, -w0), (-i w0, i w1),
// (w0, w1) for mu = 0..3.
template <int MU, int S>
__device__ __forceinline__ void ff_reconstruct(const cdacc &w0, const cdacc &w1, cdacc (&acc)[4]) {
    constexpr int P = S > 0 ? 0 : 2;  // rotation offset of the sign s
    cda_add<0>(acc[0], w0);
    cda_add<0>(acc[1], w1);
    if (MU == 0) {
        cda_add<(3 + P) % 4>(acc[2], w1);
        cda_add<(3 + P) % 4>(acc[3], w0);
    } else if (MU == 1) {
        cda_add<(0 + P) % 4>(acc[2], w1);
        cda_add<(2 + P) % 4>(acc[3], w0);
    } else if (MU == 2) {
        cda_add<(3 + P) % 4>(acc[2], w0);
        cda_add<(1 + P) % 4>(acc[3], w1);
    } else {
        cda_add<(0 + P) % 4>(acc[2], w0);
        cda_add<(0 + P) % 4>(acc[3], w1);
    }
}

// Direction mu, forward (SG = -1: (1 - g_mu) U_mu(x) psi(x + mu)) or backward
// (SG = +1: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)), for colour row a.
template <int MU, int SG>
__device__ __forceinline__ void ff_dir(const HopArgs &A, const Site &st, int cb, int a, int j, cdacc (&acc)[4]) {
    constexpr bool FWD = SG < 0;
    const int nb = FWD ? nbr_fwd(st, A.g, MU) : nbr_bwd(st, A.g, MU);
    const bool flip = (MU == 3) && (A.g.t_bc < 0) && (st.c[3] == (FWD ? A.g.L[3] - 1 : 0));
    const double *up = reinterpret_cast<const double *>(A.gauge) +
                       2 * 9 * (FWD ? ((size_t)A.p * A.g.Vh + cb) * 4 + MU : ((size_t)(1 - A.p) * A.g.Vh + nb) * 4 + MU);
    cff u[3];  // forward: row a of U; backward: column a of U (conjugated in the product)
#pragma unroll
    for (int b = 0; b < 3; ++b) u[b] = ld_ff(up + 2 * (FWD ? a * 3 + b : b * 3 + a));
    const size_t N2 = (size_t)A.N * 2;
    const double *src = reinterpret_cast<const double *>(A.in) + ((size_t)nb * 12 * A.N + j) * 2;
    cdacc w0 = cda_zero(), w1 = cda_zero();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        cff h0, h1;
        ff_project<MU, SG>(ld_ff(src + b * N2), ld_ff(src + (3 + b) * N2), ld_ff(src + (6 + b) * N2),
                           ld_ff(src + (9 + b) * N2), h0, h1);
        if (flip) {
            h0 = -h0;
            h1 = -h1;
        }
        cda_mac<!FWD>(w0, u[b], h0);
        cda_mac<!FWD>(w1, u[b], h1);
    }
    ff_reconstruct<MU, SG>(w0, w1, acc);
}

// out = c D in (PLAIN), y + c D in (XPAY) or z - y - c D in (RESID) on the
// output parity p, sites [cb_begin, cb_end); RED = RED_NORM adds <out, out>
// per right-hand side to partials (block_reduce).  blockDim.x must be a
// multiple of 3 N (three rows of N right-hand sides per site).
template <int MODE, int RED, bool YFF, bool OFF>
__global__ void __launch_bounds__(192, 4) hop_ff_rows_kernel(HopArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int G = A.N;
    const int lgG = __ffs(G) - 1;
    const long total = ((long)(A.cb_end - A.cb_begin) * 3) << lgG;
    const dfloat cD = df_from_double(A.c);
    cff red[1][1];
    red[0][0] = zero<dfloat>();
    const double *yd = reinterpret_cast<const double *>(A.y);
    const double *zd = reinterpret_cast<const double *>(A.z);
    double *od = reinterpret_cast<double *>(A.out);
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int j = (int)idx & (G - 1);
        const long q = idx >> lgG;
        const int a = (int)(q % 3);
        const int cb = A.cb_begin + (int)(q / 3);
        const Site st = decode(__ldg(A.coords + (size_t)A.p * A.g.Vh + cb), A.g);
        cdacc acc[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[s] = cda_zero();
        ff_dir<0, -1>(A, st, cb, a, j, acc);
        ff_dir<0, +1>(A, st, cb, a, j, acc);
        ff_dir<1, -1>(A, st, cb, a, j, acc);
        ff_dir<1, +1>(A, st, cb, a, j, acc);
        ff_dir<2, -1>(A, st, cb, a, j, acc);
        ff_dir<2, +1>(A, st, cb, a, j, acc);
        ff_dir<3, -1>(A, st, cb, a, j, acc);
        ff_dir<3, +1>(A, st, cb, a, j, acc);
        const size_t base = ((size_t)cb * 12 * A.N + j) * 2;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const size_t off = base + (size_t)(3 * s + a) * A.N * 2;
            cff o = mk(cD * da_norm(acc[s].re), cD * da_norm(acc[s].im));
            if (MODE == MODE_XPAY || MODE == MODE_RESID) {
                const cff yv = YFF ? ld_ff(yd + off) : ld_f64_as_ff(yd + off);
                if (MODE == MODE_XPAY) o = yv + o;
                else o = ld_f64_as_ff(zd + off) - yv - o;
            }
            if (OFF)
                *reinterpret_cast<float4 *>(od + off) = make_float4(o.re.hi, o.re.lo, o.im.hi, o.im.lo);
            else
                *reinterpret_cast<double2 *>(od + off) = make_double2(df_to_f64(o.re), df_to_f64(o.im));
            if (RED == RED_NORM) {
                red[0][0].re = df_fma(o.re, o.re, red[0][0].re);
                red[0][0].re = df_fma(o.im, o.im, red[0][0].re);
            }
        }
    }
    if (RED != RED_NONE) block_reduce<1, 1, dfloat>(red, G, A.N, A.partials, smem);
}

// dst[i] = src[i] for n complex values, FP64 -> float-float (to_ff) or back,
// with integer operations only; in place when dst == src.
static __global__ void ff_cast_kernel(const double *src, double *dst, long n, int to_ff) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if (to_ff) {
            const double2 v = reinterpret_cast<const double2 *>(src)[i];
            const dfloat re = df_from_bits((uint32_t)__double2loint(v.x), (uint32_t)__double2hiint(v.x));
            const dfloat im = df_from_bits((uint32_t)__double2loint(v.y), (uint32_t)__double2hiint(v.y));
            reinterpret_cast<float4 *>(dst)[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
        } else {
            const float4 v = reinterpret_cast<const float4 *>(src)[i];
            reinterpret_cast<double2 *>(dst)[i] =
                make_double2(df_to_f64(dfloat(v.x, v.y)), df_to_f64(dfloat(v.z, v.w)));
        }
    }
}

}  // namespace dl
