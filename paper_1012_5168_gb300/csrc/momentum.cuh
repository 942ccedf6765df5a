// Momentum projection and two-point functions (Sec. 3, Eqs. 1 and 3).
//
// Loops at spatial momentum p = 2 pi n / L (n integer):
//     L_Gamma(p, t) = sum_{x in t} exp(-i p.(x - o)) eta(x)^dag Gamma phi(x),
// and the connected meson function of a point source at y (o = y):
//     C^{BA}(p, t) = - sum_x exp(-i p.(x - y)) Tr[g5 S(x)^dag g5 Gamma_B S(x) Gamma_A].
// Both run in three steps: a per-site matrix (the 4x4 spin matrix
// phi eta^dag, or the 16x16 colour-summed product of the propagator with its
// conjugate), its Fourier sum over each timeslice against a phase table, and the
// Gamma traces.  All sums are FP64 in a fixed order.  The disconnected
// function combines per-noise loops at p and -p over pairs of distinct noise
// vectors, so no noise vector is multiplied with itself.
#pragma once

#include "common.cuh"

namespace dl {

// ph[q][s] = exp(-i 2 pi sum_i n_i (x_i - o_i) / L_i), s = x + Lx (y + Ly z).
static __global__ void phase_table_kernel(double2 *ph, const int *mom, int n_mom, Geom g, int ox, int oy, int oz) {
    const int V3 = g.L[0] * g.L[1] * g.L[2];
    const int total = n_mom * V3;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int q = idx / V3, s = idx % V3;
        const int x = s % g.L[0], y = (s / g.L[0]) % g.L[1], z = s / (g.L[0] * g.L[1]);
        const int kx = ((mom[3 * q] * (x - ox)) % g.L[0] + g.L[0]) % g.L[0];
        const int ky = ((mom[3 * q + 1] * (y - oy)) % g.L[1] + g.L[1]) % g.L[1];
        const int kz = ((mom[3 * q + 2] * (z - oz)) % g.L[2] + g.L[2]) % g.L[2];
        const double frac = (double)kx / g.L[0] + (double)ky / g.L[1] + (double)kz / g.L[2];
        double sn, cs;
        sincospi(-2.0 * frac, &sn, &cs);
        ph[idx] = make_double2(cs, sn);
    }
}

struct SiteSpinArgs {
    const double *eta;  // EO tile [2][Vh][12][N]
    const double *phi;
    const uint32_t *coords;
    Geom g;
    int N, n;           // layout width, right-hand sides in use
    int t_lo, nt;       // timeslices t_lo .. t_lo + nt - 1 (nt = 1 with tcol)
    const int *tcol;    // if set: right-hand side j lives on timeslice tcol[j]
    double2 *out;       // [n][nt][V3][16]: S_{beta alpha}(x) = sum_a phi_{beta a}(x) conj(eta_{alpha a}(x))
};

// One thread per (site of the timeslice, right-hand side); j is the fastest
// index so that a warp reads contiguous right-hand sides of the EO tile.
static __global__ void site_spin_kernel(SiteSpinArgs A) {
    const int V3 = A.g.L[0] * A.g.L[1] * A.g.L[2];
    const long total = (long)A.nt * 2 * A.g.V3h * A.n;
    const size_t half = (size_t)A.g.Vh * 12 * A.N * 2;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % A.n);
        const long sp = idx / A.n;
        const int cbl = (int)(sp % A.g.V3h);
        const int p = (int)((sp / A.g.V3h) % 2);
        const int tt = (int)(sp / (2L * A.g.V3h));
        const int t = A.tcol ? A.tcol[j] : A.t_lo + tt;
        const int cb = t * A.g.V3h + cbl;
        const Site st = decode(__ldg(A.coords + (size_t)p * A.g.Vh + cb), A.g);
        const int s = st.c[0] + A.g.L[0] * (st.c[1] + A.g.L[1] * st.c[2]);
        const size_t base = (size_t)p * half + (size_t)cb * 12 * A.N * 2 + (size_t)j * 2;
        cx<double> e[12], f[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            cx<double> v[1];
            ld_pack<double, 1, true>(A.eta + base + (size_t)c * A.N * 2, v);
            e[c] = v[0];
            ld_pack<double, 1, true>(A.phi + base + (size_t)c * A.N * 2, v);
            f[c] = v[0];
        }
        double2 *o = A.out + (((size_t)j * A.nt + tt) * V3 + s) * 16;
#pragma unroll
        for (int be = 0; be < 4; ++be)
#pragma unroll
            for (int al = 0; al < 4; ++al) {
                cx<double> acc = zero<double>();
#pragma unroll
                for (int a = 0; a < 3; ++a) cjmac(acc, e[3 * al + a], f[3 * be + a]);
                o[be * 4 + al] = make_double2(acc.re, acc.im);
            }
    }
}

// out[jt][q][e] = sum_s ph[q][s] in[jt][s][e]; grid = (J*nt, ceil(Q*E / blockDim.x)).
static __global__ void fourier_kernel(const double2 *in, const double2 *ph, int V3, int E, int Q, double2 *out) {
    const int jt = blockIdx.x;
    const int o = blockIdx.y * blockDim.x + threadIdx.x;
    if (o >= Q * E) return;
    const int q = o / E, e = o % E;
    const double2 *src = in + (size_t)jt * V3 * E + e;
    const double2 *w = ph + (size_t)q * V3;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < V3; ++s) {
        const double2 a = __ldg(w + s), b = __ldg(src + (size_t)s * E);
        re = ::fma(a.x, b.x, ::fma(-a.y, b.y, re));
        im = ::fma(a.x, b.y, ::fma(a.y, b.x, im));
    }
    out[((size_t)jt * Q + q) * E + e] = make_double2(re, im);
}

// L_Gamma(p, t) = sum_{alpha beta} Gamma_{alpha beta} S_{beta alpha}(p, t):
// S [n][nt][Q][16] -> out[j][q][G][T] at t = tcol[j] or t_lo + tt.
static __global__ void mom_gamma_kernel(const double2 *S, const double2 *gammas, int n, int nt, int Q, int T, int t_lo,
                                        const int *tcol, double2 *out) {
    const int total = n * nt * Q * 16;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int G = idx % 16;
        const int q = (idx / 16) % Q;
        const int tt = (idx / (16 * Q)) % nt;
        const int j = idx / (16 * Q * nt);
        const double2 *s = S + (((size_t)j * nt + tt) * Q + q) * 16;
        double re = 0.0, im = 0.0;
        for (int al = 0; al < 4; ++al)
            for (int be = 0; be < 4; ++be) {
                const double2 gm = gammas[(G * 4 + al) * 4 + be], v = s[be * 4 + al];
                re += gm.x * v.x - gm.y * v.y;
                im += gm.x * v.y + gm.y * v.x;
            }
        const int t = tcol ? tcol[j] : t_lo + tt;
        out[(((size_t)j * Q + q) * 16 + G) * T + t] = make_double2(re, im);
    }
}

// Per site of the point-source propagator (canonical [12][V][4][3], column
// j = 3 alpha + a): P_{(beta alpha),(beta' alpha')} = sum_{a,b}
// conj(S_{beta b, alpha a}) S_{beta' b, alpha' a}.  One thread per (site, beta,
// beta'); out [V][256] with V in lexicographic order (t slowest).
static __global__ void meson_site_kernel(const double *prop, long V, double2 *out) {
    const long total = V * 16;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int bb = (int)(idx % 16);
        const long i = idx / 16;
        const int be = bb / 4, be2 = bb % 4;
        cx<double> acc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = zero<double>();
        for (int a = 0; a < 3; ++a) {
            cx<double> u[4][3], v[4][3];
#pragma unroll
            for (int al = 0; al < 4; ++al)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const double *pu = prop + (((size_t)(3 * al + a) * V + i) * 12 + be * 3 + b) * 2;
                    const double *pv = prop + (((size_t)(3 * al + a) * V + i) * 12 + be2 * 3 + b) * 2;
                    u[al][b] = mk(__ldg(pu), __ldg(pu + 1));
                    v[al][b] = mk(__ldg(pv), __ldg(pv + 1));
                }
#pragma unroll
            for (int al = 0; al < 4; ++al)
#pragma unroll
                for (int al2 = 0; al2 < 4; ++al2)
#pragma unroll
                    for (int b = 0; b < 3; ++b) cjmac(acc[al * 4 + al2], u[al][b], v[al2][b]);
        }
        double2 *o = out + (size_t)i * 256;
#pragma unroll
        for (int al = 0; al < 4; ++al)
#pragma unroll
            for (int al2 = 0; al2 < 4; ++al2)
                o[(be * 4 + al) * 16 + be2 * 4 + al2] = make_double2(acc[al * 4 + al2].re, acc[al * 4 + al2].im);
    }
}

// C^{BA}(q, t - t_src) = - sum g5_alpha g5_beta (Gamma_B)_{beta beta'} (Gamma_A)_{alpha' alpha}
//                          F_t[q][(beta alpha),(beta' alpha')];  F [T][Q][256], out [Q][16 A][16 B][T].
static __global__ void meson_gamma_kernel(const double2 *F, const double2 *gammas, int T, int Q, int t_src,
                                          double2 *out) {
    const int total = Q * 256 * T;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int t = idx % T;
        const int B = (idx / T) % 16;
        const int A = (idx / (16 * T)) % 16;
        const int q = idx / (256 * T);
        const double2 *f = F + ((size_t)t * Q + q) * 256;
        double re = 0.0, im = 0.0;
        for (int be = 0; be < 4; ++be)
            for (int be2 = 0; be2 < 4; ++be2) {
                const double2 gb = gammas[(B * 4 + be) * 4 + be2];
                if (gb.x == 0.0 && gb.y == 0.0) continue;
                for (int al2 = 0; al2 < 4; ++al2)
                    for (int al = 0; al < 4; ++al) {
                        const double2 ga = gammas[(A * 4 + al2) * 4 + al];
                        if (ga.x == 0.0 && ga.y == 0.0) continue;
                        const double sg = ((al < 2) == (be < 2)) ? 1.0 : -1.0;  // g5_alpha g5_beta
                        const double2 g = make_double2(sg * (gb.x * ga.x - gb.y * ga.y), sg * (gb.x * ga.y + gb.y * ga.x));
                        const double2 v = f[(be * 4 + al) * 16 + be2 * 4 + al2];
                        re += g.x * v.x - g.y * v.y;
                        im += g.x * v.y + g.y * v.x;
                    }
            }
        out[(((size_t)q * 16 + A) * 16 + B) * T + (t - t_src + T) % T] = make_double2(-re, -im);
    }
}

// D^{BA}(q, dt) = -(1/(V3 T)) sum_t E[L_B(q, t + dt) L_A(-q, t)], the expectation over
// pairs of distinct noise vectors n != m that cover t + dt and t respectively:
//   E = [(sum_{n in C(t+dt)} L_B^n)(sum_{m in C(t)} L_A^m) - sum_{n in both} L_B^n L_A^n]
//       / (|C(t+dt)| |C(t)| - |C(t+dt) and C(t)|).
// L [n][Q][16][T], cover [n][T] (1: the noise vector's loop covers t), minus [Q].
static __global__ void disconnected_kernel(const double2 *L, const unsigned char *cover, const int *minus, int n, int Q,
                                           int T, double norm, double2 *out) {
    const int total = Q * 256 * T;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int dt = idx % T;
        const int B = (idx / T) % 16;
        const int A = (idx / (16 * T)) % 16;
        const int q = idx / (256 * T);
        const int qm = minus[q];
        double re = 0.0, im = 0.0;
        for (int t = 0; t < T; ++t) {
            const int t2 = (t + dt) % T;
            double xr = 0, xi = 0, yr = 0, yi = 0, zr = 0, zi = 0;
            long c1 = 0, c2 = 0, c12 = 0;
            for (int k = 0; k < n; ++k) {
                const bool in1 = cover[(size_t)k * T + t2] != 0, in2 = cover[(size_t)k * T + t] != 0;
                if (!in1 && !in2) continue;
                const double2 lb = L[(((size_t)k * Q + q) * 16 + B) * T + t2];
                const double2 la = L[(((size_t)k * Q + qm) * 16 + A) * T + t];
                if (in1) { xr += lb.x; xi += lb.y; ++c1; }
                if (in2) { yr += la.x; yi += la.y; ++c2; }
                if (in1 && in2) {
                    zr += lb.x * la.x - lb.y * la.y;
                    zi += lb.x * la.y + lb.y * la.x;
                    ++c12;
                }
            }
            const long pairs = c1 * c2 - c12;
            if (pairs <= 0) continue;
            re += ((xr * yr - xi * yi) - zr) / (double)pairs;
            im += ((xr * yi + xi * yr) - zi) / (double)pairs;
        }
        out[idx] = make_double2(-norm * re, -norm * im);
    }
}

}  // namespace dl
