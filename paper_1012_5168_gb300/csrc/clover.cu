// Clover blocks A and A^-1 per site, and A or A^-1 applied to FP64 half fields.
#include "launch.h"

namespace dl {

// The link U_mu at (x, y, z, t), coordinates taken modulo the extents, from the
// FP64 field in even-odd site order [2][Vh][4][9].
__device__ __forceinline__ void m3_load(const double2 *g64, const Geom &g, int x, int y, int z, int t, int mu,
                                        cx<double> (&u)[9]) {
    x = (x + g.L[0]) % g.L[0];
    y = (y + g.L[1]) % g.L[1];
    z = (z + g.L[2]) % g.L[2];
    t = (t + g.L[3]) % g.L[3];
    const int i = x + g.stride[1] * y + g.stride[2] * z + g.stride[3] * t;
    const int p = (x + y + z + t) & 1;
    const double2 *src = g64 + (((size_t)p * g.Vh + (i >> 1)) * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = mk(src[k].x, src[k].y);
}
// c = op(a) op(b) for 3 x 3 complex matrices, op the conjugate transpose where
// DA (for a) or DB (for b) is set.
template <bool DA, bool DB>
__device__ __forceinline__ void m3_mul(const cx<double> (&a)[9], const cx<double> (&b)[9], cx<double> (&c)[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = zero<double>();
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const cx<double> x = DA ? cj(a[k * 3 + i]) : a[i * 3 + k];
                const cx<double> y = DB ? cj(b[j * 3 + k]) : b[k * 3 + j];
                s = s + x * y;
            }
            c[i * 3 + j] = s;
        }
}

// Per site: the six F_{mu nu}, the two 6 x 6 blocks of A and their inverses
// (Gauss-Jordan with partial pivoting, FP64).  One thread per lexicographic site.
static __global__ void clover_build_kernel(const double2 *g64, Geom g, SigmaBlocks sig, double kcsw, double2 *a64,
                                           double2 *ainv64, float2 *ainv32, __nv_bfloat162 *ainv16) {
    const int V = 2 * g.Vh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
        const int x = i % g.L[0], y = (i / g.stride[1]) % g.L[1], z = (i / g.stride[2]) % g.L[2], t = i / g.stride[3];
        const int c0[4] = {x, y, z, t};
        cx<double> blk[2][6][6];
        for (int b = 0; b < 2; ++b)
            for (int r = 0; r < 6; ++r)
                for (int s = 0; s < 6; ++s) blk[b][r][s] = mk(r == s ? 1.0 : 0.0, 0.0);
        int plane = 0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
                int e[4][4];  // e[m] = unit step in direction m
                for (int m = 0; m < 4; ++m)
                    for (int k = 0; k < 4; ++k) e[m][k] = (m == k);
                auto at = [&](int dm, int dn, int dir, cx<double> (&u)[9]) {
                    m3_load(g64, g, c0[0] + dm * e[mu][0] + dn * e[nu][0], c0[1] + dm * e[mu][1] + dn * e[nu][1],
                            c0[2] + dm * e[mu][2] + dn * e[nu][2], c0[3] + dm * e[mu][3] + dn * e[nu][3], dir, u);
                };
                cx<double> q[9], u1[9], u2[9], u3[9], u4[9], t1[9], t2[9], t3[9];
                for (int k = 0; k < 9; ++k) q[k] = zero<double>();
                // x -> x+mu -> x+mu+nu -> x+nu -> x : U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
                at(0, 0, mu, u1); at(1, 0, nu, u2); at(0, 1, mu, u3); at(0, 0, nu, u4);
                m3_mul<false, false>(u1, u2, t1); m3_mul<false, true>(t1, u3, t2); m3_mul<false, true>(t2, u4, t3);
                for (int k = 0; k < 9; ++k) q[k] = q[k] + t3[k];
                // x -> x+nu -> x+nu-mu -> x-mu -> x : U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
                at(0, 0, nu, u1); at(-1, 1, mu, u2); at(-1, 0, nu, u3); at(-1, 0, mu, u4);
                m3_mul<false, true>(u1, u2, t1); m3_mul<false, true>(t1, u3, t2); m3_mul<false, false>(t2, u4, t3);
                for (int k = 0; k < 9; ++k) q[k] = q[k] + t3[k];
                // x -> x-mu -> x-mu-nu -> x-nu -> x : U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
                at(-1, 0, mu, u1); at(-1, -1, nu, u2); at(-1, -1, mu, u3); at(0, -1, nu, u4);
                m3_mul<true, true>(u1, u2, t1); m3_mul<false, false>(t1, u3, t2); m3_mul<false, false>(t2, u4, t3);
                for (int k = 0; k < 9; ++k) q[k] = q[k] + t3[k];
                // x -> x-nu -> x-nu+mu -> x+mu -> x : U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
                at(0, -1, nu, u1); at(0, -1, mu, u2); at(1, -1, nu, u3); at(0, 0, mu, u4);
                m3_mul<true, false>(u1, u2, t1); m3_mul<false, false>(t1, u3, t2); m3_mul<false, true>(t2, u4, t3);
                for (int k = 0; k < 9; ++k) q[k] = q[k] + t3[k];
                // F = (Q - Q^dag) / (8 i); z / (8 i) = (Im z, -Re z) / 8
                cx<double> F[9];
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) {
                        const cx<double> d = q[a * 3 + c] - cj(q[c * 3 + a]);
                        F[a * 3 + c] = mk(d.im / 8.0, -d.re / 8.0);
                    }
                // A -= kappa c_sw sigma (x) F on each block
                for (int b = 0; b < 2; ++b)
                    for (int s1 = 0; s1 < 2; ++s1)
                        for (int s2 = 0; s2 < 2; ++s2) {
                            const cx<double> sg = mk(sig.s[plane][b][s1][s2].x, sig.s[plane][b][s1][s2].y);
                            if (sg.re == 0.0 && sg.im == 0.0) continue;
                            for (int a = 0; a < 3; ++a)
                                for (int c = 0; c < 3; ++c)
                                    blk[b][3 * s1 + a][3 * s2 + c] = blk[b][3 * s1 + a][3 * s2 + c] - kcsw * (sg * F[a * 3 + c]);
                        }
            }
        const int p = (x + y + z + t) & 1;
        const size_t base = ((size_t)p * g.Vh + (i >> 1)) * 72;
        for (int b = 0; b < 2; ++b) {
            cx<double> aug[6][12];
            for (int r = 0; r < 6; ++r)
                for (int s = 0; s < 6; ++s) {
                    a64[base + b * 36 + r * 6 + s] = make_double2(blk[b][r][s].re, blk[b][r][s].im);
                    aug[r][s] = blk[b][r][s];
                    aug[r][6 + s] = mk(r == s ? 1.0 : 0.0, 0.0);
                }
            for (int col = 0; col < 6; ++col) {
                int piv = col;
                double best = -1.0;
                for (int r = col; r < 6; ++r) {
                    const double m = aug[r][col].re * aug[r][col].re + aug[r][col].im * aug[r][col].im;
                    if (m > best) { best = m; piv = r; }
                }
                if (piv != col)
                    for (int s = 0; s < 12; ++s) {
                        const cx<double> tmp = aug[col][s];
                        aug[col][s] = aug[piv][s];
                        aug[piv][s] = tmp;
                    }
                const cx<double> d = aug[col][col];
                const double dd = d.re * d.re + d.im * d.im;
                const cx<double> inv = mk(d.re / dd, -d.im / dd);  // 1/d (a zero pivot gives non-finite values)
                for (int s = 0; s < 12; ++s) aug[col][s] = aug[col][s] * inv;
                for (int r = 0; r < 6; ++r) {
                    if (r == col) continue;
                    const cx<double> f = aug[r][col];
                    for (int s = 0; s < 12; ++s) aug[r][s] = aug[r][s] - f * aug[col][s];
                }
            }
            for (int r = 0; r < 6; ++r)
                for (int s = 0; s < 6; ++s) {
                    const cx<double> v = aug[r][6 + s];
                    const size_t k = base + b * 36 + r * 6 + s;
                    ainv64[k] = make_double2(v.re, v.im);
                    ainv32[k] = make_float2((float)v.re, (float)v.im);
                    ainv16[k] = __floats2bfloat162_rn((float)v.re, (float)v.im);
                }
        }
    }
}

// out = mat x in on the half field of parity p ([Vh][12][N] complex doubles), or
// with s != 0 out += s (in - mat x in); one thread per (site, block, right-hand
// side); out may equal in.
static __global__ void clover_mul_kernel(const double2 *mat, int p, int Vh, int N, const double2 *in, double2 *out,
                                         double s) {
    const long total = (long)Vh * 2 * N;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int r = (int)(idx % N);
        const int b = (int)((idx / N) % 2);
        const long cb = idx / (2L * N);
        const double2 *m = mat + ((size_t)p * Vh + cb) * 72 + b * 36;
        cx<double> v[6];
        for (int j = 0; j < 6; ++j) {
            const double2 w = in[(cb * 12 + 6 * b + j) * (size_t)N + r];
            v[j] = mk(w.x, w.y);
        }
        for (int i = 0; i < 6; ++i) {
            cx<double> o = zero<double>();
            for (int j = 0; j < 6; ++j) cmac(o, mk(m[i * 6 + j].x, m[i * 6 + j].y), v[j]);
            double2 &w = out[(cb * 12 + 6 * b + i) * (size_t)N + r];
            if (s != 0.0) w = make_double2(w.x + s * (v[i].re - o.re), w.y + s * (v[i].im - o.im));
            else w = make_double2(o.re, o.im);
        }
    }
}

cudaError_t launch_clover_build(const double *g64, const Geom &g, const SigmaBlocks &sig, double kcsw, double2 *a64,
                               double2 *ainv64, float2 *ainv32, __nv_bfloat162 *ainv16, int grid, cudaStream_t s) {
    clover_build_kernel<<<grid, 128, 0, s>>>(reinterpret_cast<const double2 *>(g64), g, sig, kcsw, a64, ainv64, ainv32,
                                             ainv16);
    return cudaGetLastError();
}

cudaError_t launch_clover_mul(const double2 *mat, int p, int Vh, int N, const double *in, double *out, double acc_s,
                             int grid, cudaStream_t s) {
    clover_mul_kernel<<<grid, 256, 0, s>>>(mat, p, Vh, N, reinterpret_cast<const double2 *>(in),
                                           reinterpret_cast<double2 *>(out), acc_s);
    return cudaGetLastError();
}

}  // namespace dl
