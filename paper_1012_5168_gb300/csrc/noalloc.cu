// dl_trace_loops_noalloc: the local loop contraction without any device
// allocation.
//
// Some callers cannot call cudaMalloc.  Code running while a stream is being
// captured into a CUDA graph may not allocate.  Host programs with a fixed
// device-memory budget hand every byte to their own allocator up front.
// Plug-ins that live inside another application's CUDA context must not grow
// its footprint behind its back.  These callers cannot create a dl_ctx, which
// allocates its gauge copy and workspaces.  This entry point computes the
// same per-timeslice loops as dl_trace_loops with a local sink, directly from
// canonical fields, and keeps its per-block partial sums in a fixed-size
// file-scope device array.
//
// That array (4 MiB) belongs to the library's device module.  It comes into
// being on a device when that module is first used there (with CUDA's lazy
// module loading: the first call of any kernel of this library on that device)
// and is held until the process exits.  All calls share it and it keeps the
// contents of the last call; every slot a call reads is written earlier in
// the same call, so nothing has to start at zero.  Two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on
// the array and give wrong results: serialise them.
#include <cuda_runtime.h>

#include <cstdio>

#include "dloops.h"

namespace {

constexpr int kScratchElems = 1 << 18;  // double2 entries: 4 MiB
__device__ __align__(256) double2 g_loop_scratch[kScratchElems];

// The 16 Gamma matrices of the library's basis and order (1, g1..g4, g5,
// g5 g_mu, g_mu g_nu for mu < nu; chiral DeGrand-Rossi g_mu), [G][row][col]
// as (re, im) pairs, built at compile time so that no upload is needed.
struct Cplx {
    double re, im;
};
struct Mat4 {
    Cplx a[4][4];
};
struct GammaTable {
    double v[16 * 16 * 2];
};
constexpr Cplx cmul(Cplx x, Cplx y) { return Cplx{x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re}; }
constexpr Mat4 mmul(const Mat4 &x, const Mat4 &y) {
    Mat4 r{};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            Cplx s{0.0, 0.0};
            for (int k = 0; k < 4; ++k) {
                const Cplx p = cmul(x.a[i][k], y.a[k][j]);
                s = Cplx{s.re + p.re, s.im + p.im};
            }
            r.a[i][j] = s;
        }
    return r;
}
constexpr Mat4 gamma_mu(int mu) {
    const Cplx O{0, 0}, I{0, 1}, mI{0, -1}, P{1, 0}, mP{-1, 0};
    Mat4 g{};
    const Cplx t[4][4][4] = {
        {{O, O, O, I}, {O, O, I, O}, {O, mI, O, O}, {mI, O, O, O}},
        {{O, O, O, mP}, {O, O, P, O}, {O, P, O, O}, {mP, O, O, O}},
        {{O, O, I, O}, {O, O, O, mI}, {mI, O, O, O}, {O, I, O, O}},
        {{O, O, P, O}, {O, O, O, P}, {P, O, O, O}, {O, P, O, O}},
    };
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) g.a[i][j] = t[mu][i][j];
    return g;
}
constexpr GammaTable make_gamma_table() {
    Mat4 m[16] = {};
    for (int i = 0; i < 4; ++i) m[0].a[i][i] = Cplx{1.0, 0.0};
    for (int mu = 0; mu < 4; ++mu) m[1 + mu] = gamma_mu(mu);
    m[5] = mmul(mmul(mmul(gamma_mu(0), gamma_mu(1)), gamma_mu(2)), gamma_mu(3));
    for (int mu = 0; mu < 4; ++mu) m[6 + mu] = mmul(m[5], gamma_mu(mu));
    int n = 10;
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b) m[n++] = mmul(gamma_mu(a), gamma_mu(b));
    GammaTable t{};
    for (int G = 0; G < 16; ++G)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                t.v[((G * 4 + i) * 4 + j) * 2] = m[G].a[i][j].re;
                t.v[((G * 4 + i) * 4 + j) * 2 + 1] = m[G].a[i][j].im;
            }
    return t;
}
__constant__ GammaTable c_gamma16 = make_gamma_table();

}  // namespace

// Records the message returned by dl_last_error (defined in api.cu).
__attribute__((visibility("hidden"))) int dl_record_error(int code, const char *msg);

namespace {

int fail(int code, const char *msg) { return dl_record_error(code, msg); }

// The device address of the scratch array on the current device (host code
// may not use the symbol itself: there it names a host-side stand-in).  It is
// looked up on every call, which allocates nothing and stays valid across a
// cudaDeviceReset or a new primary context.
int scratch_address(void **ptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_loop_scratch);
    if (e != cudaSuccess || p == nullptr) {
        static thread_local char msg[160];
        snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the loop scratch array failed: %s", cudaGetErrorString(e));
        return fail(DL_ECUDA, msg);
    }
    *ptr = p;
    return DL_OK;
}

// partials[((j * nt + tt) * nbx + bx) * 16 + k] = sum over this block's sites of
// S_k, S_{beta*4+alpha} = sum_a phi_{beta a} conj(eta_{alpha a}), at timeslice t_lo + tt.
__global__ void __launch_bounds__(128) contract_canonical_kernel(const double2 *eta, const double2 *phi, long V,
                                                                 long V3, int t_lo, int nt, double2 *partials) {
    const int bx = blockIdx.x, tt = blockIdx.y, j = blockIdx.z;
    const int nbx = gridDim.x;
    double2 acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = make_double2(0.0, 0.0);
    const long site0 = (long)(t_lo + tt) * V3;
    for (long s = (long)bx * blockDim.x + threadIdx.x; s < V3; s += (long)nbx * blockDim.x) {
        const double2 *e = eta + ((size_t)j * V + site0 + s) * 12;
        const double2 *f = phi + ((size_t)j * V + site0 + s) * 12;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double2 ev[4], fv[4];
#pragma unroll
            for (int sp = 0; sp < 4; ++sp) {
                ev[sp] = e[3 * sp + a];
                fv[sp] = f[3 * sp + a];
            }
#pragma unroll
            for (int be = 0; be < 4; ++be)
#pragma unroll
                for (int al = 0; al < 4; ++al) {
                    double2 &o = acc[be * 4 + al];  // phi_be * conj(eta_al)
                    o.x += fv[be].x * ev[al].x + fv[be].y * ev[al].y;
                    o.y += fv[be].y * ev[al].x - fv[be].x * ev[al].y;
                }
        }
    }
    __shared__ double2 red[4][16];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        double x = acc[k].x, y = acc[k].y;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, off);
            y += __shfl_xor_sync(0xffffffffu, y, off);
        }
        if (lane == 0) red[warp][k] = make_double2(x, y);
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            x += red[w][threadIdx.x].x;
            y += red[w][threadIdx.x].y;
        }
        partials[(((size_t)j * nt + tt) * nbx + bx) * 16 + threadIdx.x] = make_double2(x, y);
    }
}

// out[j][G][t] = sum_{alpha beta} Gamma_{alpha beta} S_{beta alpha}(t); zero outside [t_lo, t_lo + nt).
__global__ void finish_kernel(const double2 *partials, int nbx, int nt, int t_lo, int T, int n, double2 *out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * 16 * T) return;
    const int t = idx % T;
    const int G = (idx / T) % 16;
    const int j = idx / (16 * T);
    double2 r = make_double2(0.0, 0.0);
    const int tt = t - t_lo;
    if (tt >= 0 && tt < nt) {
        double2 S[16];
        for (int k = 0; k < 16; ++k) {
            double x = 0.0, y = 0.0;
            for (int b = 0; b < nbx; ++b) {
                const double2 v = partials[(((size_t)j * nt + tt) * nbx + b) * 16 + k];
                x += v.x;
                y += v.y;
            }
            S[k] = make_double2(x, y);
        }
        for (int al = 0; al < 4; ++al)
            for (int be = 0; be < 4; ++be) {
                const double2 g = make_double2(c_gamma16.v[((G * 4 + al) * 4 + be) * 2],
                                               c_gamma16.v[((G * 4 + al) * 4 + be) * 2 + 1]);
                const double2 s = S[be * 4 + al];
                r.x += g.x * s.x - g.y * s.y;
                r.y += g.x * s.y + g.y * s.x;
            }
    }
    out[idx] = r;
}

}  // namespace

extern "C" int dl_trace_loops_noalloc(const void *dev_eta, const void *dev_phi, int n_rhs, const int dims[4], int t_lo,
                                      int t_hi, void *dev_out, void *cuda_stream) {
    if (!dims) return fail(DL_EINVAL, "null dims");
    for (int m = 0; m < 4; ++m)
        if (dims[m] < 1 || dims[m] > 256) return fail(DL_EINVAL, "lattice extents must lie in [1, 256]");
    const int T = dims[3];
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    if (t_lo < 0 || t_hi > T || t_lo >= t_hi) return fail(DL_EINVAL, "bad timeslice range");
    if (n_rhs == 0) return DL_OK;
    if (!dev_eta || !dev_phi || !dev_out) return fail(DL_EINVAL, "null field pointer");
    const int nt = t_hi - t_lo;
    if ((long)n_rhs * nt * 16 > kScratchElems)
        return fail(DL_EINVAL, "n_rhs * (t_hi - t_lo) exceeds 16384, the capacity of the fixed scratch array");
    if ((long)n_rhs > 65535 || (long)n_rhs * 16 * T > (1L << 30)) return fail(DL_EINVAL, "too many right-hand sides");
    // An error left by the caller's own earlier CUDA work is reported as such
    // and left in place (cudaPeekAtLastError does not clear it).
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        static thread_local char msg[160];
        snprintf(msg, sizeof(msg), "an earlier CUDA error is pending in this thread: %s", cudaGetErrorString(pending));
        return fail(DL_ECUDA, msg);
    }
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != DL_OK) return rc;
    const long V3 = (long)dims[0] * dims[1] * dims[2];
    const long V = V3 * T;
    const int block = 128;
    long nbx = (V3 + block - 1) / block;
    if (nbx > 64) nbx = 64;
    const long cap = kScratchElems / ((long)n_rhs * nt * 16);
    if (nbx > cap) nbx = cap;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    dim3 grid((unsigned)nbx, (unsigned)nt, (unsigned)n_rhs);
    contract_canonical_kernel<<<grid, block, 0, s>>>((const double2 *)dev_eta, (const double2 *)dev_phi, V, V3, t_lo,
                                                     nt, (double2 *)scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DL_ECUDA, "contraction kernel launch failed");
    const int cnt = n_rhs * 16 * T;
    finish_kernel<<<(cnt + 127) / 128, 128, 0, s>>>((const double2 *)scratch, (int)nbx, nt, t_lo, T, n_rhs,
                                                     (double2 *)dev_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DL_ECUDA, "Gamma-trace kernel launch failed");
    return DL_OK;
}
