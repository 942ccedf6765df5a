// Host-side launchers for the kernel templates.  Each precision's Wilson-hop
// and vector kernels are instantiated in their own translation unit
// (hop_f64.cu; hop_f32*.cu and hop_bf16*.cu, one per R) so the build compiles them in parallel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "hop.cuh"
#include "blas.cuh"

namespace dl {

// Storage precisions.  P_DFF is internal to the Wilson hop: FP64 storage
// (float-float gathered field), float-float arithmetic (defect correction).
// P_F32P: FP32 storage in the paired layout (f32p, common.cuh), the inner
// fields of FP32 solves of even width when the context uses it.
enum { P_F64 = 0, P_F32 = 1, P_BF16 = 2, P_DFF = 3, P_F32P = 4 };

struct Launch {
    int grid;
    int block;
    size_t smem;
    cudaStream_t stream;
    int num_sms;  // > 0: the launcher clamps grid to num_sms x resident blocks of the kernel
};

// Resident blocks per SM of `kernel` at this block size and dynamic shared
// memory, cached per (kernel, block, shared memory).  The cache is guarded by a
// mutex so that contexts used from several host threads may share it.  (Kernels
// of one signature share this function's statics, so the kernel must be part of
// the key: a cache keyed on the shape alone once handed the residency of a
// 255-register kernel to a 64-register one and shrank its grid fourfold.)
template <typename K>
inline int resident_blocks(K kernel, int block, size_t smem) {
    static std::mutex m;
    static std::map<std::tuple<const void *, int, size_t>, int> cache;
    const auto key = std::make_tuple(reinterpret_cast<const void *>(kernel), block, smem);
    {
        std::lock_guard<std::mutex> g(m);
        const auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess || n < 1) n = 1;
    std::lock_guard<std::mutex> g(m);
    cache[key] = n;
    return n;
}
// Largest block (a multiple of `unit` threads, at most the kernel's limit) that maximises the
// resident threads per SM of `kernel`; smem_per_warp bytes of dynamic shared
// memory per warp.  *resident receives the blocks per SM at that size.
template <typename K>
inline int widest_block(K kernel, int unit, size_t smem_per_warp, int *resident) {
    int best = unit, best_thr = 0, best_res = 1;
    cudaFuncAttributes fa;
    const int max_thr = cudaFuncGetAttributes(&fa, kernel) == cudaSuccess ? fa.maxThreadsPerBlock : 256;
    for (int b = max_thr / unit * unit; b >= unit; b -= unit) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, b, smem_per_warp * (b / 32)) != cudaSuccess) continue;
        if (n * b > best_thr) {
            best_thr = n * b;
            best = b;
            best_res = n;
        }
    }
    *resident = best_res < 1 ? 1 : best_res;
    return best;
}

// Resident blocks, at most 16 per SM (the partial-sum buffers are sized for that).
inline void clamp_grid(Launch &l, int resident) {
    if (l.num_sms > 0) {
        const int cap = l.num_sms * (resident < 16 ? resident : 16);
        if (l.grid > cap) l.grid = cap;
    }
}

// Wilson hop; R = right-hand sides per thread (1, 2 or 4).  l.grid may be
// lowered to the kernel's residency (l.num_sms > 0); the launch used is left in l.
// Returns cudaErrorInvalidValue for a combination that is not instantiated.
cudaError_t launch_hop_f64(int R, int mode, int red, const HopArgs &a, Launch &l);
// The same hop in float-float arithmetic, one colour row per thread
// (hop_ff.cuh): a.in is a float-float field, a.gauge the float-float link copy
// [2][Vh][4][9] x (re.hi, re.lo, im.hi, im.lo); fmt flags FF_Y (y float-float,
// else FP64) and FF_OUT (out float-float, else FP64); z is FP64.  l.block is a
// multiple of 3 N.
enum { FF_Y = 1, FF_OUT = 2 };
cudaError_t launch_hop_ff(int mode, int red, int fmt, const HopArgs &a, Launch &l);
// n_complex values FP64 -> float-float (to_ff = 1) or back; dst may equal src.
cudaError_t launch_ff_cast(const double *src, double *dst, size_t n_complex, int to_ff, int grid, cudaStream_t s);
// kind (low precision only): 0 direct loads; 1 cp.async prefetching kernel,
// dynamic shared memory pf_stage_bytes(prec, R) * 2 * block; 2 bulk-copy
// staged kernel, dynamic shared memory tma_smem_bytes(prec, N, block / (N/R));
// 3 direct loads with one contiguous site range per block, the widest resident
// block and one wave of blocks (the launcher sets block, grid and shared memory);
// 4 warp-staged bulk copies, one site per warp, N = 32 R only (the launcher sets
// block, grid and shared memory; other widths return cudaErrorInvalidValue).
cudaError_t launch_hop_f32(int R, int mode, int red, int kind, const HopArgs &a, Launch &l);
cudaError_t launch_hop_f32p(int R, int mode, int red, int kind, const HopArgs &a, Launch &l);
cudaError_t launch_hop_bf16(int R, int mode, int red, int kind, const HopArgs &a, Launch &l);

// TMA_STAGES stages of `sites` neighbour blocks [12][N], two link rows and two
// neighbour-table rows per site
constexpr int TMA_STAGES = 4;
inline size_t tma_smem_bytes(int prec, int N, int sites) {
    const size_t cb = prec == P_F32 ? 8 : (prec == P_BF16 ? 4 : 16);  // bytes of one complex
    return 128 + TMA_STAGES * (size_t)sites * 12 * N * cb + 2 * (size_t)sites * 72 * cb + 2 * (size_t)sites * 8 * 4;
}

inline size_t pf_stage_bytes(int prec, int R) {
    const int sb = prec == P_F32 ? 4 : (prec == P_BF16 ? 2 : 8);  // bytes of one real
    return (size_t)12 * R * 2 * sb + (size_t)9 * 2 * sb;
}

// Vector kernels of the inner iteration, per storage precision.
struct VecLaunch {
    int prec;  // P_*
    int R;
    VecArgs a;
    Launch l;
};
cudaError_t launch_axpy_s(const VecLaunch &v, const RhsState *st, const void *r, const void *vv, void *s);
cudaError_t launch_update(const VecLaunch &v, const RhsState *st, void *x, void *r, void *p, const void *s,
                          const void *t, const void *vv);
cudaError_t launch_inner_init(const VecLaunch &v, const OuterState *os, const RhsState *st, const double *r64,
                              void *x, void *r, void *rhat, void *p, double2 *partials, int restart);
cudaError_t launch_accumulate(const VecLaunch &v, const OuterState *os, const void *x, double *x64);
cudaError_t launch_norm2(const VecLaunch &v, const void *x, double2 *partials);
// CG on the normal equations (blas.cuh)
cudaError_t launch_cg_init(const VecLaunch &v, const OuterState *os, const double *r64, void *x, void *r5,
                           double2 *partials);
cudaError_t launch_cg_update(const VecLaunch &v, const RhsState *st, void *x, void *r5, const void *p, const void *w,
                             double2 *partials);
cudaError_t launch_cg_p(const VecLaunch &v, const RhsState *st, const void *u, void *p, int init);
cudaError_t launch_fill(int prec, void *x, size_t n_complex, uint32_t seed, cudaStream_t s);
cudaError_t launch_cast(int prec, double *f64, void *lo, size_t n_complex, int to_lo, int grid, cudaStream_t s);
// Clover term (clover.cu): the blocks A = 1 - kappa c_sw sum sigma F and their inverses
// from the FP64 links (kcsw = kappa c_sw), and out = mat x in on one parity's half field
// ([Vh][12][N] complex doubles; in place allowed), or, for acc_s != 0,
// out += acc_s (in - mat x in).
cudaError_t launch_clover_build(const double *g64, const Geom &g, const SigmaBlocks &sig, double kcsw, double2 *a64,
                               double2 *ainv64, float2 *ainv32, __nv_bfloat162 *ainv16, int grid, cudaStream_t s);
cudaError_t launch_clover_mul(const double2 *mat, int p, int Vh, int N, const double *in, double *out, double acc_s,
                             int grid, cudaStream_t s);

}  // namespace dl
