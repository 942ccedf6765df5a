// Wilson hop with a private bulk-copy ring per warp ("warp-staged").
//
// A warp owns one output site at a time with all N = 32 R right-hand sides of
// it (lane l holds right-hand sides l R .. l R + R - 1).  The inputs of one hop
// direction are the neighbour's spinor block [12][N] (one contiguous run of
// the even-odd tile layout) and, with the first direction of a site, the
// site's row of eight links; each is one cp.async.bulk copy (the TMA engine)
// into the warp's own ring of NST stages, completed on the stage's mbarrier.
// Lane 0 keeps NST - 1 directions in flight while the warp computes the
// current one from shared memory, so the memory system sees NST - 1 blocks
// per warp in flight without registers held for loads, and no warp ever
// waits for another: there is no block-wide barrier until the final
// reduction.  The warp walks the sites gw, gw + W, gw + 2 W, ... (W warps in
// the grid), the same interleaving as the direct kernel, so the eight reads
// of each neighbour block meet in L2.
//
// Shared memory per warp: NST stages of the neighbour block, two link rows
// (the next site's links land while the current site still uses its own) and
// the NST mbarriers.
//
// Every wait is bounded: when one runs out, the warp records A.err[0], stops,
// waits (bounded again) for the copies it has issued, and leaves the site
// loop; if a drain wait runs out as well it records A.err[1] (copies may then
// land after the block exits; the host stops using the context).
#pragma once

#include "hop_tma.cuh"

namespace dl {

constexpr int WS_WARPS = 4;  // warps per block of the warp-staged hop

// Stages per warp (NSTO = 0): enough blocks in flight to cover the memory
// latency, small enough that four 4-warp blocks fit in one SM's shared memory.
// NSTO = 2 (kernel kind 11) keeps one copy in flight and so fits about twice
// the warps per SM: on GB300 that runs the fused hops faster (their epilogue
// loads gain from the extra warps) and the plain hop slower.
template <typename S, int R, int NSTO = 0>
struct WsShape {
    static constexpr uint32_t SB = 12u * 32u * R * cbytes<S>();  // one neighbour block [12][N]
    static constexpr uint32_t LB = 8u * 9u * cbytes<S>();        // one site's eight links
    static constexpr int NST = NSTO ? NSTO : (SB <= 1536 ? 6 : (SB <= 3072 ? 4 : 3));
    static constexpr size_t WB = 64 + (size_t)NST * SB + 2 * (size_t)LB;  // bytes per warp
};

// Checkerboard index of the neighbour in hop direction d (d = 2 mu: x + mu,
// d = 2 mu + 1: x - mu), without indexing the site arrays by a run-time mu.
__device__ __forceinline__ int nbr_of_dir(const Site &s, const Geom &g, int d) {
    const int mu = d >> 1;
    const int c = mu == 0 ? s.c[0] : (mu == 1 ? s.c[1] : (mu == 2 ? s.c[2] : s.c[3]));
    const int L = mu == 0 ? g.L[0] : (mu == 1 ? g.L[1] : (mu == 2 ? g.L[2] : g.L[3]));
    const int st = mu == 0 ? g.stride[0] : (mu == 1 ? g.stride[1] : (mu == 2 ? g.stride[2] : g.stride[3]));
    int i;
    if ((d & 1) == 0) {
        i = s.i + st;
        if (c == L - 1) i -= L * st;
    } else {
        i = s.i - st;
        if (c == 0) i += L * st;
    }
    return i >> 1;
}

template <typename S, int R, int MODE, int RED, int NSTO = 0>
__global__ void __launch_bounds__(WS_WARPS * 32) hop_kernel_ws(HopArgs A) {
    typedef typename Real<S>::type T;
    typedef WsShape<S, R, NSTO> W;
    constexpr int N = 32 * R;
    constexpr int NST = W::NST;
    constexpr int NV = RedCount<RED>::n > 0 ? RedCount<RED>::n : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + (size_t)warp * W::WB;
    uint64_t *full = reinterpret_cast<uint64_t *>(wbase);
    unsigned char *stg = wbase + 64;
    unsigned char *lnk = stg + (size_t)NST * W::SB;

    const int gw = blockIdx.x * WS_WARPS + warp;
    const int tw = gridDim.x * WS_WARPS;
    const int nsite = A.cb_end - A.cb_begin;
    const int nmy = gw < nsite ? (nsite - 1 - gw) / tw + 1 : 0;
    const int nsteps = nmy * 8;
    const int r0 = lane * R;
    const T cD = from_double<T>(A.c);
    const S *in = reinterpret_cast<const S *>(A.in);
    const S *g8 = reinterpret_cast<const S *>(A.gauge8);

    if (lane == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(full + i, 1);
        mbar_fence_init();
    }
    __syncwarp();

    // Lane d < 8 holds the neighbour of direction d of the site being issued.
    int nb_issue = 0;
    auto issue = [&](int k) {
        const int j = k >> 3, d = k & 7, slot = k % NST;
        const int cb = A.cb_begin + gw + j * tw;
        if (d == 0) {
            const Site st = decode(__ldg(A.coords + (size_t)A.p * A.g.Vh + cb), A.g);
            nb_issue = lane < 8 ? nbr_of_dir(st, A.g, lane) : 0;
        }
        const int nb = __shfl_sync(0xffffffffu, nb_issue, d);
        fence_proxy_async();  // this warp's reads of the slot come before the async writes into it
        __syncwarp();
        if (lane == 0) {
            mbar_expect_tx(full + slot, W::SB + (d == 0 ? W::LB : 0u));
            bulk_copy(stg + (size_t)slot * W::SB, in + (size_t)nb * 12 * N * 2, W::SB, full + slot);
            if (d == 0)
                bulk_copy(lnk + (size_t)(j & 1) * W::LB, g8 + ((size_t)A.p * A.g.Vh + cb) * 8 * 18, W::LB,
                          full + slot);
        }
    };
    for (int k = 0; k < NST && k < nsteps; ++k) issue(k);
    int issued = nsteps < NST ? nsteps : NST;

    cx<T> red[R][NV];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int v = 0; v < NV; ++v) red[r][v] = zero<T>();

    bool ok = true;
    int k = 0;  // next step to wait for
    for (int j = 0; j < nmy && ok; ++j) {
        const int cb = A.cb_begin + gw + j * tw;
        // (the link rows carry the time boundary factor)
        const unsigned char *lrow = lnk + (size_t)(j & 1) * W::LB;
        cx<T> acc[R][12];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int cc = 0; cc < 12; ++cc) acc[r][cc] = zero<T>();
#define DL_WS_STEP(D)                                                                                  \
        if (ok) {                                                                                      \
            const int slot = k % NST;                                                                  \
            ok = __all_sync(0xffffffffu, mbar_wait(full + slot, (uint32_t)((k / NST) & 1)));           \
            if (ok) {                                                                                  \
                tma_compute<S, R, D>(stg + (size_t)slot * W::SB, lrow, N, r0,                          \
                                     false, acc);            \
                __syncwarp();                                                                          \
                if (k + NST < nsteps) {                                                                \
                    issue(k + NST);                                                                    \
                    issued = k + NST + 1;                                                              \
                }                                                                                      \
                ++k;                                                                                   \
            }                                                                                          \
        }
        DL_WS_STEP(0) DL_WS_STEP(1) DL_WS_STEP(2) DL_WS_STEP(3)
        DL_WS_STEP(4) DL_WS_STEP(5) DL_WS_STEP(6) DL_WS_STEP(7)
#undef DL_WS_STEP
        if (!ok) break;
        const size_t base = (size_t)cb * 12 * N * 2 + (size_t)r0 * 2;
        S *out = reinterpret_cast<S *>(A.out);
#pragma unroll
        for (int cc = 0; cc < 12; ++cc) {
            const size_t off = base + (size_t)cc * N * 2;
            cx<T> o[R];
            if (MODE == MODE_PLAIN) {
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = cD * acc[r][cc];
            }
            cx<T> yv[R];
            if (MODE == MODE_XPAY || MODE == MODE_RESID || RED == RED_BICG)
                ld_pack<S, R, true>(reinterpret_cast<const S *>(A.y) + off, yv);
            if (MODE == MODE_XPAY) {
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = yv[r] + cD * acc[r][cc];
            } else if (MODE == MODE_RESID) {
                cx<T> zv[R];
                ld_pack<S, R, true>(reinterpret_cast<const S *>(A.z) + off, zv);
#pragma unroll
                for (int r = 0; r < R; ++r) o[r] = zv[r] - yv[r] - cD * acc[r][cc];
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
    }
    if (!ok) {
        // record the failure, then let every copy this warp issued land (bounded
        // waits) before the block releases its shared memory
        if (lane == 0) {
            if (A.err) *(volatile int *)A.err = 1;
            bool drained = true;
            for (int kk = k; kk < issued; ++kk) drained &= mbar_wait(full + (kk % NST), (uint32_t)((kk / NST) & 1));
            if (!drained && A.err) *(volatile int *)(A.err + 1) = 1;
        }
        __syncwarp();
    }
    // No copy of this warp is pending now (all waited, or drained): retire its barriers.
    __syncwarp();
    if (lane == 0)
        for (int i = 0; i < NST; ++i) mbar_inval(full + i);
    if (RED != RED_NONE) {
        // Every warp's copies have landed and its barriers are retired: the
        // reduction reuses the staging memory from byte 64 on (WS_WARPS * 32 * R *
        // NV complex, at most 10 kB, below the WS_WARPS * WB bytes of the block).
        __syncthreads();
        block_reduce<R, NV, T>(red, 32, N, A.partials, smem + 64);
    }
}

}  // namespace dl
