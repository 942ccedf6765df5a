// Warp-staged Wilson hop on the paired FP32 layout with packed FP32
// arithmetic (kernel kind 9).
//
// The memory side is the warp-staged kernel's (hop_ws.cuh): every warp keeps
// its own ring of NST stages filled by cp.async.bulk copies (the TMA engine),
// each stage completed on its own mbarrier, so the loads of NST - 1 hop
// directions are in flight while the warp computes the current one from
// shared memory, and no warp waits for another.  The arithmetic side is the
// paired kernel's (hop_pair.cuh): a lane owns two right-hand sides, so one
// FFMA2 does the work of two FFMA.  A warp works on SPW = 64 / N sites at a
// time (16 lanes per site at N = 32).  A stage holds, per site, the
// neighbour's spinor block [12][N] and the link of that direction as nine
// (Re, Re, Im, Im) quads (144 bytes), so nothing stays in shared memory
// across sites.
//
// Every wait is bounded: when one runs out, the warp records A.err[0], stops,
// waits (bounded again) for the copies it has issued, and leaves the site
// loop; if a drain wait runs out as well it records A.err[1].
#pragma once

#include "hop_pair.cuh"
#include "hop_ws.cuh"

namespace dl {

constexpr int WSP_WARPS = 4;  // warps per block

template <int N>
struct WspShape {
    static constexpr int SPW = 64 / N;                      // sites per warp
    static constexpr uint32_t SB = 12u * N * 8u;             // one neighbour block [12][N] (FP32 complex)
    static constexpr uint32_t LQ = 9u * 16u;                 // one link as nine quads
    static constexpr uint32_t STAGE = SPW * (SB + LQ);       // bytes per stage
    static constexpr int NST = 4;                            // stages per warp
    static constexpr size_t WB = 64 + (size_t)NST * STAGE;   // bytes per warp (64: the mbarriers)
};

template <int MODE, int RED, int N>
__global__ void __launch_bounds__(WSP_WARPS * 32) hop_kernel_ws_pair(HopArgs A) {
    typedef WspShape<N> W;
    constexpr int SPW = W::SPW, NST = W::NST, G = N / 2;
    constexpr int NV = PairNV<RED>::n;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + (size_t)warp * W::WB;
    uint64_t *full = reinterpret_cast<uint64_t *>(wbase);
    unsigned char *stg = wbase + 64;

    const int gw = blockIdx.x * WSP_WARPS + warp;
    const int tw = gridDim.x * WSP_WARPS;
    const int ngroup = (A.cb_end - A.cb_begin) / SPW;  // site groups (the host checks divisibility)
    const int nmy = gw < ngroup ? (ngroup - 1 - gw) / tw + 1 : 0;
    const int nsteps = nmy * 8;
    const int h = lane / G;             // the site of this lane within the group
    const int r0 = (lane % G) * 2;      // its two right-hand sides
    const float cD = (float)A.c;
    const float2 c2 = make_float2(cD, cD);
    const float *in = reinterpret_cast<const float *>(A.in);

    if (lane == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(full + i, 1);
        mbar_fence_init();
    }
    __syncwarp();

    // lanes s * 8 + d (s < SPW, d < 8) hold the neighbour of direction d of site s of the group being issued
    int nb_issue = 0;
    auto issue = [&](int k) {
        const int j = k >> 3, d = k & 7, slot = k % NST;
        const int cbg = A.cb_begin + (gw + j * tw) * SPW;
        if (d == 0) {
            const int s = lane >> 3;
            nb_issue = 0;
            if (s < SPW) {
                const Site st = decode(__ldg(A.coords + (size_t)A.p * A.g.Vh + cbg + s), A.g);
                nb_issue = nbr_of_dir(st, A.g, lane & 7);
            }
        }
        int nb[SPW];
#pragma unroll
        for (int s = 0; s < SPW; ++s) nb[s] = __shfl_sync(0xffffffffu, nb_issue, s * 8 + d);
        fence_proxy_async();  // this warp's reads of the slot come before the async writes into it
        __syncwarp();
        if (lane == 0) {
            unsigned char *dst = stg + (size_t)slot * W::STAGE;
            mbar_expect_tx(full + slot, W::STAGE);
#pragma unroll
            for (int s = 0; s < SPW; ++s) {
                bulk_copy(dst + (size_t)s * W::SB, in + (size_t)nb[s] * 12 * N * 2, W::SB, full + slot);
                bulk_copy(dst + (size_t)SPW * W::SB + (size_t)s * W::LQ,
                          A.gauge8d + (((size_t)A.p * A.g.Vh + cbg + s) * 8 + d) * 9, W::LQ, full + slot);
            }
        }
    };
    for (int k = 0; k < NST && k < nsteps; ++k) issue(k);
    int issued = nsteps < NST ? nsteps : NST;

    float2 dr[NV], di[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) dr[v] = di[v] = make_float2(0.f, 0.f);

    bool ok = true;
    int k = 0;  // next step to wait for
    for (int j = 0; j < nmy && ok; ++j) {
        const int cb = A.cb_begin + (gw + j * tw) * SPW + h;
        P2 acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c].re = acc[c].im = make_float2(0.f, 0.f);
#define DL_WSP_STEP(D)                                                                                  \
        if (ok) {                                                                                       \
            const int slot = k % NST;                                                                   \
            ok = __all_sync(0xffffffffu, mbar_wait(full + slot, (uint32_t)((k / NST) & 1)));            \
            if (ok) {                                                                                   \
                const unsigned char *sb = stg + (size_t)slot * W::STAGE;                                \
                hop_dir_pair<(D) / 2, ((D) % 2 == 0) ? -1 : +1, ((D) % 2) != 0, false>(                 \
                    reinterpret_cast<const float *>(sb + (size_t)h * W::SB) + r0 * 2, N,                \
                    reinterpret_cast<const float4 *>(sb + (size_t)SPW * W::SB + (size_t)h * W::LQ), acc); \
                __syncwarp();                                                                           \
                if (k + NST < nsteps) {                                                                 \
                    issue(k + NST);                                                                     \
                    issued = k + NST + 1;                                                               \
                }                                                                                       \
                ++k;                                                                                    \
            }                                                                                           \
        }
        DL_WSP_STEP(0) DL_WSP_STEP(1) DL_WSP_STEP(2) DL_WSP_STEP(3)
        DL_WSP_STEP(4) DL_WSP_STEP(5) DL_WSP_STEP(6) DL_WSP_STEP(7)
#undef DL_WSP_STEP
        if (!ok) break;
        epilogue_pair<MODE, RED>(A, cb, r0, N, c2, acc, dr, di);
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
        // Every warp's copies have landed: the reduction reuses warp 0's staging
        // memory (WSP_WARPS * G * 2 * NV complex floats, below one stage).
        __syncthreads();
        reduce_pair<NV>(A, G, N, dr, di, smem + 64);
    }
}

}  // namespace dl
