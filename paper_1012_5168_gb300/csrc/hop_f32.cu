// Wilson-hop instantiations for float storage (direct and prefetching variants).
#include "launch.h"
#include "hop_tma.cuh"

namespace dl {

template <int R, int MODE, int RED>
static cudaError_t go(const HopArgs &a, Launch &l, int pf) {
    if (pf == 2) {
        static size_t opted_tma = 0;
        if (l.smem > 48 * 1024 && l.smem > opted_tma) {
            cudaError_t e = cudaFuncSetAttribute(hop_kernel_tma<float, R, MODE, RED, TMA_STAGES>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem);
            if (e != cudaSuccess) return e;
            opted_tma = l.smem;
        }
        hop_kernel_tma<float, R, MODE, RED, TMA_STAGES><<<l.grid, l.block, l.smem, l.stream>>>(a);
        return cudaGetLastError();
    }
    if (pf == 3) {
        constexpr int cap = HopRegCap<float, R, MODE, RED>::n;
        constexpr int NV = RedCount<RED>::n;
        const int G = a.N / R;
        const size_t per_warp = NV ? (size_t)(G < 32 ? G : 32) * R * NV * sizeof(cx<float>) : 0;
        static int blk = 0, res = 1, blkN = 0;  // per instantiation, for the last G seen
        auto kern = [] {
            if constexpr (cap > 0) return hop_kernel_cap<float, R, MODE, RED, cap>;
            else return hop_kernel<float, R, MODE, RED>;
        }();
        if (blk == 0 || blkN != G) {
            blk = widest_block(kern, G > 32 ? G : 32, per_warp, &res);
            blkN = G;
        }
        HopArgs b = a;
        b.blocked = 1;
        l.block = blk;
        l.smem = per_warp * (blk / 32);
        l.grid = (l.num_sms > 0 ? l.num_sms : 1) * (res < 16 ? res : 16);
        kern<<<l.grid, l.block, l.smem, l.stream>>>(b);
        return cudaGetLastError();
    }
    if (!pf) {
        constexpr int cap = HopRegCap<float, R, MODE, RED>::n;
        if constexpr (cap > 0) {
            clamp_grid(l, resident_blocks(hop_kernel_cap<float, R, MODE, RED, cap>, l.block, l.smem));
            hop_kernel_cap<float, R, MODE, RED, cap><<<l.grid, l.block, l.smem, l.stream>>>(a);
        } else {
            clamp_grid(l, resident_blocks(hop_kernel<float, R, MODE, RED>, l.block, l.smem));
            hop_kernel<float, R, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
        }
        return cudaGetLastError();
    }
    static size_t opted = 0;  // largest dynamic shared memory opted in so far
    if (l.smem > 48 * 1024 && l.smem > opted) {
        cudaError_t e = cudaFuncSetAttribute(hop_kernel_pf<float, R, MODE, RED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem);
        if (e != cudaSuccess) return e;
        opted = l.smem;
    }
    hop_kernel_pf<float, R, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hop_f32(int R, int mode, int red, int pf, const HopArgs &a, Launch &l) {
#define DL_CASE(r, m, rd) \
    if (R == r && mode == m && red == rd) return go<r, m, rd>(a, l, pf);
    DL_CASE(1, MODE_PLAIN, RED_NONE)
    DL_CASE(1, MODE_XPAY, RED_NONE)
    DL_CASE(1, MODE_XPAY, RED_R0DOT)
    DL_CASE(1, MODE_XPAY, RED_BICG)
    DL_CASE(1, MODE_XPAY, RED_NORM)
    DL_CASE(2, MODE_PLAIN, RED_NONE)
    DL_CASE(2, MODE_XPAY, RED_NONE)
    DL_CASE(2, MODE_XPAY, RED_R0DOT)
    DL_CASE(2, MODE_XPAY, RED_BICG)
    DL_CASE(2, MODE_XPAY, RED_NORM)
    DL_CASE(4, MODE_PLAIN, RED_NONE)
    DL_CASE(4, MODE_XPAY, RED_NONE)
    DL_CASE(4, MODE_XPAY, RED_R0DOT)
    DL_CASE(4, MODE_XPAY, RED_BICG)
    DL_CASE(4, MODE_XPAY, RED_NORM)
#undef DL_CASE
    return cudaErrorInvalidValue;
}

}  // namespace dl
