// Wilson-hop instantiations for the paired FP32 layout (f32p): the direct
// kernel with scalar arithmetic (kind 0; R = 1 with the FP32 register caps,
// R = 2 and 4 uncapped), the clover direct kernel, and the packed-arithmetic
// kernels (kind 7, two right-hand sides per thread; kind 8 the same under a
// 128-register cap; kind 9 warp-staged through per-warp bulk-copy rings).
#include "hop_launch.cuh"
#include "hop_ws_pair.cuh"
#include "launch.h"

namespace dl {

template <int MODE, int RED, int N>
static cudaError_t go_ws_pair(const HopArgs &a, Launch &l) {
    static size_t opted = 0;
    static std::mutex m;
    auto kern = hop_kernel_ws_pair<MODE, RED, N>;
    l.block = WSP_WARPS * 32;
    l.smem = WspShape<N>::WB * WSP_WARPS;
    const cudaError_t e = opt_in_smem(kern, l.smem, opted, m);
    if (e != cudaSuccess) return e;
    const int res = resident_blocks(kern, l.block, l.smem);
    l.grid = (l.num_sms > 0 ? l.num_sms : 1) * (res < 16 ? res : 16);
    kern<<<l.grid, l.block, l.smem, l.stream>>>(a);
    return cudaGetLastError();
}

template <int MODE, int RED>
static cudaError_t go_pair(const HopArgs &a, Launch &l, int kind, int R) {
    typedef f32p S;
    if (a.clovinv) {
        if (R != 1) return cudaErrorInvalidValue;
        clamp_grid(l, resident_blocks(hop_kernel_clov<S, MODE, RED>, l.block, l.smem));
        hop_kernel_clov<S, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
        return cudaGetLastError();
    }
    if (kind == 7 || kind == 8) {
        if (R != 2 || !a.gauge8d) return cudaErrorInvalidValue;
        // at the benchmark width the component offsets are compile-time constants
        auto k = kind == 7 ? (a.N == 32 ? hop_kernel_pair<MODE, RED, 32> : hop_kernel_pair<MODE, RED>)
                           : (a.N == 32 ? hop_kernel_pair_cap<MODE, RED, 32> : hop_kernel_pair_cap<MODE, RED>);
        clamp_grid(l, resident_blocks(k, l.block, l.smem));
        k<<<l.grid, l.block, l.smem, l.stream>>>(a);
        return cudaGetLastError();
    }
    if (kind == 9) {  // warp-staged, 64 / N sites per warp: N = 32 (site count even) or 64
        if (R != 2 || !a.gauge8d) return cudaErrorInvalidValue;
        if (a.N == 32 && (a.cb_end - a.cb_begin) % 2 == 0) return go_ws_pair<MODE, RED, 32>(a, l);
        if (a.N == 64) return go_ws_pair<MODE, RED, 64>(a, l);
        return cudaErrorInvalidValue;
    }
    if (kind != 0) return cudaErrorInvalidValue;
    if (R == 1) {
        constexpr int cap = HopRegCap<S, 1, MODE, RED>::n;
        clamp_grid(l, resident_blocks(hop_kernel_cap<S, 1, MODE, RED, cap>, l.block, l.smem));
        hop_kernel_cap<S, 1, MODE, RED, cap><<<l.grid, l.block, l.smem, l.stream>>>(a);
    } else if (R == 2) {
        clamp_grid(l, resident_blocks(hop_kernel<S, 2, MODE, RED>, l.block, l.smem));
        hop_kernel<S, 2, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
    } else if (R == 4) {
        clamp_grid(l, resident_blocks(hop_kernel<S, 4, MODE, RED>, l.block, l.smem));
        hop_kernel<S, 4, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_hop_f32p(int R, int mode, int red, int kind, const HopArgs &a, Launch &l) {
#define DL_CASE(m, rd) \
    if (mode == m && red == rd) return go_pair<m, rd>(a, l, kind, R);
    DL_CASE(MODE_PLAIN, RED_NONE)
    DL_CASE(MODE_XPAY, RED_NONE)
    DL_CASE(MODE_XPAY, RED_R0DOT)
    DL_CASE(MODE_XPAY, RED_BICG)
    DL_CASE(MODE_XPAY, RED_NORM)
#undef DL_CASE
    return cudaErrorInvalidValue;
}

}  // namespace dl
