// Launch of one Wilson-hop instantiation for a low-precision storage type S
// (float or bf16): the kernel kind picks the direct, prefetching, staged or
// blocked-mapping, warp-staged or (BF16 only) tensor-core kernel.  hop_f32*.cu
// and hop_bf16*.cu instantiate it.  The
// one-time settings (shared-memory opt-ins, the blocked kernel's block shape)
// are guarded so that contexts used from several host threads can launch
// concurrently.
#pragma once

#include <mutex>

#include <type_traits>

#include "hop_mma.cuh"
#include "launch.h"

namespace dl {

// Raise a kernel's dynamic shared-memory limit to at least `smem` (beyond the
// default 48 KiB), once per larger request.
template <typename K>
inline cudaError_t opt_in_smem(K kernel, size_t smem, size_t &opted, std::mutex &m) {
    if (smem <= 48 * 1024) return cudaSuccess;
    std::lock_guard<std::mutex> g(m);
    if (smem <= opted) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) opted = smem;
    return e;
}

template <typename S, int R, int MODE, int RED>
cudaError_t go_hop(const HopArgs &a, Launch &l, int kind) {
    if (a.clovinv) {  // clover: the direct kernel with A^-1 in the epilogue, one right-hand side per thread
        if constexpr (R == 1) {
            constexpr int ccap = HopRegCap<S, 1, MODE, RED>::n;
            if constexpr (ccap > 0) {
                if (a.N == 32) {
                    clamp_grid(l, resident_blocks(hop_kernel_clov_cap<S, MODE, RED, ccap, 32>, l.block, l.smem));
                    hop_kernel_clov_cap<S, MODE, RED, ccap, 32><<<l.grid, l.block, l.smem, l.stream>>>(a);
                    return cudaGetLastError();
                }
            }
            clamp_grid(l, resident_blocks(hop_kernel_clov<S, MODE, RED>, l.block, l.smem));
            hop_kernel_clov<S, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
            return cudaGetLastError();
        }
        return cudaErrorInvalidValue;
    }
    constexpr int cap = HopRegCap<S, R, MODE, RED>::n;
    auto direct = [] {
        if constexpr (cap > 0) return hop_kernel_cap<S, R, MODE, RED, cap>;
        else return hop_kernel<S, R, MODE, RED>;
    }();
    if (kind == 0) {
        if constexpr (cap > 0) {
            if (a.N == 32) {  // the benchmark width: offsets as compile-time constants
                clamp_grid(l, resident_blocks(hop_kernel_cap<S, R, MODE, RED, cap, 32>, l.block, l.smem));
                hop_kernel_cap<S, R, MODE, RED, cap, 32><<<l.grid, l.block, l.smem, l.stream>>>(a);
                return cudaGetLastError();
            }
        }
        clamp_grid(l, resident_blocks(direct, l.block, l.smem));
        direct<<<l.grid, l.block, l.smem, l.stream>>>(a);
        return cudaGetLastError();
    }
    if (kind == 10) {  // the direct FP32 kernel under a wider register cap (80 plain, 96 fused)
        if constexpr (std::is_same<S, float>::value && R == 1) {
            constexpr int wcap = MODE == MODE_PLAIN ? 80 : 96;
            auto k = a.N == 32 ? hop_kernel_cap<S, 1, MODE, RED, wcap, 32> : hop_kernel_cap<S, 1, MODE, RED, wcap>;
            clamp_grid(l, resident_blocks(k, l.block, l.smem));
            k<<<l.grid, l.block, l.smem, l.stream>>>(a);
            return cudaGetLastError();
        }
        return cudaErrorInvalidValue;
    }
    if (kind == 1) {
        static size_t opted = 0;
        static std::mutex m;
        const cudaError_t e = opt_in_smem(hop_kernel_pf<S, R, MODE, RED>, l.smem, opted, m);
        if (e != cudaSuccess) return e;
        hop_kernel_pf<S, R, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
        return cudaGetLastError();
    }
    if (kind == 2) {
        static size_t opted = 0;
        static std::mutex m;
        const cudaError_t e = opt_in_smem(hop_kernel_tma<S, R, MODE, RED, TMA_STAGES>, l.smem, opted, m);
        if (e != cudaSuccess) return e;
        hop_kernel_tma<S, R, MODE, RED, TMA_STAGES><<<l.grid, l.block, l.smem, l.stream>>>(a);
        return cudaGetLastError();
    }
    if (kind == 3) {
        constexpr int NV = RedCount<RED>::n;
        const int G = a.N / R;
        const size_t per_warp = NV ? (size_t)(G < 32 ? G : 32) * R * NV * sizeof(cx<float>) : 0;
        // block shape for the G last seen: block | resident << 16 | G << 24
        static std::atomic<uint32_t> shape{0};
        uint32_t sh = shape.load(std::memory_order_relaxed);
        if (sh == 0 || (int)(sh >> 24) != G) {
            int res = 1;
            const int blk = widest_block(direct, G > 32 ? G : 32, per_warp, &res);
            sh = (uint32_t)blk | ((uint32_t)(res < 16 ? res : 16) << 16) | ((uint32_t)G << 24);
            shape.store(sh, std::memory_order_relaxed);
        }
        HopArgs b = a;
        b.blocked = 1;
        l.block = (int)(sh & 0xffff);
        l.smem = per_warp * (l.block / 32);
        l.grid = (l.num_sms > 0 ? l.num_sms : 1) * (int)((sh >> 16) & 0xff);
        direct<<<l.grid, l.block, l.smem, l.stream>>>(b);
        return cudaGetLastError();
    }
    if (kind == 4 || kind == 11) {  // warp-staged: one site per warp, so N = 32 R; kind 11 with two stages
        if (a.N != 32 * R) return cudaErrorInvalidValue;
        static size_t opted = 0, opted2 = 0;
        static std::mutex m, m2;
        auto kern = kind == 4 ? hop_kernel_ws<S, R, MODE, RED> : hop_kernel_ws<S, R, MODE, RED, 2>;
        l.block = WS_WARPS * 32;
        l.smem = (kind == 4 ? WsShape<S, R>::WB : WsShape<S, R, 2>::WB) * WS_WARPS;
        const cudaError_t e = kind == 4 ? opt_in_smem(kern, l.smem, opted, m) : opt_in_smem(kern, l.smem, opted2, m2);
        if (e != cudaSuccess) return e;
        const int res = resident_blocks(kern, l.block, l.smem);
        l.grid = (l.num_sms > 0 ? l.num_sms : 1) * (res < 16 ? res : 16);
        kern<<<l.grid, l.block, l.smem, l.stream>>>(a);
        return cudaGetLastError();
    }
    if (kind == 6) {  // direct loads, packed FP32 arithmetic (FP32 storage, R = 1)
        if constexpr (std::is_same<S, float>::value && R == 1) {
            constexpr int xcap = MODE == MODE_PLAIN ? 64 : 72;
            if (a.N == 32) {
                clamp_grid(l, resident_blocks(hop_kernel_x2<MODE, RED, xcap, 32>, l.block, l.smem));
                hop_kernel_x2<MODE, RED, xcap, 32><<<l.grid, l.block, l.smem, l.stream>>>(a);
            } else {
                clamp_grid(l, resident_blocks(hop_kernel_x2<MODE, RED, xcap>, l.block, l.smem));
                hop_kernel_x2<MODE, RED, xcap><<<l.grid, l.block, l.smem, l.stream>>>(a);
            }
            return cudaGetLastError();
        }
    }
    if (kind == 5) {  // tensor cores, BF16 storage only; one site per warp, N = 32 R
        if constexpr (std::is_same<S, bf16>::value && (R == 1 || R == 2)) {
            if (a.N != 32 * R) return cudaErrorInvalidValue;
            static size_t opted = 0;
            static std::mutex m;
            auto kern = hop_kernel_mma<R, MODE, RED>;
            l.block = WS_WARPS * 32;
            l.smem = MmaShape<R>::SMEM;
            const cudaError_t e = opt_in_smem(kern, l.smem, opted, m);
            if (e != cudaSuccess) return e;
            const int res = resident_blocks(kern, l.block, l.smem);
            l.grid = (l.num_sms > 0 ? l.num_sms : 1) * (res < 16 ? res : 16);
            kern<<<l.grid, l.block, l.smem, l.stream>>>(a);
            return cudaGetLastError();
        }
    }
    return cudaErrorInvalidValue;
}

// The (MODE, RED) combinations the solvers use, for storage type S and R
// right-hand sides per thread.  Each (S, R) pair is instantiated in its own
// translation unit (hop_f32.cu, hop_f32_r2.cu, ...), so the build compiles the
// kernel variants in parallel.
template <typename S, int R>
cudaError_t launch_hop_low_r(int mode, int red, int kind, const HopArgs &a, Launch &l) {
#define DL_CASE(m, rd) \
    if (mode == m && red == rd) return go_hop<S, R, m, rd>(a, l, kind);
    DL_CASE(MODE_PLAIN, RED_NONE)
    DL_CASE(MODE_XPAY, RED_NONE)
    DL_CASE(MODE_XPAY, RED_R0DOT)
    DL_CASE(MODE_XPAY, RED_BICG)
    DL_CASE(MODE_XPAY, RED_NORM)
#undef DL_CASE
    return cudaErrorInvalidValue;
}

// The R = 2 and R = 4 instantiations (hop_*_r2.cu, hop_*_r4.cu).
cudaError_t launch_hop_f32_r2(int mode, int red, int kind, const HopArgs &a, Launch &l);
cudaError_t launch_hop_f32_r4(int mode, int red, int kind, const HopArgs &a, Launch &l);
cudaError_t launch_hop_bf16_r2(int mode, int red, int kind, const HopArgs &a, Launch &l);
cudaError_t launch_hop_bf16_r4(int mode, int red, int kind, const HopArgs &a, Launch &l);

}  // namespace dl
