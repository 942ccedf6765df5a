// Wilson hop for BF16 storage on the tensor cores (mma.sync, FP32 accumulate).
//
// A warp owns one output site with all N = 32 R right-hand sides, staged as in
// the warp-staged kernel (hop_ws.cuh): per hop direction the neighbour's spinor
// block [12][N] (bf16 pairs, one 32-bit word per complex value) lands in the
// warp's ring by one cp.async.bulk copy, the site's eight links with the first
// direction.  Each direction d then applies the 24 x 24 real operator of
// (1 -+ g_mu) x U (mma_table.h) to the block with mma.sync:
//
//   out (24 x N, FP32, in registers)  +=  O_d (24 x 24, bf16)  x  psi (24 x N, bf16),
//
// in two row tiles (output components 0..7 and 8..11) and two column steps
// (input components 0..7 by m16n8k16, 8..11 by m16n8k8), for N / 8 tiles of
// eight right-hand sides.  The B fragments are the staged spinor words as they
// are (a lane reads components t, t + 4, t + 8 of one right-hand side); the A
// fragments are link words with halves exchanged and signs flipped as the
// compile-time table says, so the spin projection, the SU(3) product and the
// reconstruction of the lower spins all happen inside the MMA.  Products of
// bf16 numbers are exact in FP32 and the eight directions accumulate in FP32,
// so the result equals the CUDA-core BF16 hop up to FP32 rounding order.
//
// Epilogue: the accumulator of a lane holds the real (even row) or imaginary
// (odd row) part of one output component for two right-hand sides; one
// shuffle with the partner lane (lane ^ 4) pairs them, then the usual epilogue
// (scale, xpay / resid, bf16 store, reductions) runs per complex value.
#pragma once

#include "hop_ws.cuh"
#include "mma_table.h"

namespace dl {

static __device__ MmaSel g_mma_sel = make_mma_sel();

__device__ __forceinline__ void mma16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                      uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// A staged neighbour block keeps the global layout (component rows N words
// apart, one bulk copy).  Padding the rows to N + 8 words would spread the
// B-fragment reads over all 32 banks, but it takes one bulk copy per row, and
// twelve 128-byte copies per direction measured slower than the bank
// conflicts they remove.
template <int R>
struct MmaShape {
    static constexpr int N = 32 * R;
    static constexpr int RS = N;                     // row stride in words
    static constexpr uint32_t RB = (uint32_t)N * 4u; // bytes of one row
    static constexpr uint32_t DB = 12u * RB;         // data bytes of one neighbour block
    static constexpr uint32_t SB = DB;               // staged bytes of one neighbour block
    static constexpr uint32_t LB = 8u * 9u * 4u;     // one site's eight links
    static constexpr int NST = SB <= 2048 ? 4 : 3;
    static constexpr size_t WB = 64 + (size_t)NST * SB + 2 * (size_t)LB;  // bytes per warp
    static constexpr size_t TAB = sizeof(MmaSel);                         // selection table, per block
    static constexpr size_t SMEM = TAB + WS_WARPS * WB;
};

// Apply direction D of the site to the staged block `sp` with links `lk` (the
// site's row of eight links), accumulating into acc[row tile][n-tile][4].
template <int R, int D>
__device__ __forceinline__ void mma_dir(const unsigned char *sp, const unsigned char *lk, const uint32_t *tcode,
                                        int lane, bool flip, float (&acc)[2][R * 4][4]) {
    constexpr int RS = MmaShape<R>::RS;
    const uint32_t fm = flip ? 0x80008000u : 0u;
    uint32_t aw[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        const uint32_t code = tcode[(D * 9 + s) * 32 + lane];
        const uint32_t w = *reinterpret_cast<const uint32_t *>(lk + D * 36 + ((code >> 16) & 0xffu));
        const uint32_t m = ((code >> 9) & 0x8000u) | ((code << 6) & 0x80000000u);
        aw[s] = __byte_perm(w, 0u, code) ^ m ^ fm;
    }
    const int g = lane >> 2, t = lane & 3;
    const uint32_t *blk = reinterpret_cast<const uint32_t *>(sp);
#pragma unroll
    for (int nt = 0; nt < R * 4; ++nt) {
        const int rhs = 8 * nt + g;
        const uint32_t b0 = blk[t * RS + rhs], b1 = blk[(4 + t) * RS + rhs], b2 = blk[(8 + t) * RS + rhs];
        mma16(acc[0][nt], aw[0], aw[3], aw[1], aw[4], b0, b1);
        mma8(acc[0][nt], aw[2], aw[5], b2);
        mma16(acc[1][nt], aw[6], 0u, aw[7], 0u, b0, b1);
        mma8(acc[1][nt], aw[8], 0u, b2);
    }
}

template <int R, int MODE, int RED>
__global__ void __launch_bounds__(WS_WARPS * 32, R == 1 ? 4 : 2) hop_kernel_mma(HopArgs A) {
    typedef MmaShape<R> W;
    constexpr int N = W::N;
    constexpr int NT = N / 8;
    constexpr int NST = W::NST;
    constexpr int NV = RedCount<RED>::n > 0 ? RedCount<RED>::n : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    uint32_t *tcode = reinterpret_cast<uint32_t *>(smem);
    unsigned char *wbase = smem + W::TAB + (size_t)warp * W::WB;
    uint64_t *full = reinterpret_cast<uint64_t *>(wbase);
    unsigned char *stg = wbase + 64;
    unsigned char *lnk = stg + (size_t)NST * W::SB;

    {  // the selection table, once per block
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&g_mma_sel);
        for (int i = threadIdx.x; i < 8 * 9 * 32; i += blockDim.x) tcode[i] = src[i];
    }

    const int gw = blockIdx.x * WS_WARPS + warp;
    const int tw = gridDim.x * WS_WARPS;
    const int nsite = A.cb_end - A.cb_begin;
    const int nmy = gw < nsite ? (nsite - 1 - gw) / tw + 1 : 0;
    const int nsteps = nmy * 8;
    const float cD = (float)A.c;
    const bf16 *in = reinterpret_cast<const bf16 *>(A.in);
    const bf16 *g8 = reinterpret_cast<const bf16 *>(A.gauge8);

    if (lane == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(full + i, 1);
        mbar_fence_init();
    }
    __syncthreads();  // table and barriers ready

    int nb_issue = 0;
    auto issue = [&](int k) {
        const int j = k >> 3, d = k & 7, slot = k % NST;
        const int cb = A.cb_begin + gw + j * tw;
        if (d == 0) {
            const Site st = decode(__ldg(A.coords + (size_t)A.p * A.g.Vh + cb), A.g);
            nb_issue = lane < 8 ? nbr_of_dir(st, A.g, lane) : 0;
        }
        const int nb = __shfl_sync(0xffffffffu, nb_issue, d);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
            mbar_expect_tx(full + slot, W::DB + (d == 0 ? W::LB : 0u));
            bulk_copy(stg + (size_t)slot * W::SB, in + (size_t)nb * 12 * N * 2, W::DB, full + slot);
            if (d == 0)
                bulk_copy(lnk + (size_t)(j & 1) * W::LB, g8 + ((size_t)A.p * A.g.Vh + cb) * 8 * 18, W::LB,
                          full + slot);
        }
    };
    for (int k = 0; k < NST && k < nsteps; ++k) issue(k);
    int issued = nsteps < NST ? nsteps : NST;

    cx<float> red[NT][NV];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int v = 0; v < NV; ++v) red[nt][v] = zero<float>();

    bool ok = true;
    int k = 0;
    for (int j = 0; j < nmy && ok; ++j) {
        const int cb = A.cb_begin + gw + j * tw;
        // (the link rows carry the time boundary factor)
        const unsigned char *lrow = lnk + (size_t)(j & 1) * W::LB;
        float acc[2][NT][4];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[m][nt][e] = 0.f;
#define DL_MMA_STEP(D)                                                                                 \
        if (ok) {                                                                                      \
            const int slot = k % NST;                                                                  \
            ok = __all_sync(0xffffffffu, mbar_wait(full + slot, (uint32_t)((k / NST) & 1)));           \
            if (ok) {                                                                                  \
                mma_dir<R, D>(stg + (size_t)slot * W::SB, lrow, tcode, lane,                           \
                              false, acc);                   \
                __syncwarp();                                                                          \
                if (k + NST < nsteps) {                                                                \
                    issue(k + NST);                                                                    \
                    issued = k + NST + 1;                                                              \
                }                                                                                      \
                ++k;                                                                                   \
            }                                                                                          \
        }
        DL_MMA_STEP(0) DL_MMA_STEP(1) DL_MMA_STEP(2) DL_MMA_STEP(3)
        DL_MMA_STEP(4) DL_MMA_STEP(5) DL_MMA_STEP(6) DL_MMA_STEP(7)
#undef DL_MMA_STEP
        if (!ok) break;
        // epilogue: lane pairs (g, g ^ 1) join the real and imaginary rows of each component
        bf16 *out = reinterpret_cast<bf16 *>(A.out);
        const size_t site = (size_t)cb * 12 * N;
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const float lo = acc[m][nt][2 * h], hi = acc[m][nt][2 * h + 1];
                    const float recv = __shfl_xor_sync(0xffffffffu, (g & 1) ? lo : hi, 4);
                    if (m == 1 && h == 1) continue;  // output components 12..15 do not exist
                    const int o = 8 * m + 4 * h + (g >> 1);
                    const int rhs = 8 * nt + 2 * t + (g & 1);
                    const cx<float> v = (g & 1) ? mk(recv, hi) : mk(lo, recv);
                    const size_t off = (site + (size_t)o * N + rhs) * 2;
                    cx<float> ov;
                    cx<float> yv = zero<float>();
                    if (MODE == MODE_XPAY || MODE == MODE_RESID || RED == RED_BICG) {
                        cx<float> tmp[1];
                        ld_pack<bf16, 1, true>(reinterpret_cast<const bf16 *>(A.y) + off, tmp);
                        yv = tmp[0];
                    }
                    if (MODE == MODE_PLAIN) {
                        ov = cD * v;
                    } else if (MODE == MODE_XPAY) {
                        ov = yv + cD * v;
                    } else {
                        cx<float> zv[1];
                        ld_pack<bf16, 1, true>(reinterpret_cast<const bf16 *>(A.z) + off, zv);
                        ov = zv[0] - yv - cD * v;
                    }
                    cx<float> st[1] = {ov};
                    st_pack<bf16, 1>(out + off, st);
                    if (RED == RED_R0DOT || RED == RED_BICG) {
                        cx<float> rh[1];
                        ld_pack<bf16, 1, true>(reinterpret_cast<const bf16 *>(A.rhat) + off, rh);
                        if (RED == RED_R0DOT) {
                            cjmac(red[nt][0], rh[0], ov);
                        } else {
                            cjmac(red[nt][0], ov, yv);
                            cjmac(red[nt][1], ov, ov);
                            cjmac(red[nt][2], rh[0], yv);
                            cjmac(red[nt][3], rh[0], ov);
                            cjmac(red[nt][4], yv, yv);
                        }
                    } else if (RED == RED_NORM) {
                        cjmac(red[nt][0], ov, ov);
                    }
                }
    }
    if (!ok) {
        if (lane == 0) {
            if (A.err) *(volatile int *)A.err = 1;
            bool drained = true;
            for (int kk = k; kk < issued; ++kk) drained &= mbar_wait(full + (kk % NST), (uint32_t)((kk / NST) & 1));
            if (!drained && A.err) *(volatile int *)(A.err + 1) = 1;
        }
    }
    __syncwarp();
    if (lane == 0)
        for (int i = 0; i < NST; ++i) mbar_inval(full + i);
    if (RED != RED_NONE) {
        // Lanes with the same (t, g & 1) hold the same right-hand sides (8 nt + 2 t + (g & 1)):
        // sum them over g >> 1 (lane bits 3 and 4), in a fixed order.
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                red[nt][v].re += __shfl_xor_sync(0xffffffffu, red[nt][v].re, 8);
                red[nt][v].im += __shfl_xor_sync(0xffffffffu, red[nt][v].im, 8);
                red[nt][v].re += __shfl_xor_sync(0xffffffffu, red[nt][v].re, 16);
                red[nt][v].im += __shfl_xor_sync(0xffffffffu, red[nt][v].im, 16);
            }
        __syncthreads();  // the table is no longer read: it takes the per-warp sums
        cx<float> *sm = reinterpret_cast<cx<float> *>(smem);  // [warp][N][NV]
        if (lane < 8) {
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int v = 0; v < NV; ++v) sm[((size_t)warp * N + 8 * nt + 2 * t + (g & 1)) * NV + v] = red[nt][v];
        }
        __syncthreads();
        for (int o = threadIdx.x; o < N * NV; o += blockDim.x) {
            double re = 0.0, im = 0.0;
            for (int w = 0; w < WS_WARPS; ++w) {
                re += (double)sm[(size_t)w * N * NV + o].re;
                im += (double)sm[(size_t)w * N * NV + o].im;
            }
            A.partials[(size_t)blockIdx.x * N * NV + o] = make_double2(re, im);
        }
    }
}

}  // namespace dl
