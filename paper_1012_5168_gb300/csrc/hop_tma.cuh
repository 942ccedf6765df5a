// Wilson hop with block-cooperative staging through shared memory by bulk
// asynchronous copies (the TMA engine's cp.async.bulk) with mbarrier
// completion.
//
// A block owns chunks of SITES consecutive output sites (all N right-hand
// sides; thread = (site, right-hand-side group)).  For one chunk the work is
// eight steps, one per hop direction.  The input of a step is, for each site
// of the chunk, its neighbour's spinor block [12][N] (one contiguous run in the
// even-odd tile layout) plus, at the first direction, the chunk's links in a
// site-major layout with all eight links of a site in one row
// ([parity][cb][8][3x3], direction d = 2 mu + (0 forward, 1 backward)).
// Each of those is a single bulk copy.  A ring of NST stages keeps NST - 1
// steps in flight while the current one is computed from shared memory, so
// the memory system sees many kilobytes in flight per block without any
// registers held for loads.
//
// Every wait on an mbarrier is bounded.  When a bound runs out the kernel
// records an error in A.err[0], stops computing, waits (bounded again) for the
// copies it has in flight, and returns; the host reports DL_ECUDA.  If one of
// those drain waits runs out too, copies may still land in shared memory after
// the block has exited; the kernel records that in A.err[1] and the host marks
// the context unusable (every later call returns DL_ECUDA).
#pragma once

#include "hop.cuh"

namespace dl {

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false when the bound ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Compute direction D of one site from a staged neighbour block (this
// thread's R right-hand sides at offset r0) and a staged link row.
template <typename S, int R, int D>
__device__ __forceinline__ void tma_compute(const unsigned char *sp, const unsigned char *lp, int N, int r0,
                                            bool flip, cx<typename Real<S>::type> (&acc)[R][12]) {
    typedef typename Real<S>::type T;
    constexpr int MU = D / 2;
    constexpr int SG = (D % 2 == 0) ? -1 : +1;
    const S *src = reinterpret_cast<const S *>(sp) + (size_t)r0 * 2;
    cx<T> hh[R][6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cx<T> q0[R], q1[R], q2[R], q3[R];
        ld_pack<S, R, false>(src + (size_t)a * N * 2, q0);
        ld_pack<S, R, false>(src + (size_t)(3 + a) * N * 2, q1);
        ld_pack<S, R, false>(src + (size_t)(6 + a) * N * 2, q2);
        ld_pack<S, R, false>(src + (size_t)(9 + a) * N * 2, q3);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const cx<T> p0 = q0[r], p1 = q1[r], p2 = q2[r], p3 = q3[r];
            if (MU == 0) {
                hh[r][a] = SG > 0 ? p0 + ti(p3) : p0 - ti(p3);
                hh[r][3 + a] = SG > 0 ? p1 + ti(p2) : p1 - ti(p2);
            } else if (MU == 1) {
                hh[r][a] = SG > 0 ? p0 - p3 : p0 + p3;
                hh[r][3 + a] = SG > 0 ? p1 + p2 : p1 - p2;
            } else if (MU == 2) {
                hh[r][a] = SG > 0 ? p0 + ti(p2) : p0 - ti(p2);
                hh[r][3 + a] = SG > 0 ? p1 - ti(p3) : p1 + ti(p3);
            } else {
                hh[r][a] = SG > 0 ? p0 + p2 : p0 - p2;
                hh[r][3 + a] = SG > 0 ? p1 + p3 : p1 - p3;
            }
        }
    }
    cx<T> u[9];
    const S *lk = reinterpret_cast<const S *>(lp) + D * 18;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        cx<T> z[1];
        ld_pack<S, 1, false>(lk + 2 * k, z);
        u[k] = z[0];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cx<T> w[6];
        cx<T>(&h)[6] = hh[r];
        if (flip) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = -h[k];
        }
        su3_mul<T, (D % 2 == 1)>(u, h, w);
        reconstruct<T, MU, SG>(w, acc[r]);
    }
}

// Issue the copies of step k (chunk j = k/8 of this block, direction d = k%8).
// Called by warp 0 only.  At d = 0 the lanes turn the chunk's packed
// coordinates (loaded one chunk ahead into `pre`) into the chunk's neighbour
// table nbr[j&1][site][8] in shared memory; later directions read the table,
// so no step waits on a global load before its copies go out.
template <typename S>
__device__ __forceinline__ void tma_issue(const HopArgs &A, int k, int SITES, int NST, uint64_t *full,
                                          unsigned char *stg, unsigned char *lnk, int *nbr, size_t SB, size_t LB,
                                          const uint32_t *pre) {
    const int lane = threadIdx.x & 31;
    const int j = k >> 3, d = k & 7;
    const int c = blockIdx.x + j * gridDim.x;
    const int cb0 = A.cb_begin + c * SITES;
    const int ns = min(SITES, A.cb_end - cb0);
    const int slot = k % NST;
    uint64_t *bar = full + slot;
    int *tab = nbr + (j & 1) * SITES * 8;
    if (d == 0) {
        for (int s = lane, q = 0; s < ns; s += 32, ++q) {
            const Site st = decode(pre[q], A.g);
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                tab[s * 8 + 2 * mu] = nbr_fwd(st, A.g, mu);
                tab[s * 8 + 2 * mu + 1] = nbr_bwd(st, A.g, mu);
            }
        }
        __syncwarp();
    }
    fence_proxy_async();  // earlier generic reads of this slot before the async writes
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)(ns * SB + (d == 0 ? ns * LB : 0)));
    __syncwarp();
    const S *in = reinterpret_cast<const S *>(A.in);
    for (int s = lane; s < ns; s += 32)
        bulk_copy(stg + (size_t)slot * SITES * SB + (size_t)s * SB, in + (size_t)tab[s * 8 + d] * 12 * A.N * 2,
                  (uint32_t)SB, bar);
    if (d == 0 && lane == 0) {
        const S *g8 = reinterpret_cast<const S *>(A.gauge8) + ((size_t)A.p * A.g.Vh + cb0) * 8 * 18;
        bulk_copy(lnk + (size_t)(j & 1) * SITES * LB, g8, (uint32_t)(ns * LB), bar);
    }
}

// Packed coordinates of chunk j's sites handled by this lane (lane, lane+32, ...).
__device__ __forceinline__ void tma_load_coords(const HopArgs &A, int j, int SITES, uint32_t (&pre)[8]) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x + j * gridDim.x;
    const int cb0 = A.cb_begin + c * SITES;
    const int ns = min(SITES, A.cb_end - cb0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int s = lane + 32 * q;
        pre[q] = s < ns ? __ldg(A.coords + (size_t)A.p * A.g.Vh + cb0 + s) : 0u;
    }
}

template <typename S, int R, int MODE, int RED, int NST>
__global__ void __launch_bounds__(256) hop_kernel_tma(HopArgs A) {
    typedef typename Real<S>::type T;
    constexpr int NV = RedCount<RED>::n > 0 ? RedCount<RED>::n : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    const int G = A.N / R;
    const int lgG = __ffs(G) - 1;
    const int SITES = blockDim.x >> lgG;
    const size_t N = (size_t)A.N;
    const size_t SB = 12 * N * cbytes<S>();  // one site's spinor block
    const size_t LB = 8 * 9 * cbytes<S>();   // one site's eight links
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    unsigned char *stg = smem + 128;
    unsigned char *lnk = stg + (size_t)NST * SITES * SB;
    int *nbr = reinterpret_cast<int *>(lnk + (size_t)2 * SITES * LB);  // [2][SITES][8]
    const int nsite = A.cb_end - A.cb_begin;
    const int nchunks = (nsite + SITES - 1) / SITES;
    const int nmy = (int)blockIdx.x < nchunks ? (nchunks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int nsteps = nmy * 8;
    const T cD = (T)A.c;
    const int s_me = threadIdx.x >> lgG;
    const int r0 = (threadIdx.x & (G - 1)) * R;
    const int warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(full + i, 1);
        mbar_fence_init();
    }
    __syncthreads();
    // warp 0 holds the packed coordinates of the next chunk to be issued
    uint32_t pre[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int pre_chunk = -1;
    auto issue = [&](int kk) {
        const int jj = kk >> 3;
        if ((kk & 7) == 0 && pre_chunk != jj) tma_load_coords(A, jj, SITES, pre);
        tma_issue<S>(A, kk, SITES, NST, full, stg, lnk, nbr, SB, LB, pre);
        if ((kk & 7) == 0) {
            pre_chunk = jj + 1;
            if (jj + 1 < nmy) tma_load_coords(A, jj + 1, SITES, pre);  // lands before it is needed
        }
    };
    if (warp == 0)
        for (int k = 0; k < NST && k < nsteps; ++k) issue(k);

    cx<T> red[R][NV];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[r][k] = zero<T>();

    bool ok = true;
    int k = 0;                           // next step to wait for
    int issued = nsteps < NST ? nsteps : NST;  // steps issued so far
    for (int j = 0; j < nmy && ok; ++j) {
        const int c = blockIdx.x + j * gridDim.x;
        const int cb0 = A.cb_begin + c * SITES;
        const int ns = min(SITES, A.cb_end - cb0);
        const bool active = s_me < ns;
        const int cb = cb0 + s_me;
        // (the link rows carry the time boundary factor)
        const unsigned char *lrow = lnk + (size_t)(j & 1) * SITES * LB + (size_t)s_me * LB;
        cx<T> acc[R][12];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int cc = 0; cc < 12; ++cc) acc[r][cc] = zero<T>();
#define DL_TMA_STEP(D)                                                                                 \
        if (ok) {                                                                                      \
            const int slot = k % NST;                                                                  \
            const bool landed = mbar_wait(full + slot, (uint32_t)((k / NST) & 1));                     \
            if (landed && active)                                                                      \
                tma_compute<S, R, D>(stg + (size_t)slot * SITES * SB + (size_t)s_me * SB, lrow, A.N, r0, \
                                     false, acc);            \
            ok = __syncthreads_and(landed) != 0; /* block-uniform; the slot is free */                 \
            if (ok) {                                                                                  \
                if (warp == 0 && k + NST < nsteps) issue(k + NST);                                     \
                if (k + NST < nsteps) issued = k + NST + 1;                                            \
                ++k;                                                                                   \
            }                                                                                          \
        }
        DL_TMA_STEP(0) DL_TMA_STEP(1) DL_TMA_STEP(2) DL_TMA_STEP(3)
        DL_TMA_STEP(4) DL_TMA_STEP(5) DL_TMA_STEP(6) DL_TMA_STEP(7)
#undef DL_TMA_STEP
        if (!ok || !active) continue;
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
        // record the failure, then let every copy already issued land (bounded
        // waits) before the block releases its shared memory
        if (threadIdx.x == 0) {
            if (A.err) *(volatile int *)A.err = 1;
            bool drained = true;
            for (int kk = k; kk < issued; ++kk)
                drained &= mbar_wait(full + (kk % NST), (uint32_t)((kk / NST) & 1));
            // A drain wait that ran out leaves copies into this block's shared memory
            // pending after it exits; the host then refuses further work on the context.
            if (!drained && A.err) *(volatile int *)(A.err + 1) = 1;
        }
        return;
    }
    if (RED != RED_NONE) {
        __syncthreads();  // the reduction reuses the staging buffer
        block_reduce<R, NV, T>(red, G, A.N, A.partials, smem + 128);
    }
}

}  // namespace dl
