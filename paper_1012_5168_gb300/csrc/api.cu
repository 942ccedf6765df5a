// C ABI of the library (include/dloops.h): context, gauge field, sources, the
// batched mixed-precision even-odd BiCGStab solver with FP64 defect
// correction, loop contractions (local and smeared), exact loops and the
// truncated-solver-method estimate.  All arithmetic of the path runs in the
// CUDA kernels of this directory; the host code only sequences launches,
// owns workspaces and moves the final loop values to the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "dloops.h"
#include "fields.cuh"
#include "launch.h"
#include "momentum.cuh"

using namespace dl;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

__attribute__((visibility("hidden"))) int dl_record_error(int code, const char *msg) { return fail(code, msg); }

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(DL_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(call)                   \
    do {                            \
        int rc_ = (call);           \
        if (rc_ != DL_OK) return rc_; \
    } while (0)

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct TimedPair {
    cudaEvent_t a, b;
    int kind;
    double bytes;
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int n_kernels = 0;
    std::vector<TimedPair> timed;
};

struct dl_ctx {
    int dims[4];
    int t_bc;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = 0;      // caller's stream
    cudaStream_t cap_stream = 0;  // private stream used for graph capture
    cudaStream_t cur = 0;         // stream kernels are enqueued on right now
    bool capturing = false;
    Geom g;
    long V = 0, Vh = 0;
    double kappa = 0.0;
    bool have_gauge = false, have_kappa = false;

    uint32_t *d_coords = nullptr;
    double *d_gauge64 = nullptr;
    float *d_gauge32 = nullptr;
    bf16 *d_gauge16 = nullptr;
    float *d_gauge_ff = nullptr;   // float-float links (smearing)
    bool smear_fp64 = false;       // smear in native FP64 instead of float-float
    float *d_gauge8_32 = nullptr;  // site-major links (staged hop)
    bf16 *d_gauge8_16 = nullptr;
    float4 *d_gauge8q = nullptr;   // FP32 link quads of the packed-arithmetic hop
    float4 *d_gauge8d = nullptr;   // FP32 link quads (Re, Re, Im, Im) of the paired-layout hop
    bool f32_pairs = false;        // FP32 inner fields of even width in the paired layout (DLOOPS_F32_PAIRS=1)
    int *h_err = nullptr;          // pinned, mapped [2]: set by the staged hop on a wait timeout
    int *d_err = nullptr;
    bool poisoned = false;         // a staged hop may have left bulk copies pending: no further work
    bool skip_inactive = true;     // direct hops skip right-hand sides that stopped (DLOOPS_HOP_SKIP=0: off)
    double2 *d_gammas = nullptr;  // [16][4][4]
    // clover term (c_sw != 0): A and A^-1 per site, [2][Vh][2 blocks][6][6] complex
    double csw = 0.0;
    bool clover_stale = true;        // rebuild before the next use (links, kappa or c_sw changed)
    double2 *d_clov64 = nullptr;     // A (FP64)
    double2 *d_clovinv64 = nullptr;  // A^-1 in FP64, FP32 and BF16
    float2 *d_clovinv32 = nullptr;
    bf16 *d_clovinv16 = nullptr;

    // batch workspace, width ws_N (power of two)
    int ws_N = 0;
    double *b64 = nullptr, *x64 = nullptr;   // full fields [2][Vh][12][N]
    double *bh64 = nullptr, *r64 = nullptr;  // even halves
    double *t64 = nullptr;                   // odd half
    double *s64a = nullptr, *s64b = nullptr; // full fields (smearing)
    void *lo[8] = {nullptr};                 // inner fields: x r rhat p v s t (even) tmp (odd)
    RhsState *d_rhs = nullptr;
    OuterState *d_outer = nullptr;
    double2 *d_partials = nullptr;
    size_t partials_cap = 0;  // double2 elements
    double2 *d_loops = nullptr;  // [N][2 sinks][16][T]
    double2 *d_acc = nullptr;    // [2 sinks][T][16] exact-loop accumulators
    double2 *d_acc2 = nullptr;   // [64][2 sinks][16][T] grouped loops
    double *d_canon = nullptr;   // N canonical fields (internal sources)
    double2 *d_noise = nullptr;  // per-noise loops (TSM)
    size_t noise_cap = 0;
    double2 *d_w = nullptr;      // gamma weights / spin matrices
    size_t w_cap = 0;
    int *d_tcol = nullptr;       // per-column timeslice of the current batch (64 ints)
    // momentum projection and correlators (grown on demand)
    struct Scratch {
        void *p = nullptr;
        size_t cap = 0;
    };
    Scratch s_phase, s_site, s_msum, s_mloops, s_mgroup, s_mom, s_cover, s_out;

    int *h_count = nullptr;  // pinned, mapped
    int *d_count = nullptr;

    std::map<std::tuple<int, int, int, int>, GraphEntry> graphs;
    bool timing = false;
    std::vector<TimedPair> pending;  // recorded eagerly, harvested at the next sync
    std::vector<cudaEvent_t> event_pool;
    dl_timing tim;
    int64_t kernel_launches = 0;
    // Launch shape of the Wilson hop per [prec][log2 N][m]: m = 0 the plain hop
    // (D_oe p, D_oe s), 1 the fused hops other than BiCGStab's second (XPAY with
    // <rhat, v> or a norm), 2 the fused hop with the five BiCGStab reductions.
    // Each is tuned on its own, so they may use different kernels.
    int hop_R[5][8][3];      // right-hand sides per thread
    int hop_block[5][8][3];  // threads per block
    int hop_kind[5][8][3];   // 0 direct, 1 cp.async prefetching, 2 bulk-copy staged, 3 blocked, 4 warp-staged,
                          // 5 tensor cores (BF16), 6 direct with packed FP32 arithmetic, 7 paired layout with
                          // packed FP32 arithmetic, 8 the same under a 128-register cap, 9 paired and
                          // warp-staged, 10 direct under a wider register cap, 11 warp-staged with two stages
    bool hop_tuned[5][8];
    bool autotune = true;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}
static int pow2_at_least(int n) { return 1 << ilog2(n < 1 ? 1 : n); }

static Launch make_launch(dl_ctx *c, long items, int block, size_t smem, int per_sm) {
    Launch l;
    l.num_sms = 0;
    long need = (items + block - 1) / block;
    long cap = (long)c->num_sms * per_sm;
    l.grid = (int)std::max(1L, std::min(need, cap));
    l.block = block;
    l.smem = smem;
    l.stream = c->cur;
    return l;
}

static size_t half_elems(dl_ctx *c, int N) { return (size_t)c->Vh * 12 * N; }  // complex per half field

static int storage_bytes(int prec) {
    return (prec == P_F64 || prec == P_DFF) ? 8 : ((prec == P_F32 || prec == P_F32P) ? 4 : 2);
}

// The storage of a solve's inner fields: FP32 of even width in the paired layout
// (two right-hand sides per 16-byte group) when the context uses it.
static int inner_prec(const dl_ctx *c, int prec, int N) {
    return (prec == P_F32 && c->f32_pairs && N >= 2) ? P_F32P : prec;
}

static cudaEvent_t get_event(dl_ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void harvest(dl_ctx *c, std::vector<TimedPair> &v, bool release) {
    for (auto &tp : v) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, tp.a, tp.b) == cudaSuccess) {
            c->tim.hop_ms[tp.kind] += ms;
            c->tim.hop_launches[tp.kind] += 1;
            c->tim.hop_bytes[tp.kind] += tp.bytes;
        }
        if (release) {
            c->event_pool.push_back(tp.a);
            c->event_pool.push_back(tp.b);
        }
    }
    if (release) v.clear();
}

static int sync(dl_ctx *c) {
    CK(cudaStreamSynchronize(c->stream));
    harvest(c, c->pending, true);
    if (c->h_err && (((volatile int *)c->h_err)[0] || ((volatile int *)c->h_err)[1])) {
        if (((volatile int *)c->h_err)[1]) c->poisoned = true;
        ((volatile int *)c->h_err)[0] = 0;
        return fail(DL_ECUDA, c->poisoned ? "staged Wilson hop: a bounded wait ran out and bulk copies may still be "
                                            "pending; the context takes no further work"
                                          : "staged Wilson hop: a bounded wait for a bulk copy ran out");
    }
    return DL_OK;
}

static void record(dl_ctx *c, cudaEvent_t e) {
    if (c->capturing) cudaEventRecordWithFlags(e, c->cur, cudaEventRecordExternal);
    else cudaEventRecord(e, c->cur);
}

// Wilson hop launch.  kind >= 0 marks launches timed with CUDA events.
// P_DFF: `in` is float-float; ffmt flags FF_Y / FF_OUT give the formats of y and out.
// The tuning class of a hop: 0 plain, 1 fused (other than BICG), 2 fused with the five reductions.
static int hop_class(int mode, int red) {
    return (mode == MODE_PLAIN && red == RED_NONE) ? 0 : (red == RED_BICG ? 2 : 1);
}

// clov: the clover solve's inner hop A^-1 D (A^-1 of the output parity p in the epilogue;
// FP64, FP32 or BF16 storage, the direct kernel with one right-hand side per thread).
static int do_hop(dl_ctx *c, int prec, int mode, int red, void *out, const void *in, const void *y, const void *z,
                  const void *rhat, int p, int N, double coef, int cb0, int cb1, double2 *partials, int *nblocks,
                  int ffmt = 0, const RhsState *act = nullptr, bool clov = false) {
    if (c->poisoned) return fail(DL_ECUDA, "context unusable: a staged hop left bulk copies pending");
    if (clov && (prec == P_DFF || !c->d_clovinv64)) return fail(DL_EINVAL, "clover hop: no A^-1 for this storage");
    HopArgs a;
    a.out = out;
    a.in = in;
    a.y = y;
    a.z = z;
    a.rhat = rhat;
    const bool wide = prec == P_F64 || prec == P_DFF;  // FP64 fields, one right-hand side per thread
    const bool f32 = prec == P_F32 || prec == P_F32P;
    a.gauge = prec == P_F64   ? (const void *)c->d_gauge64
              : prec == P_DFF ? (const void *)c->d_gauge_ff
              : f32           ? (const void *)c->d_gauge32
                              : (const void *)c->d_gauge16;
    a.coords = c->d_coords;
    a.partials = partials;
    a.p = p;
    a.N = N;
    a.cb_begin = cb0;
    a.cb_end = cb1;
    a.c = coef;
    a.g = c->g;
    a.gauge8 = f32 ? (const void *)c->d_gauge8_32 : (prec == P_BF16 ? (const void *)c->d_gauge8_16 : nullptr);
    a.gauge8d = c->d_gauge8d;
    a.err = c->d_err;
    a.blocked = 0;
    a.gauge8q = c->d_gauge8q;
    // per-RHS participation flags (BiCGStab inner iterations): next_active holds for the whole iteration
    a.act = act && c->skip_inactive ? &act[0].next_active : nullptr;
    a.act_stride = (int)(sizeof(RhsState) / sizeof(int));
    a.clovinv = !clov ? nullptr
                : prec == P_F64 ? (const void *)c->d_clovinv64
                : f32           ? (const void *)c->d_clovinv32
                                : (const void *)c->d_clovinv16;
    const int m = hop_class(mode, red);  // the shape tables' entry
    int R = (wide || clov) ? 1 : c->hop_R[prec][ilog2(N)][m];
    if (R > N) R = N;
    const int G = N / R;
    int block = prec == P_DFF ? 192 : c->hop_block[prec][ilog2(N)][m];  // P_DFF: a multiple of 3 N
    if (block % G) block = 128;  // a multiple of G (N <= 64)
    const long total = (long)(cb1 - cb0) * G * (prec == P_DFF ? 3 : 1);
    const int NV = red == RED_BICG ? 5 : (red == RED_NONE ? 0 : 1);
    const int kind = (wide || clov) ? 0 : c->hop_kind[prec][ilog2(N)][m];
    size_t smem = NV ? (size_t)(block / 32) * std::min(G, 32) * R * NV * (wide ? 16 : 8) : 0;
    int per_sm = wide ? 4 : 8;
    long items = total;
    if (kind == 1) {
        smem = std::max(smem, 2 * pf_stage_bytes(prec, R) * block);
        per_sm = 4;
    } else if (kind == 2) {
        const int sites = block / G;
        smem = std::max(smem, tma_smem_bytes(prec, N, sites));
        per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(220 * 1024) / smem));
        items = (long)((cb1 - cb0 + sites - 1) / sites) * block;  // one chunk per block at a time
    }
    Launch l = make_launch(c, items, block, smem, (kind == 0 || kind == 10) ? 16 : per_sm);
    // the direct and warp-staged kernels size their grid from residency
    if (kind == 0 || kind >= 3) l.num_sms = c->num_sms;
    const bool timed = c->timing;
    TimedPair tp;
    if (timed) {
        tp.a = get_event(c);
        tp.b = get_event(c);
        tp.kind = (wide ? 2 : 0) + (mode != MODE_PLAIN || red != RED_NONE ? 1 : 0);
        const double S = 24.0 * storage_bytes(prec), L = 18.0 * storage_bytes(prec);
        int streams = 2 + (mode != MODE_PLAIN ? 1 : 0) + (mode == MODE_RESID ? 1 : 0) +
                      ((red == RED_R0DOT || red == RED_BICG) ? 1 : 0);
        if (red == RED_BICG && mode == MODE_PLAIN) streams += 1;
        tp.bytes = (double)(cb1 - cb0) * (8.0 * L + (double)N * streams * S);
        if (clov) tp.bytes += (double)(cb1 - cb0) * 72.0 * 2.0 * storage_bytes(prec);  // A^-1 of each output site
        record(c, tp.a);
    }
    cudaError_t e;
    if (prec == P_F64) e = launch_hop_f64(R, mode, red, a, l);
    else if (prec == P_DFF) e = launch_hop_ff(mode, red, ffmt, a, l);
    else if (prec == P_F32) e = launch_hop_f32(R, mode, red, kind, a, l);
    else if (prec == P_F32P) e = launch_hop_f32p(R, mode, red, kind, a, l);
    else e = launch_hop_bf16(R, mode, red, kind, a, l);
    if (e != cudaSuccess) return fail(DL_ECUDA, std::string("hop launch: ") + cudaGetErrorString(e));
    if (nblocks) *nblocks = l.grid;
    c->kernel_launches++;
    if (timed) {
        record(c, tp.b);
        c->pending.push_back(tp);
    }
    return DL_OK;
}

static VecLaunch vec_launch(dl_ctx *c, int prec, int N, size_t smem_per_val, int per_sm = 8) {
    VecLaunch v;
    v.prec = prec;
    v.R = prec == P_F64 ? 1 : std::min(2, N);
    v.a.n_elem = (int)(c->Vh * 12);
    v.a.N = N;
    const int block = 256;  // a multiple of G (N <= 64)
    const int G = N / v.R;
    v.l = make_launch(c, (long)v.a.n_elem * G, block, (size_t)(block / 32) * std::min(G, 32) * v.R * smem_per_val,
                      per_sm);
    return v;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
static void free_ws(dl_ctx *c) {
    for (auto &kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto &tp : kv.second.timed) {
            c->event_pool.push_back(tp.a);
            c->event_pool.push_back(tp.b);
        }
    }
    c->graphs.clear();
    double **d64[] = {&c->b64, &c->x64, &c->bh64, &c->r64, &c->t64, &c->s64a, &c->s64b, &c->d_canon};
    for (auto pp : d64) {
        if (*pp) cudaFree(*pp);
        *pp = nullptr;
    }
    for (auto &p : c->lo) {
        if (p) cudaFree(p);
        p = nullptr;
    }
    if (c->d_rhs) cudaFree(c->d_rhs);
    if (c->d_outer) cudaFree(c->d_outer);
    if (c->d_loops) cudaFree(c->d_loops);
    c->d_rhs = nullptr;
    c->d_outer = nullptr;
    c->d_loops = nullptr;
    c->ws_N = 0;
}

static void invalidate_graphs(dl_ctx *c) {
    for (auto &kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto &tp : kv.second.timed) {
            c->event_pool.push_back(tp.a);
            c->event_pool.push_back(tp.b);
        }
    }
    c->graphs.clear();
}

static int ensure_ws(dl_ctx *c, int N) {
    if (c->ws_N >= N) return DL_OK;
    N = pow2_at_least(N);
    CK(cudaStreamSynchronize(c->stream));
    free_ws(c);
    const size_t half = half_elems(c, N) * 16;  // bytes of an FP64 half field
    double **full[] = {&c->b64, &c->x64, &c->s64a, &c->s64b};
    for (auto pp : full)
        if (cudaMalloc((void **)pp, 2 * half) != cudaSuccess) return fail(DL_ENOMEM, "workspace allocation failed");
    double **halves[] = {&c->bh64, &c->r64, &c->t64};
    for (auto pp : halves)
        if (cudaMalloc((void **)pp, half) != cudaSuccess) return fail(DL_ENOMEM, "workspace allocation failed");
    for (auto &p : c->lo)
        if (cudaMalloc(&p, half) != cudaSuccess) return fail(DL_ENOMEM, "workspace allocation failed");
    if (cudaMalloc((void **)&c->d_canon, 2 * half) != cudaSuccess) return fail(DL_ENOMEM, "workspace allocation failed");
    if (cudaMalloc((void **)&c->d_rhs, sizeof(RhsState) * N) != cudaSuccess ||
        cudaMalloc((void **)&c->d_outer, sizeof(OuterState) * N) != cudaSuccess ||
        cudaMalloc((void **)&c->d_loops, sizeof(double2) * N * 2 * 16 * c->dims[3]) != cudaSuccess)
        return fail(DL_ENOMEM, "workspace allocation failed");
    CK(cudaMemset(c->b64, 0, 2 * half));
    CK(cudaMemset(c->x64, 0, 2 * half));
    for (auto &p : c->lo) CK(cudaMemset(p, 0, half));
    c->ws_N = N;
    return DL_OK;
}

static int ensure_partials(dl_ctx *c, size_t elems) {
    if (c->partials_cap >= elems) return DL_OK;
    CK(cudaStreamSynchronize(c->stream));
    invalidate_graphs(c);
    if (c->d_partials) cudaFree(c->d_partials);
    c->d_partials = nullptr;
    if (cudaMalloc((void **)&c->d_partials, elems * sizeof(double2)) != cudaSuccess)
        return fail(DL_ENOMEM, "partials allocation failed");
    c->partials_cap = elems;
    return DL_OK;
}

// ---------------------------------------------------------------------------
// autotuner: right-hand sides per thread and block size of the Wilson hop
// ---------------------------------------------------------------------------
// Times, for each candidate launch shape on random fields of width N, the plain
// hop and the fused hop with the five BiCGStab reductions (one of each per
// inner half-iteration), and keeps the fastest shape for each.  Uses the inner
// workspace, so it runs before a solve fills it.
// which: bit 0 the plain hop, bit 1 the fused one with the five reductions, bit 2
// the fused one with <rhat, v>.
static int time_hops(dl_ctx *c, int prec, int N, int reps, float *ms_out, int which = 3) {
    const int Vh = (int)c->Vh;
    cudaEvent_t e0 = get_event(c), e1 = get_event(c);
    const bool was = c->timing;
    c->timing = false;
    int rc = DL_OK;
    for (int it = -1; it < reps && rc == DL_OK; ++it) {
        if (it == 0) cudaEventRecord(e0, c->cur);
        if (which & 1)
            rc = do_hop(c, prec, MODE_PLAIN, RED_NONE, c->lo[7], c->lo[3], nullptr, nullptr, nullptr, 1, N, 1.0, 0,
                        Vh, nullptr, nullptr);
        if (rc == DL_OK && (which & 2))
            rc = do_hop(c, prec, MODE_XPAY, RED_BICG, c->lo[6], c->lo[7], c->lo[5], nullptr, c->lo[2], 0, N, -0.02, 0,
                        Vh, c->d_partials, nullptr);
        if (rc == DL_OK && (which & 4))
            rc = do_hop(c, prec, MODE_XPAY, RED_R0DOT, c->lo[4], c->lo[7], c->lo[3], nullptr, c->lo[2], 0, N, -0.02, 0,
                        Vh, c->d_partials, nullptr);
    }
    cudaEventRecord(e1, c->cur);
    c->timing = was;
    float ms = 0.f;
    if (rc == DL_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    c->event_pool.push_back(e0);
    c->event_pool.push_back(e1);
    *ms_out = ms / reps;
    return rc;
}

// Whether kernel kind pf can run the hop of width N in storage prec with R
// right-hand sides per thread and B threads per block (bi: B's index in
// {64, 128, 256}).
static bool shape_ok(int prec, int N, int R, int B, int bi, int pf) {
    if (pf < 0 || pf > 11 || (prec == P_F64 && (pf != 0 || R != 1))) return false;
    if (pf == 10 && (prec != P_F32 || R != 1)) return false;       // wider-cap direct: FP32, one per thread
    if (prec == P_F32P ? (pf != 0 && (pf < 7 || pf > 9)) : (pf >= 7 && pf <= 9)) return false;  // paired: 0, 7-9
    if (pf == 11 && prec == P_F32P) return false;
    if (R > N || B % (N / R)) return false;
    if (pf == 1 && 2 * pf_stage_bytes(prec, R) * B > 200 * 1024) return false;
    if ((pf == 3 || pf == 4 || pf == 5 || pf == 11) && bi > 0) return false;  // the launcher picks the block
    if ((pf == 4 || pf == 5 || pf == 11) && N != 32 * R) return false;         // one site per warp
    if (pf == 5 && (prec != P_BF16 || R > 2)) return false;         // tensor cores: BF16 storage
    if (pf == 6 && (prec != P_F32 || R != 1)) return false;         // packed FP32 arithmetic
    if (pf >= 7 && pf <= 9 && R != 2) return false;                 // paired layout: two per thread
    if (pf == 9 && (bi > 0 || (N != 32 && N != 64))) return false;  // warp-staged pairs: N = 32, 64
    if (pf == 2 && (B / (N / R) < 1 || tma_smem_bytes(prec, N, B / (N / R)) > 200 * 1024)) return false;
    return true;
}

static int tune_hop(dl_ctx *c, int prec, int N, int force_R, int force_block, int force_pf) {
    const int l = ilog2(N);
    TRY(ensure_ws(c, N));
    TRY(ensure_partials(c, (size_t)2 * c->num_sms * 16 * N * 16));
    c->cur = c->stream;
    const size_t ne = half_elems(c, N);
    for (int k = 0; k < 8; ++k) CK(launch_fill(prec, c->lo[k], ne, 77u + k, c->stream));
    float best[3] = {1e30f, 1e30f, 1e30f}, best0[3] = {1e30f, 1e30f, 1e30f};  // per class: all kinds; kind 0
    int bR[3], bB[3], bP[3], b0R[3], b0B[3];
    const int which_of[3] = {1, 4, 2};  // the hop time_hops times for each class
    for (int m = 0; m < 3; ++m) {
        bR[m] = b0R[m] = c->hop_R[prec][l][m];
        bB[m] = b0B[m] = c->hop_block[prec][l][m];
        bP[m] = c->hop_kind[prec][l][m];
    }
    const int Rs[3] = {1, 2, 4}, Bs[3] = {64, 128, 256};
    // Two sweeps over the shapes, keeping each shape's faster time, so that a
    // shape timed while the GPU was still ramping its clocks or finishing other
    // work gets a second chance.
    for (int sweep = 0; sweep < 2; ++sweep)
    for (int pf = 0; pf < (prec == P_F64 ? 1 : 12); ++pf) {
        if (force_pf >= 0 && pf != force_pf) continue;
        for (int ri = 0; ri < 3; ++ri) {
            const int R = Rs[ri];
            if (force_R && R != force_R) continue;
            for (int bi = 0; bi < 3; ++bi) {
                const int B = Bs[bi];
                if (force_block && B != force_block) continue;
                if (!shape_ok(prec, N, R, B, bi, pf)) continue;
                for (int m = 0; m < 3; ++m) {
                    c->hop_R[prec][l][m] = R;
                    c->hop_block[prec][l][m] = B;
                    c->hop_kind[prec][l][m] = pf;
                }
                for (int m = 0; m < 3; ++m) {
                    float ms = 0.f;
                    TRY(time_hops(c, prec, N, 5, &ms, which_of[m]));
                    if (ms > 0.f && ms < best[m]) {
                        best[m] = ms;
                        bR[m] = R;
                        bB[m] = B;
                        bP[m] = pf;
                    }
                    if (pf == 0 && ms > 0.f && ms < best0[m]) {
                        best0[m] = ms;
                        b0R[m] = R;
                        b0B[m] = B;
                    }
                }
            }
        }
    }
    // Another kind replaces the direct kernel only when it is faster by more than
    // 2%: closer than that, which one wins is timing noise (on GB300 the
    // warp-staged kernel and the direct one are within 1% at some widths).
    for (int m = 0; m < 3; ++m) {
        if (bP[m] != 0 && best0[m] < 1e30f && best[m] > 0.98f * best0[m]) {
            bR[m] = b0R[m];
            bB[m] = b0B[m];
            bP[m] = 0;
        }
        c->hop_R[prec][l][m] = bR[m];
        c->hop_block[prec][l][m] = bB[m];
        c->hop_kind[prec][l][m] = bP[m];
    }
    c->hop_tuned[prec][l] = true;
    invalidate_graphs(c);
    return DL_OK;
}

extern "C" int dl_tune_hop(dl_ctx *c, int precision, int n_rhs, int force_R, int force_block, int force_pf,
                           int *R_out, int *block_out, int *pf_out, double *ms_out) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (!c->have_gauge) return fail(DL_ESTATE, "load_gauge has not been called");
    if (precision < 0 || precision > 2 || n_rhs < 1 || n_rhs > 64) return fail(DL_EINVAL, "bad arguments");
    if (force_R < 0 || force_block < 0) return fail(DL_EINVAL, "bad forced shape");
    const int N = pow2_at_least(n_rhs);
    const int ip = inner_prec(c, precision, N);
    if (force_pf >= 0 && (ip == P_F32P ? (force_pf != 0 && (force_pf < 7 || force_pf > 9))
                                       : (force_pf >= 7 && force_pf <= 9)))
        return fail(DL_EINVAL, "kernel kind not available for this storage layout");
    TRY(tune_hop(c, ip, N, force_R, force_block, force_pf));
    const int l = ilog2(N);
    if (R_out) *R_out = c->hop_R[ip][l][2];
    if (block_out) *block_out = c->hop_block[ip][l][2];
    if (pf_out) *pf_out = c->hop_kind[ip][l][2];
    if (ms_out) {
        float ms = 0.f;
        TRY(time_hops(c, ip, N, 10, &ms));
        *ms_out = ms;
    }
    return DL_OK;
}

// The launch shape the context uses for one class of hops (0 plain, 1 fused,
// 2 fused with the five reductions) of width n_rhs in the inner solver's
// storage for `precision` (no tuning).
extern "C" int dl_hop_shape(dl_ctx *c, int precision, int n_rhs, int cls, int *R_out, int *block_out,
                            int *kind_out) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (precision < 0 || precision > 2 || n_rhs < 1 || n_rhs > 64 || cls < 0 || cls > 2)
        return fail(DL_EINVAL, "bad arguments");
    const int N = pow2_at_least(n_rhs), l = ilog2(N), ip = inner_prec(c, precision, N), m = cls;
    if (R_out) *R_out = c->hop_R[ip][l][m];
    if (block_out) *block_out = c->hop_block[ip][l][m];
    if (kind_out) *kind_out = c->hop_kind[ip][l][m];
    return DL_OK;
}

// Set the launch shape of one class of hops of this width explicitly (it then
// counts as tuned).
extern "C" int dl_set_hop_shape(dl_ctx *c, int precision, int n_rhs, int cls, int R, int block, int kind) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (precision < 0 || precision > 2 || n_rhs < 1 || n_rhs > 64 || cls < 0 || cls > 2)
        return fail(DL_EINVAL, "bad arguments");
    const int N = pow2_at_least(n_rhs), l = ilog2(N), ip = inner_prec(c, precision, N), m = cls;
    const int bi = block == 64 ? 0 : (block == 128 ? 1 : (block == 256 ? 2 : -1));
    if ((R != 1 && R != 2 && R != 4) || bi < 0 || !shape_ok(ip, N, R, block, bi, kind))
        return fail(DL_EINVAL, "launch shape not available for this precision, width and layout");
    c->hop_R[ip][l][m] = R;
    c->hop_block[ip][l][m] = block;
    c->hop_kind[ip][l][m] = kind;
    c->hop_tuned[ip][l] = true;
    invalidate_graphs(c);
    return DL_OK;
}

static int maybe_tune(dl_ctx *c, int prec, int N) {
    prec = inner_prec(c, prec, N);
    if (!c->autotune || c->hop_tuned[prec][ilog2(N)]) return DL_OK;
    return tune_hop(c, prec, N, 0, 0, -1);
}

// ---------------------------------------------------------------------------
// gamma basis (chiral DeGrand-Rossi), host construction
// ---------------------------------------------------------------------------
typedef std::complex<double> zc;

static void gamma_basis(zc out[16][4][4]) {
    const zc I(0, 1), O(0, 0), one(1, 0);
    zc g[4][4][4] = {
        {{O, O, O, I}, {O, O, I, O}, {O, -I, O, O}, {-I, O, O, O}},
        {{O, O, O, -one}, {O, O, one, O}, {O, one, O, O}, {-one, O, O, O}},
        {{O, O, I, O}, {O, O, O, -I}, {-I, O, O, O}, {O, I, O, O}},
        {{O, O, one, O}, {O, O, O, one}, {one, O, O, O}, {O, one, O, O}},
    };
    auto mul = [](const zc a[4][4], const zc b[4][4], zc r[4][4]) {
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                zc s = 0;
                for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
                r[i][j] = s;
            }
    };
    zc g5[4][4], t1[4][4], t2[4][4];
    mul(g[0], g[1], t1);
    mul(t1, g[2], t2);
    mul(t2, g[3], g5);
    int n = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) out[n][i][j] = (i == j) ? one : O;
    ++n;
    for (int m = 0; m < 4; ++m, ++n)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) out[n][i][j] = g[m][i][j];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) out[n][i][j] = g5[i][j];
    ++n;
    for (int m = 0; m < 4; ++m, ++n) mul(g5, g[m], out[n]);
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b, ++n) mul(g[a], g[b], out[n]);
}

// ---------------------------------------------------------------------------
// context API
// ---------------------------------------------------------------------------
extern "C" const char *dl_last_error(void) { return g_err.c_str(); }

extern "C" const char *dl_status_string(int s) {
    switch (s) {
        case DL_OK: return "ok";
        case DL_EINVAL: return "invalid argument";
        case DL_ENOMEM: return "out of device memory";
        case DL_ECUDA: return "CUDA error";
        case DL_NOT_CONVERGED: return "not converged";
        case DL_BREAKDOWN: return "BiCGStab breakdown";
        case DL_NAN: return "non-finite value";
        case DL_ESTATE: return "call out of order";
        default: return "unknown status";
    }
}

extern "C" int dl_create(dl_ctx **out, const int dims[4], int t_bc, void *cuda_stream) {
    if (!out || !dims) return fail(DL_EINVAL, "null argument");
    *out = nullptr;
    for (int m = 0; m < 4; ++m)
        if (dims[m] < 2 || dims[m] > 256) return fail(DL_EINVAL, "lattice extents must lie in [2, 256]");
    for (int m = 0; m < 4; ++m)
        if (dims[m] % 2) return fail(DL_EINVAL, "every lattice extent must be even (even-odd preconditioning)");
    if (t_bc != 1 && t_bc != -1) return fail(DL_EINVAL, "t_bc must be +1 or -1");
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V * 32 >= (1L << 31)) return fail(DL_EINVAL, "lattice too large for 32-bit thread indexing");
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(DL_ECUDA, "no CUDA device");
    CK(cudaGetDevice(&dev));
    dl_ctx *c = new dl_ctx();
    memcpy(c->dims, dims, sizeof(c->dims));
    c->t_bc = t_bc;
    c->device = dev;
    {
        const char *e = getenv("DLOOPS_SMEAR_FP64");
        c->smear_fp64 = e && e[0] == '1';
        const char *k = getenv("DLOOPS_HOP_SKIP");
        c->skip_inactive = !(k && k[0] == '0');
        const char *pr = getenv("DLOOPS_F32_PAIRS");
        c->f32_pairs = pr && pr[0] == '1';
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    c->stream = (cudaStream_t)cuda_stream;
    c->cur = c->stream;
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return fail(DL_ECUDA, "stream creation failed");
    }
    c->V = V;
    c->Vh = V / 2;
    for (int m = 0; m < 4; ++m) c->g.L[m] = dims[m];
    c->g.stride[0] = 1;
    c->g.stride[1] = dims[0];
    c->g.stride[2] = dims[0] * dims[1];
    c->g.stride[3] = dims[0] * dims[1] * dims[2];
    c->g.Vh = (int)c->Vh;
    c->g.V3h = dims[0] * dims[1] * dims[2] / 2;
    c->g.t_bc = t_bc;
    memset(&c->tim, 0, sizeof(c->tim));
    for (int p = 0; p < 5; ++p)
        for (int l = 0; l < 8; ++l) {
            for (int m = 0; m < 3; ++m) {
                c->hop_R[p][l][m] = 2;
                c->hop_block[p][l][m] = 128;
                c->hop_kind[p][l][m] = 0;
            }
            c->hop_tuned[p][l] = false;
        }
    // coordinates table
    std::vector<uint32_t> coords(V);
    for (int t = 0; t < dims[3]; ++t)
        for (int z = 0; z < dims[2]; ++z)
            for (int y = 0; y < dims[1]; ++y)
                for (int x = 0; x < dims[0]; ++x) {
                    const long i = x + (long)dims[0] * (y + (long)dims[1] * (z + (long)dims[2] * t));
                    const int p = (x + y + z + t) & 1;
                    coords[p * c->Vh + (i >> 1)] = (uint32_t)x | ((uint32_t)y << 8) | ((uint32_t)z << 16) |
                                                   ((uint32_t)t << 24);
                }
    zc gam[16][4][4];
    gamma_basis(gam);
    std::vector<double2> gh(256);
    for (int n = 0; n < 16; ++n)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) gh[(n * 4 + i) * 4 + j] = make_double2(gam[n][i][j].real(), gam[n][i][j].imag());
    int rc = DL_OK;
    if (cudaMalloc((void **)&c->d_coords, V * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_gammas, 256 * sizeof(double2)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_acc, 2 * 16 * dims[3] * sizeof(double2)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_tcol, 64 * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&c->d_acc2, (size_t)64 * 2 * 16 * dims[3] * sizeof(double2)) != cudaSuccess ||
        cudaHostAlloc((void **)&c->h_count, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->d_count, c->h_count, 0) != cudaSuccess ||
        cudaHostAlloc((void **)&c->h_err, 2 * sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->d_err, c->h_err, 0) != cudaSuccess)
        rc = fail(DL_ENOMEM, "context allocation failed");
    if (rc == DL_OK) c->h_err[0] = c->h_err[1] = 0;
    if (rc == DL_OK &&
        (cudaMemcpy(c->d_coords, coords.data(), V * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(c->d_gammas, gh.data(), 256 * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess))
        rc = fail(DL_ECUDA, "context upload failed");
    if (rc != DL_OK) {
        dl_destroy(c);
        return rc;
    }
    *out = c;
    return DL_OK;
}

extern "C" int dl_destroy(dl_ctx *c) {
    if (!c) return DL_OK;
    cudaStreamSynchronize(c->stream);
    free_ws(c);
    for (auto e : c->event_pool) cudaEventDestroy(e);
    for (auto &tp : c->pending) {
        cudaEventDestroy(tp.a);
        cudaEventDestroy(tp.b);
    }
    void *ptrs[] = {c->d_coords,   c->d_gauge64, c->d_gauge32,  c->d_gauge16, c->d_gauge8_32, c->d_gauge8_16, c->d_gauge8q,
                    c->d_gauge8d,
                    c->d_gauge_ff, c->d_gammas,  c->d_partials, c->d_acc,     c->d_noise,     c->d_w,
                    c->d_tcol,     c->d_acc2,    c->d_clov64,   c->d_clovinv64, c->d_clovinv32, c->d_clovinv16};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (dl_ctx::Scratch *sc : {&c->s_phase, &c->s_site, &c->s_msum, &c->s_mloops, &c->s_mgroup, &c->s_mom,
                                &c->s_cover, &c->s_out})
        if (sc->p) cudaFree(sc->p);
    if (c->h_count) cudaFreeHost(c->h_count);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return DL_OK;
}

extern "C" int dl_load_gauge(dl_ctx *c, const double *U, int check) {
    if (!c || !U) return fail(DL_EINVAL, "null argument");
    const long nlink = 4 * c->V;
    if (check) {
        for (long l = 0; l < nlink; ++l) {
            const double *u = U + l * 18;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double re = 0, im = 0;  // (U U^dag)_{ab}
                    for (int k = 0; k < 3; ++k) {
                        const double ar = u[(a * 3 + k) * 2], ai = u[(a * 3 + k) * 2 + 1];
                        const double br = u[(b * 3 + k) * 2], bi = -u[(b * 3 + k) * 2 + 1];
                        re += ar * br - ai * bi;
                        im += ar * bi + ai * br;
                    }
                    if (std::fabs(re - (a == b ? 1.0 : 0.0)) > 1e-10 || std::fabs(im) > 1e-10 || !std::isfinite(re))
                        return fail(DL_EINVAL, "gauge link is not unitary");
                }
        }
    }
    const size_t n64 = (size_t)nlink * 18;
    if (!c->d_gauge64) {
        if (cudaMalloc((void **)&c->d_gauge64, n64 * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_gauge32, n64 * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_gauge16, n64 * sizeof(bf16)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_gauge8_32, 2 * n64 * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_gauge8_16, 2 * n64 * sizeof(bf16)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_gauge8q, (size_t)c->V * 72 * sizeof(float4)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_gauge8d, (size_t)c->V * 72 * sizeof(float4)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_gauge_ff, 2 * n64 * sizeof(float)) != cudaSuccess)
            return fail(DL_ENOMEM, "gauge allocation failed");
    }
    double *tmp = nullptr;
    if (cudaMalloc((void **)&tmp, n64 * sizeof(double)) != cudaSuccess) return fail(DL_ENOMEM, "gauge staging failed");
    c->cur = c->stream;
    int rc = DL_OK;
    if (cudaMemcpyAsync(tmp, U, n64 * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
        rc = fail(DL_ECUDA, "gauge upload failed");
    } else {
        const int grid = std::max(1, std::min((int)((2 * c->Vh + 255) / 256), c->num_sms * 8));
        gauge_reorder_kernel<double><<<grid, 256, 0, c->stream>>>(c->d_coords, c->g, tmp, c->d_gauge64);
        gauge_reorder_kernel<float><<<grid, 256, 0, c->stream>>>(c->d_coords, c->g, tmp, c->d_gauge32);
        gauge_reorder_kernel<bf16><<<grid, 256, 0, c->stream>>>(c->d_coords, c->g, tmp, c->d_gauge16);
        gauge8_kernel<float><<<grid, 256, 0, c->stream>>>(c->d_coords, c->g, tmp, c->d_gauge8_32);
        gauge8_kernel<bf16><<<grid, 256, 0, c->stream>>>(c->d_coords, c->g, tmp, c->d_gauge8_16);
        gauge8q_kernel<<<grid, 256, 0, c->stream>>>(c->d_coords, c->g, tmp, c->d_gauge8q);
        gauge8d_kernel<<<grid, 256, 0, c->stream>>>(c->d_coords, c->g, tmp, c->d_gauge8d);
        gauge_ff_kernel<<<grid, 256, 0, c->stream>>>(c->d_gauge64, c->d_gauge_ff, (long)n64 / 2);
        c->kernel_launches += 8;
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
            rc = fail(DL_ECUDA, "gauge reorder failed");
    }
    cudaFree(tmp);
    if (rc == DL_OK) c->have_gauge = true;
    c->clover_stale = true;
    return rc;
}

extern "C" int dl_set_kappa(dl_ctx *c, double kappa) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (!std::isfinite(kappa)) return fail(DL_EINVAL, "kappa must be finite");
    if (kappa != c->kappa) {
        invalidate_graphs(c);
        c->clover_stale = true;
    }
    c->kappa = kappa;
    c->have_kappa = true;
    return DL_OK;
}

// Clover term: A = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu} per site,
// built from the FP64 links before the next operation that needs it.
extern "C" int dl_set_clover(dl_ctx *c, double c_sw) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (!std::isfinite(c_sw)) return fail(DL_EINVAL, "c_sw must be finite");
    if (c_sw != c->csw) {
        CK(cudaStreamSynchronize(c->stream));
        invalidate_graphs(c);  // the inner hops change kernel
        c->clover_stale = true;
    }
    c->csw = c_sw;
    return DL_OK;
}

// The clover blocks for the current links, kappa and c_sw (no-op without clover or
// when they are current).  sigma_{mu nu} = (i/2)[g_mu, g_nu] from the context's
// chiral gamma matrices, whose 2 x 2 spin blocks are all it keeps.
static int ensure_clover(dl_ctx *c) {
    if (c->csw == 0.0 || !c->clover_stale) return DL_OK;
    const size_t n = (size_t)c->V * 72;  // complex entries
    if (!c->d_clov64) {
        if (cudaMalloc((void **)&c->d_clov64, n * sizeof(double2)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_clovinv64, n * sizeof(double2)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_clovinv32, n * sizeof(float2)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_clovinv16, n * 2 * sizeof(bf16)) != cudaSuccess)
            return fail(DL_ENOMEM, "clover allocation failed");
    }
    zc gam[16][4][4];
    gamma_basis(gam);
    SigmaBlocks sig;
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
            zc sg[4][4];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    zc v = 0;
                    for (int k = 0; k < 4; ++k) v += gam[1 + mu][i][k] * gam[1 + nu][k][j] - gam[1 + nu][i][k] * gam[1 + mu][k][j];
                    sg[i][j] = zc(0, 0.5) * v;
                }
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    if (i / 2 != j / 2 && std::abs(sg[i][j]) > 1e-12)
                        return fail(DL_EINVAL, "clover: sigma_{mu nu} is not block-diagonal in this gamma basis");
            for (int b = 0; b < 2; ++b)
                for (int s1 = 0; s1 < 2; ++s1)
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const zc v = sg[2 * b + s1][2 * b + s2];
                        sig.s[plane][b][s1][s2] = make_double2(v.real(), v.imag());
                    }
        }
    const int grid = (int)std::max<long>(1, std::min<long>((c->V + 127) / 128, (long)c->num_sms * 4));
    CK(launch_clover_build(c->d_gauge64, c->g, sig, c->kappa * c->csw, c->d_clov64, c->d_clovinv64, c->d_clovinv32,
                           reinterpret_cast<__nv_bfloat162 *>(c->d_clovinv16), grid, c->stream));
    c->kernel_launches++;
    c->clover_stale = false;
    return DL_OK;
}

// out = mat in on the half field of parity p (width N; in place allowed); with
// acc_s != 0, out += acc_s (in - mat in).
static int clover_mul(dl_ctx *c, const double2 *mat, int p, int N, const double *in, double *out,
                      double acc_s = 0.0) {
    const long items = c->Vh * 2L * N;
    const int grid = (int)std::max<long>(1, std::min<long>((items + 255) / 256, (long)c->num_sms * 8));
    CK(launch_clover_mul(mat, p, (int)c->Vh, N, in, out, acc_s, grid, c->cur));
    c->kernel_launches++;
    return DL_OK;
}

extern "C" int dl_set_timing(dl_ctx *c, int enable) {
    if (!c) return fail(DL_EINVAL, "null context");
    if ((enable != 0) != c->timing) invalidate_graphs(c);
    c->timing = enable != 0;
    return DL_OK;
}

extern "C" int dl_get_timing(dl_ctx *c, dl_timing *out, int reset) {
    if (!c || !out) return fail(DL_EINVAL, "null argument");
    TRY(sync(c));
    *out = c->tim;
    out->kernel_launches = c->kernel_launches;
    if (reset) {
        memset(&c->tim, 0, sizeof(c->tim));
        c->kernel_launches = 0;
    }
    return DL_OK;
}

// ---------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------
// Whole-lattice batches of width 16 to 64 convert tile by tile (fields.cuh).
static bool tiled_conversion(const dl_ctx *c, int N, int cb0, int cb1, const int *tcol) {
    return !tcol && cb0 == 0 && cb1 == c->Vh && N >= 16 && N <= CONV_TILE && c->Vh % (CONV_TILE / N) == 0;
}

static int canon_to_eo(dl_ctx *c, const double *canon, double *eo, int n, int N, int g5, int cb0, int cb1,
                       const int *tcol = nullptr) {
    ConvArgs a;
    a.tcol = tcol;
    a.coords = c->d_coords;
    a.g = c->g;
    a.cb0 = cb0;
    a.cb1 = cb1;
    a.n = n;
    a.N = N;
    a.gamma5 = g5;
    if (tiled_conversion(c, N, cb0, cb1, tcol)) {
        const size_t smem = (size_t)2 * 12 * (CONV_TILE + CONV_TILE / N) * sizeof(double2);
        const int grid = (int)std::min<long>(c->Vh / (CONV_TILE / N), (long)c->num_sms * 8);
        canon_to_eo_tiled<<<grid, 256, smem, c->cur>>>(a, canon, eo);
        c->kernel_launches++;
        CK(cudaGetLastError());
        return DL_OK;
    }
    Launch l = make_launch(c, 2L * (cb1 - cb0) * N, 256, 0, 8);
    canon_to_eo_kernel<<<l.grid, l.block, 0, l.stream>>>(a, canon, eo);
    c->kernel_launches++;
    CK(cudaGetLastError());
    return DL_OK;
}

static int eo_to_canon(dl_ctx *c, const double *eo, double *canon, int n, int N, int g5, int cb0, int cb1,
                       const int *tcol = nullptr) {
    ConvArgs a;
    a.tcol = tcol;
    a.coords = c->d_coords;
    a.g = c->g;
    a.cb0 = cb0;
    a.cb1 = cb1;
    a.n = n;
    a.N = N;
    a.gamma5 = g5;
    if (tiled_conversion(c, N, cb0, cb1, tcol)) {
        const size_t smem = (size_t)2 * 12 * (CONV_TILE + CONV_TILE / N) * sizeof(double2);
        const int grid = (int)std::min<long>(c->Vh / (CONV_TILE / N), (long)c->num_sms * 8);
        eo_to_canon_tiled<<<grid, 256, smem, c->cur>>>(a, eo, canon);
        c->kernel_launches++;
        CK(cudaGetLastError());
        return DL_OK;
    }
    Launch l = make_launch(c, 2L * (cb1 - cb0) * n, 256, 0, 8);
    eo_to_canon_kernel<<<l.grid, l.block, 0, l.stream>>>(a, eo, canon);
    c->kernel_launches++;
    CK(cudaGetLastError());
    return DL_OK;
}

// ---------------------------------------------------------------------------
// solver
// ---------------------------------------------------------------------------
static void *lo_ptr(dl_ctx *c, int k) { return c->lo[k]; }
enum { LX = 0, LR = 1, LRH = 2, LP = 3, LV = 4, LS = 5, LT = 6, LTMP = 7 };

static int enqueue_iteration(dl_ctx *c, int prec, int N) {
    const double k2 = c->kappa * c->kappa;
    const int Vh = (int)c->Vh;
    double2 *part = c->d_partials;
    int nb = 0;
    const RhsState *act = c->d_rhs;  // right-hand sides that stopped skip the direct hops' loads and stores
    const bool cl = c->csw != 0.0;   // clover: Mhat = 1 - kappa^2 A_ee^-1 D_eo A_oo^-1 D_oe
    TRY(do_hop(c, prec, MODE_PLAIN, RED_NONE, lo_ptr(c, LTMP), lo_ptr(c, LP), nullptr, nullptr, nullptr, 1, N, 1.0, 0,
               Vh, nullptr, nullptr, 0, act, cl));
    TRY(do_hop(c, prec, MODE_XPAY, RED_R0DOT, lo_ptr(c, LV), lo_ptr(c, LTMP), lo_ptr(c, LP), nullptr,
               lo_ptr(c, LRH), 0, N, -k2, 0, Vh, part, &nb, 0, act, cl));
    scalar_alpha_kernel<<<N, kScalarThreads, 0, c->cur>>>(c->d_rhs, part, nb, N);
    VecLaunch v = vec_launch(c, prec, N, 0);
    CK(launch_axpy_s(v, c->d_rhs, lo_ptr(c, LR), lo_ptr(c, LV), lo_ptr(c, LS)));
    TRY(do_hop(c, prec, MODE_PLAIN, RED_NONE, lo_ptr(c, LTMP), lo_ptr(c, LS), nullptr, nullptr, nullptr, 1, N, 1.0, 0,
               Vh, nullptr, nullptr, 0, act, cl));
    TRY(do_hop(c, prec, MODE_XPAY, RED_BICG, lo_ptr(c, LT), lo_ptr(c, LTMP), lo_ptr(c, LS), nullptr, lo_ptr(c, LRH),
               0, N, -k2, 0, Vh, part, &nb, 0, act, cl));
    scalar_omega_kernel<<<N, kScalarThreads, 0, c->cur>>>(c->d_rhs, part, nb, N);
    CK(launch_update(v, c->d_rhs, lo_ptr(c, LX), lo_ptr(c, LR), lo_ptr(c, LP), lo_ptr(c, LS), lo_ptr(c, LT),
                     lo_ptr(c, LV)));
    c->kernel_launches += 4;
    CK(cudaGetLastError());
    return DL_OK;
}

// One CGNR iteration (blas.cuh): w = Mhat p; x, g5 r updated; u = Mhat g5 r; p = g5 u + beta p.
// Fields: LX x, LR g5 r, LP p, LV w, LRH u, LTMP the odd intermediate.
static int enqueue_iteration_cg(dl_ctx *c, int prec, int N) {
    const double k2 = c->kappa * c->kappa;
    const int Vh = (int)c->Vh;
    double2 *pa = c->d_partials, *pb = c->d_partials + c->partials_cap / 2;
    int nb = 0;
    TRY(do_hop(c, prec, MODE_PLAIN, RED_NONE, lo_ptr(c, LTMP), lo_ptr(c, LP), nullptr, nullptr, nullptr, 1, N, 1.0, 0,
               Vh, nullptr, nullptr));
    TRY(do_hop(c, prec, MODE_XPAY, RED_NORM, lo_ptr(c, LV), lo_ptr(c, LTMP), lo_ptr(c, LP), nullptr, nullptr, 0, N,
               -k2, 0, Vh, pa, &nb));
    cg_alpha_kernel<<<N, kScalarThreads, 0, c->cur>>>(c->d_rhs, pa, nb, N);
    VecLaunch v = vec_launch(c, prec, N, prec == P_F64 ? 16 : 8);
    CK(launch_cg_update(v, c->d_rhs, lo_ptr(c, LX), lo_ptr(c, LR), lo_ptr(c, LP), lo_ptr(c, LV), pb));
    const int nbv = v.l.grid;
    TRY(do_hop(c, prec, MODE_PLAIN, RED_NONE, lo_ptr(c, LTMP), lo_ptr(c, LR), nullptr, nullptr, nullptr, 1, N, 1.0, 0,
               Vh, nullptr, nullptr));
    TRY(do_hop(c, prec, MODE_XPAY, RED_NORM, lo_ptr(c, LRH), lo_ptr(c, LTMP), lo_ptr(c, LR), nullptr, nullptr, 0, N,
               -k2, 0, Vh, pa, &nb));
    cg_beta_kernel<<<N, kScalarThreads, 0, c->cur>>>(c->d_rhs, pb, nbv, pa, nb, N);
    CK(launch_cg_p(vec_launch(c, prec, N, 0), c->d_rhs, lo_ptr(c, LRH), lo_ptr(c, LP), 0));
    c->kernel_launches += 4;
    CK(cudaGetLastError());
    return DL_OK;
}

// Run `iters` inner iterations (graph or eager); returns the number of right-hand
// sides still active in *active.
static int run_chunk(dl_ctx *c, int prec, int N, int iters, bool use_graph, int *active, int method) {
    if (use_graph) {
        auto key = std::make_tuple(prec + 4 * method, N, iters, c->timing ? 1 : 0);
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            GraphEntry ge;
            const int64_t k0 = c->kernel_launches;
            std::vector<TimedPair> saved;
            saved.swap(c->pending);
            c->cur = c->cap_stream;
            c->capturing = true;
            cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
            int rc = DL_OK;
            if (e == cudaSuccess) {
                for (int k = 0; k < iters && rc == DL_OK; ++k)
                    rc = method == DL_METHOD_CGNR ? enqueue_iteration_cg(c, prec, N) : enqueue_iteration(c, prec, N);
                if (rc == DL_OK) {
                    count_active_kernel<<<1, 1, 0, c->cap_stream>>>(c->d_rhs, N, c->d_count);
                    c->kernel_launches++;
                }
                cudaGraph_t graph = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
                if (rc == DL_OK && e2 == cudaSuccess) {
                    e2 = cudaGraphInstantiate(&ge.exec, graph, 0);
                    if (e2 != cudaSuccess) rc = fail(DL_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
                } else if (rc == DL_OK) {
                    rc = fail(DL_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e2));
                }
                if (graph) cudaGraphDestroy(graph);
            } else {
                rc = fail(DL_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
            }
            c->capturing = false;
            c->cur = c->stream;
            ge.timed.swap(c->pending);
            c->pending.swap(saved);
            ge.n_kernels = (int)(c->kernel_launches - k0);
            c->kernel_launches = k0;
            if (rc != DL_OK) {
                for (auto &tp : ge.timed) {
                    c->event_pool.push_back(tp.a);
                    c->event_pool.push_back(tp.b);
                }
                return rc;
            }
            it = c->graphs.emplace(key, std::move(ge)).first;
        }
        CK(cudaGraphLaunch(it->second.exec, c->stream));
        c->kernel_launches += it->second.n_kernels;
        TRY(sync(c));
        harvest(c, it->second.timed, false);
    } else {
        c->cur = c->stream;
        for (int k = 0; k < iters; ++k)
            TRY(method == DL_METHOD_CGNR ? enqueue_iteration_cg(c, prec, N) : enqueue_iteration(c, prec, N));
        count_active_kernel<<<1, 1, 0, c->stream>>>(c->d_rhs, N, c->d_count);
        c->kernel_launches++;
        CK(cudaGetLastError());
        TRY(sync(c));
    }
    *active = *(volatile int *)c->h_count;
    return DL_OK;
}

// Smallest tolerance for which mixed-precision solves form their residuals in
// float-float arithmetic: its rounding, about 1e-14 of |x|, stays three orders
// of magnitude below it.
constexpr double kFFMinTol = 1e-11;

struct SolveCfg {
    int method;    // DL_METHOD_BICGSTAB or DL_METHOD_CGNR
    bool outer_dff;   // defect-correction hops in float-float instead of FP64
    bool restart;  // restart BiCGStab every defect-correction cycle (default) instead of continuing it
    double tol;
    int prec;
    int max_iter;
    int fixed_iters;
    double delta;
    int max_outer;
    int batch;
    bool use_graph;
    int chunk;
};

static int read_params(const dl_solve_params *p, SolveCfg *s) {
    dl_solve_params d;
    memset(&d, 0, sizeof(d));
    d.tol = 1e-10;
    d.precision = DL_PREC_F32;
    d.max_iter = 20000;
    d.use_graph = 1;
    if (!p) p = &d;
    if (!(p->tol > 0.0) || !std::isfinite(p->tol)) return fail(DL_EINVAL, "tol must be positive");
    if (p->precision < 0 || p->precision > 2) return fail(DL_EINVAL, "unknown precision");
    if (p->max_iter < 0 || p->fixed_iters < 0) return fail(DL_EINVAL, "negative iteration count");
    if (p->method != DL_METHOD_BICGSTAB && p->method != DL_METHOD_CGNR) return fail(DL_EINVAL, "unknown method");
    s->method = p->method;
    s->tol = p->tol;
    s->prec = p->precision;
    s->max_iter = p->max_iter > 0 ? p->max_iter : 20000;
    s->fixed_iters = p->fixed_iters;
    s->delta = p->delta > 0 ? p->delta : (p->precision == DL_PREC_BF16 ? 1e-3 : (p->precision == DL_PREC_F32 ? 3e-6 : 1e-3 * p->tol));
    if (p->precision == DL_PREC_F64 && !(p->delta > 0)) s->delta = std::max(1e-14, 0.5 * p->tol);
    s->max_outer = p->max_outer > 0 ? p->max_outer : 60;
    int b = p->batch > 0 ? p->batch : 16;
    if (b > 64) return fail(DL_EINVAL, "batch must be <= 64");
    s->batch = pow2_at_least(b);
    s->use_graph = p->use_graph != 0;
    // Poll convergence every 2 iterations: on 16^3 x 32 with 32 right-hand sides this
    // ran 4% faster than every 8 (fewer iterations past convergence) and no slower
    // than every iteration.
    s->chunk = p->chunk > 0 ? p->chunk : 2;
    {
        // Continuing p and rhat across cycles (a reliable update) measured slower than a
        // restart on the 16^3 x 32 workload for both inner precisions; kept as an option.
        const char *e = getenv("DLOOPS_CONTINUE_CYCLES");
        s->restart = !(e && e[0] == '1');
        // Float-float defect-correction hops (the default for mixed precision);
        // DLOOPS_OUTER_DFF=0 selects FP64 ones.
        const char *f = getenv("DLOOPS_OUTER_DFF");
        s->outer_dff = !(f && f[0] == '0');
    }
    return DL_OK;
}

// State check before a solve; brings the clover blocks up to date.
static int ready(dl_ctx *c) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (c->poisoned) return fail(DL_ECUDA, "context unusable: a staged hop left bulk copies pending");
    if (!c->have_gauge) return fail(DL_ESTATE, "load_gauge has not been called");
    if (!c->have_kappa) return fail(DL_ESTATE, "set_kappa has not been called");
    return ensure_clover(c);
}

// FP64 <-> float-float copy of n_complex values (in place when dst == src).
static int ff_cast(dl_ctx *c, const double *src, double *dst, size_t n_complex, int to_ff) {
    const long grid = std::max<long>(1, std::min<long>(((long)n_complex + 255) / 256, (long)c->num_sms * 8));
    CK(launch_ff_cast(src, dst, n_complex, to_ff, (int)grid, c->cur));
    c->kernel_launches++;
    return DL_OK;
}

// The reconstruction x_o = b_o + kappa D_oe x_e and the residual
// r = b_e - x_e + kappa D_eo x_o into c->r64 with |r|^2 partials in pa.  The
// odd rows of b - M x vanish by construction of x_o (up to rounding) and the
// even rows equal bhat - Mhat x_e, so r is both the Schur residual that drives
// the next cycle and the full-lattice residual; the final solution needs no
// further hop.  op = P_DFF: b_o is float-float, x_o is left float-float and x_e
// is first copied to float-float in c->bh64.
// Clover (op = P_F64): x_o = t + kappa A_oo^-1 D_oe x_e with t = A_oo^-1 b_o held in
// c->t64, and r = b_e - A_ee x_e + kappa D_eo x_o with A_ee x_e formed in c->bh64.
static int outer_residual(dl_ctx *c, int op, int N, const double *be, const double *bo, const double *xe,
                          double *xo, double2 *pa, int *nb) {
    const double k = c->kappa;
    const int Vh = (int)c->Vh;
    if (c->csw != 0.0) {
        TRY(do_hop(c, P_F64, MODE_XPAY, RED_NONE, xo, xe, c->t64, nullptr, nullptr, 1, N, k, 0, Vh, nullptr, nullptr,
                   0, nullptr, true));
        TRY(clover_mul(c, c->d_clov64, 0, N, xe, c->bh64));
        return do_hop(c, P_F64, MODE_RESID, RED_NORM, c->r64, xo, c->bh64, be, nullptr, 0, N, -k, 0, Vh, pa, nb);
    }
    if (op == P_DFF) {
        TRY(ff_cast(c, xe, c->bh64, half_elems(c, N), 1));
        TRY(do_hop(c, op, MODE_XPAY, RED_NONE, xo, c->bh64, bo, nullptr, nullptr, 1, N, k, 0, Vh, nullptr, nullptr,
                   FF_Y | FF_OUT));
        return do_hop(c, op, MODE_RESID, RED_NORM, c->r64, xo, c->bh64, be, nullptr, 0, N, -k, 0, Vh, pa, nb, FF_Y);
    }
    TRY(do_hop(c, op, MODE_XPAY, RED_NONE, xo, xe, bo, nullptr, nullptr, 1, N, k, 0, Vh, nullptr, nullptr));
    return do_hop(c, op, MODE_RESID, RED_NORM, c->r64, xo, xe, be, nullptr, 0, N, -k, 0, Vh, pa, nb);
}

// Solve the batch held in c->b64 (n right-hand sides, layout width N); the
// solution is left in c->x64.  host_os receives the N outer states.
static int solve_batch(dl_ctx *c, int n, int N, const SolveCfg &P, std::vector<OuterState> &host_os) {
    const double k = c->kappa, k2 = k * k;
    // Defect-correction hops (bhat, residuals, reconstruction) in float-float
    // arithmetic for mixed-precision solves whose tolerance lies well above its
    // rounding (~1e-14 relative), else in FP64.  In float-float, b_o and x_o are
    // held as float-float fields until the batch ends and x_e is copied to that
    // format (into the bhat buffer, free once r = bhat) before each residual.
    const bool clov = c->csw != 0.0;
    if (clov && P.method == DL_METHOD_CGNR)  // A_ee^-1 Mhat is not gamma_5-hermitian: CGNR's gamma_5 trick fails
        return fail(DL_EINVAL, "the clover operator is solved with BiCGStab only");
    const int op = (!clov && P.prec != P_F64 && P.outer_dff && P.tol >= kFFMinTol) ? P_DFF : P_F64;
    const bool ffo = op == P_DFF;
    const int Vh = (int)c->Vh;
    const size_t half = half_elems(c, N) * 2;  // doubles
    double *be = c->b64, *bo = c->b64 + half, *xe = c->x64, *xo = c->x64 + half;
    c->cur = c->stream;
    const size_t pc = c->partials_cap / 2;
    double2 *pa = c->d_partials, *pb = c->d_partials + pc;
    int nb = 0, nb2 = 0;
    // |b|^2 over both halves.  For the float-float outer loop each right-hand
    // side is first brought to a norm in [1, 2) by an exact power of two
    // (undone on x at the end; the relative residuals do not change), so that
    // sources of any magnitude stay inside the float exponent range.
    {
        VecLaunch v = vec_launch(c, P_F64, N, 16);
        for (int pass = 0; pass < (ffo ? 2 : 1); ++pass) {
            if (pass == 1) {
                pow2_pick_kernel<<<1, 64, 0, c->stream>>>(c->d_outer, N);
                const long rows = 2L * Vh * 12;
                const long grid = std::min<long>((rows * N + 255) / 256, (long)c->num_sms * 8);  // stride: a multiple of N
                pow2_scale_kernel<<<(int)grid, 256, 0, c->stream>>>(c->b64, (size_t)rows, N, c->d_outer, +1);
                c->kernel_launches += 2;
            }
            CK(launch_norm2(v, be, pa));
            nb = v.l.grid;
            CK(launch_norm2(v, bo, pb));
            nb2 = v.l.grid;
            full_norm_kernel<<<N, kScalarThreads, 0, c->stream>>>(c->d_outer, pa, nb, pb, nb2, N, 0);
            c->kernel_launches += 3;
        }
    }
    // bhat = b_e + kappa D_eo b_o, |bhat|^2 (clover: b_o replaced by t = A_oo^-1 b_o, kept in c->t64)
    if (ffo) TRY(ff_cast(c, bo, bo, half / 2, 1));
    if (clov) TRY(clover_mul(c, c->d_clovinv64, 1, N, bo, c->t64));
    TRY(do_hop(c, op, MODE_XPAY, RED_NORM, c->bh64, clov ? c->t64 : bo, be, nullptr, nullptr, 0, N, k, 0, Vh, pa, &nb));
    outer_update_kernel<<<N, kScalarThreads, 0, c->stream>>>(c->d_outer, c->d_rhs, pa, nb, N, 0, P.tol, P.max_outer, P.max_iter);
    c->kernel_launches++;
    CK(cudaMemcpyAsync(c->r64, c->bh64, half * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(xe, 0, half * sizeof(double), c->stream));
    bool residual_current = false;  // c->r64 and x_o belong to the current x_e
    const int prec = inner_prec(c, P.prec, N);
    for (int cycle = 0; cycle < P.max_outer; ++cycle) {
        outer_count_kernel<<<1, 1, 0, c->stream>>>(c->d_outer, N, c->d_count);
        c->kernel_launches++;
        TRY(sync(c));
        if (*(volatile int *)c->h_count == 0) break;
        const int target = P.fixed_iters > 0 ? P.fixed_iters : P.max_iter;
        if (P.method == DL_METHOD_CGNR) {
            // g5 r_l and x_l = 0; u = Mhat g5 r_l (|u|^2 = |Mhat^dag r_l|^2); p = g5 u
            VecLaunch v = vec_launch(c, prec, N, prec == P_F64 ? 16 : 8);
            CK(launch_cg_init(v, c->d_outer, c->r64, lo_ptr(c, LX), lo_ptr(c, LR), pb));
            TRY(do_hop(c, prec, MODE_PLAIN, RED_NONE, lo_ptr(c, LTMP), lo_ptr(c, LR), nullptr, nullptr, nullptr, 1, N,
                       1.0, 0, Vh, nullptr, nullptr));
            TRY(do_hop(c, prec, MODE_XPAY, RED_NORM, lo_ptr(c, LRH), lo_ptr(c, LTMP), lo_ptr(c, LR), nullptr, nullptr,
                       0, N, -k2, 0, Vh, pa, &nb));
            cg_start_kernel<<<N, kScalarThreads, 0, c->stream>>>(c->d_rhs, c->d_outer, pb, v.l.grid, pa, nb, N, P.delta, target,
                                                     P.max_iter, P.fixed_iters > 0 ? 1 : 0);
            CK(launch_cg_p(vec_launch(c, prec, N, 0), c->d_rhs, lo_ptr(c, LRH), lo_ptr(c, LP), 1));
            c->kernel_launches += 3;
        } else {
            // clover: the inner system is A_ee^-1 Mhat, its source A_ee^-1 r (in c->bh64)
            if (clov) TRY(clover_mul(c, c->d_clovinv64, 0, N, c->r64, c->bh64));
            VecLaunch v = vec_launch(c, prec, N, 2 * (prec == P_F64 ? 16 : 8));
            CK(launch_inner_init(v, c->d_outer, c->d_rhs, clov ? c->bh64 : c->r64, lo_ptr(c, LX), lo_ptr(c, LR),
                                 lo_ptr(c, LRH), lo_ptr(c, LP), pa, (cycle == 0 || P.restart) ? 1 : 0));
            inner_start_kernel<<<N, kScalarThreads, 0, c->stream>>>(c->d_rhs, c->d_outer, pa, v.l.grid, N, P.delta, target,
                                                        P.max_iter, P.fixed_iters > 0 ? 1 : 0);
            c->kernel_launches += 2;
        }
        int done = 0;
        while (done < target) {
            const int kk = std::min(P.chunk, target - done);
            int active = 0;
            TRY(run_chunk(c, prec, N, kk, P.use_graph, &active, P.method));
            done += kk;
            if (active == 0) break;
        }
        c->cur = c->stream;
        CK(launch_accumulate(vec_launch(c, prec, N, 0), c->d_outer, lo_ptr(c, LX), xe));
        c->kernel_launches++;
        // The true residual, every cycle, through the reconstruction of x_o.
        TRY(outer_residual(c, op, N, be, bo, xe, xo, pa, &nb));
        residual_current = true;
        outer_update_kernel<<<N, kScalarThreads, 0, c->stream>>>(c->d_outer, c->d_rhs, pa, nb, N,
                                                                 P.fixed_iters > 0 ? 2 : 1, P.tol, P.max_outer,
                                                                 P.max_iter);
        c->kernel_launches++;
        if (P.fixed_iters > 0) break;
    }
    if (!residual_current) {  // no cycle ran (every right-hand side was zero): x = (0, b_o)
        TRY(outer_residual(c, op, N, be, bo, xe, xo, pa, &nb));
        full_norm_kernel<<<N, kScalarThreads, 0, c->stream>>>(c->d_outer, pa, nb, pb, 0, N, 1);
        c->kernel_launches++;
    }
    if (ffo) {  // back to FP64: the solution's odd half and the source; undo the scale on x
        TRY(ff_cast(c, xo, xo, half / 2, 0));
        TRY(ff_cast(c, bo, bo, half / 2, 0));
        const long rows = 2L * Vh * 12;
        const long grid = std::min<long>((rows * N + 255) / 256, (long)c->num_sms * 8);
        pow2_scale_kernel<<<(int)grid, 256, 0, c->stream>>>(c->x64, (size_t)rows, N, c->d_outer, -1);
        c->kernel_launches++;
    }
    CK(cudaGetLastError());
    host_os.resize(N);
    CK(cudaMemcpyAsync(host_os.data(), c->d_outer, N * sizeof(OuterState), cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    (void)n;
    return DL_OK;
}

static int status_of(const OuterState &o, double tol, bool fixed) {
    if (o.status == ST_NAN || !std::isfinite(o.full_r2)) return DL_NAN;
    if (fixed) return DL_OK;
    if (o.full_b2 == 0.0) return DL_OK;
    return std::sqrt(o.full_r2 / o.full_b2) <= tol ? DL_OK : DL_NOT_CONVERGED;
}

static int solve_impl(dl_ctx *c, const void *b, void *x, int n_rhs, const dl_solve_params *params,
                      dl_solve_stats *stats, int g5) {
    TRY(ready(c));
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    if (n_rhs == 0) return DL_OK;
    if (!b || !x) return fail(DL_EINVAL, "null field pointer");
    if (b == x) return fail(DL_EINVAL, "dev_x may not alias dev_b");
    SolveCfg P;
    TRY(read_params(params, &P));
    const int N = std::min(P.batch, pow2_at_least(n_rhs));
    TRY(ensure_ws(c, N));
    TRY(ensure_partials(c, (size_t)2 * c->num_sms * 16 * N * 16));
    TRY(maybe_tune(c, P.prec, N));
    TRY(maybe_tune(c, P_F64, N));
    const size_t field = (size_t)c->V * 24;  // doubles per canonical field
    int worst = DL_OK;
    std::vector<OuterState> os;
    for (int j0 = 0; j0 < n_rhs; j0 += N) {
        const int n = std::min(N, n_rhs - j0);
        c->cur = c->stream;
        TRY(canon_to_eo(c, (const double *)b + (size_t)j0 * field, c->b64, n, N, g5, 0, (int)c->Vh));
        TRY(solve_batch(c, n, N, P, os));
        TRY(eo_to_canon(c, c->x64, (double *)x + (size_t)j0 * field, n, N, g5, 0, (int)c->Vh));
        for (int j = 0; j < n; ++j) {
            const int s = status_of(os[j], P.tol, P.fixed_iters > 0);
            if (stats) {
                stats[j0 + j].status = s;
                stats[j0 + j].iters = os[j].iters;
                stats[j0 + j].outer = os[j].outer;
                stats[j0 + j].true_residual = os[j].full_b2 > 0 ? std::sqrt(os[j].full_r2 / os[j].full_b2) : 0.0;
            }
            if (s != DL_OK && worst == DL_OK) worst = s;
        }
    }
    TRY(sync(c));
    if (worst != DL_OK) fail(worst, "some right-hand sides did not converge");
    return worst;
}

extern "C" int dl_solve(dl_ctx *c, const void *b, void *x, int n, const dl_solve_params *p, dl_solve_stats *st) {
    return solve_impl(c, b, x, n, p, st, 0);
}

extern "C" int dl_solve_adjoint(dl_ctx *c, const void *b, void *x, int n, const dl_solve_params *p,
                                dl_solve_stats *st) {
    return solve_impl(c, b, x, n, p, st, 1);
}

// ---------------------------------------------------------------------------
// sources
// ---------------------------------------------------------------------------
extern "C" int dl_make_sources(dl_ctx *c, uint64_t seed, int64_t noise_first, int n_noise, unsigned dil, int t0,
                               int prec, void *out, int64_t *n_rhs) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (prec < DL_PREC_F64 || prec > DL_PREC_BF16) return fail(DL_EINVAL, "unknown output precision");
    if (n_noise < 0 || noise_first < 0) return fail(DL_EINVAL, "negative noise range");
    if (dil & ~31u) return fail(DL_EINVAL, "unknown dilution bits");
    if ((dil & DL_DIL_TIME) && t0 >= c->dims[3]) return fail(DL_EINVAL, "t0 outside the lattice");
    SourceArgs a;
    a.coords = c->d_coords;
    a.g = c->g;
    a.seed = seed;
    a.noise_first = noise_first;
    a.n_noise = n_noise;
    a.dil_spin = (dil & DL_DIL_SPIN) ? 4 : 1;
    a.dil_colour = (dil & DL_DIL_COLOUR) ? 3 : 1;
    a.dil_eo = (dil & DL_DIL_EVENODD) ? 2 : 1;
    a.dil_cubic = (dil & DL_DIL_CUBIC) ? 8 : 1;
    a.dil_time = (dil & DL_DIL_TIME) ? 1 : 0;
    a.t0 = t0;
    const int K = a.dil_spin * a.dil_colour * a.dil_eo * a.dil_cubic;
    a.k_first = 0;
    a.k_count = K;
    if (n_rhs) *n_rhs = (int64_t)n_noise * K;
    if (n_noise == 0) return DL_OK;
    if (!out) return fail(DL_EINVAL, "null output");
    c->cur = c->stream;
    Launch l = make_launch(c, (long)n_noise * K * c->V, 256, 0, 16);
    if (prec == DL_PREC_F64) z2_source_kernel<double2><<<l.grid, l.block, 0, c->stream>>>(a, (double2 *)out);
    else if (prec == DL_PREC_F32) z2_source_kernel<float2><<<l.grid, l.block, 0, c->stream>>>(a, (float2 *)out);
    else z2_source_kernel<__nv_bfloat162><<<l.grid, l.block, 0, c->stream>>>(a, (__nv_bfloat162 *)out);
    c->kernel_launches++;
    CK(cudaGetLastError());
    return DL_OK;
}

extern "C" int dl_make_point_sources(dl_ctx *c, int64_t first, int n, int prec, void *out) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (prec < DL_PREC_F64 || prec > DL_PREC_BF16) return fail(DL_EINVAL, "unknown output precision");
    if (n < 0 || first < 0 || first + n > 12 * c->V) return fail(DL_EINVAL, "point-source range outside 0..12V");
    if (n == 0) return DL_OK;
    if (!out) return fail(DL_EINVAL, "null output");
    c->cur = c->stream;
    Launch l = make_launch(c, (long)n * c->V * 12, 256, 0, 16);
    if (prec == DL_PREC_F64) point_source_kernel<double2><<<l.grid, l.block, 0, c->stream>>>(first, n, c->V, (double2 *)out);
    else if (prec == DL_PREC_F32) point_source_kernel<float2><<<l.grid, l.block, 0, c->stream>>>(first, n, c->V, (float2 *)out);
    else point_source_kernel<__nv_bfloat162><<<l.grid, l.block, 0, c->stream>>>(first, n, c->V, (__nv_bfloat162 *)out);
    c->kernel_launches++;
    CK(cudaGetLastError());
    return DL_OK;
}

// ---------------------------------------------------------------------------
// operators on canonical fields
// ---------------------------------------------------------------------------
enum { OP_D = 0, OP_M = 1, OP_DMDK = 2 };  // D, M, -dM/dkappa

static int apply_hop_impl(dl_ctx *c, const void *in, void *out, int n_rhs, int what) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (!c->have_gauge) return fail(DL_ESTATE, "load_gauge has not been called");
    const bool with_m = what == OP_M;
    if (what != OP_D && !c->have_kappa) return fail(DL_ESTATE, "set_kappa has not been called");
    // -dM/dkappa = D + c_sw sum sigma F = D + (1 - A) / kappa
    const bool dmdk_clov = what == OP_DMDK && c->csw != 0.0;
    if (dmdk_clov && c->kappa == 0.0) return fail(DL_EINVAL, "dM/dkappa with clover needs kappa != 0");
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    if (n_rhs == 0) return DL_OK;
    if (!in || !out || in == out) return fail(DL_EINVAL, "bad field pointers");
    const int N = std::min(64, pow2_at_least(n_rhs));
    TRY(ensure_ws(c, N));
    TRY(ensure_partials(c, (size_t)2 * c->num_sms * 16 * N * 16));
    const size_t field = (size_t)c->V * 24, half = half_elems(c, N) * 2;
    const int Vh = (int)c->Vh;
    const int mode = with_m ? MODE_XPAY : MODE_PLAIN;
    const double coef = with_m ? -c->kappa : 1.0;
    const char *ar = getenv("DLOOPS_HOP_ARITH");
    const bool clov = with_m && c->csw != 0.0;  // M = A - kappa D: y = A in (c->s64a), FP64
    const int op = (!clov && !dmdk_clov && ar && std::string(ar) == "dff") ? P_DFF : P_F64;
    if (clov || dmdk_clov) TRY(ensure_clover(c));
    for (int j0 = 0; j0 < n_rhs; j0 += N) {
        const int n = std::min(N, n_rhs - j0);
        c->cur = c->stream;
        TRY(canon_to_eo(c, (const double *)in + j0 * field, c->b64, n, N, 0, 0, Vh));
        if (clov) {
            TRY(clover_mul(c, c->d_clov64, 0, N, c->b64, c->s64a));
            TRY(clover_mul(c, c->d_clov64, 1, N, c->b64 + half, c->s64a + half));
            TRY(do_hop(c, op, mode, RED_NONE, c->x64, c->b64 + half, c->s64a, nullptr, nullptr, 0, N, coef, 0, Vh,
                       nullptr, nullptr));
            TRY(do_hop(c, op, mode, RED_NONE, c->x64 + half, c->b64, c->s64a + half, nullptr, nullptr, 1, N, coef, 0,
                       Vh, nullptr, nullptr));
            TRY(eo_to_canon(c, c->x64, (double *)out + j0 * field, n, N, 0, 0, Vh));
            continue;
        }
        if (dmdk_clov) {  // D in, then += (in - A in) / kappa on each half
            TRY(do_hop(c, op, MODE_PLAIN, RED_NONE, c->x64, c->b64 + half, nullptr, nullptr, nullptr, 0, N, 1.0, 0, Vh,
                       nullptr, nullptr));
            TRY(do_hop(c, op, MODE_PLAIN, RED_NONE, c->x64 + half, c->b64, nullptr, nullptr, nullptr, 1, N, 1.0, 0, Vh,
                       nullptr, nullptr));
            TRY(clover_mul(c, c->d_clov64, 0, N, c->b64, c->x64, 1.0 / c->kappa));
            TRY(clover_mul(c, c->d_clov64, 1, N, c->b64 + half, c->x64 + half, 1.0 / c->kappa));
            TRY(eo_to_canon(c, c->x64, (double *)out + j0 * field, n, N, 0, 0, Vh));
            continue;
        }
        // float-float: each half is converted in place before it is gathered
        if (op == P_DFF) TRY(ff_cast(c, c->b64 + half, c->b64 + half, half / 2, 1));
        TRY(do_hop(c, op, mode, RED_NONE, c->x64, c->b64 + half, c->b64, nullptr, nullptr, 0, N, coef, 0, Vh,
                   nullptr, nullptr));
        if (op == P_DFF) TRY(ff_cast(c, c->b64, c->b64, half / 2, 1));
        TRY(do_hop(c, op, mode, RED_NONE, c->x64 + half, c->b64, c->b64 + half, nullptr, nullptr, 1, N, coef, 0,
                   Vh, nullptr, nullptr, op == P_DFF && with_m ? FF_Y : 0));
        TRY(eo_to_canon(c, c->x64, (double *)out + j0 * field, n, N, 0, 0, Vh));
    }
    return DL_OK;
}

extern "C" int dl_apply_hop(dl_ctx *c, const void *in, void *out, int n) { return apply_hop_impl(c, in, out, n, OP_D); }

// out = D in with the inner solver's low-precision hop: both halves of `in`
// rounded to the storage type, the FP32/BF16 link copies, FP32 arithmetic, the
// kernel and launch shape the context uses for that (precision, width); the
// result widened back to FP64.
extern "C" int dl_apply_hop_prec(dl_ctx *c, int precision, const void *in, void *out, int n_rhs) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (precision == DL_PREC_F64) return apply_hop_impl(c, in, out, n_rhs, OP_D);
    if (precision != DL_PREC_F32 && precision != DL_PREC_BF16) return fail(DL_EINVAL, "unknown precision");
    if (!c->have_gauge) return fail(DL_ESTATE, "load_gauge has not been called");
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    if (n_rhs == 0) return DL_OK;
    if (!in || !out || in == out) return fail(DL_EINVAL, "bad field pointers");
    const int N = std::min(64, pow2_at_least(n_rhs));
    TRY(ensure_ws(c, N));
    TRY(ensure_partials(c, (size_t)2 * c->num_sms * 16 * N * 16));
    const size_t field = (size_t)c->V * 24, half = half_elems(c, N) * 2;
    const int Vh = (int)c->Vh;
    const size_t nc = half / 2;  // complex values per half field
    const int grid = (int)std::min<long>(((long)nc + 255) / 256, (long)c->num_sms * 8);
    const int ip = inner_prec(c, precision, N);  // storage layout the solver's inner fields use at this width
    for (int j0 = 0; j0 < n_rhs; j0 += N) {
        const int n = std::min(N, n_rhs - j0);
        c->cur = c->stream;
        TRY(canon_to_eo(c, (const double *)in + j0 * field, c->b64, n, N, 0, 0, Vh));
        CK(launch_cast(ip, c->b64, lo_ptr(c, 0), nc, 1, grid, c->stream));
        CK(launch_cast(ip, c->b64 + half, lo_ptr(c, 1), nc, 1, grid, c->stream));
        TRY(do_hop(c, ip, MODE_PLAIN, RED_NONE, lo_ptr(c, 2), lo_ptr(c, 1), nullptr, nullptr, nullptr, 0, N,
                   1.0, 0, Vh, nullptr, nullptr));
        TRY(do_hop(c, ip, MODE_PLAIN, RED_NONE, lo_ptr(c, 3), lo_ptr(c, 0), nullptr, nullptr, nullptr, 1, N,
                   1.0, 0, Vh, nullptr, nullptr));
        CK(launch_cast(ip, c->x64, lo_ptr(c, 2), nc, 0, grid, c->stream));
        CK(launch_cast(ip, c->x64 + half, lo_ptr(c, 3), nc, 0, grid, c->stream));
        c->kernel_launches += 4;
        TRY(eo_to_canon(c, c->x64, (double *)out + j0 * field, n, N, 0, 0, Vh));
    }
    return DL_OK;
}
extern "C" int dl_apply_m(dl_ctx *c, const void *in, void *out, int n) { return apply_hop_impl(c, in, out, n, OP_M); }
extern "C" int dl_apply_dm_dkappa(dl_ctx *c, const void *in, void *out, int n) {
    return apply_hop_impl(c, in, out, n, OP_DMDK);
}

// out = A in or A^-1 in, site by site (the identity without clover).
extern "C" int dl_apply_clover(dl_ctx *c, const void *in, void *out, int n_rhs, int inverse) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (!c->have_gauge) return fail(DL_ESTATE, "load_gauge has not been called");
    if (!c->have_kappa) return fail(DL_ESTATE, "set_kappa has not been called");
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    if (n_rhs == 0) return DL_OK;
    if (!in || !out || in == out) return fail(DL_EINVAL, "bad field pointers");
    const size_t field = (size_t)c->V * 24;
    c->cur = c->stream;
    if (c->csw == 0.0) {
        CK(cudaMemcpyAsync(out, in, (size_t)n_rhs * field * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        return DL_OK;
    }
    TRY(ensure_clover(c));
    const int N = std::min(64, pow2_at_least(n_rhs));
    TRY(ensure_ws(c, N));
    const size_t half = half_elems(c, N) * 2;
    const int Vh = (int)c->Vh;
    const double2 *mat = inverse ? c->d_clovinv64 : c->d_clov64;
    for (int j0 = 0; j0 < n_rhs; j0 += N) {
        const int n = std::min(N, n_rhs - j0);
        TRY(canon_to_eo(c, (const double *)in + j0 * field, c->b64, n, N, 0, 0, Vh));
        TRY(clover_mul(c, mat, 0, N, c->b64, c->x64));
        TRY(clover_mul(c, mat, 1, N, c->b64 + half, c->x64 + half));
        TRY(eo_to_canon(c, c->x64, (double *)out + j0 * field, n, N, 0, 0, Vh));
    }
    return DL_OK;
}

// Smear the EO fields at *buf (full field, width N) over cb range; returns the
// buffer holding the result (ping-pong with `spare`).
// Smear *buf (and, if buf2 is set, *buf2 in the same launches) in place over the cb
// range; spare / spare2 are scratch fields of the same shape.  On return *buf
// (*buf2) points at whichever of the pair holds the result.
static int smear_eo(dl_ctx *c, double **buf, double *spare, int N, int n, const dl_smear &s, int cb0, int cb1,
                    const int *tcol = nullptr, double **buf2 = nullptr, double *spare2 = nullptr) {
    if (buf2 && c->smear_fp64) {  // the FP64 kernel smears one field per launch
        TRY(smear_eo(c, buf, spare, N, n, s, cb0, cb1, tcol));
        return smear_eo(c, buf2, spare2, N, n, s, cb0, cb1, tcol);
    }
    SmearArgs A;
    A.in2 = nullptr;
    A.out2 = nullptr;
    A.n = n;
    A.tcol = tcol;
    A.gauge = c->d_gauge64;
    A.coords = c->d_coords;
    A.g = c->g;
    A.cb0 = cb0;
    A.cb1 = cb1;
    A.N = N;
    A.a = 1.0 / (1.0 + 6.0 * s.alpha);
    A.c = s.alpha / (1.0 + 6.0 * s.alpha);
    double *src = *buf, *dst = spare;
    Launch l = make_launch(c, 2L * (cb1 - cb0) * n, 128, 0, 8);
    if (c->smear_fp64) {
        for (int it = 0; it < s.n_iter; ++it) {
            A.in = src;
            A.out = dst;
            smear_kernel<<<l.grid, l.block, 0, c->cur>>>(A);
            c->kernel_launches++;
            std::swap(src, dst);
        }
    } else {
        double *src2 = buf2 ? *buf2 : nullptr, *dst2 = spare2;
        const int nf = buf2 ? 2 : 1;
        Launch lc = make_launch(c, 2L * (cb1 - cb0) * 12 * n, 256, 0, 8);
        ff_convert_kernel<<<lc.grid, lc.block, 0, c->cur>>>(src, (int)c->Vh, cb0, cb1, N, n, 1, tcol, c->g.V3h);
        if (buf2)
            ff_convert_kernel<<<lc.grid, lc.block, 0, c->cur>>>(src2, (int)c->Vh, cb0, cb1, N, n, 1, tcol, c->g.V3h);
        // one thread per (site, colour row, column): three times the threads of
        // the whole-site kernel, each with a third of the registers
        Launch lr = make_launch(c, 2L * (cb1 - cb0) * 3 * n, 256, 0, 6);
        for (int it = 0; it < s.n_iter; ++it) {
            A.in = src;
            A.out = dst;
            A.in2 = src2;
            A.out2 = dst2;
            smear_ff_rows_kernel<<<dim3(lr.grid, nf), lr.block, 0, c->cur>>>(A, c->d_gauge_ff);
            std::swap(src, dst);
            std::swap(src2, dst2);
        }
        ff_convert_kernel<<<lc.grid, lc.block, 0, c->cur>>>(src, (int)c->Vh, cb0, cb1, N, n, 0, tcol, c->g.V3h);
        if (buf2)
            ff_convert_kernel<<<lc.grid, lc.block, 0, c->cur>>>(src2, (int)c->Vh, cb0, cb1, N, n, 0, tcol, c->g.V3h);
        c->kernel_launches += s.n_iter + 2 * nf;
        if (buf2) *buf2 = src2;
    }
    CK(cudaGetLastError());
    *buf = src;
    return DL_OK;
}

extern "C" int dl_apply_smear(dl_ctx *c, const void *in, void *out, int n_rhs, const dl_smear *s, int t_lo, int t_hi) {
    if (!c || !s) return fail(DL_EINVAL, "null argument");
    if (!c->have_gauge) return fail(DL_ESTATE, "load_gauge has not been called");
    if (s->n_iter < 0 || !std::isfinite(s->alpha)) return fail(DL_EINVAL, "bad smearing parameters");
    if (t_lo < 0 || t_hi > c->dims[3] || t_lo >= t_hi) return fail(DL_EINVAL, "bad timeslice range");
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    if (n_rhs == 0) return DL_OK;
    if (!in || !out || in == out) return fail(DL_EINVAL, "bad field pointers");
    const int N = std::min(64, pow2_at_least(n_rhs));
    TRY(ensure_ws(c, N));
    const size_t field = (size_t)c->V * 24;
    const int cb0 = t_lo * c->g.V3h, cb1 = t_hi * c->g.V3h;
    c->cur = c->stream;
    CK(cudaMemsetAsync(out, 0, (size_t)n_rhs * field * sizeof(double), c->stream));
    for (int j0 = 0; j0 < n_rhs; j0 += N) {
        const int n = std::min(N, n_rhs - j0);
        TRY(canon_to_eo(c, (const double *)in + j0 * field, c->b64, n, N, 0, cb0, cb1));
        double *res = c->b64;
        TRY(smear_eo(c, &res, c->s64a, N, n, *s, cb0, cb1));
        TRY(eo_to_canon(c, res, (double *)out + j0 * field, n, N, 0, cb0, cb1));
    }
    return DL_OK;
}

extern "C" int dl_apply_gamma_weights(dl_ctx *c, const void *in, void *out, int n_rhs, const double *host_w, int mode,
                                      int accumulate) {
    if (!c || !host_w) return fail(DL_EINVAL, "null argument");
    if (mode != 0 && mode != 1) return fail(DL_EINVAL, "mode must be 0 or 1");
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    if (n_rhs == 0) return DL_OK;
    if (!in || !out || in == out) return fail(DL_EINVAL, "bad field pointers");
    const int T = c->dims[3];
    const size_t nw = (size_t)n_rhs * 16 * T;      // weights
    const size_t need = nw + (size_t)n_rhs * T * 16;  // + spin matrices
    if (c->w_cap < need) {
        TRY(sync(c));
        if (c->d_w) cudaFree(c->d_w);
        c->d_w = nullptr;
        if (cudaMalloc((void **)&c->d_w, need * sizeof(double2)) != cudaSuccess) return fail(DL_ENOMEM, "weights");
        c->w_cap = need;
    }
    c->cur = c->stream;
    CK(cudaMemcpyAsync(c->d_w, host_w, nw * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    double2 *W = c->d_w + nw;
    gamma_weights_kernel<<<std::max(1, (int)((n_rhs * T * 16 + 255) / 256)), 256, 0, c->stream>>>(c->d_w, n_rhs, T, mode,
                                                                                                    c->d_gammas, W);
    Launch l = make_launch(c, (long)n_rhs * c->V * 3, 256, 0, 16);
    apply_spin_matrix_kernel<<<l.grid, l.block, 0, c->stream>>>((const double *)in, (double *)out, W, n_rhs, c->V,
                                                                 2 * c->g.V3h, T, accumulate);
    c->kernel_launches += 2;
    CK(cudaGetLastError());
    TRY(sync(c));  // host_w may be reused by the caller
    return DL_OK;
}

// ---------------------------------------------------------------------------
// loops
// ---------------------------------------------------------------------------
__global__ void sum_loops_kernel(const double2 *in, int n, int stride_j, double2 *out, int count) {
    // out[e] = sum_j in[j*stride_j + e], fixed order
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        double re = 0, im = 0;
        for (int j = 0; j < n; ++j) {
            const double2 v = in[(size_t)j * stride_j + e];
            re += v.x;
            im += v.y;
        }
        out[e] = make_double2(re, im);
    }
}

__global__ void zero_kernel(double2 *p, int count) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
        p[e] = make_double2(0.0, 0.0);
}

__global__ void add_kernel(double2 *acc, const double2 *v, int count) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        acc[e].x += v[e].x;
        acc[e].y += v[e].y;
    }
}

// spin matrices S[t][beta*4+alpha] -> L[G][t]
__global__ void spin_to_gamma_kernel(const double2 *S, int T, const double2 *gammas, double2 *out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 16 * T) return;
    const int G = idx / T, t = idx % T;
    double re = 0, im = 0;
    for (int al = 0; al < 4; ++al)
        for (int be = 0; be < 4; ++be) {
            const double2 g = gammas[(G * 4 + al) * 4 + be];
            const double2 s = S[(size_t)t * 16 + be * 4 + al];
            re += g.x * s.x - g.y * s.y;
            im += g.x * s.y + g.y * s.x;
        }
    out[idx] = make_double2(re, im);
}

// Contract EO fields eta (c->b64) and phi (c->x64), width N, n right-hand sides,
// timeslices [t_lo, t_hi) into dst[j][16][T] (other timeslices zero).
static int contract_eo(dl_ctx *c, const double *eta, const double *phi, int n, int N, int t_lo, int t_hi,
                       double2 *dst, const int *tcol = nullptr) {
    const int T = c->dims[3];
    if (tcol) {  // one timeslice per column
        t_lo = 0;
        t_hi = 1;
    }
    const int nt = t_hi - t_lo;
    const int R = (N > 32 && !tcol) ? 2 : 1;
    const int G = N / R;
    const int block = R == 2 ? 64 : 128;  // a multiple of G
    int nbx = std::max(1, std::min((int)((c->g.V3h * (long)G + block - 1) / block), std::max(1, 4 * c->num_sms / (2 * nt))));
    TRY(ensure_partials(c, (size_t)nt * 2 * nbx * N * 16));
    ContractArgs A;
    A.eta = eta;
    A.phi = phi;
    A.g = c->g;
    A.t_lo = t_lo;
    A.N = N;
    A.partials = c->d_partials;
    A.tcol = tcol;
    A.n = n;
    dim3 grid(nbx, nt, 2);
    const size_t smem = (size_t)(block / 32) * std::min(G, 32) * R * 16 * sizeof(double2);
    if (R == 1) contract_kernel<1><<<grid, block, smem, c->cur>>>(A);
    else contract_kernel<2><<<grid, block, smem, c->cur>>>(A);
    const int cnt = n * 16 * T;
    zero_kernel<<<std::max(1, (cnt + 255) / 256), 256, 0, c->cur>>>(dst, cnt);
    contract_final_kernel<<<dim3(nt, n), 32, 0, c->cur>>>(c->d_partials, nbx, N, t_lo, T, c->d_gammas, dst, tcol);
    c->kernel_launches += 3;
    CK(cudaGetLastError());
    return DL_OK;
}

// Momentum-projected contraction (momentum.cuh): site spin matrices, their
// Fourier sums against the phase table, Gamma traces into dst[j][q][16][T].
struct MomSpec {
    int n_mom;
    const double2 *phase;  // [n_mom][V3]
    double2 *site;         // [N][nt][V3][16]
    double2 *msum;         // [N][nt][n_mom][16]
    double2 *dst;          // [sink slot][N][n_mom][16][T]
};

static int contract_mom_eo(dl_ctx *c, const double *eta, const double *phi, int n, int N, int t_lo, int t_hi,
                           const MomSpec &m, double2 *dst, const int *tcol) {
    const int T = c->dims[3];
    const int V3 = c->dims[0] * c->dims[1] * c->dims[2];
    const int nt = tcol ? 1 : t_hi - t_lo;
    SiteSpinArgs A;
    A.eta = eta;
    A.phi = phi;
    A.coords = c->d_coords;
    A.g = c->g;
    A.N = N;
    A.n = n;
    A.t_lo = tcol ? 0 : t_lo;
    A.nt = nt;
    A.tcol = tcol;
    A.out = m.site;
    Launch l = make_launch(c, (long)nt * 2 * c->g.V3h * n, 128, 0, 8);
    site_spin_kernel<<<l.grid, l.block, 0, c->cur>>>(A);
    fourier_kernel<<<dim3(n * nt, (m.n_mom * 16 + 255) / 256), 256, 0, c->cur>>>(m.site, m.phase, V3, 16, m.n_mom,
                                                                                 m.msum);
    const int cnt = n * m.n_mom * 16 * T;
    zero_kernel<<<std::max(1, (cnt + 255) / 256), 256, 0, c->cur>>>(dst, cnt);
    const int tot = n * nt * m.n_mom * 16;
    mom_gamma_kernel<<<std::max(1, (tot + 255) / 256), 256, 0, c->cur>>>(m.msum, c->d_gammas, n, nt, m.n_mom, T,
                                                                         A.t_lo, tcol, dst);
    c->kernel_launches += 4;
    CK(cudaGetLastError());
    return DL_OK;
}

// Loops of the EO pair (eta in *eta_buf, phi in *phi_buf) for the requested
// sinks into c->d_loops[j][sink][16][T] (or, with a MomSpec, into
// mom->dst[sink][j][q][16][T]); smearing overwrites the buffers.
static int trace_eo(dl_ctx *c, double *eta_buf, double *phi_buf, int n, int N, int sink, const dl_smear *sm, int t_lo,
                    int t_hi, int n_sinks, const int *tcol = nullptr, const MomSpec *mom = nullptr) {
    const int T = c->dims[3];
    const int cb0 = t_lo * c->g.V3h, cb1 = t_hi * c->g.V3h;
    const int per = 16 * T;
    int slot = 0;
    // per-sink contraction into a scratch [n][16][T] then interleave into d_loops
    for (int s = 0; s < 2; ++s) {
        const int flag = s == 0 ? DL_SINK_LOCAL : DL_SINK_SMEARED;
        if (!(sink & flag)) continue;
        double *e = eta_buf, *f = phi_buf;
        if (flag == DL_SINK_SMEARED) {
            const int s0 = tcol ? 0 : cb0, s1 = tcol ? c->g.V3h : cb1;
            TRY(smear_eo(c, &e, e == c->b64 ? c->s64a : c->b64, N, n, *sm, s0, s1, tcol, &f,
                         f == c->x64 ? c->s64b : c->x64));
        }
        // contract into the slot `slot` region of d_loops viewed as [sink][n][16][T]
        if (mom)
            TRY(contract_mom_eo(c, e, f, n, N, t_lo, t_hi, *mom, mom->dst + (size_t)slot * N * mom->n_mom * per, tcol));
        else
            TRY(contract_eo(c, e, f, n, N, t_lo, t_hi, c->d_loops + (size_t)slot * N * per, tcol));
        ++slot;
    }
    (void)n_sinks;
    return DL_OK;
}

// out[g][s][e] = sum over the right-hand sides of group g (consecutive, fixed order)
__global__ void group_sum_kernel(const double2 *loops /* [sink][N][per] */, int n, int N, int group, int n_sinks,
                                 int per, double2 *out /* [n/group][sink][per] */) {
    const int count = (n / group) * n_sinks * per;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += gridDim.x * blockDim.x) {
        const int e = idx % per;
        const int s = (idx / per) % n_sinks;
        const int g = idx / (per * n_sinks);
        double re = 0.0, im = 0.0;
        for (int k = 0; k < group; ++k) {
            const double2 v = loops[((size_t)s * N + g * group + k) * per + e];
            re += v.x;
            im += v.y;
        }
        out[idx] = make_double2(re, im);
    }
}

// out[r] = sum_t in[r][t] over T timeslices, in order (rows of [..][T])
__global__ void sum_t_kernel(const double2 *in, int rows, int T, double2 *out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int t = 0; t < T; ++t) {
            const double2 v = in[(size_t)r * T + t];
            re += v.x;
            im += v.y;
        }
        out[r] = make_double2(re, im);
    }
}

extern "C" int dl_trace_loops(dl_ctx *c, const void *eta, const void *phi, int n_rhs, int sink, const dl_smear *sm,
                              int t_lo, int t_hi, const int *t_of_rhs, int group, double *host_out) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    const bool sum_t = (sink & DL_SUM_T) != 0;
    sink &= ~DL_SUM_T;
    if (!(sink & (DL_SINK_LOCAL | DL_SINK_SMEARED)) || (sink & ~3)) return fail(DL_EINVAL, "bad sink mask");
    if ((sink & DL_SINK_SMEARED) && !sm) return fail(DL_EINVAL, "smeared sink needs smearing parameters");
    if ((sink & DL_SINK_SMEARED) && !c->have_gauge) return fail(DL_ESTATE, "load_gauge has not been called");
    if (sm && (sm->n_iter < 0 || !std::isfinite(sm->alpha))) return fail(DL_EINVAL, "bad smearing parameters");
    const int T = c->dims[3];
    if (!t_of_rhs && (t_lo < 0 || t_hi > T || t_lo >= t_hi)) return fail(DL_EINVAL, "bad timeslice range");
    if (!host_out) return fail(DL_EINVAL, "null output");
    if (group < 1 || (n_rhs > 0 && n_rhs % group)) return fail(DL_EINVAL, "group must divide n_rhs");
    if (t_of_rhs)
        for (int j = 0; j < n_rhs; ++j)
            if (t_of_rhs[j] < 0 || t_of_rhs[j] >= T) return fail(DL_EINVAL, "t_of_rhs entry outside the lattice");
    const int n_sinks = ((sink & DL_SINK_LOCAL) ? 1 : 0) + ((sink & DL_SINK_SMEARED) ? 1 : 0);
    const int per = 16 * T;
    const int per_out = sum_t ? 16 : per;  // values per (group, sink) written to host_out
    if (n_rhs == 0) return DL_OK;
    if (!eta || !phi) return fail(DL_EINVAL, "null field pointer");
    // A batch (layout width N) holds whole groups when a group fits in 64 right-hand
    // sides; a larger group is covered by consecutive batches of a divisor of it.
    const int N = std::min(64, pow2_at_least(n_rhs));
    int per_batch = (N / group) * group;
    if (group > 64) {
        per_batch = 1;
        for (int d = 64; d >= 1; --d)
            if (group % d == 0) {
                per_batch = d;
                break;
            }
    }
    TRY(ensure_ws(c, N));
    const size_t field = (size_t)c->V * 24;
    const int cb0 = t_of_rhs ? 0 : t_lo * c->g.V3h, cb1 = t_of_rhs ? c->g.V3h : t_hi * c->g.V3h;
    std::vector<double2> h((size_t)N * n_sinks * per);
    c->cur = c->stream;
    double2 *dsum = c->d_acc;  // running sums of a group spanning batches (group > 64)
    if (group > 64) zero_kernel<<<std::max(1, (2 * per + 255) / 256), 256, 0, c->stream>>>(dsum, 2 * per);
    int g_done = 0;
    for (int j0 = 0; j0 < n_rhs; j0 += per_batch) {
        const int n = std::min(per_batch, n_rhs - j0);
        const int *tcol = nullptr;
        if (t_of_rhs) {
            CK(cudaMemcpyAsync(c->d_tcol, t_of_rhs + j0, n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
            tcol = c->d_tcol;
        }
        TRY(canon_to_eo(c, (const double *)eta + j0 * field, c->b64, n, N, 0, cb0, cb1, tcol));
        TRY(canon_to_eo(c, (const double *)phi + j0 * field, c->x64, n, N, 0, cb0, cb1, tcol));
        TRY(trace_eo(c, c->b64, c->x64, n, N, sink, sm, t_lo, t_hi, n_sinks, tcol));
        if (group <= 64) {
            const int ng = n / group;
            group_sum_kernel<<<std::max(1, (ng * n_sinks * per + 255) / 256), 256, 0, c->stream>>>(
                c->d_loops, n, N, group, n_sinks, per, c->d_acc2);
            c->kernel_launches++;
            const double2 *res = c->d_acc2;
            if (sum_t) {  // d_loops is free again: it takes the timeslice sums
                sum_t_kernel<<<std::max(1, (ng * n_sinks * 16 + 255) / 256), 256, 0, c->stream>>>(
                    c->d_acc2, ng * n_sinks * 16, T, c->d_loops);
                c->kernel_launches++;
                res = c->d_loops;
            }
            CK(cudaMemcpyAsync(h.data(), res, sizeof(double2) * (size_t)ng * n_sinks * per_out,
                               cudaMemcpyDeviceToHost, c->stream));
            TRY(sync(c));
            memcpy(host_out + (size_t)g_done * n_sinks * per_out * 2, h.data(),
                   sizeof(double2) * (size_t)ng * n_sinks * per_out);
            g_done += ng;
        } else {
            for (int s = 0; s < n_sinks; ++s) {
                double2 *part = c->d_loops + (size_t)s * N * per;
                sum_loops_kernel<<<std::max(1, (per + 255) / 256), 256, 0, c->stream>>>(part, n, per, part, per);
                add_kernel<<<std::max(1, (per + 255) / 256), 256, 0, c->stream>>>(dsum + (size_t)s * per, part, per);
                c->kernel_launches += 2;
            }
            if ((j0 + n) % group == 0) {  // a group is complete
                const double2 *res = dsum;
                if (sum_t) {
                    sum_t_kernel<<<1, 64, 0, c->stream>>>(dsum, n_sinks * 16, T, c->d_acc2);
                    c->kernel_launches++;
                    res = c->d_acc2;
                }
                CK(cudaMemcpyAsync(host_out + (size_t)g_done * n_sinks * per_out * 2, res,
                                   sizeof(double2) * n_sinks * per_out, cudaMemcpyDeviceToHost, c->stream));
                TRY(sync(c));
                zero_kernel<<<std::max(1, (2 * per + 255) / 256), 256, 0, c->stream>>>(dsum, 2 * per);
                ++g_done;
            }
        }
    }
    TRY(sync(c));
    return DL_OK;
}

static int ensure_scratch(dl_ctx::Scratch &sc, size_t bytes) {
    if (sc.cap >= bytes) return DL_OK;
    if (sc.p) cudaFree(sc.p);
    sc.p = nullptr;
    sc.cap = 0;
    if (cudaMalloc(&sc.p, bytes) != cudaSuccess) return fail(DL_ENOMEM, "cudaMalloc (correlator scratch)");
    sc.cap = bytes;
    return DL_OK;
}

// Upload n_mom momenta and build the phase table exp(-i p.(x - o)) on the device.
static int build_phases(dl_ctx *c, const int *momenta, int n_mom, int ox, int oy, int oz) {
    const int V3 = c->dims[0] * c->dims[1] * c->dims[2];
    TRY(ensure_scratch(c->s_mom, sizeof(int) * 3 * n_mom));
    TRY(ensure_scratch(c->s_phase, sizeof(double2) * (size_t)n_mom * V3));
    CK(cudaMemcpyAsync(c->s_mom.p, momenta, sizeof(int) * 3 * n_mom, cudaMemcpyHostToDevice, c->stream));
    const int tot = n_mom * V3;
    phase_table_kernel<<<std::max(1, std::min((tot + 255) / 256, 8 * c->num_sms)), 256, 0, c->stream>>>(
        (double2 *)c->s_phase.p, (const int *)c->s_mom.p, n_mom, c->g, ox, oy, oz);
    c->kernel_launches++;
    CK(cudaGetLastError());
    return DL_OK;
}

extern "C" int dl_trace_loops_mom(dl_ctx *c, const void *eta, const void *phi, int n_rhs, int sink,
                                  const dl_smear *sm, const int *momenta, int n_mom, const int *t_of_rhs, int group,
                                  double *host_out) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (n_rhs < 0) return fail(DL_EINVAL, "n_rhs < 0");
    if (!(sink & (DL_SINK_LOCAL | DL_SINK_SMEARED)) || (sink & ~3)) return fail(DL_EINVAL, "bad sink mask");
    if ((sink & DL_SINK_SMEARED) && !sm) return fail(DL_EINVAL, "smeared sink needs smearing parameters");
    if ((sink & DL_SINK_SMEARED) && !c->have_gauge) return fail(DL_ESTATE, "load_gauge has not been called");
    if (sm && (sm->n_iter < 0 || !std::isfinite(sm->alpha))) return fail(DL_EINVAL, "bad smearing parameters");
    if (!momenta || n_mom < 1 || n_mom > 256) return fail(DL_EINVAL, "need 1..256 momenta");
    if (!host_out) return fail(DL_EINVAL, "null output");
    if (group < 1 || group > 64 || (n_rhs > 0 && n_rhs % group)) return fail(DL_EINVAL, "group must be 1..64 and divide n_rhs");
    const int T = c->dims[3];
    if (t_of_rhs)
        for (int j = 0; j < n_rhs; ++j)
            if (t_of_rhs[j] < 0 || t_of_rhs[j] >= T) return fail(DL_EINVAL, "t_of_rhs entry outside the lattice");
    if (n_rhs == 0) return DL_OK;
    if (!eta || !phi) return fail(DL_EINVAL, "null field pointer");
    const int n_sinks = ((sink & DL_SINK_LOCAL) ? 1 : 0) + ((sink & DL_SINK_SMEARED) ? 1 : 0);
    const int per = n_mom * 16 * T;
    const int V3 = c->dims[0] * c->dims[1] * c->dims[2];
    const int N = std::min(64, pow2_at_least(n_rhs));
    const int per_batch = (N / group) * group;
    const int nt = t_of_rhs ? 1 : T;
    TRY(ensure_ws(c, N));
    TRY(build_phases(c, momenta, n_mom, 0, 0, 0));
    TRY(ensure_scratch(c->s_site, sizeof(double2) * (size_t)N * nt * V3 * 16));
    TRY(ensure_scratch(c->s_msum, sizeof(double2) * (size_t)N * nt * n_mom * 16));
    TRY(ensure_scratch(c->s_mloops, sizeof(double2) * (size_t)n_sinks * N * per));
    TRY(ensure_scratch(c->s_mgroup, sizeof(double2) * (size_t)N * n_sinks * per));
    MomSpec m;
    m.n_mom = n_mom;
    m.phase = (const double2 *)c->s_phase.p;
    m.site = (double2 *)c->s_site.p;
    m.msum = (double2 *)c->s_msum.p;
    m.dst = (double2 *)c->s_mloops.p;
    const size_t field = (size_t)c->V * 24;
    const int cb0 = 0, cb1 = t_of_rhs ? c->g.V3h : (int)c->Vh;
    c->cur = c->stream;
    int g_done = 0;
    for (int j0 = 0; j0 < n_rhs; j0 += per_batch) {
        const int n = std::min(per_batch, n_rhs - j0);
        const int *tcol = nullptr;
        if (t_of_rhs) {
            CK(cudaMemcpyAsync(c->d_tcol, t_of_rhs + j0, n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
            tcol = c->d_tcol;
        }
        TRY(canon_to_eo(c, (const double *)eta + j0 * field, c->b64, n, N, 0, cb0, cb1, tcol));
        TRY(canon_to_eo(c, (const double *)phi + j0 * field, c->x64, n, N, 0, cb0, cb1, tcol));
        TRY(trace_eo(c, c->b64, c->x64, n, N, sink, sm, 0, T, n_sinks, tcol, &m));
        const int ng = n / group;
        group_sum_kernel<<<std::max(1, (ng * n_sinks * per + 255) / 256), 256, 0, c->stream>>>(
            m.dst, n, N, group, n_sinks, per, (double2 *)c->s_mgroup.p);
        c->kernel_launches++;
        CK(cudaMemcpyAsync(host_out + (size_t)g_done * n_sinks * per * 2, c->s_mgroup.p,
                           sizeof(double2) * (size_t)ng * n_sinks * per, cudaMemcpyDeviceToHost, c->stream));
        TRY(sync(c));
        g_done += ng;
    }
    return DL_OK;
}

extern "C" int dl_meson_correlators(dl_ctx *c, const void *prop, const int src[4], const int *momenta, int n_mom,
                                    double *host_out) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (!prop || !src || !momenta || !host_out) return fail(DL_EINVAL, "null pointer");
    if (n_mom < 1 || n_mom > 256) return fail(DL_EINVAL, "need 1..256 momenta");
    for (int mu = 0; mu < 4; ++mu)
        if (src[mu] < 0 || src[mu] >= c->dims[mu]) return fail(DL_EINVAL, "source outside the lattice");
    const int T = c->dims[3];
    const int V3 = c->dims[0] * c->dims[1] * c->dims[2];
    c->cur = c->stream;
    TRY(build_phases(c, momenta, n_mom, src[0], src[1], src[2]));
    TRY(ensure_scratch(c->s_site, sizeof(double2) * (size_t)c->V * 256));
    TRY(ensure_scratch(c->s_msum, sizeof(double2) * (size_t)T * n_mom * 256));
    TRY(ensure_scratch(c->s_out, sizeof(double2) * (size_t)n_mom * 256 * T));
    Launch l = make_launch(c, c->V * 16, 128, 0, 8);
    meson_site_kernel<<<l.grid, l.block, 0, c->stream>>>((const double *)prop, c->V, (double2 *)c->s_site.p);
    fourier_kernel<<<dim3(T, n_mom), 256, 0, c->stream>>>((const double2 *)c->s_site.p,
                                                          (const double2 *)c->s_phase.p, V3, 256, n_mom,
                                                          (double2 *)c->s_msum.p);
    const int tot = n_mom * 256 * T;
    meson_gamma_kernel<<<std::max(1, std::min((tot + 255) / 256, 8 * c->num_sms)), 256, 0, c->stream>>>(
        (const double2 *)c->s_msum.p, c->d_gammas, T, n_mom, src[3], (double2 *)c->s_out.p);
    c->kernel_launches += 3;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_out, c->s_out.p, sizeof(double2) * (size_t)tot, cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    return DL_OK;
}

extern "C" int dl_disconnected(dl_ctx *c, const double *host_loops, const unsigned char *host_cover, int n_noise,
                               const int *momenta, int n_mom, double *host_out) {
    if (!c) return fail(DL_EINVAL, "null context");
    if (!host_loops || !momenta || !host_out) return fail(DL_EINVAL, "null pointer");
    if (n_noise < 2) return fail(DL_EINVAL, "need at least two noise vectors");
    if (n_mom < 1 || n_mom > 256) return fail(DL_EINVAL, "need 1..256 momenta");
    std::vector<int> minus(n_mom, -1);
    for (int q = 0; q < n_mom; ++q)
        for (int r = 0; r < n_mom; ++r)
            if (momenta[3 * r] == -momenta[3 * q] && momenta[3 * r + 1] == -momenta[3 * q + 1] &&
                momenta[3 * r + 2] == -momenta[3 * q + 2]) {
                minus[q] = r;
                break;
            }
    for (int q = 0; q < n_mom; ++q)
        if (minus[q] < 0) return fail(DL_EINVAL, "the momentum list must contain -p for every p");
    const int T = c->dims[3];
    const int V3 = c->dims[0] * c->dims[1] * c->dims[2];
    const size_t nl = (size_t)n_noise * n_mom * 16 * T;
    c->cur = c->stream;
    TRY(ensure_scratch(c->s_mloops, sizeof(double2) * nl));
    TRY(ensure_scratch(c->s_cover, (size_t)n_noise * T));
    TRY(ensure_scratch(c->s_mom, sizeof(int) * n_mom));
    TRY(ensure_scratch(c->s_out, sizeof(double2) * (size_t)n_mom * 256 * T));
    CK(cudaMemcpyAsync(c->s_mloops.p, host_loops, sizeof(double2) * nl, cudaMemcpyHostToDevice, c->stream));
    if (host_cover)
        CK(cudaMemcpyAsync(c->s_cover.p, host_cover, (size_t)n_noise * T, cudaMemcpyHostToDevice, c->stream));
    else
        CK(cudaMemsetAsync(c->s_cover.p, 1, (size_t)n_noise * T, c->stream));
    CK(cudaMemcpyAsync(c->s_mom.p, minus.data(), sizeof(int) * n_mom, cudaMemcpyHostToDevice, c->stream));
    const int tot = n_mom * 256 * T;
    disconnected_kernel<<<std::max(1, std::min((tot + 255) / 256, 8 * c->num_sms)), 256, 0, c->stream>>>(
        (const double2 *)c->s_mloops.p, (const unsigned char *)c->s_cover.p, (const int *)c->s_mom.p, n_noise, n_mom,
        T, 1.0 / ((double)V3 * T), (double2 *)c->s_out.p);
    c->kernel_launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_out, c->s_out.p, sizeof(double2) * (size_t)tot, cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    return DL_OK;
}

extern "C" int dl_exact_loops(dl_ctx *c, int64_t src_first, int64_t n_src, const dl_solve_params *params, int sink,
                              const dl_smear *sm, double *host_out, dl_solve_stats *stats_sum) {
    TRY(ready(c));
    if (n_src < 0 || src_first < 0 || src_first + n_src > 12 * c->V) return fail(DL_EINVAL, "source range outside 0..12V");
    if (!(sink & (DL_SINK_LOCAL | DL_SINK_SMEARED)) || (sink & ~3)) return fail(DL_EINVAL, "bad sink mask");
    if ((sink & DL_SINK_SMEARED) && !sm) return fail(DL_EINVAL, "smeared sink needs smearing parameters");
    if (!host_out) return fail(DL_EINVAL, "null output");
    SolveCfg P;
    TRY(read_params(params, &P));
    const int T = c->dims[3];
    const int per = 16 * T;
    const int n_sinks = ((sink & DL_SINK_LOCAL) ? 1 : 0) + ((sink & DL_SINK_SMEARED) ? 1 : 0);
    const int N = P.batch;
    TRY(ensure_ws(c, N));
    TRY(ensure_partials(c, (size_t)2 * c->num_sms * 16 * N * 16));
    TRY(maybe_tune(c, P.prec, N));
    TRY(maybe_tune(c, P_F64, N));
    c->cur = c->stream;
    // accumulators: local spin matrices [T][16] at d_acc, smeared loops [16][T] at d_acc + per
    double2 *accS = c->d_acc, *accSm = c->d_acc + per;
    zero_kernel<<<std::max(1, (2 * per + 255) / 256), 256, 0, c->stream>>>(c->d_acc, 2 * per);
    int worst = DL_OK;
    long tot_it = 0, tot_outer = 0;
    double max_res = 0.0;
    std::vector<OuterState> os;
    for (int64_t s0 = src_first; s0 < src_first + n_src; s0 += N) {
        const int n = (int)std::min<int64_t>(N, src_first + n_src - s0);
        TRY(dl_make_point_sources(c, s0, n, DL_PREC_F64, c->d_canon));
        TRY(canon_to_eo(c, c->d_canon, c->b64, n, N, 0, 0, (int)c->Vh));
        TRY(solve_batch(c, n, N, P, os));
        for (int j = 0; j < n; ++j) {
            const int st = status_of(os[j], P.tol, P.fixed_iters > 0);
            if (st != DL_OK && worst == DL_OK) worst = st;
            tot_it += os[j].iters;
            tot_outer += os[j].outer;
            max_res = std::max(max_res, os[j].full_b2 > 0 ? std::sqrt(os[j].full_r2 / os[j].full_b2) : 0.0);
        }
        if (sink & DL_SINK_LOCAL) {
            point_diag_kernel<<<1, 32, 0, c->stream>>>(c->x64, c->d_coords, c->g, s0, n, N, accS);
            c->kernel_launches++;
        }
        if (sink & DL_SINK_SMEARED) {
            // timeslices touched by this batch of sources
            const long V3 = 2L * c->g.V3h;
            const int ta = (int)((s0 / 12) / V3), tb = (int)(((s0 + n - 1) / 12) / V3) + 1;
            TRY(canon_to_eo(c, c->d_canon, c->b64, n, N, 0, ta * c->g.V3h, tb * c->g.V3h));
            TRY(trace_eo(c, c->b64, c->x64, n, N, DL_SINK_SMEARED, sm, ta, tb, 1));
            sum_loops_kernel<<<std::max(1, (per + 255) / 256), 256, 0, c->stream>>>(c->d_loops, n, per, c->d_loops, per);
            add_kernel<<<std::max(1, (per + 255) / 256), 256, 0, c->stream>>>(accSm, c->d_loops, per);
            c->kernel_launches += 2;
        }
    }
    std::vector<double2> h((size_t)n_sinks * per);
    int slot = 0;
    if (sink & DL_SINK_LOCAL) {
        spin_to_gamma_kernel<<<(per + 127) / 128, 128, 0, c->stream>>>(accS, T, c->d_gammas, c->d_loops);
        c->kernel_launches++;
        CK(cudaMemcpyAsync(h.data(), c->d_loops, sizeof(double2) * per, cudaMemcpyDeviceToHost, c->stream));
        ++slot;
    }
    if (sink & DL_SINK_SMEARED) {
        CK(cudaMemcpyAsync(h.data() + (size_t)slot * per, accSm, sizeof(double2) * per, cudaMemcpyDeviceToHost,
                           c->stream));
    }
    TRY(sync(c));
    memcpy(host_out, h.data(), sizeof(double2) * n_sinks * per);
    if (stats_sum) {
        stats_sum->status = worst;
        stats_sum->iters = (int)std::min<long>(tot_it, 2147483647L);
        stats_sum->outer = (int)std::min<long>(tot_outer, 2147483647L);
        stats_sum->true_residual = max_res;
    }
    if (worst != DL_OK) fail(worst, "some point sources did not converge");
    return worst;
}

// ---------------------------------------------------------------------------
// truncated solver method
// ---------------------------------------------------------------------------
// Fold per-right-hand-side loops of a batch into per-noise sums (fixed order).
__global__ void fold_noise_kernel(const double2 *loops /* [sink][N][per] */, int n, int N, int per, int n_sinks, int K,
                                  int64_t rhs0, double2 *noise /* [noise][sink][per] */, int64_t noise_base) {
    const int count = n_sinks * per;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const int s = e / per, q = e % per;
        for (int j = 0; j < n; ++j) {
            const int64_t rhs = rhs0 + j;
            const int64_t nn = rhs / K - noise_base;
            double2 &o = noise[((size_t)nn * n_sinks + s) * per + q];
            const double2 v = loops[((size_t)s * N + j) * per + q];
            o.x += v.x;
            o.y += v.y;
        }
    }
}

// mean and variance of the mean per (sink, Gamma, t) over noise vectors covering t
__global__ void tsm_combine_kernel(const double2 *lp, int n_lp, const double2 *hp, const double2 *lph, int n_hp,
                                   int n_sinks, int T, int timed, int t0, double2 *mean, double2 *var) {
    const int per = 16 * T;
    const int count = n_sinks * per;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const int t = e % T;
        double m1r = 0, m1i = 0, c1 = 0;
        for (int i = 0; i < n_lp; ++i) {
            const int ti = t0 >= 0 ? t0 : i % T;
            if (timed && ti != t) continue;
            m1r += lp[(size_t)i * count + e].x;
            m1i += lp[(size_t)i * count + e].y;
            c1 += 1;
        }
        if (c1 > 0) { m1r /= c1; m1i /= c1; }
        double v1r = 0, v1i = 0;
        for (int i = 0; i < n_lp; ++i) {
            const int ti = t0 >= 0 ? t0 : i % T;
            if (timed && ti != t) continue;
            const double dr = lp[(size_t)i * count + e].x - m1r, di = lp[(size_t)i * count + e].y - m1i;
            v1r += dr * dr;
            v1i += di * di;
        }
        double m2r = 0, m2i = 0, c2 = 0;
        for (int i = 0; i < n_hp; ++i) {
            const int ti = t0 >= 0 ? t0 : (n_lp + i) % T;
            if (timed && ti != t) continue;
            m2r += hp[(size_t)i * count + e].x - lph[(size_t)i * count + e].x;
            m2i += hp[(size_t)i * count + e].y - lph[(size_t)i * count + e].y;
            c2 += 1;
        }
        if (c2 > 0) { m2r /= c2; m2i /= c2; }
        double v2r = 0, v2i = 0;
        for (int i = 0; i < n_hp; ++i) {
            const int ti = t0 >= 0 ? t0 : (n_lp + i) % T;
            if (timed && ti != t) continue;
            const double dr = hp[(size_t)i * count + e].x - lph[(size_t)i * count + e].x - m2r;
            const double di = hp[(size_t)i * count + e].y - lph[(size_t)i * count + e].y - m2i;
            v2r += dr * dr;
            v2i += di * di;
        }
        const double s1 = c1 > 1 ? 1.0 / ((c1 - 1) * c1) : 0.0, s2 = c2 > 1 ? 1.0 / ((c2 - 1) * c2) : 0.0;
        mean[e] = make_double2(m1r + m2r, m1i + m2i);
        var[e] = make_double2(v1r * s1 + v2r * s2, v1i * s1 + v2i * s2);
    }
}

// Solve and contract noise vectors [first, first + count) with params P; per-noise
// loops (summed over dilution classes) are added into out[noise - first].
static int tsm_pass(dl_ctx *c, uint64_t seed, int64_t first, int count, unsigned dil, int t0, const SolveCfg &P,
                    int sink, const dl_smear *sm, int n_sinks, double2 *out, int *worst) {
    const int T = c->dims[3];
    const int per = 16 * T;
    SourceArgs a;
    a.coords = c->d_coords;
    a.g = c->g;
    a.seed = seed;
    a.n_noise = 1;
    a.dil_spin = (dil & DL_DIL_SPIN) ? 4 : 1;
    a.dil_colour = (dil & DL_DIL_COLOUR) ? 3 : 1;
    a.dil_eo = (dil & DL_DIL_EVENODD) ? 2 : 1;
    a.dil_cubic = (dil & DL_DIL_CUBIC) ? 8 : 1;
    a.dil_time = (dil & DL_DIL_TIME) ? 1 : 0;
    a.t0 = t0;
    const int K = a.dil_spin * a.dil_colour * a.dil_eo * a.dil_cubic;
    const int N = P.batch;
    const int64_t total = (int64_t)count * K;
    std::vector<OuterState> os;
    const size_t field = (size_t)c->V * 24;
    for (int64_t r0 = 0; r0 < total; r0 += N) {
        const int n = (int)std::min<int64_t>(N, total - r0);
        // diluted sources r0 .. r0+n-1; a noise vector's classes may straddle batches
        for (int64_t nv = r0 / K; nv <= (r0 + n - 1) / K; ++nv) {
            const int64_t lo = std::max<int64_t>(r0, nv * K), hi = std::min<int64_t>(r0 + n, (nv + 1) * K);
            a.noise_first = first + nv;
            a.k_first = (int)(lo - nv * K);
            a.k_count = (int)(hi - lo);
            Launch l = make_launch(c, (long)a.k_count * c->V, 256, 0, 16);
            z2_source_kernel<double2><<<l.grid, l.block, 0, c->stream>>>(a, (double2 *)(c->d_canon + (size_t)(lo - r0) * field));
            c->kernel_launches++;
        }
        CK(cudaGetLastError());
        TRY(canon_to_eo(c, c->d_canon, c->b64, n, N, 0, 0, (int)c->Vh));
        TRY(solve_batch(c, n, N, P, os));
        for (int j = 0; j < n; ++j) {
            const int st = status_of(os[j], P.tol, P.fixed_iters > 0);
            if (st != DL_OK && *worst == DL_OK) *worst = st;
        }
        // eta: re-convert the sources (b64 was consumed by the solver).  Time-diluted
        // sources are contracted (and smeared) on their own timeslice only.
        const int *tcol = nullptr;
        if (dil & DL_DIL_TIME) {
            int ts[64];
            for (int j = 0; j < n; ++j) ts[j] = t0 >= 0 ? t0 : (int)((first + (r0 + j) / K) % T);
            CK(cudaMemcpyAsync(c->d_tcol, ts, n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
            tcol = c->d_tcol;
        }
        TRY(canon_to_eo(c, c->d_canon, c->b64, n, N, 0, 0, tcol ? c->g.V3h : (int)c->Vh, tcol));
        TRY(trace_eo(c, c->b64, c->x64, n, N, sink, sm, 0, T, n_sinks, tcol));
        fold_noise_kernel<<<std::max(1, (n_sinks * per + 255) / 256), 256, 0, c->stream>>>(c->d_loops, n, N, per,
                                                                                           n_sinks, K, r0, out, 0);
        c->kernel_launches++;
        CK(cudaGetLastError());
    }
    return DL_OK;
}

extern "C" int dl_tsm_estimate(dl_ctx *c, uint64_t seed, int n_lp, int n_hp, unsigned dil, int t0,
                               const dl_solve_params *lp, const dl_solve_params *hp, int sink, const dl_smear *sm,
                               double *mean_out, double *var_out, double *per_noise_out) {
    TRY(ready(c));
    if (n_lp < 1 || n_hp < 1) return fail(DL_EINVAL, "need at least one LP and one HP noise vector");
    if (dil & ~31u) return fail(DL_EINVAL, "unknown dilution bits");
    if (!(sink & (DL_SINK_LOCAL | DL_SINK_SMEARED)) || (sink & ~3)) return fail(DL_EINVAL, "bad sink mask");
    if ((sink & DL_SINK_SMEARED) && !sm) return fail(DL_EINVAL, "smeared sink needs smearing parameters");
    if (!mean_out || !var_out) return fail(DL_EINVAL, "null output");
    if ((dil & DL_DIL_TIME) && t0 >= c->dims[3]) return fail(DL_EINVAL, "t0 outside the lattice");
    SolveCfg Plp, Php;
    TRY(read_params(lp, &Plp));
    TRY(read_params(hp, &Php));
    if (Plp.batch != Php.batch) return fail(DL_EINVAL, "LP and HP batch sizes must agree");
    const int T = c->dims[3];
    const int per = 16 * T;
    const int n_sinks = ((sink & DL_SINK_LOCAL) ? 1 : 0) + ((sink & DL_SINK_SMEARED) ? 1 : 0);
    const int N = Plp.batch;
    TRY(ensure_ws(c, N));
    TRY(ensure_partials(c, (size_t)2 * c->num_sms * 16 * N * 16));
    TRY(maybe_tune(c, Plp.prec, N));
    TRY(maybe_tune(c, Php.prec, N));
    TRY(maybe_tune(c, P_F64, N));
    const size_t per_noise = (size_t)n_sinks * per;
    const size_t need = per_noise * ((size_t)n_lp + 2 * (size_t)n_hp) + 2 * per_noise;
    if (c->noise_cap < need) {
        TRY(sync(c));
        if (c->d_noise) cudaFree(c->d_noise);
        c->d_noise = nullptr;
        if (cudaMalloc((void **)&c->d_noise, need * sizeof(double2)) != cudaSuccess)
            return fail(DL_ENOMEM, "TSM buffers");
        c->noise_cap = need;
    }
    double2 *d_lp = c->d_noise, *d_hp = d_lp + per_noise * n_lp, *d_lph = d_hp + per_noise * n_hp;
    double2 *d_mean = d_lph + per_noise * n_hp, *d_var = d_mean + per_noise;
    c->cur = c->stream;
    const int cnt = (int)(per_noise * ((size_t)n_lp + 2 * (size_t)n_hp));
    zero_kernel<<<std::max(1, std::min(4096, (cnt + 255) / 256)), 256, 0, c->stream>>>(c->d_noise, cnt);
    int worst = DL_OK;
    TRY(tsm_pass(c, seed, 0, n_lp, dil, t0, Plp, sink, sm, n_sinks, d_lp, &worst));
    TRY(tsm_pass(c, seed, n_lp, n_hp, dil, t0, Php, sink, sm, n_sinks, d_hp, &worst));
    TRY(tsm_pass(c, seed, n_lp, n_hp, dil, t0, Plp, sink, sm, n_sinks, d_lph, &worst));
    tsm_combine_kernel<<<std::max(1, (int)((per_noise + 127) / 128)), 128, 0, c->stream>>>(
        d_lp, n_lp, d_hp, d_lph, n_hp, n_sinks, T, (dil & DL_DIL_TIME) ? 1 : 0, t0, d_mean, d_var);
    c->kernel_launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(mean_out, d_mean, per_noise * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(var_out, d_var, per_noise * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    if (per_noise_out)
        CK(cudaMemcpyAsync(per_noise_out, c->d_noise, (size_t)cnt * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    if (worst != DL_OK) fail(worst, "some TSM solves did not converge");
    return worst;
}

// ---------------------------------------------------------------------------
// dilution study
// ---------------------------------------------------------------------------
// sigma2[G] = mean over noise vectors n (and, without time dilution, over the
// timeslices t) of |L_n[G][t] - exact[G][t]|^2, with t = t_n on the source
// timeslice of a time-diluted vector; fixed summation order.
__global__ void dilution_error_kernel(const double2 *noise /* [n][16][T] */, int n, int T, int timed, int t0,
                                      const double2 *exact /* [16][T] */, double *sigma2) {
    const int G = threadIdx.x;
    if (G >= 16) return;
    double acc = 0.0, cnt = 0.0;
    for (int i = 0; i < n; ++i)
        for (int t = 0; t < T; ++t) {
            if (timed && t != (t0 >= 0 ? t0 : i % T)) continue;
            const double2 v = noise[((size_t)i * 16 + G) * T + t], e = exact[G * T + t];
            const double dr = v.x - e.x, di = v.y - e.y;
            acc += dr * dr + di * di;
            cnt += 1.0;
        }
    sigma2[G] = cnt > 0 ? acc / cnt : 0.0;
}

extern "C" int dl_dilution_error(dl_ctx *c, uint64_t seed, int n_noise, unsigned dil, int t0,
                                 const dl_solve_params *params, const double *host_exact, double *host_sigma2,
                                 double *per_noise_out) {
    TRY(ready(c));
    if (n_noise < 1) return fail(DL_EINVAL, "need at least one noise vector");
    if (dil & ~31u) return fail(DL_EINVAL, "unknown dilution bits");
    if ((dil & DL_DIL_TIME) && t0 >= c->dims[3]) return fail(DL_EINVAL, "t0 outside the lattice");
    if (!host_exact || !host_sigma2) return fail(DL_EINVAL, "null argument");
    SolveCfg P;
    TRY(read_params(params, &P));
    const int T = c->dims[3];
    const int per = 16 * T;
    const int N = P.batch;
    TRY(ensure_ws(c, N));
    TRY(ensure_partials(c, (size_t)2 * c->num_sms * 16 * N * 16));
    TRY(maybe_tune(c, P.prec, N));
    TRY(maybe_tune(c, P_F64, N));
    // per-noise loops, the exact loops and the 16 results (as doubles) in the noise buffer
    const size_t need = (size_t)per * n_noise + per + 8;
    if (c->noise_cap < need) {
        TRY(sync(c));
        if (c->d_noise) cudaFree(c->d_noise);
        c->d_noise = nullptr;
        if (cudaMalloc((void **)&c->d_noise, need * sizeof(double2)) != cudaSuccess)
            return fail(DL_ENOMEM, "dilution-study buffers");
        c->noise_cap = need;
    }
    double2 *d_loops = c->d_noise, *d_exact = d_loops + (size_t)per * n_noise;
    double *d_sig = reinterpret_cast<double *>(d_exact + per);
    c->cur = c->stream;
    const int cnt = per * n_noise;
    zero_kernel<<<std::max(1, std::min(4096, (cnt + 255) / 256)), 256, 0, c->stream>>>(d_loops, cnt);
    CK(cudaMemcpyAsync(d_exact, host_exact, per * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    int worst = DL_OK;
    TRY(tsm_pass(c, seed, 0, n_noise, dil, t0, P, DL_SINK_LOCAL, nullptr, 1, d_loops, &worst));
    dilution_error_kernel<<<1, 32, 0, c->stream>>>(d_loops, n_noise, T, (dil & DL_DIL_TIME) ? 1 : 0, t0, d_exact,
                                                   d_sig);
    c->kernel_launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host_sigma2, d_sig, 16 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (per_noise_out)
        CK(cudaMemcpyAsync(per_noise_out, d_loops, (size_t)cnt * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    TRY(sync(c));
    if (worst != DL_OK) fail(worst, "some solves of the dilution study did not converge");
    return worst;
}

// ---------------------------------------------------------------------------
// measurement
// ---------------------------------------------------------------------------
extern "C" int dl_bench_hop(dl_ctx *c, int precision, int n_rhs, int fused, int reps, double *ms, double *bytes) {
    TRY(ready(c));
    if (precision < 0 || precision > 2 || n_rhs < 1 || n_rhs > 64 || reps < 1 || !ms || !bytes)
        return fail(DL_EINVAL, "bad arguments");
    const int N = pow2_at_least(n_rhs);
    precision = inner_prec(c, precision, N);
    TRY(ensure_ws(c, N));
    TRY(ensure_partials(c, (size_t)2 * c->num_sms * 16 * N * 16));
    c->cur = c->stream;
    const size_t ne = half_elems(c, N);
    for (int k = 0; k < 8; ++k) CK(launch_fill(precision, c->lo[k], ne, 1234u + k, c->stream));
    const int Vh = (int)c->Vh;
    if (fused < 0 || fused > 2) return fail(DL_EINVAL, "fused must be 0, 1 or 2");
    auto once = [&]() -> int {
        if (fused == 2)
            return do_hop(c, precision, MODE_XPAY, RED_BICG, lo_ptr(c, LT), lo_ptr(c, LTMP), lo_ptr(c, LS), nullptr,
                          lo_ptr(c, LRH), 0, N, -0.02, 0, Vh, c->d_partials, nullptr);
        if (fused)
            return do_hop(c, precision, MODE_XPAY, RED_R0DOT, lo_ptr(c, LV), lo_ptr(c, LTMP), lo_ptr(c, LP), nullptr,
                          lo_ptr(c, LRH), 0, N, -0.02, 0, Vh, c->d_partials, nullptr);
        return do_hop(c, precision, MODE_PLAIN, RED_NONE, lo_ptr(c, LTMP), lo_ptr(c, LP), nullptr, nullptr, nullptr, 1,
                      N, 1.0, 0, Vh, nullptr, nullptr);
    };
    const bool was = c->timing;
    c->timing = false;
    for (int k = 0; k < 3; ++k) TRY(once());
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    for (int k = 0; k < reps; ++k) TRY(once());
    cudaEventRecord(e1, c->stream);
    c->timing = was;
    CK(cudaStreamSynchronize(c->stream));
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / reps;
    const double S = 24.0 * storage_bytes(precision), L = 18.0 * storage_bytes(precision);
    *bytes = (double)Vh * (8.0 * L + (double)N * (fused ? 4 : 2) * S);
    return DL_OK;
}
