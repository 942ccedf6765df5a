// Instantiations and launchers of the BiCGStab vector kernels for every
// storage precision and right-hand sides per thread.
#include "launch.h"

namespace dl {

#define DL_DISPATCH(PREC, R, CALL)                                  \
    do {                                                            \
        if (PREC == P_F64 && R == 1) { typedef double S; CALL(S, 1); } \
        else if (PREC == P_F32 && R == 1) { typedef float S; CALL(S, 1); } \
        else if (PREC == P_F32 && R == 2) { typedef float S; CALL(S, 2); } \
        else if (PREC == P_F32 && R == 4) { typedef float S; CALL(S, 4); } \
        else if (PREC == P_F32P && R == 1) { typedef f32p S; CALL(S, 1); } \
        else if (PREC == P_F32P && R == 2) { typedef f32p S; CALL(S, 2); } \
        else if (PREC == P_F32P && R == 4) { typedef f32p S; CALL(S, 4); } \
        else if (PREC == P_BF16 && R == 1) { typedef bf16 S; CALL(S, 1); } \
        else if (PREC == P_BF16 && R == 2) { typedef bf16 S; CALL(S, 2); } \
        else if (PREC == P_BF16 && R == 4) { typedef bf16 S; CALL(S, 4); } \
        else return cudaErrorInvalidValue;                          \
    } while (0)

cudaError_t launch_axpy_s(const VecLaunch &v, const RhsState *st, const void *r, const void *vv, void *s) {
#define CALL(S, RR)                                                                                   \
    axpy_s_kernel<S, RR><<<v.l.grid, v.l.block, 0, v.l.stream>>>(v.a, st, (const S *)r, (const S *)vv, \
                                                                 (S *)s)
    DL_DISPATCH(v.prec, v.R, CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_update(const VecLaunch &v, const RhsState *st, void *x, void *r, void *p, const void *s,
                          const void *t, const void *vv) {
#define CALL(S, RR)                                                                                   \
    update_kernel<S, RR><<<v.l.grid, v.l.block, 0, v.l.stream>>>(v.a, st, (S *)x, (S *)r, (S *)p,     \
                                                                 (const S *)s, (const S *)t, (const S *)vv)
    DL_DISPATCH(v.prec, v.R, CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_inner_init(const VecLaunch &v, const OuterState *os, const RhsState *st, const double *r64,
                              void *x, void *r, void *rhat, void *p, double2 *partials, int restart) {
#define CALL(S, RR)                                                                                       \
    inner_init_kernel<S, RR><<<v.l.grid, v.l.block, v.l.smem, v.l.stream>>>(v.a, os, st, r64, (S *)x, (S *)r, \
                                                                            (S *)rhat, (S *)p, partials, restart)
    DL_DISPATCH(v.prec, v.R, CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const VecLaunch &v, const OuterState *os, const void *x, double *x64) {
#define CALL(S, RR) \
    accumulate_kernel<S, RR><<<v.l.grid, v.l.block, 0, v.l.stream>>>(v.a, os, (const S *)x, x64)
    DL_DISPATCH(v.prec, v.R, CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_norm2(const VecLaunch &v, const void *x, double2 *partials) {
#define CALL(S, RR) \
    norm2_kernel<S, RR><<<v.l.grid, v.l.block, v.l.smem, v.l.stream>>>(v.a, (const S *)x, partials)
    DL_DISPATCH(v.prec, v.R, CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_cg_init(const VecLaunch &v, const OuterState *os, const double *r64, void *x, void *r5,
                           double2 *partials) {
#define CALL(S, RR)                                                                                     \
    cg_init_kernel<S, RR><<<v.l.grid, v.l.block, v.l.smem, v.l.stream>>>(v.a, os, r64, (S *)x, (S *)r5, \
                                                                        partials)
    DL_DISPATCH(v.prec, v.R, CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_cg_update(const VecLaunch &v, const RhsState *st, void *x, void *r5, const void *p, const void *w,
                             double2 *partials) {
#define CALL(S, RR)                                                                                      \
    cg_update_kernel<S, RR><<<v.l.grid, v.l.block, v.l.smem, v.l.stream>>>(v.a, st, (S *)x, (S *)r5,      \
                                                                          (const S *)p, (const S *)w, partials)
    DL_DISPATCH(v.prec, v.R, CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_cg_p(const VecLaunch &v, const RhsState *st, const void *u, void *p, int init) {
#define CALL(S, RR) \
    cg_p_kernel<S, RR><<<v.l.grid, v.l.block, 0, v.l.stream>>>(v.a, st, (const S *)u, (S *)p, init)
    DL_DISPATCH(v.prec, v.R, CALL);
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_cast(int prec, double *f64, void *lo, size_t n_complex, int to_lo, int grid, cudaStream_t s) {
    const int block = 256;
    if (prec == P_F32) cast_kernel<float><<<grid, block, 0, s>>>(f64, (float *)lo, n_complex, to_lo);
    else if (prec == P_F32P) cast_kernel<f32p><<<grid, block, 0, s>>>(f64, (f32p *)lo, n_complex, to_lo);
    else if (prec == P_BF16) cast_kernel<bf16><<<grid, block, 0, s>>>(f64, (bf16 *)lo, n_complex, to_lo);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_fill(int prec, void *x, size_t n_complex, uint32_t seed, cudaStream_t s) {
    const int grid = 1024, block = 256;
    if (prec == P_F64) fill_kernel<double><<<grid, block, 0, s>>>((double *)x, n_complex, seed);
    else if (prec == P_F32) fill_kernel<float><<<grid, block, 0, s>>>((float *)x, n_complex, seed);
    else if (prec == P_F32P) fill_kernel<f32p><<<grid, block, 0, s>>>((f32p *)x, n_complex, seed);
    else if (prec == P_BF16) fill_kernel<bf16><<<grid, block, 0, s>>>((bf16 *)x, n_complex, seed);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace dl
