// Wilson-hop instantiations for double storage: FP64 arithmetic, and float-float
// arithmetic (hop_ff.cuh) for the defect-correction steps of mixed-precision solves.
#include "hop_ff.cuh"
#include "launch.h"

namespace dl {

template <int R, int MODE, int RED>
static cudaError_t go(const HopArgs &a, Launch &l) {
    if (a.clovinv) {  // clover: A^-1 of the output site in the epilogue
        clamp_grid(l, resident_blocks(hop_kernel_clov<double, MODE, RED>, l.block, l.smem));
        hop_kernel_clov<double, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
        return cudaGetLastError();
    }
    clamp_grid(l, resident_blocks(hop_kernel<double, R, MODE, RED>, l.block, l.smem));
    hop_kernel<double, R, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hop_f64(int R, int mode, int red, const HopArgs &a, Launch &l) {
#define DL_CASE(r, m, rd) \
    if (R == r && mode == m && red == rd) return go<r, m, rd>(a, l);
    DL_CASE(1, MODE_PLAIN, RED_NONE)
    DL_CASE(1, MODE_XPAY, RED_NONE)
    DL_CASE(1, MODE_XPAY, RED_R0DOT)
    DL_CASE(1, MODE_XPAY, RED_BICG)
    DL_CASE(1, MODE_XPAY, RED_NORM)
    DL_CASE(1, MODE_RESID, RED_NORM)
#undef DL_CASE
    return cudaErrorInvalidValue;
}

template <int MODE, int RED, bool YFF, bool OFF>
static cudaError_t go_ff(const HopArgs &a, Launch &l) {
    clamp_grid(l, resident_blocks(hop_ff_rows_kernel<MODE, RED, YFF, OFF>, l.block, l.smem));
    hop_ff_rows_kernel<MODE, RED, YFF, OFF><<<l.grid, l.block, l.smem, l.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hop_ff(int mode, int red, int fmt, const HopArgs &a, Launch &l) {
    const bool yff = fmt & FF_Y, off = fmt & FF_OUT;
#define DL_CASE(m, rd, y, o) \
    if (mode == m && red == rd && yff == y && off == o) return go_ff<m, rd, y, o>(a, l);
    DL_CASE(MODE_PLAIN, RED_NONE, false, false)
    DL_CASE(MODE_XPAY, RED_NONE, false, false)
    DL_CASE(MODE_XPAY, RED_NONE, true, false)
    DL_CASE(MODE_XPAY, RED_NONE, true, true)
    DL_CASE(MODE_XPAY, RED_NORM, false, false)
    DL_CASE(MODE_RESID, RED_NORM, true, false)
#undef DL_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_ff_cast(const double *src, double *dst, size_t n_complex, int to_ff, int grid, cudaStream_t s) {
    ff_cast_kernel<<<grid, 256, 0, s>>>(src, dst, (long)n_complex, to_ff);
    return cudaGetLastError();
}

}  // namespace dl
