// Wilson-hop instantiations for double storage: FP64 arithmetic, and float-float
// arithmetic (dfs) for the defect-correction steps of mixed-precision solves.
#include "launch.h"

namespace dl {

template <int R, int MODE, int RED>
static cudaError_t go(const HopArgs &a, Launch &l) {
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

template <int MODE, int RED>
static cudaError_t go_dff(const HopArgs &a, Launch &l) {
    clamp_grid(l, resident_blocks(hop_kernel<dfs, 1, MODE, RED>, l.block, l.smem));
    hop_kernel<dfs, 1, MODE, RED><<<l.grid, l.block, l.smem, l.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hop_dff(int R, int mode, int red, const HopArgs &a, Launch &l) {
    if (R != 1) return cudaErrorInvalidValue;
#define DL_CASE(m, rd) \
    if (mode == m && red == rd) return go_dff<m, rd>(a, l);
    DL_CASE(MODE_PLAIN, RED_NONE)
    DL_CASE(MODE_XPAY, RED_NONE)
    DL_CASE(MODE_XPAY, RED_NORM)
    DL_CASE(MODE_RESID, RED_NORM)
#undef DL_CASE
    return cudaErrorInvalidValue;
}

}  // namespace dl
