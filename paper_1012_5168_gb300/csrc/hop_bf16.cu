// Wilson-hop instantiations for bfloat16 storage (all kernel kinds), one
// right-hand side per thread, and the dispatch over R (hop_bf16_r2.cu and
// hop_bf16_r4.cu hold R = 2 and R = 4).
#include "hop_launch.cuh"

namespace dl {

cudaError_t launch_hop_bf16(int R, int mode, int red, int kind, const HopArgs &a, Launch &l) {
    if (R == 1) return launch_hop_low_r<bf16, 1>(mode, red, kind, a, l);
    if (R == 2) return launch_hop_bf16_r2(mode, red, kind, a, l);
    if (R == 4) return launch_hop_bf16_r4(mode, red, kind, a, l);
    return cudaErrorInvalidValue;
}

}  // namespace dl
