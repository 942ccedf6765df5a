// Wilson-hop instantiations for bfloat16 storage (all kernel kinds), 4
// right-hand sides per thread.
#include "hop_launch.cuh"

namespace dl {

cudaError_t launch_hop_bf16_r4(int mode, int red, int kind, const HopArgs &a, Launch &l) {
    return launch_hop_low_r<bf16, 4>(mode, red, kind, a, l);
}

}  // namespace dl
