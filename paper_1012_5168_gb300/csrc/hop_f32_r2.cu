// Wilson-hop instantiations for float storage (all kernel kinds), 2
// right-hand sides per thread.
#include "hop_launch.cuh"

namespace dl {

cudaError_t launch_hop_f32_r2(int mode, int red, int kind, const HopArgs &a, Launch &l) {
    return launch_hop_low_r<float, 2>(mode, red, kind, a, l);
}

}  // namespace dl
