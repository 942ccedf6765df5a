// Wilson-hop instantiations for float storage (all kernel kinds).
#include "hop_launch.cuh"

namespace dl {

cudaError_t launch_hop_f32(int R, int mode, int red, int kind, const HopArgs &a, Launch &l) {
    return launch_hop_low<float>(R, mode, red, kind, a, l);
}

}  // namespace dl
