// Wilson-hop instantiations for bfloat16 storage (all kernel kinds).
#include "hop_launch.cuh"

namespace dl {

cudaError_t launch_hop_bf16(int R, int mode, int red, int kind, const HopArgs &a, Launch &l) {
    return launch_hop_low<bf16>(R, mode, red, kind, a, l);
}

}  // namespace dl
