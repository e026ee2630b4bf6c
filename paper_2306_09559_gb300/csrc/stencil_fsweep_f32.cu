// FP32 instantiations of the t-sweep kernels k_fsweep (links from global memory and staged).
#include "stencil_fsweep_w.cuh"

namespace mpmc {
namespace fsw {

int launch_f32(int var, int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s) {
    return var == 1 ? launch_s<float, 1>(nb, kind, m, g, gx, err, s) : launch_s<float, 0>(nb, kind, m, g, gx, err, s);
}

}  // namespace fsw
}  // namespace mpmc
