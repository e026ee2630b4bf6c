// FP32 instantiations of the two-sites-per-warp t-sweep kernel k_fsweep_p.
#include "stencil_fsweep_p.cuh"

namespace mpmc {
namespace fsw {

int launch_p_f32(int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s) {
    return launch_p_s<float>(nb, kind, m, g, gx, err, s);
}

}  // namespace fsw
}  // namespace mpmc
