// BF16 instantiations of the warp-per-site t-sweep kernel k_fsweep_w.
#include "stencil_fsweep_w.cuh"

namespace mpmc {
namespace fsw {

int launch_w_bf16(int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s) {
    return launch_s<__nv_bfloat16, 2>(nb, kind, m, g, gx, err, s);
}

}  // namespace fsw
}  // namespace mpmc
