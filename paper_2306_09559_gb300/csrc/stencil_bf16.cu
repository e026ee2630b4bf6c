// __nv_bfloat16 instantiation of the fused stencil kernels (stencil.cuh).
#include "stencil.cuh"

namespace mpmc {

void step_bf16(const Geom& g, const void* links, int nb, const NoiseSpec& ns, const StepArgs& a, const LaunchCfg& c,
             cudaStream_t s) {
    step_dispatch<__nv_bfloat16>(g, links, nb, ns, a, c, s);
}

void outer_bf16(const Geom& g, const void* links, int nb, const NoiseSpec& ns, const OuterArgs& a, const LaunchCfg& c,
              cudaStream_t s) {
    outer_dispatch<__nv_bfloat16>(g, links, nb, ns, a, c, s);
}

}  // namespace mpmc
