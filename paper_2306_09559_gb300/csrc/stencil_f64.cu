// double instantiation of the fused stencil kernels (stencil.cuh).
#include "stencil.cuh"

namespace mpmc {

void step_f64(const Geom& g, const void* links, int nb, const NoiseSpec& ns, const StepArgs& a, const LaunchCfg& c,
             cudaStream_t s) {
    step_dispatch<double>(g, links, nb, ns, a, c, s);
}

void outer_f64(const Geom& g, const void* links, int nb, const NoiseSpec& ns, const OuterArgs& a, const LaunchCfg& c,
              cudaStream_t s) {
    outer_dispatch<double>(g, links, nb, ns, a, c, s);
}

}  // namespace mpmc
