// Instantiations and host launchers of the t-sweep stencil kernels
// (stencil_sweep.cuh) for FP32 and BF16-stored spinors.
#include "stencil_sweep.cuh"

#include <algorithm>

namespace mpmc {

namespace {

template <class S, class A, bool DOT, int Y>
int launch_one(const CUtensorMap& map, const A& a, const SweepGeom& sg, const void* links, int nb, const NoiseKey& nk,
               int tiles, int* err, cudaStream_t s) {
    auto kern = k_sweep<S, A, DOT, Y>;
    static bool attr = false;   // one flag per instantiation
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<S>()) !=
            cudaSuccess)
            return 1;
        attr = true;
    }
    const dim3 grid(sg.nblk * ((sg.L.lt + sg.ts - 1) / sg.ts), tiles);
    kern<<<grid, 256, sweep_smem_bytes<S>(), s>>>(map, a, sg, reinterpret_cast<const typename Math<S>::T*>(links), nb,
                                                  nk, err);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

NoiseKey key_of(const NoiseSpec& ns) {
    NoiseKey nk;
    nk.k0 = (uint32_t)(ns.seed & 0xffffffffu);
    nk.k1 = (uint32_t)(ns.seed >> 32);
    nk.level = ns.level;
    nk.j0 = ns.j0;
    return nk;
}

SweepGeom geom_of(const Geom& g, const SweepCfg& c) {
    SweepGeom sg;
    sg.L.lx = g.lx; sg.L.ly = g.ly; sg.L.lz = g.lz; sg.L.lt = g.lt; sg.L.V = g.V; sg.L.bc_t = g.bc_t;
    sg.nblk = c.nblk;
    sg.ts = c.ts;
    return sg;
}

template <class S>
int step_s(const CUtensorMap& m, const StepArgs& a, const SweepGeom& sg, const void* U, int nb, const NoiseKey& nk,
           int tiles, int* err, cudaStream_t s) {
    if (a.dot) {
        if (a.ymode == 0) return launch_one<S, StepArgs, true, 0>(m, a, sg, U, nb, nk, tiles, err, s);
        if (a.ymode == 1) return launch_one<S, StepArgs, true, 1>(m, a, sg, U, nb, nk, tiles, err, s);
        return launch_one<S, StepArgs, true, 2>(m, a, sg, U, nb, nk, tiles, err, s);
    }
    if (a.ymode == 0) return launch_one<S, StepArgs, false, 0>(m, a, sg, U, nb, nk, tiles, err, s);
    if (a.ymode == 1) return launch_one<S, StepArgs, false, 1>(m, a, sg, U, nb, nk, tiles, err, s);
    return launch_one<S, StepArgs, false, 2>(m, a, sg, U, nb, nk, tiles, err, s);
}

template <class S>
int outer_s(const CUtensorMap& m, const OuterArgs& a, const SweepGeom& sg, const void* U, int nb, const NoiseKey& nk,
            int tiles, int* err, cudaStream_t s) {
    if (a.dot) return launch_one<S, OuterArgs, true, 0>(m, a, sg, U, nb, nk, tiles, err, s);
    return launch_one<S, OuterArgs, false, 0>(m, a, sg, U, nb, nk, tiles, err, s);
}

}  // namespace

bool sweep_supported(int storage, const Geom& g, int nb) {
    if (storage != ST_F32 && storage != ST_BF16) return false;
    if (g.lx % 2 || g.ly % 2 || g.lz % 2 || g.lt < 2) return false;
    // TMA row stride (nb complex) must be a multiple of 16 bytes
    return storage == ST_F32 ? nb % 2 == 0 : nb % 4 == 0;
}

SweepCfg sweep_config(const Geom& g, int nb, int ts) {
    SweepCfg c;
    c.nblk = (g.lx / 2) * (g.ly / 2) * (g.lz / 2);
    c.tiles = (nb + SWEEP_TW - 1) / SWEEP_TW;
    if (ts <= 0) {
        // the longest segment that still gives at least four CTAs per SM (two waves at two per SM)
        ts = g.lt;
        while (ts % 2 == 0 && ts > 4 && (long long)c.nblk * c.tiles * (g.lt / ts) < 4 * 152) ts /= 2;
    }
    c.ts = std::min(std::max(ts, 1), g.lt);
    c.nseg = (g.lt + c.ts - 1) / c.ts;
    c.rows = c.nblk * c.nseg;
    return c;
}

size_t sweep_map_bytes() { return sizeof(CUtensorMap); }

// Rows of nb complex values (inner dimension 2 nb scalars, V*12 rows), 32-complex x 12-row boxes.
bool sweep_make_map(void* map, int storage, const void* base, int V, int nb) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    const size_t es = storage == ST_F32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)2 * nb, (cuuint64_t)V * 12};
    cuuint64_t strides[1] = {(cuuint64_t)2 * nb * es};
    cuuint32_t box[2] = {2 * SWEEP_TW, 12};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = storage == ST_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int launch_sweep_step(int storage, const Geom& g, const void* links, int nb, const NoiseSpec& ns, const StepArgs& a0,
                      const SweepCfg& c, const void* map, int* err, cudaStream_t s) {
    StepArgs a = a0;
    fill_floats(a);
    const SweepGeom sg = geom_of(g, c);
    const CUtensorMap& m = *reinterpret_cast<const CUtensorMap*>(map);
    if (storage == ST_F32) return step_s<float>(m, a, sg, links, nb, key_of(ns), c.tiles, err, s);
    return step_s<__nv_bfloat16>(m, a, sg, links, nb, key_of(ns), c.tiles, err, s);
}

int launch_sweep_outer(int storage, const Geom& g, const void* links, int nb, const NoiseSpec& ns,
                       const OuterArgs& a0, const SweepCfg& c, const void* map, int* err, cudaStream_t s) {
    OuterArgs a = a0;
    fill_floats(a);
    const SweepGeom sg = geom_of(g, c);
    const CUtensorMap& m = *reinterpret_cast<const CUtensorMap*>(map);
    if (storage == ST_F32) return outer_s<float>(m, a, sg, links, nb, key_of(ns), c.tiles, err, s);
    return outer_s<__nv_bfloat16>(m, a, sg, links, nb, key_of(ns), c.tiles, err, s);
}

}  // namespace mpmc
