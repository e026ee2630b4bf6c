// Instantiations and host side of the t-sweep issue-lean stencil kernels
// (stencil_fsweep.cuh).
#include "stencil_fsweep.cuh"

#include <algorithm>

namespace mpmc {

namespace {

template <class S, int NB, int KIND>
int launch_one(const CUtensorMap& map, const fsw::Geom4& g, int gx, int* err, cudaStream_t s) {
    constexpr int TW = NB < 32 ? NB : 32;
    auto kern = fsw::k_fsweep<S, NB, KIND>;
    constexpr int smem = fsw::smem_bytes<S, TW>();
    static bool attr = false;   // one flag per instantiation
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        attr = true;
    }
    kern<<<dim3(gx, NB / TW), 8 * TW, smem, s>>>(map, g, err);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <class S, int NB>
int launch_nb(int kind, const CUtensorMap& m, const fsw::Geom4& g, int gx, int* err, cudaStream_t s) {
    switch (kind) {
        case 0: return launch_one<S, NB, 0>(m, g, gx, err, s);
        case 1: return launch_one<S, NB, 1>(m, g, gx, err, s);
        case 3: return launch_one<S, NB, 3>(m, g, gx, err, s);
        case 4: return launch_one<S, NB, 4>(m, g, gx, err, s);
        default: return 1;
    }
}

template <class S>
int launch_s(int nb, int kind, const CUtensorMap& m, const fsw::Geom4& g, int gx, int* err, cudaStream_t s) {
    switch (nb) {
        case 16: return launch_nb<S, 16>(kind, m, g, gx, err, s);
        case 32: return launch_nb<S, 32>(kind, m, g, gx, err, s);
        case 64: return launch_nb<S, 64>(kind, m, g, gx, err, s);
        case 128: return launch_nb<S, 128>(kind, m, g, gx, err, s);
        case 256: return launch_nb<S, 256>(kind, m, g, gx, err, s);
        case 512: return launch_nb<S, 512>(kind, m, g, gx, err, s);
        case 1024: return launch_nb<S, 1024>(kind, m, g, gx, err, s);
        default: return 1;
    }
}

}  // namespace

bool fsweep_supported(int storage, const Geom& g, int nb) {
    return fast_supported(storage, nb) && g.lx % 2 == 0 && g.ly % 2 == 0 && g.lz % 2 == 0 && g.lt >= 2;
}

SweepCfg fsweep_config(const Geom& g, int nb, int ts) {
    SweepCfg c;
    const int tw = nb < 32 ? nb : 32;
    c.nblk = (g.lx / 2) * (g.ly / 2) * (g.lz / 2);
    c.tiles = nb / tw;
    const int per_sm = 512 / (8 * tw);   // resident CTAs per SM (16 warps)
    if (ts <= 0) {
        // the longest segment that still fills two waves of the 152 SMs
        ts = g.lt;
        while (ts % 2 == 0 && ts > 4 && (long long)c.nblk * c.tiles * (g.lt / ts) < 2LL * per_sm * 152) ts /= 2;
    }
    c.ts = std::min(std::max(ts, 1), g.lt);
    c.nseg = (g.lt + c.ts - 1) / c.ts;
    c.rows = c.nblk * c.nseg;
    return c;
}

// Rows of nb complex values (inner dimension 2 nb scalars, V*12 rows), TW-complex x 12-row boxes.
bool fsweep_make_map(void* map, int storage, const void* base, int V, int nb) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    const int tw = nb < 32 ? nb : 32;
    const size_t es = storage == ST_F32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)2 * nb, (cuuint64_t)V * 12};
    cuuint64_t strides[1] = {(cuuint64_t)2 * nb * es};
    cuuint32_t box[2] = {(cuuint32_t)(2 * tw), 12};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = storage == ST_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int launch_fsweep(int storage, int nb, int kind, const FastArgs& a, const SweepCfg& c, const void* map, int* err,
                  cudaStream_t s) {
    if (!fast_supported(storage, nb)) return 1;
    fsw::Geom4 g;
    g.a = a;
    g.nblk = c.nblk;
    g.ts = c.ts;
    const CUtensorMap& m = *reinterpret_cast<const CUtensorMap*>(map);
    if (storage == ST_F32) return launch_s<float>(nb, kind, m, g, c.rows, err, s);
    return launch_s<__nv_bfloat16>(nb, kind, m, g, c.rows, err, s);
}

}  // namespace mpmc
