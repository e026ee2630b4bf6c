// Instantiations and host side of the t-sweep issue-lean stencil kernels
// (stencil_fsweep.cuh).
#include "stencil_fsweep.cuh"

#include <algorithm>
#include <utility>
#include <vector>

namespace mpmc {

namespace {

template <class S, int NB, int KIND, bool LSM>
int launch_one(const CUtensorMap& map, const fsw::Geom4& g, int gx, int* err, cudaStream_t s) {
    constexpr int TW = fsw::tile_width<NB, LSM>();
    auto kern = fsw::k_fsweep<S, NB, KIND, LSM>;
    constexpr int smem = fsw::smem_bytes<S, TW, LSM>();
    static bool attr = false;   // one flag per instantiation
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        attr = true;
    }
    kern<<<dim3(gx * (NB / TW)), 8 * TW, smem, s>>>(map, g, err);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <class S, int NB, bool LSM>
int launch_nb(int kind, const CUtensorMap& m, const fsw::Geom4& g, int gx, int* err, cudaStream_t s) {
    switch (kind) {
        case 0: return launch_one<S, NB, 0, LSM>(m, g, gx, err, s);
        case 1: return launch_one<S, NB, 1, LSM>(m, g, gx, err, s);
        case 3: return launch_one<S, NB, 3, LSM>(m, g, gx, err, s);
        case 4: return launch_one<S, NB, 4, LSM>(m, g, gx, err, s);
        default: return 1;
    }
}

template <class S, bool LSM>
int launch_s(int nb, int kind, const CUtensorMap& m, const fsw::Geom4& g, int gx, int* err, cudaStream_t s) {
    switch (nb) {
        case 16: return launch_nb<S, 16, LSM>(kind, m, g, gx, err, s);
        case 32: return launch_nb<S, 32, LSM>(kind, m, g, gx, err, s);
        case 64: return launch_nb<S, 64, LSM>(kind, m, g, gx, err, s);
        case 128: return launch_nb<S, 128, LSM>(kind, m, g, gx, err, s);
        case 256: return launch_nb<S, 256, LSM>(kind, m, g, gx, err, s);
        case 512: return launch_nb<S, 512, LSM>(kind, m, g, gx, err, s);
        case 1024: return launch_nb<S, 1024, LSM>(kind, m, g, gx, err, s);
        default: return 1;
    }
}

}  // namespace

bool fsweep_supported(int storage, const Geom& g, int nb) {
    return fast_supported(storage, nb) && g.lx % 2 == 0 && g.ly % 2 == 0 && g.lz % 2 == 0 && g.lt >= 2;
}

SweepCfg fsweep_config(const Geom& g, int nb, int ts, bool lsm) {
    SweepCfg c;
    const int tw = lsm ? 16 : (nb < 32 ? nb : 32);
    c.nblk = (g.lx / 2) * (g.ly / 2) * (g.lz / 2);
    c.tiles = nb / tw;
    const int per_sm = lsm ? 3 : 512 / (8 * tw);   // resident CTAs per SM
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

void fsweep_morton_order(const Geom& g, int* order) {
    const int hx = g.lx / 2, hy = g.ly / 2, hz = g.lz / 2, n = hx * hy * hz;
    std::vector<std::pair<uint64_t, int>> key((size_t)n);
    for (int b = 0; b < n; ++b) {
        const uint32_t c[3] = {(uint32_t)(b % hx), (uint32_t)((b / hx) % hy), (uint32_t)(b / (hx * hy))};
        uint64_t k = 0;
        for (int bit = 0; bit < 21; ++bit)
            for (int d = 0; d < 3; ++d) k |= (uint64_t)((c[d] >> bit) & 1u) << (3 * bit + d);
        key[(size_t)b] = {k, b};
    }
    std::sort(key.begin(), key.end());
    for (int i = 0; i < n; ++i) order[i] = key[(size_t)i].second;
}

// Rows of nb complex values (inner dimension 2 nb scalars, V*12 rows), TW-complex x 12-row boxes.
bool fsweep_make_map(void* map, int storage, const void* base, int V, int nb, bool lsm) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    const int tw = lsm ? 16 : (nb < 32 ? nb : 32);
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
                  cudaStream_t s, bool lsm) {
    if (!fast_supported(storage, nb)) return 1;
    if (c.tiles != nb / (lsm ? 16 : (nb < 32 ? nb : 32))) return 1;   // shape made for the other variant
    fsw::Geom4 g;
    g.a = a;
    g.nblk = c.nblk;
    g.ts = c.ts;
    g.nseg = c.nseg;
    const CUtensorMap& m = *reinterpret_cast<const CUtensorMap*>(map);
    if (storage == ST_F32)
        return lsm ? launch_s<float, true>(nb, kind, m, g, c.rows, err, s)
                   : launch_s<float, false>(nb, kind, m, g, c.rows, err, s);
    return lsm ? launch_s<__nv_bfloat16, true>(nb, kind, m, g, c.rows, err, s)
               : launch_s<__nv_bfloat16, false>(nb, kind, m, g, c.rows, err, s);
}

}  // namespace mpmc
