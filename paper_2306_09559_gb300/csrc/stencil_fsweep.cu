// Host side of the t-sweep issue-lean stencil kernels (stencil_fsweep.cuh); their
// instantiations are split over stencil_fsweep_{f32,bf16,w_f32,w_bf16,p_f32,p_bf16}.cu so that
// they compile in parallel.
#include "stencil_fsweep_p.cuh"
#include "stencil_fsweep_w.cuh"

#include <algorithm>
#include <utility>
#include <vector>

namespace mpmc {


bool fsweep_supported(int storage, const Geom& g, int nb) {
    return fast_supported(storage, nb) && g.lx % 2 == 0 && g.ly % 2 == 0 && g.lz % 2 == 0 && g.lt >= 2;
}

int fsweep_variant(int mask, int nb) {
    if (mask & 64) return 3;
    if (mask & 32) return nb >= 32 ? 2 : 1;
    return (mask & 16) ? 1 : 0;
}

int fsweep_tile(int var, int nb) { return var == 2 ? fsw::WTW : var == 3 ? fsw::PTW : var == 1 ? 16 : (nb < 32 ? nb : 32); }

SweepCfg fsweep_config(const Geom& g, int nb, int ts, int var) {
    SweepCfg c;
    const int tw = fsweep_tile(var, nb);
    c.nblk = (g.lx / 2) * (g.ly / 2) * (g.lz / 2);
    c.tiles = nb / tw;
    const int per_sm = var == 3 ? 4 : var == 2 ? 2 : var == 1 ? 3 : 512 / (8 * tw);   // resident CTAs per SM
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
bool fsweep_make_map(void* map, int storage, const void* base, int V, int nb, int tw) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || tw <= 0 || nb % tw) return false;
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
                  cudaStream_t s, int var) {
    if (!fast_supported(storage, nb) || var < 0 || var > 3) return 1;
    if (var == 2 && nb < 32) var = 1;
    if (c.tiles != nb / fsweep_tile(var, nb)) return 1;   // shape made for another variant
    fsw::Geom4 g;
    g.a = a;
    g.nblk = c.nblk;
    g.ts = c.ts;
    g.nseg = c.nseg;
    const CUtensorMap& m = *reinterpret_cast<const CUtensorMap*>(map);
    if (storage == ST_F32)
        return var == 3 ? fsw::launch_p_f32(nb, kind, m, g, c.rows, err, s)
             : var == 2 ? fsw::launch_w_f32(nb, kind, m, g, c.rows, err, s)
                        : fsw::launch_f32(var, nb, kind, m, g, c.rows, err, s);
    return var == 3 ? fsw::launch_p_bf16(nb, kind, m, g, c.rows, err, s)
         : var == 2 ? fsw::launch_w_bf16(nb, kind, m, g, c.rows, err, s)
                    : fsw::launch_bf16(var, nb, kind, m, g, c.rows, err, s);
}

}  // namespace mpmc
