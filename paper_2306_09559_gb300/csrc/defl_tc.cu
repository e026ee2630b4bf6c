// Deflation dot products on the tensor cores (paper Sec. 4.1): for a block of
// Z4 noise vectors b_c and the k deflation vectors z_i,
//     G1[i][c] = z_i^H b_c,   G2[i][c] = z_i^H gamma5 b_c,
// as one real GEMM  D[i][4c + t] = sum_K A[i][K] B[4c + t][K]  over the real
// index K = (site, spin*3 + colour, re/im) of length 24 V:
//     A[i][K]        = z_i in interleaved (re, im) order, split into two BF16
//                      planes z = hi + lo (both MMAs accumulate into one FP32
//                      TMEM accumulator, ~16 significant bits of z);
//     B[4c + 0][K]   = (Re b, Im b)          -> Re(z^H b)
//     B[4c + 1][K]   = (Im b, -Re b)         -> Im(z^H b)
//     B[4c + 2/3][K] = the same times the gamma5 sign of the spin -> z^H gamma5 b
// B holds only 0 and +-1, exact in BF16; it is generated from Philox directly
// into the swizzled shared-memory tile and never stored in HBM.  A tiles come
// in by TMA.  One elected thread issues tcgen05.mma (128 x 256 x 16 per
// instruction); the accumulator lives in TMEM and is read back with
// tcgen05.ld.  K is split over CTAs; partial sums are reduced in a fixed order.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "device.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace mpmc {

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 3;
constexpr int A_BYTES = BM * BK * 2;             // one BF16 plane of an A tile (16 KB)
constexpr int B_BYTES = BN * BK * 2;             // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t IDESC = tc::idesc_bf16_f32(BM, BN);
constexpr long long TIMEOUT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

struct TcArgs {
    int V, nb, Mpad, kblocks, kb_per_split, Npad;
    NoiseKey nk;
    float* part;       // [split][Mpad][Npad]
    int* err;          // set to a non-zero code when a wait times out
};

__device__ __forceinline__ uint16_t bf16_of(int v) { return v > 0 ? 0x3F80u : (v < 0 ? 0xBF80u : 0u); }

// Fill the B tile of global K block `kbg` for noise columns nt*64 .. nt*64+63.
// Thread t handles column t/2 and half (t%2) of the 64 K values: four rows
// (the four variants) x four 16-byte chunks.
__device__ __forceinline__ void gen_b_tile(uint8_t* sB, int kbg, int nt, int t, const TcArgs& p) {
    const int cl = t >> 1, half = t & 1;
    const int c = nt * 64 + cl;
    const int k0 = kbg * BK + half * 32;
    const int s_lo = k0 / 24;
    uint32_t wd[3] = {0, 0, 0};
    bool live[3] = {false, false, false};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int site = s_lo + j;
        if (c < p.nb && site < p.V && site * 24 < k0 + 32) {
            wd[j] = z4_word(p.nk, site, c);
            live[j] = true;
        }
    }
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        uint32_t pk[4][4];   // [variant][2 bf16 per word]
#pragma unroll
        for (int e2 = 0; e2 < 8; e2 += 2) {
            int v[4][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kg = k0 + ch * 8 + e2 + h;
                const int site = kg / 24, rem = kg - site * 24;
                const int j = site - s_lo;
                const int e = rem >> 1, reim = rem & 1;
                int br = 0, bi = 0;
                if (j >= 0 && j < 3 && live[j]) {
                    const uint32_t q = (wd[j] >> (2 * e)) & 3u;
                    br = q == 0 ? 1 : (q == 2 ? -1 : 0);
                    bi = q == 1 ? 1 : (q == 3 ? -1 : 0);
                }
                const int sg = e < 6 ? 1 : -1;
                v[0][h] = reim ? bi : br;
                v[1][h] = reim ? -br : bi;
                v[2][h] = sg * v[0][h];
                v[3][h] = sg * v[1][h];
            }
#pragma unroll
            for (int t4 = 0; t4 < 4; ++t4)
                pk[t4][e2 >> 1] = (uint32_t)bf16_of(v[t4][0]) | ((uint32_t)bf16_of(v[t4][1]) << 16);
        }
        const int chunk = half * 4 + ch;
#pragma unroll
        for (int t4 = 0; t4 < 4; ++t4) {
            const int row = cl * 4 + t4;
            uint4* dst = reinterpret_cast<uint4*>(sB + row * 128 + ((chunk ^ (row & 7)) << 4));
            *dst = make_uint4(pk[t4][0], pk[t4][1], pk[t4][2], pk[t4][3]);
        }
    }
}

__global__ void __launch_bounds__(192, 1) k_defl_tc(const __grid_constant__ CUtensorMap tmA, TcArgs p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full_a = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* full_b = full_a + STAGES;
    uint64_t* empty = full_b + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x, nt = blockIdx.y, split = blockIdx.z;
    const int kb0 = split * p.kb_per_split;
    const int kb1 = min(p.kblocks, kb0 + p.kb_per_split);
    const int nkb = max(0, kb1 - kb0);
    const long long deadline = clock64() + TIMEOUT_CYCLES;

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full_a[s], 1);
            tc::mbar_init(&full_b[s], 128);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, BN);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    auto stageA = [&](int s, int plane) { return smem + s * STAGE_BYTES + plane * A_BYTES; };
    auto stageB = [&](int s) { return smem + s * STAGE_BYTES + 2 * A_BYTES; };

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (i / STAGES) & 1;
                if (i >= STAGES && !tc::mbar_wait(&empty[s], ph ^ 1, deadline)) { s_fail = 1; break; }
                if (s_fail) break;
                tc::mbar_expect_tx(&full_a[s], 2 * A_BYTES);
                tc::tma_load_2d(stageA(s, 0), &tmA, (kb0 + i) * BK, mt * BM, &full_a[s]);
                tc::tma_load_2d(stageA(s, 1), &tmA, (kb0 + i) * BK, p.Mpad + mt * BM, &full_a[s]);
                issued = i + 1;
            }
            // never leave the CTA with copies still landing in its shared memory
            for (int i = max(0, issued - STAGES); i < issued; ++i)
                if (!tc::mbar_wait(&full_a[i % STAGES], (i / STAGES) & 1, deadline + TIMEOUT_CYCLES)) s_fail = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int i = 0; i < nkb; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (i / STAGES) & 1;
                if (!tc::mbar_wait(&full_a[s], ph, deadline) || !tc::mbar_wait(&full_b[s], ph, deadline)) {
                    s_fail = 1;
                    break;
                }
                tc::fence_after();
                const uint32_t a0 = tc::smem_u32(stageA(s, 0)), a1 = tc::smem_u32(stageA(s, 1));
                const uint32_t b = tc::smem_u32(stageB(s));
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint64_t bd = tc::sw128_desc(b + kk * 32);
                    tc::mma_bf16(tmem, tc::sw128_desc(a0 + kk * 32), bd, IDESC, (i > 0 || kk > 0) ? 1u : 0u);
                    tc::mma_bf16(tmem, tc::sw128_desc(a1 + kk * 32), bd, IDESC, 1u);
                }
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(done);
        }
    } else {
        const int t = threadIdx.x - 64;   // 0..127
        for (int i = 0; i < nkb; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (i / STAGES) & 1;
            if (i >= STAGES && !tc::mbar_wait(&empty[s], ph ^ 1, deadline)) { s_fail = 1; break; }
            gen_b_tile(stageB(s), kb0 + i, nt, t, p);
            tc::fence_proxy_async();
            tc::mbar_arrive(&full_b[s]);
        }
        // epilogue: TMEM lanes of this warp's quarter -> partial sums
        const bool ok = tc::mbar_wait(done, 0, deadline + TIMEOUT_CYCLES);
        tc::fence_after();
        const int q = warp & 3;
        const int m = mt * BM + q * 32 + lane;
        float* dst = p.part + ((size_t)split * p.Mpad + m) * p.Npad + (size_t)nt * BN;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + c0, r);
            tc::tmem_wait_ld();
            float4* d4 = reinterpret_cast<float4*>(dst + c0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float4 v;
                v.x = (ok && nkb > 0) ? __uint_as_float(r[4 * j + 0]) : 0.f;
                v.y = (ok && nkb > 0) ? __uint_as_float(r[4 * j + 1]) : 0.f;
                v.z = (ok && nkb > 0) ? __uint_as_float(r[4 * j + 2]) : 0.f;
                v.w = (ok && nkb > 0) ? __uint_as_float(r[4 * j + 3]) : 0.f;
                d4[j] = v;
            }
        }
        if (!ok) s_fail = 1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 1) tc::tmem_dealloc(tmem, BN);
    if (threadIdx.x == 0 && s_fail) atomicExch(p.err, 1);
}

// z (FP64, k vectors of n complex, vector-major) -> zhat in FP32 and its two BF16 planes:
// hi = bf16(z), lo = bf16(z - hi), zhat = hi + lo (exact in FP32).
__global__ void k_split_bf16(size_t n2, int k, int Mpad, int Kpad, const double* __restrict__ z, float* zhat,
                             __nv_bfloat16* planes) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // over Mpad * Kpad
    if (idx >= (size_t)Mpad * Kpad) return;
    const int i = (int)(idx / Kpad);
    const size_t kk = idx % Kpad;
    float hi = 0.f, lo = 0.f;
    if (i < k && kk < n2) {
        const float x = (float)z[(size_t)i * n2 + kk];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __bfloat162float(h);
        lo = __bfloat162float(__float2bfloat16_rn(x - hi));
        zhat[(size_t)i * n2 + kk] = hi + lo;
    }
    planes[idx] = __float2bfloat16_rn(hi);
    planes[(size_t)Mpad * Kpad + idx] = __float2bfloat16_rn(lo);
}

// G1[i][c], G2[i][c] (complex double) from the split partials.
__global__ void k_tc_reduce(int k, int nb, int Mpad, int Npad, int nsplit, const float* __restrict__ part, double2* G1,
                            double2* G2) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)k * nb) return;
    const int i = (int)(idx / nb), c = (int)(idx % nb);
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int s = 0; s < nsplit; ++s) {
        const float4 v = *reinterpret_cast<const float4*>(part + ((size_t)s * Mpad + i) * Npad + 4 * c);
        a0 += v.x;
        a1 += v.y;
        a2 += v.z;
        a3 += v.w;
    }
    G1[idx] = make_double2(a0, a1);
    G2[idx] = make_double2(a2, a3);
}

}  // namespace

// ================================================================== host side
// cuTensorMapEncodeTiled from the CUDA driver, looked up once (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int tc_defl_layout(int V, int k, int* Mpad, int* Kpad) {
    *Mpad = ((k + BM - 1) / BM) * BM;
    *Kpad = ((24 * V + BK - 1) / BK) * BK;
    return 0;
}

void launch_split_bf16(int V, int k, int Mpad, int Kpad, const double* z, float* zhat, void* planes, cudaStream_t s) {
    const size_t n = (size_t)Mpad * Kpad;
    k_split_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((size_t)24 * V, k, Mpad, Kpad, z, zhat,
                                                           reinterpret_cast<__nv_bfloat16*>(planes));
}

// Encode the TMA map of the two planes ([2 Mpad] rows x Kpad BF16, 128-byte swizzle, 64 x 128 boxes).
bool tc_make_map(void* map, const void* planes, int Mpad, int Kpad) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)(2 * Mpad)};
    cuuint64_t strides[1] = {(cuuint64_t)Kpad * 2};
    cuuint32_t box[2] = {BK, BM};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(planes),
                    dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t tc_map_bytes() { return sizeof(CUtensorMap); }

// Split count and partial-buffer size for a launch (grid ~ 2 waves of 152 SMs).
void tc_defl_plan(int V, int k, int nb, int* nsplit, int* kb_per_split, size_t* part_floats) {
    int Mpad, Kpad;
    tc_defl_layout(V, k, &Mpad, &Kpad);
    const int kblocks = Kpad / BK;
    const int tiles = (Mpad / BM) * ((nb + 63) / 64);
    int want = std::max(1, 304 / tiles);
    want = std::min(want, kblocks);
    const int per = (kblocks + want - 1) / want;
    *kb_per_split = per;
    *nsplit = (kblocks + per - 1) / per;
    *part_floats = (size_t)(*nsplit) * Mpad * (size_t)(((nb + 63) / 64) * BN);
}

int tc_defl_launch(const void* map, int V, int k, int nb, const NoiseSpec& ns, float* part, int nsplit,
                   int kb_per_split, double2* G1, double2* G2, int* err, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_defl_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess)
            return 1;
        attr = true;
    }
    int Mpad, Kpad;
    tc_defl_layout(V, k, &Mpad, &Kpad);
    TcArgs p;
    p.V = V;
    p.nb = nb;
    p.Mpad = Mpad;
    p.kblocks = Kpad / BK;
    p.kb_per_split = kb_per_split;
    p.Npad = ((nb + 63) / 64) * BN;
    p.nk.k0 = (uint32_t)(ns.seed & 0xffffffffu);
    p.nk.k1 = (uint32_t)(ns.seed >> 32);
    p.nk.level = ns.level;
    p.nk.j0 = ns.j0;
    p.part = part;
    p.err = err;
    const dim3 grid(Mpad / BM, (nb + 63) / 64, nsplit);
    k_defl_tc<<<grid, 192, SMEM_BYTES, s>>>(*reinterpret_cast<const CUtensorMap*>(map), p);
    const size_t n = (size_t)k * nb;
    k_tc_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(k, nb, Mpad, p.Npad, nsplit, part, G1, G2);
    return 0;
}

}  // namespace mpmc
