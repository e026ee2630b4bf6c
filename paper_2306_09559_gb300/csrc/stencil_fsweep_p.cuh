// Two-sites-per-warp form of the t-sweep kernel (k_fsweep_p) and its launches.
//
// As k_fsweep_w (stencil_fsweep_w.cuh: ring of three plane slots with the plane's links, per-warp
// release of the slots, out-of-block rows loaded ahead, hops summed into the 12 outputs), but a
// tile of 16 right-hand sides and 4 warps per CTA, each warp holding the two x-sites of the block
// that share (y, z), one per half-warp.  A 16-byte shared-memory load costs two wavefronts whether
// one address or one address per half-warp is read, so each link element reaches two sites for
// the price k_fsweep_w pays for one.  The price: the x hops' direction differs between the
// half-warps (selects between the out-of-block row and the in-block partner's row).  Four CTAs
// (16 warps) per SM at 128 registers.
#pragma once

#include "stencil_fsweep_w.cuh"

namespace mpmc {
namespace fsw {

constexpr int PRING = 3;
constexpr int PTW = 16;
template <class S> __host__ __device__ constexpr int pslot_bytes() { return plane_bytes<S, PTW>() + LINK_SLOT; }
template <class S> __host__ __device__ constexpr int psmem_bytes() { return PRING * pslot_bytes<S>() + PRING * 8 + 128; }

// KIND as k_fsweep (0 step, 1 step + dot, 3 outer, 4 outer + dot); NB >= 16.
template <class S, int NB, int KIND>
__global__ void __launch_bounds__(128, 4) k_fsweep_p(const __grid_constant__ CUtensorMap tin, const Geom4 g, int* err) {
    constexpr int TW = PTW;
    constexpr int PB = plane_bytes<S, TW>(), RB = row_bytes<S, TW>();
    constexpr int SB = pslot_bytes<S>();
    constexpr int RS = RB / (int)sizeof(S);
    constexpr bool OUTER = KIND >= 3;
    constexpr bool DOT = KIND == 1 || KIND == 4;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + PRING * SB);
    __shared__ int s_out[PRING];      // warps counted out of each slot (monotone; 4 per use)
    __shared__ volatile int s_fail;
    __shared__ volatile int s_issued; // highest plane index whose copies were issued
    __shared__ float4 ctab[4];
    double2 (*red)[TW] = reinterpret_cast<double2 (*)[TW]>(smem);   // dot reduction [site][column], over slot 0

    const FastArgs& a = g.a;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int bx = lane >> 4, by = warp & 1, bz = warp >> 1;   // x differs between the half-warps
    const int sib = bx + 2 * by + 4 * bz;      // site in block
    const int lc = lane & 15;                  // column in the tile
    const int tile = blockIdx.x % (NB / TW), row = blockIdx.x / (NB / TW);
    int blk, seg;
    if (a.blk_order) {
        seg = row % g.nseg;
        blk = __ldg(a.blk_order + row / g.nseg);
    } else {
        blk = row % g.nblk;
        seg = row / g.nblk;
    }
    const int hx = a.lx >> 1, hy = a.ly >> 1;
    const int X0 = 2 * (blk % hx), Y0 = 2 * ((blk / hx) % hy), Z0 = 2 * (blk / (hx * hy));
    const int col = tile * TW + lc;
    const int plane = a.lx * a.ly * a.lz;
    const int x = X0 + bx, y = Y0 + by, z = Z0 + bz;
    const int sxyz = (z * a.ly + y) * a.lx + x;
    const int sy = a.lx, sz = a.lx * a.ly;
    // the out-of-block neighbour of each of x, y, z (forward when the site is on the block's upper face)
    const int ox = bx ? sxyz + (x + 1 < a.lx ? 1 : 1 - a.lx) : sxyz - (x > 0 ? 1 : 1 - a.lx);
    const int oy = by ? sxyz + (y + 1 < a.ly ? sy : sy - a.ly * sy) : sxyz - (y > 0 ? sy : sy - a.ly * sy);
    const int oz = bz ? sxyz + (z + 1 < a.lz ? sz : sz - a.lz * sz) : sxyz - (z > 0 ? sz : sz - a.lz * sz);
    const int t0 = seg * g.ts;
    const int t1 = min(t0 + g.ts, a.lt);
    const int nrel = t1 - t0 + 2;              // planes t0-1 .. t1, rel = q - (t0 - 1)

    auto issue = [&](int rel) {                // one thread
        s_issued = rel;
        if (rel + 1 == a.skip_copy) return;    // test hook (1-based; 0 = off): this copy is never issued
        const int t = (t0 - 1 + rel + a.lt) % a.lt;
        uint64_t* bar = &full[rel % PRING];
        uint8_t* dst = smem + (rel % PRING) * SB;
        tc::mbar_expect_tx(bar, (uint32_t)(PB + LINK_BYTES));
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int s = t * plane + ((Z0 + (w >> 2)) * a.ly + (Y0 + ((w >> 1) & 1))) * a.lx + (X0 + (w & 1));
            tc::tma_load_2d(dst + w * RB, &tin, tile * TW * 2, s * 12, bar);
        }
        float4* L = reinterpret_cast<float4*>(dst + PB);
        const float4* Ue = a.Ue;
        const int xm = X0 > 0 ? X0 - 1 : a.lx - 1, ym = Y0 > 0 ? Y0 - 1 : a.ly - 1;
        const int zm = Z0 > 0 ? Z0 - 1 : a.lz - 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = q & 1, v = q >> 1;
            const int s0 = t * plane + ((Z0 + v) * a.ly + (Y0 + u)) * a.lx + X0;
            tc::bulk_load(L + 2 * q * 36, Ue + (size_t)s0 * 36, 2 * 36 * 16, bar);
            const int sx = t * plane + ((Z0 + v) * a.ly + (Y0 + u)) * a.lx + xm;
            tc::bulk_load(L + LINK_XB + q * 9, Ue + ((size_t)sx * 4 + 0) * 9, 9 * 16, bar);
            const int sy2 = t * plane + ((Z0 + v) * a.ly + ym) * a.lx + (X0 + u);
            tc::bulk_load(L + LINK_YB + q * 9, Ue + ((size_t)sy2 * 4 + 1) * 9, 9 * 16, bar);
            const int sz2 = t * plane + (zm * a.ly + (Y0 + v)) * a.lx + (X0 + u);
            tc::bulk_load(L + LINK_ZB + q * 9, Ue + ((size_t)sz2 * 4 + 2) * 9, 9 * 16, bar);
        }
    };
    if (tid == 0) {
        s_fail = 0;
        s_issued = -1;
        for (int b = 0; b < PRING; ++b) {
            tc::mbar_init(&full[b], 1);
            s_out[b] = 0;
        }
        tc::fence_mbar_init();
    }
    if (tid < 4) ctab[tid] = fast::z4_conj_entry(tid);
    __syncthreads();
    if (tid == 0)
        for (int rel = 0; rel < PRING && rel < nrel; ++rel) issue(rel);

    const float2 al = make_float2(a.alpha[0], a.alpha[1]);
    const float2 mk = make_float2(-a.kappa, -a.kappa);
    const long long deadline = clock64() + a.wait_limit;
    double dre = 0.0, dim = 0.0;
    float fre = 0.f, fim = 0.f;   // FP32 partial of the noise dot, moved to FP64 every 4 planes
    const S* gin = reinterpret_cast<const S*>(a.in);
    auto grow = [&](int site, float2 (&p)[12]) {
        const S* q = gin + ((size_t)site * 12 * NB + col) * 2;
#pragma unroll
        for (int e = 0; e < 12; ++e) p[e] = Row<S>::ld(q + (size_t)e * NB * 2);
    };

    float2 G[12];                              // out-of-block rows, one plane ahead for x
    grow(t0 * plane + ox, G);
    bool ok = tc::mbar_wait(&full[0], 0, deadline) && tc::mbar_wait(&full[1], 0, deadline);
    if (!ok) s_fail = 1;
    for (int t = t0; t < t1; ++t) {
        const int rel = t - t0 + 1;
        if (ok && s_fail) ok = false;          // another warp gave up: no new plane is coming
        if (ok) {
            const uint8_t* C = smem + (rel % PRING) * SB;
            const uint8_t* M = smem + ((rel - 1) % PRING) * SB;
            const uint8_t* N = smem + ((rel + 1) % PRING) * SB;
            const S* P0 = reinterpret_cast<const S*>(C) + sib * RS + lc * 2;   // own row
            auto srow = [&](const uint8_t* slot, int w) {
                const S* P = reinterpret_cast<const S*>(slot) + w * RS + lc * 2;
                return [P](int e) { return Row<S>::ld_rw(P + e * TW * 2); };
            };
            const int tp = t * plane;
            const int site = tp + sxyz;
            const bool af = a.bc_t < 0 && t + 1 == a.lt, ab = a.bc_t < 0 && t == 0;
            const float4* Lc = reinterpret_cast<const float4*>(C + PB);
            const float4* Lm = reinterpret_cast<const float4*>(M + PB);
            const float4* Lxf = Lc + (sib * 4 + 0) * 9;
            const float4* Lxb = bx ? Lc + ((sib - 1) * 4 + 0) * 9 : Lc + LINK_XB + (by + 2 * bz) * 9;
            const float4* Lyf = Lc + (sib * 4 + 1) * 9;
            const float4* Lyb = by ? Lc + ((sib - 2) * 4 + 1) * 9 : Lc + LINK_YB + (bx + 2 * bz) * 9;
            const float4* Lzf = Lc + (sib * 4 + 2) * 9;
            const float4* Lzb = bz ? Lc + ((sib - 4) * 4 + 2) * 9 : Lc + LINK_ZB + (bx + 2 * by) * 9;
            const float4* Ltf = Lc + (sib * 4 + 3) * 9;
            const float4* Ltb = Lm + (sib * 4 + 3) * 9;

            float2 acc[12], H[12];
#pragma unroll
            for (int e = 0; e < 12; ++e) acc[e] = make_float2(0.f, 0.f);
            auto reg = [](const float2 (&r)[12]) { return [&r](int e) { return r[e]; }; };
            // G holds this plane's out-of-block x row (loaded during the previous plane)
            hop_w<3, false>(srow(M, sib), Ltb, -1.f, ab, acc);
            {
                // x: the half-warps are the block's two x-sites, so the out-of-block neighbour in G
                // is the forward one for bx = 1 and the backward one for bx = 0, and the in-block
                // partner (site sib ^ 1) is the other; G and R become the forward and backward rows
                float2 R[12];
                const S* Pq = reinterpret_cast<const S*>(C) + (sib ^ 1) * RS + lc * 2;
#pragma unroll
                for (int e = 0; e < 12; ++e) {
                    const float2 q = Row<S>::ld_rw(Pq + e * TW * 2);
                    const float2 f = bx ? G[e] : q;
                    R[e] = bx ? q : G[e];
                    G[e] = f;
                }
                hop_w<0, true>(reg(G), Lxf, 1.f, false, acc);
                hop_w<0, false>(reg(R), Lxb, 1.f, false, acc);
            }
            // y and z (uniform per warp): the out-of-block rows load while the in-block hops run
            grow(tp + oy, H);
            grow(tp + oz, G);
            if (by) hop_w<1, false>(srow(C, sib - 2), Lyb, 1.f, false, acc);
            else    hop_w<1, true>(srow(C, sib + 2), Lyf, 1.f, false, acc);
            if (bz) hop_w<2, false>(srow(C, sib - 4), Lzb, 1.f, false, acc);
            else    hop_w<2, true>(srow(C, sib + 4), Lzf, 1.f, false, acc);
            if (by) hop_w<1, true>(reg(H), Lyf, 1.f, false, acc);
            else    hop_w<1, false>(reg(H), Lyb, 1.f, false, acc);
            if (bz) hop_w<2, true>(reg(G), Lzf, 1.f, false, acc);
            else    hop_w<2, false>(reg(G), Lzb, 1.f, false, acc);
            if (t + 1 < t1) grow(tp + plane + ox, G);   // the next plane's x row, ahead of the t-hop and stores
            ok = tc::mbar_wait(&full[(rel + 1) % PRING], (uint32_t)(((rel + 1) / PRING) & 1), deadline);
            if (!ok) {
                s_fail = 1;
            } else {
                hop_w<3, true>(srow(N, sib), Ltf, -1.f, af, acc);

                const size_t off = ((size_t)site * 12 * NB + col) * 2;
                const uint32_t hsr = sr_seed(a.salt, (uint32_t)site, (uint32_t)col);
                uint32_t word = 0;
                if (DOT) word = __ldg(a.words + (size_t)site * NB + col);
                float2 dA = make_float2(0.f, 0.f), dB = make_float2(0.f, 0.f);
#pragma unroll
                for (int e = 0; e < 12; ++e) {
                    const float2 own = Row<S>::ld_rw(P0 + e * TW * 2);
                    const float2 tt = fma2(mk, acc[e], own);
                    float2 v;
                    if (!OUTER) {
                        v = fast::minus_alpha2(own, al, tt);
                        Row<S>::st_sr(reinterpret_cast<S*>(a.out) + off + (size_t)e * NB * 2, v, sr_bits(hsr, e));
                    } else {
                        const float2 pa = fast::minus_alpha2(own, al, tt);
                        const size_t oe = off + (size_t)e * NB * 2;
                        const float2 wv = Row<S>::ld_rw(reinterpret_cast<const S*>(a.w) + oe);
                        float2 yv = Row<S>::ld_rw(reinterpret_cast<const S*>(a.y) + oe);
                        const float2 wn = fast::minus_alpha2(wv, make_float2(a.beta[0], a.beta[1]), sub2(wv, pa));
                        yv = fast::cmac2(yv, make_float2(a.gamma[0], a.gamma[1]), wn);
                        Row<S>::st_sr(reinterpret_cast<S*>(a.out) + oe, wn, sr_bits(hsr, e));
                        Row<S>::st_sr(reinterpret_cast<S*>(a.y) + oe, yv, sr_bits(hsr, 12 + e));
                        v = yv;
                    }
                    if (DOT) {
                        const float4 c = ctab[(word >> (2 * e)) & 3u];
                        dA = fma2(make_float2(c.x, c.y), v, dA);
                        dB = fma2(make_float2(c.z, c.w), v, dB);
                    }
                }
                if (DOT) {
                    fre += dA.x - dB.y;
                    fim += dA.y + dB.x;
                    if (((t - t0) & 3) == 3) {
                        dre += (double)fre;
                        dim += (double)fim;
                        fre = fim = 0.f;
                    }
                }
            }
        }
        // this warp is done with plane rel-1; the last of the four warps reuses its slot for rel+2
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int before = atomicAdd(&s_out[(rel - 1) % PRING], 1);
            if ((before & 3) == 3) {
                __threadfence_block();
                if (!s_fail && rel + 2 < nrel) {
                    tc::fence_proxy_async();
                    issue(rel + 2);
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0 && s_fail) {
        // wait (bounded) for the last copy issued into each slot before the CTA exits
        const long long d2 = clock64() + a.wait_limit;
        const int hi = s_issued;
        for (int b = 0; b < PRING; ++b) {
            int last = -1;
            for (int r = b; r <= hi; r += PRING)
                if (r + 1 != a.skip_copy) last = r;
            if (last >= 0) tc::mbar_wait(&full[b], (uint32_t)((last / PRING) & 1), d2);
        }
        atomicExch(err, 1);
    }
    if (DOT) {
        __syncthreads();   // red overlays ring slot 0: no copy into it is pending
        red[sib][lc] = make_double2(dre + (double)fre, dim + (double)fim);
        __syncthreads();
        if (sib == 0 && !s_fail) {
            double sr = 0.0, si = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                sr += red[w][lc].x;
                si += red[w][lc].y;
            }
            double2* pa = a.acc + (size_t)row * NB + col;
            double2 cur = *pa;
            cur.x += a.dot_w[0] * sr - a.dot_w[1] * si;
            cur.y += a.dot_w[0] * si + a.dot_w[1] * sr;
            *pa = cur;
        }
    }
}


template <class S, int NB, int KIND>
int launch_p_one(const CUtensorMap& map, const Geom4& g, int gx, int* err, cudaStream_t s) {
    constexpr int smem = psmem_bytes<S>();
    auto kern = k_fsweep_p<S, NB, KIND>;
    static bool attr = false;   // one flag per instantiation
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        // four CTAs per SM need the whole shared-memory carveout
        if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess) return 1;
        attr = true;
    }
    kern<<<dim3(gx * (NB / PTW)), 128, smem, s>>>(map, g, err);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <class S, int NB>
int launch_p_nb(int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s) {
    switch (kind) {
        case 0: return launch_p_one<S, NB, 0>(m, g, gx, err, s);
        case 1: return launch_p_one<S, NB, 1>(m, g, gx, err, s);
        case 3: return launch_p_one<S, NB, 3>(m, g, gx, err, s);
        case 4: return launch_p_one<S, NB, 4>(m, g, gx, err, s);
        default: return 1;
    }
}

template <class S>
int launch_p_s(int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s) {
    switch (nb) {
        case 16: return launch_p_nb<S, 16>(kind, m, g, gx, err, s);
        case 32: return launch_p_nb<S, 32>(kind, m, g, gx, err, s);
        case 64: return launch_p_nb<S, 64>(kind, m, g, gx, err, s);
        case 128: return launch_p_nb<S, 128>(kind, m, g, gx, err, s);
        case 256: return launch_p_nb<S, 256>(kind, m, g, gx, err, s);
        case 512: return launch_p_nb<S, 512>(kind, m, g, gx, err, s);
        case 1024: return launch_p_nb<S, 1024>(kind, m, g, gx, err, s);
        default: return 1;
    }
}

// stencil_fsweep_p_f32.cu / stencil_fsweep_p_bf16.cu
int launch_p_f32(int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s);
int launch_p_bf16(int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s);

}  // namespace fsw
}  // namespace mpmc
