// Warp-per-site form of the t-sweep kernel (k_fsweep_w) and the launch templates of every t-sweep
// form; the ring layout constants and the links-staged form k_fsweep are in stencil_fsweep.cuh.
#pragma once

#include "stencil_fsweep.cuh"

namespace mpmc {
namespace fsw {

// ---------------------------------------------------------------------------------------------
// Warp-per-site form (k_fsweep_w): TW = 32 right-hand sides, 256 threads, warp w owns site w of
// the 2 x 2 x 2 block, so which of a site's x / y / z neighbours lie outside the block is the
// same for all lanes of a warp and the hops need no per-lane selects.  Ring of three plane
// slots (spinor rows + the plane's links), two CTAs (16 warps) per SM at 128 registers.
// No CTA-wide barrier per plane: each warp counts itself out of the slot it no longer needs and
// the last of the eight issues the next plane's copies into it, so warps drift by up to a plane.
// Hop order: the out-of-block rows come from global memory (L2) ahead of use: x during the
// previous plane, y before the backward t-hop, z before the y hops; the forward t-hop, whose
// plane is the one most recently issued, comes last.
constexpr int WRING = 3;
constexpr int WTW = 32;
template <class S> __host__ __device__ constexpr int wslot_bytes() { return plane_bytes<S, WTW>() + LINK_SLOT; }
template <class S> __host__ __device__ constexpr int wsmem_bytes() { return WRING * wslot_bytes<S>() + WRING * 8 + 128; }

// One hop onto the 12 accumulators acc (spins 0-1 then 2-3, three colours each), the row given
// component by component by src(e) (a register array or shared-memory loads made where used).
// Projection, link product and reconstruction as hop_p (stencil_fast.cuh), with the lower spins
// accumulated directly: i g adds (-g.y, g.x).
template <int MU, bool FWD, class Src>
__device__ __forceinline__ void hop_w(const Src& src, const float4* __restrict__ L, float sgn, bool use_sgn,
                                      float2 (&acc)[12]) {
    float2 g0[3], g1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 p0 = src(c), p1 = src(3 + c), p2 = src(6 + c), p3 = src(9 + c);
        float2 a, b;
        if (MU == 0) {
            if (FWD) { a = make_float2(p0.x + p3.y, p0.y - p3.x); b = make_float2(p1.x + p2.y, p1.y - p2.x); }
            else     { a = make_float2(p0.x - p3.y, p0.y + p3.x); b = make_float2(p1.x - p2.y, p1.y + p2.x); }
        } else if (MU == 1) {
            if (FWD) { a = add2(p0, p3); b = sub2(p1, p2); }
            else     { a = sub2(p0, p3); b = add2(p1, p2); }
        } else if (MU == 2) {
            if (FWD) { a = make_float2(p0.x + p2.y, p0.y - p2.x); b = make_float2(p1.x - p3.y, p1.y + p3.x); }
            else     { a = make_float2(p0.x - p2.y, p0.y + p2.x); b = make_float2(p1.x + p3.y, p1.y - p3.x); }
        } else {
            if (FWD) { a = sub2(p0, p2); b = sub2(p1, p3); }
            else     { a = add2(p0, p2); b = add2(p1, p3); }
        }
        if (use_sgn) {
            a = __fmul2_rn(a, make_float2(sgn, sgn));
            b = __fmul2_rn(b, make_float2(sgn, sgn));
        }
        const float2 ia = FWD ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
        const float2 ib = FWD ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float4 u = *(L + (FWD ? 3 * r + c : 3 * c + r));
            const float2 ur = make_float2(u.x, u.y), ui = make_float2(u.z, u.w);
            if (c == 0) {
                g0[r] = fma2(ui, ia, __fmul2_rn(ur, a));
                g1[r] = fma2(ui, ib, __fmul2_rn(ur, b));
            } else {
                g0[r] = fma2(ui, ia, fma2(ur, a, g0[r]));
                g1[r] = fma2(ui, ib, fma2(ur, b, g1[r]));
            }
        }
    }
    auto addi = [](float2 x, float2 g) { return make_float2(x.x - g.y, x.y + g.x); };   // x + i g
    auto subi = [](float2 x, float2 g) { return make_float2(x.x + g.y, x.y - g.x); };   // x - i g
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        acc[r] = add2(acc[r], g0[r]);
        acc[3 + r] = add2(acc[3 + r], g1[r]);
        float2 &l0 = acc[6 + r], &l1 = acc[9 + r];
        if (MU == 0) {
            if (FWD) { l0 = addi(l0, g1[r]); l1 = addi(l1, g0[r]); }
            else     { l0 = subi(l0, g1[r]); l1 = subi(l1, g0[r]); }
        } else if (MU == 1) {
            if (FWD) { l0 = sub2(l0, g1[r]); l1 = add2(l1, g0[r]); }
            else     { l0 = add2(l0, g1[r]); l1 = sub2(l1, g0[r]); }
        } else if (MU == 2) {
            if (FWD) { l0 = addi(l0, g0[r]); l1 = subi(l1, g1[r]); }
            else     { l0 = subi(l0, g0[r]); l1 = addi(l1, g1[r]); }
        } else {
            if (FWD) { l0 = sub2(l0, g0[r]); l1 = sub2(l1, g1[r]); }
            else     { l0 = add2(l0, g0[r]); l1 = add2(l1, g1[r]); }
        }
    }
}

// KIND as k_fsweep (0 step, 1 step + dot, 3 outer, 4 outer + dot); NB >= 32.
template <class S, int NB, int KIND>
__global__ void __launch_bounds__(256, 2) k_fsweep_w(const __grid_constant__ CUtensorMap tin, const Geom4 g, int* err) {
    constexpr int TW = WTW;
    constexpr int PB = plane_bytes<S, TW>(), RB = row_bytes<S, TW>();
    constexpr int SB = wslot_bytes<S>();
    constexpr int RS = RB / (int)sizeof(S);
    constexpr bool OUTER = KIND >= 3;
    constexpr bool DOT = KIND == 1 || KIND == 4;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + WRING * SB);
    __shared__ int s_out[WRING];      // warps counted out of each slot (monotone; 8 per use)
    __shared__ volatile int s_fail;
    __shared__ volatile int s_issued; // highest plane index whose copies were issued
    __shared__ float4 ctab[4];
    double2 (*red)[TW] = reinterpret_cast<double2 (*)[TW]>(smem);   // dot reduction, over slot 0 at the end

    const FastArgs& a = g.a;
    const int tid = threadIdx.x;
    const int sib = tid >> 5;                  // site in block (warp): bx + 2 by + 4 bz
    const int lane = tid & 31;
    const int bx = sib & 1, by = (sib >> 1) & 1, bz = sib >> 2;
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
    const int col = tile * TW + lane;
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
        uint64_t* bar = &full[rel % WRING];
        uint8_t* dst = smem + (rel % WRING) * SB;
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
        for (int b = 0; b < WRING; ++b) {
            tc::mbar_init(&full[b], 1);
            s_out[b] = 0;
        }
        tc::fence_mbar_init();
    }
    if (tid < 4) ctab[tid] = fast::z4_conj_entry(tid);
    __syncthreads();
    if (tid == 0)
        for (int rel = 0; rel < WRING && rel < nrel; ++rel) issue(rel);

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
            const uint8_t* C = smem + (rel % WRING) * SB;
            const uint8_t* M = smem + ((rel - 1) % WRING) * SB;
            const uint8_t* N = smem + ((rel + 1) % WRING) * SB;
            const S* P0 = reinterpret_cast<const S*>(C) + sib * RS + lane * 2;   // own row
            auto srow = [&](const uint8_t* slot, int w) {
                const S* P = reinterpret_cast<const S*>(slot) + w * RS + lane * 2;
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
            grow(tp + oy, H);
            hop_w<3, false>(srow(M, sib), Ltb, -1.f, ab, acc);
            // x: out-of-block row (registers) and the in-block partner (shared memory); warp-uniform
            if (bx) { hop_w<0, true>(reg(G), Lxf, 1.f, false, acc); hop_w<0, false>(srow(C, sib - 1), Lxb, 1.f, false, acc); }
            else    { hop_w<0, false>(reg(G), Lxb, 1.f, false, acc); hop_w<0, true>(srow(C, sib + 1), Lxf, 1.f, false, acc); }
            grow(tp + oz, G);
            if (by) { hop_w<1, true>(reg(H), Lyf, 1.f, false, acc); hop_w<1, false>(srow(C, sib - 2), Lyb, 1.f, false, acc); }
            else    { hop_w<1, false>(reg(H), Lyb, 1.f, false, acc); hop_w<1, true>(srow(C, sib + 2), Lyf, 1.f, false, acc); }
            // z, then the next plane's x row into G, ahead of the in-block z hop, the t-hop and the stores
            if (bz) hop_w<2, true>(reg(G), Lzf, 1.f, false, acc);
            else    hop_w<2, false>(reg(G), Lzb, 1.f, false, acc);
            if (t + 1 < t1) grow(tp + plane + ox, G);
            if (bz) hop_w<2, false>(srow(C, sib - 4), Lzb, 1.f, false, acc);
            else    hop_w<2, true>(srow(C, sib + 4), Lzf, 1.f, false, acc);
            ok = tc::mbar_wait(&full[(rel + 1) % WRING], (uint32_t)(((rel + 1) / WRING) & 1), deadline);
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
        // this warp is done with plane rel-1; the last of the eight warps reuses its slot for rel+2
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int before = atomicAdd(&s_out[(rel - 1) % WRING], 1);
            if ((before & 7) == 7) {
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
        for (int b = 0; b < WRING; ++b) {
            int last = -1;
            for (int r = b; r <= hi; r += WRING)
                if (r + 1 != a.skip_copy) last = r;
            if (last >= 0) tc::mbar_wait(&full[b], (uint32_t)((last / WRING) & 1), d2);
        }
        atomicExch(err, 1);
    }
    if (DOT) {
        __syncthreads();   // red overlays ring slot 0: no copy into it is pending
        red[sib][lane] = make_double2(dre + (double)fre, dim + (double)fim);
        __syncthreads();
        if (sib == 0 && !s_fail) {
            double sr = 0.0, si = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                sr += red[w][lane].x;
                si += red[w][lane].y;
            }
            double2* pa = a.acc + (size_t)row * NB + col;
            double2 cur = *pa;
            cur.x += a.dot_w[0] * sr - a.dot_w[1] * si;
            cur.y += a.dot_w[0] * si + a.dot_w[1] * sr;
            *pa = cur;
        }
    }
}

// Launch of one instantiation: VAR 0 / 1 run k_fsweep (links from global memory / staged), VAR 2
// k_fsweep_w.  The dynamic shared-memory attribute is set once per instantiation.
template <class S, int NB, int KIND, int VAR>
int launch_one(const CUtensorMap& map, const Geom4& g, int gx, int* err, cudaStream_t s) {
    constexpr bool W = VAR == 2;
    static_assert(!W || NB >= 32, "the warp-per-site form needs tiles of 32 columns");
    constexpr int TW = W ? WTW : tile_width<NB, VAR == 1>();
    void (*kern)(const CUtensorMap, const Geom4, int*);
    if constexpr (W) kern = k_fsweep_w<S, NB, KIND>;
    else kern = k_fsweep<S, NB, KIND, VAR == 1>;
    constexpr int smem = W ? wsmem_bytes<S>() : smem_bytes<S, TW, VAR == 1>();
    constexpr int threads = W ? 256 : 8 * TW;
    static bool attr = false;   // one flag per instantiation
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
        attr = true;
    }
    kern<<<dim3(gx * (NB / TW)), threads, smem, s>>>(map, g, err);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <class S, int NB, int VAR>
int launch_nb(int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s) {
    switch (kind) {
        case 0: return launch_one<S, NB, 0, VAR>(m, g, gx, err, s);
        case 1: return launch_one<S, NB, 1, VAR>(m, g, gx, err, s);
        case 3: return launch_one<S, NB, 3, VAR>(m, g, gx, err, s);
        case 4: return launch_one<S, NB, 4, VAR>(m, g, gx, err, s);
        default: return 1;
    }
}

template <class S, int VAR>
int launch_s(int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s) {
    if constexpr (VAR != 2)
        if (nb == 16) return launch_nb<S, 16, VAR>(kind, m, g, gx, err, s);
    switch (nb) {
        case 32: return launch_nb<S, 32, VAR>(kind, m, g, gx, err, s);
        case 64: return launch_nb<S, 64, VAR>(kind, m, g, gx, err, s);
        case 128: return launch_nb<S, 128, VAR>(kind, m, g, gx, err, s);
        case 256: return launch_nb<S, 256, VAR>(kind, m, g, gx, err, s);
        case 512: return launch_nb<S, 512, VAR>(kind, m, g, gx, err, s);
        case 1024: return launch_nb<S, 1024, VAR>(kind, m, g, gx, err, s);
        default: return 1;
    }
}

// one function per translation unit (stencil_fsweep_*.cu); var 0 or 1 for launch_f32 / launch_bf16
int launch_f32(int var, int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s);
int launch_bf16(int var, int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s);
int launch_w_f32(int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s);
int launch_w_bf16(int nb, int kind, const CUtensorMap& m, const Geom4& g, int gx, int* err, cudaStream_t s);

}  // namespace fsw
}  // namespace mpmc
