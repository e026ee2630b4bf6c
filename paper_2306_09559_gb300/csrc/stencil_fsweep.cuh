// t-sweep form of the issue-lean stencil kernels (stencil_fast.cuh).
//
// k_fast does half the instructions of k_step but then waits on its
// neighbour-row loads: each hop's row must arrive before its arithmetic, and
// the resident warps cannot cover that latency.  Here most rows come from
// shared memory instead, staged ahead of use by TMA:
//  * a CTA owns a 2 x 2 x 2 block of (x, y, z) sites and a tile of TW = 16
//    or 32 right-hand sides and walks a segment [t0, t1) of t;
//  * the block's rows of the planes t0-1 .. t1 stream through a ring of four
//    plane buffers (one 12 x TW box per site, issued two planes ahead);
//  * own row, both t-neighbours and the in-block x/y/z neighbours are read
//    from shared memory; the three neighbours outside the block are read
//    from global memory (L2);
//  * with TW = 16 a warp holds the two x-partners of the block, so only the
//    x-hop loads differ between its halves.
// Arithmetic, links and noise dot as in k_fast.  Every mbarrier wait is
// bounded (a.wait_limit clock cycles from the start of the CTA): on timeout
// the CTA stops issuing copies, waits (bounded) for the copies it issued,
// sets *err and returns.  a.skip_copy (a failure-detection test hook) makes
// the producer leave out one plane copy, so that the consumers' wait for it
// runs out with no copy in flight into that buffer.
#pragma once

#include <cuda.h>

#include "stencil_fast.cuh"
#include "tc.cuh"

namespace mpmc {
namespace fsw {

using fast::add2;
using fast::fma2;
using fast::sub2;
using fast::Row;

constexpr int RING = 4;

template <class S, int TW> __host__ __device__ constexpr int row_bytes() { return 12 * TW * 2 * (int)sizeof(S); }
template <class S, int TW> __host__ __device__ constexpr int plane_bytes() { return 8 * row_bytes<S, TW>(); }
// Links staged with a plane (LSM kernels): the block's own 8 x 4 links (8 x 36 float4), then the
// out-of-block backward links of the x, y and z hops (4 sites each, 9 float4), padded so that
// every ring slot starts on a 128-byte boundary.
constexpr int LINK_OWN = 8 * 36, LINK_XB = LINK_OWN, LINK_YB = LINK_XB + 36, LINK_ZB = LINK_YB + 36;
constexpr int LINK_BYTES = (LINK_ZB + 36) * 16;                  // 6336
constexpr int LINK_SLOT = (LINK_BYTES + 127) / 128 * 128;        // 6400
template <class S, int TW, bool LSM> __host__ __device__ constexpr int slot_bytes() {
    return plane_bytes<S, TW>() + (LSM ? LINK_SLOT : 0);
}
// plane ring + mbarriers + alignment slack
template <class S, int TW, bool LSM> __host__ __device__ constexpr int smem_bytes() {
    return RING * slot_bytes<S, TW, LSM>() + RING * 8 + 128;
}
template <int NB, bool LSM> __host__ __device__ constexpr int tile_width() { return LSM ? 16 : (NB < 32 ? NB : 32); }

struct Geom4 {
    FastArgs a;
    int nblk;   // (lx/2)(ly/2)(lz/2)
    int ts;     // t-segment length
    int nseg;   // t-segments
};

// KIND: 0 step, 1 step + dot, 3 outer, 4 outer + dot (the noise-started step stays on k_fast).
// LSM = false: links read from global memory (L1 / L2); 16 resident warps per SM: 2 CTAs of 256
// threads (TW = 32) or 4 of 128 (TW = 16).
// LSM = true: each ring slot also receives, by bulk copies on the slot's mbarrier, the links the
// plane's hops use, so the only global loads left in the arithmetic are the three out-of-block
// neighbour rows; TW = 16, 3 CTAs of 128 threads per SM.
template <class S, int NB, int KIND, bool LSM>
__global__ void __launch_bounds__(LSM ? 128 : 8 * (NB < 32 ? NB : 32), LSM ? 3 : 64 / (NB < 32 ? NB : 32))
    k_fsweep(const __grid_constant__ CUtensorMap tin, const Geom4 g, int* err) {
    constexpr int TW = tile_width<NB, LSM>();
    constexpr int PB = plane_bytes<S, TW>(), RB = row_bytes<S, TW>();
    constexpr int SB = slot_bytes<S, TW, LSM>();
    constexpr int RS = RB / (int)sizeof(S);   // scalars per staged row
    constexpr bool OUTER = KIND >= 3;
    constexpr bool DOT = KIND == 1 || KIND == 4;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // 128-byte aligned ring (an offset from the shared array keeps shared-space loads)
    uint8_t* smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + RING * SB);
    __shared__ volatile int s_fail;
    __shared__ float4 ctab[4];
    // dot reduction: its own array, or (LSM, where shared memory is short) the first ring slot
    __shared__ double2 red_s[LSM ? 1 : 8][TW];
    double2 (*red)[TW] = LSM ? reinterpret_cast<double2 (*)[TW]>(smem) : red_s;

    const FastArgs& a = g.a;
    const int tid = threadIdx.x;
    const int sib = tid / TW;                  // site in block: bx + 2 by + 4 bz
    const int lane_c = tid % TW;
    const int bx = sib & 1, by = (sib >> 1) & 1, bz = sib >> 2;
    // launch index -> (site block, t-segment): plain (block fastest), or with a block order table,
    // segments fastest and the blocks in the table's order
    // (the right-hand-side tiles of one block and segment are adjacent launches: they share links)
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
    const int col = tile * TW + lane_c;
    const int plane = a.lx * a.ly * a.lz;
    const int x = X0 + bx, y = Y0 + by, z = Z0 + bz;
    const int sxyz = (z * a.ly + y) * a.lx + x;
    // plane-local neighbour offsets (x, y, z) with periodic wrap
    const int sy = a.lx, sz = a.lx * a.ly;
    const int nxf = sxyz + (x + 1 < a.lx ? 1 : 1 - a.lx), nxb = sxyz - (x > 0 ? 1 : 1 - a.lx);
    const int nyf = sxyz + (y + 1 < a.ly ? sy : sy - a.ly * sy), nyb = sxyz - (y > 0 ? sy : sy - a.ly * sy);
    const int nzf = sxyz + (z + 1 < a.lz ? sz : sz - a.lz * sz), nzb = sxyz - (z > 0 ? sz : sz - a.lz * sz);
    const int t0 = seg * g.ts;
    const int t1 = min(t0 + g.ts, a.lt);
    const int nrel = t1 - t0 + 2;              // planes t0-1 .. t1, rel = q - (t0 - 1)

    int issued_hi = -1;                        // thread 0 only
    auto issue = [&](int rel) {
        issued_hi = rel;
        if (rel + 1 == a.skip_copy) return;    // test hook (1-based; 0 = off): this copy is never issued
        const int t = (t0 - 1 + rel + a.lt) % a.lt;
        uint64_t* bar = &full[rel % RING];
        uint8_t* dst = smem + (rel % RING) * SB;
        tc::mbar_expect_tx(bar, (uint32_t)(PB + (LSM ? LINK_BYTES : 0)));
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int s = t * plane + ((Z0 + (w >> 2)) * a.ly + (Y0 + ((w >> 1) & 1))) * a.lx + (X0 + (w & 1));
            tc::tma_load_2d(dst + w * RB, &tin, tile * TW * 2, s * 12, bar);
        }
        if constexpr (LSM) {
            // links of this plane: own (site w at [w][mu][9]: one copy per x-pair of sites), and the
            // backward links of the x, y, z hops whose neighbour lies outside the block
            float4* L = reinterpret_cast<float4*>(dst + PB);
            const float4* Ue = a.Ue;
            const int xm = X0 > 0 ? X0 - 1 : a.lx - 1, ym = Y0 > 0 ? Y0 - 1 : a.ly - 1;
            const int zm = Z0 > 0 ? Z0 - 1 : a.lz - 1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int u = q & 1, v = q >> 1;
                const int s0 = t * plane + ((Z0 + v) * a.ly + (Y0 + u)) * a.lx + X0;
                tc::bulk_load(L + 2 * q * 36, Ue + (size_t)s0 * 36, 2 * 36 * 16, bar);
                const int sx = t * plane + ((Z0 + v) * a.ly + (Y0 + u)) * a.lx + xm;            // (by, bz) = (u, v)
                tc::bulk_load(L + LINK_XB + q * 9, Ue + ((size_t)sx * 4 + 0) * 9, 9 * 16, bar);
                const int sy2 = t * plane + ((Z0 + v) * a.ly + ym) * a.lx + (X0 + u);           // (bx, bz) = (u, v)
                tc::bulk_load(L + LINK_YB + q * 9, Ue + ((size_t)sy2 * 4 + 1) * 9, 9 * 16, bar);
                const int sz2 = t * plane + (zm * a.ly + (Y0 + v)) * a.lx + (X0 + u);           // (bx, by) = (u, v)
                tc::bulk_load(L + LINK_ZB + q * 9, Ue + ((size_t)sz2 * 4 + 2) * 9, 9 * 16, bar);
            }
        }
    };
    if (tid == 0) {
        s_fail = 0;
        for (int b = 0; b < RING; ++b) tc::mbar_init(&full[b], 1);
        tc::fence_mbar_init();
    }
    if (tid < 4) ctab[tid] = fast::z4_conj_entry(tid);
    __syncthreads();
    if (tid == 0)
        for (int rel = 0; rel < RING && rel < nrel; ++rel) issue(rel);

    const float2 al = make_float2(a.alpha[0], a.alpha[1]);
    const float2 mk = make_float2(-a.kappa, -a.kappa);
    const long long deadline = clock64() + a.wait_limit;
    double dre = 0.0, dim = 0.0;
    float fre = 0.f, fim = 0.f;   // FP32 partial of the noise dot, moved to FP64 every 4 planes
    const S* gin = reinterpret_cast<const S*>(a.in);

    bool ok = tc::mbar_wait(&full[0], 0, deadline) && tc::mbar_wait(&full[1], 0, deadline);
    if (!ok) s_fail = 1;
    for (int t = t0; t < t1; ++t) {
        const int rel = t - t0 + 1;
        if (ok) {
            ok = tc::mbar_wait(&full[(rel + 1) % RING], (uint32_t)(((rel + 1) / RING) & 1), deadline);
            if (!ok) s_fail = 1;
        }
        if (ok) {
            const S* P0 = reinterpret_cast<const S*>(smem + (rel % RING) * SB) + lane_c * 2;
            const S* Pm = reinterpret_cast<const S*>(smem + ((rel - 1) % RING) * SB) + lane_c * 2;
            const S* Pp = reinterpret_cast<const S*>(smem + ((rel + 1) % RING) * SB) + lane_c * 2;
            auto srow = [&](const S* P, int w, float2 (&p)[12]) {
#pragma unroll
                for (int e = 0; e < 12; ++e) p[e] = Row<S>::ld_rw(P + w * RS + e * TW * 2);
            };
            auto grow = [&](int site, float2 (&p)[12]) {
                const S* q = gin + ((size_t)site * 12 * NB + col) * 2;
#pragma unroll
                for (int e = 0; e < 12; ++e) p[e] = Row<S>::ld(q + (size_t)e * NB * 2);
            };
            const int tp = t * plane;
            const int site = tp + sxyz;
            const bool af = a.bc_t < 0 && t + 1 == a.lt, ab = a.bc_t < 0 && t == 0;
            const int tb = t > 0 ? site - plane : site - plane + a.lt * plane;
            // the link of each hop: forward hops use the site's own links, backward hops those of
            // the neighbour; staged in the ring slots (LSM) or read from global memory
            const float4* U = a.Ue;
            const float4 *Lxf, *Lxb, *Lyf, *Lyb, *Lzf, *Lzb, *Ltf, *Ltb;
            if constexpr (LSM) {
                const float4* Lc = reinterpret_cast<const float4*>(smem + (rel % RING) * SB + PB);
                const float4* Lm = reinterpret_cast<const float4*>(smem + ((rel - 1) % RING) * SB + PB);
                Lxf = Lc + (sib * 4 + 0) * 9;
                Lxb = bx ? Lc + ((sib - 1) * 4 + 0) * 9 : Lc + LINK_XB + (by + 2 * bz) * 9;
                Lyf = Lc + (sib * 4 + 1) * 9;
                Lyb = by ? Lc + ((sib - 2) * 4 + 1) * 9 : Lc + LINK_YB + (bx + 2 * bz) * 9;
                Lzf = Lc + (sib * 4 + 2) * 9;
                Lzb = bz ? Lc + ((sib - 4) * 4 + 2) * 9 : Lc + LINK_ZB + (bx + 2 * by) * 9;
                Ltf = Lc + (sib * 4 + 3) * 9;
                Ltb = Lm + (sib * 4 + 3) * 9;
            } else {
                Lxf = U + ((size_t)site * 4 + 0) * 9;
                Lxb = U + ((size_t)(tp + nxb) * 4 + 0) * 9;
                Lyf = U + ((size_t)site * 4 + 1) * 9;
                Lyb = U + ((size_t)(tp + nyb) * 4 + 1) * 9;
                Lzf = U + ((size_t)site * 4 + 2) * 9;
                Lzb = U + ((size_t)(tp + nzb) * 4 + 2) * 9;
                Ltf = U + ((size_t)site * 4 + 3) * 9;
                Ltb = U + ((size_t)tb * 4 + 3) * 9;
            }
            float2 up[6], lr[6], lj[6], p[12];
#pragma unroll
            for (int i = 0; i < 6; ++i) up[i] = lr[i] = lj[i] = make_float2(0.f, 0.f);
            if constexpr (LSM) {
                // the three out-of-block neighbour rows are the only global loads left: issue them
                // all first and start with the two t-hops from shared memory, so that their L2
                // latency overlaps arithmetic (the register budget of 3 CTAs per SM allows it)
                float2 gx[12], gy[12], gz[12];
                grow(tp + (bx ? nxf : nxb), gx);
                grow(tp + (by ? nyf : nyb), gy);
                grow(tp + (bz ? nzf : nzb), gz);
                srow(Pp, sib, p);
                fast::hop_p<3, true, LSM>(p, Ltf, -1.f, af, up, lr, lj);
                srow(Pm, sib, p);
                fast::hop_p<3, false, LSM>(p, Ltb, -1.f, ab, up, lr, lj);
                if (bx == 0) srow(P0, sib + 1, p);
                fast::hop_p<0, true, LSM>(bx == 0 ? p : gx, Lxf, 1.f, false, up, lr, lj);
                if (bx == 1) srow(P0, sib - 1, p);
                fast::hop_p<0, false, LSM>(bx == 1 ? p : gx, Lxb, 1.f, false, up, lr, lj);
                if (by == 0) srow(P0, sib + 2, p);
                fast::hop_p<1, true, LSM>(by == 0 ? p : gy, Lyf, 1.f, false, up, lr, lj);
                if (by == 1) srow(P0, sib - 2, p);
                fast::hop_p<1, false, LSM>(by == 1 ? p : gy, Lyb, 1.f, false, up, lr, lj);
                if (bz == 0) srow(P0, sib + 4, p);
                fast::hop_p<2, true, LSM>(bz == 0 ? p : gz, Lzf, 1.f, false, up, lr, lj);
                if (bz == 1) srow(P0, sib - 4, p);
                fast::hop_p<2, false, LSM>(bz == 1 ? p : gz, Lzb, 1.f, false, up, lr, lj);
            } else {
                if (bx == 0) srow(P0, sib + 1, p); else grow(tp + nxf, p);
                fast::hop_p<0, true, LSM>(p, Lxf, 1.f, false, up, lr, lj);
                if (bx == 1) srow(P0, sib - 1, p); else grow(tp + nxb, p);
                fast::hop_p<0, false, LSM>(p, Lxb, 1.f, false, up, lr, lj);
                if (by == 0) srow(P0, sib + 2, p); else grow(tp + nyf, p);
                fast::hop_p<1, true, LSM>(p, Lyf, 1.f, false, up, lr, lj);
                if (by == 1) srow(P0, sib - 2, p); else grow(tp + nyb, p);
                fast::hop_p<1, false, LSM>(p, Lyb, 1.f, false, up, lr, lj);
                if (bz == 0) srow(P0, sib + 4, p); else grow(tp + nzf, p);
                fast::hop_p<2, true, LSM>(p, Lzf, 1.f, false, up, lr, lj);
                if (bz == 1) srow(P0, sib - 4, p); else grow(tp + nzb, p);
                fast::hop_p<2, false, LSM>(p, Lzb, 1.f, false, up, lr, lj);
                srow(Pp, sib, p);
                fast::hop_p<3, true, LSM>(p, Ltf, -1.f, af, up, lr, lj);
                srow(Pm, sib, p);
                fast::hop_p<3, false, LSM>(p, Ltb, -1.f, ab, up, lr, lj);
            }
            srow(P0, sib, p);   // own row

            const size_t off = ((size_t)site * 12 * NB + col) * 2;
            const uint32_t hsr = sr_seed(a.salt, (uint32_t)site, (uint32_t)col);
            uint32_t word = 0;
            if (DOT) word = __ldg(a.words + (size_t)site * NB + col);
            float2 dA = make_float2(0.f, 0.f), dB = make_float2(0.f, 0.f);
#pragma unroll
            for (int e = 0; e < 12; ++e) {
                const float2 hw = e < 6 ? up[e] : make_float2(lr[e - 6].x - lj[e - 6].y, lr[e - 6].y + lj[e - 6].x);
                const float2 own = p[e];
                const float2 tt = fma2(mk, hw, own);
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
        __syncthreads();   // plane rel-1 is free: it takes plane rel+3
        if (tid == 0 && !s_fail && rel + 3 < nrel) issue(rel + 3);
    }
    if (tid == 0 && s_fail) {
        // wait (bounded) for the last copy issued into each buffer before the CTA exits; copies into
        // one buffer complete its phases in order, so the last one issued covers the earlier ones
        const long long d2 = clock64() + a.wait_limit;
        for (int b = 0; b < RING; ++b) {
            int last = -1;
            for (int r = b; r <= issued_hi; r += RING)
                if (r + 1 != a.skip_copy) last = r;
            if (last >= 0) tc::mbar_wait(&full[b], (uint32_t)((last / RING) & 1), d2);
        }
        atomicExch(err, 1);
    }
    if (DOT) {
        // fixed-order reduction over the 8 sites of the block, one update of this CTA's row
        if constexpr (LSM) __syncthreads();   // red overlays ring slot 0: every read of the ring is done
        red[sib][lane_c] = make_double2(dre + (double)fre, dim + (double)fim);
        __syncthreads();
        if (sib == 0 && !s_fail) {
            double sr = 0.0, si = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                sr += red[w][lane_c].x;
                si += red[w][lane_c].y;
            }
            double2* pa = a.acc + (size_t)row * NB + col;
            double2 cur = *pa;
            cur.x += a.dot_w[0] * sr - a.dot_w[1] * si;
            cur.y += a.dot_w[0] * si + a.dot_w[1] * sr;
            *pa = cur;
        }
    }
}

}  // namespace fsw
}  // namespace mpmc
