// t-sweep form of the fused stencil kernels of stencil.cuh (same per-site
// arithmetic, same hop order, so the stored vectors agree with k_step /
// k_outer up to FMA contraction).
//
// A CTA owns a 2 x 2 x 2 block of (x, y, z) sites and a tile of 32
// right-hand sides, and walks a segment [t0, t1) of the t direction; each of
// its 8 warps computes one site of the block, lane = right-hand side.  The
// block's spinor rows of the planes t0-1 .. t1 stream through a ring of four
// shared-memory plane buffers, filled by TMA tiled loads (one 12 x 32-complex
// box per site, issued two planes ahead).  Own row, both t-neighbours and
// the in-block x/y/z neighbours are read from shared memory; only the three
// neighbours outside the block go through L1/L2, so a step moves about four
// spinor rows per output site through L2 instead of nine.
//
// Every mbarrier wait is bounded: on timeout the CTA stops issuing copies,
// waits (bounded) for the copies it issued, sets *err and skips its stores.
#pragma once

#include <cuda.h>

#include "stencil.cuh"
#include "tc.cuh"

namespace mpmc {

constexpr int SWEEP_TW = 32;      // right-hand sides per tile (one per lane)
constexpr int SWEEP_SITES = 8;    // 2 x 2 x 2 block, one warp per site
constexpr int SWEEP_RING = 4;     // plane buffers
constexpr long long SWEEP_TIMEOUT = 4000000000LL;   // clock64 ticks (about 2 s)

template <class S> __host__ __device__ constexpr int sweep_row_bytes() { return 12 * SWEEP_TW * 2 * (int)sizeof(S); }
template <class S> __host__ __device__ constexpr int sweep_plane_bytes() { return SWEEP_SITES * sweep_row_bytes<S>(); }
// plane ring + mbarriers + alignment slack
template <class S> __host__ __device__ constexpr int sweep_smem_bytes() {
    return SWEEP_RING * sweep_plane_bytes<S>() + SWEEP_RING * 8 + 128;
}

struct SweepGeom {
    Lattice L;
    int nblk;   // (lx/2)(ly/2)(lz/2) site blocks
    int ts;     // t-segment length; blockIdx.x = blk + nblk * segment
};

template <class A> struct IsOuter { static constexpr bool value = false; };
template <> struct IsOuter<OuterArgs> { static constexpr bool value = true; };

template <class S, class A, bool DOT, int YMODE>
__global__ void __launch_bounds__(256, 2) k_sweep(const __grid_constant__ CUtensorMap tin, const A a, SweepGeom sg,
                                                  const typename Math<S>::T* __restrict__ U, int nb, NoiseKey nk,
                                                  int* err) {
    using T = typename Math<S>::T;
    constexpr bool OUTER = IsOuter<A>::value;
    constexpr int PB = sweep_plane_bytes<S>(), RB = sweep_row_bytes<S>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + SWEEP_RING * PB);
    __shared__ volatile int s_fail;
    __shared__ double2 red[SWEEP_SITES][SWEEP_TW];

    const Lattice& L = sg.L;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int blk = blockIdx.x % sg.nblk, seg = blockIdx.x / sg.nblk;
    const int hx = L.lx >> 1, hy = L.ly >> 1;
    const int X0 = 2 * (blk % hx), Y0 = 2 * ((blk / hx) % hy), Z0 = 2 * (blk / (hx * hy));
    const int bx = warp & 1, by = (warp >> 1) & 1, bz = warp >> 2;
    const int col = blockIdx.y * SWEEP_TW + lane;
    const bool colok = col < nb;
    const int plane = L.lx * L.ly * L.lz;
    const int sxyz = ((Z0 + bz) * L.ly + (Y0 + by)) * L.lx + (X0 + bx);
    const int t0 = seg * sg.ts;
    const int t1 = min(t0 + sg.ts, L.lt);
    const int nrel = t1 - t0 + 2;   // planes t0-1 .. t1, index rel = q - (t0 - 1)

    int issued_hi = -1;   // thread 0 only
    auto issue = [&](int rel) {
        const int t = (t0 - 1 + rel + L.lt) % L.lt;
        uint64_t* bar = &full[rel % SWEEP_RING];
        uint8_t* dst = ring + (rel % SWEEP_RING) * PB;
        tc::mbar_expect_tx(bar, (uint32_t)PB);
#pragma unroll
        for (int w = 0; w < SWEEP_SITES; ++w) {
            const int s = t * plane + ((Z0 + (w >> 2)) * L.ly + (Y0 + ((w >> 1) & 1))) * L.lx + (X0 + (w & 1));
            tc::tma_load_2d(dst + w * RB, &tin, blockIdx.y * SWEEP_TW * 2, s * 12, bar);
        }
        issued_hi = rel;
    };
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int b = 0; b < SWEEP_RING; ++b) tc::mbar_init(&full[b], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int rel = 0; rel < SWEEP_RING && rel < nrel; ++rel) issue(rel);

    const cplx<T> cal = Coef<T>::get(a.alpha, a.alphaf);
    const T kap = Coef<T>::real(a.kappa, a.kappaf);
    const long long deadline = clock64() + SWEEP_TIMEOUT;
    double dre = 0.0, dim = 0.0;

    bool ok = tc::mbar_wait(&full[0], 0, deadline) && tc::mbar_wait(&full[1], 0, deadline);
    if (!ok) s_fail = 1;
    for (int t = t0; t < t1; ++t) {
        const int rel = t - t0 + 1;
        if (ok) {
            ok = tc::mbar_wait(&full[(rel + 1) % SWEEP_RING], (uint32_t)(((rel + 1) / SWEEP_RING) & 1), deadline);
            if (!ok) s_fail = 1;
        }
        if (ok && colok) {
            const S* P0 = reinterpret_cast<const S*>(ring + (rel % SWEEP_RING) * PB);
            const S* Pm = reinterpret_cast<const S*>(ring + ((rel - 1) % SWEEP_RING) * PB);
            const S* Pp = reinterpret_cast<const S*>(ring + ((rel + 1) % SWEEP_RING) * PB);
            auto srow = [&](const S* P, int w, cplx<T> (&v)[12][1]) {
                const S* q = P + (size_t)w * (RB / sizeof(S)) + lane * 2;
#pragma unroll
                for (int e = 0; e < 12; ++e) VecIO<S, 1>::ld(q + e * SWEEP_TW * 2, v[e]);
            };
            const MemSrcR<S, 1> gsrc{reinterpret_cast<const S*>(a.in), nb};
            const int site = t * plane + sxyz;
            const Nbrs nbr = neighbours(L, site);
            cplx<T> acc[12][1], psi[12][1], u[9];
#pragma unroll
            for (int e = 0; e < 12; ++e) acc[e][0] = cz<T>();
            const T sf = (nbr.fwd_wrap_t && L.bc_t < 0) ? T(-1) : T(1);
            const T sb = (nbr.bwd_wrap_t && L.bc_t < 0) ? T(-1) : T(1);
            if (bx == 0) srow(P0, warp + 1, psi); else gsrc.get(nbr.fwd[0], col, psi);
            load_link(U, site, 0, u);      hop_r<0, true, false>(psi, u, T(1), acc);
            if (bx == 1) srow(P0, warp - 1, psi); else gsrc.get(nbr.bwd[0], col, psi);
            load_link(U, nbr.bwd[0], 0, u); hop_r<0, false, false>(psi, u, T(1), acc);
            if (by == 0) srow(P0, warp + 2, psi); else gsrc.get(nbr.fwd[1], col, psi);
            load_link(U, site, 1, u);      hop_r<1, true, false>(psi, u, T(1), acc);
            if (by == 1) srow(P0, warp - 2, psi); else gsrc.get(nbr.bwd[1], col, psi);
            load_link(U, nbr.bwd[1], 1, u); hop_r<1, false, false>(psi, u, T(1), acc);
            if (bz == 0) srow(P0, warp + 4, psi); else gsrc.get(nbr.fwd[2], col, psi);
            load_link(U, site, 2, u);      hop_r<2, true, false>(psi, u, T(1), acc);
            if (bz == 1) srow(P0, warp - 4, psi); else gsrc.get(nbr.bwd[2], col, psi);
            load_link(U, nbr.bwd[2], 2, u); hop_r<2, false, false>(psi, u, T(1), acc);
            srow(Pp, warp, psi);
            load_link(U, site, 3, u);      hop_r<3, true, true>(psi, u, sf, acc);
            srow(Pm, warp, psi);
            load_link(U, nbr.bwd[3], 3, u); hop_r<3, false, true>(psi, u, sb, acc);
            cplx<T> own[12][1];
            srow(P0, warp, own);

            const size_t off = ((size_t)site * 12 * nb + col) * 2;
            const uint32_t hsr = sr_seed(a.salt, (uint32_t)site, (uint32_t)col);
            uint32_t wq = 0;
            if (DOT) wq = z4_word(nk, site, col);
            cplx<T> dsum = cz<T>();
            if constexpr (!OUTER) {
                const cplx<T> cya = Coef<T>::get(a.ya, a.yaf), cyb = Coef<T>::get(a.yb, a.ybf);
                S* po = reinterpret_cast<S*>(a.out) + off;
                S* py = reinterpret_cast<S*>(a.y) + off;
#pragma unroll
                for (int e = 0; e < 12; ++e) {
                    cplx<T> out[1];
                    const cplx<T> tt = apply_A_elem(own[e][0], acc[e][0], kap);
                    out[0] = a.op_only ? tt : minus_alpha(own[e][0], cal, tt);
                    if (DOT) dsum = dsum + z4_conj_mul<T>(wq >> (2 * e), out[0]);
                    const uint32_t rb[1] = {sr_bits(hsr, e)}, rby[1] = {sr_bits(hsr, 12 + e)};
                    VecIO<S, 1>::st_sr(po + (size_t)e * nb * 2, out, rb);
                    if (YMODE == 1) {
                        cplx<T> yv[1];
                        yv[0] = cmul_f(cya, own[e][0]);
                        cmac(yv[0], cyb, out[0]);
                        VecIO<S, 1>::st_sr(py + (size_t)e * nb * 2, yv, rby);
                    } else if (YMODE == 2) {
                        cplx<T> yv[1];
                        VecIO<S, 1>::ld(py + (size_t)e * nb * 2, yv);
                        cmac(yv[0], cyb, out[0]);
                        VecIO<S, 1>::st_sr(py + (size_t)e * nb * 2, yv, rby);
                    }
                }
            } else {
                const cplx<T> cb = Coef<T>::get(a.beta, a.betaf), cg = Coef<T>::get(a.gamma, a.gammaf);
                const S* pw = reinterpret_cast<const S*>(a.w) + off;
                S* pwo = reinterpret_cast<S*>(a.wout) + off;
                S* py = reinterpret_cast<S*>(a.y) + off;
#pragma unroll
                for (int e = 0; e < 12; ++e) {
                    cplx<T> wv[1], yv[1];
                    VecIO<S, 1>::ld(pw + (size_t)e * nb * 2, wv);
                    VecIO<S, 1>::ld(py + (size_t)e * nb * 2, yv);
                    const cplx<T> tt = minus_alpha(own[e][0], cal, apply_A_elem(own[e][0], acc[e][0], kap));
                    const cplx<T> wn = minus_alpha(wv[0], cb, wv[0] - tt);
                    wv[0] = wn;
                    cmac(yv[0], cg, wn);
                    if (DOT) dsum = dsum + z4_conj_mul<T>(wq >> (2 * e), yv[0]);
                    const uint32_t rb[1] = {sr_bits(hsr, e)}, rby[1] = {sr_bits(hsr, 12 + e)};
                    VecIO<S, 1>::st_sr(pwo + (size_t)e * nb * 2, wv, rb);
                    VecIO<S, 1>::st_sr(py + (size_t)e * nb * 2, yv, rby);
                }
            }
            if (DOT) { dre += (double)dsum.re; dim += (double)dsum.im; }
        }
        __syncthreads();   // plane rel-1 is free: it takes plane rel+3
        if (threadIdx.x == 0 && !s_fail && rel + 3 < nrel) issue(rel + 3);
    }

    if (threadIdx.x == 0 && s_fail) {
        // wait for the last copy issued into each buffer before the CTA exits
        const long long d2 = clock64() + SWEEP_TIMEOUT;
        for (int b = 0; b < SWEEP_RING; ++b) {
            int last = -1;
            for (int r = b; r <= issued_hi; r += SWEEP_RING) last = r;
            if (last >= 0) tc::mbar_wait(&full[b], (uint32_t)((last / SWEEP_RING) & 1), d2);
        }
        atomicExch(err, 1);
    }
    if (DOT) {
        // fixed-order reduction over the 8 sites of the block, then one
        // read-modify-write of this CTA's accumulator row
        red[warp][lane] = make_double2(dre, dim);
        __syncthreads();
        if (warp == 0 && colok && !s_fail) {
            double sr = 0.0, si = 0.0;
#pragma unroll
            for (int w = 0; w < SWEEP_SITES; ++w) { sr += red[w][lane].x; si += red[w][lane].y; }
            double2* acc = a.acc + (size_t)blockIdx.x * nb + col;
            double2 cur = *acc;
            cur.x += a.dot_w[0] * sr - a.dot_w[1] * si;
            cur.y += a.dot_w[0] * si + a.dot_w[1] * sr;
            *acc = cur;
        }
    }
}

}  // namespace mpmc
