// Issue-lean form of the fused stencil kernels (k_step / k_outer of
// stencil.cuh) for FP32 and BF16-stored spinors with FP32 arithmetic.
//
// On GB300 the FP32 Wilson step at small block widths is bound by
// instruction issue, not by HBM, so this kernel is written to spend as few
// issue slots per (site, right-hand side) as the arithmetic allows:
//  * complex values are (re, im) float pairs and the SU(3) products, the
//    reconstruction and A = I - kappa H run as packed FP32x2 FMAs/adds;
//    the links are pre-expanded once per field into broadcast pairs
//    (re, re, im, im), so U h = (re,re)*h + (im,im)*(i h) needs no shuffles;
//  * the lower spin components collect their +-i terms in a separate
//    accumulator, so the reconstruction needs no swaps either;
//  * the block width NB is a compile-time constant: the 12 components of a
//    spinor row sit at immediate offsets;
//  * Z4 symbols come from a per-block table of Philox words in memory, and
//    the noise dot b^H w uses a 4-entry shared-memory table per symbol;
//  * site coordinates use multiply-high division by the lattice extents.
// Per-component rounding is that of scalar FMAs; the grouping of the sums
// differs from k_step, so results agree with it to FP32 rounding.
#pragma once

#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"

namespace mpmc {
namespace fast {

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

template <class S> struct Row;
template <> struct Row<float> {
    static __device__ __forceinline__ float2 ld(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
    static __device__ __forceinline__ float2 ld_rw(const float* p) { return *reinterpret_cast<const float2*>(p); }
    static __device__ __forceinline__ void st(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
    static __device__ __forceinline__ void st_sr(float* p, float2 v, uint32_t) { st(p, v); }
};
template <> struct Row<__nv_bfloat16> {
    static __device__ __forceinline__ float2 cvt(uint32_t w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    static __device__ __forceinline__ float2 ld(const __nv_bfloat16* p) {
        return cvt(__ldg(reinterpret_cast<const unsigned int*>(p)));
    }
    static __device__ __forceinline__ float2 ld_rw(const __nv_bfloat16* p) {
        return cvt(*reinterpret_cast<const uint32_t*>(p));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float2 v) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.x, v.y);
    }
    // stochastic rounding (zero-mean errors) for the chain vectors
    static __device__ __forceinline__ void st_sr(__nv_bfloat16* p, float2 v, uint32_t rb) {
        *reinterpret_cast<uint32_t*>(p) = bf16x2_sr(v.x, v.y, rb);
    }
};

// 12 components of column `col` of a stored block row (compile-time stride NB)
template <class S, int NB> struct MemRow {
    const S* p;
    __device__ __forceinline__ float2 get(int site, int col, int e) const {
        return Row<S>::ld(p + ((size_t)site * 12 * NB + col) * 2 + (size_t)e * NB * 2);
    }
};
// Z4 noise from the per-block word table (symbol q -> i^q from a shared table)
template <int NB> struct NoiseRow {
    const uint32_t* words;
    const float2* zval;   // shared: {1, i, -1, -i}
    __device__ __forceinline__ float2 get(int site, int col, int e) const {
        const uint32_t w = __ldg(words + (size_t)site * NB + col);
        return zval[(w >> (2 * e)) & 3u];
    }
};

// One hop on a loaded neighbour row p: projection, SU(3) product with the
// expanded link, reconstruction.  up[3*spin + c] for spins 0, 1; lower
// spins: lr (real coefficients) and lj (coefficients of i), index
// 3*(spin-2) + c.  sgn (applied when use_sgn) is the boundary sign.
// A link element: read-only global load, or (SMEM) a plain load of a copy staged in shared memory
template <bool SMEM> __device__ __forceinline__ float4 ld_link(const float4* p) {
    if constexpr (SMEM) return *p;
    else return __ldg(p);
}

template <int MU, bool FWD, bool SMEM = false>
__device__ __forceinline__ void hop_p(const float2 (&p)[12], const float4* __restrict__ L, float sgn, bool use_sgn,
                                      float2 (&up)[6], float2 (&lr)[6], float2 (&lj)[6]) {
    float2 h0[3], h1[3], i0[3], i1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        float2 a, b;
        if (MU == 0) {        // FWD: p0 - i p3, p1 - i p2;  BWD: p0 + i p3, p1 + i p2
            if (FWD) { a = make_float2(p0.x + p3.y, p0.y - p3.x); b = make_float2(p1.x + p2.y, p1.y - p2.x); }
            else     { a = make_float2(p0.x - p3.y, p0.y + p3.x); b = make_float2(p1.x - p2.y, p1.y + p2.x); }
        } else if (MU == 1) { // FWD: p0 + p3, p1 - p2;  BWD: p0 - p3, p1 + p2
            if (FWD) { a = add2(p0, p3); b = sub2(p1, p2); }
            else     { a = sub2(p0, p3); b = add2(p1, p2); }
        } else if (MU == 2) { // FWD: p0 - i p2, p1 + i p3;  BWD: p0 + i p2, p1 - i p3
            if (FWD) { a = make_float2(p0.x + p2.y, p0.y - p2.x); b = make_float2(p1.x - p3.y, p1.y + p3.x); }
            else     { a = make_float2(p0.x - p2.y, p0.y + p2.x); b = make_float2(p1.x + p3.y, p1.y - p3.x); }
        } else {              // FWD: p0 - p2, p1 - p3;  BWD: p0 + p2, p1 + p3
            if (FWD) { a = sub2(p0, p2); b = sub2(p1, p3); }
            else     { a = add2(p0, p2); b = add2(p1, p3); }
        }
        if (use_sgn) {
            a = __fmul2_rn(a, make_float2(sgn, sgn));
            b = __fmul2_rn(b, make_float2(sgn, sgn));
        }
        h0[c] = a;
        h1[c] = b;
        // i h (forward: U h = re*h + im*(i h)) or -i h (backward: conj(U) h = re*h + im*(-i h))
        i0[c] = FWD ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
        i1[c] = FWD ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float2 g0 = make_float2(0.f, 0.f), g1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 u = ld_link<SMEM>(L + (FWD ? 3 * r + c : 3 * c + r));
            const float2 ur = make_float2(u.x, u.y), ui = make_float2(u.z, u.w);
            g0 = fma2(ur, h0[c], g0);
            g0 = fma2(ui, i0[c], g0);
            g1 = fma2(ur, h1[c], g1);
            g1 = fma2(ui, i1[c], g1);
        }
        up[r] = add2(up[r], g0);
        up[3 + r] = add2(up[3 + r], g1);
        if (MU == 0) {
            if (FWD) { lj[r] = add2(lj[r], g1); lj[3 + r] = add2(lj[3 + r], g0); }
            else     { lj[r] = sub2(lj[r], g1); lj[3 + r] = sub2(lj[3 + r], g0); }
        } else if (MU == 1) {
            if (FWD) { lr[r] = sub2(lr[r], g1); lr[3 + r] = add2(lr[3 + r], g0); }
            else     { lr[r] = add2(lr[r], g1); lr[3 + r] = sub2(lr[3 + r], g0); }
        } else if (MU == 2) {
            if (FWD) { lj[r] = add2(lj[r], g0); lj[3 + r] = sub2(lj[3 + r], g1); }
            else     { lj[r] = sub2(lj[r], g0); lj[3 + r] = add2(lj[3 + r], g1); }
        } else {
            if (FWD) { lr[r] = sub2(lr[r], g0); lr[3 + r] = sub2(lr[3 + r], g1); }
            else     { lr[r] = add2(lr[r], g0); lr[3 + r] = add2(lr[3 + r], g1); }
        }
    }
}

template <int MU, bool FWD, class Src>
__device__ __forceinline__ void hop(const Src& src, int nsite, int col, const float4* __restrict__ L, float sgn,
                                    bool use_sgn, float2 (&up)[6], float2 (&lr)[6], float2 (&lj)[6]) {
    float2 p[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) p[e] = src.get(nsite, col, e);
    hop_p<MU, FWD>(p, L, sgn, use_sgn, up, lr, lj);
}

__device__ __forceinline__ uint32_t divu(uint32_t n, unsigned long long m) { return (uint32_t)__umul64hi(n, m); }

// H psi at `site` for column `col`: hw[e], e = 3*spin + colour
template <class Src>
__device__ __forceinline__ void hopping(const FastArgs& a, const Src& src, int site, int col, float2 (&hw)[12]) {
    const uint32_t s = (uint32_t)site;
    const uint32_t q1 = divu(s, a.mx), x = s - q1 * a.lx;
    const uint32_t q2 = divu(q1, a.my), y = q1 - q2 * a.ly;
    const uint32_t t = divu(q2, a.mz), z = q2 - t * a.lz;
    const int sy = a.lx, sz = a.lx * a.ly, st = sz * a.lz;
    const int xf = site + (x + 1 < (uint32_t)a.lx ? 1 : 1 - a.lx), xb = site - (x > 0 ? 1 : 1 - a.lx);
    const int yf = site + (y + 1 < (uint32_t)a.ly ? sy : sy - a.ly * sy), yb = site - (y > 0 ? sy : sy - a.ly * sy);
    const int zf = site + (z + 1 < (uint32_t)a.lz ? sz : sz - a.lz * sz), zb = site - (z > 0 ? sz : sz - a.lz * sz);
    const int tf = site + (t + 1 < (uint32_t)a.lt ? st : st - a.lt * st), tb = site - (t > 0 ? st : st - a.lt * st);
    const bool af = a.bc_t < 0 && t + 1 == (uint32_t)a.lt, ab = a.bc_t < 0 && t == 0;
    float2 up[6], lr[6], lj[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) up[i] = lr[i] = lj[i] = make_float2(0.f, 0.f);
    const float4* U = a.Ue;
    hop<0, true>(src, xf, col, U + ((size_t)site * 4 + 0) * 9, 1.f, false, up, lr, lj);
    hop<0, false>(src, xb, col, U + ((size_t)xb * 4 + 0) * 9, 1.f, false, up, lr, lj);
    hop<1, true>(src, yf, col, U + ((size_t)site * 4 + 1) * 9, 1.f, false, up, lr, lj);
    hop<1, false>(src, yb, col, U + ((size_t)yb * 4 + 1) * 9, 1.f, false, up, lr, lj);
    hop<2, true>(src, zf, col, U + ((size_t)site * 4 + 2) * 9, 1.f, false, up, lr, lj);
    hop<2, false>(src, zb, col, U + ((size_t)zb * 4 + 2) * 9, 1.f, false, up, lr, lj);
    hop<3, true>(src, tf, col, U + ((size_t)site * 4 + 3) * 9, -1.f, af, up, lr, lj);
    hop<3, false>(src, tb, col, U + ((size_t)tb * 4 + 3) * 9, -1.f, ab, up, lr, lj);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        hw[i] = up[i];
        hw[6 + i] = make_float2(lr[i].x - lj[i].y, lr[i].y + lj[i].x);
    }
}

// o = own - alpha * t, per component in the order of minus_alpha (stencil.cuh)
__device__ __forceinline__ float2 minus_alpha2(float2 own, float2 al, float2 t) {
    float2 o = fma2(make_float2(-al.x, -al.x), t, own);
    o.x = fmaf(al.y, t.y, o.x);
    o.y = fmaf(-al.y, t.x, o.y);
    return o;
}
// acc += c * v (complex), in the order of cmac (stencil.cuh)
__device__ __forceinline__ float2 cmac2(float2 acc, float2 c, float2 v) {
    acc = fma2(make_float2(c.x, c.x), v, acc);
    acc.x = fmaf(-c.y, v.y, acc.x);
    acc.y = fmaf(c.y, v.x, acc.y);
    return acc;
}

// (cr, cr, ci, ci) of conj(i^q) and i^q, for the shared tables
__device__ __forceinline__ float4 z4_conj_entry(int q) {
    const float cr = q == 0 ? 1.f : (q == 2 ? -1.f : 0.f), ci = q == 1 ? -1.f : (q == 3 ? 1.f : 0.f);
    return make_float4(cr, cr, ci, ci);
}

// KIND: 0 step, 1 step + dot, 2 step from the noise + dot, 3 outer, 4 outer + dot
template <class S, int NB, int KIND>
__global__ void __launch_bounds__(256) k_fast(const FastArgs a) {
    constexpr int TW = NB < 32 ? NB : 32;
    constexpr int SB = 256 / TW;
    constexpr bool OUTER = KIND >= 3;
    constexpr bool DOT = KIND == 1 || KIND == 2 || KIND == 4;
    constexpr bool NOISE = KIND == 2;
    __shared__ float4 ctab[4];   // (cr, cr, ci, ci) of conj(i^q)
    __shared__ float2 zval[4];   // i^q
    if (threadIdx.y == 0 && threadIdx.x < 4) {
        const float4 c = z4_conj_entry(threadIdx.x);
        ctab[threadIdx.x] = c;
        zval[threadIdx.x] = make_float2(c.x, -c.z);
    }
    __syncthreads();
    const int col = blockIdx.y * TW + threadIdx.x;
    float dre = 0.f, dim = 0.f;
    const float2 al = make_float2(a.alpha[0], a.alpha[1]);
    const float2 mk = make_float2(-a.kappa, -a.kappa);
    for (int it = 0; it < a.sl; ++it) {
        const int site = (blockIdx.x * a.sl + it) * SB + threadIdx.y;
        if (site >= a.V) break;
        float2 hw[12];
        uint32_t word = 0;
        if (NOISE) {
            const NoiseRow<NB> src{a.words, zval};
            hopping(a, src, site, col, hw);
        } else {
            const MemRow<S, NB> src{reinterpret_cast<const S*>(a.in)};
            hopping(a, src, site, col, hw);
        }
        if (DOT || NOISE) word = __ldg(a.words + (size_t)site * NB + col);
        const size_t off = ((size_t)site * 12 * NB + col) * 2;
        const S* pin = NOISE ? nullptr : reinterpret_cast<const S*>(a.in) + off;
        const uint32_t hsr = sr_seed(a.salt, (uint32_t)site, (uint32_t)col);
        float2 dA = make_float2(0.f, 0.f), dB = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < 12; ++e) {
            const float2 own = NOISE ? zval[(word >> (2 * e)) & 3u] : Row<S>::ld(pin + (size_t)e * NB * 2);
            const float2 t = fma2(mk, hw[e], own);                 // own - kappa H own
            float2 v;
            if (!OUTER) {
                v = minus_alpha2(own, al, t);                      // (I - A/theta) own
                Row<S>::st_sr(reinterpret_cast<S*>(a.out) + off + (size_t)e * NB * 2, v, sr_bits(hsr, e));
            } else {
                const float2 tt = minus_alpha2(own, al, t);        // pi_in(A) w
                const size_t oe = off + (size_t)e * NB * 2;
                const float2 wv = Row<S>::ld_rw(reinterpret_cast<const S*>(a.w) + oe);
                float2 yv = Row<S>::ld_rw(reinterpret_cast<const S*>(a.y) + oe);
                const float2 wn = minus_alpha2(wv, make_float2(a.beta[0], a.beta[1]), sub2(wv, tt));
                yv = cmac2(yv, make_float2(a.gamma[0], a.gamma[1]), wn);
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
            dre += dA.x - dB.y;
            dim += dA.y + dB.x;
        }
    }
    if (DOT) {
        __shared__ double2 red[SB][TW];
        red[threadIdx.y][threadIdx.x] = make_double2((double)dre, (double)dim);
        __syncthreads();
        if (threadIdx.y == 0) {
            double sr = 0.0, si = 0.0;
            for (int yy = 0; yy < SB; ++yy) {
                sr += red[yy][threadIdx.x].x;
                si += red[yy][threadIdx.x].y;
            }
            double2* pa = a.acc + (size_t)blockIdx.x * NB + col;
            double2 cur = *pa;
            cur.x += a.dot_w[0] * sr - a.dot_w[1] * si;
            cur.y += a.dot_w[0] * si + a.dot_w[1] * sr;
            *pa = cur;
        }
    }
}

}  // namespace fast
}  // namespace mpmc
