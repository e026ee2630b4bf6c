// The fused stencil kernels: one degree step of the root-form polynomial
// (paper Sec. 2.3) applied to a block of right-hand sides, with the Wilson
// hopping term computed in place (half-spinor projection), and the composite
// outer step of Sec. 3.2.  Each thread handles R consecutive right-hand
// sides of one site, so one link load and one neighbour-index computation
// serve R vectors and spinor components move as R-wide vector loads.
// Instantiated per storage format in stencil_{f64,f32,bf16}.cu.
#pragma once

#include "device.cuh"
#include "kernels.h"

namespace mpmc {

// ------------------------------------------------------------------ FMA-chained complex arithmetic
template <class T> __device__ __forceinline__ cplx<T> cmul_f(cplx<T> a, cplx<T> b) {
    cplx<T> r;
    r.re = a.re * b.re;
    r.re = fma(-a.im, b.im, r.re);
    r.im = a.re * b.im;
    r.im = fma(a.im, b.re, r.im);
    return r;
}
// acc += a * b
template <class T> __device__ __forceinline__ void cmac(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// conj(a) * b
template <class T> __device__ __forceinline__ cplx<T> ccmul_f(cplx<T> a, cplx<T> b) {
    cplx<T> r;
    r.re = a.re * b.re;
    r.re = fma(a.im, b.im, r.re);
    r.im = a.re * b.im;
    r.im = fma(-a.im, b.re, r.im);
    return r;
}
// acc += conj(a) * b
template <class T> __device__ __forceinline__ void ccmac(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

// ------------------------------------------------------------------ R-wide loads and stores
template <class S, int R> struct VecIO;

template <> struct VecIO<float, 1> {
    static __device__ __forceinline__ void ld(const float* p, cplx<float> (&v)[1]) {
        const float2 x = *reinterpret_cast<const float2*>(p);
        v[0] = {x.x, x.y};
    }
    static __device__ __forceinline__ void st(float* p, const cplx<float> (&v)[1]) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0].re, v[0].im);
    }
    static __device__ __forceinline__ void st_sr(float* p, const cplx<float> (&v)[1], const uint32_t (&)[1]) { st(p, v); }
};
template <> struct VecIO<float, 2> {
    static __device__ __forceinline__ void ld(const float* p, cplx<float> (&v)[2]) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        v[0] = {x.x, x.y};
        v[1] = {x.z, x.w};
    }
    static __device__ __forceinline__ void st(float* p, const cplx<float> (&v)[2]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
    }
    static __device__ __forceinline__ void st_sr(float* p, const cplx<float> (&v)[2], const uint32_t (&)[2]) { st(p, v); }
};
template <> struct VecIO<double, 1> {
    static __device__ __forceinline__ void ld(const double* p, cplx<double> (&v)[1]) {
        const double2 x = *reinterpret_cast<const double2*>(p);
        v[0] = {x.x, x.y};
    }
    static __device__ __forceinline__ void st(double* p, const cplx<double> (&v)[1]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0].re, v[0].im);
    }
    static __device__ __forceinline__ void st_sr(double* p, const cplx<double> (&v)[1], const uint32_t (&)[1]) { st(p, v); }
};
template <> struct VecIO<double, 2> {
    static __device__ __forceinline__ void ld(const double* p, cplx<double> (&v)[2]) {
        const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
        v[0] = {x.x, x.y};
        v[1] = {y.x, y.y};
    }
    static __device__ __forceinline__ void st(double* p, const cplx<double> (&v)[2]) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0].re, v[0].im);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[1].re, v[1].im);
    }
    static __device__ __forceinline__ void st_sr(double* p, const cplx<double> (&v)[2], const uint32_t (&)[2]) { st(p, v); }
};
template <> struct VecIO<__nv_bfloat16, 1> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16* p, cplx<float> (&v)[1]) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
        v[0] = {f.x, f.y};
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, const cplx<float> (&v)[1]) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v[0].re, v[0].im);
    }
    static __device__ __forceinline__ void st_sr(__nv_bfloat16* p, const cplx<float> (&v)[1], const uint32_t (&rb)[1]) {
        *reinterpret_cast<uint32_t*>(p) = bf16x2_sr(v[0].re, v[0].im, rb[0]);
    }
};
template <> struct VecIO<__nv_bfloat16, 2> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16* p, cplx<float> (&v)[2]) {
        const uint2 x = *reinterpret_cast<const uint2*>(p);
        const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x.x));
        const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x.y));
        v[0] = {f0.x, f0.y};
        v[1] = {f1.x, f1.y};
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, const cplx<float> (&v)[2]) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0].re, v[0].im), b = __floats2bfloat162_rn(v[1].re, v[1].im);
        uint2 x;
        x.x = *reinterpret_cast<uint32_t*>(&a);
        x.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = x;
    }
    static __device__ __forceinline__ void st_sr(__nv_bfloat16* p, const cplx<float> (&v)[2], const uint32_t (&rb)[2]) {
        uint2 x;
        x.x = bf16x2_sr(v[0].re, v[0].im, rb[0]);
        x.y = bf16x2_sr(v[1].re, v[1].im, rb[1]);
        *reinterpret_cast<uint2*>(p) = x;
    }
};

// Sources of the 12 x R values of a site: memory, or the noise block itself.
template <class S, int R> struct MemSrcR {
    const S* p;
    int nb;
    using T = typename Math<S>::T;
    __device__ __forceinline__ void get(int site, int col0, cplx<T> (&v)[12][R]) const {
        const S* q = p + ((size_t)site * 12 * nb + col0) * 2;
#pragma unroll
        for (int e = 0; e < 12; ++e) VecIO<S, R>::ld(q + (size_t)e * nb * 2, v[e]);
    }
};

template <class T, int R> struct NoiseSrcR {
    NoiseKey nk;
    __device__ __forceinline__ void get(int site, int col0, cplx<T> (&v)[12][R]) const {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t w = z4_word(nk, site, col0 + r);
#pragma unroll
            for (int e = 0; e < 12; ++e) v[e][r] = z4_value<T>(w >> (2 * e));
        }
    }
};

// g = U h (FWD) or U^+ h, FMA-chained
template <bool FWD, class T>
__device__ __forceinline__ void su3_apply(const cplx<T> (&u)[9], const cplx<T> (&h)[3], cplx<T> (&g)[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (FWD) {
            g[a] = cmul_f(u[3 * a], h[0]);
            cmac(g[a], u[3 * a + 1], h[1]);
            cmac(g[a], u[3 * a + 2], h[2]);
        } else {
            g[a] = ccmul_f(u[a], h[0]);
            ccmac(g[a], u[3 + a], h[1]);
            ccmac(g[a], u[6 + a], h[2]);
        }
    }
}

// One hop for R columns (projector, link multiply, reconstruction), the
// same spin algebra as `hop` in device.cuh.
template <int MU, bool FWD, bool SIGN, class T, int R>
__device__ __forceinline__ void hop_r(const cplx<T> (&psi)[12][R], const cplx<T> (&u)[9], T sgn,
                                      cplx<T> (&acc)[12][R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cplx<T> h0[3], h1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cplx<T> p0 = psi[c][r], p1 = psi[3 + c][r], p2 = psi[6 + c][r], p3 = psi[9 + c][r];
            if (MU == 0) {
                if (FWD) { h0[c] = p0 + times_mi(p3); h1[c] = p1 + times_mi(p2); }
                else     { h0[c] = p0 + times_i(p3);  h1[c] = p1 + times_i(p2); }
            } else if (MU == 1) {
                if (FWD) { h0[c] = p0 + p3; h1[c] = p1 - p2; }
                else     { h0[c] = p0 - p3; h1[c] = p1 + p2; }
            } else if (MU == 2) {
                if (FWD) { h0[c] = p0 + times_mi(p2); h1[c] = p1 + times_i(p3); }
                else     { h0[c] = p0 + times_i(p2);  h1[c] = p1 + times_mi(p3); }
            } else {
                if (FWD) { h0[c] = p0 - p2; h1[c] = p1 - p3; }
                else     { h0[c] = p0 + p2; h1[c] = p1 + p3; }
            }
            if (SIGN) { h0[c] = scale(h0[c], sgn); h1[c] = scale(h1[c], sgn); }
        }
        cplx<T> g0[3], g1[3];
        su3_apply<FWD>(u, h0, g0);
        su3_apply<FWD>(u, h1, g1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc[c][r] = acc[c][r] + g0[c];
            acc[3 + c][r] = acc[3 + c][r] + g1[c];
            if (MU == 0) {
                if (FWD) { acc[6 + c][r] = acc[6 + c][r] + times_i(g1[c]);  acc[9 + c][r] = acc[9 + c][r] + times_i(g0[c]); }
                else     { acc[6 + c][r] = acc[6 + c][r] + times_mi(g1[c]); acc[9 + c][r] = acc[9 + c][r] + times_mi(g0[c]); }
            } else if (MU == 1) {
                if (FWD) { acc[6 + c][r] = acc[6 + c][r] - g1[c]; acc[9 + c][r] = acc[9 + c][r] + g0[c]; }
                else     { acc[6 + c][r] = acc[6 + c][r] + g1[c]; acc[9 + c][r] = acc[9 + c][r] - g0[c]; }
            } else if (MU == 2) {
                if (FWD) { acc[6 + c][r] = acc[6 + c][r] + times_i(g0[c]);  acc[9 + c][r] = acc[9 + c][r] + times_mi(g1[c]); }
                else     { acc[6 + c][r] = acc[6 + c][r] + times_mi(g0[c]); acc[9 + c][r] = acc[9 + c][r] + times_i(g1[c]); }
            } else {
                if (FWD) { acc[6 + c][r] = acc[6 + c][r] - g0[c]; acc[9 + c][r] = acc[9 + c][r] - g1[c]; }
                else     { acc[6 + c][r] = acc[6 + c][r] + g0[c]; acc[9 + c][r] = acc[9 + c][r] + g1[c]; }
            }
        }
    }
}

template <class T, int R, class Src>
__device__ __forceinline__ void hopping_r(const Lattice& L, const T* __restrict__ U, const Src& src, int site,
                                          int col0, cplx<T> (&acc)[12][R]) {
    const Nbrs nb = neighbours(L, site);
#pragma unroll
    for (int e = 0; e < 12; ++e)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[e][r] = cz<T>();
    cplx<T> psi[12][R], u[9];
    const T sf = (nb.fwd_wrap_t && L.bc_t < 0) ? T(-1) : T(1);
    const T sb = (nb.bwd_wrap_t && L.bc_t < 0) ? T(-1) : T(1);
    src.get(nb.fwd[0], col0, psi); load_link(U, site, 0, u);      hop_r<0, true, false>(psi, u, T(1), acc);
    src.get(nb.bwd[0], col0, psi); load_link(U, nb.bwd[0], 0, u); hop_r<0, false, false>(psi, u, T(1), acc);
    src.get(nb.fwd[1], col0, psi); load_link(U, site, 1, u);      hop_r<1, true, false>(psi, u, T(1), acc);
    src.get(nb.bwd[1], col0, psi); load_link(U, nb.bwd[1], 1, u); hop_r<1, false, false>(psi, u, T(1), acc);
    src.get(nb.fwd[2], col0, psi); load_link(U, site, 2, u);      hop_r<2, true, false>(psi, u, T(1), acc);
    src.get(nb.bwd[2], col0, psi); load_link(U, nb.bwd[2], 2, u); hop_r<2, false, false>(psi, u, T(1), acc);
    src.get(nb.fwd[3], col0, psi); load_link(U, site, 3, u);      hop_r<3, true, true>(psi, u, sf, acc);
    src.get(nb.bwd[3], col0, psi); load_link(U, nb.bwd[3], 3, u); hop_r<3, false, true>(psi, u, sb, acc);
}

template <class T> struct Coef;
template <> struct Coef<float> {
    static __device__ __forceinline__ cplx<float> get(const double (&)[2], const float (&f)[2]) { return {f[0], f[1]}; }
    static __device__ __forceinline__ float real(double, float f) { return f; }
};
template <> struct Coef<double> {
    static __device__ __forceinline__ cplx<double> get(const double (&d)[2], const float (&)[2]) { return {d[0], d[1]}; }
    static __device__ __forceinline__ double real(double d, float) { return d; }
};

// t = own - kappa * hw  (A applied), then out = own - alpha * t
template <class T>
__device__ __forceinline__ cplx<T> apply_A_elem(cplx<T> own, cplx<T> hw, T kappa) {
    return {fma(-kappa, hw.re, own.re), fma(-kappa, hw.im, own.im)};
}
template <class T>
__device__ __forceinline__ cplx<T> minus_alpha(cplx<T> own, cplx<T> alpha, cplx<T> t) {
    cplx<T> o = own;
    cmac(o, cplx<T>{-alpha.re, -alpha.im}, t);
    return o;
}

// Reduce R per-thread partial dots over threadIdx.y in fixed order (FP64),
// then acc[blockIdx.x][col] += w * sum.
template <class T, int R>
__device__ __forceinline__ void cta_dot_r(const cplx<T> (&v)[R], int col0, bool colok, int nb, const double (&w)[2],
                                          double2* acc) {
    __shared__ double2 red[256 * R];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
    for (int r = 0; r < R; ++r) red[tid * R + r] = make_double2((double)v[r].re, (double)v[r].im);
    __syncthreads();
    if (threadIdx.y == 0 && colok) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double sr = 0.0, si = 0.0;
            for (int yy = 0; yy < (int)blockDim.y; ++yy) {
                const double2 q = red[(yy * blockDim.x + threadIdx.x) * R + r];
                sr += q.x;
                si += q.y;
            }
            double2* pa = acc + (size_t)blockIdx.x * nb + col0 + r;
            double2 cur = *pa;
            cur.x += w[0] * sr - w[1] * si;
            cur.y += w[0] * si + w[1] * sr;
            *pa = cur;
        }
    }
}

// ------------------------------------------------------------------ step
template <class S, int R, bool NOISE_IN, bool DOT, int YMODE>
__global__ void __launch_bounds__(256) k_step(StepArgs a, Lattice L, const typename Math<S>::T* __restrict__ U,
                                              int nb, NoiseKey nk, int sl) {
    using T = typename Math<S>::T;
    const int col0 = (blockIdx.y * blockDim.x + threadIdx.x) * R;
    const bool colok = col0 < nb;
    const cplx<T> cal = Coef<T>::get(a.alpha, a.alphaf);
    const T kap = Coef<T>::real(a.kappa, a.kappaf);
    const bool op_only = a.op_only;
    const cplx<T> cya = Coef<T>::get(a.ya, a.yaf), cyb = Coef<T>::get(a.yb, a.ybf);
    cplx<T> dsum[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dsum[r] = cz<T>();
    const int base = blockIdx.x * blockDim.y * sl;
    for (int it = 0; it < sl; ++it) {
        const int site = base + it * blockDim.y + threadIdx.y;
        if (site >= L.V || !colok) continue;
        cplx<T> hw[12][R], own[12][R];
        if (NOISE_IN) {
            NoiseSrcR<T, R> src{nk};
            hopping_r<T, R>(L, U, src, site, col0, hw);
            src.get(site, col0, own);
        } else {
            MemSrcR<S, R> src{reinterpret_cast<const S*>(a.in), nb};
            hopping_r<T, R>(L, U, src, site, col0, hw);
            src.get(site, col0, own);
        }
        const size_t off = ((size_t)site * 12 * nb + col0) * 2;
        S* po = reinterpret_cast<S*>(a.out) + off;
        S* py = reinterpret_cast<S*>(a.y) + off;
        uint32_t wq[R], hsr[R], rb[R], rby[R];
        if (DOT)
#pragma unroll
            for (int r = 0; r < R; ++r) wq[r] = z4_word(nk, site, col0 + r);
#pragma unroll
        for (int r = 0; r < R; ++r) hsr[r] = sr_seed(a.salt, (uint32_t)site, (uint32_t)(col0 + r));
#pragma unroll
        for (int e = 0; e < 12; ++e) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                rb[r] = sr_bits(hsr[r], e);
                rby[r] = sr_bits(hsr[r], 12 + e);
            }
            cplx<T> out[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const cplx<T> t = apply_A_elem(own[e][r], hw[e][r], kap);
                out[r] = op_only ? t : minus_alpha(own[e][r], cal, t);
                if (DOT) dsum[r] = dsum[r] + z4_conj_mul<T>(wq[r] >> (2 * e), out[r]);
            }
            VecIO<S, R>::st_sr(po + (size_t)e * nb * 2, out, rb);
            if (YMODE == 1) {
                cplx<T> yv[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    yv[r] = cmul_f(cya, own[e][r]);
                    cmac(yv[r], cyb, out[r]);
                }
                VecIO<S, R>::st_sr(py + (size_t)e * nb * 2, yv, rby);
            } else if (YMODE == 2) {
                cplx<T> yv[R];
                VecIO<S, R>::ld(py + (size_t)e * nb * 2, yv);
#pragma unroll
                for (int r = 0; r < R; ++r) cmac(yv[r], cyb, out[r]);
                VecIO<S, R>::st_sr(py + (size_t)e * nb * 2, yv, rby);
            }
        }
    }
    if (DOT) cta_dot_r<T, R>(dsum, col0, colok, nb, a.dot_w, a.acc);
}

// ------------------------------------------------------------------ outer
template <class S, int R, bool DOT>
__global__ void __launch_bounds__(256) k_outer(OuterArgs a, Lattice L, const typename Math<S>::T* __restrict__ U,
                                               int nb, NoiseKey nk, int sl) {
    using T = typename Math<S>::T;
    const int col0 = (blockIdx.y * blockDim.x + threadIdx.x) * R;
    const bool colok = col0 < nb;
    const cplx<T> cal = Coef<T>::get(a.alpha, a.alphaf);
    const T kap = Coef<T>::real(a.kappa, a.kappaf);
    const cplx<T> cb = Coef<T>::get(a.beta, a.betaf), cg = Coef<T>::get(a.gamma, a.gammaf);
    cplx<T> dsum[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dsum[r] = cz<T>();
    const int base = blockIdx.x * blockDim.y * sl;
    for (int it = 0; it < sl; ++it) {
        const int site = base + it * blockDim.y + threadIdx.y;
        if (site >= L.V || !colok) continue;
        cplx<T> hw[12][R], own[12][R];
        MemSrcR<S, R> src{reinterpret_cast<const S*>(a.in), nb};
        hopping_r<T, R>(L, U, src, site, col0, hw);
        src.get(site, col0, own);
        const size_t off = ((size_t)site * 12 * nb + col0) * 2;
        const S* pw = reinterpret_cast<const S*>(a.w) + off;
        S* pwo = reinterpret_cast<S*>(a.wout) + off;
        S* py = reinterpret_cast<S*>(a.y) + off;
        uint32_t wq[R], hsr[R], rb[R], rby[R];
        if (DOT)
#pragma unroll
            for (int r = 0; r < R; ++r) wq[r] = z4_word(nk, site, col0 + r);
#pragma unroll
        for (int r = 0; r < R; ++r) hsr[r] = sr_seed(a.salt, (uint32_t)site, (uint32_t)(col0 + r));
#pragma unroll
        for (int e = 0; e < 12; ++e) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                rb[r] = sr_bits(hsr[r], e);
                rby[r] = sr_bits(hsr[r], 12 + e);
            }
            cplx<T> wv[R], yv[R];
            VecIO<S, R>::ld(pw + (size_t)e * nb * 2, wv);
            VecIO<S, R>::ld(py + (size_t)e * nb * 2, yv);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const cplx<T> t = minus_alpha(own[e][r], cal, apply_A_elem(own[e][r], hw[e][r], kap));
                const cplx<T> wn = minus_alpha(wv[r], cb, wv[r] - t);
                wv[r] = wn;
                cmac(yv[r], cg, wn);
                if (DOT) dsum[r] = dsum[r] + z4_conj_mul<T>(wq[r] >> (2 * e), yv[r]);
            }
            VecIO<S, R>::st_sr(pwo + (size_t)e * nb * 2, wv, rb);
            VecIO<S, R>::st_sr(py + (size_t)e * nb * 2, yv, rby);
        }
    }
    if (DOT) cta_dot_r<T, R>(dsum, col0, colok, nb, a.dot_w, a.acc);
}

// ------------------------------------------------------------------ dispatch (per storage)
template <class S, int R>
void step_dispatch_r(const Geom& g, const void* links, int nb, const NoiseSpec& ns, const StepArgs& a,
                     const LaunchCfg& c, cudaStream_t s) {
    using T = typename Math<S>::T;
    const dim3 grid(c.gx, c.gy), block(c.bx, c.by);
    Lattice L;
    L.lx = g.lx; L.ly = g.ly; L.lz = g.lz; L.lt = g.lt; L.V = g.V; L.bc_t = g.bc_t;
    NoiseKey nk;
    nk.k0 = (uint32_t)(ns.seed & 0xffffffffu);
    nk.k1 = (uint32_t)(ns.seed >> 32);
    nk.level = ns.level;
    nk.j0 = ns.j0;
    const T* U = reinterpret_cast<const T*>(links);
    const bool noise = (a.in == nullptr);
#define MPMC_STEP(NI, D, Y) k_step<S, R, NI, D, Y><<<grid, block, 0, s>>>(a, L, U, nb, nk, c.sl)
    if (noise) {
        if (a.dot) {
            if (a.ymode == 0) MPMC_STEP(true, true, 0); else if (a.ymode == 1) MPMC_STEP(true, true, 1); else MPMC_STEP(true, true, 2);
        } else {
            if (a.ymode == 0) MPMC_STEP(true, false, 0); else if (a.ymode == 1) MPMC_STEP(true, false, 1); else MPMC_STEP(true, false, 2);
        }
    } else {
        if (a.dot) {
            if (a.ymode == 0) MPMC_STEP(false, true, 0); else if (a.ymode == 1) MPMC_STEP(false, true, 1); else MPMC_STEP(false, true, 2);
        } else {
            if (a.ymode == 0) MPMC_STEP(false, false, 0); else if (a.ymode == 1) MPMC_STEP(false, false, 1); else MPMC_STEP(false, false, 2);
        }
    }
#undef MPMC_STEP
}

template <class S, int R>
void outer_dispatch_r(const Geom& g, const void* links, int nb, const NoiseSpec& ns, const OuterArgs& a,
                      const LaunchCfg& c, cudaStream_t s) {
    using T = typename Math<S>::T;
    const dim3 grid(c.gx, c.gy), block(c.bx, c.by);
    Lattice L;
    L.lx = g.lx; L.ly = g.ly; L.lz = g.lz; L.lt = g.lt; L.V = g.V; L.bc_t = g.bc_t;
    NoiseKey nk;
    nk.k0 = (uint32_t)(ns.seed & 0xffffffffu);
    nk.k1 = (uint32_t)(ns.seed >> 32);
    nk.level = ns.level;
    nk.j0 = ns.j0;
    const T* U = reinterpret_cast<const T*>(links);
    if (a.dot) k_outer<S, R, true><<<grid, block, 0, s>>>(a, L, U, nb, nk, c.sl);
    else k_outer<S, R, false><<<grid, block, 0, s>>>(a, L, U, nb, nk, c.sl);
}

template <class S>
void step_dispatch(const Geom& g, const void* links, int nb, const NoiseSpec& ns, const StepArgs& a,
                   const LaunchCfg& c, cudaStream_t s) {
    if (c.R == 2) step_dispatch_r<S, 2>(g, links, nb, ns, a, c, s);
    else step_dispatch_r<S, 1>(g, links, nb, ns, a, c, s);
}

template <class S>
void outer_dispatch(const Geom& g, const void* links, int nb, const NoiseSpec& ns, const OuterArgs& a,
                    const LaunchCfg& c, cudaStream_t s) {
    if (c.R == 2) outer_dispatch_r<S, 2>(g, links, nb, ns, a, c, s);
    else outer_dispatch_r<S, 1>(g, links, nb, ns, a, c, s);
}

}  // namespace mpmc
