// Device building blocks of the GB300 hot path: complex arithmetic,
// storage formats, Philox-4x32-10 Z4 noise and the Wilson hopping term
// with half-spinor projection.  Only the CUDA path includes this file.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace mpmc {

// ---------------------------------------------------------------- complex
template <class T> struct cplx { T re, im; };

template <class T> __device__ __forceinline__ cplx<T> cz() { return {T(0), T(0)}; }
template <class T> __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a) { return {-a.re, -a.im}; }
template <class T> __device__ __forceinline__ cplx<T> mul(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <class T> __device__ __forceinline__ cplx<T> times_i(cplx<T> a) { return {-a.im, a.re}; }
template <class T> __device__ __forceinline__ cplx<T> times_mi(cplx<T> a) { return {a.im, -a.re}; }
template <class T> __device__ __forceinline__ cplx<T> scale(cplx<T> a, T s) { return {a.re * s, a.im * s}; }

// ---------------------------------------------------------------- storage
// A complex number is stored as two consecutive S values; arithmetic runs
// in Math<S>::T (double for FP64 storage, float otherwise).
template <class S> struct Math;
template <> struct Math<double> { using T = double; };
template <> struct Math<float> { using T = float; };
template <> struct Math<__nv_bfloat16> { using T = float; };

__device__ __forceinline__ cplx<double> ld(const double* p) {
    double2 v = *reinterpret_cast<const double2*>(p);
    return {v.x, v.y};
}
__device__ __forceinline__ cplx<float> ld(const float* p) {
    float2 v = *reinterpret_cast<const float2*>(p);
    return {v.x, v.y};
}
__device__ __forceinline__ cplx<float> ld(const __nv_bfloat16* p) {
    __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
    float2 f = __bfloat1622float2(v);
    return {f.x, f.y};
}
__device__ __forceinline__ void st(double* p, cplx<double> a) {
    *reinterpret_cast<double2*>(p) = make_double2(a.re, a.im);
}
__device__ __forceinline__ void st(float* p, cplx<float> a) {
    *reinterpret_cast<float2*>(p) = make_float2(a.re, a.im);
}
__device__ __forceinline__ void st(__nv_bfloat16* p, cplx<float> a) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a.re, a.im);
}

// ------------------------------------------------------------------ stochastic rounding to BF16
// Round-to-nearest of the chain vectors to BF16 leaves an error that is a fixed function of the
// stored value; when the values follow the noise vector (w = c b + neighbour terms) the error
// correlates with b and b^H p(A) b acquires a bias of ~1e-3 of its size.  The BF16 chain stores
// therefore round stochastically (the hardware conversion with random bits): up or down with
// probabilities that make every rounding error zero-mean given the value, so the chain's
// expectation is that of the unrounded arithmetic.  The random bits are a hash of the element
// index and a per-step salt: results stay deterministic.
__device__ __forceinline__ uint32_t sr_hash(uint32_t x) {   // integer mixing (xor-shift-multiply)
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// (re, im) -> two BF16 rounded stochastically with the random bits rb; re in the low half
__device__ __forceinline__ uint32_t bf16x2_sr(float re, float im, uint32_t rb) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(im), "f"(re), "r"(rb));
    return d;
}
// Stores of a storage format with stochastic rounding where it narrows (BF16); exact otherwise
__device__ __forceinline__ void st_sr(double* p, cplx<double> a, uint32_t) { st(p, a); }
__device__ __forceinline__ void st_sr(float* p, cplx<float> a, uint32_t) { st(p, a); }
__device__ __forceinline__ void st_sr(__nv_bfloat16* p, cplx<float> a, uint32_t rb) {
    *reinterpret_cast<uint32_t*>(p) = bf16x2_sr(a.re, a.im, rb);
}
// random bits of component e of the element group whose hash is h (one hash per site and column)
__device__ __forceinline__ uint32_t sr_bits(uint32_t h, int e) { return h + (uint32_t)e * 0x9E3779B9u; }
__device__ __forceinline__ uint32_t sr_seed(uint32_t salt, uint32_t site, uint32_t col) {
    return sr_hash(salt ^ sr_hash(site * 0x27d4eb2fu + col));
}

// ---------------------------------------------------------------- Philox
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers
// 0xD2511F53 and 0xCD9E8D57, key increments 0x9E3779B9 and 0xBB67AE85,
// ten rounds, key bumped between rounds.  Only output word 0 is used.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return c0;
}

struct NoiseKey {
    uint32_t k0, k1;   // seed low / high words
    uint32_t level;    // counter word 2
    uint32_t j0;       // noise index of block column 0 (counter word 0 = j0 + column)
};

// Packed Z4 symbols of (site, column): entry e is bits 2e..2e+1.
__device__ __forceinline__ uint32_t z4_word(const NoiseKey& nk, int site, int col) {
    return philox_word0(nk.j0 + (uint32_t)col, (uint32_t)site, nk.level, 0u, nk.k0, nk.k1);
}

// i^q
template <class T> __device__ __forceinline__ cplx<T> z4_value(uint32_t q) {
    const T one = T(1);
    switch (q & 3u) {
        case 0: return {one, T(0)};
        case 1: return {T(0), one};
        case 2: return {-one, T(0)};
        default: return {T(0), -one};
    }
}
// conj(i^q) * w
template <class T> __device__ __forceinline__ cplx<T> z4_conj_mul(uint32_t q, cplx<T> w) {
    switch (q & 3u) {
        case 0: return w;
        case 1: return times_mi(w);
        case 2: return -w;
        default: return times_i(w);
    }
}

// ---------------------------------------------------------------- lattice
struct Lattice {
    int lx, ly, lz, lt;
    int V;
    int bc_t;   // +1 periodic, -1 antiperiodic in t
};

struct Nbrs {
    int fwd[4], bwd[4];
    bool fwd_wrap_t, bwd_wrap_t;
};

__device__ __forceinline__ Nbrs neighbours(const Lattice& L, int s) {
    const int x = s % L.lx;
    int r = s / L.lx;
    const int y = r % L.ly;
    r /= L.ly;
    const int z = r % L.lz;
    const int t = r / L.lz;
    const int sx = 1, sy = L.lx, sz = L.lx * L.ly, stt = L.lx * L.ly * L.lz;
    Nbrs n;
    n.fwd[0] = s + (x + 1 < L.lx ? sx : sx - L.lx * sx);
    n.bwd[0] = s - (x > 0 ? sx : sx - L.lx * sx);
    n.fwd[1] = s + (y + 1 < L.ly ? sy : sy - L.ly * sy);
    n.bwd[1] = s - (y > 0 ? sy : sy - L.ly * sy);
    n.fwd[2] = s + (z + 1 < L.lz ? sz : sz - L.lz * sz);
    n.bwd[2] = s - (z > 0 ? sz : sz - L.lz * sz);
    n.fwd[3] = s + (t + 1 < L.lt ? stt : stt - L.lt * stt);
    n.bwd[3] = s - (t > 0 ? stt : stt - L.lt * stt);
    n.fwd_wrap_t = (t + 1 == L.lt);
    n.bwd_wrap_t = (t == 0);
    return n;
}

// ---------------------------------------------------------------- spinors
// Block layout: element (site, e, column) at ((site*12 + e)*nb + column)
// complex numbers.  A "source" yields the 12 components of a column at a
// site either from memory or, for the first step of a chain, as noise.
template <class S> struct MemSource {
    const S* p;
    int nb;
    __device__ __forceinline__ void get(int site, int col, cplx<typename Math<S>::T> (&v)[12]) const {
        const S* q = p + ((size_t)site * 12 * nb + col) * 2;
#pragma unroll
        for (int e = 0; e < 12; ++e) v[e] = ld(q + (size_t)e * nb * 2);
    }
};

template <class T> struct NoiseSource {
    NoiseKey nk;
    __device__ __forceinline__ void get(int site, int col, cplx<T> (&v)[12]) const {
        const uint32_t w = z4_word(nk, site, col);
#pragma unroll
        for (int e = 0; e < 12; ++e) v[e] = z4_value<T>(w >> (2 * e));
    }
};

// ---------------------------------------------------------------- links
// Device links: [site][mu][a][b] complex in the math precision.
template <class T> __device__ __forceinline__ void load_link(const T* U, int site, int mu, cplx<T> (&u)[9]) {
    const T* q = U + ((size_t)site * 4 + mu) * 18;
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = ld(q + 2 * i);
}

// g = U h (a = row)
template <class T> __device__ __forceinline__ void su3_mul(const cplx<T> (&u)[9], const cplx<T>* h, cplx<T>* g) {
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] = mul(u[3 * a], h[0]) + mul(u[3 * a + 1], h[1]) + mul(u[3 * a + 2], h[2]);
}
// g = U^+ h
template <class T> __device__ __forceinline__ void su3_adj_mul(const cplx<T> (&u)[9], const cplx<T>* h, cplx<T>* g) {
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] = cmul(u[a], h[0]) + cmul(u[3 + a], h[1]) + cmul(u[6 + a], h[2]);
}

// One hop of the Wilson term with the spin projector (1 - gamma_mu)
// (forward, FWD = true, U = U_mu(x), psi = psi(x+mu)) or (1 + gamma_mu)
// (backward, U^+ = U_mu(x-mu)^+, psi = psi(x-mu)), accumulated into acc.
// Chiral DeGrand-Rossi basis; each projector has rank 2, so only the
// half spinor (h0, h1) is multiplied by the link and the lower two spin
// components are rebuilt from it.  sgn is the boundary sign (+1 or -1).
template <int MU, bool FWD, class T>
__device__ __forceinline__ void hop(const cplx<T> (&psi)[12], const cplx<T> (&u)[9], T sgn, cplx<T> (&acc)[12]) {
    cplx<T> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<T> p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
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
        h0[c] = scale(h0[c], sgn);
        h1[c] = scale(h1[c], sgn);
    }
    cplx<T> g0[3], g1[3];
    if (FWD) { su3_mul(u, h0, g0); su3_mul(u, h1, g1); }
    else     { su3_adj_mul(u, h0, g0); su3_adj_mul(u, h1, g1); }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = acc[c] + g0[c];
        acc[3 + c] = acc[3 + c] + g1[c];
        if (MU == 0) {
            if (FWD) { acc[6 + c] = acc[6 + c] + times_i(g1[c]);  acc[9 + c] = acc[9 + c] + times_i(g0[c]); }
            else     { acc[6 + c] = acc[6 + c] + times_mi(g1[c]); acc[9 + c] = acc[9 + c] + times_mi(g0[c]); }
        } else if (MU == 1) {
            if (FWD) { acc[6 + c] = acc[6 + c] - g1[c]; acc[9 + c] = acc[9 + c] + g0[c]; }
            else     { acc[6 + c] = acc[6 + c] + g1[c]; acc[9 + c] = acc[9 + c] - g0[c]; }
        } else if (MU == 2) {
            if (FWD) { acc[6 + c] = acc[6 + c] + times_i(g0[c]);  acc[9 + c] = acc[9 + c] + times_mi(g1[c]); }
            else     { acc[6 + c] = acc[6 + c] + times_mi(g0[c]); acc[9 + c] = acc[9 + c] + times_i(g1[c]); }
        } else {
            if (FWD) { acc[6 + c] = acc[6 + c] - g0[c]; acc[9 + c] = acc[9 + c] - g1[c]; }
            else     { acc[6 + c] = acc[6 + c] + g0[c]; acc[9 + c] = acc[9 + c] + g1[c]; }
        }
    }
}

// (H psi)(site) for one column, neighbours from a source.
template <class T, class Src>
__device__ __forceinline__ void wilson_hopping(const Lattice& L, const T* U, const Src& src, int site, int col,
                                               cplx<T> (&acc)[12]) {
    const Nbrs nb = neighbours(L, site);
#pragma unroll
    for (int e = 0; e < 12; ++e) acc[e] = cz<T>();
    cplx<T> psi[12], u[9];
    const T one = T(1);
    const T sf = (nb.fwd_wrap_t && L.bc_t < 0) ? -one : one;
    const T sb = (nb.bwd_wrap_t && L.bc_t < 0) ? -one : one;

    src.get(nb.fwd[0], col, psi); load_link(U, site, 0, u); hop<0, true>(psi, u, one, acc);
    src.get(nb.bwd[0], col, psi); load_link(U, nb.bwd[0], 0, u); hop<0, false>(psi, u, one, acc);
    src.get(nb.fwd[1], col, psi); load_link(U, site, 1, u); hop<1, true>(psi, u, one, acc);
    src.get(nb.bwd[1], col, psi); load_link(U, nb.bwd[1], 1, u); hop<1, false>(psi, u, one, acc);
    src.get(nb.fwd[2], col, psi); load_link(U, site, 2, u); hop<2, true>(psi, u, one, acc);
    src.get(nb.bwd[2], col, psi); load_link(U, nb.bwd[2], 2, u); hop<2, false>(psi, u, one, acc);
    src.get(nb.fwd[3], col, psi); load_link(U, site, 3, u); hop<3, true>(psi, u, sf, acc);
    src.get(nb.bwd[3], col, psi); load_link(U, nb.bwd[3], 3, u); hop<3, false>(psi, u, sb, acc);
}

}  // namespace mpmc
