// CUDA kernels of the GB300 hot path (sm_103a): the root-form polynomial
// step fused into the multi-RHS Wilson stencil, the composite outer step,
// the level-sample assembly, the deflation dot products, and the FP64
// vector kernels of the Krylov setup.
#include "device.cuh"
#include "kernels.h"

#include <algorithm>

namespace mpmc {

namespace {

template <class T> __device__ __forceinline__ cplx<T> cdv(const double (&v)[2]) { return {T(v[0]), T(v[1])}; }

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

NoiseKey make_key(const NoiseSpec& ns) {
    NoiseKey k;
    k.k0 = (uint32_t)(ns.seed & 0xffffffffu);
    k.k1 = (uint32_t)(ns.seed >> 32);
    k.level = ns.level;
    k.j0 = ns.j0;
    return k;
}

Lattice make_lat(const Geom& g) {
    Lattice L;
    L.lx = g.lx; L.ly = g.ly; L.lz = g.lz; L.lt = g.lt; L.V = g.V; L.bc_t = g.bc_t;
    return L;
}

// ------------------------------------------------------------------ elementwise
template <class S>
__global__ void k_fill_noise(int V, int nb, NoiseKey nk, double sre, double sim, S* out) {
    using T = typename Math<S>::T;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)V * nb) return;
    const int site = (int)(idx / nb), col = (int)(idx % nb);
    const uint32_t w = z4_word(nk, site, col);
    const cplx<T> sc = {T(sre), T(sim)};
    S* p = out + ((size_t)site * 12 * nb + col) * 2;
#pragma unroll
    for (int e = 0; e < 12; ++e) st(p + (size_t)e * nb * 2, mul(sc, z4_value<T>(w >> (2 * e))));
}

__global__ void k_noise_f64(int V, NoiseKey nk, int cnt, int ld_, int c0, double* out) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)V * cnt) return;
    const int site = (int)(idx / cnt), col = (int)(idx % cnt);
    const uint32_t w = z4_word(nk, site, col);
    double* p = out + ((size_t)site * 12 * ld_ + c0 + col) * 2;
#pragma unroll
    for (int e = 0; e < 12; ++e) {
        const cplx<double> v = z4_value<double>(w >> (2 * e));
        p[(size_t)e * ld_ * 2] = v.re;
        p[(size_t)e * ld_ * 2 + 1] = v.im;
    }
}

template <class S>
__global__ void k_import(size_t nrow, const double* __restrict__ src, int ld_, int c0, int cnt, S* dst, int nb) {
    using T = typename Math<S>::T;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrow * nb) return;
    const size_t row = idx / nb;
    const int col = (int)(idx % nb);
    cplx<T> v = cz<T>();
    if (col < cnt) {
        const double* p = src + (row * ld_ + c0 + col) * 2;
        v = {T(p[0]), T(p[1])};
    }
    st(dst + idx * 2, v);
}

template <class S>
__global__ void k_export(size_t nrow, const S* __restrict__ src, int nb, double* dst, int ld_, int c0, int cnt) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrow * cnt) return;
    const size_t row = idx / cnt;
    const int col = (int)(idx % cnt);
    const auto v = ld(src + (row * nb + col) * 2);
    double* p = dst + (row * ld_ + c0 + col) * 2;
    p[0] = (double)v.re;
    p[1] = (double)v.im;
}

template <class S>
__global__ void k_scale(size_t n, const S* __restrict__ in, double sre, double sim, S* out, uint32_t salt) {
    using T = typename Math<S>::T;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const cplx<T> sc = {T(sre), T(sim)};
    st_sr(out + idx * 2, mul(sc, ld(in + idx * 2)), sr_hash(salt ^ sr_hash((uint32_t)idx)));
}

template <class T>
__global__ void k_links(int V, const double* __restrict__ src, double scale, T* dst) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // (site, mu, i)
    if (idx >= (size_t)V * 36) return;
    const int i = (int)(idx % 9);
    const int mu = (int)((idx / 9) % 4);
    const size_t site = idx / 36;
    const double* p = src + (((size_t)mu * V + site) * 9 + i) * 2;
    dst[idx * 2] = (T)(scale * p[0]);
    dst[idx * 2 + 1] = (T)(scale * p[1]);
}

template <class T>
__global__ void k_convert(size_t n, const double* __restrict__ src, T* dst) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * n) return;
    dst[idx] = (T)src[idx];
}

// ------------------------------------------------------------------ finalize
// One CTA per 32 columns; the accumulator rows are split into FIN_RG
// contiguous chunks summed in order, then the chunk sums are added in order:
// a fixed summation order independent of scheduling.
constexpr int FIN_RG = 16;

__global__ void __launch_bounds__(32 * FIN_RG) k_finalize(int ncta, int nb, int nvalid,
                                                          const double2* __restrict__ acc_hi,
                                                          const double2* __restrict__ acc_lo, double2 chi, double2 clo,
                                                          const double2* __restrict__ dterm, double2* samples,
                                                          double2* hi, double2* lo,
                                                          const double2* __restrict__ add_hi) {
    __shared__ double2 red[2][FIN_RG][32];
    const int col = blockIdx.x * 32 + threadIdx.x;
    const int chunk = (ncta + FIN_RG - 1) / FIN_RG;
    const int b0 = threadIdx.y * chunk, b1 = min(ncta, b0 + chunk);
    double2 h = make_double2(0, 0), l = make_double2(0, 0);
    if (col < nvalid) {
        for (int b = b0; b < b1; ++b) h = cadd(h, acc_hi[(size_t)b * nb + col]);
        if (acc_lo)
            for (int b = b0; b < b1; ++b) l = cadd(l, acc_lo[(size_t)b * nb + col]);
    }
    red[0][threadIdx.y][threadIdx.x] = h;
    red[1][threadIdx.y][threadIdx.x] = l;
    __syncthreads();
    if (threadIdx.y != 0 || col >= nvalid) return;
    h = chi;
    l = clo;
    if (add_hi) h = cadd(h, add_hi[col]);
    for (int g = 0; g < FIN_RG; ++g) {
        h = cadd(h, red[0][g][threadIdx.x]);
        l = cadd(l, red[1][g][threadIdx.x]);
    }
    double2 s = make_double2(h.x - l.x, h.y - l.y);
    if (dterm) s = make_double2(s.x - dterm[col].x, s.y - dterm[col].y);
    samples[col] = s;
    if (hi) hi[col] = h;
    if (lo) lo[col] = l;
}

// ------------------------------------------------------------------ deflation dots
// CTA: 32 noise columns x 4 site lanes; KT eigenvectors per CTA.  Each
// thread sums, over its sites, conj(z_i) * b separately over the upper
// (spin 0, 1) and lower (spin 2, 3) half: G1 = up + low, G2 = up - low
// (gamma5 = diag(1, 1, -1, -1)).
constexpr int DEFL_KT = 8;

template <class T>
__global__ void __launch_bounds__(128) k_defl_dots(int V, int k, const T* __restrict__ Z, int nb, NoiseKey nk,
                                                   double2* part, int nsplit) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    const int i0 = blockIdx.y * DEFL_KT;
    const int split = blockIdx.z;
    const int chunk = (V + nsplit - 1) / nsplit;
    const int s0 = split * chunk, s1 = min(V, s0 + chunk);
    cplx<T> up[DEFL_KT], lo[DEFL_KT];
#pragma unroll
    for (int q = 0; q < DEFL_KT; ++q) { up[q] = cz<T>(); lo[q] = cz<T>(); }
    const bool colok = col < nb;
    for (int site = s0 + threadIdx.y; site < s1 && colok; site += blockDim.y) {
        const uint32_t w = z4_word(nk, site, col);
#pragma unroll
        for (int q = 0; q < DEFL_KT; ++q) {
            const int i = i0 + q;
            if (i >= k) break;
            const T* zp = Z + ((size_t)i * V + site) * 24;
#pragma unroll
            for (int e = 0; e < 12; ++e) {
                const cplx<T> z = ld(zp + 2 * e);
                // conj(z) * i^q
                const cplx<T> t = mul(cplx<T>{z.re, -z.im}, z4_value<T>(w >> (2 * e)));
                if (e < 6) up[q] = up[q] + t; else lo[q] = lo[q] + t;
            }
        }
    }
    __shared__ double2 red[128][2];
    const int tid = threadIdx.y * 32 + threadIdx.x;
#pragma unroll
    for (int q = 0; q < DEFL_KT; ++q) {
        red[tid][0] = make_double2((double)up[q].re, (double)up[q].im);
        red[tid][1] = make_double2((double)lo[q].re, (double)lo[q].im);
        __syncthreads();
        if (threadIdx.y == 0 && colok && i0 + q < k) {
            double2 u = make_double2(0, 0), l = make_double2(0, 0);
            for (int yy = 0; yy < (int)blockDim.y; ++yy) {
                u = cadd(u, red[yy * 32 + threadIdx.x][0]);
                l = cadd(l, red[yy * 32 + threadIdx.x][1]);
            }
            double2* p = part + (((size_t)split * k + (i0 + q)) * nb + col) * 2;
            p[0] = make_double2(u.x + l.x, u.y + l.y);
            p[1] = make_double2(u.x - l.x, u.y - l.y);
        }
        __syncthreads();
    }
}

__global__ void k_defl_sum(int k, int nb, int nsplit, const double2* __restrict__ part, double2* G1, double2* G2) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)k * nb) return;
    double2 g1 = make_double2(0, 0), g2 = make_double2(0, 0);
    for (int s = 0; s < nsplit; ++s) {
        const double2* p = part + (((size_t)s * k) * nb + idx) * 2;
        g1 = cadd(g1, p[0]);
        g2 = cadd(g2, p[1]);
    }
    G1[idx] = g1;
    G2[idx] = g2;
}

__global__ void k_defl_term(int k, int nb, const double2* __restrict__ coef, const int* __restrict__ pair,
                            const double2* __restrict__ G1, const double2* __restrict__ G2, double2* term) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= nb) return;
    double2 s = make_double2(0, 0);
    for (int i = 0; i < k; ++i) {
        const double2 bz = conjd(G1[(size_t)i * nb + col]);           // b^H z_i
        const double2 ub = G2[(size_t)pair[i] * nb + col];            // z_pair^H gamma5 b
        s = cadd(s, cmuld(coef[i], cmuld(bz, ub)));
    }
    term[col] = s;
}

template <class T>
__global__ void k_defl_norms(int V, int k, const T* __restrict__ Z, const int* __restrict__ pair, double2* d) {
    // one CTA per i; fixed-order tree over the CTA
    const int i = blockIdx.x;
    const T* zi = Z + (size_t)i * V * 24;
    const T* zp = Z + (size_t)pair[i] * V * 24;
    double sr = 0, si = 0;
    for (size_t p = threadIdx.x; p < (size_t)V * 12; p += blockDim.x) {
        const double ar = zp[2 * p], ai = zp[2 * p + 1], br = zi[2 * p], bi = zi[2 * p + 1];
        const double g = ((p % 12) < 6) ? 1.0 : -1.0;
        sr += g * (ar * br + ai * bi);
        si += g * (ar * bi - ai * br);
    }
    __shared__ double rr[256], ri[256];
    rr[threadIdx.x] = sr;
    ri[threadIdx.x] = si;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) { rr[threadIdx.x] += rr[threadIdx.x + w]; ri[threadIdx.x] += ri[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) d[i] = make_double2(rr[0], ri[0]);
}

// ------------------------------------------------------------------ FP64 Krylov vectors
constexpr int MDOT_THREADS = 256;

__global__ void k_mdot_part(size_t n, int m, const double2* __restrict__ Vb, const double2* __restrict__ w,
                            double2* part) {
    __shared__ double2 red[MDOT_THREADS];
    const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const size_t p0 = blockIdx.x * chunk, p1 = min(n, p0 + chunk);
    for (int j = 0; j < m; ++j) {
        const double2* v = Vb + (size_t)j * n;
        double2 s = make_double2(0, 0);
        for (size_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) s = cadd(s, cmuld(conjd(v[p]), w[p]));
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + h]);
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * m + j] = red[0];
        __syncthreads();
    }
}

__global__ void k_mdot_sum(int nparts, int m, const double2* __restrict__ part, double2* h) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double2 s = make_double2(0, 0);
    for (int b = 0; b < nparts; ++b) s = cadd(s, part[(size_t)b * m + j]);
    h[j] = s;
}

__global__ void k_maxpy(size_t n, int m, const double2* __restrict__ Vb, const double2* __restrict__ h, double2* w) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double2 s = w[p];
    for (int j = 0; j < m; ++j) {
        const double2 t = cmuld(h[j], Vb[(size_t)j * n + p]);
        s = make_double2(s.x - t.x, s.y - t.y);
    }
    w[p] = s;
}

__global__ void k_norm2_part(size_t n, const double2* __restrict__ w, double* part) {
    __shared__ double red[MDOT_THREADS];
    double s = 0;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        s += w[p].x * w[p].x + w[p].y * w[p].y;
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_scalar(int nparts, const double* __restrict__ part, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0;
        for (int b = 0; b < nparts; ++b) s += part[b];
        *out = s;
    }
}

__global__ void k_normalize(size_t n, const double2* __restrict__ w, const double* __restrict__ nrm2, double2* dst) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double inv = 1.0 / sqrt(*nrm2);
    dst[p] = make_double2(w[p].x * inv, w[p].y * inv);
}

__global__ void k_combine(size_t n, int m, const double2* __restrict__ Vb, const double2* __restrict__ Y, int k,
                          double2* Z) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (p >= n) return;
    double2 s = make_double2(0, 0);
    for (int j = 0; j < m; ++j) s = cadd(s, cmuld(Vb[(size_t)j * n + p], Y[(size_t)j * k + i]));
    Z[(size_t)i * n + p] = s;
}

inline unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------ probing
// Probe vectors of the period-m distance colouring: column q = 12 * colour + e,
// colour = x%m + m (y%m) + m^2 (z%m) + m^3 (t%m).
__device__ __forceinline__ int probe_colour(int site, int lx, int ly, int lz, int m) {
    const int x = site % lx;
    int r = site / lx;
    const int y = r % ly;
    r /= ly;
    const int z = r % lz;
    const int t = r / lz;
    return (x % m) + m * ((y % m) + m * ((z % m) + m * (t % m)));
}

// Colour of a site: from a per-site table (any distance colouring) or, without one,
// the period-m formula.
__device__ __forceinline__ int site_colour(const int* tab, int site, int lx, int ly, int lz, int m) {
    return tab ? __ldg(tab + site) : probe_colour(site, lx, ly, lz, m);
}

template <class S>
__global__ void k_probe_block(int V, int lx, int ly, int lz, int m, const int* __restrict__ tab, int q0, int nq,
                              int nb, S* __restrict__ out) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // (site, e, col)
    if (idx >= (size_t)V * 12 * nb) return;
    const int col = (int)(idx % nb);
    const int e = (int)((idx / nb) % 12);
    const int site = (int)(idx / ((size_t)12 * nb));
    const int q = q0 + col;
    const bool one = col < nq && e == q % 12 && site_colour(tab, site, lx, ly, lz, m) == q / 12;
    using T = typename Math<S>::T;
    st(out + idx * 2, cplx<T>{one ? T(1) : T(0), T(0)});
}

// part[chunk][col] = sum over the chunk's sites of colour c(q) of X[site][e(q)][col] (FP64, site order)
template <class S>
__global__ void k_probe_dot(int V, int lx, int ly, int lz, int m, const int* __restrict__ tab, int q0, int nq, int nb,
                            int nchunk, const S* __restrict__ X, double2* __restrict__ part) {
    const int col = blockIdx.y * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.x;
    if (col >= nb) return;
    double sr = 0.0, si = 0.0;
    if (col < nq) {
        const int q = q0 + col, c = q / 12, e = q % 12;
        const int per = (V + nchunk - 1) / nchunk;
        const int s1 = min(V, (chunk + 1) * per);
        for (int site = chunk * per; site < s1; ++site) {
            if (site_colour(tab, site, lx, ly, lz, m) != c) continue;
            const auto v = ld(X + (((size_t)site * 12 + e) * nb + col) * 2);
            sr += (double)v.re;
            si += (double)v.im;
        }
    }
    part[(size_t)chunk * nb + col] = make_double2(sr, si);
}

// total += sum over columns (in order) of the chunk sums (in order): one thread
__global__ void k_probe_sum(int nchunk, int nb, int nq, const double2* __restrict__ part, double2* total) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double tr = total->x, ti = total->y;
    for (int col = 0; col < nq; ++col) {
        double sr = 0.0, si = 0.0;
        for (int ch = 0; ch < nchunk; ++ch) {
            sr += part[(size_t)ch * nb + col].x;
            si += part[(size_t)ch * nb + col].y;
        }
        tr += sr;
        ti += si;
    }
    *total = make_double2(tr, ti);
}

// ================================================================== host side
LaunchCfg chain_config(const Geom& g, int nb, int bx_max, int sl, int R) {
    LaunchCfg c;
    c.R = (R == 2 && nb % 2 == 0) ? 2 : 1;
    const int groups = nb / c.R;                        // column groups of R
    c.bx = std::min(groups, bx_max);
    c.by = std::max(1, 256 / c.bx);
    c.sl = std::max(1, sl);
    c.gx = (g.V + c.by * c.sl - 1) / (c.by * c.sl);   // site blocks (x: no 65535 limit)
    c.gy = (groups + c.bx - 1) / c.bx;                 // column blocks
    return c;
}

void fill_floats(StepArgs& a) {
    for (int i = 0; i < 2; ++i) {
        a.alphaf[i] = (float)a.alpha[i];
        a.yaf[i] = (float)a.ya[i];
        a.ybf[i] = (float)a.yb[i];
    }
    a.kappaf = (float)a.kappa;
}

void fill_floats(OuterArgs& a) {
    for (int i = 0; i < 2; ++i) {
        a.alphaf[i] = (float)a.alpha[i];
        a.betaf[i] = (float)a.beta[i];
        a.gammaf[i] = (float)a.gamma[i];
    }
    a.kappaf = (float)a.kappa;
}

void launch_step(int storage, const Geom& g, const void* links, int nb, const NoiseSpec& ns, const StepArgs& a0,
                 const LaunchCfg& c, cudaStream_t s) {
    StepArgs a = a0;
    fill_floats(a);
    if (storage == ST_F64) step_f64(g, links, nb, ns, a, c, s);
    else if (storage == ST_F32) step_f32(g, links, nb, ns, a, c, s);
    else step_bf16(g, links, nb, ns, a, c, s);
}

void launch_outer(int storage, const Geom& g, const void* links, int nb, const NoiseSpec& ns, const OuterArgs& a0,
                  const LaunchCfg& c, cudaStream_t s) {
    OuterArgs a = a0;
    fill_floats(a);
    if (storage == ST_F64) outer_f64(g, links, nb, ns, a, c, s);
    else if (storage == ST_F32) outer_f32(g, links, nb, ns, a, c, s);
    else outer_bf16(g, links, nb, ns, a, c, s);
}

void launch_fill_noise(int storage, const Geom& g, int nb, const NoiseSpec& ns, const double sc[2], void* out,
                       cudaStream_t s) {
    const size_t n = (size_t)g.V * nb;
    const NoiseKey nk = make_key(ns);
    if (storage == ST_F64) k_fill_noise<double><<<blocks_for(n, 256), 256, 0, s>>>(g.V, nb, nk, sc[0], sc[1], (double*)out);
    else if (storage == ST_F32) k_fill_noise<float><<<blocks_for(n, 256), 256, 0, s>>>(g.V, nb, nk, sc[0], sc[1], (float*)out);
    else k_fill_noise<__nv_bfloat16><<<blocks_for(n, 256), 256, 0, s>>>(g.V, nb, nk, sc[0], sc[1], (__nv_bfloat16*)out);
}

void launch_noise_f64(const Geom& g, const NoiseSpec& ns, int cnt, int ld_, int c0, double* out, cudaStream_t s) {
    const size_t n = (size_t)g.V * cnt;
    k_noise_f64<<<blocks_for(n, 256), 256, 0, s>>>(g.V, make_key(ns), cnt, ld_, c0, out);
}

void launch_import(int storage, int V, const double* src, int ld_, int c0, int cnt, void* dst, int nb,
                   cudaStream_t s) {
    const size_t nrow = (size_t)V * 12, n = nrow * nb;
    if (storage == ST_F64) k_import<double><<<blocks_for(n, 256), 256, 0, s>>>(nrow, src, ld_, c0, cnt, (double*)dst, nb);
    else if (storage == ST_F32) k_import<float><<<blocks_for(n, 256), 256, 0, s>>>(nrow, src, ld_, c0, cnt, (float*)dst, nb);
    else k_import<__nv_bfloat16><<<blocks_for(n, 256), 256, 0, s>>>(nrow, src, ld_, c0, cnt, (__nv_bfloat16*)dst, nb);
}

void launch_export(int storage, int V, const void* src, int nb, double* dst, int ld_, int c0, int cnt,
                   cudaStream_t s) {
    const size_t nrow = (size_t)V * 12, n = nrow * cnt;
    if (storage == ST_F64) k_export<double><<<blocks_for(n, 256), 256, 0, s>>>(nrow, (const double*)src, nb, dst, ld_, c0, cnt);
    else if (storage == ST_F32) k_export<float><<<blocks_for(n, 256), 256, 0, s>>>(nrow, (const float*)src, nb, dst, ld_, c0, cnt);
    else k_export<__nv_bfloat16><<<blocks_for(n, 256), 256, 0, s>>>(nrow, (const __nv_bfloat16*)src, nb, dst, ld_, c0, cnt);
}

void launch_scale(int storage, size_t ncplx, const void* in, const double sc[2], void* out, cudaStream_t s,
                  uint32_t salt) {
    const size_t n = ncplx;
    if (storage == ST_F64) k_scale<double><<<blocks_for(n, 256), 256, 0, s>>>(n, (const double*)in, sc[0], sc[1], (double*)out, salt);
    else if (storage == ST_F32) k_scale<float><<<blocks_for(n, 256), 256, 0, s>>>(n, (const float*)in, sc[0], sc[1], (float*)out, salt);
    else k_scale<__nv_bfloat16><<<blocks_for(n, 256), 256, 0, s>>>(n, (const __nv_bfloat16*)in, sc[0], sc[1], (__nv_bfloat16*)out, salt);
}

void launch_links(int storage, int V, const double* src, void* dst, cudaStream_t s, double scale) {
    const size_t n = (size_t)V * 36;
    if (storage == ST_F64) k_links<double><<<blocks_for(n, 256), 256, 0, s>>>(V, src, scale, (double*)dst);
    else k_links<float><<<blocks_for(n, 256), 256, 0, s>>>(V, src, scale, (float*)dst);
}

void launch_convert_vectors(int storage, size_t ncplx, const double* src, void* dst, cudaStream_t s) {
    if (storage == ST_F64) k_convert<double><<<blocks_for(2 * ncplx, 256), 256, 0, s>>>(ncplx, src, (double*)dst);
    else k_convert<float><<<blocks_for(2 * ncplx, 256), 256, 0, s>>>(ncplx, src, (float*)dst);
}

void launch_finalize(int ncta, int nb, int nvalid, const double2* acc_hi, const double2* acc_lo, const double c_hi[2],
                     const double c_lo[2], const double2* dterm, double2* samples, double2* hi, double2* lo,
                     cudaStream_t s, const double2* add_hi) {
    k_finalize<<<blocks_for(nvalid, 32), dim3(32, FIN_RG), 0, s>>>(ncta, nb, nvalid, acc_hi, acc_lo,
                                                                    make_double2(c_hi[0], c_hi[1]),
                                                                    make_double2(c_lo[0], c_lo[1]), dterm, samples, hi, lo,
                                                                    add_hi);
}

int defl_nsplit(int V) { return std::max(1, std::min(64, V / 128)); }

void launch_defl_dots(int storage, const Geom& g, int k, const void* Z, int nb, const NoiseSpec& ns, double2* part,
                      int nsplit, cudaStream_t s) {
    const dim3 grid((nb + 31) / 32, (k + DEFL_KT - 1) / DEFL_KT, nsplit), block(32, 4);
    if (storage == ST_F64) k_defl_dots<double><<<grid, block, 0, s>>>(g.V, k, (const double*)Z, nb, make_key(ns), part, nsplit);
    else k_defl_dots<float><<<grid, block, 0, s>>>(g.V, k, (const float*)Z, nb, make_key(ns), part, nsplit);
}

void launch_defl_reduce(int k, int nb, int nsplit, const double2* part, const double2* coef, const int* pair,
                        double2* G1, double2* G2, double2* term, cudaStream_t s) {
    const size_t n = (size_t)k * nb;
    k_defl_sum<<<blocks_for(n, 256), 256, 0, s>>>(k, nb, nsplit, part, G1, G2);
    k_defl_term<<<blocks_for(nb, 128), 128, 0, s>>>(k, nb, coef, pair, G1, G2, term);
}

void launch_defl_term(int k, int nb, const double2* coef, const int* pair, const double2* G1, const double2* G2,
                      double2* term, cudaStream_t s) {
    k_defl_term<<<blocks_for(nb, 128), 128, 0, s>>>(k, nb, coef, pair, G1, G2, term);
}

void launch_defl_norms(int storage, int V, int k, const void* Z, const int* pair, double2* d, cudaStream_t s) {
    if (storage == ST_F64) k_defl_norms<double><<<k, 256, 0, s>>>(V, k, (const double*)Z, pair, d);
    else k_defl_norms<float><<<k, 256, 0, s>>>(V, k, (const float*)Z, pair, d);
}

int mdot_parts(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>(304, n / 1024)); }

void launch_mdot(size_t n, int m, const double2* Vb, const double2* w, double2* part, double2* h, cudaStream_t s) {
    const int np = mdot_parts(n);
    k_mdot_part<<<np, MDOT_THREADS, 0, s>>>(n, m, Vb, w, part);
    k_mdot_sum<<<blocks_for(m, 128), 128, 0, s>>>(np, m, part, h);
}

void launch_maxpy(size_t n, int m, const double2* Vb, const double2* h, double2* w, cudaStream_t s) {
    k_maxpy<<<blocks_for(n, 256), 256, 0, s>>>(n, m, Vb, h, w);
}

void launch_norm2(size_t n, const double2* w, double* part, double* out, cudaStream_t s) {
    const int np = mdot_parts(n);
    k_norm2_part<<<np, MDOT_THREADS, 0, s>>>(n, w, part);
    k_sum_scalar<<<1, 32, 0, s>>>(np, part, out);
}

void launch_normalize(size_t n, const double2* w, const double* nrm2, double2* dst, cudaStream_t s) {
    k_normalize<<<blocks_for(n, 256), 256, 0, s>>>(n, w, nrm2, dst);
}

void launch_combine(size_t n, int m, const double2* Vb, const double2* Y, int k, double2* Z, cudaStream_t s) {
    const dim3 grid(blocks_for(n, 256), k);
    k_combine<<<grid, 256, 0, s>>>(n, m, Vb, Y, k, Z);
}

}  // namespace mpmc

namespace mpmc {

void launch_probe_block(int storage, const Geom& g, int m, const int* tab, int q0, int nq, int nb, void* out,
                        cudaStream_t s) {
    const size_t n = (size_t)g.V * 12 * nb;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (storage == ST_F64)
        k_probe_block<double><<<blocks, 256, 0, s>>>(g.V, g.lx, g.ly, g.lz, m, tab, q0, nq, nb, (double*)out);
    else if (storage == ST_F32)
        k_probe_block<float><<<blocks, 256, 0, s>>>(g.V, g.lx, g.ly, g.lz, m, tab, q0, nq, nb, (float*)out);
    else
        k_probe_block<__nv_bfloat16><<<blocks, 256, 0, s>>>(g.V, g.lx, g.ly, g.lz, m, tab, q0, nq, nb,
                                                           (__nv_bfloat16*)out);
}

void launch_probe_trace(int storage, const Geom& g, int m, const int* tab, int q0, int nq, int nb, const void* X,
                        int nchunk, double2* part, double2* total, cudaStream_t s) {
    const dim3 grid(nchunk, (nb + 63) / 64);
    if (storage == ST_F64)
        k_probe_dot<double><<<grid, 64, 0, s>>>(g.V, g.lx, g.ly, g.lz, m, tab, q0, nq, nb, nchunk, (const double*)X,
                                                part);
    else if (storage == ST_F32)
        k_probe_dot<float><<<grid, 64, 0, s>>>(g.V, g.lx, g.ly, g.lz, m, tab, q0, nq, nb, nchunk, (const float*)X,
                                               part);
    else
        k_probe_dot<__nv_bfloat16><<<grid, 64, 0, s>>>(g.V, g.lx, g.ly, g.lz, m, tab, q0, nq, nb, nchunk,
                                                      (const __nv_bfloat16*)X, part);
    k_probe_sum<<<1, 32, 0, s>>>(nchunk, nb, nq, part, total);
}

}  // namespace mpmc
