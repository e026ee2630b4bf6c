// Instantiations and host side of the issue-lean stencil kernels
// (stencil_fast.cuh): per-block Z4 word table, expanded links, launcher.
#include "stencil_fast.cuh"

namespace mpmc {

namespace {

__global__ void k_noise_words(int V, int nb, NoiseKey nk, uint32_t* __restrict__ out) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)V * nb) return;
    const int col = (int)(idx % nb);
    const int site = (int)(idx / nb);
    out[idx] = z4_word(nk, site, col);
}

__global__ void k_links_expanded(int V, const double* __restrict__ src, double scale, float4* __restrict__ dst) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // (site, mu, i)
    if (idx >= (size_t)V * 36) return;
    const int i = (int)(idx % 9);
    const int mu = (int)((idx / 9) % 4);
    const size_t site = idx / 36;
    const double* p = src + (((size_t)mu * V + site) * 9 + i) * 2;
    const float re = (float)(scale * p[0]), im = (float)(scale * p[1]);
    dst[idx] = make_float4(re, re, im, im);
}

template <class S, int NB>
int launch_nb(int kind, const FastArgs& a, int gx, cudaStream_t s) {
    constexpr int TW = NB < 32 ? NB : 32;
    const dim3 grid(gx, NB / TW), block(TW, 256 / TW);
    switch (kind) {
        case 0: fast::k_fast<S, NB, 0><<<grid, block, 0, s>>>(a); break;
        case 1: fast::k_fast<S, NB, 1><<<grid, block, 0, s>>>(a); break;
        case 2: fast::k_fast<S, NB, 2><<<grid, block, 0, s>>>(a); break;
        case 3: fast::k_fast<S, NB, 3><<<grid, block, 0, s>>>(a); break;
        default: fast::k_fast<S, NB, 4><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <class S>
int launch_s(int nb, int kind, const FastArgs& a, int gx, cudaStream_t s) {
    switch (nb) {
        case 16: return launch_nb<S, 16>(kind, a, gx, s);
        case 32: return launch_nb<S, 32>(kind, a, gx, s);
        case 64: return launch_nb<S, 64>(kind, a, gx, s);
        case 128: return launch_nb<S, 128>(kind, a, gx, s);
        case 256: return launch_nb<S, 256>(kind, a, gx, s);
        case 512: return launch_nb<S, 512>(kind, a, gx, s);
        case 1024: return launch_nb<S, 1024>(kind, a, gx, s);
        default: return 1;
    }
}

// floor(2^64 / d) + 1 (d >= 2): umulhi(n, m) = floor(n / d) for every 32-bit n
unsigned long long magic(int d) { return ~0ULL / (unsigned long long)d + 1ULL; }

}  // namespace

bool fast_supported(int storage, int nb) {
    if (storage != ST_F32 && storage != ST_BF16) return false;
    return nb == 16 || nb == 32 || nb == 64 || nb == 128 || nb == 256 || nb == 512 || nb == 1024;
}

int fast_sites_per_cta(int nb) { return 256 / (nb < 32 ? nb : 32); }

void fast_geometry(const Geom& g, FastArgs& a) {
    a.lx = g.lx; a.ly = g.ly; a.lz = g.lz; a.lt = g.lt; a.V = g.V; a.bc_t = g.bc_t;
    a.mx = magic(g.lx);
    a.my = magic(g.ly);
    a.mz = magic(g.lz);
}

int launch_fast(int storage, int nb, int kind, const FastArgs& a, int gx, cudaStream_t s) {
    if (!fast_supported(storage, nb) || kind < 0 || kind > 4 || a.sl < 1) return 1;
    if (storage == ST_F32) return launch_s<float>(nb, kind, a, gx, s);
    return launch_s<__nv_bfloat16>(nb, kind, a, gx, s);
}

void launch_noise_words(const Geom& g, int nb, const NoiseSpec& ns, uint32_t* words, cudaStream_t s) {
    NoiseKey nk;
    nk.k0 = (uint32_t)(ns.seed & 0xffffffffu);
    nk.k1 = (uint32_t)(ns.seed >> 32);
    nk.level = ns.level;
    nk.j0 = ns.j0;
    const size_t n = (size_t)g.V * nb;
    k_noise_words<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g.V, nb, nk, words);
}

void launch_links_expanded(int V, const double* src, float4* dst, cudaStream_t s, double scale) {
    const size_t n = (size_t)V * 36;
    k_links_expanded<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, src, scale, dst);
}

}  // namespace mpmc
