// The projected ("deflated") composite polynomial of paper Sec. 4.3, read as a
// Left-right Projection (Sec. 2.1) followed by the composite polynomial:
//     M_1 b = Z D + p_1(A) (b - (A Z) D),   D = H^{-1} U^H b,   H = U^H A Z,
// with u_i = gamma5 z_pair(i) / conj(d_i) (u_i^H z_i = 1).  The kernels here
// form H (setup), D and b^H Z D per noise column, and the rank-k updates
// r = b - (A Z) D and x += Z D.  Vectors are in block layout
// [site][spin*3 + colour][column] like the stencil's.
#include <type_traits>

#include "device.cuh"
#include "kernels.h"
#include "stencil.cuh"

namespace mpmc {

namespace {

__device__ __forceinline__ double2 cadd2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <class S> __device__ __forceinline__ double2 ld_d(const S* p) {
    const auto v = ld(p);
    return make_double2((double)v.re, (double)v.im);
}

// part[split][i*ky + j] = sum over the split's sites, e of conj(X[site][e][i]) s_e Y[site][e][j]
// (s_e = gamma5 sign when g5 != 0), accumulated in FP64.
// Double-float accumulation (FP32 hi + lo pair, error-free transformations; Dekker 1971, Knuth's
// TwoSum): acc += a * b with the product split exactly into p + e (fmaf) and the sum hi + p
// split exactly into s + err.  The pair carries about 48 bits of the running sum, so a Gram
// entry of FP32 (or BF16) inputs is accurate to the FP64 level at FP32-pipe cost, where
// GB300's FP64 units run at about 1/70 of its FP32 rate.  The _rn intrinsics keep the
// compiler from contracting the additions into FMAs, which would break the transformations.
struct DF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void mac(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <class SX, class SY>
__global__ void k_block_gram(int V, const SX* __restrict__ X, int kx, const SY* __restrict__ Y, int ky, int g5,
                             double2* part, int nsplit) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)kx * ky) return;
    const int i = (int)(idx / ky), j = (int)(idx % ky);
    const int split = blockIdx.y;
    const int chunk = (V + nsplit - 1) / nsplit;
    const int s0 = split * chunk, s1 = min(V, s0 + chunk);
    if constexpr (!std::is_same<SX, double>::value && !std::is_same<SY, double>::value) {
        // FP32 / BF16 inputs (exact in FP32): double-float sums, a fresh pair per site (24
        // products each) whose value is then added in FP64
        double ar = 0, ai = 0;
        for (int site = s0; site < s1; ++site) {
            DF sr, si;
#pragma unroll
            for (int e = 0; e < 12; ++e) {
                const size_t row = (size_t)site * 12 + e;
                const auto x = ld(X + (row * kx + i) * 2);
                auto y = ld(Y + (row * ky + j) * 2);
                const float yr = (g5 && e >= 6) ? -(float)y.re : (float)y.re;
                const float yi = (g5 && e >= 6) ? -(float)y.im : (float)y.im;
                sr.mac((float)x.re, yr);
                sr.mac((float)x.im, yi);
                si.mac((float)x.re, yi);
                si.mac(-(float)x.im, yr);
            }
            ar += sr.value();
            ai += si.value();
        }
        part[(size_t)split * kx * ky + idx] = make_double2(ar, ai);
        return;
    }
    double ar = 0, ai = 0;
    for (int site = s0; site < s1; ++site) {
#pragma unroll
        for (int e = 0; e < 12; ++e) {
            const size_t row = (size_t)site * 12 + e;
            const double2 x = ld_d(X + (row * kx + i) * 2);
            double2 y = ld_d(Y + (row * ky + j) * 2);
            if (g5 && e >= 6) y = make_double2(-y.x, -y.y);
            ar += x.x * y.x + x.y * y.y;
            ai += x.x * y.y - x.y * y.x;
        }
    }
    part[(size_t)split * kx * ky + idx] = make_double2(ar, ai);
}

__global__ void k_gram_reduce(size_t n, int nsplit, const double2* __restrict__ part, double2* out) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    double2 s = make_double2(0, 0);
    for (int p = 0; p < nsplit; ++p) s = cadd2(s, part[(size_t)p * n + idx]);
    out[idx] = s;
}

// Per noise column c: Ub_j = G2[pair[j]][c] * inv_d[j] (u_j^H b), D[i][c] = sum_j Hinv[i][j] Ub_j,
// xz[c] = sum_i conj(G1[i][c]) D[i][c] (b^H Z D) when G1 is given.
__global__ void k_proj_coef(int k, int nb, const int* __restrict__ pair, const double2* __restrict__ inv_d,
                            const double2* __restrict__ Hinv, const double2* __restrict__ G1,
                            const double2* __restrict__ G2, double2* D64, float2* D32, double2* xz) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nb) return;
    double2 acc_xz = make_double2(0, 0);
    for (int i = 0; i < k; ++i) {
        double2 d = make_double2(0, 0);
        for (int j = 0; j < k; ++j) {
            const double2 ub = cmul2(G2[(size_t)pair[j] * nb + c], inv_d[j]);
            d = cadd2(d, cmul2(Hinv[(size_t)i * k + j], ub));
        }
        D64[(size_t)i * nb + c] = d;
        D32[(size_t)i * nb + c] = make_float2((float)d.x, (float)d.y);
        if (G1) {
            const double2 g = G1[(size_t)i * nb + c];
            acc_xz = cadd2(acc_xz, cmul2(make_double2(g.x, -g.y), d));
        }
    }
    if (xz) xz[c] = acc_xz;
}

template <class T> struct DTy;
template <> struct DTy<double> { using type = double2; };
template <> struct DTy<float> { using type = float2; };

// out[site][e][c] = base[site][e][c] + sign * sum_i Y[site][e][i] D[i][c]; base = noise when null.
template <class S, class T>
__global__ void k_rank_update(int V, int nb, const T* __restrict__ Y, int k, const typename DTy<T>::type* __restrict__ D,
                              T sign, const S* base, NoiseKey nk, S* out, uint32_t salt) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)V * nb) return;
    const int site = (int)(idx / nb), c = (int)(idx % nb);
    cplx<T> acc[12];
    if (base) {
        const S* pb = base + ((size_t)site * 12 * nb + c) * 2;
#pragma unroll
        for (int e = 0; e < 12; ++e) {
            const auto v = ld(pb + (size_t)e * nb * 2);
            acc[e] = {(T)v.re, (T)v.im};
        }
    } else {
        const uint32_t w = z4_word(nk, site, c);
#pragma unroll
        for (int e = 0; e < 12; ++e) acc[e] = z4_value<T>(w >> (2 * e));
    }
    const T* py = Y + (size_t)site * 12 * k * 2;
    for (int i = 0; i < k; ++i) {
        const auto dv = D[(size_t)i * nb + c];
        const cplx<T> d = {sign * (T)dv.x, sign * (T)dv.y};
#pragma unroll
        for (int e = 0; e < 12; ++e) {
            const T* q = py + ((size_t)e * k + i) * 2;
            cmac(acc[e], cplx<T>{q[0], q[1]}, d);
        }
    }
    using MS = typename Math<S>::T;   // arithmetic type of the storage format
    S* po = out + ((size_t)site * 12 * nb + c) * 2;
#pragma unroll
    for (int e = 0; e < 12; ++e)   // BF16: stochastic rounding (zero-mean errors), see device.cuh
        st_sr(po + (size_t)e * nb * 2, cplx<MS>{(MS)acc[e].re, (MS)acc[e].im},
              sr_bits(sr_seed(salt, (uint32_t)site, (uint32_t)c), e));
}

// vector-major [k][V*12] -> block layout [site][e][k]
template <class TS, class TD>
__global__ void k_vec_to_block(int V, int k, const TS* __restrict__ src, TD* dst) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // over V*12*k (block order)
    if (idx >= (size_t)V * 12 * k) return;
    const size_t row = idx / k;
    const int i = (int)(idx % k);
    dst[idx * 2] = (TD)src[((size_t)i * V * 12 + row) * 2];
    dst[idx * 2 + 1] = (TD)src[((size_t)i * V * 12 + row) * 2 + 1];
}

// Per column c of two blocks X, Y ([site][e][nb], FP64): partial sums of |x|^2, |y|^2, x^H y.
__global__ void k_col_stats(int V, int nb, const double* __restrict__ X, const double* __restrict__ Y, double* part,
                            int nsplit) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int split = blockIdx.y;
    if (c >= nb) return;
    const int chunk = (V + nsplit - 1) / nsplit;
    const int s0 = split * chunk, s1 = min(V, s0 + chunk);
    double xx = 0, yy = 0, re = 0, im = 0;
    for (int site = s0; site < s1; ++site)
        for (int e = 0; e < 12; ++e) {
            const size_t o = (((size_t)site * 12 + e) * nb + c) * 2;
            const double xr = X[o], xi = X[o + 1], yr = Y[o], yi = Y[o + 1];
            xx += xr * xr + xi * xi;
            yy += yr * yr + yi * yi;
            re += xr * yr + xi * yi;
            im += xr * yi - xi * yr;
        }
    double* q = part + ((size_t)split * nb + c) * 4;
    q[0] = xx; q[1] = yy; q[2] = re; q[3] = im;
}

__global__ void k_col_stats_reduce(int nb, int nsplit, const double* __restrict__ part, double* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nb) return;
    double a[4] = {0, 0, 0, 0};
    for (int s = 0; s < nsplit; ++s)
        for (int t = 0; t < 4; ++t) a[t] += part[((size_t)s * nb + c) * 4 + t];
    for (int t = 0; t < 4; ++t) out[(size_t)c * 4 + t] = a[t];
}

NoiseKey key_of(const NoiseSpec& ns) {
    NoiseKey nk;
    nk.k0 = (uint32_t)(ns.seed & 0xffffffffu);
    nk.k1 = (uint32_t)(ns.seed >> 32);
    nk.level = ns.level;
    nk.j0 = ns.j0;
    return nk;
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int gram_nsplit(int V) { return std::max(1, std::min(128, V / 64)); }

// math: ST_F64 (X double) or ST_F32 (X float); sy: storage of Y
void launch_block_gram(int math, int V, const void* X, int kx, int sy, const void* Y, int ky, int g5, double2* part,
                       int nsplit, double2* out, cudaStream_t s) {
    const size_t n = (size_t)kx * ky;
    const dim3 grid(nblk(n, 128), nsplit);
    if (math == ST_F64) {
        if (sy == ST_F64) k_block_gram<double, double><<<grid, 128, 0, s>>>(V, (const double*)X, kx, (const double*)Y, ky, g5, part, nsplit);
        else if (sy == ST_F32) k_block_gram<double, float><<<grid, 128, 0, s>>>(V, (const double*)X, kx, (const float*)Y, ky, g5, part, nsplit);
        else k_block_gram<double, __nv_bfloat16><<<grid, 128, 0, s>>>(V, (const double*)X, kx, (const __nv_bfloat16*)Y, ky, g5, part, nsplit);
    } else {
        if (sy == ST_F64) k_block_gram<float, double><<<grid, 128, 0, s>>>(V, (const float*)X, kx, (const double*)Y, ky, g5, part, nsplit);
        else if (sy == ST_F32) k_block_gram<float, float><<<grid, 128, 0, s>>>(V, (const float*)X, kx, (const float*)Y, ky, g5, part, nsplit);
        else k_block_gram<float, __nv_bfloat16><<<grid, 128, 0, s>>>(V, (const float*)X, kx, (const __nv_bfloat16*)Y, ky, g5, part, nsplit);
    }
    k_gram_reduce<<<nblk(n, 256), 256, 0, s>>>(n, nsplit, part, out);
}

void launch_proj_coef(int k, int nb, const int* pair, const double2* inv_d, const double2* Hinv, const double2* G1,
                      const double2* G2, double2* D64, float2* D32, double2* xz, cudaStream_t s) {
    k_proj_coef<<<nblk(nb, 64), 64, 0, s>>>(k, nb, pair, inv_d, Hinv, G1, G2, D64, D32, xz);
}

// math: precision of Y and D (ST_F64 -> double Y, D64; otherwise float Y, D32); storage: of base/out
void launch_rank_update(int math, int storage, int V, int nb, const void* Y, int k, const double2* D64,
                        const float2* D32, double sign, const void* base, const NoiseSpec& ns, void* out,
                        cudaStream_t s, uint32_t salt) {
    const size_t n = (size_t)V * nb;
    const NoiseKey nk = key_of(ns);
    if (math == ST_F64 && storage == ST_F64) {
        k_rank_update<double, double><<<nblk(n, 128), 128, 0, s>>>(V, nb, (const double*)Y, k, D64, sign,
                                                                (const double*)base, nk, (double*)out, salt);
    } else if (math == ST_F64 && storage == ST_F32) {
        // FP64 projection of a reduced-precision block: the sum is formed in FP64 and rounded once
        k_rank_update<float, double><<<nblk(n, 128), 128, 0, s>>>(V, nb, (const double*)Y, k, D64, sign,
                                                               (const float*)base, nk, (float*)out, salt);
    } else if (math == ST_F64) {
        k_rank_update<__nv_bfloat16, double><<<nblk(n, 128), 128, 0, s>>>(V, nb, (const double*)Y, k, D64, sign,
                                                                       (const __nv_bfloat16*)base, nk,
                                                                       (__nv_bfloat16*)out, salt);
    } else if (storage == ST_F32) {
        k_rank_update<float, float><<<nblk(n, 128), 128, 0, s>>>(V, nb, (const float*)Y, k, D32, (float)sign,
                                                              (const float*)base, nk, (float*)out, salt);
    } else {
        k_rank_update<__nv_bfloat16, float><<<nblk(n, 128), 128, 0, s>>>(V, nb, (const float*)Y, k, D32, (float)sign,
                                                                      (const __nv_bfloat16*)base, nk,
                                                                      (__nv_bfloat16*)out, salt);
    }
}

void launch_col_stats(int V, int nb, const double* X, const double* Y, double* part, int nsplit, double* out,
                      cudaStream_t s) {
    k_col_stats<<<dim3(nblk(nb, 64), nsplit), 64, 0, s>>>(V, nb, X, Y, part, nsplit);
    k_col_stats_reduce<<<nblk(nb, 64), 64, 0, s>>>(nb, nsplit, part, out);
}

void launch_vec_to_block(int math, int V, int k, const void* src, void* dst, cudaStream_t s, int src_storage) {
    const size_t n = (size_t)V * 12 * k;
    if (src_storage < 0) src_storage = math;
    if (math == ST_F64 && src_storage == ST_F64)
        k_vec_to_block<double, double><<<nblk(n, 256), 256, 0, s>>>(V, k, (const double*)src, (double*)dst);
    else if (math == ST_F64)   // vectors held in FP32 (exactly), widened to FP64
        k_vec_to_block<float, double><<<nblk(n, 256), 256, 0, s>>>(V, k, (const float*)src, (double*)dst);
    else
        k_vec_to_block<float, float><<<nblk(n, 256), 256, 0, s>>>(V, k, (const float*)src, (float*)dst);
}

}  // namespace mpmc
