// Host-side launch interface of the CUDA kernels (no templates, no torch).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpmc {

enum Storage { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2 };

struct Geom {
    int lx, ly, lz, lt, V, bc_t;
};

struct NoiseSpec {
    uint64_t seed;
    uint32_t level;
    uint32_t j0;
};

// One degree step of the root form (Sec. 2.3), in the order that keeps the
// matrix the same at every step whatever the working precision:
//   t   = in - kappa * H in                 (t = A in)
//   out = in - alpha * t                    (out = (I - A/theta) in, alpha = 1/theta)
// (op_only: out = t).  Optional:  y = ya * in + yb * out (ymode 1)  or
// y += yb * out (ymode 2);  acc[cta][col] += dot_w * sum_sites b^H out
// (b = the column's Z4 noise).  in == nullptr means "in is the noise block".
struct StepArgs {
    const void* in;
    void* out;
    void* y;
    int ymode;
    bool dot;
    bool op_only;
    double alpha[2], ya[2], yb[2];
    double dot_w[2];
    double2* acc;
    double kappa;
    float alphaf[2], yaf[2], ybf[2], kappaf;   // the same in FP32 (filled by launch_step)
    uint32_t salt;                              // random-bit salt of stochastically rounded BF16 stores
};

// Last inner step of a composite outer step (Sec. 3.2):
//   t  = in - alpha * (in - kappa H in)       (t = pi_in(A) w, not stored)
//   wn = w - beta * (w - t)                   (wn = (I - B/eta) w, B = A p_in(A))
//   y += gamma * wn;  optional acc += dot_w * b^H y
struct OuterArgs {
    const void* in;
    const void* w;
    void* wout;
    void* y;
    double alpha[2], beta[2], gamma[2];
    bool dot;
    double dot_w[2];
    double2* acc;
    double kappa;
    float alphaf[2], betaf[2], gammaf[2], kappaf;
    uint32_t salt;                              // as StepArgs
};

struct LaunchCfg {
    int bx, by, sl, gx, gy;   // block (bx, by), site loop sl, grid (gx, gy)
    int R;                    // right-hand sides per thread (1 or 2)
};

// bx: threads per CTA along the columns (each handles R columns), 256/bx sites per CTA
LaunchCfg chain_config(const Geom& g, int nb, int bx_max, int sl, int R = 1);

// per-storage stencil launchers (stencil_f64.cu, stencil_f32.cu, stencil_bf16.cu)
void step_f64(const Geom&, const void*, int, const NoiseSpec&, const StepArgs&, const LaunchCfg&, cudaStream_t);
void step_f32(const Geom&, const void*, int, const NoiseSpec&, const StepArgs&, const LaunchCfg&, cudaStream_t);
void step_bf16(const Geom&, const void*, int, const NoiseSpec&, const StepArgs&, const LaunchCfg&, cudaStream_t);
void outer_f64(const Geom&, const void*, int, const NoiseSpec&, const OuterArgs&, const LaunchCfg&, cudaStream_t);
void outer_f32(const Geom&, const void*, int, const NoiseSpec&, const OuterArgs&, const LaunchCfg&, cudaStream_t);
void outer_bf16(const Geom&, const void*, int, const NoiseSpec&, const OuterArgs&, const LaunchCfg&, cudaStream_t);

// FP32 copies of the coefficients (what the FP32 / BF16 kernels use)
void fill_floats(StepArgs& a);
void fill_floats(OuterArgs& a);

void launch_step(int storage, const Geom& g, const void* links, int nb, const NoiseSpec& ns,
                 const StepArgs& a, const LaunchCfg& cfg, cudaStream_t s);
void launch_outer(int storage, const Geom& g, const void* links, int nb, const NoiseSpec& ns,
                  const OuterArgs& a, const LaunchCfg& cfg, cudaStream_t s);

// Shape of a t-sweep launch: site blocks, right-hand-side tiles, t-segment
// length and count, accumulator rows (blocks x segments).
struct SweepCfg {
    int nblk, tiles, ts, nseg, rows;
};

// Issue-lean FP32-arithmetic stencil kernels (stencil_fast.cuh): FP32 /
// BF16 storage, block widths NB in {16, 32, 64, 128, 256, 512, 1024}
// (compile-time row stride), links expanded to broadcast pairs, Z4 symbols
// from a per-block word table.  Same step / outer semantics as StepArgs /
// OuterArgs (ymode 0 only).  Accumulator rows: ceil(V / (sites per CTA * sl)).
struct FastArgs {
    const void* in;          // input block (unused when the input is the noise)
    void* out;               // step: output;  outer: w_out
    const void* w;           // outer: w
    void* y;                 // outer: y
    const uint32_t* words;   // Z4 words [V][NB] of the noise block
    const float4* Ue;        // expanded links [V][4][9] (re, re, im, im)
    double2* acc;
    double dot_w[2];
    float alpha[2], beta[2], gamma[2], kappa;
    uint32_t salt;                   // random-bit salt of stochastically rounded BF16 stores
    int lx, ly, lz, lt, V, bc_t, sl;
    unsigned long long mx, my, mz;   // floor(2^64 / extent) + 1
    const int* blk_order;            // t-sweep: site block of each launch-order index (null: plain order)
    long long wait_limit;            // t-sweep: bound of each mbarrier wait in SM clock cycles
    int skip_copy;                   // t-sweep test hook: the q-th plane copy of each CTA (q >= 1) is
                                     // not issued; 0: none
};
bool fast_supported(int storage, int nb);
int fast_sites_per_cta(int nb);
// kind: 0 step, 1 step + dot, 2 step from the noise + dot, 3 outer, 4 outer + dot
int launch_fast(int storage, int nb, int kind, const FastArgs& a, int gx, cudaStream_t s);
void fast_geometry(const Geom& g, FastArgs& a);
// t-sweep form of the issue-lean kernels (stencil_fsweep.cu): kinds 0, 1,
// 3, 4; even lx, ly, lz; the input block read by TMA through a tensor map
// made by fsweep_make_map; accumulator rows cfg.rows.
// var: 0 links read from global memory (tile width min(nb, 32)); 1 each plane's links staged in
// shared memory with its spinor rows (tile width 16); 2 warp-per-site form with staged links (tile
// width 32, nb >= 32; nb = 16 runs variant 1); 3 two-sites-per-warp form with staged links (tile
// width 16).  fsweep_variant maps the sweep option mask (bit 4: staged links, bit 5: warp-per-site,
// bit 6: two sites per warp) and nb to var; fsweep_tile gives its tile width.
bool fsweep_supported(int storage, const Geom& g, int nb);
int fsweep_variant(int mask, int nb);
int fsweep_tile(int var, int nb);
SweepCfg fsweep_config(const Geom& g, int nb, int ts, int var);
// Launch order of the (lx/2)(ly/2)(lz/2) site blocks along a Morton (Z-order) curve of the
// block grid, so that CTAs running at the same time cover compact regions of the lattice
void fsweep_morton_order(const Geom& g, int* order);
bool fsweep_make_map(void* map, int storage, const void* base, int V, int nb, int tw);
int launch_fsweep(int storage, int nb, int kind, const FastArgs& a, const SweepCfg& c, const void* map, int* err,
                  cudaStream_t s, int var);
// Z4 words of a noise block: words[site][col] = Philox word 0 of (j0 + col, site, level)
void launch_noise_words(const Geom& g, int nb, const NoiseSpec& ns, uint32_t* words, cudaStream_t s);
// expanded links (re, re, im, im) in float from scale * complex-double [mu][site][3][3]
void launch_links_expanded(int V, const double* src, float4* dst, cudaStream_t s, double scale = 1.0);

// t-sweep form of the step / outer kernels (stencil_sweep.cu): FP32 and
// BF16 storage, even lx, ly, lz; the input block is read by TMA through a
// tensor map made by sweep_make_map for that buffer.  Accumulator rows:
// cfg.rows (one per site block and t-segment).
bool sweep_supported(int storage, const Geom& g, int nb);
SweepCfg sweep_config(const Geom& g, int nb, int ts);   // ts <= 0: automatic segment length
size_t sweep_map_bytes();
bool sweep_make_map(void* map, int storage, const void* base, int V, int nb);
int launch_sweep_step(int storage, const Geom& g, const void* links, int nb, const NoiseSpec& ns, const StepArgs& a,
                      const SweepCfg& c, const void* map, int* err, cudaStream_t s);
int launch_sweep_outer(int storage, const Geom& g, const void* links, int nb, const NoiseSpec& ns,
                       const OuterArgs& a, const SweepCfg& c, const void* map, int* err, cudaStream_t s);

// out = scale * noise block (all nb columns)
void launch_fill_noise(int storage, const Geom& g, int nb, const NoiseSpec& ns, const double scale[2],
                       void* out, cudaStream_t s);
// noise block as complex double in the C-ABI layout [site][e][ld] columns c0..c0+cnt
void launch_noise_f64(const Geom& g, const NoiseSpec& ns, int cnt, int ld, int c0, double* out, cudaStream_t s);
// dst (storage, [site][e][nb]) = src columns c0..c0+cnt of a complex-double [site][e][ld] block; zero pad
void launch_import(int storage, int V, const double* src, int ld, int c0, int cnt, void* dst, int nb,
                   cudaStream_t s);
// dst columns c0..c0+cnt of complex-double [site][e][ld] = src (storage) columns 0..cnt
void launch_export(int storage, int V, const void* src, int nb, double* dst, int ld, int c0, int cnt,
                   cudaStream_t s);
// out = s * in (storage buffers of V*12*nb complex)
// (BF16 output rounded stochastically with random bits salted by `salt`)
void launch_scale(int storage, size_t ncplx, const void* in, const double sc[2], void* out, cudaStream_t s,
                  uint32_t salt = 0);
// links: scale * complex double [mu][site][3][3] -> math precision [site][mu][3][3] (the product
// formed in FP64, then rounded once per element)
void launch_links(int storage, int V, const double* src, void* dst, cudaStream_t s, double scale = 1.0);

// samples[j0 + col] = sum_cta acc_hi + const_hi - (sum_cta acc_lo + const_lo) - dterm[col]
// also hi/lo parts (may be null).  acc_lo/dterm may be null.
void launch_finalize(int ncta, int nb, int nvalid, const double2* acc_hi, const double2* acc_lo,
                     const double c_hi[2], const double c_lo[2], const double2* dterm,
                     double2* samples, double2* hi, double2* lo, cudaStream_t s,
                     const double2* add_hi = nullptr);

// Projection of the projected composite polynomial (proj.cu)
int gram_nsplit(int V);
void launch_block_gram(int math, int V, const void* X, int kx, int sy, const void* Y, int ky, int g5, double2* part,
                       int nsplit, double2* out, cudaStream_t s);
void launch_proj_coef(int k, int nb, const int* pair, const double2* inv_d, const double2* Hinv, const double2* G1,
                      const double2* G2, double2* D64, float2* D32, double2* xz, cudaStream_t s);
void launch_rank_update(int math, int storage, int V, int nb, const void* Y, int k, const double2* D64,
                        const float2* D32, double sign, const void* base, const NoiseSpec& ns, void* out,
                        cudaStream_t s, uint32_t salt = 0);
// vector-major [k][V*12] -> block layout [site][e][k] in the math precision; src_storage: the
// precision of src (default: math; FP32 src with FP64 math is widened exactly)
void launch_vec_to_block(int math, int V, int k, const void* src, void* dst, cudaStream_t s, int src_storage = -1);
// out[c] = (|x_c|^2, |y_c|^2, Re x_c^H y_c, Im x_c^H y_c) for FP64 blocks of nb columns
void launch_col_stats(int V, int nb, const double* X, const double* Y, double* part, int nsplit, double* out,
                      cudaStream_t s);

// Deflation dots of Sec. 4.1 for a noise block:
//   G1[i][col] = z_i^H b_col,  G2[i][col] = z_i^H gamma5 b_col
// Z: math precision, k vectors of V*12 complex.  part: scratch [nsplit][k][nb][2] double2.
int defl_nsplit(int V);
void launch_defl_dots(int storage, const Geom& g, int k, const void* Z, int nb, const NoiseSpec& ns,
                      double2* part, int nsplit, cudaStream_t s);
// term[col] = sum_i coef[i] * conj(G1[i][col]) * G2[pair[i]][col]; G1, G2 written too (k x nb each)
void launch_defl_reduce(int k, int nb, int nsplit, const double2* part, const double2* coef, const int* pair,
                        double2* G1, double2* G2, double2* term, cudaStream_t s);
// term[col] only, from G1, G2 already formed
void launch_defl_term(int k, int nb, const double2* coef, const int* pair, const double2* G1, const double2* G2,
                      double2* term, cudaStream_t s);

// Tensor-core deflation dots (defl_tc.cu)
int tc_defl_layout(int V, int k, int* Mpad, int* Kpad);
void launch_split_bf16(int V, int k, int Mpad, int Kpad, const double* z, float* zhat, void* planes, cudaStream_t s);
bool tc_make_map(void* map, const void* planes, int Mpad, int Kpad);
size_t tc_map_bytes();
void tc_defl_plan(int V, int k, int nb, int* nsplit, int* kb_per_split, size_t* part_floats);
int tc_defl_launch(const void* map, int V, int k, int nb, const NoiseSpec& ns, float* part, int nsplit,
                   int kb_per_split, double2* G1, double2* G2, int* err, cudaStream_t s);

// d[i] = z_pair[i]^H gamma5 z_i (FP64 accumulation of the stored vectors)
void launch_defl_norms(int storage, int V, int k, const void* Z, const int* pair, double2* d, cudaStream_t s);
// Z (math precision) from complex double host-layout vectors
void launch_convert_vectors(int storage, size_t ncplx, const double* src, void* dst, cudaStream_t s);

// FP64 Krylov helpers on complex-double vectors of n complex
// h[j] = V_j^H w for j < m (two-level fixed-order reduction through part)
void launch_mdot(size_t n, int m, const double2* Vb, const double2* w, double2* part, double2* h,
                 cudaStream_t s);
// w -= sum_j h[j] V_j
void launch_maxpy(size_t n, int m, const double2* Vb, const double2* h, double2* w, cudaStream_t s);
// out[0] = ||w||^2
void launch_norm2(size_t n, const double2* w, double* part, double* out, cudaStream_t s);
// dst = w * (1/nrm)   where *nrm2 is ||w||^2 on the device
void launch_normalize(size_t n, const double2* w, const double* nrm2, double2* dst, cudaStream_t s);
// Z_i = sum_j V_j Y[j][i]
void launch_combine(size_t n, int m, const double2* Vb, const double2* Y, int k, double2* Z, cudaStream_t s);
// complex double [site][e][1] <-> storage conversions for a single vector are import/export with nb = 1

// Probing: out = probe block of columns q0 .. q0+nq-1 (zero beyond nq); total += sum of X
// over the probe entries of those columns (FP64, fixed order; part: nchunk x nb scratch).
// Site colours from the device table tab (V entries), or with tab == nullptr from the
// period-m colouring x%m + m (y%m) + m^2 (z%m) + m^3 (t%m).
void launch_probe_block(int storage, const Geom& g, int m, const int* tab, int q0, int nq, int nb, void* out,
                        cudaStream_t s);
void launch_probe_trace(int storage, const Geom& g, int m, const int* tab, int q0, int nq, int nb, const void* X,
                        int nchunk, double2* part, double2* total, cudaStream_t s);

int mdot_parts(size_t n);

}  // namespace mpmc
