/*
 * mpmc.h -- C ABI of the GB300 hot path of Multipolynomial Monte Carlo
 * (Lashomb, Morgan, Whyte, Wilcox, arXiv:2306.09559).
 *
 * The library estimates the traces of the multilevel decomposition of
 * Sec. 3.1, Eq. (2), with polynomials p_j(A) of the Wilson-Dirac matrix
 * A = I - kappa*H applied to blocks of Z4 noise vectors (Sec. 1) in root
 * form (Sec. 2.3), composite ("double") polynomials (Secs. 2.4, 3.2) and
 * eigenvector deflation of the polynomial-difference levels (Sec. 4.1).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Complex numbers are two consecutive doubles (re, im).
 *  - dims = {Lx, Ly, Lz, Lt}, each >= 2.  V = Lx*Ly*Lz*Lt sites, n = 12 V.
 *  - Site index s = ((t*Lz + z)*Ly + y)*Lx + x; unknown index within a
 *    site e = spin*3 + colour (spin 0..3, colour 0..2).
 *  - Links: U[mu][s][a][b], mu = 0..3 for x, y, z, t, each a 3x3 complex
 *    matrix (row a, column b): 4*V*9 complex = 72 V doubles.
 *  - A = I - kappa * sum_mu [(1 - gamma_mu) U_mu(x) delta_{x+mu,y}
 *                           + (1 + gamma_mu) U_mu(x-mu)^+ delta_{x-mu,y}]
 *    with Hermitian gamma matrices in the chiral DeGrand-Rossi basis,
 *    gamma5 = diag(1, 1, -1, -1); periodic boundaries (bc_t = -1 makes the
 *    t direction antiperiodic).  The paper names the matrix only
 *    ("quenched Wilson-Dirac", Sec. 5, Examples 2 and 3); this is the
 *    reading every part of the project uses.
 *  - Vector blocks passed to mpmc_apply_*: complex doubles laid out
 *    [s][e][r] (right-hand side r innermost), i.e. element (unknown
 *    12 s + e, column r) at offset (12 s + e) * nrhs + r complex numbers.
 *  - Z4 noise (Sec. 1): vector j of level l has entry e of site s equal to
 *    i^q, q = bits 2e..2e+1 of word 0 of Philox-4x32-10 (Salmon et al.,
 *    SC'11) with key (seed & 0xffffffff, seed >> 32) and counter
 *    (j, s, l, 0).
 *
 * Ownership: every input is copied into library-owned device memory
 * before the call returns; the caller keeps its buffers.  Calls on one
 * handle must not overlap (a handle is not thread-safe); different handles
 * are independent.  All work is enqueued on the handle's stream (its own,
 * or the one given by mpmc_set_stream); calls that return host results
 * synchronise that stream.
 *
 * Errors: every call returns MPMC_OK (0) or a positive code below.  No
 * call aborts the process.  mpmc_last_error() gives a message for the last
 * failing call on a handle.
 */
#ifndef MPMC_H
#define MPMC_H

#include <stdint.h>

#if defined(__GNUC__)
#define MPMC_API __attribute__((visibility("default")))
#else
#define MPMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpmc_ctx* mpmc_handle;

enum {
    MPMC_OK = 0,
    MPMC_EINVAL = 1,      /* bad argument: dims < 2, kappa not finite, nroots < 1, k > n, ... */
    MPMC_ENOMEM = 2,      /* device or host allocation failed */
    MPMC_ENOTSUP = 3,     /* precision or mode not supported */
    MPMC_ETIMEOUT = 4,    /* a bounded device wait gave up */
    MPMC_ENONFINITE = 5,  /* a non-finite root, eigenvalue or sample */
    MPMC_ECUDA = 6,       /* a CUDA runtime call failed (message in mpmc_last_error) */
    MPMC_ESTATE = 7       /* call out of order: e.g. trace before any polynomial is set */
};

/* Arithmetic of the stencil and polynomial chain. */
enum {
    MPMC_FP64 = 0,   /* FP64 vectors, links and arithmetic */
    MPMC_FP32 = 1,   /* FP32 vectors and links, FP32 arithmetic, FP64 b^H x accumulation */
    MPMC_BF16S = 2   /* BF16-stored vectors, FP32 links and arithmetic, FP64 accumulation */
};

/* Polynomial kinds (mpmc_set_poly). */
enum {
    MPMC_SINGLE = 0,             /* p(A) from one GMRES run, Secs. 2.3, 3.1 */
    MPMC_COMPOSITE = 1,          /* p_in(A) p_out(A p_in(A)), Secs. 2.4, 3.2 */
    MPMC_DEFLATED_COMPOSITE = 2  /* projection then composite, Sec. 4.3 */
};

/*
 * mpmc_create: a handle for one lattice.  links: host array described
 * above (copied).  kappa: hopping parameter (finite).  precision: one of
 * MPMC_FP64/FP32/BF16S.  bc_t: +1 periodic or -1 antiperiodic in t.
 * Defines the matrix A of Secs. 1 and 5 (see the conventions).
 * Errors: EINVAL (dims, kappa, bc_t), ENOTSUP (precision), ENOMEM, ECUDA.
 * *h is NULL on failure.
 */
MPMC_API int mpmc_create(mpmc_handle* h, const int dims[4], const double* links,
                double kappa, int precision, int bc_t);

/* mpmc_destroy: frees all device memory of the handle; NULL is accepted. */
MPMC_API int mpmc_destroy(mpmc_handle h);

/* mpmc_strerror: static text for an error code. */
MPMC_API const char* mpmc_strerror(int code);

/* mpmc_last_error: message of the last failing call on h (never NULL). */
MPMC_API const char* mpmc_last_error(mpmc_handle h);

/*
 * mpmc_set_stream: enqueue all further work of h on the CUDA stream
 * `stream` (a cudaStream_t, owned by the caller, which must outlive its
 * use); NULL restores the handle's own stream.
 */
MPMC_API int mpmc_set_stream(mpmc_handle h, void* stream);

/*
 * mpmc_set_block: number of right-hand sides processed per launch
 * (1..MPMC_MAX_BLOCK).  0 restores the default.  Only performance depends
 * on it: samples and applied vectors do not.
 */
#define MPMC_MAX_BLOCK 1024
MPMC_API int mpmc_set_block(mpmc_handle h, int nrhs_block);

/*
 * mpmc_set_poly: polynomial number `index` (0 <= index < MPMC_MAX_POLYS).
 * roots: nroots complex values theta_1..theta_m, the harmonic Ritz values
 * of the GMRES run that defines p through pi(alpha) = 1 - alpha p(alpha)
 * (Sec. 3.1); p has degree m - 1 and is applied in root form
 * p(A) v = sum_i theta_i^{-1} prod_{j<i} (I - A/theta_j) v (Sec. 2.3).
 * For the composite kinds, roots are those of p_in and outer (nouter
 * values) those of p_out, found by GMRES on A p_in(A); the polynomial is
 * p_in(A) p_out(A p_in(A)) of degree nroots*nouter - 1 (Sec. 3.2).  The
 * deflated kind adds the projection of Sec. 4.3 with the eigenpairs of
 * mpmc_set_deflation (which must be called first).
 * leja: flags.  Bit 0 (MPMC_POLY_LEJA) reorders each root list into
 * modified Leja order (first the root of largest modulus, then each next root
 * maximising the product of distances to those taken; ties to the lowest
 * index); without it the caller's order is kept.  Bit 1
 * (MPMC_POLY_FP32_COEFS) replaces every root theta by 1/c with c = 1/theta
 * rounded to the nearest FP32 complex number, on any handle.  The product
 * form applies the coefficients 1/theta; FP32 and BF16S handles apply them in
 * FP32, so without this flag they use the polynomial with those rounded roots
 * while an FP64 handle uses the exact one.  With it, handles of every
 * precision apply the same polynomial, and the traces of a reduced-precision
 * estimate differ from FP64 ones only by arithmetic rounding (a root moves
 * by at most ~6e-8 of its modulus).
 * Polynomials 0..L-1 define the levels of mpmc_trace_levels: level l < L-1
 * is Tr(p_l - p_{l+1}), level L-1 is Tr(p_{L-1}) (Eq. (2)).
 * Errors: EINVAL (index, kind, counts, NULL roots), ENONFINITE (a root is
 * zero or not finite), ESTATE (deflated kind without deflation).
 */
#define MPMC_MAX_POLYS 8
#define MPMC_POLY_LEJA 1
#define MPMC_POLY_FP32_COEFS 2
MPMC_API int mpmc_set_poly(mpmc_handle h, int index, int kind,
                  const double* roots, int nroots,
                  const double* outer, int nouter, int leja);

/* mpmc_get_roots: copies the (possibly reordered) roots of polynomial
 * `index` to roots[0..2*nroots) and outer[0..2*nouter) (either may be
 * NULL).  Errors: EINVAL, ESTATE (not set). */
MPMC_API int mpmc_get_roots(mpmc_handle h, int index, double* roots, double* outer);

/*
 * mpmc_set_deflation: eigenpairs for the Monte Carlo deflation of Sec. 4.1
 * and the projection of Sec. 4.3.  Z: host, k right eigenvectors, vector i
 * at Z + 2*n*i (complex, unknown order); lambda: k complex eigenvalues;
 * pair[i] = j says the left eigenvector of lambda_i is gamma5 z_j (j = i
 * for real lambda_i, the conjugate partner otherwise; Sec. 4).  The
 * library scales u_i so that u_i^H z_i = 1 using the vectors as stored in
 * its working precision, so the exact correction sum_i c_i u_i^H z_i and
 * the sampled term use the same vectors.  k = 0 removes the deflation.
 * Errors: EINVAL (k < 0, k > n, pair out of range or not an involution,
 * NULL pointers with k > 0), ENONFINITE (u_i^H z_i = 0 or NaN).
 */
MPMC_API int mpmc_set_deflation(mpmc_handle h, const double* Z, const double* lambda,
                       const int* pair, int k);

/*
 * mpmc_apply_op: Y = A X for nrhs vectors in the block layout above.
 * on_device != 0: X and Y are device pointers (complex double, same
 * layout) usable on the handle's stream; otherwise host pointers.
 * The product runs in the handle's precision.
 */
MPMC_API int mpmc_apply_op(mpmc_handle h, const double* X, double* Y, int nrhs, int on_device);

/*
 * mpmc_apply_poly: X = p_index(A) B (root form of Sec. 2.3, composite of
 * Sec. 3.2, or the projected composite of Sec. 4.3), layout and on_device
 * as for mpmc_apply_op.  Errors: EINVAL, ESTATE (polynomial not set).
 */
MPMC_API int mpmc_apply_poly(mpmc_handle h, int index, const double* B, double* X,
                    int nrhs, int on_device);

/*
 * mpmc_trace_levels: the Monte Carlo of every level (Eq. (2), Sec. 4.1).
 * For level l and j = first .. first+nsamples-1 it draws Z4 noise b_j
 * (level id l), and forms
 *     s_j = b_j^H p_l(A) b_j - b_j^H p_{l+1}(A) b_j
 *           - sum_i c_i (b_j^H z_i)(u_i^H b_j),   c_i = p_l(lambda_i) - p_{l+1}(lambda_i)
 * (p_{l+1} = 0 and no deflation for the last level; c_i uses
 * 1/lambda_i for a deflated composite).  Outputs (host, any may be NULL):
 *   mean[2*l..2*l+1]   estimate = sample mean + sum_i c_i u_i^H z_i (complex)
 *   var[l]             sample variance of Re s_j (unbiased)
 *   samples[2*(l*nsamples + j) ...]   s_j (complex)
 * nsamples >= 1 (variance needs >= 2; var = NaN for 1).
 * Errors: EINVAL, ESTATE (no polynomial), ENONFINITE (a sample is not
 * finite), ECUDA.
 */
MPMC_API int mpmc_trace_levels(mpmc_handle h, uint64_t seed, int nsamples, int first,
                      double* mean, double* var, double* samples);

/*
 * mpmc_level_info: for level l, the exact deflation correction
 * sum_i c_i u_i^H z_i (complex, 2 doubles) and the number of products with
 * A per noise vector (the "MVP" count of Tables 1-8).  Either output may
 * be NULL.  Errors: EINVAL, ESTATE.
 */
MPMC_API int mpmc_level_info(mpmc_handle h, int level, double* correction, long long* matvecs);

/*
 * mpmc_noise: writes noise vectors first .. first+nrhs-1 of level `level`
 * as complex doubles in the block layout (host or device per on_device).
 * The same bits the trace kernels regenerate internally.
 */
MPMC_API int mpmc_noise(mpmc_handle h, uint64_t seed, int level, int first, int nrhs,
               double* B, int on_device);

/*
 * mpmc_arnoldi: m steps of FP64 Arnoldi with two passes of classical
 * Gram-Schmidt on the operator A (op_poly < 0) or A p_{op_poly}(A)
 * (the polynomial preconditioned operator of Secs. 2.3, 3.2, 4), started
 * from the host vector v0 (n complex).  hbar (host, (m+1) x m complex,
 * row-major, entry (i, j) at 2*(i*m + j)) receives the Hessenberg matrix;
 * basis (device, n x (m+1) complex, vector j at basis + 2*n*j) receives the
 * orthonormal basis when not NULL.  Used for the setup of Sec. 5, step 2.
 * Returns the number of completed steps in *steps (< m on breakdown).
 * All vector work is FP64 on the GPU whatever the handle's precision.
 */
MPMC_API int mpmc_arnoldi(mpmc_handle h, int op_poly, const double* v0, int m,
                 double* hbar, double* basis, int* steps);

/*
 * mpmc_combine: Z = Vb * Y on the device in FP64: Vb n x m (device, vector
 * j at Vb + 2*n*j), Y m x k (host, row-major complex), Z n x k (device,
 * vector i at Z + 2*n*i).  Forms Ritz vectors from an Arnoldi basis.
 */
MPMC_API int mpmc_combine(mpmc_handle h, const double* Vb, int m, const double* Y, int k, double* Z);

/*
 * mpmc_set_links: replace the gauge links of h (same lattice; layout and
 * copy semantics as in mpmc_create).  Polynomials and deflation vectors
 * are kept: they belong to the caller's setup for the new field.
 */
MPMC_API int mpmc_set_links(mpmc_handle h, const double* links);

/*
 * Profiling: with mpmc_profile(h, 1) every kernel launch of the classes
 * below is bracketed by CUDA events on the handle's stream; the elapsed
 * device time, the launch count and the algorithmic bytes of the launches
 * (vector reads and writes counted once per launch, links once per launch,
 * deflation vectors once per launch) accumulate until mpmc_profile(h, 1)
 * clears them; mpmc_profile(h, 0) stops recording.  mpmc_profile_read
 * synchronises the stream and returns the totals of one class.  The
 * stencil launches are also counted by kernel: the t-sweep issue-lean kernel
 * (MPMC_PROF_K_FSWEEP), the issue-lean one (K_FAST), the site-parallel one
 * (K_SITE) and the t-sweep site-parallel one (K_SWEEP).
 */
enum { MPMC_PROF_STENCIL = 0, MPMC_PROF_DEFLATION = 1, MPMC_PROF_OTHER = 2, MPMC_PROF_K_FSWEEP = 3,
       MPMC_PROF_K_FAST = 4, MPMC_PROF_K_SITE = 5, MPMC_PROF_K_SWEEP = 6 };
MPMC_API int mpmc_profile(mpmc_handle h, int enable);
MPMC_API int mpmc_profile_read(mpmc_handle h, int cls, double* ms, long long* launches, double* bytes);

/* Device counter of kernel launches made by the library since the handle
 * was created (the count a caller reports for its timed region). */
MPMC_API long long mpmc_launch_count(mpmc_handle h);

/*
 * Launch shape of the stencil kernels (performance only; results do not
 * depend on it beyond FP rounding order of the per-site sums):
 * R = right-hand sides per thread (1 or 2), bx = threads along the
 * right-hand sides per CTA (power of two <= 256), sl = sites per thread.
 * 0 selects the default (1, 64, 1).  mpmc_get_launch reports the current
 * shape and block width.  mpmc_autotune times short noise-started chains of
 * `steps` fused steps (the trace-mode kernel) for block widths up to max_nb
 * and the shapes above on this handle's lattice and precision, then (where
 * the options below allow) the issue-lean kernels and the t-sweep with t-segment
 * lengths Lt, Lt/2, ... , and keeps the fastest per site and right-hand
 * side (block width as mpmc_set_block; sweep on/off and segment length as
 * the two options below).
 */
MPMC_API int mpmc_set_launch(mpmc_handle h, int R, int bx, int sl);
MPMC_API int mpmc_get_launch(mpmc_handle h, int* nb, int* R, int* bx, int* sl);
MPMC_API int mpmc_autotune(mpmc_handle h, int max_nb, int steps);

/*
 * Options.  MPMC_OPT_TENSOR_CORE_DEFLATION (default 1): on FP32 / BF16S
 * handles, form the deflation dots of Sec. 4.1 with the tcgen05 tensor-core
 * kernel (BF16 hi + lo split of the vectors, FP32 accumulation) instead of
 * the CUDA-core kernel.  Both use the same stored vectors zhat = hi + lo, so
 * the exact correction matches either way.  mpmc_get_option reports whether
 * the tensor-core path is in use (1) or not (0).
 * Stencil step classes (bits of the two masks below): 1 the dotted steps
 * (single and projected chains, including the noise-started first step),
 * 2 the undotted inner steps of composite chains, 4 the outer steps of
 * composite chains.
 * MPMC_OPT_FAST_STENCIL (mask 0 .. 7, default 7): classes that run the
 * issue-lean kernels on FP32 / BF16S handles with block widths 16, 32, 64,
 * ..., 1024: packed FP32x2 arithmetic on (re, im) pairs, links expanded
 * once per field to (re, re, im, im) pairs (16 bytes per link element),
 * compile-time block width, Z4 symbols from a per-block word table (4 bytes
 * per site and right-hand side) and a table-driven noise dot.  Same
 * per-component FMA rounding as the site-parallel kernels; the grouping of
 * the hopping sums differs (FP32 rounding level).  mpmc_get_option returns
 * the mask in effect for the current block width (0 where they do not
 * apply).
 * MPMC_OPT_FAST_SITES: sites per thread of those kernels (1 .. 16, default 1).
 * MPMC_OPT_SWEEP_STENCIL (mask 0 .. 127, default 55): t-sweep form of the
 * stencil steps whose input is a stored block, on handles whose x, y, z
 * extents are even: a CTA walks t over a 2 x 2 x 2 block of sites and a
 * tile of right-hand sides, with the block's spinor planes staged in shared
 * memory by TMA, and reads only the three neighbours outside the block from
 * global memory.  Bits 1, 2, 4: the issue-lean kernels of that class run in
 * t-sweep form; bit 8: steps outside the issue-lean set (other FP32 / BF16S
 * block widths with 16-byte rows, or classes not in the fast mask) run the
 * site-parallel arithmetic in t-sweep form; bit 16: each plane's links are
 * staged in shared memory with its spinor rows (tiles of 16 right-hand
 * sides, three CTAs per SM); bit 32: the warp-per-site form of that kernel
 * (tiles of 32 right-hand sides, one warp per site of the block, a ring of
 * three planes, no CTA-wide barrier per plane; blocks of 32 or more columns,
 * others run the bit-16 form); bit 64: the two-sites-per-warp form (tiles
 * of 16 right-hand sides, each warp holding the block's two x-sites, one
 * per half-warp, so that one 16-byte link load serves both; a ring of three
 * planes, no CTA-wide barrier per plane, four CTAs per SM; opt-in).  Same
 * arithmetic per site as the non-sweep
 * kernel; the order in which the eight hops are summed and the order of the
 * FP64 per-block dot sums differ.  mpmc_autotune times the forms the mask
 * allows and keeps the fastest; mpmc_get_option returns the mask in effect
 * (class bits, plus 16, 32 or 64 for the form that runs at the current block).
 * MPMC_OPT_SWEEP_ORDER (default 1): order in which the t-sweep CTAs take the
 * (2 x 2 x 2 site block, t-segment) pairs: 0 blocks in row order (x fastest)
 * for each segment in turn; 1 the segments of one block one after another,
 * the blocks along a Morton curve of the block grid, so that CTAs running at
 * the same time cover a compact region of the lattice and the neighbour rows
 * and shared t-planes they read from each other are still in L2.
 * MPMC_OPT_WAIT_LIMIT: bound of every wait of the t-sweep issue-lean kernels
 * on their TMA pipeline, in thousands of SM clock cycles (1 .. 4000000;
 * default 4000000, about 2 s).  A wait that runs out makes the CTA stop
 * issuing copies, wait (bounded) for the copies it issued and leave; the
 * call then returns MPMC_ETIMEOUT and the handle stays usable.
 * MPMC_OPT_TEST_SKIP_COPY (failure-detection test hook, default 0 = off):
 * value q >= 1 makes every t-sweep CTA leave out the copy of the q-th plane of
 * its ring, so that the wait for it runs out with nothing in flight into
 * that buffer.  Not for production use.
 * MPMC_OPT_SWEEP_SEGMENT: t-extent walked by one CTA (0 = automatic, else
 * 1 .. Lt); mpmc_get_option returns the length in effect.  mpmc_autotune
 * sets all four options: block width and the dotted class's kernel from
 * noise-started trace chains, then per class the faster of the
 * site-parallel, issue-lean and t-sweep kernels on chains of that class,
 * and, when polynomials are set, the fastest of a few class assignments on
 * one block of the handle's own mpmc_trace_levels.
 */
enum {
    MPMC_OPT_TENSOR_CORE_DEFLATION = 1,
    MPMC_OPT_SWEEP_STENCIL = 2,
    MPMC_OPT_SWEEP_SEGMENT = 3,
    MPMC_OPT_FAST_STENCIL = 4,
    MPMC_OPT_FAST_SITES = 5,
    MPMC_OPT_WAIT_LIMIT = 6,
    MPMC_OPT_TEST_SKIP_COPY = 7,
    MPMC_OPT_SWEEP_ORDER = 8
};
MPMC_API int mpmc_set_option(mpmc_handle h, int option, int value);
MPMC_API int mpmc_get_option(mpmc_handle h, int option, int* value);

/*
 * mpmc_deflation_dots: the deflation inner products of Sec. 4.1 for noise
 * vectors first .. first+nrhs-1 of level `level`: G1[i][c] = z_i^H b_c and
 * G2[i][c] = z_i^H gamma5 b_c (host outputs, k x nrhs complex, row i at
 * offset 2*i*nrhs), computed by the path the handle uses in
 * mpmc_trace_levels (tensor cores or CUDA cores), with z_i as stored.
 * Errors: ESTATE (no deflation), EINVAL, ETIMEOUT, ECUDA.
 */
MPMC_API int mpmc_deflation_dots(mpmc_handle h, uint64_t seed, int level, int first, int nrhs, double* G1,
                                 double* G2);

/*
 * mpmc_set_deflation_device: as mpmc_set_deflation, with Z a device
 * pointer (same layout); lambda and pair stay on the host.
 */
MPMC_API int mpmc_set_deflation_device(mpmc_handle h, const double* Z, const double* lambda, const int* pair, int k);

/*
 * mpmc_deflation_norms: d_i = z_pair(i)^H gamma5 z_i (k complex values,
 * interleaved re/im) of the deflation vectors as the handle stores them
 * (FP64, or the BF16 hi + lo split on reduced-precision handles).  The left
 * vectors are u_i = gamma5 z_pair(i) / conj(d_i), so that u_i^H z_i = 1
 * (Secs. 2.2, 4.1); |u_i| = 1 / |d_i| for unit z, and the deflation term of
 * a level sample grows like 1 / |d_i|, so a caller can drop pairs whose
 * |d_i| is too small to normalise stably.  Errors: ESTATE (no deflation).
 */
MPMC_API int mpmc_deflation_norms(mpmc_handle h, double* d);

/*
 * mpmc_solve: x = A^{-1} b for nrhs right-hand sides (layout of
 * mpmc_apply_poly; host or device per on_device) by restarted GMRES(m) on the
 * polynomial-preconditioned operator A p_in(A) (Sec. 2.4; polynomial `pin`,
 * a single polynomial, or pin < 0 for plain GMRES), with a Left-right
 * Projection with the deflation vectors before every cycle when they are set
 * (Secs. 2.1 and 5, step 3a).  FP64 handles only.  Stops when
 * |b - A x| <= rtol |b| or after maxcycles cycles; relres (optional, nrhs)
 * receives the final relative residuals, matvecs (optional) the products
 * with A.  Errors: ENOTSUP (precision, p_in kind), EINVAL, ESTATE.
 *
 * mpmc_trace_inverse: samples of the level Tr(A^{-1} - p_1(A)) (Sec. 3.1,
 * Eq. (2); the first Monte Carlo of Sec. 5, step 3a): for Z4 noise b_j
 * (level id 0xFFFF, noise index first + j), s_j = b_j^H x_j - b_j^H p_1(A) b_j
 * - sum_i c_i (b_j^H z_i)(u_i^H b_j) with x_j from mpmc_solve and
 * c_i = 1/lambda_i - p_1(lambda_i); mean (1 complex) adds sum_i c_i.  var: the
 * variance of Re s; samples optional (nsamples complex).  FP64 handles only.
 * p_1 may be the projected composite (Sec. 4.3): then b^H M_1 b with
 * M_1 b = Z D + p_1(A)(b - (A Z) D), D = H^{-1} U^H b, and c_i = 0 (A^{-1}
 * and M_1 both map z_i to z_i / lambda_i).
 */
MPMC_API int mpmc_solve(mpmc_handle h, int pin, const double* B, double* X, int nrhs, double rtol, int m,
                        int maxcycles, int on_device, double* relres, long long* matvecs);
MPMC_API int mpmc_trace_inverse(mpmc_handle h, int p1, int pin, uint64_t seed, int nsamples, int first, double rtol,
                                int m, int maxcycles, double* mean, double* var, double* samples);

/*
 * mpmc_trace_probing: the probing estimate of Tr p(A) for polynomial `index`
 * (single or composite), used for the lowest-degree level in place of its
 * Monte Carlo (Sec. 5, step 3c: the trace of the cheapest polynomial can be
 * found exactly).  Probe vectors: for each colour c of the period-m
 * colouring colour(x) = x%m + m (y%m) + m^2 (z%m) + m^3 (t%m) and each of the
 * 12 spin-colour components e, the indicator of {sites of colour c} x {e};
 * trace = sum over the 12 m^4 vectors of v^H p(A) v (complex, interleaved).
 * Sites of one colour are m or more hops apart, so the estimate is exact for
 * polynomials of degree below m, and for any degree when m equals every
 * extent.  m must divide every lattice extent.  The vectors run through the
 * same chain kernels as mpmc_apply_poly in blocks of the handle's width; the
 * in-colour sums are FP64 in a fixed order.  Errors: EINVAL (m), ESTATE (no
 * polynomial), ENOTSUP (projected composite).
 */
MPMC_API int mpmc_trace_probing(mpmc_handle h, int index, int m, double* trace);

/*
 * mpmc_colouring: a distance-`distance` colouring of the graph of A on the
 * periodic lattice `dims` (Sec. 3.1: p_3 is chosen of low enough degree for
 * its trace to be found by probing with a distance colouring of that graph;
 * Sec. 5, step 3d).  Sites whose hop distance on the periodic lattice is at
 * most `distance` get different colours, so probing with it is exact for
 * polynomials of degree <= distance.  colours: V ints (host, caller-owned)
 * receiving colour(site) in 0 .. *ncolours-1.  Greedy colouring in the
 * order of a linear colouring of Z^4; host only (no GPU, no handle);
 * deterministic.  About 110 colours for distance 4 on 24^3 x 32.
 * Errors: EINVAL (dims < 2, distance < 0, NULL pointer), ENOTSUP (a greedy
 * pass of more than 8e9 neighbour checks).
 *
 * mpmc_trace_probing_colours: the probing estimate of Tr p(A) for polynomial
 * `index` with any site colouring (colours: V host ints in 0 .. ncolours-1,
 * copied): the sum over the 12 * ncolours vectors "indicator of the sites of
 * colour c, component e" of v^H p(A) v, through the same chain kernels and
 * FP64 fixed-order sums as mpmc_trace_probing.  Exact when same-coloured
 * sites are more hops apart than the degree of p (e.g. a colouring from
 * mpmc_colouring with distance >= degree).  Errors: EINVAL (colour out of
 * range, ncolours < 1), ESTATE, ENOTSUP as mpmc_trace_probing.
 */
MPMC_API int mpmc_colouring(const int dims[4], int distance, int* colours, int* ncolours);

/*
 * mpmc_fma_peak: measured FMA throughput of the CUDA cores of the current
 * device in TFLOP/s (2 flops per FMA), for precision MPMC_FP64 or MPMC_FP32:
 * independent FMA chains on every SM, timed with CUDA events after a warm-up
 * launch.  The ALU roofline of the FP64 stencil path, which is bound by FP64
 * arithmetic rather than HBM on GB300.  The paper has no counterpart (it
 * reports desktop-CPU wall times only).  Allocates one small device buffer.
 * Errors: EINVAL (NULL), ENOTSUP (precision), ENOMEM, ECUDA.
 */
MPMC_API int mpmc_fma_peak(int precision, double* tflops);
MPMC_API int mpmc_trace_probing_colours(mpmc_handle h, int index, const int* colours, int ncolours,
                                        double* trace);

/*
 * mpmc_trace_level: one level of mpmc_trace_levels on its own (the same
 * samples, noise indices first .. first+nsamples-1 of that level), for the
 * sequential stopping rule of Sec. 5, step 3, which runs the Monte Carlos one
 * after another, each until its standard error meets its share of the
 * tolerance.  mean: 1 complex (with the level's exact correction), var: 1,
 * samples: nsamples complex (optional).  Errors: as mpmc_trace_levels.
 */
MPMC_API int mpmc_trace_level(mpmc_handle h, int level, uint64_t seed, int nsamples, int first, double* mean,
                              double* var, double* samples);

/*
 * mpmc_vector_stats: for k device vectors z_i (vector-major, complex double,
 * vector i at Z + 2*n*i) writes stats[4i..4i+3] = (|z_i|^2, |A z_i|^2,
 * Re z_i^H A z_i, Im z_i^H A z_i), with A applied in FP64.  These give the
 * Rayleigh quotient lambda_i = z_i^H A z_i / |z_i|^2 and every residual norm
 * |A z_i - mu z_i| the eigen selection of Sec. 4 needs in closed form.
 */
MPMC_API int mpmc_vector_stats(mpmc_handle h, const double* Z, int k, double* stats);

/*
 * mpmc_project: the Left-right Projection of Sec. 2.1 with the deflation
 * vectors (V = Z, U = the gamma5 left vectors): R = B - A Z H^{-1} U^H B,
 * H = U^H A Z, for nrhs vectors in the block layout (host or device per
 * on_device).  Sec. 5, step 2c starts the PP-GMRES of the deflated
 * polynomial from such a projected Z4 vector.
 */
MPMC_API int mpmc_project(mpmc_handle h, const double* B, double* R, int nrhs, int on_device);

/*
 * Batches of independent instances (lattices of uneven size, their own kappa,
 * polynomials, deflation and precision): the multilevel estimates of all
 * handles in a batch run as parallel branches of one captured CUDA graph, so
 * that small instances overlap on the GPU and the batch costs one graph
 * launch on the host.  The paper treats one lattice at a time; this is the
 * batched form of mpmc_trace_levels for many of them.
 *
 * mpmc_batch_create: handles are borrowed (the caller keeps and destroys
 * them, after the batch); each must be on its own stream (not the legacy or
 * per-thread default stream, which cannot be captured).  mpmc_batch_trace_levels: noise vectors first ..
 * first+nsamples-1 of every handle (each with its own noise seed `seed`
 * and level ids as in mpmc_trace_levels); mean[2*(i*MPMC_MAX_POLYS + l)]
 * (complex) and var[i*MPMC_MAX_POLYS + l] receive level l of handle i (as
 * mpmc_trace_levels would return them, bit for bit).  The graph is captured
 * on the first call (after one plain run, which does any lazy allocation)
 * and replayed while (seed, nsamples, first) and every handle's state stay
 * the same; changing a handle (polynomials, deflation, links, options,
 * block, stream, autotune), or any call on it that allocates a device
 * buffer (a longer trace, an apply or deflation dots with another block
 * width), recaptures it.  mpmc_batch_launch_count: kernel
 * nodes replayed so far.  Errors: as mpmc_trace_levels, EINVAL (a handle on
 * the legacy default stream), ECUDA (capture or launch failed).
 */
typedef struct mpmc_batch* mpmc_batch_handle;
MPMC_API int mpmc_batch_create(mpmc_batch_handle* b, int n, const mpmc_handle* handles);
MPMC_API int mpmc_batch_trace_levels(mpmc_batch_handle b, uint64_t seed, int nsamples, int first, double* mean,
                                     double* var);
MPMC_API long long mpmc_batch_launch_count(mpmc_batch_handle b);
MPMC_API int mpmc_batch_destroy(mpmc_batch_handle b);

/*
 * mpmc_trace_poly_noalloc: Hutchinson samples s_j = b_j^H p(A) b_j of one
 * polynomial, j = first .. first+nsamples-1 (Z4 noise of level id `level`,
 * same bits as mpmc_noise), computed without allocating any device memory.
 * The paper has no counterpart: this is a deployment variant of the
 * single-polynomial trace of mpmc_trace_levels (same kernels, FP64).
 *
 * Who it is for: callers that cannot call cudaMalloc -- an application whose
 * framework owns the whole GPU through its own caching allocator, or code on a
 * latency-critical path where cudaMalloc's implicit device synchronisation is
 * not acceptable.  The call makes no cudaMalloc, cudaFree or other allocating
 * call and needs no handle.
 *
 * All intermediates (links in kernel layout, two chain vectors, FP64
 * accumulators, samples) live in one file-scope device array of
 * MPMC_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library
 * holds until the process exits.  Noise is processed in blocks of at most 64
 * vectors, narrowed until the block fits; a lattice whose single-vector
 * working set does not fit, 2*12*V*16 + 36*V*16 (+ 36*V*16 for host links)
 * bytes plus a few KB, is rejected with MPMC_EINVAL before any GPU work.
 *
 * Arguments: dims, kappa, bc_t as in mpmc_create; links in the mpmc_create
 * layout; roots: nroots complex values used in the given order (no Leja
 * reordering); samples: nsamples complex outputs.  on_device != 0: links and
 * samples are device pointers and the call is asynchronous on `stream`;
 * otherwise both are host pointers and the call synchronises `stream`.
 * stream: a cudaStream_t (NULL = legacy default stream).
 *
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (once per device, with that device current); make that
 * first call before any stream capture.  Every call shares the array and
 * leaves its contents behind (accumulators are cleared at the start of each
 * call): calls that overlap on the GPU -- from different streams or host
 * threads -- race on it and must be serialised by the caller.
 * Errors: EINVAL (arguments, or the lattice exceeds the array), ENONFINITE
 * (a zero or non-finite root), ENOTSUP (device index >= 128), ECUDA.
 */
#define MPMC_NOALLOC_SCRATCH_BYTES (32u << 20)
MPMC_API int mpmc_trace_poly_noalloc(const int dims[4], const double* links, double kappa, int bc_t,
                                     const double* roots, int nroots, uint64_t seed, int level,
                                     int first, int nsamples, double* samples, int on_device,
                                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPMC_H */
