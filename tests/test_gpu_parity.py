"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  * noise: bit-exact (integer work);
  * FP64 path: 1e-13 relative for one product with A, 1e-11 for polynomial
    applies, 1e-12 relative per level sample (relative to the magnitude of
    the summed terms |b^H p_l b| + |b^H p_{l+1} b| + |deflation term|);
  * FP32 path: 3e-6 relative for A; for level samples the paired bound on
    identical noise (conftest.paired_bound): bias |mean(s32 - s64)| <=
    0.1 SE64 + 3 std(s32 - s64)/sqrt(N), noise std(s32 - s64) <=
    max(0.3 std(s64), u32 <|b^H p_l b| + |b^H p_{l+1} b|>);
  * BF16-stored path: 1.5e-2 relative for A (inputs rounded to bf16).
"""

import functools

import numpy as np
import pytest

from conftest import fp32_polys, fp32_resolution, links, operator, paired_bound
from oracle import krylov as K
from oracle import mpmc as M
from oracle import philox
from oracle import polynomial as P
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G
from paper_2306_09559_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


def handle(dims, kind="haar", seed=0, kappa=0.12, eps=0.3, prec=G.FP64, bc_t=1):
    return G.Handle(links(dims, kind, seed, eps), kappa, prec, bc_t)


@functools.lru_cache(maxsize=None)
def small_setup(dims=(4, 4, 4, 4), seed=0, kappa=0.12):
    """Roots and deflation vectors from the oracle's setup (Sec. 5, step 2)."""
    op = operator(dims, "haar", seed, kappa)
    b0 = synth.random_unit_vector(op.n, 17)
    p_hi, p_lo, p_in = K.gmres_polynomials(op, b0, [24, 9, 4])
    p_out, _, _ = K.pp_gmres_roots(op, p_in, b0, m_out=6)
    lam, Z = K.pp_arnoldi_ritz(op, p_in, b0, m=120, nev=24)
    lam_s, Z_s, pair = K.select_deflation(op, op.gamma5, lam, Z)
    if lam_s.size < 4:          # any vectors define a valid (unbiased) deflation
        lam_s, Z_s, pair = lam[:8], Z[:, :8], np.arange(8)
    polys = [{"kind": "composite", "inner": p_in, "outer": p_out},
             {"kind": "single", "roots": p_hi},
             {"kind": "single", "roots": p_lo}]
    return op, polys, lam_s, Z_s, pair


def set_polys(h, polys):
    for i, p in enumerate(polys):
        if p["kind"] == "single":
            h.mpmc_set_poly(i, G.SINGLE, p["roots"], leja=False)
        else:
            kind = G.COMPOSITE if p["kind"] == "composite" else G.DEFLATED_COMPOSITE
            h.mpmc_set_poly(i, kind, p["inner"], p["outer"], leja=False)


# ---------------------------------------------------------------- noise
@pytest.mark.parametrize("seed,level,first,nrhs", [(0, 0, 0, 3), (1001, 2, 37, 5), ((7 << 32) + 5, 1, 1000, 2)])
def test_noise_bit_exact(seed, level, first, nrhs):
    with handle((4, 4, 2, 4)) as h:
        got = h.mpmc_noise(seed, level, first, nrhs)
        ref = philox.z4_block(seed, level, first, nrhs, h.V)
        assert np.array_equal(got, ref)


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), 1), ((2, 2, 2, 2), 1), ((3, 2, 5, 4), -1), ((6, 4, 2, 2), 1)])
@pytest.mark.parametrize("nrhs,block", [(1, 0), (5, 0), (70, 32), (33, 8)])
def test_apply_op_fp64(dims, bc_t, nrhs, block):
    op = operator(dims, "haar", 1, 0.13, 0.3, bc_t)
    X = synth.random_block(op.n, nrhs, 3)
    with handle(dims, "haar", 1, 0.13, 0.3, G.FP64, bc_t) as h:
        if block:
            h.mpmc_set_block(block)
        Y = h.mpmc_apply_op(X)
    ref = op(X)
    assert np.max(np.abs(Y - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,tol", [(G.FP32, 3e-6), (G.BF16S, 1.5e-2)])
def test_apply_op_reduced_precision(prec, tol):
    dims = (4, 4, 4, 4)
    op = operator(dims, "near_identity", 2, 0.123, 0.3)
    X = synth.random_block(op.n, 40, 4)
    with handle(dims, "near_identity", 2, 0.123, 0.3, prec) as h:
        Y = h.mpmc_apply_op(X)
    ref = op(X)
    assert np.max(np.abs(Y - ref)) <= tol * np.max(np.abs(ref))


def test_apply_op_device_pointers():
    torch = pytest.importorskip("torch")
    dims = (4, 4, 2, 4)
    op = operator(dims, "haar", 0, 0.12)
    X = synth.random_block(op.n, 7, 9)
    with handle(dims) as h:
        h.mpmc_set_stream(torch.cuda.current_stream())
        Xd = torch.from_numpy(X).cuda()
        Yd = h.mpmc_apply_op(Xd)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy()
    assert np.max(np.abs(Y - op(X))) <= 1e-13 * np.max(np.abs(Y))


# ---------------------------------------------------------------- polynomials
@pytest.mark.parametrize("which", [0, 1, 2])
def test_apply_poly_fp64(which):
    op, polys, *_ = small_setup()
    B = synth.random_block(op.n, 19, 5)
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_block(8)
        set_polys(h, polys)
        X = h.mpmc_apply_poly(which, B)
    ref = M.apply_spec(op, polys[which], B)
    assert np.linalg.norm(X - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("m_in,m_out", [(1, 4), (3, 1), (1, 1), (2, 2)])
def test_apply_composite_degenerate_shapes(m_in, m_out):
    op = operator((2, 2, 2, 4), "haar", 0, 0.12)
    inner = np.linspace(0.6, 1.4, m_in) + 0.2j
    outer = np.linspace(0.7, 1.3, m_out) - 0.1j
    B = synth.random_block(op.n, 3, 6)
    with handle((2, 2, 2, 4)) as h:
        h.mpmc_set_poly(0, G.COMPOSITE, inner, outer, leja=False)
        X = h.mpmc_apply_poly(0, B)
    ref = P.apply_composite(op, inner, outer, B)
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)


def test_single_root_polynomial():
    op = operator((2, 2, 2, 4), "haar", 0, 0.12)
    B = synth.random_block(op.n, 2, 1)
    with handle((2, 2, 2, 4)) as h:
        h.mpmc_set_poly(0, G.SINGLE, [0.8 + 0.1j], leja=False)
        X = h.mpmc_apply_poly(0, B)
        mean, var, s = h.mpmc_trace_levels(3, 4)
    assert np.allclose(X, B / (0.8 + 0.1j), rtol=1e-15, atol=0)
    assert np.allclose(s[0], op.n / (0.8 + 0.1j), rtol=1e-14)


def test_leja_order_matches_oracle(rng):
    for trial in range(4):
        r = rng.standard_normal(23) + 1j * rng.standard_normal(23)
        with handle((2, 2, 2, 2)) as h:
            h.mpmc_set_poly(0, G.SINGLE, r, leja=True)
            got = h.mpmc_get_roots(0, r.size)
        assert np.array_equal(got, r[P.leja_order(r)])


# ---------------------------------------------------------------- level samples
def test_trace_levels_fp64_per_sample():
    op, polys, lam, Z, pair = small_setup()
    defl = M.Deflation(op, Z, lam, pair)
    N = 21                                  # ragged against the block of 8
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_block(8)
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, polys)
        mean, var, s = h.mpmc_trace_levels(seed=1234, nsamples=N, first=5)
        corr = [h.mpmc_level_info(l)[0] for l in range(3)]
    for level in range(3):
        ref, hi, lo, dt = M.level_sample_parts(op, polys, level, 1234, N, defl, first=5)
        scale = np.abs(hi) + np.abs(lo) + np.abs(dt)
        assert np.max(np.abs(s[level] - ref) / scale) < 1e-12, level
        assert abs(corr[level] - M.exact_correction(polys, level, defl)) < 1e-10 * (1 + abs(corr[level]))
        assert abs(mean[level] - (ref.mean() + corr[level])) < 1e-10 * np.max(scale)
        assert np.isclose(var[level], np.var(ref.real, ddof=1), rtol=1e-8)


def test_trace_levels_fp32_paired_bound():
    op, polys, lam, Z, pair = small_setup()
    polys = fp32_polys(polys)           # the polynomial an FP32 chain applies, on both sides
    defl = M.Deflation(op, Z, lam, pair)
    N = 48
    with handle((4, 4, 4, 4), prec=G.FP32) as h:
        h.mpmc_set_block(16)
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, polys)
        _, _, s = h.mpmc_trace_levels(seed=99, nsamples=N)
    for level in range(3):
        ref, hi, lo, dt = M.level_sample_parts(op, polys, level, 99, N, defl)
        paired_bound(s[level] - ref, ref, resolution=fp32_resolution(hi, lo))


@pytest.mark.parametrize("prec", [G.FP64, G.FP32])
def test_launch_shapes_do_not_change_samples(prec):
    op, polys, lam, Z, pair = small_setup()
    out = []
    shapes = [(8, 1, 64, 1), (16, 2, 32, 1), (32, 2, 64, 2), (12, 2, 32, 4), (7, 2, 32, 1), (64, 1, 32, 2)]
    for nb, R, bx, sl in shapes:
        with handle((4, 4, 4, 4), prec=prec) as h:
            h.mpmc_set_block(nb)
            h.mpmc_set_launch(R, bx, sl)
            h.mpmc_set_deflation(Z, lam, pair)
            set_polys(h, polys)
            out.append(h.mpmc_trace_levels(seed=5, nsamples=30)[2])
    tol = 1e-12 if prec == G.FP64 else 2e-6
    for o in out[1:]:
        assert np.max(np.abs(o - out[0])) < tol * op.n


def test_autotune_picks_a_valid_shape():
    op, polys, lam, Z, pair = small_setup()
    with handle((4, 4, 4, 4), prec=G.FP32) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, polys)
        cfg = h.mpmc_autotune(64)
        assert cfg["nb"] in (16, 32, 64) and cfg["R"] in (1, 2) and cfg["bx"] in (32, 64) and cfg["sl"] in (1, 2)
        s = h.mpmc_trace_levels(seed=5, nsamples=20)[2]
    ref = M.level_samples(op, polys, 2, 5, 20)
    assert np.max(np.abs(s[2] - ref)) < 1e-5 * op.n


def test_trace_block_size_does_not_change_samples():
    op, polys, lam, Z, pair = small_setup()
    out = []
    for nb in (1, 7, 32):
        with handle((4, 4, 4, 4)) as h:
            h.mpmc_set_block(nb)
            h.mpmc_set_deflation(Z, lam, pair)
            set_polys(h, polys)
            out.append(h.mpmc_trace_levels(seed=5, nsamples=9)[2])
    # level samples cancel terms of size ~n; summation order may differ by block
    for o in out[1:]:
        assert np.max(np.abs(o - out[0])) < 1e-12 * op.n


# ---------------------------------------------------------------- projected composite (Sec. 4.3)
def _projected(polys):
    return [dict(polys[0], kind="deflated_composite")] + list(polys[1:])


def test_apply_projected_composite_fp64():
    op, polys, lam, Z, pair = small_setup()
    defl = M.Deflation(op, Z, lam, pair)
    pp = _projected(polys)
    B = synth.random_block(op.n, 11, 13)
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_block(8)
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, pp)
        X = h.mpmc_apply_poly(0, B)
    ref = M.apply_spec(op, pp[0], B, defl)
    assert np.linalg.norm(X - ref) <= 1e-11 * np.linalg.norm(ref)
    # it maps A z_i to z_i (the projection is exact on the deflation space)
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, pp)
        AZ = h.mpmc_apply_op(Z)
        back = h.mpmc_apply_poly(0, AZ)
    assert np.linalg.norm(back - Z) < 1e-9 * np.linalg.norm(Z)


@pytest.mark.parametrize("nsamples,block", [(21, 8), (9, 32)])
def test_trace_projected_composite_fp64_per_sample(nsamples, block):
    op, polys, lam, Z, pair = small_setup()
    defl = M.Deflation(op, Z, lam, pair)
    pp = _projected(polys)
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_block(block)
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, pp)
        mean, var, s = h.mpmc_trace_levels(seed=808, nsamples=nsamples, first=2)
        corr = h.mpmc_level_info(0)[0]
    ref, hi, lo, dt = M.level_sample_parts(op, pp, 0, 808, nsamples, defl, first=2)
    scale = np.abs(hi) + np.abs(lo) + np.abs(dt)
    assert np.max(np.abs(s[0] - ref) / scale) < 1e-12
    assert abs(corr - M.exact_correction(pp, 0, defl)) < 1e-10 * (1 + abs(corr))
    # the other levels are unchanged
    for level in (1, 2):
        r2, hi2, lo2, dt2 = M.level_sample_parts(op, pp, level, 808, nsamples, defl, first=2)
        assert np.max(np.abs(s[level] - r2) / (np.abs(hi2) + np.abs(lo2) + np.abs(dt2))) < 1e-12


def test_trace_projected_composite_fp32_paired():
    op, polys, lam, Z, pair = small_setup()
    polys = fp32_polys(polys)
    defl = M.Deflation(op, Z, lam, pair)
    pp = _projected(polys)
    N = 40
    with handle((4, 4, 4, 4), prec=G.FP32) as h:
        h.mpmc_set_block(20)
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, pp)
        _, _, s = h.mpmc_trace_levels(seed=9, nsamples=N)
    ref, hi, lo, dt = M.level_sample_parts(op, pp, 0, 9, N, defl)
    paired_bound(s[0] - ref, ref, resolution=fp32_resolution(hi, lo))


def test_projected_composite_only_at_the_top():
    with handle((2, 2, 2, 2)) as h:
        Z = synth.random_block(h.n, 2, 3)
        h.mpmc_set_deflation(Z, [1.0 + 0.1j, 1.0 - 0.1j], [1, 0])
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_set_poly(1, G.DEFLATED_COMPOSITE, [1.0], [1.0, 2.0])
        assert e.value.code == G.MPMC_EINVAL


# ---------------------------------------------------------------- deflation dots
def _zhat(Z):
    """z rounded as the reduced-precision handles store it: hi = bf16(z), lo = bf16(z - hi)."""
    torch = pytest.importorskip("torch")
    Zc = np.ascontiguousarray(Z)
    x = torch.from_numpy(Zc.view(np.float64)).float()
    hi = x.bfloat16().float()
    lo = (x - hi).bfloat16().float()
    return np.ascontiguousarray((hi + lo).double().numpy()).view(np.complex128).reshape(Zc.shape)


@pytest.mark.parametrize("nrhs", [1, 37, 64, 130])
def test_deflation_dots_tensor_core_vs_cuda_core_vs_oracle(nrhs):
    op, polys, lam, Z, pair = small_setup()
    with handle((4, 4, 4, 4), prec=G.FP32) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        assert h.mpmc_get_option(G.OPT_TENSOR_CORE_DEFLATION) == 1
        T1, T2 = h.mpmc_deflation_dots(31, 1, 7, nrhs, lam.size)
        h.mpmc_set_option(G.OPT_TENSOR_CORE_DEFLATION, 0)
        assert h.mpmc_get_option(G.OPT_TENSOR_CORE_DEFLATION) == 0
        C1, C2 = h.mpmc_deflation_dots(31, 1, 7, nrhs, lam.size)
    B = philox.z4_block(31, 1, 7, nrhs, op.n // 12)
    Zh = _zhat(Z)
    R1 = Zh.conj().T @ B
    R2 = Zh.conj().T @ op.gamma5(B)
    scale = np.max(np.abs(R1))
    # both device paths use zhat with FP32 accumulation
    for got in (T1, C1):
        assert np.max(np.abs(got - R1)) < 2e-6 * scale
    for got in (T2, C2):
        assert np.max(np.abs(got - R2)) < 2e-6 * scale
    # and zhat is within the BF16 hi + lo precision of z
    assert np.max(np.abs(Z.conj().T @ B - R1)) < 1e-3 * scale


def test_deflation_dots_fp64_path():
    op, polys, lam, Z, pair = small_setup()
    with handle((4, 4, 4, 4), prec=G.FP64) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        assert h.mpmc_get_option(G.OPT_TENSOR_CORE_DEFLATION) == 0
        G1, G2 = h.mpmc_deflation_dots(5, 0, 0, 9, lam.size)
    B = philox.z4_block(5, 0, 0, 9, op.n // 12)
    assert np.max(np.abs(G1 - Z.conj().T @ B)) < 1e-12 * np.max(np.abs(G1))
    assert np.max(np.abs(G2 - Z.conj().T @ op.gamma5(B))) < 1e-12 * np.max(np.abs(G2))


def test_trace_with_tensor_core_deflation_matches_cuda_core():
    op, polys, lam, Z, pair = small_setup()
    out = []
    for tcore in (1, 0):
        with handle((4, 4, 4, 4), prec=G.FP32) as h:
            h.mpmc_set_block(32)
            h.mpmc_set_deflation(Z, lam, pair)
            h.mpmc_set_option(G.OPT_TENSOR_CORE_DEFLATION, tcore)
            set_polys(h, polys)
            out.append(h.mpmc_trace_levels(seed=3, nsamples=40)[2])
    assert np.max(np.abs(out[0] - out[1])) < 1e-8 * op.n


# ---------------------------------------------------------------- setup kernels
def test_arnoldi_fp64_matches_oracle():
    dims = (4, 4, 4, 4)
    op = operator(dims, "haar", 0, 0.12)
    v0 = synth.random_unit_vector(op.n, 3)
    m = 25
    V, Hb, beta = K.arnoldi(op, v0, m)
    with handle(dims, prec=G.FP32) as h:          # setup is FP64 on any handle
        Hg, steps = h.mpmc_arnoldi(-1, v0, m)
    assert steps == m
    assert np.max(np.abs(Hg - Hb)) < 1e-11 * np.max(np.abs(Hb))


def test_pp_arnoldi_fp64_matches_oracle():
    op, polys, *_ = small_setup()
    p_in = polys[0]["inner"]
    v0 = synth.random_unit_vector(op.n, 4)
    m = 12
    V, Hb, beta = K.arnoldi(K.pp_operator(op, p_in), v0, m)
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_poly(0, G.SINGLE, p_in, leja=False)
        Hg, steps = h.mpmc_arnoldi(0, v0, m)
    assert np.max(np.abs(Hg - Hb)) < 1e-11 * np.max(np.abs(Hb))


def test_combine_forms_ritz_vectors():
    torch = pytest.importorskip("torch")
    dims = (4, 4, 2, 4)
    op = operator(dims, "haar", 0, 0.12)
    v0 = synth.random_unit_vector(op.n, 8)
    m = 10
    V, Hb, _ = K.arnoldi(op, v0, m)
    Y = np.random.default_rng(1).standard_normal((m, 3)) + 0j
    with handle(dims) as h:
        basis = torch.zeros((m + 1, op.n), dtype=torch.complex128, device="cuda")
        h.mpmc_arnoldi(-1, v0, m, basis=basis)
        Zd = torch.zeros((3, op.n), dtype=torch.complex128, device="cuda")
        h.mpmc_combine(basis, m, Y, Zd)
        Zg = Zd.cpu().numpy().T
    assert np.max(np.abs(Zg - V[:, :m] @ Y)) < 1e-12 * np.max(np.abs(Zg))


# ---------------------------------------------------------------- product-side setup
def test_product_setup_matches_oracle_setup():
    """Roots and accepted eigenpairs of the GPU setup agree with the oracle's (Sec. 5, step 2)."""
    from paper_2306_09559_gb300 import krylov_setup
    dims, kappa = (4, 4, 4, 4), 0.12
    op = operator(dims, "haar", 0, kappa)
    v0 = synth.random_unit_vector(op.n, 17)
    with handle(dims, kappa=kappa) as h:
        S = krylov_setup.Setup(h)
        r24, r4 = S.single_roots(v0, [24, 4])
        Zd, lam, pair = S.eigenpairs(r4, v0, m=120, ndefinit=24)
        out5, _ = S.pp_roots(r4, v0, m_out=6)
    o24, o4 = K.gmres_polynomials(op, v0, [24, 4])
    oout, _, _ = K.pp_gmres_roots(op, o4, v0, m_out=6)
    for got, ref in ((r24, o24), (r4, o4), (out5, oout)):
        d = np.abs(got[:, None] - ref[None, :])
        assert np.max(np.min(d, axis=1)) < 1e-8 and np.max(np.min(d, axis=0)) < 1e-8
    olam, oZ = K.pp_arnoldi_ritz(op, o4, v0, m=120, nev=24)
    olam_s, _, opair = K.select_deflation(op, op.gamma5, olam, oZ)
    assert lam.size == olam_s.size and lam.size > 0
    d = np.abs(lam[:, None] - olam_s[None, :])
    assert np.max(np.min(d, axis=1)) < 1e-8
    assert np.array_equal(np.sort(pair - np.arange(pair.size)), np.sort(opair - np.arange(opair.size)))
    # the accepted vectors are eigenvectors of A to the selection tolerance
    Z = Zd.cpu().numpy().T
    assert np.max(np.linalg.norm(op(Z) - Z * lam, axis=0)) < K.EVECTOL


def test_left_right_projection_matches_oracle():
    op, polys, lam, Z, pair = small_setup()
    defl = M.Deflation(op, Z, lam, pair)
    B = synth.random_block(op.n, 5, 21)
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        R = h.mpmc_project(B)
    ref = K.left_right_projection(op, defl.Z, defl.U, B)[1]
    assert np.linalg.norm(R - ref) < 1e-11 * np.linalg.norm(ref)
    assert np.linalg.norm(defl.U.conj().T @ R) < 1e-10 * np.linalg.norm(B)


# ---------------------------------------------------------------- errors
def test_error_codes():
    with handle((2, 2, 2, 2)) as h:
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_trace_levels(1, 4)
        assert e.value.code == G.MPMC_ESTATE
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_set_poly(0, G.SINGLE, [0.0])
        assert e.value.code == G.MPMC_ENONFINITE
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_set_poly(9, G.SINGLE, [1.0])
        assert e.value.code == G.MPMC_EINVAL
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_set_poly(0, G.DEFLATED_COMPOSITE, [1.0], [1.0, 2.0])
        assert e.value.code == G.MPMC_ESTATE
        Z = np.ones((h.n, 2), dtype=complex)
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_set_deflation(Z, [1.0, 2.0], [1, 1])
        assert e.value.code == G.MPMC_EINVAL
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_set_block(5000)
        assert e.value.code == G.MPMC_EINVAL


def test_deflation_norms_match_oracle():
    """d_i = z_pair(i)^H gamma5 z_i as stored (FP64 handle) against the oracle's normalisation."""
    op, polys, lam, Z, pair = small_setup()
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        d = h.mpmc_deflation_norms()
    ref = np.einsum('ni,ni->i', op.gamma5(Z[:, pair]).conj(), Z)
    assert np.max(np.abs(d - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
