import os
import sys
import functools

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libmpmc.so")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@functools.lru_cache(maxsize=None)
def links(dims, kind="haar", seed=0, eps=0.3):
    from paper_2306_09559_gb300 import synth
    return synth.gauge_field(dims, kind=kind, seed=seed, eps=eps)


@functools.lru_cache(maxsize=None)
def operator(dims, kind="haar", seed=0, kappa=0.12, eps=0.3, bc_t=1):
    from oracle.lattice import WilsonOperator
    return WilsonOperator(links(dims, kind, seed, eps), kappa, bc_t)


@functools.lru_cache(maxsize=None)
def dense(dims, kind="haar", seed=0, kappa=0.12, eps=0.3, bc_t=1):
    from oracle.lattice import dense_A
    return dense_A(links(dims, kind, seed, eps), kappa, bc_t)


@pytest.fixture
def rng():
    return np.random.Generator(np.random.PCG64(12345))


U32 = 2.0 ** -24     # unit roundoff of FP32


def fp32_resolution(hi, lo):
    """FP32 resolution of one level sample: u32 times the mean size of the two traced terms
    |b^H p_l b| + |b^H p_{l+1} b|, whose difference the sample is."""
    return U32 * float(np.mean(np.abs(hi) + np.abs(lo)))


def paired_bound(d, ref, noise_frac=0.3, resolution=0.0):
    """The mixed-precision bound on identical noise, for the paired differences
    d = s_mixed - s_64 of N samples and the FP64 samples ref (real parts):

      bias:   |mean d| <= 0.1 SE_64 + 3 std(d) / sqrt(N)
      noise:  std(d)   <= max(noise_frac std(s_64), resolution)   (skipped when noise_frac is None)

    The bias test allows for the sampling noise of the N differences at three
    standard deviations; a bias above a tenth of the FP64 standard error that
    the pairing resolves fails it.  The noise test's second term is the
    resolution of one sample in the mixed precision (fp32_resolution): a level
    whose FP64 spread lies below it is resolved only to it.  Returns (bias,
    allowed bias, noise ratio)."""
    d = np.asarray(d).real
    ref = np.asarray(ref).real
    N = d.size
    se = np.std(ref, ddof=1) / np.sqrt(N)
    allowed = 0.1 * se + 3.0 * np.std(d, ddof=1) / np.sqrt(N)
    bias = abs(np.mean(d))
    ratio = np.std(d, ddof=1) / np.std(ref, ddof=1)
    assert bias <= allowed, f"bias {bias:.3e} > {allowed:.3e} (SE64 {se:.3e}, std(d)/std64 {ratio:.3e})"
    if noise_frac is not None:
        sd = np.std(d, ddof=1)
        assert sd <= max(noise_frac * np.std(ref, ddof=1), resolution), \
            f"std(d)/std64 = {ratio:.3e} > {noise_frac} and std(d) = {sd:.3e} > resolution {resolution:.3e}"
    return bias, allowed, ratio


def fp32_coefs(roots):
    """theta -> 1 / fl32(1 / theta): roots whose product-form coefficients 1/theta are FP32
    numbers, as MPMC_POLY_FP32_COEFS makes them.  Given to the oracle and to an FP32 handle, both
    apply the same polynomial, and their samples differ by arithmetic rounding alone."""
    c = 1.0 / np.asarray(roots, dtype=np.complex128)
    return 1.0 / c.astype(np.complex64).astype(np.complex128)


def fp32_polys(polys):
    """A level set with every root list passed through fp32_coefs."""
    out = []
    for p in polys:
        q = dict(p)
        for key in ("roots", "inner", "outer"):
            if key in q:
                q[key] = fp32_coefs(q[key])
        out.append(q)
    return out
