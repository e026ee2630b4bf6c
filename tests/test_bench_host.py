"""Host logic of bench.py (no GPU): the t-sweep form named by a sweep mask, and the lookup of
captured DRAM traffic in profiles/dram_traffic.md.

The traffic table is keyed by a digest of each form's kernel sources.  The last test asks
that the default form (the warp-per-site kernel) has a row that matches the sources as they
stand, so that a change to the kernel without a new capture shows up here, not as a null
`roofline.traffic` in a bench line."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("mask,form", [(7, "k_fsweep"), (23, "k_fsweep_lsm"), (39, "k_fsweep_w"),
                                       (55, "k_fsweep_w"), (0, "k_fsweep"), (71, "k_fsweep_p")])
def test_fsweep_form(mask, form):
    assert bench.fsweep_form(mask) == form


def test_digest_depends_on_the_form_sources():
    d_lsm, d_w = bench.kernel_sources_digest("k_fsweep_lsm"), bench.kernel_sources_digest("k_fsweep_w")
    assert len(d_lsm) == 16 and len(d_w) == 16 and d_lsm != d_w
    assert bench.kernel_sources_digest("k_fsweep") == d_lsm   # same sources, other launch option


def test_captured_traffic_scales_by_sites():
    V = 24 ** 3 * 32
    got, src = bench.captured_traffic("k_fsweep_w", "fp32", 32, V)
    assert got is not None, "no capture of the default t-sweep form matches its current sources"
    small, _ = bench.captured_traffic("k_fsweep_w", "fp32", 32, V // 4)
    assert got == pytest.approx(4 * small)
    assert "scaled by" in src


def test_captured_traffic_misses():
    assert bench.captured_traffic("k_fsweep_w", "bf16s", 32, 1000) == (None, None)
    assert bench.captured_traffic("k_fsweep_w", "fp32", 64, 1000) == (None, None)
    assert bench.captured_traffic("no_such_kernel", "fp32", 32, 1000) == (None, None)
