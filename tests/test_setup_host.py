"""Host-side logic of the GPU setup that needs no GPU: the conditioning
filter on deflation pairs (left vectors u_i = gamma5 z_pair(i) / conj(d_i)
of norm 1/|d_i|; Secs. 2.2 and 4)."""

import numpy as np

from paper_2306_09559_gb300 import krylov_setup


def test_well_conditioned_keeps_pairs_together():
    # 0: real, fine; 1: real, tiny d; 2, 3: conjugate pair, fine; 4, 5: pair with one tiny d
    d = np.array([0.9, 1e-6, 0.3 + 0.2j, 0.3 - 0.2j, 0.5, 2e-3])
    pair = np.array([0, 1, 3, 2, 5, 4])
    keep, pmap = krylov_setup.Setup.well_conditioned(d, pair, 1e-2)
    assert keep.tolist() == [0, 2, 3]
    assert pmap.tolist() == [0, 2, 1]
    # every kept entry's partner is kept and maps back
    assert all(pmap[pmap[i]] == i for i in range(keep.size))


def test_well_conditioned_keeps_everything_above_the_limit():
    d = np.array([0.5, 0.4j, 0.2])
    pair = np.array([0, 1, 2])
    keep, pmap = krylov_setup.Setup.well_conditioned(d, pair)
    assert keep.tolist() == [0, 1, 2] and pmap.tolist() == [0, 1, 2]
