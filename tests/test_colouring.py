"""The library's distance colourings (mpmc_colouring, host code): every pair
of same-coloured sites is more than `distance` hops apart on the periodic
lattice (checked over all pairs with a distance written out here), the
special distances give one colour and one colour per site, and distance 4 on
the 24^3 x 32 lattice needs about a hundred colours, not the 4096 of the
period-8 colouring."""

import numpy as np
import pytest

from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


def _coords(dims):
    V = int(np.prod(dims))
    s = np.arange(V)
    out = []
    for L in dims:
        out.append(s % L)
        s = s // L
    return np.stack(out, axis=1)


def _pair_distances(dims):
    c = _coords(dims)
    d = np.zeros((len(c), len(c)), dtype=np.int64)
    for mu, L in enumerate(dims):
        r = np.abs(c[:, None, mu] - c[None, :, mu])
        d += np.minimum(r, L - r)
    return d


@pytest.mark.parametrize("dims,distance", [((4, 4, 4, 4), 4), ((6, 4, 4, 8), 4), ((4, 2, 6, 4), 2),
                                           ((6, 6, 4, 4), 3), ((2, 2, 2, 2), 1)])
def test_same_colour_sites_are_farther_apart_than_the_distance(dims, distance):
    colours, nc = G.mpmc_colouring(dims, distance)
    assert colours.min() == 0 and colours.max() == nc - 1
    d = _pair_distances(dims)
    same = colours[:, None] == colours[None, :]
    np.fill_diagonal(same, False)
    assert np.all(d[same] > distance)


def test_degenerate_distances():
    c, n = G.mpmc_colouring((4, 2, 2, 4), 0)
    assert n == 1 and np.all(c == 0)
    c, n = G.mpmc_colouring((4, 2, 2, 4), 6)          # 2 + 1 + 1 + 2: every site within reach
    assert n == 64 and np.array_equal(c, np.arange(64))
    with pytest.raises(G.MpmcError):
        G.mpmc_colouring((4, 1, 2, 4), 2)
    with pytest.raises(G.MpmcError):
        G.mpmc_colouring((4, 2, 2, 4), -1)


def test_distance_four_on_the_large_lattice_needs_about_a_hundred_colours():
    colours, nc = G.mpmc_colouring((24, 24, 24, 32), 4)
    assert 41 <= nc <= 120
    counts = np.bincount(colours, minlength=nc)
    assert counts.sum() == 24 ** 3 * 32 and counts.min() > 0
