"""Philox-4x32-10 and Z4 noise (oracle; test infrastructure only).

The method samples Z4 noise vectors, entries drawn uniformly from
{1, -1, i, -i} (Sec. 1; Sec. 5, step 3).  The paper does not say how they
are drawn.  The project reads it as a counter-based generator so that any
noise vector can be regenerated anywhere from its index:

* generator: Philox-4x32-10 of Salmon, Moraes, Dror and Shaw ("Parallel
  random numbers: as easy as 1, 2, 3", SC'11), written here from that
  paper's definition: multipliers 0xD2511F53 and 0xCD9E8D57, Weyl key
  increments 0x9E3779B9 and 0xBB67AE85, ten rounds, the key bumped between
  consecutive rounds;
* key = (seed & 0xffffffff, seed >> 32);
* counter = (noise index j, site index, level id, 0);
* the 12 entries of a site (spin*3 + colour = e) take bits 2e and 2e+1 of
  output word 0 as q in {0, 1, 2, 3} and map it to i**q, i.e.
  0 -> 1, 1 -> i, 2 -> -1, 3 -> -i.

The GPU library implements the same definition independently.

Parity unpinned (bit pattern): no published known-answer vector of
Philox-4x32-10 is available offline, so the exact output bits are pinned
only by agreement of the two independent implementations; the statistical
tests pin uniformity and independence of the Z4 symbols.
"""

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds on uint32 counter words (numpy arrays, broadcast)."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


_Z4 = np.array([1, 1j, -1, -1j], dtype=np.complex128)


def z4_symbols(seed, level, noise_index, nsites):
    """Integer symbols q[site, e] in 0..3 for one noise vector."""
    sites = np.arange(nsites, dtype=np.uint64)
    w0, _, _, _ = philox4x32_10(np.uint64(noise_index), sites, np.uint64(level), np.uint64(0),
                                np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32))
    w0 = w0.astype(np.uint64)
    shifts = (2 * np.arange(12, dtype=np.uint64))[None, :]
    return ((w0[:, None] >> shifts) & np.uint64(3)).astype(np.int64)


def z4_noise(seed, level, noise_index, nsites):
    """One Z4 noise vector as a flat complex n-vector (n = 12 * nsites)."""
    return _Z4[z4_symbols(seed, level, noise_index, nsites)].reshape(-1)


def z4_block(seed, level, first_index, count, nsites):
    """Noise vectors first_index .. first_index+count-1 as an n x count block."""
    cols = [z4_noise(seed, level, first_index + j, nsites) for j in range(count)]
    return np.stack(cols, axis=1)
