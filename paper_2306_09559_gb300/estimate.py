"""Sequential multilevel estimate and sample allocation (Sec. 5, step 3; Eq. (3)).

Sequential stopping rule: the K Monte Carlos of the estimate run one after
another; the k-th (k = 0 .. K-1) stops at the first check point where its
standard error is at most sqrt((eps^2 - currerr^2) / (K - k)), currerr^2 being
the sum of the squared standard errors of the Monte Carlos before it (so the
total standard error sqrt(sum SE^2) ends at or below eps).  Check points
follow the paper: the first Monte Carlo from two noises on, the second from
three and every three, the later ones from six and every three.

Samples are drawn from the library in chunks (one GPU launch sequence per
chunk); since a sample depends only on its noise index, drawing ahead and
then finding the first check point that meets the tolerance stops exactly
where checking after every group of noises would.
"""

import math

import numpy as np

START = (2, 3, 6)     # first check point of the 1st, 2nd, 3rd and later Monte Carlos
STEP = (1, 3, 3)      # distance between check points


def schedule(k):
    i = min(k, len(START) - 1)
    return START[i], STEP[i]


def standard_error(re, n):
    """Standard error of the mean of the first n real parts (n - 1 in the variance)."""
    x = np.asarray(re[:n], dtype=np.float64)
    return math.sqrt(np.var(x, ddof=1) / n) if n > 1 else math.inf


def stop_point(re, tol, start, step):
    """First n in start, start+step, ... (n <= len(re)) with SE(n) <= tol, or None."""
    n = start
    while n <= len(re):
        if standard_error(re, n) <= tol:
            return n
        n += step
    return None


def sequential_estimate(sampler, levels, eps, chunk=64, nmax=1 << 15):
    """sampler(level, first, count) -> (complex samples, exact correction of the level).

    Returns {"levels": [{"estimate", "se", "n", "tol"}], "total", "err"}.
    """
    out, currerr2 = [], 0.0
    K = len(levels)
    for k, level in enumerate(levels):
        tol = math.sqrt(max(eps * eps - currerr2, 0.0) / (K - k))
        start, step = schedule(k)
        samples = np.zeros(0, dtype=np.complex128)
        corr = 0j
        n = None
        while n is None and samples.size < nmax:
            want = max(start, samples.size + chunk)
            if samples.size >= 2:
                # draw up to the predicted stopping size (rounded up to the check grid)
                se = standard_error(samples.real, samples.size)
                need = int(math.ceil(samples.size * (se / tol) ** 2)) if tol > 0 else nmax
                want = max(want, min(nmax, need + step))
            want = min(want, nmax)
            s, corr = sampler(level, samples.size, want - samples.size)
            samples = np.concatenate([samples, np.asarray(s, dtype=np.complex128)])
            n = stop_point(samples.real, tol, start, step)
        if n is None:
            n = samples.size
        se = standard_error(samples.real, n)
        currerr2 += se * se
        out.append({"level": level, "estimate": complex(np.mean(samples[:n]) + corr), "se": se, "n": int(n),
                    "tol": tol})
    return {"levels": out, "total": sum(x["estimate"] for x in out), "err": math.sqrt(currerr2)}


def library_sampler(h, seed):
    """Sampler over a handle: the level's samples and its exact deflation correction."""
    def sample(level, first, count):
        mean, _, s = h.mpmc_trace_level(level, seed, count, first)
        return s, mean - np.mean(s)
    return sample


def full_estimate(h_inv, h_lev, eps, seed, pin, colours, ncolours, *, h_probe=None, chunk=16, rtol=1e-10, m=40,
                  maxcycles=50, nmax=1 << 15):
    """The whole multipolynomial estimate of Tr A^{-1} (Sec. 5, step 3 (a) - (e); Eq. (2)):

        Tr A^{-1} = Tr(A^{-1} - p_1) + Tr(p_1 - p_2) + Tr(p_2 - p_3) + Tr(p_3).

    The handles hold the polynomials p_1 = q_0, p_2 = q_1, p_3 = q_2 (and p_in,
    a single polynomial, at index `pin` of h_inv).  The three Monte Carlos run one
    after another with the sequential rule: Tr(A^{-1} - p_1) on the FP64 handle
    h_inv (deflated PP-GMRES solves, mpmc_trace_inverse) to eps / sqrt(3) with
    checks from two noises; the deflated difference levels on h_lev with the
    checks 3, 6, ... and 6, 9, ...; then Tr(p_3) by probing with the given
    colouring (exact when it is a distance-d colouring, d >= degree of p_3).
    Returns {"levels": [...], "probing", "total", "err"}: total = the sum of the
    three Monte Carlo estimates and the probing trace, err = their combined
    standard error (currerr of step 3e).  nmax caps the noise vectors of each
    Monte Carlo (a level that has not met its tolerance by then stops there)."""
    def sample(level, first, count):
        if level == "inverse":
            mean, _, s = h_inv.mpmc_trace_inverse(0, seed, count, first, pin=pin, rtol=rtol, m=m,
                                                  maxcycles=maxcycles)
        else:
            mean, _, s = h_lev.mpmc_trace_level(level, seed, count, first)
        return s, mean - np.mean(s)
    nlev = h_lev.nlevels
    out = sequential_estimate(sample, ["inverse"] + list(range(nlev - 1)), eps, chunk=chunk, nmax=nmax)
    probing = (h_probe or h_lev).mpmc_trace_probing_colours(nlev - 1, colours, ncolours)
    out["probing"] = probing
    out["total"] = out["total"] + probing
    return out


def allocation(variances, costs, eps):
    """Samples per level minimising the cost for total standard error eps (Eq. (3)):
    N_l = eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k); returns (N_l rounded up, cost)."""
    v = np.asarray(variances, dtype=np.float64)
    c = np.asarray(costs, dtype=np.float64)
    s = float(np.sum(np.sqrt(v * c)))
    n = np.ceil(np.sqrt(v / c) * s / eps ** 2).astype(np.int64)
    return n, s * s / eps ** 2
