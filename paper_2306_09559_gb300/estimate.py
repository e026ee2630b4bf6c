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


def precision_corrected_level(h_mix, h64, level, seed, nsamples, ncorr, first=0):
    """One level estimated in reduced precision with an FP64 correction level.

    The telescoping of Eq. (2) applied across precisions: E[s_64] = E[s_mix] +
    E[s_64 - s_mix].  The mixed-precision handle draws `nsamples` samples; the
    FP64 handle (same polynomials and deflation) draws the first `ncorr` of the
    same noise vectors, and the mean of the paired differences d = s_64 - s_mix
    is added.  The estimate is then unbiased with respect to the FP64 level
    whatever the rounding of the mixed path does; d is small, so few FP64
    samples suffice.  With m the mixed samples and d the differences,
    Var = Var(m)/N + Var(d)/n + 2 Cov(m, d)/N (the n pairs share their noise with
    the first n mixed samples).  Returns {"estimate", "se", "mixed", "correction",
    "var_mixed", "var_diff", "n", "ncorr"}."""
    if ncorr < 2:
        raise ValueError("the correction level needs at least two samples")
    mean_m, _, sm = h_mix.mpmc_trace_level(level, seed, nsamples, first)
    _, _, s64 = h64.mpmc_trace_level(level, seed, ncorr, first)
    corr_m = mean_m - np.mean(sm)                  # the level's exact deflation correction
    d = s64 - sm[:ncorr]
    m = sm.real
    var_m = float(np.var(m, ddof=1)) if nsamples > 1 else 0.0
    var_d = float(np.var(d.real, ddof=1))
    cov = float(np.cov(m[:ncorr], d.real, ddof=1)[0, 1])
    var = var_m / nsamples + var_d / ncorr + 2 * cov / nsamples
    est = complex(np.mean(sm) + corr_m + np.mean(d))
    return {"estimate": est, "se": math.sqrt(max(var, 0.0)), "mixed": complex(mean_m),
            "correction": complex(np.mean(d)), "var_mixed": var_m, "var_diff": var_d, "n": int(nsamples),
            "ncorr": int(ncorr)}


def correction_samples(var_mixed, var_diff, cost_mixed, cost_64, nsamples):
    """Paired FP64 samples for a correction level at the least total cost for the variance
    of `nsamples` mixed samples (the allocation of Eq. (3) for the two terms):
    n = N sqrt((V_d / C_64) / (V_m / C_m)), at least 2."""
    if var_mixed <= 0:
        return 2
    n = nsamples * math.sqrt((var_diff / cost_64) / (var_mixed / cost_mixed))
    return max(2, int(math.ceil(n)))


def allocation(variances, costs, eps):
    """Samples per level minimising the cost for total standard error eps (Eq. (3)):
    N_l = eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k); returns (N_l rounded up, cost)."""
    v = np.asarray(variances, dtype=np.float64)
    c = np.asarray(costs, dtype=np.float64)
    s = float(np.sum(np.sqrt(v * c)))
    n = np.ceil(np.sqrt(v / c) * s / eps ** 2).astype(np.int64)
    return n, s * s / eps ** 2


def choose_degree(h, index, candidates, roots_for, eps, seed, pilot=32, first=0):
    """The degree of polynomial `index` chosen by the cost model, Eq. (3) (the paper
    leaves the degrees to the user and names choosing them from the level
    variances and costs as future work, Sec. 7).

    For each candidate degree d the handle's polynomial `index` is set to the
    single polynomial roots_for(d); every level is sampled on `pilot` noise vectors
    (the pilot variances V_l) and priced with its matvecs per sample C_l
    (mpmc_level_info); the level set costs eps^-2 (sum_l sqrt(V_l C_l))^2 matvecs
    for total standard error eps.  The handle is left with the cheapest candidate.
    Returns (best degree, {degree: Eq. (3) cost})."""
    from . import mpmc as G
    costs = {}
    for d in candidates:
        h.mpmc_set_poly(index, G.SINGLE, roots_for(d), leja=True)
        _, var, _ = h.mpmc_trace_levels(seed, pilot, first, want_samples=False)
        C = [h.mpmc_level_info(level)[1] for level in range(h.nlevels)]
        costs[d] = allocation(var, C, eps)[1]
    best = min(costs, key=costs.get)
    h.mpmc_set_poly(index, G.SINGLE, roots_for(best), leja=True)
    return best, costs

