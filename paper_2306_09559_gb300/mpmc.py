"""Thin ctypes binding of libmpmc.so (the C ABI of include/mpmc.h).

Only argument marshalling happens here: numpy arrays become host pointers,
torch CUDA tensors become device pointers, and every computation runs in
the library's CUDA kernels.  If the library is missing, :func:`lib` raises;
there is no fallback path.

Vector blocks use the library layout: complex128 arrays of shape
(V, 4, 3, nrhs) (site, spin, colour, column), i.e. an n x nrhs matrix in
unknown order with the column index fastest.
"""

import ctypes
import os

import numpy as np

from . import build as _build

MPMC_OK, MPMC_EINVAL, MPMC_ENOMEM, MPMC_ENOTSUP, MPMC_ETIMEOUT, MPMC_ENONFINITE, MPMC_ECUDA, MPMC_ESTATE = range(8)
FP64, FP32, BF16S = 0, 1, 2
SINGLE, COMPOSITE, DEFLATED_COMPOSITE = 0, 1, 2
MAX_POLYS = 8
POLY_LEJA, POLY_FP32_COEFS = 1, 2
MAX_BLOCK = 1024

_LIB = None

_SIGS = {
    "mpmc_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    "mpmc_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "mpmc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mpmc_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "mpmc_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mpmc_set_block": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mpmc_set_poly": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "mpmc_get_roots": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "mpmc_set_deflation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int]),
    "mpmc_apply_op": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "mpmc_apply_poly": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_int]),
    "mpmc_trace_levels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mpmc_level_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_longlong)]),
    "mpmc_noise": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_int]),
    "mpmc_arnoldi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "mpmc_combine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_void_p]),
    "mpmc_launch_count": (ctypes.c_longlong, [ctypes.c_void_p]),
    "mpmc_set_links": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mpmc_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mpmc_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]),
    "mpmc_trace_poly_noalloc": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_double,
                                               ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_int, ctypes.c_void_p]),
    "mpmc_set_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mpmc_get_launch": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 4),
    "mpmc_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "mpmc_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "mpmc_get_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mpmc_set_deflation_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_int]),
    "mpmc_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]),
    "mpmc_batch_trace_levels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "mpmc_batch_launch_count": (ctypes.c_longlong, [ctypes.c_void_p]),
    "mpmc_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "mpmc_trace_probing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "mpmc_colouring": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_int)]),
    "mpmc_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "mpmc_trace_probing_colours": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.c_void_p]),
    "mpmc_trace_level": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mpmc_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_longlong)]),
    "mpmc_trace_inverse": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "mpmc_deflation_norms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mpmc_vector_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "mpmc_project": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "mpmc_deflation_dots": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_void_p]),
}

OPT_TENSOR_CORE_DEFLATION = 1
OPT_SWEEP_STENCIL = 2
OPT_SWEEP_SEGMENT = 3
OPT_FAST_STENCIL = 4
OPT_FAST_SITES = 5
OPT_WAIT_LIMIT = 6
OPT_TEST_SKIP_COPY = 7
OPT_SWEEP_ORDER = 8

PROF_STENCIL, PROF_DEFLATION, PROF_OTHER = 0, 1, 2
PROF_K_FSWEEP, PROF_K_FAST, PROF_K_SITE, PROF_K_SWEEP = 3, 4, 5, 6
PROF_KERNEL_NAMES = {PROF_K_FSWEEP: "k_fsweep", PROF_K_FAST: "k_fast", PROF_K_SITE: "k_step/k_outer",
                     PROF_K_SWEEP: "k_sweep"}
NOALLOC_SCRATCH_BYTES = 32 << 20


def exported_symbols():
    """Names every build of the library must export (the declarations of include/mpmc.h)."""
    return sorted(_SIGS)


def lib(path=None):
    """The loaded library (loaded once).  Raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2306_09559_gb300.build.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


class MpmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def _ptr(a):
    """Host pointer of a C-contiguous numpy array, or device pointer of a torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _is_device(a):
    return hasattr(a, "is_cuda") and a.is_cuda


class Handle:
    """One lattice: links, kappa, precision (mpmc_create ... mpmc_destroy)."""

    def __init__(self, links, kappa, precision=FP64, bc_t=1):
        L = lib()
        links = _c128(links)
        lt, lz, ly, lx = links.shape[1:5]
        self.dims = (lx, ly, lz, lt)
        self.V = lx * ly * lz * lt
        self.n = 12 * self.V
        self.k = 0
        self.precision = precision
        self.kappa = kappa
        dims = (ctypes.c_int * 4)(lx, ly, lz, lt)
        h = ctypes.c_void_p()
        rc = L.mpmc_create(ctypes.byref(h), dims, _ptr(links), float(kappa), int(precision), int(bc_t))
        if rc != MPMC_OK:
            raise MpmcError(rc, "mpmc_create: " + L.mpmc_strerror(rc).decode())
        self._h = h
        self._L = L
        self._set = set()

    @property
    def nlevels(self):
        """Levels of mpmc_trace_levels: polynomials 0..L-1 set without a gap."""
        L = 0
        while L in self._set:
            L += 1
        return L

    def _check(self, rc, what):
        if rc != MPMC_OK:
            msg = self._L.mpmc_last_error(self._h).decode()
            raise MpmcError(rc, f"{what}: {self._L.mpmc_strerror(rc).decode()}: {msg}")

    def close(self):
        if getattr(self, "_h", None):
            self._L.mpmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ----------------------------------------------------------------- config
    def mpmc_set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self._L.mpmc_set_stream(self._h, ctypes.c_void_p(raw) if raw else None), "mpmc_set_stream")

    def mpmc_set_block(self, nb):
        self._check(self._L.mpmc_set_block(self._h, int(nb)), "mpmc_set_block")

    def mpmc_set_poly(self, index, kind, roots, outer=None, leja=True, fp32_coefs=False):
        """leja: Leja-order the roots; fp32_coefs: round every 1/theta to FP32 (MPMC_POLY_FP32_COEFS),
        so that handles of every precision apply the same polynomial."""
        r = _c128(roots)
        o = _c128(outer) if outer is not None else None
        flags = (POLY_LEJA if leja else 0) | (POLY_FP32_COEFS if fp32_coefs else 0)
        rc = self._L.mpmc_set_poly(self._h, int(index), int(kind), _ptr(r), r.size, _ptr(o),
                                   0 if o is None else o.size, flags)
        self._check(rc, "mpmc_set_poly")
        self._set.add(int(index))

    def mpmc_get_roots(self, index, nroots, nouter=0):
        r = np.zeros(nroots, dtype=np.complex128)
        o = np.zeros(max(nouter, 1), dtype=np.complex128)
        self._check(self._L.mpmc_get_roots(self._h, int(index), _ptr(r), _ptr(o)), "mpmc_get_roots")
        return (r, o[:nouter]) if nouter else r

    def mpmc_set_deflation(self, Z, lam, pair, rows=False):
        """Z: n x k complex (column i = z_i), lam: k, pair: k ints.

        rows=True: Z is already k x n (vector i contiguous, the library
        layout), e.g. a pinned torch tensor; it is passed without a copy.
        """
        if rows:
            k = Z.shape[0]
            Zt = Z if hasattr(Z, "data_ptr") else _c128(Z)
        else:
            Z = np.asarray(Z)
            k = 0 if Z.size == 0 else Z.shape[1]
            Zt = _c128(Z.T) if k else None
        lam = _c128(lam) if k else None
        pr = np.ascontiguousarray(pair, dtype=np.int32) if k else None
        self._check(self._L.mpmc_set_deflation(self._h, _ptr(Zt), _ptr(lam), _ptr(pr), k), "mpmc_set_deflation")
        self.k = k

    # ----------------------------------------------------------------- compute
    def _block_call(self, fn, what, X, *pre):
        if _is_device(X):
            import torch
            nrhs = X.shape[-1] if X.dim() > 1 else 1
            Y = torch.empty_like(X)
            self._check(fn(self._h, *pre, _ptr(X), _ptr(Y), nrhs, 1), what)
            return Y
        X = _c128(X)
        nrhs = X.shape[-1] if X.ndim > 1 else 1
        Y = np.empty_like(X)
        self._check(fn(self._h, *pre, _ptr(X), _ptr(Y), nrhs, 0), what)
        return Y

    def mpmc_apply_op(self, X):
        """A X for X of shape (n, nrhs) (or (n,)), host numpy or device torch complex128."""
        return self._block_call(self._L.mpmc_apply_op, "mpmc_apply_op", X)

    def mpmc_apply_poly(self, index, B):
        return self._block_call(self._L.mpmc_apply_poly, "mpmc_apply_poly", B, int(index))

    def mpmc_trace_levels(self, seed, nsamples, first=0, want_samples=True):
        L = self.nlevels
        mean = np.zeros(L, dtype=np.complex128)
        var = np.zeros(L, dtype=np.float64)
        samples = np.zeros((L, nsamples), dtype=np.complex128) if want_samples else None
        rc = self._L.mpmc_trace_levels(self._h, ctypes.c_uint64(seed), int(nsamples), int(first), _ptr(mean),
                                       _ptr(var), _ptr(samples))
        self._check(rc, "mpmc_trace_levels")
        return mean, var, samples

    def mpmc_level_info(self, level):
        corr = np.zeros(1, dtype=np.complex128)
        mv = ctypes.c_longlong()
        self._check(self._L.mpmc_level_info(self._h, int(level), _ptr(corr), ctypes.byref(mv)), "mpmc_level_info")
        return corr[0], mv.value

    def mpmc_noise(self, seed, level, first, nrhs):
        B = np.zeros((self.n, nrhs), dtype=np.complex128)
        self._check(self._L.mpmc_noise(self._h, ctypes.c_uint64(seed), int(level), int(first), int(nrhs), _ptr(B), 0),
                    "mpmc_noise")
        return B

    def mpmc_arnoldi(self, op_poly, v0, m, basis=None):
        """Hbar ((m+1) x m) and completed steps; basis: optional torch complex128 (m+1, n) device tensor."""
        v0 = _c128(v0)
        hbar = np.zeros((m + 1, m), dtype=np.complex128)
        steps = ctypes.c_int()
        rc = self._L.mpmc_arnoldi(self._h, int(op_poly), _ptr(v0), int(m), _ptr(hbar), _ptr(basis),
                                  ctypes.byref(steps))
        self._check(rc, "mpmc_arnoldi")
        return hbar, steps.value

    def mpmc_combine(self, basis, m, Y, Z):
        """Z (device, (k, n)) = sum_j basis[j] Y[j, :] for j < m."""
        Y = _c128(Y)
        self._check(self._L.mpmc_combine(self._h, _ptr(basis), int(m), _ptr(Y), Y.shape[1], _ptr(Z)), "mpmc_combine")

    def mpmc_launch_count(self):
        return int(self._L.mpmc_launch_count(self._h))

    def mpmc_set_launch(self, R=0, bx=0, sl=0):
        self._check(self._L.mpmc_set_launch(self._h, int(R), int(bx), int(sl)), "mpmc_set_launch")

    def mpmc_get_launch(self):
        v = [ctypes.c_int() for _ in range(4)]
        self._check(self._L.mpmc_get_launch(self._h, *[ctypes.byref(x) for x in v]), "mpmc_get_launch")
        return dict(zip(("nb", "R", "bx", "sl"), (x.value for x in v)))

    def mpmc_autotune(self, max_nb, steps=6):
        self._check(self._L.mpmc_autotune(self._h, int(max_nb), int(steps)), "mpmc_autotune")
        return self.mpmc_get_launch()

    def mpmc_set_option(self, option, value):
        self._check(self._L.mpmc_set_option(self._h, int(option), int(value)), "mpmc_set_option")

    def mpmc_get_option(self, option):
        v = ctypes.c_int()
        self._check(self._L.mpmc_get_option(self._h, int(option), ctypes.byref(v)), "mpmc_get_option")
        return v.value

    def mpmc_trace_probing(self, index, m):
        """Probing estimate of Tr p(A) (period-m colouring; exact below degree m)."""
        t = np.zeros(1, dtype=np.complex128)
        self._check(self._L.mpmc_trace_probing(self._h, int(index), int(m), _ptr(t)), "mpmc_trace_probing")
        return complex(t[0])

    def mpmc_trace_probing_colours(self, index, colours, ncolours):
        """Probing estimate of Tr p(A) with a site colouring (exact when same-coloured
        sites are more hops apart than the degree of p)."""
        c = np.ascontiguousarray(colours, dtype=np.int32)
        if c.size != self.V:
            raise ValueError(f"colours must have {self.V} entries")
        t = np.zeros(1, dtype=np.complex128)
        self._check(self._L.mpmc_trace_probing_colours(self._h, int(index), _ptr(c), int(ncolours), _ptr(t)),
                    "mpmc_trace_probing_colours")
        return complex(t[0])

    def mpmc_trace_level(self, level, seed, nsamples, first=0):
        """(mean with exact correction, variance of Re, samples) of one level."""
        mean = np.zeros(1, dtype=np.complex128)
        var = np.zeros(1, dtype=np.float64)
        samples = np.zeros(nsamples, dtype=np.complex128)
        rc = self._L.mpmc_trace_level(self._h, int(level), ctypes.c_uint64(seed), int(nsamples), int(first),
                                      _ptr(mean), _ptr(var), _ptr(samples))
        self._check(rc, "mpmc_trace_level")
        return complex(mean[0]), float(var[0]), samples

    def mpmc_solve(self, B, pin=-1, rtol=1e-10, m=40, maxcycles=50):
        """x = A^{-1} B (host numpy (n, nrhs) or (n,)); returns (X, relres, matvecs)."""
        B = _c128(B)
        nrhs = B.shape[-1] if B.ndim > 1 else 1
        X = np.empty_like(B)
        rr = np.zeros(nrhs)
        mv = ctypes.c_longlong()
        self._check(self._L.mpmc_solve(self._h, int(pin), _ptr(B), _ptr(X), nrhs, float(rtol), int(m), int(maxcycles),
                                       0, _ptr(rr), ctypes.byref(mv)), "mpmc_solve")
        return X, rr, mv.value

    def mpmc_trace_inverse(self, p1, seed, nsamples, first=0, pin=-1, rtol=1e-10, m=40, maxcycles=50):
        """(mean with exact correction, variance of Re, samples) of Tr(A^{-1} - p_1(A))."""
        mean = np.zeros(1, dtype=np.complex128)
        var = np.zeros(1)
        s = np.zeros(nsamples, dtype=np.complex128)
        self._check(self._L.mpmc_trace_inverse(self._h, int(p1), int(pin), ctypes.c_uint64(seed), int(nsamples),
                                               int(first), float(rtol), int(m), int(maxcycles), _ptr(mean), _ptr(var),
                                               _ptr(s)), "mpmc_trace_inverse")
        return complex(mean[0]), float(var[0]), s

    def mpmc_deflation_norms(self):
        """d_i = z_pair(i)^H gamma5 z_i of the stored deflation vectors (complex, length k)."""
        k = self.k
        d = np.zeros(k, dtype=np.complex128)
        self._check(self._L.mpmc_deflation_norms(self._h, _ptr(d)), "mpmc_deflation_norms")
        return d

    def mpmc_set_deflation_device(self, Zd, lam, pair):
        """Zd: CUDA complex128 tensor (k, n), row i = z_i."""
        lam = _c128(lam)
        pr = np.ascontiguousarray(pair, dtype=np.int32)
        self._check(self._L.mpmc_set_deflation_device(self._h, _ptr(Zd), _ptr(lam), _ptr(pr), int(Zd.shape[0])),
                    "mpmc_set_deflation_device")
        self.k = int(Zd.shape[0])

    def mpmc_vector_stats(self, Zd):
        """Zd: CUDA complex128 tensor (k, n); returns (k, 4) float64 stats."""
        k = int(Zd.shape[0])
        out = np.zeros((k, 4), dtype=np.float64)
        self._check(self._L.mpmc_vector_stats(self._h, _ptr(Zd), k, _ptr(out)), "mpmc_vector_stats")
        return out

    def mpmc_project(self, B):
        return self._block_call(self._L.mpmc_project, "mpmc_project", B)

    def mpmc_deflation_dots(self, seed, level, first, nrhs, k):
        G1 = np.zeros((k, nrhs), dtype=np.complex128)
        G2 = np.zeros((k, nrhs), dtype=np.complex128)
        self._check(self._L.mpmc_deflation_dots(self._h, ctypes.c_uint64(seed), int(level), int(first), int(nrhs),
                                                _ptr(G1), _ptr(G2)), "mpmc_deflation_dots")
        return G1, G2

    def mpmc_set_links(self, links):
        """links: (4, Lt, Lz, Ly, Lx, 3, 3) complex128 numpy array or a pinned torch tensor of the same bytes."""
        ptr = _ptr(links) if hasattr(links, "data_ptr") else _ptr(_c128(links))
        self._check(self._L.mpmc_set_links(self._h, ptr), "mpmc_set_links")

    def mpmc_profile(self, enable):
        self._check(self._L.mpmc_profile(self._h, 1 if enable else 0), "mpmc_profile")

    def mpmc_profile_read(self, cls):
        ms, n, b = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        self._check(self._L.mpmc_profile_read(self._h, int(cls), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)),
                    "mpmc_profile_read")
        return ms.value, n.value, b.value


class Batch:
    """Independent handles whose multilevel traces run as one captured CUDA graph.

    The handles are borrowed: keep them alive (and destroy them) after the
    batch.  Each needs its own stream (the handles' default).
    """

    def __init__(self, handles):
        self._L = lib()
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h._h for h in self.handles])
        b = ctypes.c_void_p()
        rc = self._L.mpmc_batch_create(ctypes.byref(b), len(self.handles), ctypes.cast(arr, ctypes.c_void_p))
        if rc:
            raise MpmcError(rc, "mpmc_batch_create")
        self._b = b

    def mpmc_batch_trace_levels(self, seed, nsamples, first=0):
        """(mean, var) arrays of shape (n_handles, MAX_POLYS); entries past a handle's levels are unused."""
        n = len(self.handles)
        mean = np.zeros((n, MAX_POLYS), dtype=np.complex128)
        var = np.zeros((n, MAX_POLYS), dtype=np.float64)
        rc = self._L.mpmc_batch_trace_levels(self._b, ctypes.c_uint64(seed), int(nsamples), int(first), _ptr(mean),
                                             _ptr(var))
        if rc:
            msgs = [self._L.mpmc_last_error(h._h).decode() for h in self.handles]
            raise MpmcError(rc, "mpmc_batch_trace_levels: " + "; ".join(m for m in msgs if m))
        return mean, var

    def mpmc_batch_launch_count(self):
        return int(self._L.mpmc_batch_launch_count(self._b))

    def close(self):
        if self._b is not None:
            self._L.mpmc_batch_destroy(self._b)
            self._b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def mpmc_fma_peak(precision):
    """Measured FMA throughput (TFLOP/s) of the current device's CUDA cores in FP64 or FP32."""
    L = lib()
    v = ctypes.c_double()
    rc = L.mpmc_fma_peak(int(precision), ctypes.byref(v))
    if rc != MPMC_OK:
        raise MpmcError(rc, "mpmc_fma_peak: " + L.mpmc_strerror(rc).decode())
    return v.value


def mpmc_colouring(dims, distance):
    """(colours, ncolours): a distance-`distance` colouring of the periodic lattice
    dims = (Lx, Ly, Lz, Lt) from the library (host code, no GPU needed)."""
    L = lib()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    V = int(np.prod(dims))
    colours = np.zeros(V, dtype=np.int32)
    nc = ctypes.c_int()
    rc = L.mpmc_colouring(d, int(distance), _ptr(colours), ctypes.byref(nc))
    if rc != MPMC_OK:
        raise MpmcError(rc, "mpmc_colouring: " + L.mpmc_strerror(rc).decode())
    return colours, nc.value


def mpmc_trace_poly_noalloc(links, kappa, roots, seed, level, first, nsamples, out=None, bc_t=1, stream=None):
    """Samples b_j^H p(A) b_j without any device allocation inside the library.

    links: host complex128 array (4, Lt, Lz, Ly, Lx, 3, 3) or a CUDA tensor of
    the same layout; out: None (host result) or a CUDA complex128 tensor of
    nsamples entries (then links must be on the device too and the call is
    asynchronous on `stream`).  Returns the samples (host array or `out`).
    """
    L = lib()
    if len(links.shape) != 7 or tuple(links.shape[0:1]) + tuple(links.shape[5:]) != (4, 3, 3):
        raise ValueError("links must have shape (4, Lt, Lz, Ly, Lx, 3, 3)")
    lt, lz, ly, lx = (int(e) for e in links.shape[1:5])
    dims = (ctypes.c_int * 4)(lx, ly, lz, lt)
    r = _c128(roots)
    on_dev = 1 if out is not None else 0
    if on_dev:
        # the library reads links and writes out through raw device pointers: both must be
        # contiguous complex128 CUDA tensors of the stated sizes on one device
        for name, t in (("links", links), ("out", out)):
            if not _is_device(t):
                raise ValueError(f"with out= given, {name} must be a CUDA tensor")
            if str(t.dtype) != "torch.complex128" or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous complex128 tensor")
        if links.device != out.device:
            raise ValueError("links and out must be on the same device")
        if links.numel() != 36 * lx * ly * lz * lt:
            raise ValueError("links has the wrong number of entries")
        if out.numel() < nsamples:
            raise ValueError(f"out holds {out.numel()} entries, fewer than nsamples = {nsamples}")
        res = out
        lk = links
    else:
        if _is_device(links):
            raise ValueError("device links need a device result: pass out=")
        res = np.zeros(nsamples, dtype=np.complex128)
        lk = _c128(links)
    raw = getattr(stream, "cuda_stream", stream)
    rc = L.mpmc_trace_poly_noalloc(dims, _ptr(lk), float(kappa), int(bc_t), _ptr(r), r.size, ctypes.c_uint64(seed),
                                   int(level), int(first), int(nsamples), _ptr(res), on_dev,
                                   ctypes.c_void_p(raw) if raw else None)
    if rc != MPMC_OK:
        raise MpmcError(rc, "mpmc_trace_poly_noalloc: " + L.mpmc_strerror(rc).decode())
    return res
