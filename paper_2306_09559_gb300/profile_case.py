"""Stand-alone driver of the fused stencil step for timing and ncu captures.

One composite level p_in(A) p_out(A p_in(A)) and one single polynomial p_1(A) (Sec. 3 and
Sec. 4 of the paper, roots from GMRES runs on the lattice itself) are set on a handle of
the chosen precision; `--reps` traces of level 0 on `--nb` Z4 noise columns then run
through the public API with the stencil options given, and the per-launch time and
algorithmic bandwidth of the stencil kernels (the handle's own profiling counters) are
printed.  Example, the 24^3 x 8 FP32 case of the 24^3 x 32 workload's dominant kernel:

    python -m paper_2306_09559_gb300.profile_case --dims 24 24 24 8 --nb 32 --precision fp32

Under ncu, capture a few launches of one kernel class, e.g.
`ncu --clock-control none -k regex:k_fsweep -c 3 ... python -m ...profile_case --reps 1`.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import krylov_setup, synth
from . import mpmc as G


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--dims", type=int, nargs=4, default=[24, 24, 24, 8], metavar=("LX", "LY", "LZ", "LT"))
    ap.add_argument("--nb", type=int, default=32, help="noise columns per launch")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16s", "fp64"])
    ap.add_argument("--fast", type=int, default=7, help="MPMC_OPT_FAST_STENCIL step-class mask")
    ap.add_argument("--sweep", type=int, default=55,
                    help="MPMC_OPT_SWEEP_STENCIL mask (bit 16: links staged, bit 32: warp-per-site form)")
    ap.add_argument("--segment", type=int, default=0, help="MPMC_OPT_SWEEP_SEGMENT (0: whole t extent)")
    ap.add_argument("--order", type=int, default=1, help="MPMC_OPT_SWEEP_ORDER")
    ap.add_argument("--launch", type=int, nargs=2, default=[1, 64], metavar=("R", "BX"))
    ap.add_argument("--m-out", type=int, default=5, help="outer degree of the composite")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--kappa", type=float, default=0.124)
    args = ap.parse_args(argv)

    G.lib()
    dims = tuple(args.dims)
    nsite = int(np.prod(dims))
    U = synth.gauge_field(dims, "near_identity", 3, 0.2)
    h64 = G.Handle(U, args.kappa, G.FP64)
    setup = krylov_setup.Setup(h64)
    v0 = synth.random_unit_vector(12 * nsite, 7)
    inner, single = setup.single_roots(v0, [19, 16])
    outer, _ = setup.pp_roots(inner, v0, m_out=args.m_out)
    prec = {"fp32": G.FP32, "bf16s": G.BF16S, "fp64": G.FP64}[args.precision]
    h = G.Handle(U, args.kappa, prec)
    stream = torch.cuda.Stream()
    h.mpmc_set_stream(stream)
    h.mpmc_set_poly(0, G.COMPOSITE, inner, outer, leja=True)
    h.mpmc_set_poly(1, G.SINGLE, single, leja=True)
    h.mpmc_set_block(args.nb)
    for opt, val in ((G.OPT_FAST_STENCIL, args.fast), (G.OPT_SWEEP_STENCIL, args.sweep),
                     (G.OPT_SWEEP_SEGMENT, args.segment), (G.OPT_SWEEP_ORDER, args.order)):
        h.mpmc_set_option(opt, val)
    h.mpmc_set_launch(args.launch[0], args.launch[1], 1)
    h.mpmc_trace_levels(1, args.nb, 0, want_samples=False)     # warm-up (first-use allocations)
    torch.cuda.synchronize()
    h.mpmc_profile(True)
    t0 = time.perf_counter()
    for _ in range(args.reps):
        h.mpmc_trace_levels(1, args.nb, 0, want_samples=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms, n, nbytes = h.mpmc_profile_read(G.PROF_STENCIL)
    out = {"dims": list(dims), "nb": args.nb, "precision": args.precision, "fast": args.fast,
           "sweep": args.sweep, "segment": args.segment, "order": args.order, "launch": args.launch,
           "stencil_launches": n, "avg_launch_ms": ms / max(n, 1), "bytes_per_launch": nbytes / max(n, 1),
           "algorithmic_gbs": nbytes / (ms / 1e3) / 1e9 if ms > 0 else None, "wall_s": wall}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
