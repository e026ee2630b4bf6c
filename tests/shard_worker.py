"""One rank of the CPU (gloo) sharding test: computes its share of level
samples with the oracle, one noise index at a time, gathers on rank 0 and
writes the gathered samples and statistics there.  Run as a process with
RANK, WORLD_SIZE, MASTER_ADDR, MASTER_PORT set."""

import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(out_path, nsamples):
    import torch.distributed as dist

    from oracle import krylov as K
    from oracle import mpmc as M
    from oracle.lattice import WilsonOperator
    from paper_2306_09559_gb300 import shard, synth

    dist.init_process_group("gloo")
    U = synth.gauge_field((2, 2, 2, 2), "haar", seed=4)
    op = WilsonOperator(U, 0.11)
    p_hi, p_lo = K.gmres_polynomials(op, synth.random_unit_vector(op.n, 2), [7, 3])
    polys = [{"kind": "single", "roots": p_hi}, {"kind": "single", "roots": p_lo}]

    def compute(first, count):
        out = np.zeros((2, count), dtype=np.complex128)
        for i in range(count):
            for level in range(2):
                out[level, i] = M.level_sample_parts(op, polys, level, 91, 1, None, first=first + i)[0][0]
        return out

    res = shard.sharded_trace(compute, nsamples)
    if dist.get_rank() == 0:
        samples, mean, var = res
        np.savez(out_path, samples=samples, mean=mean, var=var)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]))
