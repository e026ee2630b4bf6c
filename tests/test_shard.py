"""Noise sharding across ranks (paper_2306_09559_gb300.shard): the partition
of noise indices, the statistics, and a two-rank gloo run on the CPU whose
gathered samples and statistics equal a single process's bit for bit."""

import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_2306_09559_gb300 import shard

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_partition_tiles_the_indices(world):
    for n in list(range(0, 20)) + [511, 512, 1000]:
        parts = [shard.partition(n, world, r) for r in range(world)]
        nxt = 0
        for first, cnt in parts:
            assert first == nxt and cnt >= 0
            nxt += cnt
        assert nxt == n
        counts = [c for _, c in parts]
        assert max(counts) - min(counts) <= 1


def test_partition_rejects_bad_arguments():
    for args in [(10, 0, 0), (10, 2, 2), (10, 2, -1), (-1, 2, 0)]:
        with pytest.raises(ValueError):
            shard.partition(*args)


def test_level_statistics():
    rng = np.random.default_rng(3)
    s = rng.normal(size=(3, 57)) + 1j * rng.normal(size=(3, 57))
    mean, var = shard.level_statistics(s)
    assert np.allclose(mean, s.mean(axis=1), rtol=1e-14, atol=0)
    assert np.allclose(var, np.var(s.real, axis=1, ddof=1), rtol=1e-12, atol=0)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("nsamples", [9, 2])
def test_two_gloo_ranks_equal_one_process(tmp_path, nsamples):
    pytest.importorskip("torch")
    out = str(tmp_path / "gathered.npz")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, os.path.join(HERE, "shard_worker.py"), out, str(nsamples)],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    logs = []
    for p in procs:
        try:
            logs.append(p.communicate(timeout=300)[0])
        except subprocess.TimeoutExpired:
            p.kill()
            raise
    assert all(p.returncode == 0 for p in procs), "\n".join(logs)
    got = np.load(out)

    # the same computation in one process, one noise index at a time
    sys.path.insert(0, HERE)
    from oracle import krylov as K
    from oracle import mpmc as M
    from oracle.lattice import WilsonOperator
    from paper_2306_09559_gb300 import synth
    U = synth.gauge_field((2, 2, 2, 2), "haar", seed=4)
    op = WilsonOperator(U, 0.11)
    p_hi, p_lo = K.gmres_polynomials(op, synth.random_unit_vector(op.n, 2), [7, 3])
    polys = [{"kind": "single", "roots": p_hi}, {"kind": "single", "roots": p_lo}]
    ref = np.zeros((2, nsamples), dtype=np.complex128)
    for j in range(nsamples):
        for level in range(2):
            ref[level, j] = M.level_sample_parts(op, polys, level, 91, 1, None, first=j)[0][0]
    mean, var = shard.level_statistics(ref)
    assert np.array_equal(got["samples"], ref)
    assert np.array_equal(got["mean"], mean)
    assert np.array_equal(got["var"], var, equal_nan=True)
