"""The multi-rank host path on two gloo ranks (no GPU).

Rows of a batch are independent, so a batch split over ranks with
``replicas.shard`` and marched separately must reassemble, on rank 0, into
exactly the unsplit result; timing reductions take the maximum over ranks.
The march here is the oracle's (it stands in for one GPU's work).
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from paper_2601_06340_gb300 import inputs, replicas  # noqa: E402


def test_shard_partitions_rows():
    for n in (0, 1, 5, 6, 7, 256, 257):
        for world in (1, 2, 3, 4, 8):
            spans = [replicas.shard(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (b0, e0), (b1, e1) in zip(spans, spans[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _small_batch():
    return inputs.pulse_batched(nx=64, nz=30, n_energy=5, dx_um=0.4, record_every=0)


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    from oracle import run as orun
    rk = replicas.Ranks(backend="gloo")
    try:
        assert (rk.rank, rk.world) == (rank, world)
        rk.barrier()
        assert rk.max(1.5 + rank) == 1.5 + world - 1
        assert rk.sum(1.0) == float(world)
        wl = _small_batch()
        b, e = replicas.shard(wl.batch, rank, world)
        part = orun.run_workload(wl, rows=list(range(b, e)))
        psi = rk.gather_rows(part.psi, wl.batch)
        pw = rk.gather_rows(part.powers, wl.batch)
        if rank == 0:
            np.save(os.path.join(out_dir, "psi.npy"), psi)
            np.save(os.path.join(out_dir, "pw.npy"), pw)
        else:
            assert psi is None and pw is None
        rk.barrier()
    finally:
        rk.close()


def test_two_gloo_ranks_split_batch_equals_whole(tmp_path):
    from oracle import run as orun
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    wl = _small_batch()
    whole = orun.run_workload(wl)
    psi = np.load(tmp_path / "psi.npy")
    pw = np.load(tmp_path / "pw.npy")
    assert psi.shape == whole.psi.shape and pw.shape == whole.powers.shape
    assert np.array_equal(psi, whole.psi)
    assert np.array_equal(pw, whole.powers)
