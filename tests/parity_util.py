"""Shared helpers of the GPU parity tests (relative L2 per band, runners)."""

import numpy as np

from oracle import run as oracle_run
from paper_2601_06340_gb300 import binding

# Tolerances (relative L2 per band over the final fields and every record).
TOL_FP64 = 1e-10
TOL_FP32 = 2e-4


def band_errors(got_psi, ref_psi, got_rec=None, ref_rec=None):
    """max over rows of the per-band relative L2 error, fields and records
    together; a band whose reference norm is below 1e-12 of the other
    band's is skipped (it carries no signal)."""
    worst = [0.0, 0.0]
    for r in range(ref_psi.shape[0]):
        norms = [0.0, 0.0]
        errs = [0.0, 0.0]
        for b in range(2):
            g = [np.asarray(got_psi[r, b], np.complex128).ravel()]
            f = [np.asarray(ref_psi[r, b]).ravel()]
            if ref_rec is not None and ref_rec.shape[1] > 0:
                g.append(np.asarray(got_rec[r, :, b], np.complex128).ravel())
                f.append(np.asarray(ref_rec[r, :, b]).ravel())
            g = np.concatenate(g)
            f = np.concatenate(f)
            norms[b] = np.linalg.norm(f)
            errs[b] = np.linalg.norm(g - f)
        for b in range(2):
            if norms[b] < 1e-12 * norms[1 - b]:
                continue
            worst[b] = max(worst[b], errs[b] / norms[b])
    return worst


def run_gpu(wl, precision, n_begin=0, n_end=None, psi_in=None):
    with binding.Plan(wl, precision) as plan:
        out = plan.propagate(psi_in, n_begin, n_end)
    return out


def run_ref(wl, **kw):
    return oracle_run.run_workload(wl, **kw)


_POOL = None


def oracle_pool():
    """A process pool for oracle marches, started with 'spawn' (never forked
    from a process that holds a CUDA context).  The oracle is single-threaded
    numpy, so independent marches run side by side on the host cores while
    the GPU works."""
    global _POOL
    if _POOL is None:
        import concurrent.futures
        import multiprocessing
        import os
        workers = max(1, min(8, (os.cpu_count() or 2) - 1))
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(var, "1")    # one core per oracle worker
        _POOL = concurrent.futures.ProcessPoolExecutor(
            workers, mp_context=multiprocessing.get_context("spawn"))
    return _POOL


def submit_ref(wl, **kw):
    """The oracle march of ``wl`` in the pool (a future of its MarchResult)."""
    return oracle_pool().submit(oracle_run.run_workload, wl, **kw)
