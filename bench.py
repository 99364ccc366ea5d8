"""Benchmark of the two-beam FFT-BPM z-march on GB300.

Default workload (the one the headline metric is quoted on): symmetric
Bragg, cylindrically bent crystal (R = 1 m), Nx = 4096, Nz = 8000, one
photon energy.  One benchmark "step" is one whole march of that solve
(8000 z-steps of forward FFT, propagator, inverse FFT and coupling for both
envelopes).  ``value`` is cell-updates/s of the fused FP32 path with inputs
resident in device memory; ``e2e`` is the same metric through the host
C-ABI call (pinned host buffers, copies inside the timed region).  The line
also carries the plain FP64 GPU path, both paths' relative L2 errors
against the FP64 oracle, single-solve latency percentiles, the batched
256-energy workload, the 256-angle rocking-curve scan, the serving run, the roofline of the
dominant kernel and the oracle's own throughput on the host cores.

``--impl reference`` times the FP64 oracle instead (bounded samples of the
same march on the host cores).  Multi-GPU runs (torchrun) are independent
replicas: every rank marches its own copy, there is no collective on the
data path.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BPM cell-updates/s, fused FP32 vs plain FP64 GPU at stated err; p50/p99 latency"
UNIT = "cell-updates/s"
WORKLOAD = ("bragg_bent: 2D symmetric Bragg, bent crystal R=1 m nu=0.28, 8 keV, "
            "theta_B=23.65 deg, 200 um slab, Nx=4096, Nz=8000, dx=0.2 um, dz=0.1 um, "
            "one energy, Gaussian 50 um FWHM")
FLOPS_PER_CELL = lambda n: 4 * 5 * math.log2(n)      # 4 FFTs x 5 N log2 N / N
# the single-solve march kernel by launch layout (bpm_launch_shape): name, SMs
MARCH_KERNELS = {
    2: ("fused4s_march_kernel (4-CTA cluster per solve: two half-band parts per band, "
        "8 points per thread)", 4),
    8: ("fused4e_march_kernel<11> (4-CTA cluster per solve: two half-band parts per band, "
        "16 points per thread)", 4),
    1: ("fused3_march_kernel<12> (2-CTA cluster per solve, one band per CTA)", 2),
    -1: ("fused3_march_kernel<12> (2-CTA cluster per solve, one band per CTA)", 2),
}

KERNEL_SOURCES = ["paper_2601_06340_gb300/csrc/radix.cuh",
                  "paper_2601_06340_gb300/csrc/fused4s_kernel.cuh",
                  "paper_2601_06340_gb300/csrc/fused_kernel.cuh",
                  "paper_2601_06340_gb300/csrc/fused2_kernel.cuh",
                  "paper_2601_06340_gb300/csrc/fused3_kernel.cuh",
                  "paper_2601_06340_gb300/csrc/fused4_kernel.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(name: str):
    """dram bytes per launch from a committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_hash():
        return None
    return float(m_bytes.group(1))


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def host_info():
    """Core count and CPU model of the host (for the CPU baselines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model,
            "machine": os.uname().machine}


def oracle_job(wl, kw, three_d=False):
    """One oracle march in a pool worker: (MarchResult, seconds)."""
    from oracle import run as orun
    t0 = time.perf_counter()
    res = orun.run_workload3d(wl, **kw) if three_d else orun.run_workload(wl, **kw)
    return res, time.perf_counter() - t0


def _warm_worker(_):
    import oracle.run  # noqa: F401  (imports done before a timed batch)
    return os.getpid()


def row_workload(wl, r: int):
    """Row r of a batched workload as a one-row workload (so that a pool
    task carries one row's input, not the whole batch's)."""
    import dataclasses
    return dataclasses.replace(wl, energies_ev=np.asarray(wl.energies_ev)[r:r + 1],
                               psi0=np.asarray(wl.psi0)[r:r + 1])


def make_oracle_pool(workers: int):
    """Process pool for oracle marches, started with 'spawn' (the oracle is
    single-threaded numpy; one worker per host core)."""
    import concurrent.futures
    import multiprocessing
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    pool = concurrent.futures.ProcessPoolExecutor(
        workers, mp_context=multiprocessing.get_context("spawn"))
    list(pool.map(_warm_worker, range(workers)))
    return pool


def cpu_baselines(pool, workers: int, head_steps: int, batch_steps: int):
    """The oracle, as it stands, on bounded samples: the headline solve on
    one core (its march is sequential in z) and the pulse batch on every
    host core in parallel over energies (one row per core)."""
    from oracle import run as orun
    from paper_2601_06340_gb300 import inputs
    info = host_info()
    wl = inputs.bragg_bent()
    t0 = time.perf_counter()
    orun.run_workload(wl, 0, head_steps, record_every=0)
    dt = time.perf_counter() - t0
    head = {"value": wl.nx * head_steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {head_steps} of the {wl.nz} z-steps of the bragg_bent march "
                      f"(Nx={wl.nx}), numpy float64, single thread", **info}
    wb = inputs.pulse_batched(nz=batch_steps)
    rows = list(range(0, wb.batch, max(1, wb.batch // workers)))[:workers]
    tasks = [row_workload(wb, r) for r in rows]
    t0 = time.perf_counter()
    futs = [pool.submit(oracle_job, w, dict(record_every=0)) for w in tasks]
    for f in futs:
        f.result()
    dt = time.perf_counter() - t0
    batch = {"value": len(rows) * wb.nx * batch_steps / dt, "unit": UNIT,
             "cores": workers, "kind": "oracle",
             "sample": f"{len(rows)} of the 256 energy rows of pulse_batched (Nx={wb.nx}), "
                       f"first {batch_steps} of 6000 z-steps each, one row per process, "
                       f"{workers} processes in parallel, numpy float64", **info}
    return head, batch


def rel_l2_bands(got, ref):
    out = []
    for b in range(2):
        den = np.linalg.norm(ref[:, b])
        out.append(float(np.linalg.norm(got[:, b] - ref[:, b]) / den) if den > 0 else 0.0)
    return out


# --------------------------------------------------------------------------
def serving_sample(n_requests: int, warm: int, n: int) -> list[int]:
    """Indices of the timed requests whose results are checked (seeded)."""
    rng = np.random.default_rng(7)
    n = min(n, n_requests - warm)
    return sorted(int(i) for i in rng.choice(np.arange(warm, n_requests), n, replace=False))


def serving_run(n_requests: int, rate: float, warm: int = 40, n_check: int = 8,
                oracle_refs=None):
    """Replay a seeded Poisson stream of mixed solves (Nx 512..16384) in real
    time through bpm_submit / bpm_poll; latency = completion - submission as
    stamped by the server.  The first `warm` requests are excluded from the
    statistics.  `n_check` sampled requests are re-run alone for parity, and
    the requests in `oracle_refs` (index -> future of the oracle march) are
    compared with the oracle."""
    import threading
    from paper_2601_06340_gb300 import binding, inputs
    FP32 = binding.BPM_FP32_FUSED
    reqs = inputs.serving_requests(n_requests, rate_per_s=rate)
    binding.bpm_server_configure(0.6, 256, 256, 100000)
    tickets = [None] * len(reqs)
    outs = [np.empty_like(r.workload.psi0) for r in reqs]
    plans = [None] * len(reqs)
    done = [None] * len(reqs)

    def poller():
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(1e-4)
            binding.bpm_poll(tickets[i], -1)
            done[i] = binding.bpm_ticket_times(tickets[i])
    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        wait = t0 + r.arrival_s - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        plans[i] = binding.Plan(r.workload, FP32)
        tickets[i] = binding.bpm_submit(plans[i].handle, r.workload.psi0, outs[i])
    th.join()
    times = np.array(done[warm:])
    lat_ms = (times[:, 2] - times[:, 0]) * 1e3
    wait_ms = (times[:, 1] - times[:, 0]) * 1e3
    span = times[:, 2].max() - times[:, 0].min()
    cells = sum(r.workload.cell_updates for r in reqs[warm:])
    flops = sum(r.workload.cell_updates * FLOPS_PER_CELL(r.workload.nx) for r in reqs[warm:])
    errs = []
    for i in serving_sample(len(reqs), warm, n_check):
        alone = plans[i].propagate(records=False, powers=False).psi
        for b in range(2):
            den = np.linalg.norm(alone[0, b])
            if den > 0:
                errs.append(float(np.linalg.norm(outs[i][0, b] - alone[0, b]) / den))
    for p in plans:
        p.close()
    vs_oracle = None
    if oracle_refs:
        per = []
        for i, fut in sorted(oracle_refs.items()):
            ref, _ = fut.result()
            per.append(max(rel_l2_bands(outs[i], ref.psi)))
        vs_oracle = {"requests": len(per), "max_rel_l2": max(per),
                     "median_rel_l2": float(np.median(per)), "tolerance": 2e-4,
                     "sample": "seeded uniform draw among the timed requests"}
    per_nx = {}
    svc_ms = (times[:, 2] - times[:, 1]) * 1e3
    for nx in sorted({r.workload.nx for r in reqs[warm:]}):
        sel = np.array([r.workload.nx == nx for r in reqs[warm:]])
        nzs = np.array([r.workload.nz for r in reqs[warm:]])[sel]
        per_nx[str(nx)] = {"count": int(sel.sum()),
                           "latency_p50_ms": float(np.percentile(lat_ms[sel], 50)),
                           "service_us_per_step_p50": float(np.percentile(
                               svc_ms[sel] * 1e3 / nzs, 50))}
    return {"requests": len(reqs) - warm, "warmup_requests": warm, "rate_per_s": rate,
            "per_nx": per_nx,
            "mean_active": float(np.sum(times[:, 2] - times[:, 1]) / span),
            "nx_choices": [512, 1024, 2048, 4096, 8192, 16384], "nz_range": [500, 20000],
            "throughput": cells / span, "unit": UNIT,
            "achieved_tflops": flops / span / 1e12,
            "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                           "p99": float(np.percentile(lat_ms, 99)),
                           "max": float(lat_ms.max())},
            "queue_wait_ms_p99": float(np.percentile(wait_ms, 99)),
            "alone_vs_mix_max_rel_l2": max(errs) if errs else None,
            "vs_oracle": vs_oracle}


def curve_fwhm(x: np.ndarray, y: np.ndarray) -> float:
    """Full width at half maximum of a sampled curve (linear interpolation
    at the outermost half-maximum crossings around the peak)."""
    i = int(np.argmax(y))
    half = 0.5 * y[i]
    lo = i
    while lo > 0 and y[lo - 1] >= half:
        lo -= 1
    hi = i
    while hi < len(y) - 1 and y[hi + 1] >= half:
        hi += 1
    xl = x[lo] if lo == 0 else x[lo - 1] + (half - y[lo - 1]) * (x[lo] - x[lo - 1]) / (y[lo] - y[lo - 1])
    xr = x[hi] if hi == len(y) - 1 else x[hi] + (y[hi] - half) * (x[hi + 1] - x[hi]) / (y[hi] - y[hi + 1])
    return float(xr - xl)


ROCKING_ROWS = [128, 140]
BATCH_ROWS = [0, 131, 255]

# Every timed march runs after a write of twice the 129 MB L2 (outside the
# timed region), so no input or table of the previous march is served from
# L2: the separable slices keep the inputs of a solve far below L2.
L2_FLUSH_BYTES = 256 << 20
L2_NOTE = "L2 flushed before every timed march (256 MB write outside the timed region)"


def timed_ms(fn, steps, stream, flush):
    """Device times (ms) of `steps` calls of fn on `stream`, each after an L2
    flush; CUDA events bracket the call alone.  The caller synchronizes."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    return ev


def elapsed(ev) -> list[float]:
    return [a.elapsed_time(b) for a, b in ev]


def rocking_run(dev, stream, barrier, max_over_ranks, world, rank, refs=None, steps=3):
    """256 incidence angles of a Laue slab as the rows of one batched march;
    reflectivity per row from the FP64 band powers."""
    import torch
    from paper_2601_06340_gb300 import binding, inputs
    FP32 = binding.BPM_FP32_FUSED
    wr = inputs.rocking_scan()
    plan = binding.Plan(wr, FP32)
    x = torch.from_numpy(wr.psi0.astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    pw = torch.zeros((wr.batch, 1, 2), dtype=torch.float64, device=dev)

    def march():
        binding.bpm_propagate_device(plan.handle, x, y, None, pw, 0, wr.nz, stream.cuda_stream)
    march()
    barrier()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = timed_ms(march, steps, stream, flush)
    barrier()
    ms = max_over_ranks(sum(elapsed(ev))) / steps
    del flush
    p_in = wr.dx_um * np.sum(np.abs(wr.psi0[:, 0]) ** 2, axis=-1)
    refl = pw[:, -1, 1].cpu().numpy() / p_in
    angles = wr.meta["angles_urad"]
    out = {"workload": "rocking_scan: symmetric Laue slab 100 um, 8 keV, 256 incidence angles "
                       "over +-50 urad, Nx=2048, Nz=2000, Gaussian 200 um FWHM, one batch",
           "value": world * wr.cell_updates / (ms * 1e-3), "unit": UNIT, "ms_per_scan": ms,
           "l2": L2_NOTE,
           "reflectivity": {"peak": float(refl.max()),
                            "peak_angle_urad": float(angles[int(np.argmax(refl))]),
                            "fwhm_urad": curve_fwhm(angles, refl)}}
    if refs:
        got = y.cpu().numpy().astype(np.complex128)
        errs = [rel_l2_bands(got[r:r + 1], f.result()[0].psi) for r, f in zip(ROCKING_ROWS, refs)]
        out["rel_l2_err_sampled_rows"] = [max(e[0] for e in errs), max(e[1] for e in errs)]
        out["sampled_rows"] = ROCKING_ROWS
    plan.close()
    return out


def volume_run(dev, stream, barrier, max_over_ranks, world, rank, ref=None, steps=3):
    """The 3D stand-in workload (both transverse coordinates): one solve of
    512 x 256 x 300 cells.  The paper's only timing (its 3D example, 300 x 200
    x 300 cells, ~13 s on a Perlmutter node) is quoted as context."""
    import torch
    from paper_2601_06340_gb300 import binding, inputs
    FP32 = binding.BPM_FP32_FUSED
    wv = inputs.cube_dislocation_3d()
    plan = binding.Plan(wv, FP32)
    x = torch.from_numpy(wv.psi0.astype(np.complex64)).to(dev)
    y = torch.empty_like(x)

    def march():
        binding.bpm_propagate_device(plan.handle, x, y, None, None, 0, wv.nz, stream.cuda_stream)
    march()
    barrier()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ev = timed_ms(march, steps, stream, flush)
    barrier()
    ms = max_over_ranks(sum(elapsed(ev))) / steps
    del flush
    out = {"workload": "cube_dislocation_3d: Si(440)-like at 17.45 keV, 10 um box crystal, "
                       "edge dislocation along y, Nx=512, Ny=256, Nz=300, dx=dy=dz=0.05 um",
           "value": world * wv.cell_updates / (ms * 1e-3), "unit": UNIT, "ms_per_march": ms,
           "launches_per_march": 2 * wv.nz + 2, "l2": L2_NOTE,
           "paper_context": {"seconds": 13.0, "grid": "300 x 200 x 300",
                             "hardware": "one Perlmutter node (CPU vs GPU not stated)"}}
    if ref is not None:
        res, sec = ref.result()
        out["oracle_seconds_1core"] = sec
        out["rel_l2_err"] = rel_l2_bands(y.cpu().numpy().astype(np.complex128), res.psi)
    plan.close()
    return out


def configs_run(dev, stream, barrier, max_over_ranks, world, rank, refs=None, steps=3):
    """The single-solve configurations besides the headline one: the
    symmetric Laue crystal (Nx=1024, Nz=2000) and the asymmetric Bragg slab
    with a polygonal shape and an edge dislocation (Nx=8192, Nz=12000): the
    fused FP32 and plain FP64 GPU paths, the FP64 oracle on one host core,
    and both paths' errors against it."""
    import torch
    from paper_2601_06340_gb300 import binding, inputs
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for name, make in (("laue_perfect", inputs.laue_perfect),
                       ("asym_dislocation", inputs.asym_dislocation)):
        wl = make()
        wl.record_every = 0
        row = {"nx": wl.nx, "nz": wl.nz}
        psi = {}
        for prec, key in ((binding.BPM_FP32_FUSED, "fused_fp32"),
                          (binding.BPM_FP64_PLAIN, "plain_fp64")):
            plan = binding.Plan(wl, prec)
            dt = torch.complex64 if prec == binding.BPM_FP32_FUSED else torch.complex128
            x = torch.from_numpy(wl.psi0).to(dev).to(dt)
            y = torch.empty_like(x)

            def march():
                binding.bpm_propagate_device(plan.handle, x, y, None, None, 0, wl.nz,
                                             stream.cuda_stream)
            march()
            barrier()
            n = steps if prec == binding.BPM_FP32_FUSED else 1
            ev = timed_ms(march, n, stream, flush)
            barrier()
            ms = max_over_ranks(sum(elapsed(ev))) / n
            row[key] = {"value": world * wl.cell_updates / (ms * 1e-3), "unit": UNIT,
                        "ms_per_march": ms}
            psi[key] = y.cpu().numpy().astype(np.complex128)
            plan.close()
        row["fused_speedup"] = row["fused_fp32"]["value"] / row["plain_fp64"]["value"]
        if refs:
            ref, cpu_s = refs[name].result()
            row["oracle_1core"] = {"value": wl.cell_updates / cpu_s, "unit": UNIT, "cores": 1}
            row["fused_fp32"]["rel_l2_err"] = rel_l2_bands(psi["fused_fp32"], ref.psi)
            row["plain_fp64"]["rel_l2_err"] = rel_l2_bands(psi["plain_fp64"], ref.psi)
        out[name] = row
    out["l2"] = L2_NOTE
    return out


SPLIT_CHECK_STEPS = 600
SPLIT_SIZES = (4096, 8192)
SPLIT_METHODS = (("first_order", "BPM_SPLIT_FIRST_ORDER"), ("verlet", "BPM_SPLIT_VERLET"),
                 ("forest_ruth", "BPM_SPLIT_FOREST_RUTH"))


def split_workload(nx: int):
    """The bent Bragg solve (Nz = 8000) at Nx = 4096 (the headline workload)
    or 8192 (dx halved: the same 819 um window at twice the resolution)."""
    from paper_2601_06340_gb300 import inputs
    return inputs.bragg_bent(nx=nx, dx_um=min(0.2, 800.0 / nx))


def splitting_run(dev, stream, barrier, max_over_ranks, world, rank, refs=None, steps=3):
    """The operator splittings of Eq. split-op on the fused FP32 path: each
    scheme's whole 8000-step march of the bent solve at Nx = 4096 and 8192
    (the launch shape the rule picks), and the error of its first
    SPLIT_CHECK_STEPS steps against the oracle's march with the same scheme."""
    import torch
    from paper_2601_06340_gb300 import binding
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for nx in SPLIT_SIZES:
        wl = split_workload(nx)
        wl.record_every = 0
        row = {"nx": wl.nx, "nz": wl.nz}
        for name, const in SPLIT_METHODS:
            plan = binding.Plan(wl, binding.BPM_FP32_FUSED, splitting=getattr(binding, const))
            x = torch.from_numpy(wl.psi0.astype(np.complex64)).to(dev)
            y = torch.empty_like(x)

            def march(n_end=wl.nz):
                binding.bpm_propagate_device(plan.handle, x, y, None, None, 0, n_end,
                                             stream.cuda_stream)
            march()
            barrier()
            ev = timed_ms(march, steps, stream, flush)
            barrier()
            ms = max_over_ranks(sum(elapsed(ev))) / steps
            r = {"value": world * wl.cell_updates / (ms * 1e-3), "unit": UNIT,
                 "ms_per_march": ms, "us_per_step": 1e3 * ms / wl.nz,
                 "launch_layout": binding.bpm_launch_shape(plan.handle)[0],
                 "slice_form": ["stream", "separable"][binding.bpm_slice_form(plan.handle)[0]]}
            if refs:
                march(SPLIT_CHECK_STEPS)
                torch.cuda.synchronize()
                ref, _ = refs[(nx, name)].result()
                r["rel_l2_err_first_%d_steps" % SPLIT_CHECK_STEPS] = rel_l2_bands(
                    y.cpu().numpy().astype(np.complex128), ref.psi)
            row[name] = r
            plan.close()
        out[str(nx)] = row
    out["tolerance"] = 2e-4
    out["l2"] = L2_NOTE
    return out


def run_reference(args, rank, world):
    """FP64 oracle on the host cores: each step is a bounded sample (the
    first `sample_steps` z-steps of the march)."""
    if rank != 0:
        return
    from oracle import run as orun
    from paper_2601_06340_gb300 import inputs
    wl = inputs.bragg_bent()
    sample_steps = args.ref_sample_steps
    for _ in range(args.warmup):
        orun.run_workload(wl, 0, sample_steps, record_every=0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orun.run_workload(wl, 0, sample_steps, record_every=0)
    dt = (time.perf_counter() - t0) / args.steps
    cells = wl.nx * sample_steps
    value = cells / dt
    sample = (f"first {sample_steps} of the {wl.nz} z-steps of the bragg_bent march "
              f"(Nx={wl.nx}, one energy) per step, numpy float64, single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_gpu(args, rks):
    import torch
    from paper_2601_06340_gb300 import binding, inputs
    import __graft_entry__
    __graft_entry__.build()
    binding.load()
    rank, world = rks.rank, rks.world
    dev = rks.device
    stream = torch.cuda.current_stream()
    FP32, FP64 = binding.BPM_FP32_FUSED, binding.BPM_FP64_PLAIN

    def barrier():
        rks.barrier(torch.cuda.synchronize)

    max_over_ranks = rks.max

    if args.only == "serving":
        if rank == 0:
            print(json.dumps({"only": "serving",
                              **serving_run(args.serving_requests, args.serving_rate)}),
                  flush=True)
        return

    if args.only == "volume":
        r = volume_run(dev, stream, barrier, max_over_ranks, world, rank, ref=None,
                       steps=args.steps)
        if rank == 0:
            print(json.dumps({"only": "volume", **r}), flush=True)
        return

    if args.only == "rocking":
        r = rocking_run(dev, stream, barrier, max_over_ranks, world, rank, refs=None,
                        steps=args.steps)
        if rank == 0:
            print(json.dumps({"only": "rocking", **r}), flush=True)
        return

    if args.only == "batched":
        wb = inputs.pulse_batched()
        planb = binding.Plan(wb, FP32)
        xb = torch.from_numpy(wb.psi0.astype(np.complex64)).to(dev)
        yb = torch.empty_like(xb)
        def march_b():
            binding.bpm_propagate_device(planb.handle, xb, yb, None, None, 0, wb.nz,
                                         stream.cuda_stream)
        for _ in range(args.warmup):
            march_b()
        barrier()
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        ev = timed_ms(march_b, args.steps, stream, flush)
        barrier()
        ms = max_over_ranks(sum(elapsed(ev))) / args.steps
        if rank == 0:
            print(json.dumps({"only": "batched", "value": world * wb.cell_updates / (ms * 1e-3),
                              "unit": UNIT, "ms_per_step": ms}), flush=True)
        planb.close()
        return

    wl = inputs.bragg_bent()
    cells = wl.cell_updates

    # ---- the oracle on the host cores: CPU baselines first (idle host), then
    # every parity reference of this run in a spawn pool, beside the GPU work
    pool, jobs = None, {}
    cpu_baseline = batch_cpu = None
    if rank == 0 and not args.skip_oracle:
        workers = max(1, os.cpu_count() or 1)
        pool = make_oracle_pool(workers)
        cpu_baseline, batch_cpu = cpu_baselines(pool, workers, args.ref_sample_steps,
                                                args.batch_sample_steps)

    def submit_jobs():
        """Every parity reference of the run, into the pool (after the
        headline and end-to-end timings, which need a quiet host)."""
        if pool is None:
            return
        sub = lambda w, **kw: pool.submit(oracle_job, w, kw)
        jobs["head"] = sub(wl, record_every=0)
        if not args.skip_batched:
            wb_all = inputs.pulse_batched()
            jobs["batched"] = [sub(row_workload(wb_all, r), record_every=0) for r in BATCH_ROWS]
        if not args.skip_rocking:
            wr_all = inputs.rocking_scan()
            jobs["rocking"] = [sub(row_workload(wr_all, r)) for r in ROCKING_ROWS]
        if not args.skip_configs:
            jobs["configs"] = {"laue_perfect": sub(inputs.laue_perfect(), record_every=0),
                               "asym_dislocation": sub(inputs.asym_dislocation(),
                                                       record_every=0)}
        if not args.skip_splitting:
            jobs["splitting"] = {(nx, name): sub(split_workload(nx), record_every=0,
                                                 n_end=SPLIT_CHECK_STEPS, method=name)
                                 for nx in SPLIT_SIZES for name, _ in SPLIT_METHODS}
        if not args.skip_volume:
            jobs["volume"] = pool.submit(oracle_job, inputs.cube_dislocation_3d(),
                                         dict(record_every=0), True)
        if not args.skip_serving and args.serving_check > 0:
            reqs = inputs.serving_requests(args.serving_requests, rate_per_s=args.serving_rate)
            jobs["serving"] = {i: sub(reqs[i].workload, record_every=0)
                               for i in serving_sample(len(reqs), 40, args.serving_check)}

    plan32 = binding.Plan(wl, FP32)
    n_rec = plan32.n_rec
    x = torch.from_numpy(wl.psi0.astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    rec = torch.zeros((1, n_rec, 2, wl.nx), dtype=torch.complex64, device=dev)
    pw = torch.zeros((1, n_rec + 1, 2), dtype=torch.float64, device=dev)

    def march32():
        binding.bpm_propagate_device(plan32.handle, x, y, rec, pw, 0, wl.nz, stream.cuda_stream)

    # ---- fused FP32, device-resident (the headline value) -----------------
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        march32()
    barrier()
    with ClockSampler(dev.index) as clk:
        barrier()
        ev = timed_ms(march32, args.steps, stream, flush)
        barrier()
    per_ms = elapsed(ev)
    total_ms = max_over_ranks(sum(per_ms))
    value = world * args.steps * cells / (total_ms * 1e-3)
    clocks = clk.summary()
    march_layout, _ = binding.bpm_launch_shape(plan32.handle)

    if args.only == "fused":
        if rank == 0:
            print(json.dumps({"only": "fused", "value": value, "unit": UNIT,
                              "ms_per_step": total_ms / args.steps}), flush=True)
        plan32.close()
        return

    # ---- measured arithmetic peaks (the roofline denominators) ------------
    with ClockSampler(dev.index) as clk_peak:
        f32a, _ = binding.bpm_fp_peak(binding.BPM_PEAK_FP32_FFMA, 96000)
        f32b, _ = binding.bpm_fp_peak(binding.BPM_PEAK_FP32_FFMA2, 48000)
        f64, _ = binding.bpm_fp_peak(binding.BPM_PEAK_FP64_DFMA, 1500)
    peaks = {"fp32_tflops": max(f32a, f32b) / 1e12, "fp32_ffma_tflops": f32a / 1e12,
             "fp32_ffma2_tflops": f32b / 1e12, "fp64_tflops": f64 / 1e12,
             "sm_mhz": clk_peak.summary().get("sm_mhz"),
             "how": "bpm_fp_peak: 8 CTAs x 256 threads per SM, 8 independent FMA chains per "
                    "thread, CUDA events, after a warm-up launch; 1 FMA = 2 flops"}

    fused_psi = y.cpu().numpy().astype(np.complex128)

    # ---- end to end through the host C-ABI (pinned host buffers) ----------
    pin_in = torch.from_numpy(wl.psi0.astype(np.complex128)).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    pin_rec = torch.empty((1, n_rec, 2, wl.nx), dtype=torch.complex64).pin_memory()
    pin_pw = torch.empty((1, n_rec + 1, 2), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, args.steps // 2)
    binding.bpm_propagate(plan32.handle, pin_in, pin_out, pin_rec, pin_pw, 0, wl.nz)
    barrier()
    e2e_s = 0.0
    for _ in range(e2e_steps):
        flush.zero_()                        # L2 flushed outside the timed call
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        binding.bpm_propagate(plan32.handle, pin_in, pin_out, pin_rec, pin_pw, 0, wl.nz)
        _ = float(pin_pw[0, -1, 1])          # read the step's result on the host
        e2e_s += time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s)
    e2e_value = world * e2e_steps * cells / e2e_s
    h2d = pin_in.numel() * 16
    d2h = pin_out.numel() * 16 + pin_rec.numel() * 8 + pin_pw.numel() * 8
    plan32.close()

    # the oracle's references, computed on the host from here on
    submit_jobs()

    # ---- plain FP64 per-step GPU path (same workload) ----------------------
    plan64 = binding.Plan(wl, FP64)
    x64 = torch.from_numpy(wl.psi0).to(dev)
    y64 = torch.empty_like(x64)
    binding.bpm_propagate_device(plan64.handle, x64, y64, None, None, 0, wl.nz,
                                 stream.cuda_stream)
    barrier()
    s64 = max(1, args.steps // 5)
    ev64 = timed_ms(lambda: binding.bpm_propagate_device(plan64.handle, x64, y64, None, None,
                                                         0, wl.nz, stream.cuda_stream),
                    s64, stream, flush)
    barrier()
    ms64 = max_over_ranks(sum(elapsed(ev64))) / s64
    value64 = world * cells / (ms64 * 1e-3)
    psi64 = y64.cpu().numpy()
    plan64.close()
    # ---- parity on the timed workload (the oracle's reference) -------------
    ref = jobs["head"].result()[0] if "head" in jobs else None
    err32 = rel_l2_bands(fused_psi, ref.psi) if ref is not None else None
    err64 = rel_l2_bands(psi64, ref.psi) if ref is not None else None

    # ---- batched: 256 photon energies (pulse), one launch + energy->time --
    batched = None
    if not args.skip_batched:
        wb = inputs.pulse_batched()
        planb = binding.Plan(wb, FP32)
        xb = torch.from_numpy(wb.psi0.astype(np.complex64)).to(dev)
        yb = torch.empty_like(xb)
        tb = torch.empty((2, wb.nx, wb.batch), dtype=torch.complex64, device=dev)

        def march_b():
            binding.bpm_propagate_device(planb.handle, xb, yb, None, None, 0, wb.nz,
                                         stream.cuda_stream)
            binding.bpm_omega_to_t_device(yb, tb, wb.batch, wb.nx, FP32, stream.cuda_stream)
        march_b()
        barrier()
        kb = 3
        evb = timed_ms(march_b, kb, stream, flush)
        barrier()
        msb = max_over_ranks(sum(elapsed(evb))) / kb
        cells_b = wb.cell_updates
        layout, chunk = binding.bpm_launch_shape(planb.handle)
        batched = {"workload": "pulse_batched: 256 energies 9 keV +- 5 eV, Laue 300 um, "
                               "bent R=2 m, Nx=4096, Nz=6000, + energy->time synthesis",
                   "value": world * cells_b / (msb * 1e-3), "unit": UNIT,
                   "ms_per_march": msb, "cpu_baseline": batch_cpu, "l2": L2_NOTE,
                   "launch_shape": {"layout": {2: "split4", 1: "cluster", 0: "cta", -1: "rule"}[layout],
                                    "rotation_chunk": chunk,
                                    "autotune": os.environ.get("BPM_AUTOTUNE", "1") != "0"}}
        if "batched" in jobs:
            gotb = yb.cpu().numpy().astype(np.complex128)
            eb = [rel_l2_bands(gotb[r:r + 1], f.result()[0].psi)
                  for r, f in zip(BATCH_ROWS, jobs["batched"])]
            batched["rel_l2_err_sampled_rows"] = [max(e[0] for e in eb), max(e[1] for e in eb)]
            batched["sampled_rows"] = BATCH_ROWS
            batched["tolerance"] = 2e-4
        planb.close()

    # ---- rocking curve: incidence angles as the rows of one batch ----------
    rocking = None
    if not args.skip_rocking:
        rocking = rocking_run(dev, stream, barrier, max_over_ranks, world, rank,
                              refs=jobs.get("rocking"))

    # ---- the other single-solve configurations ------------------------------
    configs = None
    if not args.skip_configs:
        configs = configs_run(dev, stream, barrier, max_over_ranks, world, rank,
                              refs=jobs.get("configs"))

    # ---- operator splittings (Eq. split-op) on the fused path --------------
    splitting = None
    if not args.skip_splitting:
        splitting = splitting_run(dev, stream, barrier, max_over_ranks, world, rank,
                                  refs=jobs.get("splitting"))

    # ---- 3D: both transverse coordinates -----------------------------------
    volume = None
    if not args.skip_volume:
        volume = volume_run(dev, stream, barrier, max_over_ranks, world, rank,
                            ref=jobs.get("volume"))

    # ---- serving: Poisson stream of mixed solves through submit/poll ------
    serving = None
    if not args.skip_serving and rank == 0:
        # the host must be quiet for a real-time replay: wait for the pool
        for key in ("head", "batched", "rocking", "configs", "splitting", "volume"):
            fl = jobs.get(key)
            for f in (fl.values() if isinstance(fl, dict) else fl if isinstance(fl, list)
                      else [fl] if fl is not None else []):
                f.result()
        if "serving" in jobs:
            for f in jobs["serving"].values():
                f.result()
        serving = serving_run(args.serving_requests, args.serving_rate,
                              oracle_refs=jobs.get("serving"))
        # the same mix arriving far faster than it can be served: the GPU
        # stays saturated, so the throughput is the server's capacity
        sat = serving_run(args.capacity_requests, args.capacity_rate, warm=0, n_check=0)
        serving["capacity"] = {"requests": sat["requests"], "rate_per_s": sat["rate_per_s"],
                               "throughput": sat["throughput"], "unit": UNIT,
                               "achieved_tflops": sat["achieved_tflops"],
                               "mean_active": sat["mean_active"]}

    # ---- roofline of the dominant kernel (fused march) ---------------------
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    derived_tflops = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    peak_tflops = peaks["fp32_tflops"]
    avg_launch_s = float(np.mean(per_ms)) * 1e-3
    achieved = cells * FLOPS_PER_CELL(wl.nx) / avg_launch_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops,
                "traffic": profiled_traffic("fused_march_bragg_bent.md"),
                "kernel": MARCH_KERNELS[march_layout][0],
                "peak_basis": "measured: FP32 FMA throughput kernel (bpm_fp_peak, the faster "
                              "of FFMA and packed FFMA2) on this GPU in this run",
                "peak_derived": derived_tflops,
                "peak_derived_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
                # the solve occupies one cluster: the fraction of its SMs' peak
                "cluster_sms": MARCH_KERNELS[march_layout][1],
                "cluster_frac": achieved / (MARCH_KERNELS[march_layout][1] * peak_tflops / sms),
                "flops_per_cell_update": FLOPS_PER_CELL(wl.nx)}
    if batched is not None:
        ach_b = batched["value"] / world * FLOPS_PER_CELL(4096) / 1e12
        batched["roofline"] = {"bound": "alu", "achieved": ach_b, "peak": peak_tflops,
                               "unit": "TFLOP/s", "frac": ach_b / peak_tflops}
    if serving is not None:
        for part in (serving, serving.get("capacity")):
            if part is not None:
                part["roofline"] = {"bound": "alu", "achieved": part["achieved_tflops"],
                                    "peak": peak_tflops, "unit": "TFLOP/s",
                                    "frac": part["achieved_tflops"] / peak_tflops}
    if volume is not None:
        # two 2D FFTs per band and step: 4 x 5 log2(Nx Ny) flops per cell-update
        ach_v = volume["value"] / world * FLOPS_PER_CELL(512 * 256) / 1e12
        volume["roofline"] = {"bound": "alu", "achieved": ach_v, "peak": peak_tflops,
                              "unit": "TFLOP/s", "frac": ach_v / peak_tflops}
    if rocking is not None:
        ach_r = rocking["value"] / world * FLOPS_PER_CELL(2048) / 1e12
        rocking["roofline"] = {"bound": "alu", "achieved": ach_r, "peak": peak_tflops,
                               "unit": "TFLOP/s", "frac": ach_r / peak_tflops}

    if rank == 0:
        lat = np.array(per_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas{world}",
                       "l2": L2_NOTE},
            "rel_l2_err": err32,
            "tolerance": 2e-4,
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99))},
            "fp64_plain": {"value": value64, "unit": UNIT, "ms_per_step": ms64,
                           "rel_l2_err": err64, "tolerance": 1e-10,
                           "fused_speedup": value / value64,
                           "roofline": {"bound": "fp64 alu / launches",
                                        "achieved": value64 * FLOPS_PER_CELL(wl.nx) / 1e12,
                                        "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                                        "frac": value64 * FLOPS_PER_CELL(wl.nx) / 1e12
                                        / peaks["fp64_tflops"],
                                        "launches_per_step": 2 * (wl.nx.bit_length() // 2) + 2,
                                        "peak_basis": "measured: FP64 DFMA throughput kernel "
                                                      "(bpm_fp_peak)"}},
            "peaks": peaks,
            "batched": batched,
            "configs": configs,
            "splitting": splitting,
            "rocking": rocking,
            "volume": volume,
            "serving": serving,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": 2 * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu_baseline,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if pool is not None:
        pool.shutdown(wait=False, cancel_futures=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-sample-steps", type=int, default=2000,
                    help="z-steps of the oracle's headline sample (CPU baseline)")
    ap.add_argument("--batch-sample-steps", type=int, default=1500,
                    help="z-steps per energy row of the oracle's all-cores batch sample")
    ap.add_argument("--serving-check", type=int, default=32,
                    help="served requests compared with the oracle")
    ap.add_argument("--skip-oracle", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-rocking", action="store_true")
    ap.add_argument("--skip-splitting", action="store_true")
    ap.add_argument("--skip-volume", action="store_true")
    ap.add_argument("--skip-configs", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=440)
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--capacity-requests", type=int, default=600)
    ap.add_argument("--capacity-rate", type=float, default=3000.0)
    ap.add_argument("--only", default="all", choices=["all", "fused", "batched", "rocking", "volume", "serving"],
                    help="time only the fused single-solve march, the 256-energy batch, "
                         "the 256-angle rocking scan, the 3D solve or the serving run "
                         "(profiling runs)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_2601_06340_gb300 import replicas
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    rks = replicas.Ranks(backend="nccl", device=dev)   # replicas: no data-path collective
    try:
        run_gpu(args, rks)
    finally:
        rks.close()


if __name__ == "__main__":
    main()
