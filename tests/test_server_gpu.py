"""Continuous-batching server (bpm_submit / bpm_poll) on the GPU.

Requests of different sizes, lengths and geometries are admitted while
others run and share fused launches; each result must equal the same solve
run alone through bpm_propagate within the FP32 tolerance.  Host-side
policies (arrival-order admission under a memory budget, queue overflow,
oversized requests, plans locked while a request is in flight) are checked
through the C ABI."""

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, inputs

from parity_util import TOL_FP32, band_errors

pytestmark = pytest.mark.gpu

FP32 = binding.BPM_FP32_FUSED


def _mix(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.choice([512, 1024, 2048, 4096, 8192]))
        nz = int(rng.integers(100, 700))
        out.append(inputs.serving_request(rng, nx, nz))
    return out


def _alone(wl):
    with binding.Plan(wl, FP32) as plan:
        return plan.propagate(records=False, powers=False).psi


def test_mix_equals_alone(bpm_lib):
    binding.bpm_server_configure(0.6, 64, 128, 1000)
    reqs = _mix(12, 1)
    plans, outs, tickets = [], [], []
    for wl in reqs:
        plan = binding.Plan(wl, FP32)
        out = np.empty_like(wl.psi0)
        tickets.append(binding.bpm_submit(plan.handle, wl.psi0, out))
        plans.append(plan)
        outs.append(out)
    for t in tickets:
        assert binding.bpm_poll(t, -1) == binding.BPM_OK
    for wl, out in zip(reqs, outs):
        errs = band_errors(out, _alone(wl))
        assert max(errs) <= TOL_FP32, errs
    for t in tickets:
        ts, ta, td = binding.bpm_ticket_times(t)
        assert 0 < ts <= ta <= td
    for p in plans:
        p.close()


def test_injected_launch_failure_fails_only_that_size(bpm_lib):
    # host-side fault injection: the next batch launch of N = 1024 fails as a
    # failed kernel launch would; N = 2048 requests are not affected and the
    # server serves N = 1024 again afterwards
    binding.bpm_server_configure(0.6, 64, 128, 1000)
    rng = np.random.default_rng(11)
    wls = [inputs.serving_request(rng, nx, 400) for nx in (1024, 2048, 1024, 2048)]
    plans, outs, tickets = [], [], []
    binding.bpm_server_inject_launch_failure(1024, 1)
    try:
        for wl in wls:
            plan = binding.Plan(wl, FP32)
            out = np.empty_like(wl.psi0)
            tickets.append(binding.bpm_submit(plan.handle, wl.psi0, out))
            plans.append(plan)
            outs.append(out)
        codes = []
        for t in tickets:
            try:
                codes.append(binding.bpm_poll(t, -1))
            except binding.BpmError as e:
                codes.append(e.code)
    finally:
        binding.bpm_server_inject_launch_failure(1024, 0)
    assert codes[0] == binding.BPM_ERR_CUDA
    # the second N = 1024 request failed with it if it shared the bucket then
    assert codes[2] in (binding.BPM_OK, binding.BPM_ERR_CUDA)
    for k in (1, 3) if codes[2] != binding.BPM_OK else (1, 2, 3):
        assert codes[k] == binding.BPM_OK
        assert max(band_errors(outs[k], _alone(wls[k]))) <= TOL_FP32
    # a new N = 1024 request on a failed request's plan succeeds
    out = np.empty_like(wls[0].psi0)
    t = binding.bpm_submit(plans[0].handle, wls[0].psi0, out)
    assert binding.bpm_poll(t, -1) == binding.BPM_OK
    assert max(band_errors(out, _alone(wls[0]))) <= TOL_FP32
    for p in plans:
        p.close()


def test_verlet_requests_share_the_server_with_first_order_ones(bpm_lib, monkeypatch):
    # FP32 plans set to Verlet or Forest-Ruth march in their own launch
    # groups (N <= 4096 one CTA per row on the half-step or fourth-order
    # kernel, N = 8192 and 16384 on the split-band forms); each result
    # equals the same plan marched alone (on the same kernel: the solo march
    # is forced to one CTA, which the split-band sizes do not have)
    binding.bpm_server_configure(0.6, 64, 128, 1000)
    V, F = binding.BPM_SPLIT_VERLET, binding.BPM_SPLIT_FIRST_ORDER
    R = binding.BPM_SPLIT_FOREST_RUTH
    specs = [(512, V), (512, F), (1024, V), (4096, V), (4096, F), (2048, F), (1024, R),
             (4096, R), (8192, V), (8192, R), (16384, V), (8192, F)]
    rng = np.random.default_rng(21)
    wls = [inputs.serving_request(rng, nx, 300) for nx, _ in specs]
    plans = [binding.Plan(wl, FP32, splitting=sp) for wl, (_, sp) in zip(wls, specs)]
    outs = [np.empty_like(wl.psi0) for wl in wls]
    try:
        tickets = [binding.bpm_submit(p.handle, wl.psi0, o) for p, wl, o in zip(plans, wls, outs)]
        for t in tickets:
            assert binding.bpm_poll(t, -1) == binding.BPM_OK
        monkeypatch.setenv("BPM_FUSED_LAYOUT", "cta")
        for p, wl, o, (_, sp) in zip(plans, wls, outs, specs):
            alone = p.propagate(records=False, powers=False).psi
            errs = band_errors(o, alone)
            # the same kernel and steps: Verlet and Forest-Ruth rows agree to
            # rounding
            assert max(errs) <= (TOL_FP32 if sp == F else 1e-6), (sp, errs)
    finally:
        for p in plans:
            p.close()


def test_admission_respects_memory_budget_and_order(bpm_lib):
    # budget big enough for about one request at a time
    wl = inputs.serving_request(np.random.default_rng(5), 4096, 300)
    binding.bpm_server_configure(1e-4, 64, 64, 1000)
    plans, outs, tickets = [], [], []
    try:
        for i in range(4):
            plan = binding.Plan(wl, FP32)
            out = np.empty_like(wl.psi0)
            tickets.append(binding.bpm_submit(plan.handle, wl.psi0, out))
            plans.append(plan)
            outs.append(out)
        for t in tickets:
            assert binding.bpm_poll(t, -1) == binding.BPM_OK
        times = [binding.bpm_ticket_times(t) for t in tickets]
        admits = [t[1] for t in times]
        assert admits == sorted(admits)
        ref = _alone(wl)
        for out in outs:
            assert max(band_errors(out, ref)) <= TOL_FP32
    finally:
        for p in plans:
            p.close()
        binding.bpm_server_configure(0.6, 256, 256, 100000)


def test_queue_overflow_oversized_request_and_busy_plan(bpm_lib):
    wl = inputs.serving_request(np.random.default_rng(6), 1024, 2000)
    binding.bpm_server_configure(0.6, 1, 64, 1)
    plans = [binding.Plan(wl, FP32) for _ in range(3)]
    outs = [np.empty_like(wl.psi0) for _ in range(3)]
    try:
        t0 = binding.bpm_submit(plans[0].handle, wl.psi0, outs[0])
        # same plan twice: busy; plan locked against changes while in flight
        with pytest.raises(binding.BpmError) as e:
            binding.bpm_submit(plans[0].handle, wl.psi0, outs[0])
        assert e.value.code == binding.BPM_ERR_BUSY
        st = binding.BPM_OK
        try:
            binding.bpm_set_strain(plans[0].handle, inputs.STRAIN_NONE)
        except binding.BpmError as err:
            st = err.code
        # either still pending (busy) or already finished (ok)
        assert st in (binding.BPM_OK, binding.BPM_ERR_BUSY)
        # max_active = 1 and max_queue = 1: a burst overflows the queue
        codes = []
        tickets = [t0]
        for p, o in zip(plans[1:], outs[1:]):
            try:
                tickets.append(binding.bpm_submit(p.handle, wl.psi0, o))
            except binding.BpmError as err:
                codes.append(err.code)
        for t in tickets:
            assert binding.bpm_poll(t, -1) == binding.BPM_OK
        assert all(c == binding.BPM_ERR_BUSY for c in codes)
        # a request larger than the whole budget is refused up front
        binding.bpm_server_configure(1e-9, 0, 0, 0)
        with pytest.raises(binding.BpmError) as e:
            binding.bpm_submit(plans[1].handle, wl.psi0, outs[1])
        assert e.value.code == binding.BPM_ERR_OOM
    finally:
        binding.bpm_server_configure(0.6, 256, 256, 100000)
        for p in plans:
            p.close()


def test_staged_forest_ruth_refused_by_the_server(bpm_lib):
    """A Forest-Ruth plan of N = 16384 marches stage by stage, which does not
    fit a shared launch: bpm_submit refuses it up front."""
    wl = inputs.serving_request(np.random.default_rng(9), 16384, 50)
    with binding.Plan(wl, FP32, splitting=binding.BPM_SPLIT_FOREST_RUTH) as plan:
        out = np.empty_like(wl.psi0)
        with pytest.raises(binding.BpmError) as e:
            binding.bpm_submit(plan.handle, wl.psi0, out)
        assert e.value.code == binding.BPM_ERR_INVALID


def test_poll_timeout_and_collection(bpm_lib):
    binding.bpm_server_configure(0.6, 64, 64, 100)
    wl = inputs.serving_request(np.random.default_rng(7), 2048, 3000)
    with binding.Plan(wl, FP32) as plan:
        out = np.empty_like(wl.psi0)
        t = binding.bpm_submit(plan.handle, wl.psi0, out)
        first = binding.bpm_poll(t, 0)
        assert first in (binding.BPM_OK, binding.BPM_NOT_READY)
        if first == binding.BPM_NOT_READY:
            assert binding.bpm_poll(t, -1) == binding.BPM_OK
        with pytest.raises(binding.BpmError):
            binding.bpm_poll(t, 0)           # already collected


def test_concurrent_submits_on_one_plan_admit_exactly_one(bpm_lib):
    """Two threads submit on the same plan at the same moment: the plan takes
    one request at a time, so exactly one submit is accepted and the other
    returns BPM_ERR_BUSY (never both: two requests would share the plan's
    device state).  Repeated so that the two calls overlap in most trials."""
    import ctypes
    import threading
    binding.bpm_server_configure(0.6, 64, 128, 1000)
    rng = np.random.default_rng(5)
    wl = inputs.serving_request(rng, 512, 64)
    lib = binding.load()
    psi_in = np.ascontiguousarray(wl.psi0)
    with binding.Plan(wl, FP32) as plan:
        for _ in range(40):
            outs = [np.empty_like(psi_in) for _ in range(2)]
            tickets = [ctypes.c_uint64(0) for _ in range(2)]
            codes = [None, None]
            go = threading.Barrier(2)

            def submit(i):
                go.wait()
                codes[i] = lib.bpm_submit(plan.handle, binding._ptr(psi_in),
                                          binding._ptr(outs[i]), None, None,
                                          ctypes.byref(tickets[i]))
            th = [threading.Thread(target=submit, args=(i,)) for i in range(2)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            assert sorted(codes) == [binding.BPM_ERR_BUSY, binding.BPM_OK], codes
            won = codes.index(binding.BPM_OK)
            assert binding.bpm_poll(tickets[won].value, -1) == binding.BPM_OK


def test_served_mix_matches_oracle(bpm_lib):
    """Requests of every transform size the server takes (512..16384, two
    each, 500-3000 steps) plus three long ones (512 x 20000, 2048 x 12000,
    4096 x 8000), submitted together so that they overlap on the GPU: every
    served result against the FP64 oracle at the FP32 bound (not only
    against the same request run alone)."""
    from parity_util import submit_ref
    binding.bpm_server_configure(0.6, 64, 256, 1000)
    rng = np.random.default_rng(29)
    sizes = [(nx, int(rng.integers(500, 3001)))
             for nx in (512, 1024, 2048, 4096, 8192, 16384) for _ in range(2)]
    sizes += [(512, 20000), (2048, 12000), (4096, 8000)]
    reqs = [inputs.serving_request(rng, nx, nz) for nx, nz in sizes]
    refs = [submit_ref(wl, record_every=0) for wl in reqs]
    plans, outs, tickets = [], [], []
    for wl in reqs:
        plan = binding.Plan(wl, FP32)
        out = np.empty_like(wl.psi0)
        tickets.append(binding.bpm_submit(plan.handle, wl.psi0, out))
        plans.append(plan)
        outs.append(out)
    for t in tickets:
        assert binding.bpm_poll(t, -1) == binding.BPM_OK
    for p in plans:
        p.close()
    worst = []
    for wl, out, fut in zip(reqs, outs, refs):
        errs = band_errors(out, fut.result().psi)
        worst.append((max(errs), wl.nx, wl.nz))
        assert max(errs) <= TOL_FP32, (wl.nx, wl.nz, errs)
