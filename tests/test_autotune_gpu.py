"""Launch-shape autotuning of batch marches.

A batch that can run as one 2-CTA cluster per row or one CTA per row, or as a
rotation with several chunk lengths, is timed in each shape on its first
march and runs in the fastest.  The chosen shape must be one of the
candidates, the result must match the oracle, and rotation chunks must not
change a single bit of the fields and records (rows are independent and each
chunk resumes from the stored FP32 state).
"""

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, inputs
from parity_util import band_errors, run_ref

pytestmark = pytest.mark.gpu

FP32 = binding.BPM_FP32_FUSED


def _march(wl, monkeypatch, tune):
    monkeypatch.setenv("BPM_AUTOTUNE", "1" if tune else "0")
    with binding.Plan(wl, FP32) as plan:
        out = plan.propagate()
        shape = binding.bpm_launch_shape(plan.handle)
    return out, shape


def test_layout_search_for_a_small_batch(bpm_lib, monkeypatch):
    wl = inputs.pulse_batched(nx=2048, nz=200, n_energy=40, record_every=60)
    out, shape = _march(wl, monkeypatch, True)
    assert shape[0] in (0, 1, 2) and shape[1] == 0, shape
    rule, rshape = _march(wl, monkeypatch, False)
    assert rshape == (-1, 0)
    rows = [0, 21, 39]
    ref = run_ref(wl, rows=rows)
    for o in (out, rule):
        errs = band_errors(o.psi[rows], ref.psi, o.records[rows], ref.records)
        assert max(errs) <= 2e-5, errs
    # the tuned shape is kept for the process: a second plan of the same
    # shape reuses it without a search
    again, shape2 = _march(wl, monkeypatch, True)
    assert shape2 == shape
    assert np.array_equal(again.psi, out.psi)


def test_rotation_chunk_search_is_bit_exact(bpm_lib, monkeypatch):
    wl = inputs.pulse_batched(nx=4096, nz=300, n_energy=200, record_every=100)
    out, shape = _march(wl, monkeypatch, True)
    assert shape[0] == 0 and shape[1] in (64, 128, 256, 300), shape
    rule, rshape = _march(wl, monkeypatch, False)
    assert rshape == (-1, 64)
    assert np.array_equal(out.psi, rule.psi)
    assert np.array_equal(out.records, rule.records)
    # the rule runs a rotation's short tail launches on the 2-CTA cluster
    # kernel, which sums the same FP64 per-thread partial powers in another
    # tree order: equal to FP64 rounding, not bit for bit
    assert np.allclose(out.powers, rule.powers, rtol=1e-14, atol=0)
    rows = [7, 199]
    ref = run_ref(wl, rows=rows)
    assert max(band_errors(out.psi[rows], ref.psi)) <= 2e-5
