"""N = 4096 solves in their launch layouts: the half-band split on a 4-CTA
cluster with 8 points per thread (the rule while every row gets four SMs)
or 16 (forced), the 2-CTA cluster and one CTA per row.  Each must match the oracle within the FP32 tolerance,
on the final field alone (the stricter reading when a band has decayed) and
on every record, over marches long enough for per-step errors to build up.
"""

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, inputs
from parity_util import TOL_FP32, band_errors, run_ref

pytestmark = pytest.mark.gpu

FP32 = binding.BPM_FP32_FUSED


def _march(wl, monkeypatch, layout):
    if layout:
        monkeypatch.setenv("BPM_FUSED_LAYOUT", layout)
    else:
        monkeypatch.delenv("BPM_FUSED_LAYOUT", raising=False)
    with binding.Plan(wl, FP32) as plan:
        out = plan.propagate()
        shape = binding.bpm_launch_shape(plan.handle)
    return out, shape


@pytest.mark.parametrize("seed", [0, 1])
def test_layouts_against_oracle(bpm_lib, monkeypatch, seed):
    rng = np.random.default_rng(40 + seed)
    wl = inputs.serving_request(rng, 4096, 3000)
    wl.record_every = 700
    ref = run_ref(wl)
    outs = {}
    for layout, want in ((None, 2), ("split16", 8), ("cluster", -1), ("cta", -1)):
        out, shape = _march(wl, monkeypatch, layout)
        assert shape[0] == want, (layout, shape)
        final = band_errors(out.psi, ref.psi)
        full = band_errors(out.psi, ref.psi, out.records, ref.records)
        assert max(final) <= TOL_FP32 and max(full) <= TOL_FP32, (layout, final, full)
        assert np.allclose(out.powers, ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())
        outs[layout] = out
    # the layouts differ only by FP32 rounding
    assert max(band_errors(outs[None].psi, outs["cluster"].psi)) <= 1e-4


def test_split_bragg_bent_full_march(bpm_lib, monkeypatch):
    """The 8000-step bent Bragg solve: its weak transmitted band at the
    exit is the hardest reading of the bound."""
    wl = inputs.bragg_bent()
    ref = run_ref(wl)
    out, shape = _march(wl, monkeypatch, None)
    assert shape[0] == 2
    final = band_errors(out.psi, ref.psi)
    assert max(final) <= TOL_FP32, final


def test_split_resume_and_small_batch(bpm_lib, monkeypatch):
    """A march resumed half-way equals the whole march (the half-band kernel
    reloads its state and tables per launch), and an 8-row N = 4096 batch
    (every row still gets four SMs) matches the oracle row by row."""
    monkeypatch.delenv("BPM_FUSED_LAYOUT", raising=False)
    wl = inputs.bragg_bent(nx=4096, nz=1400, record_every=200)
    with binding.Plan(wl, FP32) as plan:
        full = plan.propagate()
        assert binding.bpm_launch_shape(plan.handle)[0] == 2
        first = plan.propagate(n_end=700)
        rec = first.records.copy()
        pw = first.powers.copy()
        second = plan.propagate(first.psi, n_begin=700,
                                out=binding.MarchOutput(np.empty_like(first.psi), rec, pw))
    assert max(band_errors(second.psi, full.psi, second.records, full.records)) <= 1e-5
    wb = inputs.pulse_batched(nx=4096, nz=300, n_energy=8, record_every=100)
    with binding.Plan(wb, FP32) as plan:
        out = plan.propagate()
        assert binding.bpm_launch_shape(plan.handle)[0] in (0, 1, 2)
    rows = [0, 7]
    ref = run_ref(wb, rows=rows)
    assert max(band_errors(out.psi[rows], ref.psi, out.records[rows], ref.records)) <= 2e-5


def test_split16_bragg_bent_full_march(bpm_lib, monkeypatch):
    """The 16-points-per-thread form of the half-band split (forced; the rule
    takes the 8-point form) on the 8000-step bent Bragg solve: fields,
    records and powers against the oracle, and a march resumed at step 3000
    through the host API also within the bound."""
    wl = inputs.bragg_bent()
    ref = run_ref(wl)
    out, shape = _march(wl, monkeypatch, "split16")
    assert shape[0] == 8
    assert max(band_errors(out.psi, ref.psi)) <= TOL_FP32
    assert max(band_errors(out.psi, ref.psi, out.records, ref.records)) <= TOL_FP32
    assert np.allclose(out.powers, ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())
    with binding.Plan(wl, FP32) as plan:
        first = plan.propagate(n_end=3000)
        rest = plan.propagate(first.psi, n_begin=3000)
    assert max(band_errors(rest.psi, ref.psi)) <= TOL_FP32
