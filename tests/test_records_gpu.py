"""Records at every step (record_every = 1) in every fused kernel family.

A record multiplies the field by the common phase g^(n+1) of Eq. fov10's
output, which one thread per row computes in FP64 at the step's start and
the others read when they record.  Warps of a row run out of step by up to
a step, so with a record at every step the phase of step n + 1 is written
while a slower warp may still read step n's: it is kept in two slots by step
parity.  Records and band powers of every step must match the oracle's.
"""

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, inputs
from parity_util import TOL_FP32, band_errors, submit_ref

pytestmark = pytest.mark.gpu

FP32 = binding.BPM_FP32_FUSED
FIRST = binding.BPM_SPLIT_FIRST_ORDER
VERLET = binding.BPM_SPLIT_VERLET
FR = binding.BPM_SPLIT_FOREST_RUTH

# (nx, BPM_FUSED_LAYOUT, splitting): one CTA, the 2-CTA cluster, the
# half-band split (8 and 16 points per thread), the split bands (N = 8192
# with each step form: the next slice staged in the peer spectrum buffer)
CASES = [
    (64, None, FIRST),
    (1024, "cta", FIRST),
    (1024, "cluster", FIRST),
    (1024, "cluster", VERLET),
    (1024, "cluster", FR),
    (1024, "cta", FR),
    (4096, None, FIRST),
    (4096, "split16", FIRST),
    (4096, None, VERLET),
    (4096, None, FR),
    (8192, None, FIRST),
    (8192, None, VERLET),
    (8192, None, FR),
    (16384, None, FIRST),
]


def _workload(nx):
    return inputs.bragg_bent(nx=nx, nz=60, dx_um=min(0.2, 800.0 / nx), record_every=1)


@pytest.fixture(scope="module")
def refs():
    method = {FIRST: "first_order", VERLET: "verlet", FR: "forest_ruth"}
    keys = sorted({(nx, split) for nx, _, split in CASES})
    return {k: submit_ref(_workload(k[0]), method=method[k[1]]) for k in keys}


@pytest.mark.parametrize("nx,layout,split", CASES)
def test_every_step_records(bpm_lib, monkeypatch, refs, nx, layout, split):
    if layout:
        monkeypatch.setenv("BPM_FUSED_LAYOUT", layout)
    else:
        monkeypatch.delenv("BPM_FUSED_LAYOUT", raising=False)
    wl = _workload(nx)
    with binding.Plan(wl, FP32, splitting=split) as plan:
        out = plan.propagate()
    ref = refs[(nx, split)].result()
    assert out.records.shape[1] == wl.nz
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= TOL_FP32, errs
    # every record on its own (a wrong phase on one record would hide in the
    # sum over 60 of them)
    for k in range(wl.nz):
        e = band_errors(out.records[:, k], ref.records[:, k])
        assert max(e) <= TOL_FP32, (k, e)
    assert np.allclose(out.powers, ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())
