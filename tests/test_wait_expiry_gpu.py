"""Bounded device waits give up without a fault and leave the context usable.

Every march kernel waits on its mbarriers (strain-slice bulk copies, data
from peer CTAs) through one bounded polling loop and reports an expired wait
as a status bit that the host turns into BPM_ERR_TIMEOUT.  The self-test
kernel arms a barrier for bytes that no copy delivers -- a message nobody
sends -- so the wait runs to its limit; the test checks the status word, that
the limit is short, and that a march on the same context afterwards still
equals the oracle."""

import pytest

from paper_2601_06340_gb300 import binding, inputs

from parity_util import TOL_FP32, band_errors, run_ref

pytestmark = pytest.mark.gpu


def test_expired_wait_sets_status_and_context_stays_usable(bpm_lib):
    status, seconds = binding.bpm_selftest_wait_expiry()
    assert status == 1
    assert 0.0 < seconds < 5.0, seconds
    print(f"bounded wait gave up after {seconds:.3f} s")
    wl = inputs.laue_perfect(nx=1024, nz=300)
    ref = run_ref(wl)
    with binding.Plan(wl, binding.BPM_FP32_FUSED) as plan:
        out = plan.propagate()
    assert max(band_errors(out.psi, ref.psi)) <= TOL_FP32
