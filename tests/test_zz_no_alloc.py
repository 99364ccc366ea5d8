"""The allocation-free FP64 march (bpm_march_f64_noalloc) against the plan
based march (bpm_propagate_device on an FP64 plan).

Callers that cannot allocate device memory use the allocation-free entry
point with their own buffers; its working memory is static and shared by
every call.  A first call of another size (other twiddles, row descriptors
and scratch contents) precedes two checked calls in a row, so a call that
depended on what an earlier one left behind would fail here."""

import math

import numpy as np
import pytest

from oracle import run as orun
from paper_2601_06340_gb300 import binding, inputs

from parity_util import TOL_FP64, band_errors

pytestmark = pytest.mark.gpu


def test_noalloc_march_matches_plan_march_on_two_calls(bpm_lib):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    wl = inputs.bragg_bent(nx=1024, nz=600, record_every=0)
    with binding.Plan(wl, binding.BPM_FP64_PLAIN) as plan:
        _, phasor = plan.slices()
        x = torch.from_numpy(wl.psi0).to(dev)
        ref = torch.empty_like(x)
        binding.bpm_propagate_device(plan.handle, x, ref, None, None, 0, wl.nz, st.cuda_stream)
        st.synchronize()
    ref = ref.cpu().numpy()

    # Inputs of the allocation-free call: propagators and coupling of Eq. fov10
    # from the FP64 plan constants, the strain phasor the plan prepared.
    p = orun.plans_for(wl)[0]
    d_prop = torch.from_numpy(np.stack([p.prop_plus, p.prop_minus])[None] / wl.nx).to(dev)
    d_ab = torch.from_numpy(np.array([[p.a, p.b]], dtype=np.complex128)).to(dev)
    d_ph = torch.from_numpy(np.ascontiguousarray(phasor)).to(dev)
    gph = math.fmod(p.dzh * p.c, 2 * math.pi)
    ang = math.fmod(wl.nz * gph, 2 * math.pi)
    g = complex(math.cos(ang), math.sin(ang))
    # A call of another size first (nx = 2048, two rows, random data): it
    # leaves different twiddles, row descriptors and scratch behind.
    rng = np.random.default_rng(3)
    nd, rd, sd = 2048, 2, 5

    def crand(*shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    dummy_psi = torch.from_numpy(crand(rd, 2, nd)).to(dev)
    dummy_prop = torch.from_numpy(np.exp(1j * rng.uniform(0, 6.28, (rd, 2, nd))) / nd).to(dev)
    dummy_ab = torch.from_numpy(0.5 * crand(rd, 2)).to(dev)
    dummy_ph = torch.from_numpy(np.exp(1j * rng.uniform(0, 6.28, (sd, nd)))).to(dev)
    binding.bpm_march_f64_noalloc(dummy_psi, nd, rd, dummy_prop, dummy_ab, dummy_ph, 0, sd,
                                  st.cuda_stream)
    st.synchronize()
    for _ in range(2):
        y = torch.from_numpy(wl.psi0.copy()).to(dev)
        binding.bpm_march_f64_noalloc(y, wl.nx, 1, d_prop, d_ab, d_ph, 0, wl.nz, st.cuda_stream)
        st.synchronize()
        got = y.cpu().numpy() * g
        errs = band_errors(got, ref)
        assert max(errs) <= TOL_FP64, errs


def test_noalloc_march_rejects_sizes_beyond_its_static_scratch(bpm_lib):
    dummy = 256
    with pytest.raises(binding.BpmError) as err:
        binding.bpm_march_f64_noalloc(dummy, 8192, 128, dummy, dummy, dummy, 0, 1)
    assert err.value.code == binding.BPM_ERR_INVALID
    assert "static scratch" in str(err.value)
    with pytest.raises(binding.BpmError):
        binding.bpm_march_f64_noalloc(dummy, 16384, 1, dummy, dummy, dummy, 0, 1)
