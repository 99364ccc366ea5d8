"""GPU parity: the CUDA paths (through the C ABI) against the FP64 oracle.

FP64 plain path: relative L2 per band <= 1e-10; fused FP32 path: <= 2e-4,
over the final fields and every record (see ``parity_util.band_errors``).
Masks are compared bit for bit (the decision is taken in FP64 with the same
operation order on both sides).
"""

import math

import numpy as np
import pytest

from oracle import bpm as obpm
from oracle import run as orun
from oracle import timeaxis
from paper_2601_06340_gb300 import binding, inputs

from parity_util import TOL_FP32, TOL_FP64, band_errors, run_gpu, run_ref

pytestmark = pytest.mark.gpu

FP64, FP32 = binding.BPM_FP64_PLAIN, binding.BPM_FP32_FUSED


def _reduced(name):
    if name == "laue_perfect":
        return inputs.laue_perfect(nx=512, nz=1000, record_every=90)
    if name == "bragg_bent":
        return inputs.bragg_bent(nx=1024, nz=2000, record_every=150)
    if name == "asym_dislocation":
        return inputs.asym_dislocation(nx=1024, nz=3000, record_every=250)
    if name == "pulse_batched":
        return inputs.pulse_batched(nx=512, nz=600, n_energy=8, record_every=70)
    raise KeyError(name)


CONFIGS = ["laue_perfect", "bragg_bent", "asym_dislocation", "pulse_batched"]


@pytest.fixture(scope="module")
def refs():
    return {name: (_reduced(name), run_ref(_reduced(name))) for name in CONFIGS}


@pytest.mark.parametrize("name", CONFIGS)
def test_fp64_plain_matches_oracle(bpm_lib, refs, name):
    wl, ref = refs[name]
    out = run_gpu(wl, FP64)
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= TOL_FP64, errs
    assert np.allclose(out.powers, ref.powers, rtol=1e-10, atol=0)


@pytest.mark.parametrize("name", CONFIGS)
def test_fp32_fused_matches_oracle(bpm_lib, refs, name):
    wl, ref = refs[name]
    out = run_gpu(wl, FP32)
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= TOL_FP32, errs
    assert np.allclose(out.powers, ref.powers, rtol=4e-4, atol=1e-12 * np.max(ref.powers))


@pytest.mark.parametrize("nx", [8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384])
def test_every_transform_size(bpm_lib, nx):
    """Random two-band input, masked strained bulk, 37 steps with a ragged
    record tail (37 = 3 * 12 + 1): exercises every radix decomposition."""
    rng = np.random.default_rng(nx)
    nz = 37
    wl = inputs.laue_perfect(nx=nx, nz=nz, dx_um=0.4, record_every=12)
    wl.psi0 = (rng.standard_normal((1, 2, nx)) + 1j * rng.standard_normal((1, 2, nx)))
    wl.crystal = dict(kind=inputs.CRYSTAL_MASK, mask=(rng.uniform(size=(nz, nx)) < 0.8))
    wl.strain = dict(kind=inputs.STRAIN_ARRAY, ux=rng.uniform(-1e-3, 1e-3, (nz, nx)))
    ref = run_ref(wl)
    out64 = run_gpu(wl, FP64)
    e64 = band_errors(out64.psi, ref.psi, out64.records, ref.records)
    assert max(e64) <= TOL_FP64, e64
    out32 = run_gpu(wl, FP32)
    e32 = band_errors(out32.psi, ref.psi, out32.records, ref.records)
    assert max(e32) <= 2e-6, e32


@pytest.mark.parametrize("name", ["laue_perfect", "bragg_bent", "asym_dislocation"])
def test_mask_is_bit_exact(bpm_lib, name):
    wl = _reduced(name)
    for prec in (FP32, FP64):
        with binding.Plan(wl, prec) as plan:
            mask, ph = plan.slices()
        ref = orun.mask_of(wl)
        assert np.array_equal(mask.astype(bool), ref)


def test_strain_phasor_fp64(bpm_lib):
    wl = _reduced("asym_dislocation")
    with binding.Plan(wl, FP64) as plan:
        mask, ph = plan.slices()
    cr = orun.crystal_for(wl)
    for n in range(0, wl.nz, 97):
        inside, theta = cr(n)
        ref = np.where(inside, np.exp(1j * theta), 0)
        assert np.max(np.abs(ph[n] - ref)) < 1e-12


@pytest.mark.parametrize("name", ["bragg_bent", "asym_dislocation"])
def test_strain_phasor_fp32(bpm_lib, name):
    """FP32 plans: the unit phasor of every inside cell to FP32 accuracy (the
    bent phase reaches hundreds of radians, so this also checks its FP64
    reduction), zero outside."""
    wl = _reduced(name)
    with binding.Plan(wl, FP32) as plan:
        mask, ph = plan.slices()
    cr = orun.crystal_for(wl)
    for n in range(0, wl.nz, 61):
        inside, theta = cr(n)
        ref = np.where(inside, np.exp(1j * theta), 0)
        assert np.max(np.abs(ph[n] - ref)) < 4e-6, n


def test_split_band_slices_fp32(bpm_lib):
    """Mask and phasor of FP32 plans at N = 8192 and 16384 (stored per part
    on the device) against the oracle, in natural order."""
    rng = np.random.default_rng(33)
    for nx in (8192, 16384):
        for _ in range(2):
            wl = inputs.serving_request(rng, nx, 200)
            with binding.Plan(wl, FP32) as plan:
                mask, ph = plan.slices()
            assert np.array_equal(mask.astype(bool), orun.mask_of(wl))
            cr = orun.crystal_for(wl)
            for n in range(0, wl.nz, 37):
                inside, theta = cr(n)
                ref = np.where(inside, np.exp(1j * theta), 0)
                assert np.max(np.abs(ph[n] - ref)) < 4e-6, (nx, n)


def _check_full(out, ref, tol):
    """Bound both readings: every record plus the final field, and the final
    field alone (the stricter one when a band has decayed)."""
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    final = band_errors(out.psi, ref.psi)
    assert max(errs) <= tol and max(final) <= tol, (errs, final)


def test_full_size_laue_perfect(bpm_lib):
    wl = inputs.laue_perfect()
    ref = run_ref(wl)
    for prec, tol in ((FP64, TOL_FP64), (FP32, TOL_FP32)):
        _check_full(run_gpu(wl, prec), ref, tol)


def test_full_size_bragg_bent(bpm_lib):
    wl = inputs.bragg_bent()
    ref = run_ref(wl)
    for prec, tol in ((FP64, TOL_FP64), (FP32, TOL_FP32)):
        _check_full(run_gpu(wl, prec), ref, tol)


def test_full_size_asym_dislocation_fp32(bpm_lib):
    wl = inputs.asym_dislocation()
    with binding.Plan(wl, FP32) as plan:
        mask, _ = plan.slices()
        out = plan.propagate()
    assert np.array_equal(mask.astype(bool), orun.mask_of(wl))
    ref = run_ref(wl)
    _check_full(out, ref, TOL_FP32)


def test_full_size_pulse_batched_sampled_rows(bpm_lib):
    """All 256 energies on the GPU in one launch; the oracle checks rows 0,
    131 and 255 one by one."""
    wl = inputs.pulse_batched()
    out = run_gpu(wl, FP32)
    rows = [0, 131, 255]
    ref = run_ref(wl, rows=rows)
    errs = band_errors(out.psi[rows], ref.psi)
    assert max(errs) <= TOL_FP32, errs


def test_resume_split_equals_unsplit(bpm_lib):
    wl = _reduced("bragg_bent")
    for prec, tol in ((FP64, 1e-12), (FP32, 1e-5)):
        with binding.Plan(wl, prec) as plan:
            full = plan.propagate()
            first = plan.propagate(n_end=700)
            rec = first.records.copy()
            pw = first.powers.copy()
            second = plan.propagate(first.psi, n_begin=700,
                                    out=binding.MarchOutput(np.empty_like(first.psi), rec, pw))
        e = band_errors(second.psi, full.psi, second.records, full.records)
        assert max(e) <= tol, (prec, e)


def test_repeat_runs_are_bitwise_equal(bpm_lib):
    wl = _reduced("asym_dislocation")
    for prec in (FP32, FP64):
        with binding.Plan(wl, prec) as plan:
            a = plan.propagate()
            b = plan.propagate()
        assert np.array_equal(a.psi, b.psi) and np.array_equal(a.records, b.records)
        assert np.array_equal(a.powers, b.powers)


def test_batch_rows_are_independent(bpm_lib):
    """A row's result does not depend on the rows launched beside it."""
    wl = inputs.pulse_batched(nx=256, nz=300, n_energy=12)
    full = run_gpu(wl, FP32)
    for r in (0, 5, 11):
        one = inputs.pulse_batched(nx=256, nz=300, n_energy=12)
        one.energies_ev = one.energies_ev[r:r + 1]
        one.psi0 = one.psi0[r:r + 1]
        single = run_gpu(one, FP32)
        assert np.array_equal(single.psi[0], full.psi[r])


def test_edge_cases(bpm_lib):
    # one step, records coarser than the march, smallest grid
    wl = inputs.laue_perfect(nx=8, nz=1, dx_um=0.4, record_every=5)
    ref = run_ref(wl)
    for prec in (FP32, FP64):
        out = run_gpu(wl, prec)
        assert out.records.shape[1] == 0
        assert max(band_errors(out.psi, ref.psi)) <= 1e-6
    # record on every step
    wl = inputs.bragg_bent(nx=256, nz=50, record_every=1)
    ref = run_ref(wl)
    out = run_gpu(wl, FP32)
    assert max(band_errors(out.psi, ref.psi, out.records, ref.records)) <= 1e-5
    # vacuum: fields only propagate; zero input stays zero
    wl = inputs.laue_perfect(nx=128, nz=20)
    wl.crystal = dict(kind=inputs.CRYSTAL_VACUUM)
    wl.psi0 = np.zeros_like(wl.psi0)
    out = run_gpu(wl, FP32)
    assert np.all(out.psi == 0)


def test_device_api_with_torch_tensors(bpm_lib):
    torch = pytest.importorskip("torch")
    wl = _reduced("bragg_bent")
    ref = run_gpu(wl, FP32)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(wl.psi0.astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    with binding.Plan(wl, FP32) as plan:
        rec = torch.zeros((1, plan.n_rec, 2, wl.nx), dtype=torch.complex64, device=dev)
        pw = torch.zeros((1, plan.n_rec + 1, 2), dtype=torch.float64, device=dev)
        st = torch.cuda.current_stream()
        binding.bpm_propagate_device(plan.handle, x, y, rec, pw, 0, wl.nz, st.cuda_stream)
        # no bounded device wait expired in the march
        assert binding.bpm_device_status(plan.handle, st.cuda_stream) == binding.BPM_OK
        st.synchronize()
    assert np.array_equal(y.cpu().numpy().astype(np.complex128), ref.psi.astype(np.complex64))
    assert np.array_equal(rec.cpu().numpy(), ref.records)


def _capture_case(name):
    rng = np.random.default_rng(8)
    if name == "cluster N=1024":
        return inputs.serving_request(rng, 1024, 300), binding.BPM_SPLIT_FIRST_ORDER
    if name == "split N=4096":
        return inputs.serving_request(rng, 4096, 300), binding.BPM_SPLIT_FIRST_ORDER
    if name == "rotated batch 160x4096":
        return (inputs.pulse_batched(nx=4096, nz=300, n_energy=160, record_every=100),
                binding.BPM_SPLIT_FIRST_ORDER)
    if name == "Verlet N=1024":
        return inputs.serving_request(rng, 1024, 300), binding.BPM_SPLIT_VERLET
    if name == "Verlet N=4096":
        return inputs.serving_request(rng, 4096, 300), binding.BPM_SPLIT_VERLET
    if name == "Forest-Ruth N=1024":
        return inputs.serving_request(rng, 1024, 200), binding.BPM_SPLIT_FOREST_RUTH
    if name == "Forest-Ruth N=4096":
        return inputs.serving_request(rng, 4096, 200), binding.BPM_SPLIT_FOREST_RUTH
    if name == "Forest-Ruth N=8192":
        return inputs.serving_request(rng, 8192, 200), binding.BPM_SPLIT_FOREST_RUTH
    return (inputs.cube_dislocation_3d(nx=256, ny=256, nz=40, dx_um=0.08, dy_um=0.08,
                                       dz_um=0.1, cube_um=5.0, fwhm_um=1.5, record_every=10),
            binding.BPM_SPLIT_VERLET if name.endswith("Verlet") else binding.BPM_SPLIT_FIRST_ORDER)


@pytest.mark.parametrize("name", ["cluster N=1024", "split N=4096", "rotated batch 160x4096",
                                  "Verlet N=1024", "Verlet N=4096", "Forest-Ruth N=1024",
                                  "Forest-Ruth N=4096",
                                  "Forest-Ruth N=8192", "3D 256x256", "3D 256x256 Verlet"])
def test_device_api_graph_capture_replays(bpm_lib, monkeypatch, name):
    """A device-API march captured into a CUDA graph (its per-call uploads go
    through kernel parameters) replays to the same bits as the march run
    directly, twice in a row."""
    torch = pytest.importorskip("torch")
    monkeypatch.setenv("BPM_AUTOTUNE", "0")   # both marches take the fixed rule's shape
    wl, split = _capture_case(name)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(wl.psi0.astype(np.complex64)).to(dev)
    with binding.Plan(wl, FP32, splitting=split) as plan:
        shape_rec = (wl.batch, plan.n_rec) + tuple(wl.psi0.shape[1:])
        outs = [(torch.empty_like(x), torch.zeros(shape_rec, dtype=torch.complex64, device=dev),
                 torch.zeros((wl.batch, plan.n_rec + 1, 2), dtype=torch.float64, device=dev))
                for _ in range(2)]
        s = torch.cuda.Stream()
        y, rec, pw = outs[0]
        binding.bpm_propagate_device(plan.handle, x, y, rec, pw, 0, wl.nz, s.cuda_stream)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        y2, rec2, pw2 = outs[1]
        with torch.cuda.graph(g, stream=s):
            binding.bpm_propagate_device(plan.handle, x, y2, rec2, pw2, 0, wl.nz, s.cuda_stream)
        for _ in range(2):
            y2.zero_()
            rec2.zero_()
            pw2.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(y2, y) and torch.equal(rec2, rec) and torch.equal(pw2, pw)
        assert binding.bpm_device_status(plan.handle, s.cuda_stream) == binding.BPM_OK
        del g
    assert torch.isfinite(torch.view_as_real(y)).all() and y.abs().max() > 0


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_device_api_capture_refusals(bpm_lib):
    """What cannot be captured is refused before anything is enqueued: FP64
    plans, and plans whose strain slices are not prepared yet."""
    torch = pytest.importorskip("torch")
    wl = _reduced("laue_perfect")
    dev = torch.device("cuda:0")
    for precision, dtype in ((FP64, torch.complex128), (FP32, torch.complex64)):
        x = torch.from_numpy(wl.psi0.astype(np.complex128)).to(dev).to(dtype)
        y = torch.empty_like(x)
        with binding.Plan(wl, precision) as plan:   # never marched: slices not prepared
            s = torch.cuda.Stream()
            g = torch.cuda.CUDAGraph()
            with pytest.raises(binding.BpmError) as e:
                with torch.cuda.graph(g, stream=s):
                    binding.bpm_propagate_device(plan.handle, x, y, None, None, 0, wl.nz,
                                                 s.cuda_stream)
            assert e.value.code == binding.BPM_ERR_INVALID
            torch.cuda.synchronize()
            # the plan still marches outside a capture
            binding.bpm_propagate_device(plan.handle, x, y, None, None, 0, wl.nz,
                                         torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
        ref = run_gpu(wl, precision)
        got = y.cpu().numpy().astype(np.complex128)
        assert np.array_equal(got, ref.psi if precision == FP64 else
                              ref.psi.astype(np.complex64).astype(np.complex128))


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_staged_forest_ruth_capture_refused(bpm_lib):
    """A Forest-Ruth plan that marches stage by stage (N = 16384) is refused
    under capture before anything is enqueued, and still marches outside."""
    torch = pytest.importorskip("torch")
    wl = inputs.serving_request(np.random.default_rng(3), 16384, 20)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(wl.psi0.astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    with binding.Plan(wl, FP32, splitting=binding.BPM_SPLIT_FOREST_RUTH) as plan:
        s = torch.cuda.Stream()
        binding.bpm_propagate_device(plan.handle, x, y, None, None, 0, wl.nz, s.cuda_stream)
        s.synchronize()
        assert binding.bpm_launch_shape(plan.handle)[0] == 7
        first = y.clone()
        g = torch.cuda.CUDAGraph()
        with pytest.raises(binding.BpmError) as e:
            with torch.cuda.graph(g, stream=s):
                binding.bpm_propagate_device(plan.handle, x, y, None, None, 0, wl.nz,
                                             s.cuda_stream)
        assert e.value.code == binding.BPM_ERR_INVALID
        torch.cuda.synchronize()
        binding.bpm_propagate_device(plan.handle, x, y, None, None, 0, wl.nz,
                                     torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(y, first)


def test_omega_to_t_matches_oracle(bpm_lib):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    nb, nx = 64, 48
    f = rng.standard_normal((nb, 2, nx)) + 1j * rng.standard_normal((nb, 2, nx))
    ref = timeaxis.omega_to_t(f)
    dev = torch.device("cuda:0")
    for prec, dt, tol in ((FP64, torch.complex128, 1e-13), (FP32, torch.complex64, 3e-6)):
        x = torch.from_numpy(f.astype(np.complex128)).to(dtype=dt, device=dev).contiguous()
        y = torch.empty((2, nx, nb), dtype=dt, device=dev)
        binding.bpm_omega_to_t_device(x, y, nb, nx, prec, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_rotated_schedule_matches_single_launch(bpm_lib):
    """200 rows of N=4096 exceed what one launch keeps resident: the march is
    split into (row, chunk) launches (64-step chunks plus a 36-step
    remainder round).  Rows must come out bit-identical to a batch small
    enough for one launch, and match the oracle."""
    big = inputs.pulse_batched(nx=4096, nz=100, n_energy=200)
    small = inputs.pulse_batched(nx=4096, nz=100, n_energy=200)
    small.energies_ev = small.energies_ev[:100]
    small.psi0 = small.psi0[:100]
    out_big = run_gpu(big, FP32)
    out_small = run_gpu(small, FP32)
    assert np.array_equal(out_big.psi[:100], out_small.psi)
    rows = [3, 150, 199]
    ref = run_ref(big, rows=rows)
    assert max(band_errors(out_big.psi[rows], ref.psi)) <= 2e-5


def test_split_band_sizes_against_oracle(bpm_lib):
    """N = 8192 and 16384 run as bands split over 2 and 4 CTAs per band:
    a few hundred steps of a dislocated asymmetric Bragg request against the
    oracle, the strain stream fetched back in natural order."""
    rng = np.random.default_rng(21)
    for nx in (8192, 16384):
        wl = inputs.serving_request(rng, nx, 300)
        wl.record_every = 100
        ref = run_ref(wl)
        for prec, tol in ((FP32, 2e-5), (FP64, TOL_FP64)):
            with binding.Plan(wl, prec) as plan:
                mask, _ = plan.slices()
                out = plan.propagate()
            assert np.array_equal(mask.astype(bool), orun.mask_of(wl))
            errs = band_errors(out.psi, ref.psi, out.records, ref.records)
            assert max(errs) <= tol, (nx, prec, errs)
