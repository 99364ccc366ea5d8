"""ctypes binding of the C ABI declared in include/bpm.h.

The module-level functions carry the C names (``bpm_plan``,
``bpm_set_crystal``, ...) and only marshal arguments: numpy arrays become
pointers, torch tensors pass ``data_ptr()`` and their stream handle.  Every
step of the march runs in the CUDA library; if the library is missing this
module raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbpm.so")

BPM_OK, BPM_NOT_READY = 0, 1
BPM_ERR_INVALID, BPM_ERR_OOM, BPM_ERR_CUDA = -1, -2, -3
BPM_ERR_BUSY, BPM_ERR_TIMEOUT, BPM_ERR_NUMERIC = -4, -5, -6
BPM_FP64_PLAIN, BPM_FP32_FUSED = 0, 1
BPM_CRYSTAL_BOX = 6
BPM_SPLIT_FIRST_ORDER, BPM_SPLIT_VERLET, BPM_SPLIT_FOREST_RUTH = 0, 1, 2

_STATUS_NAMES = {0: "OK", 1: "NOT_READY", -1: "ERR_INVALID", -2: "ERR_OOM",
                 -3: "ERR_CUDA", -4: "ERR_BUSY", -5: "ERR_TIMEOUT", -6: "ERR_NUMERIC"}


class BpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class bpm_problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dx_um", ctypes.c_double), ("dz_um", ctypes.c_double), ("x0_um", ctypes.c_double),
        ("n_energy", ctypes.c_int32), ("energy_ev", ctypes.POINTER(ctypes.c_double)),
        ("e_ref_ev", ctypes.c_double), ("theta_b_ref_rad", ctypes.c_double),
        ("chi0_re", ctypes.c_double), ("chi0_im", ctypes.c_double),
        ("chih_re", ctypes.c_double), ("chih_im", ctypes.c_double),
        ("record_every", ctypes.c_int32), ("precision", ctypes.c_int32),
    ]


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int32
_D = ctypes.c_double
_SIGS = {
    "bpm_plan": ([ctypes.POINTER(bpm_problem), ctypes.POINTER(_P)], ctypes.c_int),
    "bpm_plan3d": ([ctypes.POINTER(bpm_problem), _I, _D, _D, ctypes.POINTER(_P)], ctypes.c_int),
    "bpm_set_crystal_box": ([_P, _P], ctypes.c_int),
    "bpm_set_splitting": ([_P, _I], ctypes.c_int),
    "bpm_set_crystal": ([_P, _I, _D, _D, _D, _D, _P, _P, _I], ctypes.c_int),
    "bpm_set_strain": ([_P, _I, _P, _P, _I], ctypes.c_int),
    "bpm_propagate": ([_P, _P, _P, _P, _P, _I, _I], ctypes.c_int),
    "bpm_propagate_device": ([_P, _P, _P, _P, _P, _I, _I, _P], ctypes.c_int),
    "bpm_omega_to_t_device": ([_P, _P, _I, _I, _I, _P], ctypes.c_int),
    "bpm_submit": ([_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "bpm_poll": ([ctypes.c_uint64, _I], ctypes.c_int),
    "bpm_server_configure": ([_D, _I, _I, _I], ctypes.c_int),
    "bpm_ticket_times": ([ctypes.c_uint64, ctypes.POINTER(_D), ctypes.POINTER(_D),
                          ctypes.POINTER(_D)], ctypes.c_int),
    "bpm_fetch_slices": ([_P, _P, _P], ctypes.c_int),
    "bpm_march_f64_noalloc": ([_P, _I, _I, _P, _P, _P, _I, _I, _P], ctypes.c_int),
    "bpm_launch_shape": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I)], ctypes.c_int),
    "bpm_slice_form": ([_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "bpm_destroy": ([_P], ctypes.c_int),
    "bpm_last_error": ([], ctypes.c_char_p),
    "bpm_version": ([], ctypes.c_char_p),
    "bpm_selftest_wait_expiry": ([ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "bpm_server_inject_launch_failure": ([_I, _I], ctypes.c_int),
    "bpm_device_status": ([_P, _P], ctypes.c_int),
    "bpm_fp_peak": ([_I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)], ctypes.c_int),
}


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(code: int) -> int:
    if code < 0:
        raise BpmError(code, load().bpm_last_error().decode())
    return code


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return int(a)


# ---- C names, marshalling only -------------------------------------------

def bpm_plan(problem: bpm_problem) -> int:
    h = ctypes.c_void_p()
    _check(load().bpm_plan(ctypes.byref(problem), ctypes.byref(h)))
    return h.value


def bpm_plan3d(problem: bpm_problem, ny: int, dy_um: float, y0_um: float) -> int:
    h = ctypes.c_void_p()
    _check(load().bpm_plan3d(ctypes.byref(problem), int(ny), float(dy_um), float(y0_um),
                             ctypes.byref(h)))
    return h.value


def bpm_set_splitting(plan, method: int):
    return _check(load().bpm_set_splitting(plan, int(method)))


def bpm_set_crystal_box(plan, box_um):
    b = np.ascontiguousarray(box_um, dtype=np.float64)
    assert b.size == 6
    return _check(load().bpm_set_crystal_box(plan, _ptr(b)))


def bpm_set_crystal(plan, kind, asym_angle_rad=0.0, thickness_um=0.0, surf_x_um=0.0,
                    surf_z_um=0.0, mask=None, poly_xz_um=None):
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    p = None if poly_xz_um is None else np.ascontiguousarray(poly_xz_um, dtype=np.float64)
    nv = 0 if p is None else p.size // 2
    return _check(load().bpm_set_crystal(plan, int(kind), float(asym_angle_rad),
                                         float(thickness_um), float(surf_x_um),
                                         float(surf_z_um), _ptr(m), _ptr(p), nv))


def bpm_set_strain(plan, kind, ux_um=None, params=None):
    u = None if ux_um is None else np.ascontiguousarray(ux_um, dtype=np.float64)
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    return _check(load().bpm_set_strain(plan, int(kind), _ptr(u), _ptr(p),
                                        0 if p is None else p.size))


def bpm_propagate(plan, psi_in, psi_out, records, powers, n_begin, n_end):
    return _check(load().bpm_propagate(plan, _ptr(psi_in), _ptr(psi_out), _ptr(records),
                                       _ptr(powers), int(n_begin), int(n_end)))


def bpm_propagate_device(plan, d_psi_in, d_psi_out, d_records, d_powers, n_begin, n_end,
                         stream=None):
    return _check(load().bpm_propagate_device(plan, _ptr(d_psi_in), _ptr(d_psi_out),
                                              _ptr(d_records), _ptr(d_powers), int(n_begin),
                                              int(n_end), stream))


def bpm_omega_to_t_device(d_in, d_out, n_energy, nx, precision, stream=None):
    return _check(load().bpm_omega_to_t_device(_ptr(d_in), _ptr(d_out), int(n_energy),
                                               int(nx), int(precision), stream))


def bpm_submit(plan, psi_in, psi_out, records=None, powers=None) -> int:
    t = ctypes.c_uint64()
    _check(load().bpm_submit(plan, _ptr(psi_in), _ptr(psi_out), _ptr(records), _ptr(powers),
                             ctypes.byref(t)))
    return t.value


def bpm_poll(ticket, timeout_ms=0) -> int:
    return _check(load().bpm_poll(ctypes.c_uint64(ticket), int(timeout_ms)))


def bpm_server_configure(mem_fraction=0.0, max_active=0, epoch_steps=0, max_queue=0):
    return _check(load().bpm_server_configure(float(mem_fraction), int(max_active),
                                              int(epoch_steps), int(max_queue)))


def bpm_device_status(plan, stream=None) -> int:
    """BPM_OK, or raises BpmError (BPM_ERR_TIMEOUT) if a bounded device wait
    expired in the plan's device marches enqueued on `stream` so far."""
    return _check(load().bpm_device_status(plan, stream))


def bpm_server_inject_launch_failure(nx: int, count: int):
    """Test hook: the next `count` FP32 batch launches of size nx fail on the
    host with BPM_ERR_CUDA (0 clears it)."""
    return _check(load().bpm_server_inject_launch_failure(int(nx), int(count)))


def bpm_ticket_times(ticket):
    a, b, c = _D(), _D(), _D()
    _check(load().bpm_ticket_times(ctypes.c_uint64(ticket), ctypes.byref(a), ctypes.byref(b),
                                   ctypes.byref(c)))
    return a.value, b.value, c.value


def bpm_fetch_slices(plan, mask=None, phasor=None):
    return _check(load().bpm_fetch_slices(plan, _ptr(mask), _ptr(phasor)))


def bpm_march_f64_noalloc(d_psi, nx, n_rows, d_prop, d_coupling, d_phasor, n_begin, n_end,
                          stream=None):
    return _check(load().bpm_march_f64_noalloc(_ptr(d_psi), int(nx), int(n_rows), _ptr(d_prop),
                                                _ptr(d_coupling), _ptr(d_phasor), int(n_begin),
                                                int(n_end), stream))


def bpm_launch_shape(plan) -> tuple[int, int]:
    """(layout, chunk) of the plan's last FP32 march: layout 10 the
    Forest-Ruth step on a two-CTA cluster per row (N = 512-4096), 9 the
    Forest-Ruth step on the N = 4096 half-band split or the N = 8192 split
    band, 8 the 16-point form of the N = 4096 split (forced), 7 the
    Forest-Ruth step stage by stage (N = 16384; N = 8192 forced), 6 the
    Forest-Ruth step on one CTA per row; layouts 5, 4, 3 the Verlet step on
    a split-band cluster (N = 4096, 8192, 16384), a two-CTA cluster or one
    CTA per row; 2 four-CTA cluster per row (N = 4096 half-band
    split), 1 two-CTA cluster per row, 0 CTA per row, -1 the fixed rule;
    chunk 0 for one launch."""
    layout, chunk = _I(0), _I(0)
    _check(load().bpm_launch_shape(plan, ctypes.byref(layout), ctypes.byref(chunk)))
    return layout.value, chunk.value


def bpm_slice_form(plan) -> tuple[int, int]:
    """(form, bytes) of the plan's prepared slices: form 1 separable (one
    row per z-step and one phasor per column; the kernels form each cell),
    0 the per-cell stream, -1 not prepared yet; bytes of device memory."""
    form, nbytes = _I(0), ctypes.c_int64(0)
    _check(load().bpm_slice_form(plan, ctypes.byref(form), ctypes.byref(nbytes)))
    return form.value, nbytes.value


def bpm_selftest_wait_expiry() -> tuple[int, float]:
    """(status word, seconds) of the bounded-wait self-test kernel: status 1
    means the wait gave up and the kernel returned."""
    status, seconds = _I(0), ctypes.c_double(0.0)
    _check(load().bpm_selftest_wait_expiry(ctypes.byref(status), ctypes.byref(seconds)))
    return status.value, seconds.value


BPM_PEAK_FP64_DFMA, BPM_PEAK_FP32_FFMA, BPM_PEAK_FP32_FFMA2 = 0, 1, 2


def bpm_fp_peak(kind: int, iters: int) -> tuple[float, float]:
    """(flops/s, seconds) of the FMA-throughput kernel of `kind` on the
    current device (one FMA = 2 flops, a packed FFMA2 = 4)."""
    rate, sec = _D(0.0), _D(0.0)
    _check(load().bpm_fp_peak(int(kind), int(iters), ctypes.byref(rate), ctypes.byref(sec)))
    return rate.value, sec.value


def bpm_destroy(plan):
    return _check(load().bpm_destroy(plan))


def bpm_last_error() -> str:
    return load().bpm_last_error().decode()


def bpm_version() -> str:
    return load().bpm_version().decode()


# ---- convenience wrapper over the same calls -------------------------------

@dataclass
class MarchOutput:
    psi: np.ndarray        # [B][2][N] complex128
    records: np.ndarray    # [B][n_rec][2][N] complex64 (FP32) / complex128 (FP64)
    powers: np.ndarray     # [B][n_rec+1][2]


class Plan:
    """Owns one bpm plan built from a workload (see ``inputs.Workload``)."""

    def __init__(self, wl, precision: int = BPM_FP32_FUSED, record_every: int | None = None,
                 splitting: int = BPM_SPLIT_FIRST_ORDER):
        self.wl = wl
        self.precision = precision
        self.record_every = wl.record_every if record_every is None else record_every
        self._energies = np.ascontiguousarray(wl.energies_ev, dtype=np.float64)
        prob = bpm_problem(
            nx=wl.nx, nz=wl.nz, dx_um=wl.dx_um, dz_um=wl.dz_um, x0_um=wl.x0_um,
            n_energy=len(self._energies),
            energy_ev=self._energies.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            e_ref_ev=wl.e_ref_ev, theta_b_ref_rad=wl.theta_b_ref_rad,
            chi0_re=wl.chi0.real, chi0_im=wl.chi0.imag, chih_re=wl.chih.real,
            chih_im=wl.chih.imag, record_every=self.record_every, precision=precision)
        self.ny = int(getattr(wl, "ny", 1))
        if self.ny > 1:
            self.handle = bpm_plan3d(prob, self.ny, wl.dy_um, wl.y0_um)
        else:
            self.handle = bpm_plan(prob)
        c = dict(wl.crystal)
        kind = c.pop("kind")
        if kind == BPM_CRYSTAL_BOX:
            bpm_set_crystal_box(self.handle, c["box_um"])
        else:
            bpm_set_crystal(self.handle, kind, c.get("asym_angle_rad", 0.0),
                            c.get("thickness_um", 0.0), c.get("surf_x_um", 0.0),
                            c.get("surf_z_um", 0.0), c.get("mask"), c.get("polygon"))
        st = dict(wl.strain)
        bpm_set_strain(self.handle, st.pop("kind"), st.get("ux"), st.get("params"))
        if splitting != BPM_SPLIT_FIRST_ORDER:
            bpm_set_splitting(self.handle, splitting)
        self.n_rec = (wl.nz // self.record_every) if self.record_every > 0 else 0

    @property
    def rec_dtype(self):
        return np.complex64 if self.precision == BPM_FP32_FUSED else np.complex128

    def propagate(self, psi_in=None, n_begin=0, n_end=None, records=True, powers=True,
                  out: MarchOutput | None = None) -> MarchOutput:
        wl = self.wl
        psi_in = np.ascontiguousarray(wl.psi0 if psi_in is None else psi_in,
                                      dtype=np.complex128)
        n_end = wl.nz if n_end is None else n_end
        if out is None:
            out = MarchOutput(np.empty_like(psi_in),
                              np.zeros((wl.batch, self.n_rec) + psi_in.shape[1:], self.rec_dtype),
                              np.zeros((wl.batch, self.n_rec + 1, 2)))
        bpm_propagate(self.handle, psi_in, out.psi, out.records if records else None,
                      out.powers if powers else None, n_begin, n_end)
        return out

    def slices(self):
        shape = (self.wl.nz, self.ny, self.wl.nx) if self.ny > 1 else (self.wl.nz, self.wl.nx)
        mask = np.zeros(shape, np.uint8)
        ph = np.zeros(shape, np.complex128)
        bpm_fetch_slices(self.handle, mask, ph)
        return mask, ph

    def close(self):
        if self.handle:
            bpm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
