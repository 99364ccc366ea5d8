"""Oracle: the two-beam FFT-BPM z-march with both transverse coordinates.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. fov4 is written for psi(x^, y^, z^) with the angular-spectrum operator
exp(i dz^ sqrt(1 - kx^2 - ky^2)).  The two-beam envelopes of Eqs. fov6-fov10
carry the Bragg shift k_d/2 along x only (k_d is parallel to x^, Sec. 2), so
with both transverse coordinates:

* each band's propagator is exp(i dz^ sqrt(1 - (qx +- s)^2 - qy^2)), written
  as g * exp(i dz^ delta_+-) with g = exp(i dz^ cos(alpha)) and
  delta_+-(qx, qy) = sqrt(1 - (qx +- s)^2 - qy^2) - cos(alpha)
                   = -(qx (qx +- 2 s) + qy^2) / (sqrt(1 - (qx +- s)^2 - qy^2) + cos(alpha));
* the coupling of Eq. fov10 (Eqs. fov11, fov12, Authier) is unchanged and
  pointwise in (x, y), with Pi(x, y, z) and u_x(x, y, z);
* band powers are dx dy sum |psi|^2.

The paper says the generalisation from (x, z) is straightforward (Sec. 2)
and runs 3D cases (Sec. 7).  Readings: the 2D DFT over (y, x) (the oracle's own, ``oracle.fft``);
qx = 2 pi fftfreq(Nx, dx^), qy = 2 pi fftfreq(Ny, dy^); cells at
(x_j, y_i, z_n) = (x0 + j dx, y0 + i dy, n dz); the 2D crystal kinds and
strain fields apply at every y; a box crystal {x0 <= x <= x1, y0 <= y <= y1,
z0 <= z <= z1} and [nz][ny][nx] mask / u_x arrays cover the rest.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import bpm, geometry
from . import fft as dft

CRYSTAL_BOX = 6


@dataclass
class Plan3D:
    base: bpm.EnergyPlan      # scalars (k, s, c, dz^, a, b, g) of the energy
    dyh: float                # dy^ = k dy
    qx: np.ndarray            # [Nx]
    qy: np.ndarray            # [Ny]
    prop_plus: np.ndarray     # [Ny][Nx] exp(i dz^ delta_+(qx, qy))
    prop_minus: np.ndarray    # [Ny][Nx] exp(i dz^ delta_-(qx, qy))
    delta_plus: np.ndarray    # [Ny][Nx] delta_+(qx, qy) (fractional steps of Eq. split-op)
    delta_minus: np.ndarray   # [Ny][Nx] delta_-(qx, qy)


def energy_plan3d(energy_ev: float, e_ref_ev: float, theta_b_ref_rad: float,
                  chi0: complex, chih: complex, nx: int, ny: int, dx_um: float,
                  dy_um: float, dz_um: float) -> Plan3D:
    base = bpm.energy_plan(energy_ev, e_ref_ev, theta_b_ref_rad, chi0, chih, nx, dx_um, dz_um)
    s, c, dzh = base.s, base.c, base.dzh
    dyh = base.k_um * dy_um
    qx = 2.0 * math.pi * dft.fftfreq(nx, base.dxh)
    qy = 2.0 * math.pi * dft.fftfreq(ny, dyh)
    QX, QY = np.meshgrid(qx, qy)          # [Ny][Nx]
    props, deltas = [], []
    for sign in (+1.0, -1.0):
        root = np.sqrt(1.0 - (QX + sign * s) ** 2 - QY ** 2)
        delta = -(QX * (QX + sign * 2.0 * s) + QY ** 2) / (root + c)
        deltas.append(delta)
        props.append(np.exp(1j * dzh * delta))
    return Plan3D(base, dyh, qx, qy, props[0], props[1], deltas[0], deltas[1])


class Crystal3D:
    """Slice provider n -> (Pi[n][:, :], h*u_x[n][:, :]) on the (y, x) grid."""

    def __init__(self, nx: int, ny: int, x0_um: float, y0_um: float, dx_um: float,
                 dy_um: float, dz_um: float, d_spacing_um: float):
        self.nx, self.ny = nx, ny
        self.dz_um = dz_um
        self.x = geometry.grid_x(nx, x0_um, dx_um)
        self.y = y0_um + np.arange(ny, dtype=np.float64) * dy_um
        self.h = 2.0 * math.pi / d_spacing_um
        self.plane = geometry.Crystal(nx, x0_um, dx_um, dz_um, d_spacing_um)
        self.kind = geometry.CRYSTAL_VACUUM
        self.box = None
        self.mask3 = None
        self.ux3 = None

    def set_crystal(self, kind: int, box=None, mask3=None, **plane_args):
        """2D kinds (geometry.Crystal arguments) hold at every y; CRYSTAL_BOX
        takes box = (x0, x1, y0, y1, z0, z1) in um; CRYSTAL_MASK takes a
        [nz][ny][nx] array."""
        self.kind = kind
        if kind == CRYSTAL_BOX:
            self.box = tuple(float(v) for v in box)
        elif kind == geometry.CRYSTAL_MASK:
            self.mask3 = np.asarray(mask3) != 0
        else:
            self.plane.set_crystal(kind, **plane_args)
        return self

    def set_strain(self, kind: int, ux3=None, params=None):
        self.strain_kind = kind
        if kind == geometry.STRAIN_ARRAY:
            self.ux3 = np.asarray(ux3, dtype=np.float64)
        else:
            self.plane.set_strain(kind, params=params)
        return self

    def inside(self, n: int) -> np.ndarray:
        if self.kind == CRYSTAL_BOX:
            x0, x1, y0, y1, z0, z1 = self.box
            z = geometry.grid_z(n, self.dz_um)
            if not (z0 <= z <= z1):
                return np.zeros((self.ny, self.nx), dtype=bool)
            return ((self.y[:, None] >= y0) & (self.y[:, None] <= y1)
                    & (self.x[None, :] >= x0) & (self.x[None, :] <= x1))
        if self.kind == geometry.CRYSTAL_MASK:
            return self.mask3[n].copy()
        return np.broadcast_to(self.plane.inside(n), (self.ny, self.nx)).copy()

    def theta(self, n: int) -> np.ndarray:
        if getattr(self, "strain_kind", geometry.STRAIN_NONE) == geometry.STRAIN_ARRAY:
            return self.h * self.ux3[n]
        return np.broadcast_to(self.plane.theta(n), (self.ny, self.nx)).copy()

    def __call__(self, n: int):
        return self.inside(n), self.theta(n)


def march3d(plans: list[Plan3D], psi0: np.ndarray, slices, n_begin: int, n_end: int,
            record_every: int, dx_um: float, dy_um: float, method: str = "first_order",
            chi: tuple[complex, complex] | None = None) -> bpm.MarchResult:
    """Eq. fov10 on [B][2][Ny][Nx] fields: each envelope through its own 2D
    angular-spectrum operator, then the pointwise two-beam coupling.
    Records / powers as in ``bpm.march`` (powers = dx dy sum |psi|^2).
    ``method`` selects the operator splitting of Eq. split-op as in
    ``bpm.march`` (stages of step n on the slice of z_n; a stage of a_i dz
    propagates with exp(i a_i dz^ delta_+-) and the common phase g is applied
    once per step); ``chi`` = (chi_0, chi_h) is needed for it."""
    psi0 = np.asarray(psi0, dtype=np.complex128)
    nb, nbands, ny, nx = psi0.shape
    assert nbands == 2 and len(plans) == nb
    n_rec = (n_end // record_every) if record_every > 0 else 0
    records = np.zeros((nb, n_rec, 2, ny, nx), dtype=np.complex128)
    powers = np.zeros((nb, n_rec + 1, 2), dtype=np.float64)
    prop_p = np.stack([p.prop_plus for p in plans])
    prop_m = np.stack([p.prop_minus for p in plans])
    g = np.array([p.base.g for p in plans])[:, None, None]
    a = np.array([p.base.a for p in plans])[:, None, None]
    b = np.array([p.base.b for p in plans])[:, None, None]

    def power(f):
        return dx_um * dy_um * np.sum(f.real ** 2 + f.imag ** 2, axis=(-2, -1))

    # stages: (propagator pair or None, a, b) per row; first order keeps the
    # plan's propagators and applies g with them
    stages = []
    if method != "first_order":
        chi0, chih = chi
        for frac_a, frac_b in bpm.split_stages(method):
            props = None
            if frac_a != 0.0:
                props = (np.stack([np.exp(1j * frac_a * p.base.dzh * p.delta_plus) for p in plans]),
                         np.stack([np.exp(1j * frac_a * p.base.dzh * p.delta_minus) for p in plans]))
            ab = [bpm.coupling_coefficients(p.base, frac_b, chi0, chih) for p in plans]
            stages.append((props, np.array([x[0] for x in ab])[:, None, None],
                           np.array([x[1] for x in ab])[:, None, None]))

    psi_p = psi0[:, 0].copy()
    psi_m = psi0[:, 1].copy()
    for step in range(n_begin, n_end):
        inside, theta = slices(step)
        e_plus = np.exp(1j * theta)
        e_minus = np.exp(-1j * theta)
        if method == "first_order":
            pp = dft.ifft2(dft.fft2(psi_p) * prop_p) * g
            pm = dft.ifft2(dft.fft2(psi_m) * prop_m) * g
            new_p = np.where(inside, a * pp + b * e_plus * pm, pp)
            new_m = np.where(inside, a * pm + b * e_minus * pp, pm)
            psi_p, psi_m = new_p, new_m
        else:
            for props, a_s, b_s in stages:
                if props is not None:
                    psi_p = dft.ifft2(dft.fft2(psi_p) * props[0])
                    psi_m = dft.ifft2(dft.fft2(psi_m) * props[1])
                new_p = np.where(inside, a_s * psi_p + b_s * e_plus * psi_m, psi_p)
                new_m = np.where(inside, a_s * psi_m + b_s * e_minus * psi_p, psi_m)
                psi_p, psi_m = new_p, new_m
            psi_p = psi_p * g
            psi_m = psi_m * g
        if record_every > 0 and (step + 1) % record_every == 0:
            slot = (step + 1) // record_every - 1
            records[:, slot, 0] = psi_p
            records[:, slot, 1] = psi_m
            powers[:, slot, 0] = power(psi_p)
            powers[:, slot, 1] = power(psi_m)
    powers[:, n_rec, 0] = power(psi_p)
    powers[:, n_rec, 1] = power(psi_m)
    return bpm.MarchResult(np.stack([psi_p, psi_m], axis=1), records, powers)
