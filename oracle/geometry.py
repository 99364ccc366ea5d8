"""Oracle: crystal-shape masks Pi(x, z) and strain phases h*u_x(x, z).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper defines the crystal by a 0/1 map Pi (Eqs. fov11-fov12: 1 in the
crystal, 0 elsewhere), either as a slab whose surface normal is
set by ``asymm_angle`` (Section 4: 0 deg = Bragg, 90 deg = Laue, in between
= asymmetric) or as an arbitrary map (Section 7).  The deformation enters
only through u_x (Eq. Authier), here from

* a cylindrical bend, Eq. fov110 in the configured form
  u_x = (x'^2 + nu z'^2) / (2 R) with x' measured from the entrance surface
  and z' from the beam's hit point on it;
* a straight edge dislocation, Eq. fov120 with the Burgers vector b along x
  and the line normal to the (x, z) plane, which leaves
  u_x = b / (2 pi) [atan2(z', x') + x' z' / (2 (1 - nu) (x'^2 + z'^2))];
* a user array.

Readings of the paper taken here:

* Pi is binary; a cell is inside when its centre x_j = x0 + j dx,
  z_n = n dz is inside (slab test with <= on both faces, even-odd rule with
  the half-open crossing test for polygons).
* Slab normal n = (cos a, sin a) in (x, z); a component whose magnitude is
  below 1e-12 is set to exactly 0 (so a = 90 deg gives an exact Laue slab).
  Crystal = {0 <= n . (r - r_s) <= T}.
* The atan2 branch cut of the dislocation runs along -x' from the core and
  u_x = 0 at the core itself.
"""

from __future__ import annotations

import math

import numpy as np

from .bpm import TWO_PI

# Mask kinds (mirrors the C-ABI enumeration in include/bpm.h).
CRYSTAL_VACUUM = 0
CRYSTAL_BULK = 1
CRYSTAL_SLAB = 2
CRYSTAL_MASK = 3
CRYSTAL_SLAB_AND_MASK = 4
CRYSTAL_SLAB_AND_POLYGON = 5

# Strain kinds.
STRAIN_NONE = 0
STRAIN_ARRAY = 1
STRAIN_BENT = 2
STRAIN_EDGE_DISLOCATION = 3


def grid_x(nx: int, x0_um: float, dx_um: float) -> np.ndarray:
    """Cell centres x_j = x0 + j dx (one multiply, one add, in that order)."""
    return x0_um + np.arange(nx, dtype=np.float64) * dx_um


def grid_z(n: int, dz_um: float) -> float:
    """z_n = n dz: the mask and strain of step n are sampled here."""
    return float(n) * dz_um


def slab_normal(asym_angle_rad: float) -> tuple[float, float]:
    cx = math.cos(asym_angle_rad)
    sz = math.sin(asym_angle_rad)
    if abs(cx) < 1e-12:
        cx, sz = 0.0, math.copysign(1.0, sz)
    elif abs(sz) < 1e-12:
        cx, sz = math.copysign(1.0, cx), 0.0
    return cx, sz


def slab_row(x: np.ndarray, z: float, asym_angle_rad: float,
             thickness_um: float, surf_x_um: float, surf_z_um: float
             ) -> np.ndarray:
    """Inside test of the slab {0 <= n.(r - r_s) <= T} for one row z."""
    cx, sz = slab_normal(asym_angle_rad)
    depth = cx * (x - surf_x_um) + sz * (z - surf_z_um)
    return (depth >= 0.0) & (depth <= thickness_um)


def polygon_row(x: np.ndarray, z: float, px: np.ndarray, pz: np.ndarray
                ) -> np.ndarray:
    """Even-odd point-in-polygon test for one row z (vertices in order).

    Edge (i, i+1) is crossed by the ray from (x, z) towards +x when exactly
    one end lies above z and x is left of the edge's crossing abscissa.
    """
    inside = np.zeros(x.shape, dtype=bool)
    nv = len(px)
    for i in range(nv):
        j = (i + 1) % nv
        if (pz[i] > z) != (pz[j] > z):
            xc = (px[j] - px[i]) * (z - pz[i]) / (pz[j] - pz[i]) + px[i]
            inside ^= x < xc
    return inside


def bent_ux(x: np.ndarray, z: float, radius_um: float, nu: float,
            x_ref_um: float, z_ref_um: float) -> np.ndarray:
    """u_x = (x'^2 + nu z'^2) / (2 R) (configured form of Eq. fov110)."""
    xp = x - x_ref_um
    zp = z - z_ref_um
    return (xp * xp + nu * (zp * zp)) / (2.0 * radius_um)


def edge_dislocation_ux(x: np.ndarray, z: float, burgers_um: float, nu: float,
                        xc_um: float, zc_um: float) -> np.ndarray:
    """u_x of a straight edge dislocation (Eq. fov120, b along x, line along y)."""
    xp = x - xc_um
    zp = z - zc_um
    r2 = xp * xp + zp * zp
    with np.errstate(divide="ignore", invalid="ignore"):
        u = burgers_um / TWO_PI * (np.arctan2(zp, xp)
                                   + xp * zp / (2.0 * (1.0 - nu) * r2))
    return np.where(r2 == 0.0, 0.0, u)


class Crystal:
    """Row provider n -> (Pi[n][:], h*u_x[n][:]) for ``bpm.march``."""

    def __init__(self, nx: int, x0_um: float, dx_um: float, dz_um: float,
                 d_spacing_um: float):
        self.nx = nx
        self.dz_um = dz_um
        self.x = grid_x(nx, x0_um, dx_um)
        self.h = TWO_PI / d_spacing_um
        self.crystal_kind = CRYSTAL_VACUUM
        self.strain_kind = STRAIN_NONE

    # -- shape -------------------------------------------------------------
    def set_crystal(self, kind: int, asym_angle_rad: float = 0.0,
                    thickness_um: float = 0.0, surf_x_um: float = 0.0,
                    surf_z_um: float = 0.0, mask=None, polygon=None):
        self.crystal_kind = kind
        self.slab = (asym_angle_rad, thickness_um, surf_x_um, surf_z_um)
        self.mask = None if mask is None else np.asarray(mask) != 0
        if polygon is not None:
            poly = np.asarray(polygon, dtype=np.float64).reshape(-1, 2)
            self.px, self.pz = poly[:, 0].copy(), poly[:, 1].copy()
        return self

    def inside(self, n: int) -> np.ndarray:
        z = grid_z(n, self.dz_um)
        k = self.crystal_kind
        if k == CRYSTAL_VACUUM:
            return np.zeros(self.nx, dtype=bool)
        if k == CRYSTAL_BULK:
            return np.ones(self.nx, dtype=bool)
        if k == CRYSTAL_MASK:
            return self.mask[n].copy()
        slab = slab_row(self.x, z, *self.slab)
        if k == CRYSTAL_SLAB:
            return slab
        if k == CRYSTAL_SLAB_AND_MASK:
            return slab & self.mask[n]
        if k == CRYSTAL_SLAB_AND_POLYGON:
            return slab & polygon_row(self.x, z, self.px, self.pz)
        raise ValueError(f"unknown crystal kind {k}")

    # -- deformation --------------------------------------------------------
    def set_strain(self, kind: int, ux=None, params=None):
        self.strain_kind = kind
        self.ux = None if ux is None else np.asarray(ux, dtype=np.float64)
        self.params = None if params is None else [float(p) for p in params]
        return self

    def ux_row(self, n: int) -> np.ndarray:
        z = grid_z(n, self.dz_um)
        k = self.strain_kind
        if k == STRAIN_NONE:
            return np.zeros(self.nx)
        if k == STRAIN_ARRAY:
            return self.ux[n].copy()
        if k == STRAIN_BENT:
            return bent_ux(self.x, z, *self.params[:4])
        if k == STRAIN_EDGE_DISLOCATION:
            return edge_dislocation_ux(self.x, z, *self.params[:4])
        raise ValueError(f"unknown strain kind {k}")

    def theta(self, n: int) -> np.ndarray:
        """Strain phase h * u_x (Eq. Authier, k_d . u with k_d along x)."""
        return self.h * self.ux_row(n)

    def __call__(self, n: int):
        return self.inside(n), self.theta(n)
