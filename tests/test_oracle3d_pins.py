"""Pins of the 3D oracle (oracle/bpm3d.py) against the 2D march, closed
forms and brute force.  CPU only."""

import math

import numpy as np
import pytest

from oracle import bpm, bpm3d, geometry

E = 8000.0
THETA = math.radians(23.65)
CHI0 = complex(-1.51e-5, 3.5e-7)
CHIH = complex(-9.1e-6, 3.4e-7)


def _plan3(nx, ny, dx, dy, dz, chi0=CHI0, chih=CHIH):
    return bpm3d.energy_plan3d(E, E, THETA, chi0, chih, nx, ny, dx, dy, dz)


def _crystal3(nx, ny, x0, y0, dx, dy, dz):
    return bpm3d.Crystal3D(nx, ny, x0, y0, dx, dy, dz, bpm.d_spacing_um(E, THETA))


def test_y_uniform_field_reduces_to_the_2d_march():
    """A field constant along y through a y-independent crystal only has
    qy = 0 content, where the 3D propagator is the 2D one: every y line of
    the 3D march equals the 2D march (bent Bragg slab, records included)."""
    nx, ny, dx, dy, dz, nz = 128, 8, 0.4, 0.3, 0.1, 240
    x0 = -0.5 * nx * dx
    rng = np.random.default_rng(3)
    line = np.zeros((1, 2, nx), complex)
    line[0, 0] = np.exp(-((x0 + dx * np.arange(nx) + 8.0) / 6.0) ** 2) * np.exp(
        1j * rng.uniform(-0.2, 0.2, nx))
    slab = dict(asym_angle_rad=0.0, thickness_um=20.0, surf_x_um=0.0, surf_z_um=0.0)
    bend = [0.5e6, 0.28, 0.0, 10.0]
    p2 = bpm.energy_plan(E, E, THETA, CHI0, CHIH, nx, dx, dz)
    c2 = geometry.Crystal(nx, x0, dx, dz, bpm.d_spacing_um(E, THETA))
    c2.set_crystal(geometry.CRYSTAL_SLAB, **slab).set_strain(geometry.STRAIN_BENT, params=bend)
    r2 = bpm.march([p2], line, c2, 0, nz, 60, dx)
    c3 = _crystal3(nx, ny, x0, -1.0, dx, dy, dz)
    c3.set_crystal(geometry.CRYSTAL_SLAB, **slab).set_strain(geometry.STRAIN_BENT, params=bend)
    psi3 = np.repeat(line[:, :, None, :], ny, axis=2)
    r3 = bpm3d.march3d([_plan3(nx, ny, dx, dy, dz)], psi3, c3, 0, nz, 60, dx, dy)
    scale = np.abs(r2.psi).max()
    for i in range(ny):
        assert np.max(np.abs(r3.psi[:, :, i] - r2.psi)) < 1e-12 * scale
        assert np.max(np.abs(r3.records[:, :, :, i] - r2.records)) < 1e-12 * scale
    # powers: dx dy sum over the plane = ny dy x the 2D line power
    assert np.allclose(r3.powers, r2.powers * ny * dy, rtol=1e-12)


@pytest.mark.parametrize("method", ["verlet", "forest_ruth"])
def test_y_uniform_split_march_reduces_to_the_2d_split_march(method):
    """The same reduction for the higher-order splittings of Eq. split-op:
    every y line of the 3D Verlet / Forest-Ruth march equals the 2D march of
    the same scheme (bent Bragg slab, records included)."""
    nx, ny, dx, dy, dz, nz = 128, 4, 0.4, 0.3, 0.1, 120
    x0 = -0.5 * nx * dx
    line = np.zeros((1, 2, nx), complex)
    line[0, 0] = np.exp(-((x0 + dx * np.arange(nx) + 8.0) / 6.0) ** 2)
    slab = dict(asym_angle_rad=0.0, thickness_um=20.0, surf_x_um=0.0, surf_z_um=0.0)
    bend = [0.5e6, 0.28, 0.0, 10.0]
    p2 = bpm.energy_plan(E, E, THETA, CHI0, CHIH, nx, dx, dz)
    c2 = geometry.Crystal(nx, x0, dx, dz, bpm.d_spacing_um(E, THETA))
    c2.set_crystal(geometry.CRYSTAL_SLAB, **slab).set_strain(geometry.STRAIN_BENT, params=bend)
    r2 = bpm.march([p2], line, c2, 0, nz, 40, dx, method=method, chi=(CHI0, CHIH))
    c3 = _crystal3(nx, ny, x0, -1.0, dx, dy, dz)
    c3.set_crystal(geometry.CRYSTAL_SLAB, **slab).set_strain(geometry.STRAIN_BENT, params=bend)
    psi3 = np.repeat(line[:, :, None, :], ny, axis=2)
    r3 = bpm3d.march3d([_plan3(nx, ny, dx, dy, dz)], psi3, c3, 0, nz, 40, dx, dy,
                       method=method, chi=(CHI0, CHIH))
    scale = np.abs(r2.psi).max()
    for i in range(ny):
        assert np.max(np.abs(r3.psi[:, :, i] - r2.psi)) < 1e-12 * scale
        assert np.max(np.abs(r3.records[:, :, :, i] - r2.records)) < 1e-12 * scale
    # and the scheme matters: the first-order 3D march differs
    r1 = bpm3d.march3d([_plan3(nx, ny, dx, dy, dz)], psi3, c3, 0, nz, 40, dx, dy)
    assert np.max(np.abs(r1.psi - r3.psi)) > 1e-6 * scale


def test_plane_wave_mode_in_vacuum():
    """One grid mode exp(i (qx x^ + qy y^)) in psi_+ through vacuum gains the
    exact angular-spectrum phase exp(i dz^ sqrt(1 - (qx + s)^2 - qy^2)) per
    step (qx, qy from the grid definition, the root evaluated directly)."""
    nx, ny, dx, dy, dz, nz = 16, 16, 0.3, 0.2, 0.05, 40
    p = _plan3(nx, ny, dx, dy, dz)
    k = 2.0 * math.pi / bpm.wavelength_um(E)
    s = math.sin(THETA)
    xh = k * dx * np.arange(nx)
    yh = k * dy * np.arange(ny)
    cr = _crystal3(nx, ny, 0.0, 0.0, dx, dy, dz)
    for mx, my in ((0, 0), (3, 5), (nx - 2, 1), (nx // 2, ny // 2), (1, ny - 3)):
        qx = 2.0 * math.pi * (mx if mx < nx // 2 else mx - nx) / (nx * k * dx)
        qy = 2.0 * math.pi * (my if my < ny // 2 else my - ny) / (ny * k * dy)
        mode = np.exp(1j * (qy * yh[:, None] + qx * xh[None, :]))
        psi0 = np.zeros((1, 2, ny, nx), complex)
        psi0[0, 0] = mode
        res = bpm3d.march3d([p], psi0, cr, 0, nz, 0, dx, dy)
        want = np.exp(1j * nz * k * dz * math.sqrt(1.0 - (qx + s) ** 2 - qy ** 2))
        assert np.max(np.abs(res.psi[0, 0] - want * mode)) < 1e-9
        assert np.max(np.abs(res.psi[0, 1])) == 0.0


def test_box_crystal_is_the_closed_box_at_cell_centres():
    nx, ny, dx, dy, dz = 32, 16, 0.5, 0.7, 0.25
    x0, y0 = -3.0, -4.0
    box = (0.0, 5.0, -2.1, 2.1, 1.0, 3.0)
    cr = _crystal3(nx, ny, x0, y0, dx, dy, dz).set_crystal(bpm3d.CRYSTAL_BOX, box=box)
    for n in range(0, 20):
        got = cr.inside(n)
        z = n * dz
        for i in range(ny):
            for j in range(nx):
                x, y = x0 + j * dx, y0 + i * dy
                want = (0.0 <= x <= 5.0) and (-2.1 <= y <= 2.1) and (1.0 <= z <= 3.0)
                assert bool(got[i, j]) == want


def test_vacuum_conserves_power_in_3d():
    nx, ny, dx, dy, dz, nz = 32, 32, 0.2, 0.2, 0.1, 50
    rng = np.random.default_rng(5)
    psi0 = rng.standard_normal((1, 2, ny, nx)) + 1j * rng.standard_normal((1, 2, ny, nx))
    cr = _crystal3(nx, ny, 0.0, 0.0, dx, dy, dz)
    res = bpm3d.march3d([_plan3(nx, ny, dx, dy, dz)], psi0, cr, 0, nz, 0, dx, dy)
    p0 = dx * dy * np.sum(np.abs(psi0) ** 2, axis=(-2, -1))
    assert np.allclose(res.powers[:, -1], p0, rtol=1e-12)
