"""Oracle: run a whole workload through the FP64 march.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  ``wl`` is any object
with the fields of a workload (grid, energies, chi values, crystal and strain
descriptions, incident field); nothing from the product package is imported.
"""

from __future__ import annotations

import numpy as np

from . import bpm, geometry


def plans_for(wl, rows=None):
    idx = range(len(wl.energies_ev)) if rows is None else rows
    return [bpm.energy_plan(float(wl.energies_ev[r]), wl.e_ref_ev, wl.theta_b_ref_rad,
                            complex(wl.chi0), complex(wl.chih), wl.nx, wl.dx_um, wl.dz_um)
            for r in idx]


def crystal_for(wl) -> geometry.Crystal:
    cr = geometry.Crystal(wl.nx, wl.x0_um, wl.dx_um, wl.dz_um,
                          bpm.d_spacing_um(wl.e_ref_ev, wl.theta_b_ref_rad))
    c = dict(wl.crystal)
    kind = c.pop("kind")
    cr.set_crystal(kind, c.get("asym_angle_rad", 0.0), c.get("thickness_um", 0.0),
                   c.get("surf_x_um", 0.0), c.get("surf_z_um", 0.0), c.get("mask"),
                   c.get("polygon"))
    s = dict(wl.strain)
    cr.set_strain(s.pop("kind"), s.get("ux"), s.get("params"))
    return cr


def run_workload(wl, n_begin=0, n_end=None, rows=None, psi_in=None,
                 record_every=None, method="first_order") -> bpm.MarchResult:
    """March rows ``rows`` (default all) of ``wl`` from n_begin to n_end with
    the operator splitting ``method`` (see ``bpm.split_stages``)."""
    n_end = wl.nz if n_end is None else n_end
    plans = plans_for(wl, rows)
    psi = wl.psi0 if psi_in is None else psi_in
    if rows is not None:
        psi = np.asarray(psi)[list(rows)]
    rec = wl.record_every if record_every is None else record_every
    return bpm.march(plans, psi, crystal_for(wl), n_begin, n_end, rec, wl.dx_um,
                     method=method, chi=(complex(wl.chi0), complex(wl.chih)))


def mask_of(wl) -> np.ndarray:
    cr = crystal_for(wl)
    return np.stack([cr.inside(n) for n in range(wl.nz)])


def run_workload3d(wl, n_begin=0, n_end=None, psi_in=None, record_every=None,
                   method="first_order"):
    """March a 3D workload (fields [B][2][Ny][Nx]) from n_begin to n_end with
    the operator splitting ``method`` (see ``bpm.split_stages``)."""
    from . import bpm3d
    n_end = wl.nz if n_end is None else n_end
    plans = [bpm3d.energy_plan3d(float(e), wl.e_ref_ev, wl.theta_b_ref_rad, complex(wl.chi0),
                                 complex(wl.chih), wl.nx, wl.ny, wl.dx_um, wl.dy_um, wl.dz_um)
             for e in wl.energies_ev]
    cr = bpm3d.Crystal3D(wl.nx, wl.ny, wl.x0_um, wl.y0_um, wl.dx_um, wl.dy_um, wl.dz_um,
                         bpm.d_spacing_um(wl.e_ref_ev, wl.theta_b_ref_rad))
    c = dict(wl.crystal)
    kind = c.pop("kind")
    if kind == bpm3d.CRYSTAL_BOX:
        cr.set_crystal(kind, box=c["box_um"])
    elif kind == geometry.CRYSTAL_MASK:
        cr.set_crystal(kind, mask3=c["mask"])
    else:
        cr.set_crystal(kind, asym_angle_rad=c.get("asym_angle_rad", 0.0),
                       thickness_um=c.get("thickness_um", 0.0), surf_x_um=c.get("surf_x_um", 0.0),
                       surf_z_um=c.get("surf_z_um", 0.0), polygon=c.get("polygon"))
    s = dict(wl.strain)
    cr.set_strain(s.pop("kind"), ux3=s.get("ux"), params=s.get("params"))
    psi = wl.psi0 if psi_in is None else psi_in
    rec = wl.record_every if record_every is None else record_every
    return bpm3d.march3d(plans, psi, cr, n_begin, n_end, rec, wl.dx_um, wl.dy_um,
                         method=method, chi=(complex(wl.chi0), complex(wl.chih)))
