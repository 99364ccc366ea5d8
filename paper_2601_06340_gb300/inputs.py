"""Seeded synthetic inputs for the two-beam FFT-BPM z-march.

This module is shared by the tests, the benchmark and users who want the
standard workloads.  It builds *inputs only* -- grids, photon energies,
incident envelopes, crystal-shape descriptors, displacement descriptors --
and holds none of the march's arithmetic (no propagators, no coupling, no
FFTs).  Every random draw comes from ``numpy.random.default_rng`` with a
fixed seed (base seed 20260106, workload i uses base + i).

The five workloads are the problem classes the paper simulates (Laue and
Bragg slabs, bent crystals, dislocations in arbitrarily shaped crystals,
time-dependent pulses as batches of photon energies) with the sizes of the
project's benchmark table:

1. ``laue_perfect``      symmetric Laue, perfect, 8 keV, 100 um, Nx=1024, Nz=2000
2. ``bragg_bent``        symmetric Bragg, bent R = 1 m, 200 um, Nx=4096, Nz=8000
3. ``asym_dislocation``  asymmetric Bragg (10 deg) slab cut by a seeded star
                         polygon, edge dislocation, Nx=8192, Nz=12000
4. ``pulse_batched``     256 energies over 9 keV +- 5 eV, Laue, bent R = 2 m,
                         Nx=4096, Nz=6000, SASE-like random spectral phases
5. ``serving_stream``    Poisson request stream of mixed solves (see
                         ``serving_requests``)
6. ``rocking_scan``      256 incidence angles over +-50 urad through one Laue
                         slab (100 um), Nx=2048, Nz=2000, one batched launch
7. ``cube_dislocation_3d`` both transverse coordinates: a 10 um box crystal with
                         a dislocation at 17.45 keV, 512 x 256 x 300 cells

Each builder takes optional smaller ``nx`` / ``nz`` so that the same
geometry can be run at sizes the FP64 oracle finishes in seconds.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20260106
HC_EV_ANGSTROM = 12398.419843320026

# Kind codes (same values as include/bpm.h).
CRYSTAL_VACUUM, CRYSTAL_BULK, CRYSTAL_SLAB, CRYSTAL_MASK = 0, 1, 2, 3
CRYSTAL_SLAB_AND_MASK, CRYSTAL_SLAB_AND_POLYGON = 4, 5
STRAIN_NONE, STRAIN_ARRAY, STRAIN_BENT, STRAIN_EDGE_DISLOCATION = 0, 1, 2, 3

# Si(220)-like reflection at 8 keV as configured (Bragg angle 23.65 deg).
E_REF_EV = 8000.0
THETA_B_REF = math.radians(23.65)
CHI0 = complex(-1.51e-5, 3.5e-7)
CHIH = complex(-9.1e-6, 3.4e-7)


@dataclass
class Workload:
    name: str
    nx: int
    nz: int
    dx_um: float
    dz_um: float
    x0_um: float
    energies_ev: np.ndarray
    e_ref_ev: float
    theta_b_ref_rad: float
    chi0: complex
    chih: complex
    record_every: int
    crystal: dict
    strain: dict
    psi0: np.ndarray                      # [B][2][N] complex128
    meta: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return len(self.energies_ev)

    @property
    def cell_updates(self) -> int:
        return self.batch * self.nx * self.nz


@dataclass
class Workload3D(Workload):
    """A workload with both transverse coordinates: fields [B][2][Ny][Nx]."""
    ny: int = 1
    dy_um: float = 1.0
    y0_um: float = 0.0

    @property
    def cell_updates(self) -> int:
        return self.batch * self.nx * self.ny * self.nz


CRYSTAL_BOX = 6


def gaussian_envelope(nx: int, x0_um: float, dx_um: float, centre_um: float,
                      fwhm_um: float, cos_theta: float,
                      tilt_per_um: float = 0.0) -> np.ndarray:
    """Incident psi_+(x, z=0): intensity FWHM ``fwhm_um`` measured normal to
    the beam, so the trace on the z = 0 plane has FWHM fwhm / cos(theta);
    ``tilt_per_um`` adds a linear envelope phase (rad / um) about the centre.
    """
    x = x0_um + np.arange(nx, dtype=np.float64) * dx_um
    wx = fwhm_um / cos_theta
    amp = np.exp(-2.0 * math.log(2.0) * ((x - centre_um) / wx) ** 2)
    return amp * np.exp(1j * tilt_per_um * (x - centre_um))


def slit_field(nx: int, x0_um: float, dx_um: float, centre_um: float, width_um: float,
               tilt_per_um: float = 0.0) -> np.ndarray:
    """Incident psi_+ shaped by a slit (section topography, Sec. 5: a 5 um
    slit): unit amplitude on the cells whose centres lie within
    ``width_um`` / 2 of ``centre_um``, zero elsewhere, with an optional
    linear envelope phase; psi_- = 0.  Shape [1][2][nx]."""
    x = x0_um + np.arange(nx, dtype=np.float64) * dx_um
    amp = (np.abs(x - centre_um) <= 0.5 * width_um).astype(np.float64)
    return _two_band(amp * np.exp(1j * tilt_per_um * (x - centre_um)))


def far_field_step(exit_field: np.ndarray, nx: int, dx_um: float, x0_um: float,
                   distance_um: float, energy_ev: float = E_REF_EV,
                   theta_b_ref_rad: float = THETA_B_REF) -> "Workload":
    """One free-space step of ``distance_um`` applied to a march's exit
    field (both envelopes, each through its own angular-spectrum operator):
    a vacuum plan with chi = 0, nz = 1, dz = distance (the far-field images
    of Secs. 5-6 are taken 2-4 m behind the crystal)."""
    return Workload(
        "far_field", nx, 1, dx_um, distance_um, x0_um, np.array([energy_ev]), energy_ev,
        theta_b_ref_rad, 0j, 0j, 0, crystal=dict(kind=CRYSTAL_VACUUM),
        strain=dict(kind=STRAIN_NONE), psi0=np.asarray(exit_field, dtype=np.complex128))


def _two_band(psi_plus: np.ndarray) -> np.ndarray:
    out = np.zeros((1, 2, psi_plus.shape[-1]), dtype=np.complex128)
    out[0, 0] = psi_plus
    return out


def laue_perfect(nx: int = 1024, nz: int = 2000, dx_um: float = 0.4,
                 dz_um: float = 0.05, record_every: int = 100) -> Workload:
    """Symmetric Laue slab of 100 um (Pi = 1 on every step of the march)."""
    x0 = -0.5 * nx * dx_um
    c = math.cos(THETA_B_REF)
    psi0 = _two_band(gaussian_envelope(nx, x0, dx_um, 0.0, 20.0, c))
    return Workload(
        "laue_perfect", nx, nz, dx_um, dz_um, x0, np.array([E_REF_EV]),
        E_REF_EV, THETA_B_REF, CHI0, CHIH, record_every,
        crystal=dict(kind=CRYSTAL_SLAB, asym_angle_rad=math.pi / 2,
                     thickness_um=100.0, surf_x_um=0.0, surf_z_um=0.0),
        strain=dict(kind=STRAIN_NONE), psi0=psi0)


def bragg_bent(nx: int = 4096, nz: int = 8000, dx_um: float = 0.2,
               dz_um: float = 0.1, record_every: int = 100,
               radius_um: float = 1.0e6, nu: float = 0.28) -> Workload:
    """Symmetric Bragg slab x in [0, 200] um, bent (u = (x^2 + nu z'^2)/2R).

    The beam (50 um FWHM) starts at z = 0 and hits the surface x = 0 at
    z_hit = (march length) * 5/16 (250 um for the full 800 um march).
    """
    x0 = -0.5 * nx * dx_um
    tan_t = math.tan(THETA_B_REF)
    z_hit = nz * dz_um * 5.0 / 16.0
    xc = -tan_t * z_hit
    psi0 = _two_band(gaussian_envelope(nx, x0, dx_um, xc, 50.0,
                                       math.cos(THETA_B_REF)))
    return Workload(
        "bragg_bent", nx, nz, dx_um, dz_um, x0, np.array([E_REF_EV]),
        E_REF_EV, THETA_B_REF, CHI0, CHIH, record_every,
        crystal=dict(kind=CRYSTAL_SLAB, asym_angle_rad=0.0,
                     thickness_um=200.0, surf_x_um=0.0, surf_z_um=0.0),
        strain=dict(kind=STRAIN_BENT, params=[radius_um, nu, 0.0, z_hit]),
        psi0=psi0, meta=dict(z_hit_um=z_hit))


def star_polygon(rng: np.random.Generator, centre: tuple[float, float],
                 extent_um: float, nv: int) -> np.ndarray:
    """Seeded star-shaped polygon: sorted angles, radii U[0.5, 1] * D/2."""
    ang = np.sort(rng.uniform(0.0, 2.0 * math.pi, nv))
    rad = rng.uniform(0.5, 1.0, nv) * extent_um / 2.0
    return np.stack([centre[0] + rad * np.cos(ang),
                     centre[1] + rad * np.sin(ang)], axis=1)


def asym_dislocation(nx: int = 8192, nz: int = 12000, dx_um: float = 0.1,
                     dz_um: float = 0.05, record_every: int = 200,
                     asym_deg: float = 10.0, seed: int = BASE_SEED + 3,
                     burgers_um: float = 3.84e-4, nu: float = 0.28,
                     core_depth_um: float = 20.0) -> Workload:
    """Asymmetric Bragg slab (300 um) cut by a seeded star polygon, with an
    edge dislocation 20 um below the entrance surface at the beam hit point.
    """
    rng = np.random.default_rng(seed)
    nv = int(rng.integers(5, 9))
    extent = float(rng.uniform(50.0, 300.0))
    x0 = -0.5 * nx * dx_um
    a = math.radians(asym_deg)
    nrm = (math.cos(a), math.sin(a))
    z_hit = nz * dz_um / 2.0
    tan_t = math.tan(THETA_B_REF)
    xb = -tan_t * z_hit                        # beam centre at z = 0
    surf = (0.0, z_hit)                        # hit point on the surface
    centre = (surf[0] + nrm[0] * extent / 2.0, surf[1] + nrm[1] * extent / 2.0)
    poly = star_polygon(rng, centre, extent, nv)
    core = (surf[0] + nrm[0] * core_depth_um, surf[1] + nrm[1] * core_depth_um)
    psi0 = _two_band(gaussian_envelope(nx, x0, dx_um, xb, 50.0,
                                       math.cos(THETA_B_REF)))
    return Workload(
        "asym_dislocation", nx, nz, dx_um, dz_um, x0, np.array([E_REF_EV]),
        E_REF_EV, THETA_B_REF, CHI0, CHIH, record_every,
        crystal=dict(kind=CRYSTAL_SLAB_AND_POLYGON, asym_angle_rad=a,
                     thickness_um=300.0, surf_x_um=surf[0], surf_z_um=surf[1],
                     polygon=poly),
        strain=dict(kind=STRAIN_EDGE_DISLOCATION,
                    params=[burgers_um, nu, core[0], core[1]]),
        psi0=psi0, meta=dict(nv=nv, extent_um=extent))


def pulse_energies(n_energy: int = 256, centre_ev: float = 9000.0,
                   span_ev: float = 10.0) -> np.ndarray:
    """E_j = centre - span/2 + span * j / B, ascending."""
    return centre_ev - span_ev / 2.0 + span_ev * np.arange(n_energy) / n_energy


def pulse_batched(nx: int = 4096, nz: int = 6000, n_energy: int = 256,
                  dx_um: float = 0.1, dz_um: float = 0.05,
                  record_every: int = 0, sigma_ev: float = 1.5,
                  radius_um: float = 2.0e6, nu: float = 0.28,
                  seed: int = BASE_SEED + 4) -> Workload:
    """Batch of photon energies through one bent Laue slab (300 um).

    The crystal is set at the Bragg angle of the centre energy, so row j's
    incident envelope carries the tilt (sin theta_0 - s_j) k_j: its carrier
    is the fixed incident direction while the band centre s_j = lambda_j/2d
    moves with energy.  Spectral amplitudes: Gaussian envelope (intensity
    RMS sigma) times seeded uniform random phases (SASE-like).
    """
    rng = np.random.default_rng(seed)
    energies = pulse_energies(n_energy)
    phases = rng.uniform(0.0, 2.0 * math.pi, n_energy)
    centre_ev = 9000.0
    s_ref = math.sin(THETA_B_REF)
    s0 = s_ref * E_REF_EV / centre_ev
    c0 = math.sqrt(1.0 - s0 * s0)
    x0 = -0.5 * nx * dx_um
    thickness = 300.0
    xb = -0.5 * thickness * s0 / c0             # centre the Borrmann fan
    psi0 = np.zeros((n_energy, 2, nx), dtype=np.complex128)
    for j, e in enumerate(energies):
        k = 2.0 * math.pi / (HC_EV_ANGSTROM / e * 1e-4)
        sj = s_ref * E_REF_EV / e
        amp = math.exp(-((e - centre_ev) ** 2) / (4.0 * sigma_ev ** 2))
        env = gaussian_envelope(nx, x0, dx_um, xb, 50.0, c0,
                                tilt_per_um=(s0 - sj) * k)
        psi0[j, 0] = amp * complex(math.cos(phases[j]), math.sin(phases[j])) * env
    return Workload(
        "pulse_batched", nx, nz, dx_um, dz_um, x0, energies, E_REF_EV,
        THETA_B_REF, CHI0, CHIH, record_every,
        crystal=dict(kind=CRYSTAL_SLAB, asym_angle_rad=math.pi / 2,
                     thickness_um=thickness, surf_x_um=0.0, surf_z_um=0.0),
        strain=dict(kind=STRAIN_BENT, params=[radius_um, nu, 0.0, 0.0]),
        psi0=psi0, meta=dict(centre_ev=centre_ev, sigma_ev=sigma_ev))


def rocking_angles_urad(n_angles: int = 256, span_urad: float = 100.0) -> np.ndarray:
    """Incidence offsets from the Bragg angle, evenly spaced over
    [-span/2, span/2), ascending (urad)."""
    return -0.5 * span_urad + span_urad * np.arange(n_angles) / n_angles


def rocking_scan(nx: int = 2048, nz: int = 2000, n_angles: int = 256,
                 span_urad: float = 100.0, dx_um: float = 0.4,
                 dz_um: float = 0.05, fwhm_um: float = 200.0,
                 radius_um: float | None = None, nu: float = 0.28) -> Workload:
    """Rocking curve of a symmetric Laue slab (Sec. 3: rocking curves as
    independent solves over the incidence angle; Sec. 4: the Laue-geometry
    rocking curve): every row is the same photon energy (8 keV)
    with the incident beam turned by dtheta_b from the Bragg angle, i.e. the
    envelope of psi_+ carries the tilt k cos(theta_B) dtheta_b.  The slab is
    as thick as the march (nz dz); the beam (``fwhm_um``, wide enough that
    its divergence is far below the Darwin width) is centred on the Borrmann
    fan.  Optional cylindrical bend (radius, Poisson ratio).  The
    reflectivity of row b is its final P_- over its incident P_+.
    """
    angles = rocking_angles_urad(n_angles, span_urad)
    x0 = -0.5 * nx * dx_um
    s = math.sin(THETA_B_REF)
    c = math.cos(THETA_B_REF)
    thickness = nz * dz_um
    k = 2.0 * math.pi / (HC_EV_ANGSTROM / E_REF_EV * 1e-4)
    xb = -0.5 * thickness * s / c
    psi0 = np.zeros((n_angles, 2, nx), dtype=np.complex128)
    for b, a in enumerate(angles):
        psi0[b, 0] = gaussian_envelope(nx, x0, dx_um, xb, fwhm_um, c,
                                       tilt_per_um=k * c * a * 1e-6)
    strain = dict(kind=STRAIN_NONE)
    if radius_um is not None:
        strain = dict(kind=STRAIN_BENT, params=[radius_um, nu, 0.0, 0.0])
    return Workload(
        "rocking_scan", nx, nz, dx_um, dz_um, x0,
        np.full(n_angles, E_REF_EV), E_REF_EV, THETA_B_REF, CHI0, CHIH, 0,
        crystal=dict(kind=CRYSTAL_SLAB, asym_angle_rad=math.pi / 2,
                     thickness_um=thickness, surf_x_um=0.0, surf_z_um=0.0),
        strain=strain, psi0=psi0, meta=dict(angles_urad=angles))


# Si(440)-like reflection at 17.45 keV (d = a / sqrt(32), a = 5.4309 A):
# chi values scaled from the 8 keV Si values (chi_0 ~ lambda^2, chi_h by the
# (440) form-factor ratio) -- synthetic stand-ins, not tabulated values.
E_440_EV = 17450.0
D_440_UM = 5.4309e-4 / math.sqrt(32.0)
THETA_440 = math.asin(HC_EV_ANGSTROM / E_440_EV * 1e-4 / (2.0 * D_440_UM))
CHI0_440 = complex(-3.17e-6, 1.6e-8)
CHIH_440 = complex(-1.45e-6, 1.2e-8)


def cube_dislocation_3d(nx: int = 512, ny: int = 256, nz: int = 300, dx_um: float = 0.05,
                        dy_um: float = 0.05, dz_um: float = 0.05, cube_um: float = 10.0,
                        fwhm_um: float = 2.0, record_every: int = 0) -> Workload3D:
    """Stand-in for the 3D example of Sec. 7 (Si(440) at 17.45 keV from a
    10 um cube with a dislocation, 300 x 200 x 300 grid): a box crystal
    x in [0, cube], |y| <= cube/2, z in [cube/4, 5 cube/4]; an edge
    dislocation (b = 0.384 nm, nu = 0.28) along y through the cube centre
    (the paper's mixed 60 deg dislocation also has a screw part, not
    modelled); a Gaussian beam (``fwhm_um`` in x and y) at the Bragg angle
    hitting the face x = 0 at mid-height; grid padded to powers of two.
    """
    x0 = -0.42 * nx * dx_um
    y0 = -0.5 * ny * dy_um
    s = math.sin(THETA_440)
    c = math.cos(THETA_440)
    z_hit = 0.75 * cube_um
    xb = -s / c * z_hit
    x = x0 + np.arange(nx) * dx_um
    y = y0 + np.arange(ny) * dy_um
    gx = np.exp(-2.0 * math.log(2.0) * ((x - xb) / (fwhm_um / c)) ** 2)
    gy = np.exp(-2.0 * math.log(2.0) * (y / fwhm_um) ** 2)
    psi0 = np.zeros((1, 2, ny, nx), dtype=np.complex128)
    psi0[0, 0] = gy[:, None] * gx[None, :]
    box = [0.0, cube_um, -0.5 * cube_um, 0.5 * cube_um, 0.25 * cube_um, 1.25 * cube_um]
    core = (0.5 * cube_um, 0.75 * cube_um)
    return Workload3D(
        "cube_dislocation_3d", nx, nz, dx_um, dz_um, x0, np.array([E_440_EV]), E_440_EV,
        THETA_440, CHI0_440, CHIH_440, record_every,
        crystal=dict(kind=CRYSTAL_BOX, box_um=box),
        strain=dict(kind=STRAIN_EDGE_DISLOCATION, params=[3.84e-4, 0.28, core[0], core[1]]),
        psi0=psi0, meta=dict(cube_um=cube_um), ny=ny, dy_um=dy_um, y0_um=y0)


@dataclass
class Request:
    arrival_s: float
    workload: Workload


def serving_request(rng: np.random.Generator, nx: int, nz: int,
                    dx_um: float = 0.1, dz_um: float = 0.05) -> Workload:
    """One mixed solve: Bragg / Laue / asymmetric, bent or dislocated."""
    geom = int(rng.integers(0, 3))
    x0 = -0.5 * nx * dx_um
    tan_t = math.tan(THETA_B_REF)
    c = math.cos(THETA_B_REF)
    length = nz * dz_um
    if geom == 0:                                  # symmetric Bragg
        a, surf = 0.0, (0.0, length * 0.25)
        xb = -tan_t * surf[1]
    elif geom == 1:                                # symmetric Laue
        a, surf = math.pi / 2, (0.0, 0.0)
        xb = -0.5 * length * tan_t
    else:                                          # asymmetric Bragg
        a = math.radians(float(rng.uniform(5.0, 30.0)))
        surf = (0.0, length * 0.25)
        xb = -tan_t * surf[1]
    xb = max(xb, x0 + 0.25 * nx * dx_um)
    nrm = (math.cos(a), math.sin(a))
    if rng.uniform() < 0.5:
        strain = dict(kind=STRAIN_BENT,
                      params=[float(rng.uniform(0.5e6, 5.0e6)), 0.28,
                              surf[0], surf[1]])
    else:
        depth = 20.0
        strain = dict(kind=STRAIN_EDGE_DISLOCATION,
                      params=[3.84e-4, 0.28, surf[0] + nrm[0] * depth,
                              surf[1] + nrm[1] * depth])
    fwhm = min(50.0, 0.1 * nx * dx_um)
    psi0 = _two_band(gaussian_envelope(nx, x0, dx_um, xb, fwhm, c))
    return Workload(
        "serving_request", nx, nz, dx_um, dz_um, x0, np.array([E_REF_EV]),
        E_REF_EV, THETA_B_REF, CHI0, CHIH, 0,
        crystal=dict(kind=CRYSTAL_SLAB, asym_angle_rad=a, thickness_um=300.0,
                     surf_x_um=surf[0], surf_z_um=surf[1]),
        strain=strain, psi0=psi0, meta=dict(geometry=geom))


def serving_requests(n: int, rate_per_s: float = 200.0,
                     nx_choices=(512, 1024, 2048, 4096, 8192, 16384),
                     nz_range=(500, 20000), seed: int = BASE_SEED + 5
                     ) -> list[Request]:
    """Poisson arrivals (mean ``rate_per_s``) of mixed solves."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        nx = int(rng.choice(nx_choices))
        nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
        out.append(Request(t, serving_request(rng, nx, nz)))
    return out


WORKLOADS = {
    "laue_perfect": laue_perfect,
    "bragg_bent": bragg_bent,
    "asym_dislocation": asym_dislocation,
    "pulse_batched": pulse_batched,
}
