"""Oracle: the first-order two-beam FFT-BPM z-march in float64 / complex128.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper (arXiv 2601.06340, Section 2 "Theoretical
approach"):

* hatted coordinates x^ = k x, z^ = k z with k = 2 pi / lambda (Eq. fov2);
* the two envelopes psi_+ (transmitted, carrier e^{+i k_d x^/2}) and psi_-
  (reflected, carrier e^{-i k_d x^/2}) of Eqs. fov6-fov7, with
  k_d / 2 = lambda / (2 d) = sin(theta_B) =: s in units of k;
* the susceptibility delta_eps = chi_0 + 2 chi_h cos(k_d x^) (Eq. fov8);
* its Jacobi-Anger expansion truncated to n = 0, +-1 (Eqs. fov9, fov11,
  fov12), read with the step length dz^ = k dz in place of z^:
      Delta_eps_0   = J0(w) exp(i phi0),
      Delta_eps_+-1 = i J1(w) exp(i phi0),
      w = dz^ chi_h / cos(alpha),   phi0 = dz^ chi_0 / (2 cos(alpha)),
  inside the crystal (Pi = 1) and Delta_eps_0 = 1, Delta_eps_+-1 = 0
  outside (Pi = 0);
* cos(alpha) = sqrt(1 - s^2) for both bands (Eq. fov4 with the angular
  spectrum centred on +-s);
* the deformation phase Delta_eps'_n = Delta_eps_n exp(i n h u_x)
  (Eq. Authier), h = 2 pi / d;
* the march of Eq. fov10,
      psi_+(z^+dz^) = psi_p+ Delta_eps_0 + psi_p- Delta_eps'_{+1},
      psi_-(z^+dz^) = psi_p- Delta_eps_0 + psi_p+ Delta_eps'_{-1},
  where psi_p+- is each envelope propagated through its own angular-spectrum
  operator exp(i dz^ sqrt(1 - kx^2)) centred on its own carrier.

Readings where the paper is silent or ambiguous:

* FFT convention: forward kernel e^{-2 pi i m j / N} (numpy's), computed by
  the oracle's own DFT / radix-2 FFT (``oracle.fft``).  With it the
  + envelope's spectrum sits at kx = q + s, so its propagator uses
  sqrt(1 - (q + s)^2) and the - envelope's uses sqrt(1 - (q - s)^2).  The
  paper's "p_-+" pairing is the same statement under the opposite sign
  convention of F.
* q_m = 2 pi fftfreq(N, dx^), i.e. index N/2 is the negative Nyquist mode.
* The propagator is written as g * exp(i dz^ delta_+-(q)) with
  g = exp(i (dz^ cos(alpha) mod 2 pi)) and
  delta_+-(q) = sqrt(1 - (q +- s)^2) - cos(alpha) in the cancellation-free
  form -q (q +- 2 s) / (sqrt(1 - (q +- s)^2) + cos(alpha)).  The product is
  algebraically exp(i dz^ sqrt(1 - (q +- s)^2)) of Eq. fov10; the split only
  keeps the FP64 argument of the per-mode exponential small.  The "-1" of
  Eq. fov2 is not applied (Eqs. fov4 and fov10 omit it).
* Mask and strain are sampled at the start of each step, z_n = n dz, and at
  the cell centres x_j = x0 + j dx (Eq. fov10 evaluates Delta_eps at z^).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import fft as dft

# h*c in eV * Angstrom (CODATA 2018: h and c exact, e exact).
HC_EV_ANGSTROM = 12398.419843320026
TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------
# Bessel functions of complex argument (Eqs. fov11-fov12 need J0 and J1)
# --------------------------------------------------------------------------

def bessel_series(nu: int, w: complex, skip_first: bool = False) -> complex:
    """J_nu(w) = sum_m (-1)^m (w/2)^(2m+nu) / (m! (m+nu)!), complex w.

    Summed term by term until a term falls below 1e-18 of the first
    term's magnitude (|w| is ~0.02 on the configured grids, so a handful of
    terms suffice).  ``skip_first`` drops the m = 0 term, which for nu = 0
    gives J0(w) - 1 without cancellation.
    """
    half = complex(w) / 2.0
    term = half ** nu / math.factorial(nu)
    scale = max(abs(term), 1e-300)
    total = 0j if skip_first else term
    m = 0
    while True:
        m += 1
        term = term * (-(half * half)) / (m * (m + nu))
        total += term
        if abs(term) < 1e-18 * scale or m > 200:
            break
    return total


# --------------------------------------------------------------------------
# Plan scalars and propagator tables for one photon energy
# --------------------------------------------------------------------------

@dataclass
class EnergyPlan:
    energy_ev: float
    k_um: float          # wave number 2 pi / lambda in 1/um
    s: float             # k_d / 2 in units of k = sin(theta_B(E))
    c: float             # cos(alpha) = sqrt(1 - s^2)
    dzh: float           # dz^ = k dz
    dxh: float           # dx^ = k dx
    w: complex           # dz^ chi_h / cos(alpha)
    phi0: complex        # dz^ chi_0 / (2 cos(alpha))
    a: complex           # Delta_eps_0 inside the crystal
    b: complex           # Delta_eps_{+1} = Delta_eps_{-1} inside, before strain
    g: complex           # common per-step phase exp(i (dz^ c mod 2 pi))
    q: np.ndarray        # transverse wave numbers in units of k, fft order
    delta_plus: np.ndarray
    delta_minus: np.ndarray
    prop_plus: np.ndarray    # exp(i dz^ delta_+(q)), applied to psi_+
    prop_minus: np.ndarray   # exp(i dz^ delta_-(q)), applied to psi_-


def wavelength_um(energy_ev: float) -> float:
    lam_angstrom = HC_EV_ANGSTROM / energy_ev
    return lam_angstrom * 1e-4


def sin_bragg(energy_ev: float, e_ref_ev: float, theta_b_ref_rad: float) -> float:
    """s(E) = lambda(E) / (2 d) with d fixed by the Bragg angle at E_ref.

    lambda is proportional to 1/E, so s(E) = sin(theta_B(E_ref)) E_ref / E.
    """
    return math.sin(theta_b_ref_rad) * (e_ref_ev / energy_ev)


def d_spacing_um(e_ref_ev: float, theta_b_ref_rad: float) -> float:
    """Lattice-plane spacing implied by Bragg's law at the reference energy."""
    return wavelength_um(e_ref_ev) / (2.0 * math.sin(theta_b_ref_rad))


def energy_plan(energy_ev: float, e_ref_ev: float, theta_b_ref_rad: float,
                chi0: complex, chih: complex, nx: int, dx_um: float,
                dz_um: float) -> EnergyPlan:
    """All per-energy constants of one first-order step (Eqs. fov4-fov12)."""
    lam = wavelength_um(energy_ev)
    k = TWO_PI / lam
    s = sin_bragg(energy_ev, e_ref_ev, theta_b_ref_rad)
    c = math.sqrt((1.0 - s) * (1.0 + s))
    dzh = k * dz_um
    dxh = k * dx_um

    # Jacobi-Anger coefficients, Eqs. fov11-fov12 with z^ read as dz^.
    w = dzh * complex(chih) / c
    phi0 = dzh * complex(chi0) / (2.0 * c)
    e_phi0 = complex(math.exp(-phi0.imag) * math.cos(phi0.real),
                     math.exp(-phi0.imag) * math.sin(phi0.real))
    a = bessel_series(0, w) * e_phi0
    b = 1j * bessel_series(1, w) * e_phi0

    # Angular-spectrum propagators of Eq. fov10, each centred on its carrier.
    q = TWO_PI * dft.fftfreq(nx, dxh)
    root_plus = np.sqrt(1.0 - (q + s) ** 2)
    root_minus = np.sqrt(1.0 - (q - s) ** 2)
    delta_plus = -q * (q + 2.0 * s) / (root_plus + c)
    delta_minus = -q * (q - 2.0 * s) / (root_minus + c)
    prop_plus = np.exp(1j * dzh * delta_plus)
    prop_minus = np.exp(1j * dzh * delta_minus)
    gphase = math.fmod(dzh * c, TWO_PI)
    g = complex(math.cos(gphase), math.sin(gphase))
    return EnergyPlan(energy_ev, k, s, c, dzh, dxh, w, phi0, a, b, g, q,
                      delta_plus, delta_minus, prop_plus, prop_minus)


# --------------------------------------------------------------------------
# The march (Eq. fov10)
# --------------------------------------------------------------------------

@dataclass
class MarchResult:
    psi: np.ndarray       # [B][2][N] complex128 after the last step
    records: np.ndarray   # [B][n_rec][2][N] complex128
    powers: np.ndarray    # [B][n_rec + 1][2] float64, dx * sum |psi|^2


FOREST_RUTH_T = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))   # 1.3512..., printed as 1.3512


def split_stages(method: str) -> list[tuple[float, float]]:
    """Stage coefficients (a_i, b_i) of the operator splitting of Eq.
    split-op: the step applies A(a_1 dz), B(b_1 dz), A(a_2 dz), B(b_2 dz), ...
    in that order, A the angular-spectrum propagation and B the coupling.
    first_order: a = (1), b = (1) -- Eq. fov10 itself;
    verlet:      a = (0, 1), b = (1/2, 1/2);
    forest_ruth: a = (0, t, 1 - 2t, t), b = (t/2, (1-t)/2, (1-t)/2, t/2),
                 t = 1 / (2 - 2^(1/3)) (the paper prints t = 1.3512)."""
    if method == "first_order":
        return [(1.0, 1.0)]
    if method == "verlet":
        return [(0.0, 0.5), (1.0, 0.5)]
    if method == "forest_ruth":
        t = FOREST_RUTH_T
        return [(0.0, t / 2.0), (t, (1.0 - t) / 2.0), (1.0 - 2.0 * t, (1.0 - t) / 2.0),
                (t, t / 2.0)]
    raise ValueError(f"unknown splitting method {method}")


def coupling_coefficients(plan: "EnergyPlan", frac: float, chi0: complex, chih: complex
                          ) -> tuple[complex, complex]:
    """(Delta_eps_0, Delta_eps_+-1) of Eqs. fov11-fov12 for a coupling step
    of frac * dz (frac = b_i of Eq. split-op)."""
    w = frac * plan.dzh * complex(chih) / plan.c
    phi0 = frac * plan.dzh * complex(chi0) / (2.0 * plan.c)
    e_phi0 = complex(math.exp(-phi0.imag) * math.cos(phi0.real),
                     math.exp(-phi0.imag) * math.sin(phi0.real))
    return bessel_series(0, w) * e_phi0, 1j * bessel_series(1, w) * e_phi0


def band_power(psi: np.ndarray, dx_um: float) -> np.ndarray:
    """P = dx * sum_j |psi_j|^2 along the last axis."""
    return dx_um * np.sum(psi.real ** 2 + psi.imag ** 2, axis=-1)


def march(plans: list[EnergyPlan], psi0: np.ndarray, slices, n_begin: int,
          n_end: int, record_every: int, dx_um: float,
          prop_override: tuple[np.ndarray, np.ndarray] | None = None,
          method: str = "first_order", chi: tuple[complex, complex] | None = None
          ) -> MarchResult:
    """Advance psi0 (state after ``n_begin`` steps) to the state after ``n_end``.

    plans   : one EnergyPlan per batch row (photon energy).
    psi0    : [B][2][N] complex; band 0 = psi_+, band 1 = psi_-.
    slices  : callable n -> (inside bool[N], theta float64[N]) giving the
              mask Pi and the strain phase h*u_x at z_n = n dz.  Mask and
              strain do not depend on the photon energy.
    record_every : record psi after step n (0-based) when
              (n + 1) % record_every == 0; 0 disables records.  Records are
              indexed by (n + 1) // record_every - 1 over the whole march
              [0, n_end), so a resumed march fills the later slots.
    prop_override : optional (P+, P-) replacing exp(i dz^ delta_+-) (same
              table for every row); used only by the gauge-identity test.
    method  : operator splitting of Eq. split-op (see ``split_stages``); the
              stages of step n all use the mask and strain of z_n (the
              equation evaluates delta_eps at the step's z^).  Higher orders
              need ``chi`` = (chi_0, chi_h) to form the fractional couplings.

    Powers: row r, record i holds the two band powers at that record; the
    last entry holds the powers of the returned state.
    """
    psi0 = np.asarray(psi0, dtype=np.complex128)
    nb, nbands, n = psi0.shape
    assert nbands == 2 and len(plans) == nb
    n_rec = (n_end // record_every) if record_every > 0 else 0
    records = np.zeros((nb, n_rec, 2, n), dtype=np.complex128)
    powers = np.zeros((nb, n_rec + 1, 2), dtype=np.float64)

    if prop_override is None:
        prop_p = np.stack([p.prop_plus for p in plans])
        prop_m = np.stack([p.prop_minus for p in plans])
    else:
        prop_p = np.broadcast_to(prop_override[0], (nb, n))
        prop_m = np.broadcast_to(prop_override[1], (nb, n))
    g = np.array([p.g for p in plans])[:, None]
    a = np.array([p.a for p in plans])[:, None]
    b = np.array([p.b for p in plans])[:, None]

    # stages: (propagator pair or None, common-phase factor, a, b) per row.
    # A stage of a_i dz propagates with g^{a_i} exp(i a_i dz^ delta_+-); the
    # factors g^{a_i} multiply both bands, commute with the coupling and
    # multiply to g per step (sum a_i = 1), so higher-order schemes apply g
    # once, after the step's last stage.
    stages = []
    if method == "first_order":
        stages.append(((prop_p, prop_m), g[:, :, None], a, b))
    else:
        chi0, chih = chi
        for frac_a, frac_b in split_stages(method):
            props = None
            if frac_a != 0.0:
                props = (np.stack([np.exp(1j * frac_a * p.dzh * p.delta_plus) for p in plans]),
                         np.stack([np.exp(1j * frac_a * p.dzh * p.delta_minus) for p in plans]))
            ab = [coupling_coefficients(p, frac_b, chi0, chih) for p in plans]
            stages.append((props, 1.0, np.array([x[0] for x in ab])[:, None],
                           np.array([x[1] for x in ab])[:, None]))

    # band axis 1: psi[:, 0] = psi_+, psi[:, 1] = psi_-; each band's
    # propagator table sits at the same index of the stacked tables.
    stage_props = [None if props is None else np.stack(props, axis=1)
                   for props, _, _, _ in stages]
    psi = psi0.copy()
    for step in range(n_begin, n_end):
        inside, theta = slices(step)
        e_plus = np.exp(1j * theta)     # exp(+i h u_x) on Delta_eps'_{+1}
        e_minus = np.exp(-1j * theta)   # exp(-i h u_x) on Delta_eps'_{-1}
        for (_, gs, a_s, b_s), props in zip(stages, stage_props):
            if props is not None:
                # Free propagation of each envelope through its own band operator.
                psi = dft.ifft(dft.fft(psi) * props) * gs
            psi_p, psi_m = psi[:, 0], psi[:, 1]
            # Real-space coupling through chi_0, chi_h, the strain phase and Pi.
            new_p = np.where(inside, a_s * psi_p + b_s * e_plus * psi_m, psi_p)
            new_m = np.where(inside, a_s * psi_m + b_s * e_minus * psi_p, psi_m)
            psi = np.stack([new_p, new_m], axis=1)
        if method != "first_order":
            psi = psi * g[:, :, None]
        psi_p, psi_m = psi[:, 0], psi[:, 1]
        if record_every > 0 and (step + 1) % record_every == 0:
            slot = (step + 1) // record_every - 1
            records[:, slot, 0, :] = psi_p
            records[:, slot, 1, :] = psi_m
            powers[:, slot, 0] = band_power(psi_p, dx_um)
            powers[:, slot, 1] = band_power(psi_m, dx_um)
    psi_p, psi_m = psi[:, 0], psi[:, 1]
    powers[:, n_rec, 0] = band_power(psi_p, dx_um)
    powers[:, n_rec, 1] = band_power(psi_m, dx_um)
    return MarchResult(np.stack([psi_p, psi_m], axis=1), records, powers)


def rel_l2(x: np.ndarray, ref: np.ndarray) -> float:
    """||x - ref||_2 / ||ref||_2 over all elements."""
    num = np.linalg.norm((np.asarray(x) - np.asarray(ref)).ravel())
    den = np.linalg.norm(np.asarray(ref).ravel())
    return float(num / den) if den > 0 else float(num)
