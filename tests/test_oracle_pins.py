"""Pins of the FP64 oracle against things other than itself.

Each test fixes part of ``oracle/`` with a closed form, a textbook law, an
invariant of the equations, brute force, or an independent library routine,
chosen so that a plausible slip (a dropped factor, a wrong sign or index, a
swapped band) fails at least one of them.  None of them needs a GPU.
"""

import math

import numpy as np
import pytest
import scipy.special

from oracle import bpm, geometry, timeaxis
from oracle import fft as dft

E = 8000.0
THETA = math.radians(23.65)
CHI0 = complex(-1.51e-5, 3.5e-7)
CHIH = complex(-9.1e-6, 3.4e-7)


def _plan(nx, dx, dz, chi0=CHI0, chih=CHIH, energy=E):
    return bpm.energy_plan(energy, E, THETA, chi0, chih, nx, dx, dz)


def _crystal(nx, x0, dx, dz, kind):
    cr = geometry.Crystal(nx, x0, dx, dz, bpm.d_spacing_um(E, THETA))
    return cr.set_crystal(kind)


# ---------------------------------------------------------------- P1 -------
def test_p1_fft_convention_and_q_grid():
    """The oracle's own transforms (``oracle.fft``): the O(N^2) definition
    and the radix-2 FFT equal a brute-force sum with the e^{-2 pi i m j/N}
    kernel written out term by term here (N = 8..512) and numpy's FFT, an
    independent library routine (N up to 16384); the inverse undoes the
    forward transform.  The oracle's q_m is the wave number of DFT bin m:
    a sampled plane wave exp(i q_m x^) transforms to a single spike at m."""
    rng = np.random.default_rng(1)
    for n in (8, 16, 64, 256, 512):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        brute = np.zeros(n, dtype=np.complex128)
        for m in range(n):
            for j in range(n):
                ang = -2.0 * math.pi * ((m * j) % n) / n
                brute[m] += x[j] * complex(math.cos(ang), math.sin(ang))
        assert np.max(np.abs(dft.fft(x) - brute)) <= 1e-13 * np.max(np.abs(brute))
    for n in (8, 256, 512, 1024, 4096, 16384):
        x = rng.standard_normal((3, 2, n)) + 1j * rng.standard_normal((3, 2, n))
        ref = np.fft.fft(x, axis=-1)
        assert np.max(np.abs(dft.fft(x) - ref)) <= 2e-15 * np.max(np.abs(ref))
        assert np.max(np.abs(dft.ifft(ref) - x)) <= 2e-15 * np.max(np.abs(x))
        assert np.array_equal(dft.fftfreq(n, 0.37), np.fft.fftfreq(n, 0.37))
    y = rng.standard_normal((3, 32, 512)) + 1j * rng.standard_normal((3, 32, 512))
    assert np.max(np.abs(dft.fft2(y) - np.fft.fft2(y))) <= 1e-14 * np.max(np.abs(np.fft.fft2(y)))
    nx, dx = 64, 0.3
    p = _plan(nx, dx, 0.05)
    xh = p.k_um * (-7.0 + np.arange(nx) * dx)
    for m in (0, 1, 5, nx // 2 - 1, nx // 2, nx // 2 + 3, nx - 1):
        spec = dft.fft(np.exp(1j * p.q[m] * xh))
        others = np.delete(np.abs(spec), m)
        assert abs(abs(spec[m]) - nx) < 1e-9 and np.max(others) < 1e-9


# ---------------------------------------------------------------- P2 -------
def _angular_spectrum_closed_form(xh_eval, sigma_h, xh_c, s, dzh_total):
    """(1/2pi) int A(q) exp(i q x^) exp(i Z^ sqrt(1 - (q + s)^2)) dq for the
    Gaussian psi(x^) = exp(-(x^ - x^_c)^2 / (2 sigma^2)), by a fine
    trapezoid rule in q, with the exponent taken in 40-digit arithmetic."""
    import mpmath
    mpmath.mp.dps = 40
    nq = 6001
    qmax = 14.0 / sigma_h
    q = np.linspace(-qmax, qmax, nq)
    hq = q[1] - q[0]
    amp = sigma_h * math.sqrt(2.0 * math.pi) * np.exp(-0.5 * (q * sigma_h) ** 2)
    prop = np.empty(nq, dtype=np.complex128)
    s_mp = mpmath.mpf(s)
    z_mp = mpmath.mpf(dzh_total)
    for i, qi in enumerate(q):
        ph = z_mp * mpmath.sqrt(1 - (mpmath.mpf(qi) + s_mp) ** 2)
        ph = ph - 2 * mpmath.pi * mpmath.floor(ph / (2 * mpmath.pi))
        prop[i] = complex(mpmath.cos(ph), mpmath.sin(ph))
    out = []
    for xh in xh_eval:
        integrand = amp * np.exp(1j * q * (xh - xh_c)) * prop
        out.append(hq * np.sum(integrand) / (2.0 * math.pi))
    return np.array(out)


def test_p2_free_space_gaussian_matches_angular_spectrum_integral():
    """Pi = 0: the march is pure angular-spectrum propagation of psi_+.
    Compare with the continuum integral (exact square root, no delta split,
    no global-phase split).  Fixes the propagator's sign and centring on
    +s, dz^ = k dz, the q grid and the per-step common phase g."""
    nx, dx, dz, nsteps = 1024, 0.4, 0.05, 400
    x0 = -0.5 * nx * dx
    sigma = 10.0
    p = _plan(nx, dx, dz)
    x = x0 + np.arange(nx) * dx
    psi0 = np.zeros((1, 2, nx), dtype=complex)
    psi0[0, 0] = np.exp(-0.5 * ((x + 3.0) / sigma) ** 2)
    cr = _crystal(nx, x0, dx, dz, geometry.CRYSTAL_VACUUM)
    res = bpm.march([p], psi0, cr, 0, nsteps, 0, dx)
    drift = nsteps * dz * math.tan(THETA)
    idx = np.searchsorted(x, np.linspace(-3.0 + drift - 20, -3.0 + drift + 20, 16))
    ref = _angular_spectrum_closed_form(p.k_um * x[idx], p.k_um * sigma,
                                        p.k_um * (-3.0), p.s, nsteps * p.dzh)
    got = res.psi[0, 0, idx]
    # g is rounded once per step (|error| <= ulp(dz^ c)/2 = 1.2e-13 rad).
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(res.psi[0, 1])) == 0.0


def test_p2_free_space_drift_is_along_plus_x_at_tan_theta():
    """The + envelope is the beam travelling at +theta_B to z: its intensity
    centroid moves by z tan(theta_B) (ray optics), the - envelope's by
    -z tan(theta_B)."""
    nx, dx, dz, nsteps = 512, 0.4, 0.05, 1000
    x0 = -0.5 * nx * dx
    p = _plan(nx, dx, dz)
    x = x0 + np.arange(nx) * dx
    g = np.exp(-0.5 * (x / 8.0) ** 2)
    psi0 = np.stack([g, g])[None].astype(complex)
    cr = _crystal(nx, x0, dx, dz, geometry.CRYSTAL_VACUUM)
    res = bpm.march([p], psi0, cr, 0, nsteps, 0, dx)
    for band, sign in ((0, 1.0), (1, -1.0)):
        inten = np.abs(res.psi[0, band]) ** 2
        cen = np.sum(x * inten) / np.sum(inten)
        assert abs(cen - sign * nsteps * dz * math.tan(THETA)) < 1e-6


def test_p2b_free_space_power_is_conserved():
    """Parseval with |P+-| = 1: vacuum conserves each band's power."""
    nx, dx, dz = 256, 0.4, 0.05
    rng = np.random.default_rng(2)
    psi0 = (rng.standard_normal((1, 2, nx)) + 1j * rng.standard_normal((1, 2, nx)))
    cr = _crystal(nx, -50.0, dx, dz, geometry.CRYSTAL_VACUUM)
    res = bpm.march([_plan(nx, dx, dz)], psi0, cr, 0, 300, 100, dx)
    p0 = bpm.band_power(psi0[0], dx)
    for rec in range(4):
        assert np.allclose(res.powers[0, rec], p0, rtol=300 * 1e-13, atol=0)


# ---------------------------------------------------------------- P3 -------
def test_p3_single_mode_is_a_2x2_matrix_power():
    """One grid mode q_m in both bands, Pi = 1, no strain: the step is the
    2x2 map v -> [[a, b], [b, a]] diag(g P+(m), g P-(m)) v.  Compare the
    march (FFTs, masks, records) with the matrix power."""
    nx, dx, dz, nsteps = 32, 0.5, 0.05, 250
    x0 = -8.0
    p = _plan(nx, dx, dz)
    xh = p.k_um * (x0 + np.arange(nx) * dx)
    for m in (0, 3, nx - 2, nx // 2):
        mode = np.exp(1j * p.q[m] * xh)
        v0 = np.array([0.7 - 0.2j, 0.1 + 0.4j])
        psi0 = np.stack([v0[0] * mode, v0[1] * mode])[None]
        cr = _crystal(nx, x0, dx, dz, geometry.CRYSTAL_BULK)
        res = bpm.march([p], psi0, cr, 0, nsteps, 0, dx)
        mat = np.array([[p.a, p.b], [p.b, p.a]]) @ np.diag(
            [p.g * p.prop_plus[m], p.g * p.prop_minus[m]])
        v = np.linalg.matrix_power(mat, nsteps) @ v0
        got = res.psi[0] / mode
        assert np.max(np.abs(got - v[:, None])) < 1e-12


# ---------------------------------------------------------------- P4 -------
def test_p4_pendelloesung_period_symmetric_laue():
    """Plane wave at the exact Bragg angle in a perfect symmetric Laue
    crystal (no absorption): the reflected fraction follows the textbook
    Pendelloesung law sin^2(pi z / Lambda0), Lambda0 = lambda cos(theta_B)
    / |chi_h| (15.6 um here).  The truncated expansion (Eqs. fov11-12)
    deviates by O(w^3) per step, < 1e-3 over two periods at dz = 0.05 um."""
    nx, dx, dz, nsteps = 16, 1.0, 0.05, 700
    chi0, chih = complex(-1.51e-5, 0.0), complex(-9.1e-6, 0.0)
    p = _plan(nx, dx, dz, chi0, chih)
    psi0 = np.zeros((1, 2, nx), dtype=complex)
    psi0[0, 0] = 1.0
    cr = _crystal(nx, 0.0, dx, dz, geometry.CRYSTAL_BULK)
    res = bpm.march([p], psi0, cr, 0, nsteps, 1, dx)
    pw = res.powers[0, :nsteps]
    frac = pw[:, 1] / (pw[:, 0] + pw[:, 1])
    lam = bpm.HC_EV_ANGSTROM / E * 1e-4
    lam0 = lam * math.cos(THETA) / abs(chih)
    assert abs(lam0 - 15.60) < 0.01
    z = dz * np.arange(1, nsteps + 1)
    assert np.max(np.abs(frac - np.sin(np.pi * z / lam0) ** 2)) < 1e-3


def test_p5_laue_rocking_curve_matches_two_beam_theory():
    """Rocking curve of a non-absorbing symmetric Laue crystal.  A comb of
    plane waves exp(i q_m x^), one per grid mode, enters psi_+; in a perfect
    crystal the modes do not mix, and two-beam dynamical theory gives the
    reflected fraction of mode m after thickness Z^ = k T as
        R(q) = kappa^2 sin^2(Z^ Omega) / Omega^2,
        Omega^2 = kappa^2 + Delta^2,  kappa = |chi_h| / (2 cos theta_B),
        Delta = (sqrt(1 - (q + s)^2) - sqrt(1 - (q - s)^2)) / 2
    (Pendelloesung at q = 0, the angular width of the Darwin scale away from
    it).  Measured as |psi_-|^2 / (|psi_+|^2 + |psi_-|^2) per mode, which
    divides out the discretisation's uniform power factor (P6).  The grid
    spans Delta = -6.6 .. 6.8 kappa; first-order splitting leaves 2.6e-5 at
    dz = 0.02 um (1.6e-4 at 0.05, 6.5e-6 at 0.01: second order in dz)."""
    nx, dx, dz, thick = 64, 1.0, 0.02, 50.0
    nsteps = int(round(thick / dz))
    chi0, chih = complex(-1.51e-5, 0.0), complex(-9.1e-6, 0.0)
    p = _plan(nx, dx, dz, chi0, chih)
    k = 2.0 * math.pi / bpm.wavelength_um(E)
    q = 2.0 * math.pi * np.fft.fftfreq(nx, k * dx)
    xh = k * dx * np.arange(nx)
    psi0 = np.zeros((1, 2, nx), dtype=complex)
    psi0[0, 0] = np.exp(1j * q[:, None] * xh[None, :]).sum(axis=0)
    cr = _crystal(nx, 0.0, dx, dz, geometry.CRYSTAL_BULK)
    res = bpm.march([p], psi0, cr, 0, nsteps, 0, dx)
    fp = np.fft.fft(res.psi[0, 0]) / nx
    fm = np.fft.fft(res.psi[0, 1]) / nx
    got = np.abs(fm) ** 2 / (np.abs(fp) ** 2 + np.abs(fm) ** 2)
    s, c = math.sin(THETA), math.cos(THETA)
    kappa = abs(chih) / (2.0 * c)
    delta = 0.5 * (np.sqrt(1.0 - (q + s) ** 2) - np.sqrt(1.0 - (q - s) ** 2))
    omega = np.sqrt(kappa ** 2 + delta ** 2)
    want = kappa ** 2 * np.sin(omega * k * nsteps * dz) ** 2 / omega ** 2
    assert np.max(np.abs(got - want)) < 1e-4
    assert want.max() > 0.8 and np.abs(delta).max() > 6 * kappa


def _bragg_reflectivity(angles_urad, dz, nx=1024, dx=0.8, fwhm=100.0, march_um=1000.0):
    """Reflectivity of a thick symmetric Bragg slab (x in [0, 400] um) for a
    wide Gaussian beam turned by each angle offset: P_- at the end of the
    march over the incident P_+."""
    nz = int(round(march_um / dz))
    chi0, chih = complex(-1.51e-5, 3.5e-7), complex(-9.1e-6, 3.4e-7)
    x0 = -0.75 * nx * dx
    s, c = math.sin(THETA), math.cos(THETA)
    k = 2.0 * math.pi / bpm.wavelength_um(E)
    xb = -s / c * 0.35 * march_um            # hits x = 0 at 35 % of the march
    x = x0 + dx * np.arange(nx)
    psi0 = np.zeros((len(angles_urad), 2, nx), complex)
    for i, a in enumerate(angles_urad):
        psi0[i, 0] = np.exp(-2.0 * math.log(2.0) * ((x - xb) / (fwhm / c)) ** 2) * np.exp(
            1j * k * c * a * 1e-6 * (x - xb))
    plans = [_plan(nx, dx, dz, chi0, chih) for _ in angles_urad]
    cr = geometry.Crystal(nx, x0, dx, dz, bpm.d_spacing_um(E, THETA)).set_crystal(
        geometry.CRYSTAL_SLAB, asym_angle_rad=0.0, thickness_um=400.0)
    res = bpm.march(plans, psi0, cr, 0, nz, 0, dx)
    return res.powers[:, -1, 1] / (dx * np.sum(np.abs(psi0[:, 0]) ** 2, axis=-1))


def test_p5b_bragg_darwin_curve():
    """Thick symmetric Bragg crystal against the two-beam (Darwin-Prins)
    reflectivity with absorption: R = min |eta -+ sqrt(eta^2 - 1)|^2,
    eta = (-dtheta sin 2 theta_B - chi_0) / sqrt(chi_h chi_-h) (chi_-h = chi_h
    for a centrosymmetric crystal): total reflection over a width
    2|chi_h|/sin 2 theta_B = 24.8 urad centred at the refraction shift
    -chi_0'/sin 2 theta_B = +20.5 urad.  The march's truncated coupling loses
    power at O(dz) (P6), so the reflectivity is extrapolated to dz -> 0 from
    dz = 0.2 and 0.1 um (first order); a 100 um beam diverges by < 1 urad.
    The tail point and the plateau then agree to 1 % (the steep edges,
    where a fraction of a microradian matters, are not compared)."""
    angles = [2.0, 14.0, 20.0, 26.0]
    r1 = _bragg_reflectivity(angles, 0.2)
    r2 = _bragg_reflectivity(angles, 0.1)
    got = 2.0 * r2 - r1
    chi0, chih = complex(-1.51e-5, 3.5e-7), complex(-9.1e-6, 3.4e-7)
    th = np.array(angles) * 1e-6
    eta = (-th * math.sin(2.0 * THETA) - chi0) / np.sqrt(chih * chih)
    root = np.sqrt(eta ** 2 - 1.0 + 0j)
    want = np.minimum(np.abs(eta - root) ** 2, np.abs(eta + root) ** 2)
    assert np.all(np.abs(got - want) <= 0.01 * np.maximum(want, 0.1)), (got, want)
    assert got[0] < 0.2 and min(got[1:]) > 0.85       # refraction shift is +20 urad


def _laue_modes_error(method, dz, thick=50.0):
    """max over grid modes of |R - R_two_beam| (the P5 problem)."""
    nx, dx = 64, 1.0
    nsteps = int(round(thick / dz))
    chi0, chih = complex(-1.51e-5, 0.0), complex(-9.1e-6, 0.0)
    p = _plan(nx, dx, dz, chi0, chih)
    k = 2.0 * math.pi / bpm.wavelength_um(E)
    q = 2.0 * math.pi * np.fft.fftfreq(nx, k * dx)
    xh = k * dx * np.arange(nx)
    psi0 = np.zeros((1, 2, nx), dtype=complex)
    psi0[0, 0] = np.exp(1j * q[:, None] * xh[None, :]).sum(axis=0)
    cr = _crystal(nx, 0.0, dx, dz, geometry.CRYSTAL_BULK)
    res = bpm.march([p], psi0, cr, 0, nsteps, 0, dx, method=method, chi=(chi0, chih))
    fp = np.fft.fft(res.psi[0, 0]) / nx
    fm = np.fft.fft(res.psi[0, 1]) / nx
    got = np.abs(fm) ** 2 / (np.abs(fp) ** 2 + np.abs(fm) ** 2)
    s, c = math.sin(THETA), math.cos(THETA)
    kappa = abs(chih) / (2.0 * c)
    delta = 0.5 * (np.sqrt(1.0 - (q + s) ** 2) - np.sqrt(1.0 - (q - s) ** 2))
    omega = np.sqrt(kappa ** 2 + delta ** 2)
    want = kappa ** 2 * np.sin(omega * k * nsteps * dz) ** 2 / omega ** 2
    return float(np.max(np.abs(got - want)))


def test_p12_splitting_coefficients():
    """Eq. split-op's schemes are consistent (sum a = sum b = 1), symmetric
    (palindromic in the application order A(a1) B(b1) A(a2) ...), and
    Forest-Ruth's t solves its fourth-order condition 2 t^3 + (1 - 2t)^3 = 0."""
    for m in ("first_order", "verlet", "forest_ruth"):
        st = bpm.split_stages(m)
        assert abs(sum(a for a, _ in st) - 1.0) < 1e-15
        assert abs(sum(b for _, b in st) - 1.0) < 1e-15
    for m in ("verlet", "forest_ruth"):
        seq = [x for a, b in bpm.split_stages(m) for x in (a, b)][1:]   # drop A(0)
        assert np.allclose(seq, seq[::-1])
    t = bpm.FOREST_RUTH_T
    assert abs(2.0 * t ** 3 + (1.0 - 2.0 * t) ** 3) < 1e-14
    assert abs(t - 1.3512) < 1e-4


def test_p12_higher_order_splitting_on_the_laue_rocking_curve():
    """The P5 problem marched with each scheme of Eq. split-op.  All three
    converge to the two-beam result at second order in dz (the truncated
    Jacobi-Anger coupling of Eqs. fov11-12 is not an exact flow: its angle
    per step is w/2 + w^3/48 + ..., which caps every scheme at O(dz^2));
    at dz = 0.05 um the errors are 1.6e-4 (first order), 8.2e-5 (Verlet) and
    9.9e-5 (Forest-Ruth)."""
    err = {m: [_laue_modes_error(m, dz) for dz in (0.05, 0.025)]
           for m in ("first_order", "verlet", "forest_ruth")}
    for m, (e1, e2) in err.items():
        assert e1 < 2e-4, (m, e1)
        assert 3.5 < e1 / e2 < 4.5, (m, e1 / e2)
    assert err["verlet"][0] < err["first_order"][0] / 1.8
    assert err["verlet"][0] < err["forest_ruth"][0] < err["first_order"][0]


def test_p4b_beer_lambert_and_refraction_phase():
    """chi_h = 0, uniform field in bulk: the wave only refracts and is
    absorbed.  Intensity falls as exp(-mu z / cos(theta_B)) with
    mu = 4 pi beta / lambda, beta = Im(chi_0)/2, and the phase (after the
    vacuum phase g^n) advances by k (Re chi_0 / 2) z / cos(theta_B)."""
    nx, dx, dz, nsteps = 8, 1.0, 0.05, 2000
    chi0 = complex(-1.51e-5, 3.5e-7)
    p = _plan(nx, dx, dz, chi0, 0j)
    psi0 = np.zeros((1, 2, nx), dtype=complex)
    psi0[0, 0] = 1.0
    cr = _crystal(nx, 0.0, dx, dz, geometry.CRYSTAL_BULK)
    res = bpm.march([p], psi0, cr, 0, nsteps, 0, dx)
    lam = bpm.HC_EV_ANGSTROM / E * 1e-4
    z = nsteps * dz
    mu = 4.0 * math.pi * (chi0.imag / 2.0) / lam
    assert abs(abs(res.psi[0, 0, 0]) ** 2 / math.exp(-mu * z / math.cos(THETA)) - 1) < 1e-12
    phase = np.angle(res.psi[0, 0, 0] / p.g ** nsteps)
    expect = math.remainder(2 * math.pi / lam * chi0.real / 2 * z / math.cos(THETA),
                            2 * math.pi)
    assert abs(phase - expect) < 1e-10


# ---------------------------------------------------------------- P6 -------
def test_p6_zero_absorption_power_law():
    """Real chi_0, chi_h, Pi = 1 everywhere, arbitrary beam and strain: the
    coupling matrix M satisfies M^H M = (J0(w)^2 + J1(w)^2) I for any strain
    phase, so the total power after n steps is sigma^n P_0 exactly (sigma
    from scipy's Bessel functions, independent of the oracle's series)."""
    nx, dx, dz, nsteps = 128, 0.4, 0.05, 300
    chi0, chih = complex(-1.51e-5, 0.0), complex(-9.1e-6, 0.0)
    p = _plan(nx, dx, dz, chi0, chih)
    rng = np.random.default_rng(3)
    psi0 = rng.standard_normal((1, 2, nx)) + 1j * rng.standard_normal((1, 2, nx))
    cr = _crystal(nx, -25.0, dx, dz, geometry.CRYSTAL_BULK)
    ux = rng.uniform(-1e-3, 1e-3, (nsteps, nx))
    cr.set_strain(geometry.STRAIN_ARRAY, ux=ux)
    res = bpm.march([p], psi0, cr, 0, nsteps, 100, dx)
    w = p.dzh * chih.real / p.c
    sigma = scipy.special.jv(0, w) ** 2 + scipy.special.jv(1, w) ** 2
    p0 = np.sum(bpm.band_power(psi0[0], dx))
    for rec, n in enumerate((100, 200, 300)):
        assert abs(np.sum(res.powers[0, rec]) / (sigma ** n * p0) - 1) < 1e-12


# ---------------------------------------------------------------- P7 -------
def test_p7_strain_gauge_identity():
    """A commensurate linear strain phase theta = G x^ (G k dx = 2 pi m0/N)
    is a gauge: (psi_+, e^{i theta} psi_-) follows the unstrained march with
    psi_-'s propagator shifted by m0 bins.  Fixes which band gets e^{+i
    theta} and that the strain phase multiplies Delta_eps_{+-1} only."""
    nx, dx, dz, nsteps, m0 = 64, 0.4, 0.05, 120, 3
    x0 = -12.0
    p = _plan(nx, dx, dz)
    x = x0 + np.arange(nx) * dx
    gk = 2 * np.pi * m0 / (nx * dx)                   # theta = gk * x
    rng = np.random.default_rng(4)
    psi0 = (rng.standard_normal((1, 2, nx)) + 1j * rng.standard_normal((1, 2, nx)))
    inside = rng.uniform(size=(nsteps, nx)) < 0.7
    h = 2 * np.pi / bpm.d_spacing_um(E, THETA)

    cr_s = geometry.Crystal(nx, x0, dx, dz, bpm.d_spacing_um(E, THETA))
    cr_s.set_crystal(geometry.CRYSTAL_MASK, mask=inside)
    cr_s.set_strain(geometry.STRAIN_ARRAY, ux=np.tile(gk * x / h, (nsteps, 1)))
    strained = bpm.march([p], psi0, cr_s, 0, nsteps, 0, dx)

    cr_u = geometry.Crystal(nx, x0, dx, dz, bpm.d_spacing_um(E, THETA))
    cr_u.set_crystal(geometry.CRYSTAL_MASK, mask=inside)
    gauge = np.exp(1j * gk * x)
    psi0_g = psi0.copy()
    psi0_g[0, 1] *= gauge
    plain = bpm.march([p], psi0_g, cr_u, 0, nsteps, 0, dx,
                      prop_override=(p.prop_plus, np.roll(p.prop_minus, m0)))
    assert np.max(np.abs(strained.psi[0, 0] - plain.psi[0, 0])) < 1e-12
    assert np.max(np.abs(strained.psi[0, 1] * gauge - plain.psi[0, 1])) < 1e-12


# ---------------------------------------------------------------- P8 -------
def test_p8_one_lattice_spacing_is_invisible():
    """u_x -> u_x + d changes h u_x by exactly 2 pi."""
    nx, dx, dz, nsteps = 64, 0.4, 0.05, 50
    p = _plan(nx, dx, dz)
    d = bpm.d_spacing_um(E, THETA)
    rng = np.random.default_rng(5)
    psi0 = rng.standard_normal((1, 2, nx)) + 0j
    ux = rng.uniform(-0.01, 0.01, (nsteps, nx))
    runs = []
    for shift in (0.0, d, -3 * d):
        cr = geometry.Crystal(nx, -10.0, dx, dz, d).set_crystal(geometry.CRYSTAL_BULK)
        cr.set_strain(geometry.STRAIN_ARRAY, ux=ux + shift)
        runs.append(bpm.march([p], psi0, cr, 0, nsteps, 0, dx).psi)
    assert np.max(np.abs(runs[1] - runs[0])) < 1e-12
    assert np.max(np.abs(runs[2] - runs[0])) < 1e-12


# ---------------------------------------------------------------- P9 -------
@pytest.mark.parametrize("w", [0.0201 - 0.00075j, -0.02014 + 0.00075j, 0.3 + 0.2j,
                               1e-9 + 0j, 0j, 1.7 - 0.4j])
def test_p9_bessel_series_matches_scipy(w):
    for nu in (0, 1):
        ref = scipy.special.jv(nu, w)
        got = bpm.bessel_series(nu, w)
        assert abs(got - ref) <= 2e-15 * max(1.0, abs(ref))
    # J0 - 1 without cancellation, against 40-digit mpmath.
    import mpmath
    mpmath.mp.dps = 40
    ref_m1 = complex(mpmath.besselj(0, mpmath.mpc(w.real, w.imag)) - 1)
    got_m1 = bpm.bessel_series(0, w, skip_first=True)
    assert abs(got_m1 - ref_m1) <= 1e-15 * abs(ref_m1) + 1e-300


# ---------------------------------------------------------------- P10 ------
def test_p10_linearity_and_batch_independence():
    nx, dx, dz, nsteps = 64, 0.4, 0.05, 60
    rng = np.random.default_rng(6)
    psi_a = rng.standard_normal((1, 2, nx)) + 1j * rng.standard_normal((1, 2, nx))
    psi_b = rng.standard_normal((1, 2, nx)) + 1j * rng.standard_normal((1, 2, nx))
    cr = _crystal(nx, -12.0, dx, dz, geometry.CRYSTAL_BULK)
    cr.set_strain(geometry.STRAIN_BENT, params=[1e5, 0.28, 0.0, 0.0])
    pa, pb = _plan(nx, dx, dz), _plan(nx, dx, dz, energy=8003.0)
    alpha = 0.3 - 1.7j
    ra = bpm.march([pa], psi_a, cr, 0, nsteps, 0, dx).psi
    r_scaled = bpm.march([pa], alpha * psi_a, cr, 0, nsteps, 0, dx).psi
    assert np.max(np.abs(r_scaled - alpha * ra)) < 1e-13 * np.max(np.abs(r_scaled))
    rb = bpm.march([pb], psi_b, cr, 0, nsteps, 0, dx).psi
    both = bpm.march([pa, pb], np.concatenate([psi_a, psi_b]), cr, 0, nsteps, 0, dx).psi
    assert np.array_equal(both[0], ra[0]) or np.max(np.abs(both[0] - ra[0])) < 1e-14
    assert np.max(np.abs(both[1] - rb[0])) < 1e-14


def test_resume_equals_unsplit_march():
    """The state after n steps is (psi_+, psi_-): a march split at n equals
    the unsplit march, records included."""
    nx, dx, dz = 64, 0.4, 0.05
    rng = np.random.default_rng(9)
    psi0 = rng.standard_normal((1, 2, nx)) + 1j * rng.standard_normal((1, 2, nx))
    cr = _crystal(nx, -12.0, dx, dz, geometry.CRYSTAL_BULK)
    p = _plan(nx, dx, dz)
    full = bpm.march([p], psi0, cr, 0, 100, 10, dx)
    first = bpm.march([p], psi0, cr, 0, 40, 10, dx)
    second = bpm.march([p], first.psi, cr, 40, 100, 10, dx)
    assert np.array_equal(second.psi, full.psi)
    assert np.array_equal(second.records[:, 4:], full.records[:, 4:])


# ---------------------------------------------------------------- P11 ------
def test_p11_chi_h_sign_only_flips_psi_minus():
    """chi_h -> -chi_h sends b -> -b, which is the same as psi_- -> -psi_-:
    intensities of both bands are unchanged."""
    nx, dx, dz, nsteps = 64, 0.4, 0.05, 200
    rng = np.random.default_rng(7)
    psi0 = np.zeros((1, 2, nx), dtype=complex)
    psi0[0, 0] = rng.standard_normal(nx) + 1j * rng.standard_normal(nx)
    cr = _crystal(nx, -12.0, dx, dz, geometry.CRYSTAL_BULK)
    r1 = bpm.march([_plan(nx, dx, dz, chih=CHIH)], psi0, cr, 0, nsteps, 0, dx).psi
    r2 = bpm.march([_plan(nx, dx, dz, chih=-CHIH)], psi0, cr, 0, nsteps, 0, dx).psi
    assert np.max(np.abs(r1[0, 0] - r2[0, 0])) < 1e-13
    assert np.max(np.abs(r1[0, 1] + r2[0, 1])) < 1e-13


# ---------------------------------------------------- geometry pins ---------
def test_slab_bragg_laue_and_rotated_frame():
    nx, dx, dz = 200, 0.5, 0.25
    x0 = -50.0
    x = x0 + np.arange(nx) * dx
    # a = 0: Bragg slab x in [xs, xs + T] on every row.
    for n in (0, 7, 100):
        row = geometry.slab_row(x, n * dz, 0.0, 20.0, 3.0, 0.0)
        assert np.array_equal(row, (x >= 3.0) & (x <= 23.0))
    # a = 90 deg: Laue slab z in [zs, zs + T], whole rows.
    for n in range(0, 200, 13):
        row = geometry.slab_row(x, n * dz, math.pi / 2, 10.0, 0.0, 5.0)
        z = n * dz
        assert row.all() == (5.0 <= z <= 15.0) and (row.any() == row.all())
    # Any angle: same set as the distance to the surface line measured with
    # the cross product against the surface direction (independent form).
    a, t, xs, zs = math.radians(10.0), 30.0, 2.0, 20.0
    tdir = np.array([-math.sin(a), math.cos(a)])
    for n in range(0, 200, 7):
        z = n * dz
        row = geometry.slab_row(x, z, a, t, xs, zs)
        depth = (x - xs) * tdir[1] - (z - zs) * tdir[0]       # cross(t, r - rs)
        away = (np.abs(depth) > 1e-9) & (np.abs(depth - t) > 1e-9)
        assert np.array_equal(row[away], ((depth >= 0) & (depth <= t))[away])


def test_polygon_even_odd_matches_winding_number():
    rng = np.random.default_rng(8)
    from paper_2601_06340_gb300 import inputs
    poly = inputs.star_polygon(rng, (1.0, 2.0), 40.0, 7)
    x = -25.0 + 0.37 * np.arange(150)
    for z in np.linspace(-25.0, 25.0, 41):
        row = geometry.polygon_row(x, z, poly[:, 0], poly[:, 1])
        vx = poly[:, 0][None, :] - x[:, None]
        vz = poly[:, 1][None, :] - z
        ang = np.arctan2(vz, vx)
        dang = np.diff(np.concatenate([ang, ang[:, :1]], axis=1), axis=1)
        dang = (dang + np.pi) % (2 * np.pi) - np.pi
        winding = np.rint(np.sum(dang, axis=1) / (2 * np.pi)) != 0
        assert np.array_equal(row, winding)


def test_bent_displacement_curvatures():
    """Second derivatives of the bend field: d2u/dx2 = 1/R, d2u/dz2 = nu/R,
    and u = 0 at the reference point."""
    r, nu, xr, zr = 2.0e6, 0.28, 5.0, 40.0
    x = np.array([xr - 1.0, xr, xr + 1.0])
    u0 = geometry.bent_ux(x, zr, r, nu, xr, zr)
    assert u0[1] == 0.0
    assert abs((u0[0] - 2 * u0[1] + u0[2]) - 1.0 / r) < 1e-18
    uz = [geometry.bent_ux(np.array([xr]), zr + dzz, r, nu, xr, zr)[0]
          for dzz in (-1.0, 0.0, 1.0)]
    assert abs((uz[0] - 2 * uz[1] + uz[2]) - nu / r) < 1e-18


def test_edge_dislocation_burgers_circuit():
    """A closed circuit around the core gains exactly one Burgers vector in
    u_x; the elastic term vanishes on the axes through the core."""
    b, nu, xc, zc = 3.84e-4, 0.28, 1.0, -2.0
    ang = np.linspace(-np.pi + 1e-3, np.pi - 1e-3, 4001)
    rad = 5.0
    xs, zs = xc + rad * np.cos(ang), zc + rad * np.sin(ang)
    u = np.array([geometry.edge_dislocation_ux(np.array([xs[i]]), zs[i], b, nu, xc, zc)[0]
                  for i in range(len(ang))])
    jumps = np.diff(u)
    # continuous along the circuit except across the cut on -x'
    assert np.max(np.abs(jumps)) < 1e-3 * b
    # ... and the whole circuit's closure failure sits in the jump across
    # the cut, which is exactly one Burgers vector.
    eta = 1e-9
    up = geometry.edge_dislocation_ux(np.array([xc - rad]), zc + eta, b, nu, xc, zc)[0]
    dn = geometry.edge_dislocation_ux(np.array([xc - rad]), zc - eta, b, nu, xc, zc)[0]
    assert abs((up - dn) - b) < 1e-9 * b
    on_axis = geometry.edge_dislocation_ux(np.array([xc + 3.0, xc - 0.0]), zc, b, nu, xc, zc)
    assert on_axis[0] == 0.0 and on_axis[1] == 0.0


# ---------------------------------------------------- time axis -------------
# Physical constants typed here independently of the oracle's own.
C_UM_PER_FS = 0.299792458                  # speed of light, um / fs (exact)
HBAR_EV_FS = 6.62607015e-34 / 1.602176634e-19 * 1e15 / (2.0 * math.pi)


def _vacuum_pulse(n_energy=64, de=10.0 / 256, e0=9000.0, sigma_ev=0.1, nx=512, dx=0.5,
                  dz=0.1, nsteps=100, fwhm=60.0):
    """A transform-limited pulse (Gaussian spectrum, flat phase) crossing the
    origin at t = 0 along the Bragg direction of e0, marched through vacuum
    (chi = 0) by the oracle, one energy per row (theta_B per energy, fixed
    incident direction: row j's envelope tilt (sin theta_0 - s_j) k_j)."""
    energies = e0 + de * (np.arange(n_energy) - n_energy // 2)
    s0 = math.sin(THETA) * E / e0
    theta0 = math.asin(s0)
    x = (np.arange(nx) - nx // 2) * dx
    plans, psi0 = [], np.zeros((n_energy, 2, nx), dtype=np.complex128)
    for j, ej in enumerate(energies):
        p = bpm.energy_plan(float(ej), E, THETA, 0j, 0j, nx, dx, dz)
        plans.append(p)
        amp = math.exp(-((ej - e0) ** 2) / (4.0 * sigma_ev ** 2))
        beam = np.exp(-2.0 * math.log(2.0) * (x * math.cos(theta0)) ** 2 / fwhm ** 2)
        psi0[j, 0] = amp * beam * np.exp(1j * p.k_um * (s0 - p.s) * x)

    def vacuum(n):
        return np.zeros(nx, dtype=bool), np.zeros(nx)
    out = bpm.march(plans, psi0, vacuum, 0, nsteps, 0, dx)
    return energies, theta0, x, psi0, out.psi


def _peak_time(t, intensity):
    """Time of the maximum of a sampled periodic pulse, refined by a parabola
    through the three samples around it."""
    m = int(np.argmax(intensity))
    nb = len(intensity)
    ym, y0, yp = intensity[(m - 1) % nb], intensity[m], intensity[(m + 1) % nb]
    frac = 0.5 * (ym - yp) / (ym - 2.0 * y0 + yp)
    return (m + frac) * (t[1] - t[0])


def test_time_axis_a_pulse_through_vacuum_arrives_after_its_flight_time():
    """A pulse marched a distance L through vacuum must reach the point x of
    the exit plane at t = (x sin theta_0 + L cos theta_0) / c: the plane wave
    front moving along (sin theta_0, cos theta_0) at the speed of light,
    later than it entered, never earlier.  Fixes the sign of the exponent,
    the ascending energy order and the time step h / (B dE) (a flipped sign
    puts the peak at -t, i.e. at window - t)."""
    nsteps, dz = 100, 0.1
    energies, theta0, x, psi_in, psi_out = _vacuum_pulse(nsteps=nsteps, dz=dz)
    t = timeaxis.time_axis_fs(energies)
    window = t[1] * len(t)
    length = nsteps * dz
    for label, field, zz in (("entrance", psi_in, 0.0), ("exit", psi_out, length)):
        sig = timeaxis.omega_to_t(field)            # [2][N][B]
        for xi in (-10.0, 0.0, 12.0):
            j = int(np.argmin(np.abs(x - xi)))
            want = (x[j] * math.sin(theta0) + zz * math.cos(theta0)) / C_UM_PER_FS
            got = _peak_time(t, np.abs(sig[0, j]) ** 2)
            diff = (got - want + 0.5 * window) % window - 0.5 * window
            assert abs(diff) < 0.05 * t[1], (label, xi, got, want)
    # the flight over L = 10 um takes about 31 fs: far from its mirror image
    assert 25.0 < length * math.cos(theta0) / C_UM_PER_FS < 0.5 * window


def test_time_axis_pulse_duration_is_the_transform_limit():
    """A Gaussian spectrum of intensity RMS sigma_E and flat phase is a pulse
    of intensity RMS duration hbar / (2 sigma_E) (time-bandwidth product of
    a Gaussian): fixes the scale of the time axis independently of the
    flight time."""
    sigma_ev = 0.1
    energies, _, x, psi_in, _ = _vacuum_pulse(sigma_ev=sigma_ev, nsteps=1)
    t = timeaxis.time_axis_fs(energies)
    sig = timeaxis.omega_to_t(psi_in)
    j = int(np.argmin(np.abs(x)))
    inten = np.abs(sig[0, j]) ** 2
    window = t[1] * len(t)
    tc = (t + 0.5 * window) % window - 0.5 * window     # centred on t = 0
    mean = np.sum(tc * inten) / np.sum(inten)
    rms = math.sqrt(np.sum((tc - mean) ** 2 * inten) / np.sum(inten))
    assert abs(rms / (HBAR_EV_FS / (2.0 * sigma_ev)) - 1.0) < 1e-3


def test_time_axis_a_monochromatic_field_keeps_its_amplitude():
    """One energy alone is a monochromatic wave: its amplitude is the same at
    every instant and equals the solve's own (superposition of the
    monochromatic solutions, no rescaling); B lines of equal energy spacing
    are orthogonal over the window (Parseval: sum_m |psi(t_m)|^2 =
    B sum_j |psi_j|^2)."""
    rng = np.random.default_rng(10)
    nb, nx = 32, 5
    f = np.zeros((nb, 2, nx), dtype=np.complex128)
    f[7] = rng.standard_normal((2, nx)) + 1j * rng.standard_normal((2, nx))
    out = timeaxis.omega_to_t(f)
    assert np.max(np.abs(np.abs(out) - np.abs(f[7])[:, :, None])) < 1e-14
    g = rng.standard_normal((nb, 2, nx)) + 1j * rng.standard_normal((nb, 2, nx))
    lhs = np.sum(np.abs(timeaxis.omega_to_t(g)) ** 2, axis=-1)
    rhs = nb * np.sum(np.abs(g) ** 2, axis=0)
    assert np.max(np.abs(lhs / rhs - 1.0)) < 1e-13
