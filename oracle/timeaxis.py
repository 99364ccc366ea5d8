"""Oracle: energy -> time synthesis of a batch of exit fields.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper treats a pulse as independent solves over photon energy followed
by a Fourier transform from frequency to time (Section "Time-Dependent
Simulation of Reflection from Distorted Crystals"; the ``time_dependent`` /
``tgrid`` keys of the parameter table).  It does not write the discrete
form out; the reading used here follows from the rest of the paper:

* Eq. fov4 advances a field along +z by multiplying its angular spectrum
  with exp(+i dz^ sqrt(1 - k_x^2)), so a wave travelling towards +z has the
  spatial phase exp(+i k z) and, for a forward wave, the time dependence
  exp(-i omega t);
* the equations are linear, so the field of the pulse is the superposition
  of the monochromatic solutions, each with its own exp(-i omega_j t).

With the B energies E_j = E_0 + j dE sorted ascending, the time grid
t_m = m dt, dt = h / (B dE) (window h / dE) and the common carrier
exp(-i omega_0 t) taken out, this is

    psi(x, t_m) = sum_j psi_j(x) exp(-2 pi i j m / B),

the forward DFT along the energy axis (computed by ``oracle.fft``).  A
monochromatic component keeps its own amplitude at every instant, and a
pulse that travels a distance arrives later, not earlier.
"""

from __future__ import annotations

import numpy as np

from . import fft as dft

# Planck's constant in eV * fs (SI 2019: h and e exact).
H_EV_FS = 6.62607015e-34 / 1.602176634e-19 * 1e15


def omega_to_t(fields: np.ndarray) -> np.ndarray:
    """fields [B][2][N] (energy-major, energies ascending) -> [2][N][B]
    (time-minor): out[b][x][m] = sum_j fields[j][b][x] exp(-2 pi i j m / B)."""
    f = np.asarray(fields, dtype=np.complex128)
    return dft.fft(np.transpose(f, (1, 2, 0)))


def time_axis_fs(energies_ev: np.ndarray) -> np.ndarray:
    """t_m = m h / (B dE) in femtoseconds for B equally spaced energies."""
    e = np.asarray(energies_ev, dtype=np.float64)
    nb = e.size
    de = (e[-1] - e[0]) / (nb - 1)
    return np.arange(nb) * (H_EV_FS / (nb * de))
