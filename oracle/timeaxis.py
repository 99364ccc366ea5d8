"""Oracle: energy -> time synthesis of a batch of exit fields.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper treats a pulse as independent solves over photon energy followed
by an inverse Fourier transform from frequency to time (Section
"Time-Dependent Simulation of Reflection from Distorted Crystals"; the
``time_dependent`` / ``tgrid`` keys of the parameter table).  It does not fix
the discrete convention; the reading used here is

    psi(x, t_m) = (1 / B) * sum_j psi_j(x) * exp(+2 pi i j m / B),

over the B energies E_j sorted ascending, with the time window
h / (E_{j+1} - E_j).  This is exactly numpy's inverse DFT along the energy
axis, which is how it is written below (a library FFT as one step).
"""

from __future__ import annotations

import numpy as np


def omega_to_t(fields: np.ndarray) -> np.ndarray:
    """fields [B][2][N] (energy-major) -> [2][N][B] (time-minor)."""
    f = np.asarray(fields, dtype=np.complex128)
    return np.fft.ifft(np.transpose(f, (1, 2, 0)), axis=-1)


def omega_to_t_direct(fields: np.ndarray) -> np.ndarray:
    """The same sum written out as an O(B^2) loop (brute-force cross-check)."""
    f = np.asarray(fields, dtype=np.complex128)
    nb = f.shape[0]
    out = np.zeros((f.shape[1], f.shape[2], nb), dtype=np.complex128)
    for m in range(nb):
        acc = np.zeros(f.shape[1:], dtype=np.complex128)
        for j in range(nb):
            acc += f[j] * np.exp(2j * np.pi * j * m / nb)
        out[:, :, m] = acc / nb
    return out
