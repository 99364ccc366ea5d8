"""FP64 CPU oracle for the two-beam FFT beam-propagation z-march.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
unoptimised restatement of the method of Krzywinski & Halavanau,
"Simulation package for solving dynamic diffraction problems in deformed
crystals using beam propagation method" (arXiv 2601.06340), written in
numpy float64 / complex128 so that a reader can check it against the paper's
equations by eye.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2601_06340_gb300``) never imports, links or runs
anything here, and this package imports nothing from the product path.

Modules
-------
``fft``       the discrete Fourier transform written out: the O(N^2)
              definition for N <= 256, radix-2 decimation in time above
              (no library FFT on the march's path).
``bpm``       plan scalars (Eqs. fov3-fov12), Bessel series, the first-order
              two-beam march (Eq. fov10) and the splitting schemes of Eq.
              split-op, powers and records.
``geometry``  crystal-shape masks (slab of any asymmetry angle, polygon) and
              displacement fields (cylindrical bend, Eq. fov110; edge
              dislocation, Eq. fov120 with the Burgers vector normal to the
              line), and the strain phase h*u_x of Eq. (Authier).
``timeaxis``  the energy -> time synthesis of a batch of exit fields
              (Section "Time-Dependent Simulation of Reflection").
``bpm3d``     the same march with both transverse coordinates (x, y):
              2D angular-spectrum propagators, box crystals, 3D arrays.

Every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` (3D: ``tests/test_oracle3d_pins.py``) against
closed forms, physical laws, invariants, brute force or an independent
library routine; none is left unpinned.
"""
