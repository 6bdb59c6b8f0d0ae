"""CPU oracle for GridFF's hot path (test infrastructure, not product code).

Plain, slow, obviously-correct numpy / PyTorch-CPU code in float64 (with a
float32 mirror of the grid interpolation).  It shares no code with the CUDA
library: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
legs may import it (the timed CPU baseline and reference arm, and the FP64
pairwise reference that the accuracy keys compare finished GPU results
with, outside every timed region).  The CUDA product path never calls it.

Modules
-------
bspline    cubic B-spline basis (Eq. Bspline), 1D collocation, exact and
           gradient-descent coefficient fits (Sec. 5), tricubic evaluation
           with analytic gradient in the 16/4/1 order of Sec. 5.
substrate  factorised Morse channels (Eqs. E_Morse, V_Morse), direct Morse
           pair sums, 3D Ewald with slab dipole correction (Sec. 4), the
           exact 2D-periodic Fourier sum used to pin it, the FP64 pairwise
           reference energies and forces (Eqs. E, E_Coulomb, E_Morse).
grid       node coordinates and grid construction (node values + fit).
intra      reduced UFF-like intramolecular force field (Sec. 6, Sec. 8).
dynamics   rigid-body kinematics, FIRE (flexible and rigid), velocity Verlet
           and the NO_SQUISH rigid-body NVE splitting.

Every function names the passage of the paper it follows.  Where the paper
is silent the docstring states the reading taken.
"""
