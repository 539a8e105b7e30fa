"""FP64 CPU oracle for the twisted-mass disconnected-loop path (arXiv:1401.6749).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product (the CUDA library and its Python binding) never imports, links or
executes anything here, and nothing here imports the product.

Every function is a plain, slow restatement of the mathematics in the paper (and
of the operator definition that the paper takes from the twisted-mass
formulation), in numpy complex128.  Fields use the canonical layout of the
library's C-ABI:

* spinor  ``psi[T, Z, Y, X, 4, 3]``  (lexicographic site x + Lx(y + Ly(z + Lz t)),
  then Dirac index, then colour), complex128;
* gauge   ``U[4, T, Z, Y, X, 3, 3]`` with ``U[mu]`` the link from x to x + mu_hat,
  mu = 0..3 for the x, y, z, t directions;
* a batch of fields carries one more leading axis.

Modules
-------
gamma     Dirac matrices (DeGrand-Rossi chiral basis) and the 16 Gamma products.
lattice   lattice shifts with the antiperiodic time boundary.
philox    Philox4x32-10 counter-based generator and Z4 noise (Sec. 2, Eqs. 1-2).
operator  twisted-mass Wilson operator M, its adjoint and D_W; dense matrix.
cg        conjugate gradient on the normal equations M^dag M x = M^dag eta.
loops     local (16 Gamma) and one-derivative loop contractions, three estimators
          (standard, one-end trick Eq. 5, generalised one-end trick Eq. 6).
tsm       Truncated Solver Method combination, Eq. 4.

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against closed forms, dense inversion, symmetry identities or a library routine;
none is marked "parity unpinned".
"""
