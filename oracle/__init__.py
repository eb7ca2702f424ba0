"""FP64 CPU oracle for the MD-PNOP transport path -- TEST INFRASTRUCTURE ONLY.

This package is the independent, plain, slow reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import it.  The
CUDA path never imports, links or calls anything here, and nothing here comes
from the CUDA path: the two share no code, tables or constants.

Layout
  sn_sweep.c   plain-C diamond-difference sweeps (1D slab, 2D x-y), FP64
  native.py    compiles and loads sn_sweep.c (gcc, ctypes)
  quadrature.py  Gauss-Legendre (1D) and level-symmetric S8 (2D) sets
  transport.py source iteration, power iteration, multigroup (Sec. 5.1-5.3)
  neural.py    DeepONet / FNO forward and backward, MSE, Adam (Sec. 4, App. A1)
  recast.py    equation-recast iteration, Eq. 7/8 and Eq. 24, and the
               simple-preconditioning eigen solve (App. A2, Eq. A5-A6)
  dsa.py       diffusion synthetic acceleration of slab source iteration
               (a classical accelerator, not the paper's method, kept for
               comparison with the warm start)

Pins (what fixes each function independently of itself) live in
``tests/test_oracle_*.py``; functions without such a pin say "parity unpinned"
in their docstring.
"""
