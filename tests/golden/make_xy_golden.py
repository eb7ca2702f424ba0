"""Write tests/golden/xy_checkerboard_8g.txt: the FP64 oracle's converged
dominant eigenpair of the 256x256, 8-group, level-symmetric S8 checkerboard
(the x-y multigroup eigenproblem of Sec. 5.3 Eq. 27-29 taken to two
dimensions as in Sec. 6; inputs from workloads.checkerboard_xy_8g).

The script calls only oracle/ (and the seeded input recipe).  The flux is
normalised to unit production (the oracle's convention), and the file keeps k,
the per-group flux integrals and the flux at 4096 cells drawn by a seeded
generator, enough for a relative L2 comparison of sampled values.

    python tests/golden/make_xy_golden.py      # several minutes on one core
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import quadrature as Qd  # noqa: E402
from oracle import transport as T  # noqa: E402

OUT = os.path.join(HERE, "xy_checkerboard_8g.txt")
N_SAMPLES = 4096
SAMPLE_SEED = 44
TOL_K, TOL_PHI, TOL_INNER = 1e-12, 1e-10, 1e-11


def problem():
    c = W.checkerboard_xy_8g()
    bc = {k: (T.REFLECTIVE if v else T.VACUUM) for k, v in c.bc.items()}
    return c, T.XY(dx=c.Lx / c.nx, dy=c.Ly / c.ny, sigt=c.sigt, sigs=c.sigs,
                   nusigf=c.nusigf, chi=c.chi, bc=bc)


def sample_index(G, ny, nx):
    """The (g, j, i) cells the golden file keeps: a seeded draw without repeats."""
    rng = np.random.default_rng(SAMPLE_SEED)
    flat = rng.choice(G * ny * nx, size=N_SAMPLES, replace=False)
    flat.sort()
    g, r = np.divmod(flat, ny * nx)
    j, i = np.divmod(r, nx)
    return g, j, i


def main():
    c, P = problem()
    t0 = time.time()
    r = T.power_iteration(P, Qd.level_symmetric_s8(), tol_k=TOL_K, tol_phi=TOL_PHI,
                          tol_inner=TOL_INNER)
    el = time.time() - t0
    G, ny, nx = P.sigt.shape
    g, j, i = sample_index(G, ny, nx)
    area = P.dx * P.dy
    with open(OUT, "w") as f:
        f.write("# FP64 oracle (oracle.transport.power_iteration, oracle.quadrature."
                "level_symmetric_s8)\n")
        f.write("# workload: workloads.checkerboard_xy_8g() (256x256, 8 groups, LS S8, "
                "reflective x=0/y=0, vacuum x=L/y=L)\n")
        f.write("# written by tests/golden/make_xy_golden.py; tol_k %g tol_phi %g tol_inner %g; "
                "%d outer, %d inner iterations, %.0f s\n" % (TOL_K, TOL_PHI, TOL_INNER, r.outer,
                                                             r.inner_total, el))
        f.write("# flux normalised to unit production: sum nuSigma_f phi dx dy = 1\n")
        f.write("k %.15f\n" % r.k)
        f.write("outer %d\ninner %d\n" % (r.outer, r.inner_total))
        for gg in range(G):
            f.write("group_integral %d %.15e\n" % (gg, float(np.sum(r.phi[gg]) * area)))
        f.write("sample_seed %d\nsamples %d\n" % (SAMPLE_SEED, N_SAMPLES))
        for a, b, cc in zip(g, j, i):
            f.write("%d %d %d %.15e\n" % (a, b, cc, r.phi[a, b, cc]))
    print("k = %.12f, %d outer, %d inner, %.0f s" % (r.k, r.outer, r.inner_total, el))


if __name__ == "__main__":
    main()
