"""Training data and training runs for the neural operator, through the C ABI.

The operator is trained once at p* on solutions the solver itself produces
(Sec. 5.1: a single constant cross-section pair; App. A1: GRF sources of unit
integral, MSE loss, Adam).  Every step here is a library call: the batch of
p* problems is solved by nop_solve_fixed_source, the branch inputs come from
the operator's input map nop_no_sensors, and the optimisation runs in
nop_no_train.  The random sources and the sample order are inputs.
"""
import numpy as np


def deeponet_training_set(solver, cfg, sources, order=32, tol=1e-7, itmax=100000):
    """Solve the p* problem for every source row (n x I cells over cfg.length).

    Returns (branch inputs [n, sensors], trunk coordinates [I], targets [n, I]).
    The operator `cfg` must be installed (its sensor count defines the input map).
    """
    n, I = sources.shape
    st, ss = cfg.sigma_t_star, cfg.sigma_s_star
    solver.set_slabs(np.full(n, I), np.full(n, cfg.length), np.full(n, order),
                     np.full(n * I, st), np.full(n * I, ss), source=sources.reshape(-1))
    phi, info = solver.solve_fixed_source(tol=tol, itmax=itmax, precision=0)
    U = solver.no_sensors(sources.reshape(-1))
    X = (np.arange(I) + 0.5) / I
    return U, X, phi.reshape(n, I), info


def diffusion_training_set(solver, cfg, sources):
    """The diffusion batch at p* = (D*, Sigma_a*) = (cfg.sigma_t_star,
    cfg.sigma_s_star) for every source row (n x I cells over cfg.length),
    solved by nop_diffusion_solve (Table 1's recast takes its operator from
    one parameter setting).  Returns (branch inputs [n, sensors], trunk
    coordinates [I], targets [n, I])."""
    n, I = sources.shape
    solver.set_diffusion(np.full(n, I), np.full(n, cfg.length),
                         np.full(n * I, cfg.sigma_t_star), sources.reshape(-1),
                         absorption=np.full(n * I, cfg.sigma_s_star))
    u = solver.diffusion_solve()
    U = solver.no_sensors(sources.reshape(-1))
    X = (np.arange(I) + 0.5) / I
    return U, X, u.reshape(n, I)


def fno1d_training_set(solver, cfg, sources, order=32, tol=1e-7, itmax=100000):
    """Solve the p* slab for every source row (n x I cells over cfg.length).

    Returns (inputs [n, I] = the sources, targets [n, I] = the fluxes, info):
    the FNO-1D maps a source on the grid to the flux on the same grid.
    """
    n, I = sources.shape
    st, ss = cfg.sigma_t_star, cfg.sigma_s_star
    solver.set_slabs(np.full(n, I), np.full(n, cfg.length), np.full(n, order),
                     np.full(n * I, st), np.full(n * I, ss), source=sources.reshape(-1))
    phi, info = solver.solve_fixed_source(tol=tol, itmax=itmax, precision=0)
    return sources.astype(np.float32), phi.reshape(n, I), info


def fno2d_training_set(solver, cfg, sources, tol=1e-7, itmax=100000, bc=(0, 0, 0, 0)):
    """Solve the p* square (cfg.length, vacuum unless bc says otherwise) for
    every source field (n x ny x nx, row-major [y][x]); returns (inputs [n, ny*nx],
    targets [n, ny*nx])."""
    n, ny, nx = sources.shape
    st, ss = cfg.sigma_t_star, cfg.sigma_s_star
    Y = np.zeros((n, ny * nx))
    for b in range(n):
        solver.set_xy(nx, ny, cfg.length, cfg.length, np.full(nx * ny, st),
                      np.full(nx * ny, ss), source=sources[b].reshape(-1), bc=bc)
        phi, _ = solver.solve_fixed_source(tol=tol, itmax=itmax, precision=0)
        Y[b] = phi
    return sources.reshape(n, -1).astype(np.float32), Y


def train_fno(solver, S, Y, steps, batch, seed, lr=1e-3):
    """Adam on FNO pairs (S, Y) with a seeded sample order (grid from S's width
    for FNO-1D, from the current x-y problem for FNO-2D)."""
    rng = np.random.default_rng(seed)
    n = S.shape[0]
    order = np.concatenate([rng.permutation(n) for _ in range((steps * batch) // n + 1)])
    return solver.no_train(S, Y, np.zeros(S.shape[1], dtype=np.float32), steps=steps,
                           batch=batch, lr=lr, order=order[:steps * batch])


def train(solver, U, X, Y, steps, batch, seed, lr=1e-3):
    """Adam on (U, X, Y) with a seeded sample order; returns the loss history."""
    rng = np.random.default_rng(seed)
    n = U.shape[0]
    order = np.concatenate([rng.permutation(n) for _ in range((steps * batch) // n + 1)])
    return solver.no_train(U, Y, X, steps=steps, batch=batch, lr=lr,
                           order=order[:steps * batch])
