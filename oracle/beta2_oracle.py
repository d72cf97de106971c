"""Oracle (test infrastructure only): the time step of Eq. (nonl_CH_nm) with beta2 > 0.

Only tests may import this module.  It shares nothing with the GPU library.

Reading of the step (Section 4 names implicit Euler with the convolution explicit; the paper's
own solver for the resulting obstacle problem is in work it only cites).  With
g = gamma * u^{k-1} + c_F u^{k-1} (explicit) and the convex part c_gamma u + dI(u) implicit:
    (u - u^{k-1}) / tau + beta1 w - beta2 Lap_h w = 0,
    w in c_gamma u - g + dI(u),
where Lap_h is the periodic 5-point Laplacian with spacing h.  The inclusion is inverted by the
resolvent of the indicator, u = P_[-1,1]((w + g) / c_gamma), which leaves one equation in w,
    F(w) = tau A w + P_[-1,1]((w + g) / c_gamma) - u^{k-1} = 0,    A = beta1 I - beta2 Lap_h,
strongly monotone because tau A is symmetric positive definite and the projection is monotone.
It is solved by a semismooth Newton iteration (a primal-dual active-set method): with the
inactive set I = { |w + g| < c_gamma }, the generalised Jacobian is J = tau A + diag(1_I) / c_gamma,
and the iteration stops when the active set repeats and the residual is at rounding level.
With beta2 = 0 the equation is pointwise and the step is the projection formula of the
beta2 = 0 scheme.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def laplacian(n: int, h: float) -> sp.csr_matrix:
    """Periodic 5-point Laplacian on the n x n lattice (row-major, x fastest), spacing h."""
    N = n * n
    idx = np.arange(N).reshape(n, n)
    rows, cols, vals = [], [], []
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        rows.append(idx.ravel())
        cols.append(np.roll(np.roll(idx, -dy, axis=0), -dx, axis=1).ravel())
        vals.append(np.full(N, 1.0 / h ** 2))
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(np.full(N, -4.0 / h ** 2))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def step(model, u_old: np.ndarray, eps: float, beta2: float, max_newton: int = 100):
    """One step from u_old (n x n, FP64) of `model` (an oracle.OracleModel, periodic) with the
    given beta2.  Returns (u, w, newton_iterations)."""
    n = model.n
    h = 1.0 / n
    tau, b1, cF = model.tau, model.beta1, model.c_F
    _, cg = model.weights(eps)
    g = (model.convolve(u_old, eps) + cF * u_old).ravel()
    uo = u_old.ravel()
    N = n * n
    A = b1 * sp.identity(N, format="csr") - beta2 * laplacian(n, h)
    # start from the beta2 = 0 step: w = c_gamma u0 - g reproduces u0 = P((w + g)/c_gamma)
    u0 = np.clip((uo + tau * b1 * g) / (1.0 + tau * b1 * cg), -1.0, 1.0)
    w = cg * u0 - g
    prev = None
    for it in range(1, max_newton + 1):
        x = (w + g) / cg
        inactive = np.abs(x) < 1.0
        F = tau * (A @ w) + np.clip(x, -1.0, 1.0) - uo
        if prev is not None and np.array_equal(inactive, prev) and np.abs(F).max() <= 1e-13:
            break
        J = (tau * A + sp.diags(inactive.astype(np.float64) / cg)).tocsc()
        w = w + spla.spsolve(J, -F)
        prev = inactive
    else:
        raise RuntimeError("semismooth Newton did not converge")
    u = np.clip((w + g) / cg, -1.0, 1.0)
    return u.reshape(n, n), w.reshape(n, n), it


def solve(model, u0: np.ndarray, eps: float, beta2: float, nsteps: int):
    """nsteps steps from u0; returns (u(T), mean of u(T))."""
    u = np.asarray(u0, dtype=np.float64).copy()
    for _ in range(nsteps):
        u, _, _ = step(model, u, eps, beta2)
    return u, float(u.mean())


def solve_sample(model, seed: int, beta2: float, nsteps=None):
    """Initial field from the seed (as the beta2 = 0 oracle), solve, and return (f, mean, u(T), eps)."""
    eps = model.sample_eps(seed)
    u0 = model.initial_field(seed)
    uT, mean = solve(model, u0, eps, beta2, model.nsteps if nsteps is None else nsteps)
    return 0.5 * (1.0 + mean), mean, uT, eps
