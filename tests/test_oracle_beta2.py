"""Pins of the beta2 > 0 step oracle (oracle/beta2_oracle.py) against what the mathematics
fixes, independent of its Newton iteration: the beta2 = 0 limit, the exact linear-regime
response of a Fourier mode, the minimiser of the step's box-constrained quadratic program found
by a general bound-constrained optimiser, and the mass balance of the periodic Laplacian."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import beta2_oracle as B2


def model(**kw):
    base = dict(n=16, delta=3 / 16, kernel=0, eps=0.03, c_F=1.0, beta1=1.0, tau=0.01, nsteps=5, ic=2)
    base.update(kw)
    return O.OracleModel(**base)


def test_beta2_zero_is_the_projection_step():
    m = model(n=24, delta=4 / 24)
    u0 = m.initial_field(3)
    u, _, it = B2.step(m, u0, 0.03, 0.0)
    assert np.abs(u - m.step(u0, 0.03)).max() <= 1e-15
    assert it <= 4   # points exactly on |x| = 1 may flip once


@pytest.mark.parametrize("p,q", [(1, 0), (2, 3), (5, 5)])
@pytest.mark.parametrize("kernel", [0, 1])
def test_linear_regime_fourier_mode_closed_form(p, q, kernel):
    # no active point: u_new = (1 + tau a(k) (Gamma(k) + c_F)) / (1 + tau a(k) c_gamma) u_old with
    # a(k) = beta1 + beta2 lambda(k), lambda(k) = (4 / h^2)(sin^2(pi p / n) + sin^2(pi q / n)) and
    # Gamma(k) = sum_z w_z cos(k . z) the symbol of the convolution
    n, R, eps, beta2, tau = 32, 3, 0.03, 0.05, 0.01
    m = model(n=n, delta=R / n, kernel=kernel, delta_hf=R / n, tau=tau)
    w, cg = m.weights(eps)
    dx, dy = m.offsets()
    gam = float(np.sum(w * np.cos(2 * np.pi * (p * dx + q * dy) / n)))
    lam = 4 * n * n * (math.sin(math.pi * p / n) ** 2 + math.sin(math.pi * q / n) ** 2)
    a = 1.0 + beta2 * lam
    r = (1 + tau * a * (gam + 1.0)) / (1 + tau * a * cg)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u0 = 0.01 * np.cos(2 * np.pi * (p * xx + q * yy) / n)
    u, _, _ = B2.step(m, u0, eps, beta2)
    assert np.abs(u - r * u0).max() <= 1e-15
    assert abs(r - 1.0) > 1e-6   # the mode does change


def test_step_is_the_minimiser_of_the_box_constrained_qp():
    # The step minimises Phi(v) = 1/2 (v - u0)^T (tau A)^{-1} (v - u0) + c_gamma/2 |v|^2 - g^T v
    # over [-1, 1]^N (its optimality conditions are the step's equations); found here by
    # L-BFGS-B on an 8 x 8 lattice with many points on the obstacle.
    from scipy.optimize import minimize
    n, eps, beta2 = 8, 0.2, 0.05
    m = model(n=n, delta=2 / n, tau=0.05)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u0 = np.clip(1.6 * np.sin(2 * np.pi * xx / n) * np.cos(2 * np.pi * yy / n) + 0.1, -1.0, 1.0)
    u, _, _ = B2.step(m, u0, eps, beta2)
    assert 0 < np.sum(np.abs(u) == 1.0) < n * n   # the obstacle is active somewhere
    _, cg = m.weights(eps)
    g = (m.convolve(u0, eps) + u0).ravel()
    A = np.eye(n * n) - beta2 * B2.laplacian(n, 1.0 / n).toarray()
    Minv = np.linalg.inv(m.tau * A)
    uo = u0.ravel()

    def phi(v):
        d = v - uo
        return 0.5 * d @ Minv @ d + 0.5 * cg * v @ v - g @ v, Minv @ d + cg * v - g

    res = minimize(phi, np.clip(uo, -1, 1), jac=True, method="L-BFGS-B", bounds=[(-1.0, 1.0)] * (n * n),
                   options=dict(ftol=1e-15, gtol=1e-12, maxiter=20000))
    assert np.abs(res.x - u.ravel()).max() <= 1e-6


def test_mass_balance_and_bounds():
    # sum_i (u_i - u0_i) = -tau beta1 sum_i w_i: the periodic Laplacian's columns sum to zero
    m = model(n=24, delta=4 / 24, tau=0.02)
    u0 = m.initial_field(9)
    u, w, _ = B2.step(m, u0, 0.03, 0.05)
    assert abs((u - u0).sum() + m.tau * m.beta1 * w.sum()) <= 1e-10
    assert np.abs(u).max() <= 1.0
    assert np.sum(np.abs(u) == 1.0) > 0


@pytest.mark.parametrize("c", [-1.0, 1.0])
def test_pure_phases_are_stationary(c):
    m = model(n=16, delta=3 / 16)
    u = np.full((16, 16), c)
    for _ in range(3):
        u, _, _ = B2.step(m, u, 0.03, 0.05)
    assert np.all(u == c)
