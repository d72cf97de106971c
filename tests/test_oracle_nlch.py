"""Pins of the model oracle (oracle/nlch_oracle.c) against what the paper and the
mathematics fix, independent of the oracle's own formulas."""
import math

import numpy as np
import pytest

import oracle as O
from tests.conftest import read_golden


def model(**kw):
    base = dict(n=64, delta=4 / 64, kernel=0, eps=0.03, c_F=1.0, beta1=1.0, tau=1e-3,
                nsteps=200, ic=0, ic_amp=0.05)
    base.update(kw)
    return O.OracleModel(**base)


# --------------------------------------------------------------------------- RNG
def test_splitmix64_reference_vector():
    want = [int(r[0]) for r in read_golden("splitmix64_seed1234567.txt")]
    got = [O.splitmix64(1234567, k) for k in range(1, 6)]
    assert got == want


def test_uniform_and_normal_moments():
    xs = np.array([O.uniform(20231016, 1, i) for i in range(20000)])
    assert xs.min() >= 0.0 and xs.max() < 1.0
    assert abs(xs.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(xs))
    m = model(n=128, ic=1, ic_amp=1.0)
    # the smoothed field is (5 iid normals)/5 per node: variance 1/5 before clipping
    u = m.initial_field(7)
    assert abs(u.mean()) < 4 * math.sqrt(0.2 / u.size) * 3
    assert abs(u.var() - 0.2) < 0.02


def test_streams_are_distinct_windows():
    assert O.draw(5, 0, 0) == O.splitmix64(5, 1)
    assert O.draw(5, 1, 0) == O.splitmix64(5, (1 << 32) + 1)
    assert O.draw(5, 2, 7) == O.splitmix64(5, (2 << 32) + 8)


# --------------------------------------------------------------------------- disc
def test_disc_counts_match_lattice_point_counts():
    for R, cnt in read_golden("disc_counts.txt"):
        dx, dy = O.disc(float(R))
        assert len(dx) == int(cnt)
        # brute force count in plain Python
        Ri = int(R)
        brute = sum(1 for i in range(-Ri, Ri + 1) for j in range(-Ri, Ri + 1) if i * i + j * j <= Ri * Ri)
        assert brute == int(cnt)


def test_constant_kernel_second_moment_is_4eps2():
    # int_{B_delta} gamma |z|^2 dz = 4 eps^2, so that L -> -eps^2 Laplace (Section 4)
    eps, delta = 0.03, 0.1
    A = O.gamma(0, 0.0, eps, delta, delta)
    # midpoint quadrature of the radial integral
    N = 200000
    r = (np.arange(N) + 0.5) * delta / N
    moment = np.sum(A * r ** 2 * 2 * np.pi * r) * delta / N
    assert moment == pytest.approx(4 * eps * eps, rel=1e-8)
    assert O.gamma(0, delta * 1.01, eps, delta, delta) == 0.0


def test_gaussian_kernel_matches_paper_xi():
    # Section 4: c_F = 1, eps^2 = 0.00178, delta_hf = 0.25 give xi = c_gamma - c_F ~ 0.0253
    # and c_gamma ~ 36 eps^2 / delta^2 (continuum).  The lattice c_gamma at h = 1/128
    # must be close to the continuum value.
    eps = math.sqrt(0.00178)
    m = O.OracleModel(n=128, delta=0.25, kernel=1, delta_hf=0.25, eps=eps)
    _, cg = m.weights(eps)
    assert 36 * eps ** 2 / 0.25 ** 2 == pytest.approx(1.02528, rel=1e-4)
    assert cg - 1.0 == pytest.approx(0.0253, abs=0.004)
    # exact continuum value of the truncated Gaussian: (1 - e^{-9}) 4 eps^2 / s^2
    s = 0.25 / 3
    assert cg == pytest.approx((1 - math.exp(-9)) * 4 * eps ** 2 / s ** 2, rel=5e-3)


# --------------------------------------------------------------------------- operator
def test_L_vanishes_on_constants():
    for kernel in (0, 1):
        m = model(n=32, delta=3 / 32, kernel=kernel, delta_hf=3 / 32)
        for c in (0.0, 1.0, -0.37, 0.123456789):
            Lu = m.apply_L(np.full((32, 32), c), 0.03)
            assert np.all(Lu == 0.0)


def test_L_on_quadratic_closed_form():
    # L_h(x^2)_i = -h^2 a sum_{z in D} dx^2 on a non-wrapping patch, with
    # sum_{z in D} dx^2 = sum_dy w(w+1)(2w+1)/3, w = floor(sqrt(R^2 - dy^2)).
    n, R, eps = 64, 4, 0.03
    m = model(n=n, delta=R / n, eps=eps)
    h = 1.0 / n
    x = np.arange(n) * h
    u = np.tile(x ** 2, (n, 1))
    Lu = m.apply_L_open(u, eps)
    A = 8 * eps * eps / (math.pi * (R * h) ** 4)
    s2 = sum(w * (w + 1) * (2 * w + 1) // 3 for w in
             (int(math.isqrt(R * R - dy * dy)) for dy in range(-R, R + 1)))
    assert s2 == 192
    closed = -h * h * (A * h * h) * s2
    inner = Lu[R:n - R, R:n - R]
    assert np.allclose(inner, closed, rtol=1e-12, atol=0)
    assert closed == pytest.approx(-1.71887e-3, rel=1e-5)
    # continuum limit -eps^2 * Laplace(x^2) = -2 eps^2 within the lattice error
    assert closed == pytest.approx(-2 * eps * eps, rel=0.06)


@pytest.mark.parametrize("n,delta", [(64, 4.5 / 64), (88, 0.1875)])
def test_non_integer_horizon_disc_and_operator(n, delta):
    # delta/h = 4.5, and the paper's h = 1/88, delta = 0.1875 (delta/h = 16.5): the disc is the
    # lattice ball { z : |z|^2 <= (delta/h)^2 } (brute force over its bounding square), L
    # vanishes on constants, and L(x^2) = -h^2 a sum_{z in D} dx^2 on a non-wrapping patch
    eps = 0.03
    m = model(n=n, delta=delta, eps=eps)
    rad = delta * n
    Ri = int(math.floor(rad))
    ball = {(i, j) for i in range(-Ri, Ri + 1) for j in range(-Ri, Ri + 1) if i * i + j * j <= rad * rad}
    dx, dy = m.offsets()
    assert len(dx) == len(ball) and set(zip(np.asarray(dx).tolist(), np.asarray(dy).tolist())) == ball
    if n == 88:
        assert len(ball) == 861
    assert np.all(m.apply_L(np.full((n, n), -0.4375), eps) == 0.0)
    h = 1.0 / n
    u = np.tile((np.arange(n) * h) ** 2, (n, 1))
    A = 8 * eps * eps / (math.pi * delta ** 4)
    closed = -h * h * (A * h * h) * sum(i * i for i, _ in ball)
    inner = m.apply_L_open(u, eps)[Ri:n - Ri, Ri:n - Ri]
    assert np.allclose(inner, closed, rtol=1e-12, atol=0)


def test_L_on_fourier_modes_matches_fft_symbol():
    n, R, eps = 32, 3, 0.03
    for kernel in (0, 1):
        m = model(n=n, delta=R / n, kernel=kernel, delta_hf=R / n)
        w, cg = m.weights(eps)
        dx, dy = m.offsets()
        stencil = np.zeros((n, n))
        for k in range(len(w)):
            stencil[dy[k] % n, dx[k] % n] += w[k]
        fft_sym = cg - np.real(np.fft.fft2(stencil))
        yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        for p, q in ((0, 0), (1, 0), (0, 3), (5, 7), (16, 16)):
            mode = np.cos(2 * np.pi * (p * xx + q * yy) / n)
            Lm = m.apply_L(mode, eps)
            lam = m.symbol(p, q, eps)
            assert np.allclose(Lm, lam * mode, atol=1e-13)
            assert lam == pytest.approx(fft_sym[q, p], abs=1e-13)


# --------------------------------------------------------------------------- step
def test_pure_phases_and_zero_are_stationary():
    m = model(n=32, delta=4 / 32)
    for c in (1.0, -1.0, 0.0):
        u = np.full((32, 32), c)
        uT, mean = m.solve(u, 0.03, nsteps=25)
        assert np.all(uT == c)


def test_step_solves_the_implicit_inclusion():
    # (u^k - u^{k-1})/tau + beta1 w = 0 with
    # w - (c_gamma u^k - gamma*u^{k-1} - c_F u^{k-1}) in dI(u^k):
    # zero where |u^k| < 1, >= 0 where u^k = 1, <= 0 where u^k = -1.
    m = model(n=64, delta=4 / 64, ic=2, tau=5e-3)
    eps = 0.03
    u = m.initial_field(11)
    _, cg = m.weights(eps)
    hit_lo = hit_hi = False
    for _ in range(40):
        unew = m.step(u, eps)
        w = -(unew - u) / (m.tau * m.beta1)
        g = m.convolve(u, eps) + m.c_F * u
        res = w - (cg * unew - g)
        inner = np.abs(unew) < 1
        assert np.all(np.abs(res[inner]) < 1e-10)
        assert np.all(res[unew == 1.0] >= -1e-10)
        assert np.all(res[unew == -1.0] <= 1e-10)
        hit_hi |= bool((unew == 1.0).any())
        hit_lo |= bool((unew == -1.0).any())
        u = unew
    assert hit_hi and hit_lo          # both sides of the obstacle were active


def test_bounds_and_max_norm_growth():
    m = model(n=64, delta=4 / 64, ic=0)
    eps = 0.03
    u0 = m.initial_field(3)
    grow = 1 + m.tau * m.beta1 * m.c_F
    u = u0
    for k in range(1, 41):
        u = m.step(u, eps)
        assert np.abs(u).max() <= np.abs(u0).max() * grow ** k * (1 + 1e-14)
    mn = model(n=64, delta=4 / 64, ic=2)
    v = mn.initial_field(4)
    for _ in range(10):
        v = mn.step(v, eps)
        assert np.abs(v).max() <= 1.0


def test_step_is_lipschitz_with_factor_1_plus_tau_cF():
    m = model(n=32, delta=3 / 32, ic=2)
    eps = 0.03
    a = m.initial_field(1)
    b = m.initial_field(2)
    d0 = np.abs(a - b).max()
    grow = 1 + m.tau * m.beta1 * m.c_F
    for k in range(1, 11):
        a, b = m.step(a, eps), m.step(b, eps)
        assert np.abs(a - b).max() <= d0 * grow ** k * (1 + 1e-13)


def test_energy_decreases_when_splitting_condition_holds():
    # E_h is non-increasing for the convex-concave splitting when the explicit part
    # (gamma * + c_F) is positive semidefinite: min over modes of the stencil DFT >= -c_F.
    for ic in (0, 2):
        m = model(n=32, delta=4 / 32, ic=ic, tau=2e-2, ic_amp=0.5)
        eps = 0.03
        w, _ = m.weights(eps)
        dx, dy = m.offsets()
        st = np.zeros((32, 32))
        for k in range(len(w)):
            st[dy[k] % 32, dx[k] % 32] += w[k]
        assert np.real(np.fft.fft2(st)).min() >= -m.c_F
        u = m.initial_field(9)
        e = m.energy(u, eps)
        for _ in range(30):
            u = m.step(u, eps)
            e2 = m.energy(u, eps)
            assert e2 <= e + 1e-14
            e = e2


@pytest.mark.parametrize("kernel", [0, 1])
def test_energy_closed_form_on_fourier_modes(kernel):
    # E_h(u) = h^2 [1/4 sum_i sum_z w_z (u_i - u_{i+z})^2 + sum_i (c_F/2)(1 - u_i^2)]
    # (Section 2, the nonlocal free energy with the obstacle potential; |u| <= 1).
    # On u = A cos(2 pi (p x + q y)) at the nodes x = j h, with 2p, 2q not both = 0 mod n:
    # averaged over the lattice, cos^2 = 1/2 and (cos t - cos(t + phi))^2 = 1 - cos phi, so
    #   E_h = (A^2 / 4) sum_z w_z (1 - cos(k.z)) + (c_F / 2)(1 - A^2 / 2)     (h^2 n^2 = 1).
    # The symbol sum_z w_z (1 - cos(k.z)) is taken from numpy's FFT of the stencil.
    n = 32
    m = model(n=n, delta=5 / n, kernel=kernel, delta_hf=6 / n, c_F=1.0)
    eps = 0.03
    w, cg = m.weights(eps)
    dx, dy = m.offsets()
    st = np.zeros((n, n))
    for k in range(len(w)):
        st[dy[k] % n, dx[k] % n] += w[k]
    spec = np.fft.fft2(st)
    y, x = np.meshgrid(np.arange(n) / n, np.arange(n) / n, indexing="ij")
    for (p, q), A in (((3, 5), 0.8), ((1, 0), 1.0), ((0, 7), -0.35), ((11, 2), 0.5)):
        u = A * np.cos(2 * np.pi * (p * x + q * y))
        sym = cg - spec[q, p].real
        want = 0.25 * A * A * sym + 0.5 * m.c_F * (1 - A * A / 2)
        assert m.energy(u, eps) == pytest.approx(want, rel=1e-12, abs=1e-15)
    # pure phases: no interaction, no potential energy
    assert m.energy(np.ones((n, n)), eps) == 0.0
    assert m.energy(-np.ones((n, n)), eps) == 0.0
    # a plausible slip (1/2 for the 1/4, a dropped h^2) would change the value by O(1)
    u = 0.8 * np.cos(2 * np.pi * (3 * x + 5 * y))
    assert abs(m.energy(u, eps) - (0.5 * 0.64 * (cg - spec[5, 3].real) + 0.5 * (1 - 0.32))) > 1e-3


@pytest.mark.parametrize("b", [1, 2, 4])
def test_base_lattice_block_mean(b):
    # Noise ICs shared across lattices: node (y, x) of the n-lattice takes the mean of the
    # b x b base nodes centred on it, rows and columns b y + a, a in [-(b // 2), b - b // 2).
    n = 8
    B = b * n
    rng = np.random.default_rng(b)
    f = rng.standard_normal((B, B))
    u = O.block_mean(f, n)
    # b = 1 is the identity, bit for bit
    if b == 1:
        assert np.array_equal(u, f)
    # the n-lattice mean equals the base-lattice mean (the blocks tile the base torus)
    assert u.mean() == pytest.approx(f.mean(), rel=1e-13, abs=1e-15)
    # a single base node lands, with weight 1 / b^2, in exactly one n-node: the one whose
    # block [b y - b // 2, b y + b - b // 2) contains it (periodically)
    for Y, X in ((0, 0), (1, 2), (B - 1, B - 1), (b // 2, B - b // 2 - 1), (3 * b - 1, 5 * b)):
        e = np.zeros((B, B))
        e[Y % B, X % B] = 1.0
        ue = O.block_mean(e, n)
        ys, xs = np.nonzero(ue)
        assert len(ys) == 1 and ue[ys[0], xs[0]] == 1.0 / (b * b)
        assert ys[0] == ((Y % B) + b // 2) // b % n and xs[0] == ((X % B) + b // 2) // b % n
    # the block centroid sits within half a base cell of the node (exactly on it for odd b)
    cen = np.mean([b * 3 + a for a in range(-(b // 2), b - b // 2)])
    assert abs(cen - 3 * b) <= 0.5
    # the oracle's noise IC on the n-lattice is this block mean of its base-lattice field
    # (both fields are rounded to FP32 after they are formed: agreement to 2 FP32 ulps)
    for ic in (0, 1):
        base = model(n=B, ic=ic, ic_amp=0.05)
        coarse = model(n=n, ic=ic, ic_amp=0.05, ic_base_n=B)
        want = O.block_mean(base.initial_field(17), n)
        assert np.abs(coarse.initial_field(17) - want).max() <= 2 ** -22 * np.abs(want).max()
        fb = base.initial_field(17)
        assert abs(coarse.initial_field(17).mean() - fb.mean()) <= 2 ** -23 * np.abs(fb).max()


def test_ooi_values():
    n = 16
    assert O.ooi(np.ones((n, n))) == 1.0
    assert O.ooi(-np.ones((n, n))) == 0.0
    u = np.ones((n, n))
    u[:, : n // 2] = -1
    assert O.ooi(u) == 0.5


# --------------------------------------------------------------------------- ICs
def test_nuclei_initial_condition():
    m = model(n=128, ic=2)
    mu = np.array([0.9815, 0.9276, 0.9162, 0.9417])
    eta = np.array([[0.0072, -0.0039], [0.0232, 0.0208], [-0.0220, 0.0041], [-0.0099, 0.0118]])
    u = m.initial_field(0, theta=(mu, eta))
    assert np.abs(u).max() <= 1.0
    # far from the four nuclei the field is ~1; at a nucleus centre it is 1 - 2 mu (to
    # within the other nuclei's tails), and the four nuclei have area in phase -1
    assert u[0, 0] == pytest.approx(1.0, abs=1e-3)
    # nucleus 1 at (0.25, 0.5) + eta_1, nearest node
    iy, ix = round((0.5 + eta[0, 1]) * 128), round((0.25 + eta[0, 0]) * 128)
    # own Gaussian gives at most 1 - 2 mu_1 exp(-36 d^2) with d <= h/sqrt(2) to the node;
    # the other nuclei's tails only lower it further, and the clip keeps it >= -1
    h = 1 / 128
    assert -1.0 <= u[iy, ix] <= 1 - 2 * mu[0] * math.exp(-36 * h * h / 2) + 1e-12
    assert (u < 0).sum() > 4 * 50
    mu2, eta2 = m.draw_theta(5)
    assert np.all((mu2 >= 0.9) & (mu2 <= 1.0)) and np.all(np.abs(eta2) <= 0.025)


def test_uniform_ic_and_rounding_to_fp32():
    m = model(n=32, ic=0, ic_amp=0.05)
    u = m.initial_field(20231016)
    assert np.abs(u).max() <= 0.05
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    eps = m.sample_eps(1)
    assert eps == 0.03
    m2 = model(eps_lo=0.024, eps_hi=0.036)
    e2 = m2.sample_eps(1)
    assert 0.024 <= e2 <= 0.036 and e2 == 0.024 + 0.012 * O.uniform(1, 0, 0)


# --------------------------------------------------------------------------- collar boundary
def _outside_counts(n, R):
    """For every node of an n x n lattice: how many points of the radius-R lattice disc
    around it lie outside the lattice (counted by brute force over the disc)."""
    pts = [(dx, dy) for dy in range(-R, R + 1) for dx in range(-R, R + 1) if dx * dx + dy * dy <= R * R]
    cnt = np.zeros((n, n), dtype=np.int64)
    for y in range(n):
        for x in range(n):
            cnt[y, x] = sum(1 for dx, dy in pts if not (0 <= y + dy < n and 0 <= x + dx < n))
    return cnt


@pytest.mark.parametrize("R,uI", [(3, -1.0), (4, 0.25)])
def test_collar_L_on_constant_interior_counts_collar_points(R, uI):
    # u = c on Omega, uI on the collar: every disc point in the collar contributes
    # A h^2 (c - uI) and every interior one nothing, with A = 8 eps^2 / (pi delta^4)
    n, eps, c = 24, 0.03, 0.3
    m = model(n=n, delta=R / n, bc=1, bc_value=uI)
    A = 8 * eps ** 2 / (math.pi * (R / n) ** 4)
    got = m.apply_L(np.full((n, n), c), eps)
    want = A / n ** 2 * (c - uI) * _outside_counts(n, R)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-14)
    assert np.all(got[R:n - R, R:n - R] == 0.0)


def test_collar_one_step_closed_form():
    # one step from u = c on Omega: (c (1 + tau beta1 (c_gamma + c_F)) - tau beta1 A h^2
    # (c - uI) count) / (1 + tau beta1 c_gamma), clipped; c_gamma = A h^2 |D|
    n, R, eps, c, uI, tau = 20, 3, 0.05, 0.6, -1.0, 0.02
    m = model(n=n, delta=R / n, eps=eps, tau=tau, bc=1, bc_value=uI)
    Ah2 = 8 * eps ** 2 / (math.pi * (R / n) ** 4) / n ** 2
    D = sum(1 for dy in range(-R, R + 1) for dx in range(-R, R + 1) if dx * dx + dy * dy <= R * R)
    cg = Ah2 * D
    v = (c * (1 + tau * (cg + 1.0)) - tau * Ah2 * (c - uI) * _outside_counts(n, R)) / (1 + tau * cg)
    want = np.clip(v, -1.0, 1.0)
    got = m.step(np.full((n, n), c), eps)
    assert np.allclose(got, want, rtol=0, atol=1e-14)
    assert got[n // 2, n // 2] == pytest.approx(c * (1 + tau * (cg + 1)) / (1 + tau * cg), abs=1e-15)


def test_collar_agrees_with_periodic_away_from_the_edges():
    n, R = 32, 4
    rng = np.random.default_rng(3)
    u = rng.uniform(-1, 1, (n, n))
    per = model(n=n, delta=R / n).apply_L(u, 0.03)
    col = model(n=n, delta=R / n, bc=1, bc_value=0.7).apply_L(u, 0.03)
    assert np.array_equal(per[R:n - R, R:n - R], col[R:n - R, R:n - R])
    assert not np.allclose(per[:R], col[:R])


@pytest.mark.parametrize("uI", [-1.0, 0.0, 1.0])
def test_collar_pure_phase_matching_the_collar_is_stationary(uI):
    m = model(n=16, delta=3 / 16, tau=0.01, bc=1, bc_value=uI)
    u = np.full((16, 16), uI)
    for _ in range(3):
        u = m.step(u, 0.03)
    assert np.all(u == uI)


def test_collar_keeps_reflection_symmetry_and_bounds():
    # the collar is symmetric under x -> n-1-x, so a symmetric initial field stays symmetric
    n, R = 24, 3
    m = model(n=n, delta=R / n, tau=5e-3, bc=1, bc_value=-1.0, ic=2)
    u0 = m.initial_field(11)
    u0 = 0.5 * (u0 + u0[:, ::-1])
    uT, _ = m.solve(u0, 0.03, nsteps=40)
    assert np.abs(uT - uT[:, ::-1]).max() <= 1e-13
    assert np.abs(uT).max() <= 1.0
    # the -1 collar pulls the field down near the edges relative to the periodic solve
    uP, _ = model(n=n, delta=R / n, tau=5e-3, ic=2).solve(u0, 0.03, nsteps=40)
    assert uT.mean() < uP.mean()
