"""Oracle package (test infrastructure only).

A plain, slow FP64 CPU reference of what the GPU library computes, written from the
paper: ``nlch_oracle.c`` holds the model, its time step and the output of interest
(Section 2 and Section 4, beta2 = 0; periodic lattice or a collar holding fixed data);
``beta2_oracle.py`` holds the beta2 > 0 step (a semismooth Newton solve per step); ``mfmc_oracle.py`` holds the multifidelity
Monte Carlo statistics, model selection, allocation and estimator (Section 3).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It imports nothing from the GPU library and
the GPU library imports nothing from it.
"""
import ctypes
import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load (building first if needed) the oracle's C library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_draw.restype = ctypes.c_uint64
        L.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_uniform.restype = ctypes.c_double
        L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_normal.restype = ctypes.c_double
        L.orc_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_disc.restype = ctypes.c_int
        L.orc_disc.argtypes = [ctypes.c_double, _ip, _ip, ctypes.c_int]
        L.orc_gamma.restype = ctypes.c_double
        L.orc_gamma.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4
        L.orc_weights.restype = ctypes.c_double
        L.orc_weights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, _ip, _ip, ctypes.c_int, _dp]
        for name in ("orc_convolve", "orc_apply_L"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [ctypes.c_int, _dp, _ip, _ip, _dp, ctypes.c_int, _dp]
        L.orc_apply_L_open.restype = None
        L.orc_apply_L_open.argtypes = [ctypes.c_int, _dp, _ip, _ip, _dp, ctypes.c_int,
                                       ctypes.c_int, _dp]
        L.orc_step.restype = None
        L.orc_step.argtypes = [ctypes.c_int, _dp, _dp, _ip, _ip, _dp, ctypes.c_int,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double]
        L.orc_mean.restype = ctypes.c_double
        L.orc_mean.argtypes = [ctypes.c_int, _dp]
        L.orc_ooi.restype = ctypes.c_double
        L.orc_ooi.argtypes = [ctypes.c_int, _dp]
        L.orc_energy.restype = ctypes.c_double
        L.orc_energy.argtypes = [ctypes.c_int, _dp, _ip, _ip, _dp, ctypes.c_int, ctypes.c_double]
        L.orc_symbol.restype = ctypes.c_double
        L.orc_symbol.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _ip, _dp,
                                 ctypes.c_int]
        L.orc_initial_field.restype = None
        L.orc_initial_field.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_uint64, _dp, _dp, ctypes.c_int, _dp]
        L.orc_block_mean.restype = None
        L.orc_block_mean.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.orc_draw_theta.restype = None
        L.orc_draw_theta.argtypes = [ctypes.c_uint64, _dp, _dp]
        L.orc_sample_eps.restype = ctypes.c_double
        L.orc_sample_eps.argtypes = [ctypes.c_uint64] + [ctypes.c_double] * 3
        L.orc_solve.restype = ctypes.c_double
        L.orc_solve.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _ip, _ip, _dp, ctypes.c_int,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double]
        for name in ("orc_convolve_collar", "orc_apply_L_collar"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [ctypes.c_int, _dp, _ip, _ip, _dp, ctypes.c_int, ctypes.c_double, _dp]
        L.orc_step_collar.restype = None
        L.orc_step_collar.argtypes = [ctypes.c_int, _dp, _dp, _ip, _ip, _dp, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double]
        L.orc_solve_collar.restype = ctypes.c_double
        L.orc_solve_collar.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _ip, _ip, _dp, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_threads.restype = None
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    return a.ctypes.data_as(_ip)


# ----------------------------------------------------------------------------- RNG
def splitmix64(seed: int, pos: int) -> int:
    """Output number ``pos`` (>= 1) of the SplitMix64 sequence started at ``seed``."""
    return lib().orc_splitmix64(seed, pos)


def draw(seed: int, stream: int, idx: int) -> int:
    return lib().orc_draw(seed, stream, idx)


def uniform(seed: int, stream: int, idx: int) -> float:
    return lib().orc_uniform(seed, stream, idx)


# ----------------------------------------------------------------------------- disc
def disc(rad: float):
    """Lattice offsets (dx, dy) with dx^2 + dy^2 <= rad^2, rows of dy ascending."""
    L = lib()
    cap = (2 * int(rad) + 3) ** 2
    dx = np.zeros(cap, dtype=np.int32)
    dy = np.zeros(cap, dtype=np.int32)
    cnt = L.orc_disc(rad, _i(dx), _i(dy), cap)
    return dx[:cnt].copy(), dy[:cnt].copy()


def gamma(kind: int, r: float, eps: float, delta: float, delta_hf: float) -> float:
    return lib().orc_gamma(kind, r, eps, delta, delta_hf)


@dataclass
class OracleModel:
    """One fidelity of the model: lattice, horizon, kernel and time stepping."""
    n: int
    delta: float
    kernel: int = 0            # 0 constant on the disc, 1 truncated Gaussian
    delta_hf: float = 0.0      # Gaussian width s = delta_hf/3 (kernel 1 only)
    eps: float = 0.03
    eps_lo: float = 0.0
    eps_hi: float = 0.0
    c_F: float = 1.0
    beta1: float = 1.0
    tau: float = 1e-3
    nsteps: int = 200
    ic: int = 0                # 0 uniform, 1 smoothed Gaussian noise, 2 four nuclei
    ic_amp: float = 0.05
    ic_base_n: int = 0         # noise ICs: base lattice of the shared random field (0 = n)
    bc: int = 0                # 0 periodic lattice, 1 collar Omega_I holding the fixed value bc_value
    bc_value: float = -1.0
    _disc: Optional[tuple] = field(default=None, repr=False)

    @property
    def rad(self) -> float:
        return self.delta * self.n

    def offsets(self):
        if self._disc is None:
            self._disc = disc(self.rad)
        return self._disc

    def weights(self, eps: float):
        """Quadrature weights w_z = h^2 gamma(|z| h) and c_gamma = sum_z w_z."""
        dx, dy = self.offsets()
        w = np.zeros(len(dx), dtype=np.float64)
        cg = lib().orc_weights(self.kernel, self.n, self.delta, eps,
                               self.delta_hf if self.kernel == 1 else self.delta,
                               _i(dx), _i(dy), len(dx), _d(w))
        return w, cg

    def sample_eps(self, seed: int, eps_override: float = 0.0) -> float:
        if eps_override > 0:
            return eps_override
        return lib().orc_sample_eps(seed, self.eps, self.eps_lo, self.eps_hi)

    def initial_field(self, seed: int, theta=None) -> np.ndarray:
        """FP64 initial field rounded to FP32 values, shape (n, n)."""
        mu = np.zeros(4)
        eta = np.zeros(8)
        if self.ic == 2:
            if theta is None:
                lib().orc_draw_theta(seed, _d(mu), _d(eta))
            else:
                mu[:] = theta[0]
                eta[:] = np.asarray(theta[1], dtype=np.float64).reshape(8)
        u0 = np.zeros(self.n * self.n)
        lib().orc_initial_field(self.n, self.ic, self.ic_amp, seed, _d(mu), _d(eta),
                                self.ic_base_n, _d(u0))
        return u0.reshape(self.n, self.n)

    def draw_theta(self, seed: int):
        mu = np.zeros(4)
        eta = np.zeros(8)
        lib().orc_draw_theta(seed, _d(mu), _d(eta))
        return mu, eta.reshape(4, 2)

    # -- operators -------------------------------------------------------------
    def convolve(self, u: np.ndarray, eps: float) -> np.ndarray:
        dx, dy = self.offsets()
        w, _ = self.weights(eps)
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        if self.bc == 1:
            lib().orc_convolve_collar(self.n, _d(u), _i(dx), _i(dy), _d(w), len(dx), self.bc_value, _d(out))
        else:
            lib().orc_convolve(self.n, _d(u), _i(dx), _i(dy), _d(w), len(dx), _d(out))
        return out

    def apply_L(self, u: np.ndarray, eps: float) -> np.ndarray:
        dx, dy = self.offsets()
        w, _ = self.weights(eps)
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        if self.bc == 1:
            lib().orc_apply_L_collar(self.n, _d(u), _i(dx), _i(dy), _d(w), len(dx), self.bc_value, _d(out))
        else:
            lib().orc_apply_L(self.n, _d(u), _i(dx), _i(dy), _d(w), len(dx), _d(out))
        return out

    def apply_L_open(self, u: np.ndarray, eps: float) -> np.ndarray:
        dx, dy = self.offsets()
        w, _ = self.weights(eps)
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        lib().orc_apply_L_open(self.n, _d(u), _i(dx), _i(dy), _d(w), len(dx),
                               int(math.floor(self.rad + 1e-9)), _d(out))
        return out

    def symbol(self, p: int, q: int, eps: float) -> float:
        dx, dy = self.offsets()
        w, _ = self.weights(eps)
        return lib().orc_symbol(self.n, p, q, _i(dx), _i(dy), _d(w), len(dx))

    def energy(self, u: np.ndarray, eps: float) -> float:
        dx, dy = self.offsets()
        w, _ = self.weights(eps)
        u = np.ascontiguousarray(u, dtype=np.float64)
        return lib().orc_energy(self.n, _d(u), _i(dx), _i(dy), _d(w), len(dx), self.c_F)

    def step(self, u: np.ndarray, eps: float) -> np.ndarray:
        dx, dy = self.offsets()
        w, cg = self.weights(eps)
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        if self.bc == 1:
            lib().orc_step_collar(self.n, _d(u), _d(out), _i(dx), _i(dy), _d(w), len(dx), cg, self.c_F,
                                  self.tau, self.beta1, self.bc_value)
        else:
            lib().orc_step(self.n, _d(u), _d(out), _i(dx), _i(dy), _d(w), len(dx), cg, self.c_F,
                           self.tau, self.beta1)
        return out

    def solve(self, u0: np.ndarray, eps: float, nsteps: Optional[int] = None):
        """Run the time steps from u0; returns (u(T), mean of u(T))."""
        dx, dy = self.offsets()
        w, cg = self.weights(eps)
        u = np.ascontiguousarray(u0, dtype=np.float64).copy()
        k = self.nsteps if nsteps is None else nsteps
        if self.bc == 1:
            mean = lib().orc_solve_collar(self.n, _d(u), k, _i(dx), _i(dy), _d(w), len(dx), cg, self.c_F,
                                          self.tau, self.beta1, self.bc_value)
        else:
            mean = lib().orc_solve(self.n, _d(u), k, _i(dx), _i(dy), _d(w), len(dx), cg, self.c_F,
                                   self.tau, self.beta1)
        return u, mean

    def solve_sample(self, seed: int, eps_override: float = 0.0, theta=None,
                     nsteps: Optional[int] = None):
        """Initial field from the seed, solve, and return (f, mean, u(T), eps)."""
        eps = self.sample_eps(seed, eps_override)
        u0 = self.initial_field(seed, theta)
        uT, mean = self.solve(u0, eps, nsteps)
        return 0.5 * (1.0 + mean), mean, uT, eps


def block_mean(f: np.ndarray, n: int) -> np.ndarray:
    """Mean of the b x b base-lattice blocks of f (B x B, B = b n) around each n-lattice node,
    the map the noise initial conditions use to share one random field across lattices."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    u = np.zeros((n, n))
    lib().orc_block_mean(n, f.shape[0], _d(f), _d(u))
    return u


def ooi(u: np.ndarray) -> float:
    """Eq. (ooi) on a lattice field."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_ooi(u.shape[0], _d(u))


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(t: int) -> None:
    lib().orc_set_threads(t)
