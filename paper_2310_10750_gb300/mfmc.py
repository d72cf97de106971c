"""Python binding of libmfmc (argument marshalling only).

Every function here has the name of the C entry point it calls (include/mfmc.h) and
does nothing but convert arguments: all numerical work runs in the CUDA library.
Device pointers may be passed as integers or as torch CUDA tensors (their data_ptr).
The library must have been built (``paper_2310_10750_gb300.build.build()``); importing
this module without it raises, there is no fallback.
"""
import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmfmc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libmfmc.so is not built ({LIB_PATH}); run paper_2310_10750_gb300.build.build()")

_L = ctypes.CDLL(LIB_PATH)

# ----------------------------------------------------------------------------- enums
MFMC_OK, MFMC_EINVAL, MFMC_ENOMEM, MFMC_ECUDA, MFMC_ETIMEOUT, MFMC_EBUDGET, MFMC_EBUSY, MFMC_ENOTFOUND = range(8)
KERNEL_CONSTANT, KERNEL_GAUSSIAN = 0, 1
BC_PERIODIC = 0
BC_COLLAR = 1
IC_UNIFORM, IC_SMOOTHED_GAUSS, IC_NUCLEI = 0, 1, 2
ALGO_AUTO, ALGO_DIRECT, ALGO_PREFIX, ALGO_PREFIX_KAHAN, ALGO_RESIDENT, ALGO_PLAIN, ALGO_PREFIX_TMA, ALGO_ROWS, ALGO_FFT, \
    ALGO_ACTIVE_SET, ALGO_WEIGHTED, ALGO_SPECTRAL = range(12)
MAX_MODELS = 16


class MfmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mfmc status {status}: {msg}")
        self.status = status


class mfmc_model_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("delta", ctypes.c_double), ("kernel", ctypes.c_int),
                ("delta_hf", ctypes.c_double), ("eps", ctypes.c_double), ("eps_lo", ctypes.c_double),
                ("eps_hi", ctypes.c_double), ("c_F", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("tau", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("bc", ctypes.c_int), ("ic", ctypes.c_int), ("ic_amp", ctypes.c_double),
                ("ic_base_n", ctypes.c_int), ("algo", ctypes.c_int), ("bc_value", ctypes.c_double)]


class mfmc_sample_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("has_theta", ctypes.c_int), ("mu", ctypes.c_double * 4),
                ("eta", (ctypes.c_double * 2) * 4), ("nsteps", ctypes.c_int)]


class mfmc_model_info(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int), ("disc_points", ctypes.c_int), ("c_gamma", ctypes.c_double),
                ("xi", ctypes.c_double), ("algo", ctypes.c_int), ("field_bytes", ctypes.c_size_t),
                ("tile_variant", ctypes.c_int), ("band_height", ctypes.c_int),
                ("columns_per_thread", ctypes.c_int)]


_D16 = ctypes.c_double * MAX_MODELS


class mfmc_plan_t(ctypes.Structure):
    _fields_ = [("K_sel", ctypes.c_int), ("idx", ctypes.c_int * MAX_MODELS), ("rho", _D16), ("sigma", _D16),
                ("cost", _D16), ("alpha", _D16), ("r", _D16), ("m_real", _D16),
                ("m", ctypes.c_int64 * MAX_MODELS), ("V", ctypes.c_double), ("Bmin", ctypes.c_double),
                ("mse_theory", ctypes.c_double), ("budget", ctypes.c_double),
                ("below_min_budget", ctypes.c_int), ("n_feasible", ctypes.c_int), ("n_models", ctypes.c_int),
                ("rho_all", _D16), ("sigma_all", _D16), ("mean_all", _D16)]

    def as_dict(self):
        k = self.K_sel
        return dict(K_sel=k, idx=list(self.idx[:k]), rho=list(self.rho[:k]), sigma=list(self.sigma[:k]),
                    cost=list(self.cost[:k]), alpha=list(self.alpha[:k]), r=list(self.r[:k]),
                    m_real=list(self.m_real[:k]), m=list(self.m[:k]), V=self.V, Bmin=self.Bmin,
                    mse_theory=self.mse_theory, budget=self.budget, below_min_budget=bool(self.below_min_budget),
                    n_feasible=self.n_feasible, rho_all=list(self.rho_all[:self.n_models]),
                    sigma_all=list(self.sigma_all[:self.n_models]), mean_all=list(self.mean_all[:self.n_models]))


_vp = ctypes.c_void_p
_st = ctypes.c_int


def _sig(name, res, args):
    f = getattr(_L, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("mfmc_version", ctypes.c_char_p, [])
_sig("mfmc_last_error", ctypes.c_char_p, [])
_sig("mfmc_model_create", _st, [ctypes.POINTER(mfmc_model_desc), ctypes.POINTER(_vp)])
_sig("mfmc_model_destroy", None, [_vp])
_sig("mfmc_model_query", _st, [_vp, ctypes.POINTER(mfmc_model_info)])
_sig("mfmc_model_set_tile_variant", _st, [_vp, ctypes.c_int])
_sig("mfmc_model_solver_stats", _st, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)])
_sig("mfmc_model_set_iteration_limits", _st, [_vp, ctypes.c_int, ctypes.c_int])
_sig("mfmc_model_set_band_height", _st, [_vp, ctypes.c_int, ctypes.c_int])
_sig("mfmc_sample_eps", _st, [_vp, _vp, _vp, ctypes.c_size_t, _vp])
_sig("mfmc_init_fields", _st, [_vp, _vp, _vp, ctypes.c_size_t, _vp, _vp])
_sig("mfmc_solve_fields", _st, [_vp, _vp, _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp])
_sig("mfmc_solve_fields_algo", _st, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp])
_sig("mfmc_solve_batch", _st, [_vp, _vp, _vp, ctypes.c_size_t, _vp, _vp])
_sig("mfmc_solve_batch_mixed", _st, [_vp, _vp, _vp, ctypes.c_size_t, _vp, _vp])
_sig("mfmc_pilot_stats", _st, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp])
_sig("mfmc_plan", _st, [ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_double, ctypes.c_int, _vp, ctypes.c_int,
                        ctypes.POINTER(mfmc_plan_t)])
_sig("mfmc_plan_from_stats", _st, [ctypes.c_int, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _vp, ctypes.c_int,
                                    ctypes.POINTER(mfmc_plan_t)])
_sig("mfmc_estimate", _st, [ctypes.POINTER(mfmc_plan_t), _vp, _vp])
_sig("mfmc_estimate_device", _st, [ctypes.POINTER(mfmc_plan_t), _vp, _vp, _vp])
_sig("mfmc_run", _st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, _vp,
                       ctypes.POINTER(mfmc_plan_t), _vp])


class mfmc_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("p50_latency_s", ctypes.c_double), ("p99_latency_s", ctypes.c_double),
                ("mean_latency_s", ctypes.c_double), ("samples_per_s", ctypes.c_double),
                ("peak_bytes", ctypes.c_size_t), ("peak_inflight", ctypes.c_int)]


_sig("mfmc_server_create", _st, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_vp)])
_sig("mfmc_submit", _st, [_vp, _vp, _vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)])
_sig("mfmc_poll", _st, [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)])
_sig("mfmc_request_times", _st, [_vp, ctypes.c_uint64] + [ctypes.POINTER(ctypes.c_double)] * 3)
_sig("mfmc_server_drain", _st, [_vp])
_sig("mfmc_server_get_stats", _st, [_vp, ctypes.POINTER(mfmc_server_stats)])
_sig("mfmc_server_destroy", None, [_vp])
_sig("mfmc_solve_fields_noalloc", _st, [_vp, _vp, _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp])


class mfmc_trace_record(ctypes.Structure):
    _fields_ = [("t0_ns", ctypes.c_uint64), ("t1_ns", ctypes.c_uint64), ("item", ctypes.c_uint32),
                ("sm", ctypes.c_uint32), ("kind", ctypes.c_uint32), ("step", ctypes.c_uint32)]


_sig("mfmc_trace_enable", _st, [ctypes.c_size_t])
_sig("mfmc_trace_read", _st, [ctypes.POINTER(mfmc_trace_record), ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                              ctypes.POINTER(ctypes.c_uint64)])


def _check(status):
    if status != MFMC_OK:
        raise MfmcError(status, _L.mfmc_last_error().decode())


def _ptr(x):
    """Device/host pointer from an int, None, a torch tensor or a numpy array."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def mfmc_version() -> str:
    return _L.mfmc_version().decode()


def mfmc_last_error() -> str:
    return _L.mfmc_last_error().decode()


class Model:
    """Owning wrapper of an mfmc_model handle."""

    def __init__(self, n, delta, kernel=KERNEL_CONSTANT, delta_hf=0.0, eps=0.03, eps_lo=0.0, eps_hi=0.0,
                 c_F=1.0, beta1=1.0, beta2=0.0, tau=1e-3, nsteps=200, ic=IC_UNIFORM, ic_amp=0.05, ic_base_n=0,
                 algo=ALGO_AUTO, bc=BC_PERIODIC, bc_value=-1.0):
        self.desc = mfmc_model_desc(n, delta, kernel, delta_hf, eps, eps_lo, eps_hi, c_F, beta1, beta2, tau,
                                    nsteps, bc, ic, ic_amp, ic_base_n, algo, bc_value)
        h = _vp()
        _check(_L.mfmc_model_create(ctypes.byref(self.desc), ctypes.byref(h)))
        self.handle = h.value
        self.n = n
        self.nsteps = nsteps

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _L.mfmc_model_destroy(h)
            self.handle = None

    def set_tile_variant(self, variant: int):
        _check(_L.mfmc_model_set_tile_variant(self.handle, variant))

    def set_band_height(self, rows: int, columns_per_thread: int = 4):
        _check(_L.mfmc_model_set_band_height(self.handle, rows, columns_per_thread))

    def set_iteration_limits(self, newton_max: int = 0, cg_max: int = 0):
        _check(_L.mfmc_model_set_iteration_limits(self.handle, newton_max, cg_max))

    def info(self) -> mfmc_model_info:
        out = mfmc_model_info()
        _check(_L.mfmc_model_query(self.handle, ctypes.byref(out)))
        return out


def mfmc_model_create(**kw) -> Model:
    return Model(**kw)


def mfmc_model_set_tile_variant(model: Model, variant: int):
    model.set_tile_variant(variant)


def mfmc_model_set_iteration_limits(model: Model, newton_max: int = 0, cg_max: int = 0):
    model.set_iteration_limits(newton_max, cg_max)


def mfmc_model_solver_stats(model: Model):
    """(Newton iterations, CG iterations) of the model's last beta2 > 0 solve, summed over its
    samples and steps (synchronise that solve's stream first)."""
    nw, cgi = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_L.mfmc_model_solver_stats(model.handle, ctypes.byref(nw), ctypes.byref(cgi)))
    return int(nw.value), int(cgi.value)


TRACE_SPECTRAL_QUEUE, TRACE_MIXED_STEP, TRACE_ACTIVE_SET = 1, 2, 3


def mfmc_trace_enable(capacity: int):
    """Per-work-item trace on the current device with a ring of `capacity` records (0: off)."""
    _check(_L.mfmc_trace_enable(capacity))


def mfmc_trace_read(max_records: int = 1 << 20):
    """Records written since the last read (oldest first) as a numpy structured array with
    fields t0_ns, t1_ns, item, sm, kind, step, and the count of records not returned."""
    buf = (mfmc_trace_record * max_records)()
    n, dropped = ctypes.c_size_t(0), ctypes.c_uint64(0)
    _check(_L.mfmc_trace_read(buf, max_records, ctypes.byref(n), ctypes.byref(dropped)))
    dt = np.dtype([("t0_ns", np.uint64), ("t1_ns", np.uint64), ("item", np.uint32), ("sm", np.uint32),
                   ("kind", np.uint32), ("step", np.uint32)])
    arr = np.frombuffer(bytes(buf)[:n.value * ctypes.sizeof(mfmc_trace_record)], dtype=dt).copy()
    return arr, int(dropped.value)


def make_params(ns, eps=None, theta=None, nsteps=None):
    """Array of mfmc_sample_params (eps per sample, optional nuclei theta = (mu[4], eta[4,2]),
    optional per-sample step counts)."""
    arr = (mfmc_sample_params * ns)()
    for i in range(ns):
        if eps is not None:
            arr[i].eps = float(eps[i])
        if nsteps is not None:
            arr[i].nsteps = int(nsteps[i])
        if theta is not None and theta[i] is not None:
            mu, eta = theta[i]
            arr[i].has_theta = 1
            for k in range(4):
                arr[i].mu[k] = float(mu[k])
                arr[i].eta[k][0] = float(eta[k][0])
                arr[i].eta[k][1] = float(eta[k][1])
    return arr


def _seeds(seeds):
    return np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))


def mfmc_sample_eps(model: Model, seeds, params=None) -> np.ndarray:
    s = _seeds(seeds)
    out = np.zeros(len(s))
    _check(_L.mfmc_sample_eps(model.handle, ctypes.addressof(params) if params is not None else None,
                              s.ctypes.data, len(s), out.ctypes.data))
    return out


def mfmc_init_fields(model: Model, seeds, u0, params=None, stream=None):
    s = _seeds(seeds)
    _check(_L.mfmc_init_fields(model.handle, ctypes.addressof(params) if params is not None else None,
                               s.ctypes.data, len(s), _ptr(u0), _stream(stream)))


def mfmc_solve_fields(model: Model, u0, ns, eps=None, uT=None, ubar=None, ooi=None, stream=None):
    _check(_L.mfmc_solve_fields(model.handle, _ptr(eps), _ptr(u0), ns, _ptr(uT), _ptr(ubar), _ptr(ooi),
                                _stream(stream)))


def mfmc_solve_fields_algo(model: Model, algo, u0, ns, eps=None, uT=None, ubar=None, ooi=None, stream=None):
    _check(_L.mfmc_solve_fields_algo(model.handle, algo, _ptr(eps), _ptr(u0), ns, _ptr(uT), _ptr(ubar),
                                     _ptr(ooi), _stream(stream)))


def mfmc_solve_batch(models: Sequence[Model], seeds, params=None):
    """Host seeds (and optional params) -> (ooi, ubar) host arrays."""
    s = _seeds(seeds)
    ns = len(s)
    handles = (_vp * ns)(*[m.handle for m in models])
    ooi = np.zeros(ns)
    ubar = np.zeros(ns)
    _check(_L.mfmc_solve_batch(ctypes.addressof(handles), ctypes.addressof(params) if params is not None else None,
                               s.ctypes.data, ns, ooi.ctypes.data, ubar.ctypes.data))
    return ooi, ubar


def mfmc_solve_batch_mixed(models: Sequence[Model], seeds, params=None):
    """mfmc_solve_batch with one mixed-fidelity launch per step -> (ooi, ubar) host arrays."""
    s = _seeds(seeds)
    ns = len(s)
    handles = (_vp * ns)(*[m.handle for m in models])
    ooi = np.zeros(ns)
    ubar = np.zeros(ns)
    _check(_L.mfmc_solve_batch_mixed(ctypes.addressof(handles),
                                     ctypes.addressof(params) if params is not None else None,
                                     s.ctypes.data, ns, ooi.ctypes.data, ubar.ctypes.data))
    return ooi, ubar


def mfmc_pilot_stats(K, n, ooi_dev, stream=None):
    mean, sigma, rho = np.zeros(K), np.zeros(K), np.zeros(K)
    _check(_L.mfmc_pilot_stats(K, n, _ptr(ooi_dev), mean.ctypes.data, sigma.ctypes.data, rho.ctypes.data,
                               _stream(stream)))
    return mean, sigma, rho


def mfmc_plan(pilot_ooi, costs, budget, policy=0, explicit=None) -> mfmc_plan_t:
    P = np.ascontiguousarray(np.asarray(pilot_ooi, dtype=np.float64))
    C = np.ascontiguousarray(np.asarray(costs, dtype=np.float64))
    K, n = P.shape
    out = mfmc_plan_t()
    ex = None if explicit is None else np.ascontiguousarray(np.asarray(explicit, dtype=np.int32))
    _check(_L.mfmc_plan(K, n, P.ctypes.data, C.ctypes.data, float(budget), policy,
                        None if ex is None else ex.ctypes.data, 0 if ex is None else len(ex), ctypes.byref(out)))
    return out


def mfmc_plan_from_stats(rho, sigma, costs, budget, policy=0, explicit=None) -> mfmc_plan_t:
    R = np.ascontiguousarray(np.asarray(rho, dtype=np.float64))
    S = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    C = np.ascontiguousarray(np.asarray(costs, dtype=np.float64))
    if not (len(R) == len(S) == len(C)):
        raise ValueError("rho, sigma and costs must have one entry per model")
    out = mfmc_plan_t()
    ex = None if explicit is None else np.ascontiguousarray(np.asarray(explicit, dtype=np.int32))
    _check(_L.mfmc_plan_from_stats(len(R), R.ctypes.data, S.ctypes.data, C.ctypes.data, float(budget), policy,
                                   None if ex is None else ex.ctypes.data, 0 if ex is None else len(ex),
                                   ctypes.byref(out)))
    return out


def mfmc_estimate(plan: mfmc_plan_t, lists) -> float:
    arrs = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in lists]
    ptrs = (_vp * len(arrs))(*[a.ctypes.data for a in arrs])
    est = ctypes.c_double()
    _check(_L.mfmc_estimate(ctypes.byref(plan), ctypes.addressof(ptrs), ctypes.addressof(est)))
    return est.value


def mfmc_estimate_device(plan: mfmc_plan_t, lists_dev, estimate_dev, stream=None):
    ptrs = (_vp * len(lists_dev))(*[_ptr(x) for x in lists_dev])
    _check(_L.mfmc_estimate_device(ctypes.byref(plan), ctypes.addressof(ptrs), _ptr(estimate_dev),
                                   _stream(stream)))


def mfmc_run(models: Sequence[Model], n_pilot, budget, policy=0, seed_base=0, costs=None):
    K = len(models)
    handles = (_vp * K)(*[m.handle for m in models])
    C = None if costs is None else np.ascontiguousarray(np.asarray(costs, dtype=np.float64))
    plan = mfmc_plan_t()
    est = ctypes.c_double()
    _check(_L.mfmc_run(ctypes.addressof(handles), K, n_pilot, float(budget), policy, seed_base,
                       None if C is None else C.ctypes.data, ctypes.byref(plan), ctypes.addressof(est)))
    return plan, est.value


class Server:
    """Owning wrapper of an mfmc_server (continuous-batching request loop)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int):
        h = _vp()
        _check(_L.mfmc_server_create(hbm_budget_bytes, max_slots, ctypes.byref(h)))
        self.handle = h.value

    def submit(self, model: Model, seed: int, params=None) -> int:
        t = ctypes.c_uint64()
        p = None if params is None else ctypes.addressof(params)
        _check(_L.mfmc_submit(self.handle, model.handle, p, seed, ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """(ooi, latency_s) when done, None while busy; raises for unknown tickets."""
        f, lat = ctypes.c_double(), ctypes.c_double()
        st = _L.mfmc_poll(self.handle, ticket, ctypes.byref(f), ctypes.byref(lat))
        if st == MFMC_EBUSY:
            return None
        _check(st)
        return f.value, lat.value

    def times(self, ticket: int):
        """(submit_s, admit_s, done_s) of a finished request, seconds since the server started;
        None while it runs."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = _L.mfmc_request_times(self.handle, ticket, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        if st == MFMC_EBUSY:
            return None
        _check(st)
        return a.value, b.value, c.value

    def drain(self):
        _check(_L.mfmc_server_drain(self.handle))

    def stats(self) -> dict:
        s = mfmc_server_stats()
        _check(_L.mfmc_server_get_stats(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "handle", None):
            _L.mfmc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def mfmc_server_create(hbm_budget_bytes: int, max_slots: int) -> Server:
    return Server(hbm_budget_bytes, max_slots)
