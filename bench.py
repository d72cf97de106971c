"""Benchmark of the hot path: batched time integration of the nonlocal Cahn-Hilliard
model (constant kernel, obstacle projection, OoI reduction) on one GB300 per rank.

Workload: single fidelity, 256 x 256 lattice, delta = 8h (197-point disc), 1000 steps,
512 samples per GPU, eps = 0.02 U[0.8, 1.2], initial field = Gaussian noise (sigma 0.05)
averaged over the 5-point stencil and clipped.  One bench step = one solve of the whole
batch.  The two field buffers (2 x 128 MiB) exceed the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Profiling cases (for ncu captures, never bench values): --nsteps, --samples and --algo
shrink or pin the solve, --no-e2e / --no-plain / --no-cpu-baseline drop the extra legs.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded sample of
the same workload.  Under torchrun each rank solves its own 512 samples (weak scaling,
replicas: no collective on the data path; only the timing max uses one).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_LATTICE, R_CELLS, NSTEPS, NSAMPLES = 256, 8, 1000, 512
EPS, EPS_LO, EPS_HI, TAU, SIGMA = 0.02, 0.016, 0.024, 1e-3, 0.05
SEED_BASE = 20231016 + 1000003 * 1
METRIC = "grid-pt updates/s"
WORKLOAD = "single fidelity 256x256, delta=8h (197-pt disc), constant kernel, 1000 steps, 512 samples/GPU"


BC = 0            # 0 periodic (the headline), 1 collar holding BC_VALUE (--bc collar)
BC_VALUE = -1.0


def config(algo=None):
    c = {"workload": WORKLOAD if (NSTEPS, NSAMPLES) == (1000, 512) else "profiling case: " + WORKLOAD,
         "n": N_LATTICE, "R": R_CELLS, "disc_points": 197, "nsteps": NSTEPS, "samples_per_gpu": NSAMPLES, "tau": TAU, "eps": "0.02*U[0.8,1.2]", "ic": "smoothed Gaussian sigma=0.05",
         "l2": "inputs larger than L2 (2 x 128 MiB field buffers per solve, L2 129 MB)"}
    if algo is not None:
        c["algo"] = algo
    if BC == 1:
        c["workload"] += f", collar boundary (fixed value {BC_VALUE:g} on the interaction collar)"
        c["boundary"] = {"kind": "collar", "value": BC_VALUE}
    return c


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()) if rows else None,
                "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(seconds=12.0):
    """The FP64 oracle on the host cores on a bounded sample of the workload: samples 0, 1, ...
    of the 512, each for as many of its 1000 steps as fit, until about `seconds` of CPU work.
    Returns the baseline record and the oracle's solutions (seed, steps, f, mean, u(T))."""
    import oracle
    o = oracle.OracleModel(n=N_LATTICE, delta=R_CELLS / N_LATTICE, eps=EPS, eps_lo=EPS_LO, eps_hi=EPS_HI,
                           tau=TAU, nsteps=NSTEPS, ic=1, ic_amp=SIGMA, bc=BC, bc_value=BC_VALUE)
    seed = SEED_BASE
    eps = o.sample_eps(seed)
    u0 = o.initial_field(seed)
    t = time.perf_counter()
    o.solve(u0, eps, nsteps=10)
    dt10 = time.perf_counter() - t
    steps = int(max(10, min(NSTEPS, 10 * seconds / max(dt10, 1e-6))))
    pts, dt, done, sols = 0, 0.0, 0, []
    while done < 64 and (dt < seconds or done == 0):
        s = SEED_BASE + done
        eps, u0 = o.sample_eps(s), o.initial_field(s)
        t = time.perf_counter()
        uT, mean = o.solve(u0, eps, nsteps=steps)
        dt += time.perf_counter() - t
        pts += N_LATTICE * N_LATTICE * steps
        sols.append((s, steps, 0.5 * (1.0 + mean), mean, uT))
        done += 1
    return ({"value": pts / dt, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
             "sample": f"{done} sample(s) of 256x256, {steps} of 1000 steps each, FP64 direct disc sum ({dt:.1f} s)"},
            sols)


def oracle_check(mfmc, sols, algo_req):
    """The GPU path (the benchmark's algorithm, one batch) on the samples the CPU baseline solved,
    against the FP64 oracle's solutions: OoI (relative), mean of u and the field (absolute), and
    the bounds [-1, 1]."""
    import numpy as np
    import torch
    if not sols:
        return None
    steps = sols[0][1]
    g = mfmc.Model(n=N_LATTICE, delta=R_CELLS / N_LATTICE, eps=EPS, eps_lo=EPS_LO, eps_hi=EPS_HI, tau=TAU,
                   nsteps=steps, ic=mfmc.IC_SMOOTHED_GAUSS, ic_amp=SIGMA, algo=algo_req, bc=BC, bc_value=BC_VALUE)
    seeds = np.array([s for s, _, _, _, _ in sols], dtype=np.uint64)
    k = len(seeds)
    u0 = torch.empty((k, N_LATTICE, N_LATTICE), dtype=torch.float32, device="cuda")
    uT = torch.empty_like(u0)
    f = torch.empty(k, dtype=torch.float64, device="cuda")
    ubar = torch.empty(k, dtype=torch.float64, device="cuda")
    eps = torch.tensor(mfmc.mfmc_sample_eps(g, seeds), dtype=torch.float64, device="cuda")
    mfmc.mfmc_init_fields(g, seeds, u0)
    mfmc.mfmc_solve_fields(g, u0, k, eps=eps, uT=uT, ubar=ubar, ooi=f)
    torch.cuda.synchronize()
    uT, f, ubar = uT.cpu().numpy().astype(np.float64), f.cpu().numpy(), ubar.cpu().numpy()
    rel, dm, du = 0.0, 0.0, 0.0
    for i, (_, _, fr, mr, ur) in enumerate(sols):
        rel = max(rel, abs(f[i] - fr) / abs(fr))
        dm = max(dm, abs(ubar[i] - mr))
        du = max(du, float(np.abs(uT[i] - ur).max()))
    return {"samples": k, "steps": steps, "max_rel_ooi_err": rel, "max_abs_ubar_err": dm,
            "max_abs_field_err": du, "bounds_exact": bool(np.abs(uT).max() <= 1.0),
            "target_rel_ooi_err": 1e-5, "algo": g.info().algo,
            "what": "GPU (FP32 fields) vs FP64 CPU oracle, the first samples of the timed batch's seeds"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    o = oracle.OracleModel(n=N_LATTICE, delta=R_CELLS / N_LATTICE, eps=EPS, eps_lo=EPS_LO, eps_hi=EPS_HI,
                           tau=TAU, nsteps=NSTEPS, ic=1, ic_amp=SIGMA)
    seed = SEED_BASE
    eps = o.sample_eps(seed)
    u0 = o.initial_field(seed)
    steps_per = 20
    for _ in range(args.warmup):
        o.solve(u0, eps, nsteps=2)
    t = time.perf_counter()
    for k in range(args.steps):
        o.solve(u0, eps, nsteps=steps_per)
    dt = time.perf_counter() - t
    pts = N_LATTICE * N_LATTICE * steps_per * args.steps
    v = pts / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config("oracle FP64 direct sum"),
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"each step: sample 0 of the workload, {steps_per} of 1000 time steps"},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    global NSTEPS, NSAMPLES, BC, BC_VALUE
    NSTEPS = args.nsteps or NSTEPS
    NSAMPLES = args.samples or NSAMPLES
    BC = 1 if args.bc == "collar" else 0
    BC_VALUE = args.bc_value
    ws, rank, local = dist_env()
    from paper_2310_10750_gb300 import build as pkg_build
    if rank == 0:
        pkg_build.build()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
    else:
        torch.cuda.set_device(local)
    from paper_2310_10750_gb300 import mfmc, replicas
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    algo_req = {"auto": mfmc.ALGO_AUTO, "prefix": mfmc.ALGO_PREFIX, "direct": mfmc.ALGO_DIRECT,
                "kahan": mfmc.ALGO_PREFIX_KAHAN, "tma": mfmc.ALGO_PREFIX_TMA, "rows": mfmc.ALGO_ROWS,
                "fft": mfmc.ALGO_FFT}[args.algo]
    model = mfmc.Model(n=N_LATTICE, delta=R_CELLS / N_LATTICE, eps=EPS, eps_lo=EPS_LO, eps_hi=EPS_HI, tau=TAU,
                       nsteps=NSTEPS, ic=mfmc.IC_SMOOTHED_GAUSS, ic_amp=SIGMA, algo=algo_req, bc=BC,
                       bc_value=BC_VALUE)
    if args.tile_variant >= 0:
        model.set_tile_variant(args.tile_variant)
    if args.band_height >= 0:
        model.set_band_height(args.band_height, args.columns)
    ns = NSAMPLES
    first, last = replicas.shard(ws * ns, ws, rank)  # this rank's own ns samples (weak scaling)
    seeds = np.arange(first, last, dtype=np.uint64) + np.uint64(SEED_BASE)
    u0 = torch.empty((ns, N_LATTICE, N_LATTICE), dtype=torch.float32, device="cuda")
    ooi = torch.empty(ns, dtype=torch.float64, device="cuda")
    eps = torch.tensor(mfmc.mfmc_sample_eps(model, seeds), dtype=torch.float64, device="cuda")
    mfmc.mfmc_init_fields(model, seeds, u0, stream=stream)
    for _ in range(args.warmup):
        mfmc.mfmc_solve_fields(model, u0, ns, eps=eps, ooi=ooi, stream=stream)
    torch.cuda.synchronize()
    algo_names = {1: "direct", 2: "prefix", 3: "prefix-kahan", 4: "resident", 5: "plain", 6: "prefix-tma",
                  7: "row-stream", 8: "fft"}
    algo = algo_names.get(model.info().algo, str(model.info().algo))
    if algo == "prefix-tma":
        algo += f" (tile variant {model.info().tile_variant})"
    if algo == "row-stream":
        algo += f" (band height {model.info().band_height}, {model.info().columns_per_thread} columns/thread)"

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            mfmc.mfmc_solve_fields(model, u0, ns, eps=eps, ooi=ooi, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), ws)
    ms_step = ms / args.steps
    pts_step = ws * ns * N_LATTICE * N_LATTICE * NSTEPS
    value = pts_step / (ms_step * 1e-3)
    clocks = clk.summary()

    # end to end through the batch call: host seeds in, host OoIs out
    e2e_s = None
    h2d = ns * (8 + 8 + 12 * 8)       # seeds, eps, nuclei parameters (uploaded for every IC)
    d2h = ns * 2 * 8                  # OoI and mean per sample
    if not args.no_e2e:
        models = [model] * ns
        mfmc.mfmc_solve_batch(models, seeds)          # warm the batch buffers
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t = time.perf_counter()
        for _ in range(args.steps):
            f_host, _ = mfmc.mfmc_solve_batch(models, seeds)
        e2e_s = replicas.max_over_ranks((time.perf_counter() - t) / args.steps, ws)

    # plain form: one sample per launch, one launch per step (same GPU), on 4 samples
    plain_sps = None
    if not args.no_plain:
        plain_ns = 4
        ooi_p = torch.empty(plain_ns, dtype=torch.float64, device="cuda")
        mfmc.mfmc_solve_fields_algo(model, mfmc.ALGO_PLAIN, u0, 1, eps=eps, ooi=ooi_p, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        mfmc.mfmc_solve_fields_algo(model, mfmc.ALGO_PLAIN, u0, plain_ns, eps=eps, ooi=ooi_p, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plain_sps = plain_ns / (e0.elapsed_time(e1) * 1e-3)
    batched_sps = ws * ns / (ms_step * 1e-3)

    peak_gbs, sm_max, peak_kind = load_peaks()
    # step kernels, then coefficients and the OoI finalisation, and either the padding kernel (tile
    # kernels) or the field reduction (row-streaming kernel, whose initial copy is a memcpy)
    launches_per_solve = NSTEPS + 3
    kernel_ms = ms_step / NSTEPS  # average step-kernel launch (upper bound: includes launch gaps)
    bytes_launch = 8.0 * ns * N_LATTICE * N_LATTICE
    achieved = bytes_launch / (kernel_ms * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            tr = json.load(open(tpath))
            key = f"{N_LATTICE}_{R_CELLS}_{algo.split(' (')[0]}" + ("_collar" if BC == 1 else "")
            if key in tr:
                traffic = tr[key]
        except Exception:
            traffic = None
    instr_per_pt = 4 * R_CELLS + 9
    alu_peak = 152 * 128 * sm_max * 1e6 / 1e12
    alu_achieved = instr_per_pt * ns * N_LATTICE * N_LATTICE / (kernel_ms * 1e-3) / 1e12

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(algo),
                "samples_per_s": batched_sps,
                "plain_form": None if plain_sps is None else {
                    "samples_per_s": plain_sps, "speedup_batched_vs_plain": batched_sps / plain_sps,
                    "what": "one sample per launch, one launch per step, direct disc sum"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                             "frac": achieved / peak_gbs, "traffic": traffic, "peak_kind": peak_kind,
                             "kernel": ("step_rows_kernel" if algo.startswith("row-stream") else
                                        "step_tma_kernel" if algo.startswith("prefix-tma") else "step_tile_kernel")
                                       + f" ({algo})", "algorithmic_bytes_per_launch": bytes_launch,
                             "avg_launch_ms": kernel_ms},
                "roofline_alu": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "T instr/s",
                                 "frac": alu_achieved / alu_peak, "instr_per_point": instr_per_pt},
                "e2e": None if e2e_s is None else {
                    "value": ws * ns * N_LATTICE * N_LATTICE * NSTEPS / e2e_s, "unit": METRIC,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "what": "mfmc_solve_batch: host seeds -> device initial fields -> solve -> host OoIs"},
                "gpu_launches": args.steps * launches_per_solve,
                "clocks": clocks}
        if not args.no_cpu_baseline:
            line["cpu_baseline"], sols = cpu_baseline()
            line["oracle_check"] = oracle_check(mfmc, sols, algo_req)
        if not args.no_extras and ws == 1:
            # the metric's other parts run after the headline is measured; a failure among them
            # is reported in the line instead of losing the line
            try:
                line.update(extra_metrics(mfmc, model, algo_req, ns, ms_step, args))
            except Exception as e:  # noqa: BLE001
                line["extras_error"] = f"{type(e).__name__}: {e}"
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------- other workloads
def _seeds(base, count, offset=0):
    import numpy as np
    return (np.arange(count, dtype=np.uint64) + np.uint64(base + offset))


def _batched_cost(mfmc, model, ns, seed_base):
    """GPU seconds per sample of a batched solve (fields built on the device)."""
    import numpy as np
    import torch
    n = model.n
    seeds = _seeds(seed_base, ns)
    u0 = torch.empty((ns, n, n), dtype=torch.float32, device="cuda")
    ooi = torch.empty(ns, dtype=torch.float64, device="cuda")
    eps = torch.tensor(mfmc.mfmc_sample_eps(model, seeds), dtype=torch.float64, device="cuda")
    mfmc.mfmc_init_fields(model, seeds, u0)
    mfmc.mfmc_solve_fields(model, u0, ns, eps=eps, ooi=ooi)      # tune + warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    mfmc.mfmc_solve_fields(model, u0, ns, eps=eps, ooi=ooi)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / ns


def hierarchy_metrics(mfmc, n_val, budgets=(10.0, 30.0, 100.0, 300.0), reps=10, plain=True):
    """MFMC hierarchy with a fixed physical horizon delta = 1/32 (512^2/R=16, 256^2/8,
    128^2/4, 64^2/2), 1000 steps, the four-nuclei initial condition of Eq. (ic) whose
    theta is the shared random input, eps = 0.02 U[0.8, 1.2].  Pilot of 64 samples,
    costs measured as batched GPU seconds per sample, `reps` replicate MC and MFMC estimates
    per budget B = b C_1, MSE against a validation mean of n_val HF samples (Section 3,
    Eqs. mse_error and error_theory)."""
    import numpy as np
    import torch
    base = 20231016 + 1000003 * 2
    levels = [(512, 16), (256, 8), (128, 4), (64, 2)]
    common = dict(eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, nsteps=1000, ic=mfmc.IC_NUCLEI)
    models = [mfmc.Model(n=n, delta=R / n, **common) for n, R in levels]
    cost = [_batched_cost(mfmc, m, bs, base + 10 ** 7) for m, bs in zip(models, (128, 512, 1024, 2048))]
    names = {1: "direct", 2: "prefix", 4: "resident", 6: "prefix-tma", 7: "row-stream"}
    algos = [names.get(m.info().algo, str(m.info().algo)) for m in models]
    plain_cost = None
    if plain:
        m0 = models[0]
        u0 = torch.empty((1, 512, 512), dtype=torch.float32, device="cuda")
        mfmc.mfmc_init_fields(m0, _seeds(base, 1), u0)
        ooi = torch.empty(1, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mfmc.mfmc_solve_fields_algo(m0, mfmc.ALGO_PLAIN, u0, 1, ooi=ooi)
        e1.record()
        torch.cuda.synchronize()
        plain_cost = e0.elapsed_time(e1) * 1e-3
    # pilot on shared seeds
    n_pilot = 64
    pilot = np.stack([mfmc.mfmc_solve_batch([m] * n_pilot, _seeds(base, n_pilot))[0] for m in models])
    # validation mean of the high-fidelity OoI
    t = time.perf_counter()
    chunk = 4096                                         # bounded device memory per call
    fval = np.concatenate([mfmc.mfmc_solve_batch([models[0]] * min(chunk, n_val - o),
                                                 _seeds(base, min(chunk, n_val - o), 5 * 10 ** 6 + o))[0]
                           for o in range(0, n_val, chunk)])
    q_val = float(np.mean(fval))
    t_val = time.perf_counter() - t
    rows = []
    next_seed = [base + 10 ** 5]

    def take(count):
        s0 = next_seed[0]
        next_seed[0] += count
        return s0

    plan = None
    for b in budgets:
        B = b * cost[0]
        plan = mfmc.mfmc_plan(pilot, cost, B, 0)
        p = plan.as_dict()
        est_mfmc, est_mc = [], []
        for r in range(reps):
            s0 = take(p["m"][-1])
            lists = []
            for j, i in enumerate(p["idx"]):
                f, _ = mfmc.mfmc_solve_batch([models[i]] * p["m"][j], _seeds(s0, p["m"][j]))
                lists.append(f)
            est_mfmc.append(mfmc.mfmc_estimate(plan, lists))
            m_mc = max(1, int(B // cost[0]))
            s1 = take(m_mc)
            f, _ = mfmc.mfmc_solve_batch([models[0]] * m_mc, _seeds(s1, m_mc))
            est_mc.append(float(np.mean(f)))
        mse_mfmc = float(np.mean((np.array(est_mfmc) - q_val) ** 2))
        mse_mc = float(np.mean((np.array(est_mc) - q_val) ** 2))
        sig1 = p["sigma_all"][0]
        row = {"budget_gpu_s": B, "budget_over_C1": b, "subset": p["idx"], "m": p["m"],
               "below_min_budget": p["below_min_budget"], "mse_mfmc": mse_mfmc, "mse_mc": mse_mc,
               "mse_mfmc_per_gpu_s": mse_mfmc * B, "mse_mc_per_gpu_s": mse_mc * B,
               "mse_mfmc_theory": p["mse_theory"], "mse_mc_theory": sig1 ** 2 / max(1, int(B // cost[0])),
               "mse_ratio_mc_over_mfmc": mse_mc / mse_mfmc if mse_mfmc > 0 else None,
               "validation_mse_floor": float(np.var(fval, ddof=1)) / n_val}
        if plain_cost:
            row["mse_mc_plain_loop_theory"] = sig1 ** 2 / max(1e-9, B / plain_cost)
        rows.append(row)
    return {"workload": "MFMC hierarchy delta=1/32: 512^2/R16, 256^2/R8, 128^2/R4, 64^2/R2, 1000 steps, nuclei IC "
                        f"(Eq. ic), pilot 64, {reps} replicates per budget, validation mean of {n_val} HF samples",
            "algos": algos, "cost_gpu_s_per_sample": cost, "samples_per_s_per_fidelity": [1.0 / c for c in cost],
            "plain_loop_cost_gpu_s_per_hf_sample": plain_cost,
            "pilot_rho": plan.as_dict()["rho_all"], "pilot_sigma": plan.as_dict()["sigma_all"],
            "q_validation": q_val, "n_validation": n_val, "validation_s": t_val, "budgets": rows}


def run_hierarchy(args):
    from paper_2310_10750_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2310_10750_gb300 import mfmc
    h = hierarchy_metrics(mfmc, args.validation, plain=not args.no_plain)
    rows = h["budgets"]
    line = {"metric": "MFMC MSE per GPU-s (hierarchy)", "value": rows[2]["mse_mfmc"], "unit": "MSE at B = 100 C_1",
            "higher_is_better": False, "data": "synthetic", "config": {"workload": h["workload"], "algos": h["algos"]}}
    line.update({k: v for k, v in h.items() if k not in ("workload", "algos")})
    print(json.dumps(line), flush=True)
    return 0


def serving_metrics(mfmc, total, load=0.8):
    """Poisson stream of solve requests of mixed fidelity (64^2 .. 1024^2 in 40/30/20/8/2 %,
    delta = 1/32, 500-2000 steps each) through the continuous-batching server: the capacity
    (2000 requests submitted at once), then `total` requests at `load` x that capacity (above 1:
    an overload, in which requests wait for slots and the latencies grow with the backlog)."""
    import numpy as np
    rng = np.random.default_rng(20231016 + 1000003 * 3)
    sizes = [64, 128, 256, 512, 1024]
    probs = [0.40, 0.30, 0.20, 0.08, 0.02]
    models = {n: mfmc.Model(n=n, delta=(n // 32) / n, eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3,
                            nsteps=1000, ic=mfmc.IC_SMOOTHED_GAUSS, ic_amp=0.05) for n in sizes}
    for n, m in models.items():                           # tune each fidelity before serving
        mfmc.mfmc_solve_batch([m] * 8, _seeds(1, 8))
    kinds = rng.choice(sizes, size=total, p=probs)
    steps = rng.integers(500, 2001, size=total)

    def run_stream(count, rate):
        srv = mfmc.Server(120 << 30, 8192)
        gaps = rng.exponential(1.0 / rate, size=count) if rate else np.zeros(count)
        t0 = time.perf_counter()
        t_next = t0
        tickets = []
        for i in range(count):
            t_next += gaps[i]
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                time.sleep(min(0.0005, t_next - now))
            p = mfmc.make_params(1, nsteps=[int(steps[i])])
            tickets.append(srv.submit(models[int(kinds[i])], 7 + i, params=p[0]))
        srv.drain()
        wall = time.perf_counter() - t0
        st = srv.stats()
        for t in tickets:
            srv.poll(t)
        srv.close()
        return st, wall

    cap_n = min(2000, total)
    st_cap, wall_cap = run_stream(cap_n, 0.0)              # all at once: capacity
    capacity = cap_n / wall_cap
    st, wall = run_stream(total, load * capacity)
    return {"workload": f"{total} requests, Poisson at {load:g} x measured capacity, n in 64..1024 "
                        "(40/30/20/8/2 %), R = n/32, 500-2000 steps, 120 GB budget",
            "p50_latency_s": st["p50_latency_s"], "p99_latency_s": st["p99_latency_s"],
            "mean_latency_s": st["mean_latency_s"], "samples_per_s": st["samples_per_s"],
            "capacity_samples_per_s": capacity, "arrival_rate": load * capacity, "wall_s": wall,
            "completed": st["completed"], "peak_inflight": st["peak_inflight"], "peak_bytes": st["peak_bytes"]}


def run_serving(args):
    from paper_2310_10750_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2310_10750_gb300 import mfmc
    sv = serving_metrics(mfmc, args.requests, args.load)
    line = {"metric": "p50/p99 solve latency (serving)", "value": sv["p99_latency_s"], "unit": "s (p99)",
            "higher_is_better": False, "data": "synthetic", "config": {"workload": sv["workload"]}}
    line.update({k: v for k, v in sv.items() if k != "workload"})
    print(json.dumps(line), flush=True)
    return 0


def fidelity_roofline(mfmc, n, algo, pts_per_s, peak_gbs, sm_max):
    """Fractions of a fidelity's step roofline: the HBM term (algorithmic bytes per point-step at
    the measured copy bandwidth: 8 B of field for the streamed disc-sum kernels; the half
    spectrum read and written by both passes plus the field for the streamed spectral form;
    none for the forms that keep the whole solve on chip) and the ALU term in units of the
    prefix form's 4R + 9 instructions per point against 152 SMs x 128 FP32 lanes."""
    R = n // 32
    on_chip = algo == mfmc.ALGO_RESIDENT or (algo == mfmc.ALGO_SPECTRAL and n <= 128)
    if algo == mfmc.ALGO_SPECTRAL and not on_chip:
        bytes_pt = (4 * n * (n // 2 + 1) * 8 + 2 * n * n * 4) / (n * n)
    else:
        bytes_pt = 8.0
    return {"hbm_frac": None if on_chip else pts_per_s * bytes_pt / (peak_gbs * 1e9),
            "hbm_bytes_per_point_step": None if on_chip else bytes_pt,
            "alu_frac_prefix_model": pts_per_s * (4 * R + 9) / (152 * 128 * sm_max * 1e6)}


def fidelity_rates(mfmc):
    """Batched samples/s of each fidelity of the serving mix (delta = 1/32: n = 64 .. 1024,
    R = n/32, 1000 steps, smoothed-noise IC), each batch large enough to fill the GPU, with the
    fractions of its step roofline."""
    peak_gbs, sm_max, _ = load_peaks()
    base = 20231016 + 1000003 * 6
    out = {}
    for n, bs in ((64, 4096), (128, 2048), (256, 512), (512, 128), (1024, 64)):
        m = mfmc.Model(n=n, delta=(n // 32) / n, eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, nsteps=1000,
                       ic=mfmc.IC_SMOOTHED_GAUSS, ic_amp=0.05)
        c = _batched_cost(mfmc, m, bs, base)
        algo = m.info().algo
        pps = n * n * 1000 / c
        out[f"{n}x{n}_R{n // 32}"] = {"samples_per_s": 1.0 / c, "batch": bs, "algo": algo,
                                      "grid_pt_updates_per_s": pps,
                                      "roofline": fidelity_roofline(mfmc, n, algo, pps, peak_gbs, sm_max)}
    return out


def extra_metrics(mfmc, model, algo_req, ns, ms_step, args):
    """The metric's other parts, measured after the headline timing so that they cannot
    perturb it: the plain form on the benchmark's own kernel, samples/s per fidelity, serving
    latency (the full request stream) and MFMC MSE per GPU-second at B = 100 C_1."""
    import numpy as np
    import torch
    out = {}
    # one sample per launch, one launch per step, with the kernel the batched path uses
    k = 4
    algo = model.info().algo
    seeds = np.arange(k, dtype=np.uint64) + np.uint64(SEED_BASE)
    u0 = torch.empty((k, N_LATTICE, N_LATTICE), dtype=torch.float32, device="cuda")
    ooi = torch.empty(k, dtype=torch.float64, device="cuda")
    eps = torch.tensor(mfmc.mfmc_sample_eps(model, seeds), dtype=torch.float64, device="cuda")
    mfmc.mfmc_init_fields(model, seeds, u0)
    mfmc.mfmc_solve_fields_algo(model, algo, u0[:1], 1, eps=eps[:1], ooi=ooi[:1])  # warm (graph capture)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(k):
        mfmc.mfmc_solve_fields_algo(model, algo, u0[i:i + 1], 1, eps=eps[i:i + 1], ooi=ooi[i:i + 1])
    e1.record()
    torch.cuda.synchronize()
    plain_sps = k / (e0.elapsed_time(e1) * 1e-3)
    batched_sps = ns / (ms_step * 1e-3)
    out["plain_form_same_kernel"] = {"samples_per_s": plain_sps, "speedup_batched_vs_plain": batched_sps / plain_sps,
                                     "algo": algo, "what": "the batched path's own kernel, one sample per launch, "
                                                           "one launch per step (4 samples)"}
    t = time.perf_counter()
    out["samples_per_s_per_fidelity"] = fidelity_rates(mfmc)
    out["serving"] = serving_metrics(mfmc, args.requests)
    h = hierarchy_metrics(mfmc, args.validation, budgets=(100.0,), reps=10, plain=False)
    r = h["budgets"][0]
    out["mfmc"] = {"workload": h["workload"], "budget_over_C1": 100.0, "budget_gpu_s": r["budget_gpu_s"],
                   "mse_mfmc": r["mse_mfmc"], "mse_mc": r["mse_mc"], "mse_mfmc_per_gpu_s": r["mse_mfmc_per_gpu_s"],
                   "mse_mc_per_gpu_s": r["mse_mc_per_gpu_s"], "mse_ratio_mc_over_mfmc": r["mse_ratio_mc_over_mfmc"],
                   "mse_mfmc_theory": r["mse_mfmc_theory"], "mse_mc_theory": r["mse_mc_theory"],
                   "validation_mse_floor": r["validation_mse_floor"], "n_validation": h["n_validation"],
                   "subset": r["subset"], "m": r["m"], "cost_gpu_s_per_sample": h["cost_gpu_s_per_sample"],
                   "algos": h["algos"]}
    out["extras_wall_s"] = time.perf_counter() - t
    return out


def run_large(args):
    """1024^2, delta = 32h (3209-point disc), 2000 steps, 64 samples: throughput of the
    autotuned algorithm, of the direct sum and of the spectral (cuFFT) form of the disc sum.
    (The FP32 / compensated sums against the oracle are a test: tests/test_large_hf_gpu.py.)"""
    from paper_2310_10750_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2310_10750_gb300 import mfmc
    n, R, steps, ns = 1024, 32, 2000, 64
    profiling = args.nsteps > 0  # a short solve for ncu: the main model only
    if profiling:
        steps = args.nsteps
    if args.samples > 0:
        ns = args.samples
    base = 20231016 + 1000003 * 4
    kw = dict(n=n, delta=R / n, eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, ic=mfmc.IC_SMOOTHED_GAUSS,
              ic_amp=0.05)
    pin = {"auto": mfmc.ALGO_AUTO, "spectral": mfmc.ALGO_SPECTRAL, "fft": mfmc.ALGO_FFT,
           "tma": mfmc.ALGO_PREFIX_TMA}.get(args.algo, mfmc.ALGO_AUTO)
    model = mfmc.Model(nsteps=steps, algo=pin, **kw)
    c = _batched_cost(mfmc, model, ns, base)
    names = {1: "direct", 2: "prefix", 4: "resident", 6: "prefix-tma", 7: "row-stream", 8: "fft", 11: "spectral"}
    algo = names.get(model.info().algo, str(model.info().algo))
    if algo == "prefix-tma":
        algo += f" (tile variant {model.info().tile_variant})"
    direct_c = fft_c = spec_c = None
    if not args.no_plain and not profiling:
        md = mfmc.Model(nsteps=20, algo=mfmc.ALGO_DIRECT, **kw)
        direct_c = _batched_cost(mfmc, md, ns, base) * steps / 20
    if not profiling:
        mf_ = mfmc.Model(nsteps=200, algo=mfmc.ALGO_FFT, **kw)
        fft_c = _batched_cost(mfmc, mf_, ns, base) * steps / 200
        ms_ = mfmc.Model(nsteps=200, algo=mfmc.ALGO_SPECTRAL, **kw)
        spec_c = _batched_cost(mfmc, ms_, ns, base) * steps / 200
    pts = ns * n * n * steps
    peak_gbs, sm_max, peak_kind = load_peaks()
    per_step = c / steps  # GPU seconds per sample-step
    if algo == "spectral":
        # per sample-step: the column pass reads and writes the half spectrum (1024 x 513 complex
        # FP32), the row pass reads the spectrum and the field and writes both
        spec_b, field_b = 1024 * 513 * 8, 1024 * 1024 * 4
        bytes_ss = 4 * spec_b + 2 * field_b
        roof = {"bound": "hbm", "kernel": "spectral_column_kernel + spectral_row_kernel",
                "algorithmic_bytes_per_sample_step": bytes_ss, "achieved": bytes_ss / per_step / 1e9,
                "peak": peak_gbs, "unit": "GB/s", "frac": bytes_ss / per_step / 1e9 / peak_gbs,
                "peak_kind": peak_kind}
    else:
        # the disc-sum kernels: 8 B per point-step of field traffic
        bytes_ss = 8 * n * n
        roof = {"bound": "hbm", "kernel": algo, "algorithmic_bytes_per_sample_step": bytes_ss,
                "achieved": bytes_ss / per_step / 1e9, "peak": peak_gbs, "unit": "GB/s",
                "frac": bytes_ss / per_step / 1e9 / peak_gbs, "peak_kind": peak_kind}
    line = {"metric": "grid-pt updates/s (large HF)", "value": pts / (c * ns), "unit": METRIC,
            "roofline": roof,
            "prefix_form_alu_model": {"instr_per_point": 4 * R + 9,
                                      "frac_of_alu_peak": (4 * R + 9) * pts / (c * ns) / (152 * 128 * sm_max * 1e6),
                                      "what": "the throughput in units of the register-tiled prefix form's "
                                              "instruction count (4R + 9 per point) against 152 SMs x 128 FP32 lanes"},
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"1024^2, delta=32h (3209-pt disc), {steps} steps, {ns} samples", "algo": algo},
            "gpu_s_per_sample": c, "direct_sum_gpu_s_per_sample": direct_c,
            "fft_gpu_s_per_sample": fft_c, "spectral_gpu_s_per_sample": spec_c,
            "spectral_what": "own FFT kernels: column pass + fused row pass per step (200 steps scaled)",
            "fft_what": "cuFFT R2C/C2R per step + product + fused update (library comparison point, 200 steps scaled)"}
    print(json.dumps(line), flush=True)
    return 0

def run_mixed(args):
    """One MFMC replicate's samples of the delta = 1/32 hierarchy (512^2/R16, 256^2/R8,
    128^2/R4, 64^2/R2, 1000 steps, nuclei IC), solved three ways: one mfmc_solve_batch
    call per model in turn; one mfmc_solve_batch call over all samples (per-model streams);
    one mfmc_solve_batch_mixed call (one launch per time step over every model's tiles).
    Allocations: the MFMC plans measured at B = 100 C_1 and 300 C_1, and a small allocation
    in which no level fills the GPU alone.  Wall time of the synchronous calls, best of 3
    after a warm-up call (autotuning, graph capture)."""
    import numpy as np
    from paper_2310_10750_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2310_10750_gb300 import mfmc
    base = 20231016 + 1000003 * 4
    levels = [(512, 16), (256, 8), (128, 4), (64, 2)]
    common = dict(eps=0.02, eps_lo=0.016, eps_hi=0.024, tau=1e-3, nsteps=1000, ic=mfmc.IC_NUCLEI)
    models = [mfmc.Model(n=n, delta=R / n, **common) for n, R in levels]
    allocations = {"plan B=100 C_1": [1, 3, 91, 47259], "plan B=300 C_1": [4, 11, 273, 141778],
                   "small levels": [2, 8, 32, 128]}

    def timed(fn):
        fn()
        best, out = 1e30, None
        for _ in range(3):
            t = time.perf_counter()
            out = fn()
            best = min(best, time.perf_counter() - t)
        return best, out

    rows = []
    for name, m in allocations.items():
        seeds = [_seeds(base, k, 10 ** 7 * j) for j, k in enumerate(m)]
        flat_models = [models[j] for j, k in enumerate(m) for _ in range(k)]
        flat_seeds = np.concatenate(seeds)

        def per_model():
            return np.concatenate([mfmc.mfmc_solve_batch([models[j]] * k, seeds[j])[0] for j, k in enumerate(m)])

        t_seq, f_seq = timed(per_model)
        t_batch, (f_batch, _) = timed(lambda: mfmc.mfmc_solve_batch(flat_models, flat_seeds))
        t_mixed, (f_mixed, _) = timed(lambda: mfmc.mfmc_solve_batch_mixed(flat_models, flat_seeds))
        pts = sum(k * n * n for k, (n, _) in zip(m, levels)) * 1000
        rows.append({"allocation": name, "m": m, "grid_pt_updates": pts,
                     "per_model_calls_s": t_seq, "one_batch_call_s": t_batch, "mixed_one_launch_per_step_s": t_mixed,
                     "mixed_speedup_vs_batch_call": t_batch / t_mixed,
                     "max_rel_ooi_diff_mixed_vs_batch": float(np.max(np.abs(f_mixed - f_batch) / f_batch)),
                     "max_rel_ooi_diff_batch_vs_per_model": float(np.max(np.abs(f_batch - f_seq) / f_seq))})
    algos = {1: "direct", 2: "prefix", 4: "resident", 6: "prefix-tma", 7: "row-stream"}
    line = {"metric": "hierarchy replicate wall time", "value": rows[2]["mixed_one_launch_per_step_s"], "unit": "s",
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "MFMC replicate of the delta=1/32 hierarchy (512^2/R16, 256^2/R8, 128^2/R4, "
                                   "64^2/R2), 1000 steps, nuclei IC; value = small-levels allocation, mixed call",
                       "per_model_algos": [algos.get(g.info().algo, str(g.info().algo)) for g in models]},
            "allocations": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_paper(args):
    """The paper's own nine models (Section 4, Table 1): truncated Gaussian kernel,
    delta_hf = 0.25, eps^2 = 0.00178, tau = 0.01, T = 1 (100 steps), the four-nuclei initial
    condition whose theta is the shared random input, h in {1/128, 1/88, 1/64} x delta in
    {0.25, 0.1875, 0.125}, on the periodic lattice with beta2 = 0 by default (the paper's beta2 = 0.05
    step is the active-set solver, --beta2 0.05).  50 pilot samples on shared seeds give rho_{1,k} and sigma_k; the cost
    of a model is GPU seconds per sample of a batched solve; the MFMC plan (policy 0) is printed
    for budgets of 10 .. 1000 C_1 together with the number of feasible subsets."""
    import numpy as np
    from paper_2310_10750_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2310_10750_gb300 import mfmc
    base = 20231016 + 1000003 * 5
    levels = [(128, 0.25), (128, 0.1875), (88, 0.1875), (88, 0.25), (128, 0.125), (88, 0.125),
              (64, 0.1875), (64, 0.25), (64, 0.125)]
    common = dict(kernel=mfmc.KERNEL_GAUSSIAN, delta_hf=0.25, eps=math.sqrt(0.00178), tau=0.01, nsteps=100,
                  ic=mfmc.IC_NUCLEI, beta2=args.beta2)
    models = [mfmc.Model(n=n, delta=d, **common) for n, d in levels]
    n_pilot = 50
    t = time.perf_counter()
    pilot = np.stack([mfmc.mfmc_solve_batch([m] * n_pilot, _seeds(base, n_pilot))[0] for m in models])
    t_pilot = time.perf_counter() - t
    cost, iters = [], []
    for m in models:
        ns_cost = 256 if args.beta2 == 0 else 152
        cost.append(_batched_cost(mfmc, m, ns_cost, base + 10 ** 7))
        if args.beta2 > 0:  # Newton and CG iterations per sample and step of the timed solve
            nw, cgi = mfmc.mfmc_model_solver_stats(m)
            iters.append((nw / (ns_cost * m.nsteps), cgi / (ns_cost * m.nsteps)))
    if args.beta2 == 0:
        fft_models = [mfmc.Model(n=n, delta=d, algo=mfmc.ALGO_FFT, **common) for n, d in levels]
        fft_cost = [_batched_cost(mfmc, m, 256, base + 10 ** 7) for m in fft_models]
        # the own-FFT spectral form (register transforms on 64 and 128, mixed-radix on 88)
        spec_cost = [_batched_cost(mfmc, mfmc.Model(n=n, delta=d, algo=mfmc.ALGO_SPECTRAL, **common), 256,
                                   base + 10 ** 7) for n, d in levels]
    else:
        fft_cost = spec_cost = [None] * len(models)
    paper = {}
    gpath = os.path.join(ROOT, "tests", "golden", "table1_pilot_statistics.txt")
    if os.path.exists(gpath):
        for line in open(gpath):
            if line.strip() and not line.startswith("#"):
                f = line.split()
                paper[int(f[0])] = {"rho": float(f[3]), "cost_ratio": float(f[4]), "sigma": float(f[5])}
    plans = []
    for b in (10.0, 100.0, 1000.0):
        p = mfmc.mfmc_plan(pilot, cost, b * cost[0], 0).as_dict()
        plans.append({"budget_over_C1": b, "subset": [i + 1 for i in p["idx"]], "m": p["m"], "V": p["V"],
                      "Bmin_over_C1": p["Bmin"] / cost[0], "below_min_budget": p["below_min_budget"],
                      "n_feasible_subsets": p["n_feasible"]})
    mixed = []
    if args.beta2 == 0:
        # the hierarchy in one launch (mfmc_solve_batch_mixed: the resident spectral queue over
        # every model's samples) beside one mfmc_solve_batch call per model and one call over all
        # samples; the pilot allocation and the plan at B = 1000 C_1; best of 3 after a warm-up
        def timed(fn):
            fn()
            best, out = 1e30, None
            for _ in range(3):
                t = time.perf_counter()
                out = fn()
                best = min(best, time.perf_counter() - t)
            return best, out

        p1000 = mfmc.mfmc_plan(pilot, cost, 1000 * cost[0], 0).as_dict()
        allocs = {"pilot: 50 samples of each model": [(k, n_pilot) for k in range(len(models))],
                  "MFMC plan at B = 1000 C_1": [(i, int(k)) for i, k in zip(p1000["idx"], p1000["m"]) if k > 0]}
        for name, al in allocs.items():
            seeds = [_seeds(base + 10 ** 8, k, 10 ** 6 * j) for j, (_, k) in enumerate(al)]
            flat_models = [models[i] for i, k in al for _ in range(k)]
            flat_seeds = np.concatenate(seeds)

            def per_model():
                return np.concatenate([mfmc.mfmc_solve_batch([models[i]] * k, seeds[j])[0]
                                       for j, (i, k) in enumerate(al)])

            t_seq, f_seq = timed(per_model)
            t_batch, (f_batch, _) = timed(lambda: mfmc.mfmc_solve_batch(flat_models, flat_seeds))
            t_mixed, (f_mixed, _) = timed(lambda: mfmc.mfmc_solve_batch_mixed(flat_models, flat_seeds))
            mixed.append({"allocation": name, "models": [i + 1 for i, _ in al], "m": [k for _, k in al],
                          "per_model_calls_s": t_seq, "one_batch_call_s": t_batch, "mixed_one_launch_s": t_mixed,
                          "mixed_speedup_vs_per_model_calls": t_seq / t_mixed,
                          "mixed_speedup_vs_batch_call": t_batch / t_mixed,
                          "max_rel_ooi_diff_mixed_vs_per_model": float(np.max(np.abs(f_mixed - f_seq) / f_seq))})
    p0 = mfmc.mfmc_plan(pilot, cost, 100 * cost[0], 0).as_dict()
    table = []
    for k, ((n, d), m) in enumerate(zip(levels, models)):
        algo_names = {1: "direct (generic)", 5: "plain", 8: "fft", 9: "active-set", 10: "weighted-tma",
                      11: "spectral"}
        row = {"model": k + 1, "h": f"1/{n}", "delta": d, "delta_over_h": d * n, "disc_points": m.info().disc_points,
               "algo": algo_names.get(m.info().algo, str(m.info().algo)),
               "rho_1k": p0["rho_all"][k], "cost_ratio": cost[k] / cost[0], "sigma": p0["sigma_all"][k],
               "gpu_s_per_sample": cost[k], "fft_gpu_s_per_sample": fft_cost[k],
               "spectral_gpu_s_per_sample": spec_cost[k]}
        if iters:
            row["newton_per_step"], row["cg_per_step"] = iters[k]
        if k + 1 in paper:
            row["paper"] = paper[k + 1]
        table.append(row)
    line = {"metric": "HF samples/s (paper's nine models)", "value": 1.0 / cost[0], "unit": "samples/s",
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "Section 4 models: Gaussian kernel delta_hf=0.25, eps^2=0.00178, tau=0.01, "
                                   "100 steps, nuclei IC, h in {1/128,1/88,1/64} x delta in {0.25,0.1875,0.125}, "
                                   f"periodic lattice, beta1 = 1, beta2 = {args.beta2:g}; pilot 50 shared seeds",
                       "algo": "autotuned per model (see table1[].algo)" if args.beta2 == 0 else
                               "active-set Newton-CG step (FP64, one CTA per sample)"},
            "pilot_wall_s": t_pilot, "table1": table, "plans": plans, "mixed": mixed,
            "paper_C1_s": 63.089}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="single", choices=["single", "hierarchy", "serving", "large", "mixed", "paper"],
                    help="single (the headline, default), or one of the other measured configurations")
    ap.add_argument("--validation", type=int, default=16384, help="hierarchy: HF samples of the validation mean")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the serving, per-fidelity and MFMC measurements")
    ap.add_argument("--requests", type=int, default=20000, help="serving: requests in the stream")
    ap.add_argument("--load", type=float, default=0.8, help="serving: arrival rate over the measured capacity")
    ap.add_argument("--beta2", type=float, default=0.0, help="paper: beta2 of the nine models (the paper's 0.05)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--nsteps", type=int, default=0, help="profiling: time steps per solve")
    ap.add_argument("--samples", type=int, default=0, help="profiling: samples per GPU")
    ap.add_argument("--algo", default="auto", choices=["auto", "prefix", "direct", "kahan", "tma", "rows", "fft", "spectral"])
    ap.add_argument("--band-height", type=int, default=-1,
                    help="profiling: pin the row-streaming work split (rows per range, 0 = even split)")
    ap.add_argument("--columns", type=int, default=4, help="profiling: row-streaming columns per thread")
    ap.add_argument("--tile-variant", type=int, default=-1, help="profiling: pin the TMA tile shape")
    ap.add_argument("--bc", default="periodic", choices=["periodic", "collar"],
                    help="boundary of the single-fidelity workload (collar: volume constraint)")
    ap.add_argument("--bc-value", type=float, default=-1.0, help="collar value for --bc collar")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "hierarchy":
        return run_hierarchy(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "large":
        return run_large(args)
    if args.workload == "mixed":
        return run_mixed(args)
    if args.workload == "paper":
        return run_paper(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
