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


def config(algo=None):
    c = {"workload": WORKLOAD if (NSTEPS, NSAMPLES) == (1000, 512) else "profiling case: " + WORKLOAD,
         "n": N_LATTICE, "R": R_CELLS, "disc_points": 197, "nsteps": NSTEPS, "samples_per_gpu": NSAMPLES, "tau": TAU, "eps": "0.02*U[0.8,1.2]", "ic": "smoothed Gaussian sigma=0.05",
         "l2": "inputs larger than L2 (2 x 128 MiB field buffers per solve, L2 129 MB)"}
    if algo is not None:
        c["algo"] = algo
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
    """The FP64 oracle on the host cores on a bounded sample: sample 0 of the workload
    for as many steps as fit in about `seconds`."""
    import numpy as np
    import oracle
    o = oracle.OracleModel(n=N_LATTICE, delta=R_CELLS / N_LATTICE, eps=EPS, eps_lo=EPS_LO, eps_hi=EPS_HI,
                           tau=TAU, nsteps=NSTEPS, ic=1, ic_amp=SIGMA)
    seed = SEED_BASE
    eps = o.sample_eps(seed)
    u0 = o.initial_field(seed)
    t = time.perf_counter()
    o.solve(u0, eps, nsteps=10)
    dt10 = time.perf_counter() - t
    steps = int(max(10, min(NSTEPS, 10 * seconds / max(dt10, 1e-6))))
    t = time.perf_counter()
    o.solve(u0, eps, nsteps=steps)
    dt = time.perf_counter() - t
    pts = N_LATTICE * N_LATTICE * steps
    return {"value": pts / dt, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"1 sample of 256x256, {steps} of 1000 steps, FP64 direct disc sum ({dt:.1f} s)"}


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
    global NSTEPS, NSAMPLES
    NSTEPS = args.nsteps or NSTEPS
    NSAMPLES = args.samples or NSAMPLES
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
    from paper_2310_10750_gb300 import mfmc
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    algo_req = {"auto": mfmc.ALGO_AUTO, "prefix": mfmc.ALGO_PREFIX, "direct": mfmc.ALGO_DIRECT,
                "kahan": mfmc.ALGO_PREFIX_KAHAN, "tma": mfmc.ALGO_PREFIX_TMA, "rows": mfmc.ALGO_ROWS}[args.algo]
    model = mfmc.Model(n=N_LATTICE, delta=R_CELLS / N_LATTICE, eps=EPS, eps_lo=EPS_LO, eps_hi=EPS_HI, tau=TAU,
                       nsteps=NSTEPS, ic=mfmc.IC_SMOOTHED_GAUSS, ic_amp=SIGMA, algo=algo_req)
    if args.tile_variant >= 0:
        model.set_tile_variant(args.tile_variant)
    if args.band_height > 0:
        model.set_band_height(args.band_height, args.columns)
    ns = NSAMPLES
    seeds = np.arange(ns, dtype=np.uint64) + SEED_BASE + rank * ns
    u0 = torch.empty((ns, N_LATTICE, N_LATTICE), dtype=torch.float32, device="cuda")
    ooi = torch.empty(ns, dtype=torch.float64, device="cuda")
    eps = torch.tensor(mfmc.mfmc_sample_eps(model, seeds), dtype=torch.float64, device="cuda")
    mfmc.mfmc_init_fields(model, seeds, u0, stream=stream)
    for _ in range(args.warmup):
        mfmc.mfmc_solve_fields(model, u0, ns, eps=eps, ooi=ooi, stream=stream)
    torch.cuda.synchronize()
    algo_names = {1: "direct", 2: "prefix", 3: "prefix-kahan", 4: "resident", 5: "plain", 6: "prefix-tma",
                  7: "row-stream"}
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
    ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
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
        e2e_s = (time.perf_counter() - t) / args.steps
        if ws > 1:
            tt = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_s = float(tt.item())

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
    launches_per_solve = NSTEPS + 2
    kernel_ms = ms_step / NSTEPS  # average step-kernel launch (upper bound: includes launch gaps)
    bytes_launch = 8.0 * ns * N_LATTICE * N_LATTICE
    achieved = bytes_launch / (kernel_ms * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            tr = json.load(open(tpath))
            key = f"{N_LATTICE}_{R_CELLS}_{algo}"
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
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--nsteps", type=int, default=0, help="profiling: time steps per solve")
    ap.add_argument("--samples", type=int, default=0, help="profiling: samples per GPU")
    ap.add_argument("--algo", default="auto", choices=["auto", "prefix", "direct", "kahan", "tma", "rows"])
    ap.add_argument("--band-height", type=int, default=0, help="profiling: pin the row-streaming band height")
    ap.add_argument("--columns", type=int, default=2, help="profiling: row-streaming columns per thread")
    ap.add_argument("--tile-variant", type=int, default=-1, help="profiling: pin the TMA tile shape")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
