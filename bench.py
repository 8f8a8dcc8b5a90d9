"""Benchmark: meshless D3Q19 TRT LBM steps on GB300, node-steps/s, and time to a
steady permeability within 1e-4 of the FP64 oracle.

Headline (one step = one MLBM time step of the whole cell, stream + bounce-back
+ TRT collision fused in one kernel): the periodic simple-cubic sphere cell of
radius 0.40 with an h-refined advancing-front fill h(d) = 0.008 + 0.032
min(1, d / 0.2) (about 150k nodes, 31k on the wall), N_L = 30 nearest
neighbours, PHS r^3 + quadratic monomials, TRT Lambda = 3/16, tau+ = 0.8,
nu = 1, g = (1, 0, 0), dx = h_min / 2 = 0.004, FP32 shifted populations.
Inputs are synthetic (seeded node cloud); the weights (324 MB) exceed the
129 MB L2, so every step streams them from HBM.  `value` times exactly K steps;
the same K-step replay then repeats back to back for --sustain-s seconds inside
the same nvidia-smi clock window (`sustained`, `clocks`).

The default line also carries
  tts        time to 1e-4 of the FP64 oracle's steady k/d^2 (stored in
             tests/golden/steady_references.json): the config-1 MNS cell (FP64,
             FP32, compensated FP32 from rest; compensated FP32 and FP64 from the
             trained network) and the config-2 MLBM cell (FP64, FP32, refined FP32);
  workloads  the config-4 ACM step (3M nodes) and the config-3 64-cell batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload W] [--precision fp32|fp32c|fp64] [--variant V]
                  [--no-tts] [--no-workloads] [--sustain-s S]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same
workload (the paper's own code is a single-threaded CPU program that is not
available here).  Under torchrun (N > 1) every rank runs an independent replica
of the cell on its own GPU (weak scaling, no collective on the data path).

Other workloads (--workload), same line format:
  acm-config4    ACM steps on a ~3M-node cell (r = 0.45, PHS r^5 + m = 3, N_L = 40)
  batch-config3  64 cells stepped in one persistent launch
  mlp-train      warm-start network training steps (fused tensor-core kernels)
  tts-config1    the time-to-steady block alone
  tts-config4-family  its config-4-family arms alone (FP64, compensated and plain FP32
                 to residual 1e-7 on a 52,941-node cell, against the oracle)
  warmstart-config5  the learned warm start at the configured node counts: the
                 network trained on steady fields of --cells cells (h = 1/40,
                 41k-58k nodes) and evaluated on five held-out radii against the
                 oracle's steady k/d^2
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-steps/s; time-to-steady-permeability (1e-4 rel) vs plain FP64 on same GPU"
UNIT = "node-steps/s"
R, H_MIN, H_MAX, RAMP, SEED = 0.40, 0.008, 0.04, 0.2, 2
N_L, Q, DX, TAU_P, MAGIC = 30, 19, 0.004, 0.8, 3.0 / 16.0
KERNELS = {0: "k_lbm_step<float,19> (256)", 1: "k_lbm_step_pairs<float,19,5>", 2: "k_lbm_step<float,19> (128)",
           3: "k_lbm_step_pairs<float,19,3>", 4: "k_lbm_step_pairs<float,19,6>", 5: "k_lbm_step_pairs<float,19,2>",
           6: "k_lbm_step_records<float,19,4> (256)", 7: "k_lbm_step_records<float,19,5> (256)",
           8: "k_lbm_step_records<float,19,4> (128)", 9: "k_lbm_step_records<float,19,4> (64)",
           10: "k_lbm_step_records<float,19,4,PDL> (256)"}


def workload():
    import synth
    return synth.refined_cell(r=R, h_min=H_MIN, h_max=H_MAX, ramp=RAMP, seed=SEED)


def bytes_per_node_step(q=Q, n_l=N_L, elt=4):
    """Algorithmic bytes of one fused LBM step per node: the q-1 interpolation
    weight rows and the stencil indices streamed once, every population read
    once and written once (elt: 4 for FP32, 8 for FP64)."""
    return elt * (q - 1) * n_l + 4 * n_l + 2 * elt * q


def prec_code(rbf, name):
    return {"fp32": rbf.RBF_FP32, "fp32c": rbf.RBF_FP32C, "fp64": rbf.RBF_FP64, "fp32r": rbf.RBF_FP32R}[name]


def config_dict(n, nb, prec="fp32"):
    return {
        "workload": (f"MLBM D3Q19 TRT {prec.upper()} step, periodic SC sphere cell r={R}, h-refined fill "
                     f"h(d)={H_MIN}+{H_MAX - H_MIN:.3f}*min(1,d/{RAMP}), N={n} nodes ({nb} wall), "
                     f"N_L={N_L}, PHS r^3 + m=2, dx={DX}"),
        "nodes": n, "wall_nodes": nb, "n_l": N_L, "q": Q, "precision": f"{prec} populations+weights, fp64 weight solve",
        "l2": "inputs larger than L2 (324 MB FP32 / 648 MB FP64 weights streamed per step)",
        "seed": SEED,
    }


class Clocks:
    """nvidia-smi clock and throttle samples during a region.  A background thread
    runs one-shot queries back to back (each process exits, so no sample is lost to
    output buffering; ~10 samples per second); __enter__ returns after the first
    sample, so the region that follows is covered."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.ok = False
        self._stop = None
        self._thread = None

    def _query(self):
        r = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
        return [[x.strip() for x in line.split(",")] for line in r.stdout.splitlines() if line.count(",") >= 8]

    def _run(self):
        while not self._stop.is_set():
            try:
                self.rows += self._query()
            except Exception:
                return

    def __enter__(self):
        import threading
        try:
            self.rows += self._query()
            self.ok = True
        except Exception:
            self.ok = False
            return self
        self._stop = threading.Event()
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *a):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=15)

    def summary(self):
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_traffic(kernel):
    """DRAM bytes per launch of the timed kernel from the committed ncu summary,
    valid only for that kernel and while its source is unchanged."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "lbm_step_traffic.json")))
        src = open(os.path.join(ROOT, "paper_2404_14195_gb300", "csrc", "lbm.cu"), "rb").read()
        if rec.get("lbm_cu_sha256") == hashlib.sha256(src).hexdigest() and rec.get("nodes_full"):
            return rec["kernels"][kernel]["dram_bytes_per_launch_full"]
    except Exception:
        pass
    return None


def oracle_baseline(case, budget_s=12.0, max_steps=200):
    """The CPU oracle (FP64, all host cores via OpenMP) on the same cell: stencils
    and weights untimed, then a bounded number of timed steps."""
    import oracle
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    idx = oracle.knn(case["xyz"], case["xyz"], N_L, grid=True)
    wk = oracle.lbm_weights(case["xyz"], idx, Q, DX)
    u = oracle.lbm_units(1.0, TAU_P, DX, (1.0, 0.0, 0.0))
    tm = oracle.tau_minus(TAU_P, MAGIC)
    f = oracle.lbm_equilibrium(Q, np.ones(case.n), np.zeros((case.n, 3)))
    t0 = time.perf_counter()
    f = oracle.lbm_run(f, Q, case, idx, wk, TAU_P, tm, u["g_lb"], 1)
    t1 = time.perf_counter() - t0
    steps = int(max(1, min(max_steps, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    oracle.lbm_run(f, Q, case, idx, wk, TAU_P, tm, u["g_lb"], steps)
    dt = time.perf_counter() - t0
    return {"value": case.n * steps / dt, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", cores)),
            "kind": "oracle",
            "sample": f"{steps} FP64 oracle MLBM steps of the full {case.n}-node cell (stencils and weights untimed)",
            "seconds": dt, "steps": steps}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    case = workload()
    base = oracle_baseline(case, budget_s=60.0, max_steps=max(args.steps, 3))
    line = {"metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": base["steps"],
            "warmup": 0, "ms_per_step": 1e3 * base["seconds"] / base["steps"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config_dict(case.n, int((case["type"] == 1).sum())),
            "cpu_baseline": {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": "FP64 CPU oracle of the paper's method (the paper's own CPU code is not available)"}
    print(json.dumps(line), flush=True)
    return 0


SUB_STEPS = 2000  # timed steps of each extra workload block of the default line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--variant", type=int, default=-1,
                    help="LBM step schedule (rbf_set_kernel_variant code); -1 = autotune on the case")
    ap.add_argument("--workload", default="lbm-config2",
                    choices=["lbm-config2", "acm-config4", "batch-config3", "mlp-train", "tts-config1",
                             "tts-config4-family", "warmstart-config5"],
                    help="lbm-config2 (default, the headline); acm-config4: ~3M-node ACM cell, r^5, m=3, N_L=40, "
                         "FP32; batch-config3: 64-cell porosity sweep in one persistent launch; mlp-train: "
                         "warm-start network training steps on the tensor cores")
    ap.add_argument("--mlp-batch", type=int, default=16384,
                    help="mlp-train: samples per training step (a multiple of 128)")
    ap.add_argument("--cfg4-ramp", type=float, default=0.32, help="acm-config4 refinement ramp (0.32: ~3M nodes)")
    ap.add_argument("--cells", type=int, default=64, help="batch-config3: number of cells")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32c", "fp64", "fp32r"],
                    help="storage and arithmetic of the steps (fp32c: compensated FP32 state, ACM workloads only; "
                         "fp32r: refined FP32 populations, the MLBM headline only)")
    ap.add_argument("--no-tts", action="store_true", help="default line without the time-to-steady block")
    ap.add_argument("--no-workloads", action="store_true",
                    help="default line without the config-4 and config-3 blocks")
    ap.add_argument("--sustain-s", type=float, default=1.5,
                    help="seconds of back-to-back repeats of the timed K-step replay inside the clock window")
    args = ap.parse_args()
    if args.precision == "fp32c" and args.workload == "lbm-config2":
        ap.error("--precision fp32c applies to the ACM workloads")
    if args.precision == "fp32r" and args.workload != "lbm-config2":
        ap.error("--precision fp32r applies to the MLBM headline")
    if args.workload != "lbm-config2":
        return run_workload(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        args.warmup = 3

    ws, rank, local = dist_env()
    # config-3 cells come from a spawn pool, before any GPU use
    cells3 = None if (args.no_workloads or ws > 1) else config3_cells(args.cells)

    import torch
    import paper_2404_14195_gb300 as rbf

    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    rbf._build.build()
    case = workload()
    n, nb = case.n, int((case["type"] == 1).sum())

    s = rbf.Solver(local)
    s.set_case(case)
    s.build_stencils(N_L)
    s.compute_weights(k=3, m=2, solver=rbf.RBF_SOLVER_LBM, q=Q, dx=DX)
    s.init(precision=prec_code(rbf, args.precision), nu=1.0, g=(1.0, 0.0, 0.0), tau_plus=TAU_P, magic=MAGIC)
    tune = None
    if args.variant >= 0:
        s.set_kernel_variant(args.variant)
        chosen = args.variant
    else:
        tune, chosen = s.autotune(40)
    s.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    l0 = s.launch_count()
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(args.steps)
        total_ms, per_launch_ms, nlaunch = s.last_step_timing()  # waits for the events
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier()
        launches = s.launch_count() - l0
        # the same K-step replay back to back for --sustain-s seconds in the same
        # nvidia-smi window, so that the clock record covers the load around the
        # (millisecond-long) timed region
        reps = max(1, int(np.ceil(args.sustain_s * 1e3 / max(total_ms, 1e-3))))
        sus_ms = []
        for _ in range(reps):
            s.step(args.steps)
            sus_ms.append(s.last_step_timing()[0])
        torch.cuda.synchronize()
    tmax_ms = _max_over_ranks(total_ms, dist)
    value = whole_job_rate(n * args.steps, ws, tmax_ms / 1e3)

    # per-launch kernel time with event pairs (eager launches, after the timed region)
    prof_ms = float(s.profile_steps(200)[0])
    k, _ = s.permeability(32)

    # end to end through the public API with pinned host buffers: every step uploads
    # its input populations and reads back the step's fields
    f_host = torch.empty((Q, n), dtype=torch.float64, pin_memory=True).numpy()
    f_host[:] = s.lbm_get_populations()
    out_host = torch.empty((n, 4), dtype=torch.float64, pin_memory=True).numpy()
    for _ in range(3):
        s.lbm_set_populations(f_host); s.step(1); s.get_fields(out_host)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        s.lbm_set_populations(f_host)
        s.step(1)
        s.get_fields(out_host)  # the device-to-host copy writes the pinned buffer
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = whole_job_rate(n * args.e2e_steps, ws, _max_over_ranks(e2e_s, dist))

    if rank != 0:
        dist.destroy_process_group()
        return 0
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    elt = 8 if args.precision == "fp64" else 4
    # refined FP32: the profiled launches are the correction steps, which also read
    # the residual (4 B per population)
    bpl = (bytes_per_node_step(elt=elt) + (4 * Q if args.precision == "fp32r" else 0)) * n
    achieved = bpl / (per_launch_ms / 1e3) / 1e9
    kname = KERNELS[chosen] if elt == 4 else (KERNELS[chosen].replace("float", "double")
                                              .replace(",19,4>", ",19,2>").replace(",19,5>", ",19,3>"))
    cpu = None if (args.no_cpu_baseline or ws > 1) else oracle_baseline(case)
    refs = golden_references()
    tts = None
    if not args.no_tts and ws == 1:
        tts = {"acm_config1": _tts_acm_config1(rbf, local, refs.get("mns_config1_vref2")),
               "mlbm_config2": _tts_mlbm_config2(rbf, local, case, refs.get("mlbm_config2")),
               "acm_config4_family": _tts_acm_config4_family(rbf, local, refs.get("mns_config4_family"))}
    blocks = None
    if not args.no_workloads and ws == 1:
        sub = argparse.Namespace(**vars(args))
        sub.no_cpu_baseline, sub.e2e_steps = True, 10
        # at most SUB_STEPS timed steps per block (5.3 s of config-4 steps, 11.6 s of config-3
        # steps), so the default line stays within a few minutes at the headline's K = 20,000
        sub.steps = min(args.steps, SUB_STEPS)
        blocks = {}
        for name, fn in (("acm_config4", lambda: _acm_config4(sub, rbf, local, None, 1, peaks)),
                         ("batch_config3", lambda: _batch_config3(sub, rbf, local, None, 1, peaks, cells3))):
            r = fn()
            blocks[name] = {k: r.get(k) for k in ("metric", "value", "unit", "steps", "warmup", "ms_per_step",
                                                 "dtype", "config", "roofline", "e2e", "gpu_launches", "clocks")}
        if not args.no_cpu_baseline:  # after every timed region: bounded oracle samples
            blocks["acm_config4"]["cpu_baseline"] = _cpu_sample_config4()
            blocks["batch_config3"]["cpu_baseline"] = _cpu_sample_config3(cells3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tmax_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if elt == 8 else "f32",
        "data": "synthetic (seeded node cloud; the paper's datasets are not used)",
        "config": config_dict(n, nb, args.precision) | {"parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": kernel_traffic(kname),
                     "kernel": kname,
                     "schedule": chosen, "autotune_ms_per_step": tune,
                     "bytes_per_launch": bpl,
                     "per_launch_ms_timed_region": per_launch_ms, "per_launch_ms_event_pairs": prof_ms,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)" if peaks else "fallback"},
        "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(Q * n * 8),
                "d2h_bytes_per_step": int(4 * n * 8), "steps": args.e2e_steps},
        "gpu_launches": int(launches),
        "clocks": clk.summary() | {"window": f"timed region plus {reps} back-to-back repeats of it "
                                             f"({sum(sus_ms) / 1e3:.2f} s)"},
        "sustained": {"repeats": reps, "ms_per_step": sum(sus_ms) / (reps * args.steps),
                      "value": n * reps * args.steps / (sum(sus_ms) / 1e3), "unit": UNIT},
        "k_over_d2_after_run": k,
        "wall_s_timed": wall,
        "tts": tts,
        "workloads": blocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# further workloads (same JSON line; `metric` names what is measured)
# ---------------------------------------------------------------------------
CFG4 = dict(r=0.45, h_min=0.003, h_max=0.02, seed=4, n_l=40, k=5, m=3)


def acm_kernel_bytes(n_l, prec="fp32"):
    """Algorithmic bytes per node of each ACM sweep (wall pressure: per wall
    node): stencil indices (4 B) and weights streamed once, the node's own field
    values read / written once (neighbour gathers hit L1/L2).  FP32: predictor
    20 N_L + 24, pressure 16 N_L + 20, correction 16 N_L + 28, wall 8 N_L + 8;
    FP64 doubles every floating-point byte; compensated FP32 adds the low words
    (predictor +24, pressure +8, correction +24)."""
    if prec == "fp64":
        return {"predict": 36 * n_l + 48, "pressure": 28 * n_l + 40, "wall_pressure": 12 * n_l + 12,
                "correct": 28 * n_l + 56}
    extra = prec == "fp32c"
    return {"predict": 20 * n_l + 24 + 24 * extra, "pressure": 16 * n_l + 20 + 8 * extra,
            "wall_pressure": 8 * n_l + 8, "correct": 16 * n_l + 28 + 24 * extra}


def acm_bytes(n_l, prec="fp32", n_p=3):
    """Algorithmic bytes per ACM node-step (one predictor, n_p x pressure and
    correction; wall pressure counted separately): FP32 116 N_L + 168, FP64
    204 N_L + 336, compensated FP32 116 N_L + 288."""
    kb = acm_kernel_bytes(n_l, prec)
    return kb["predict"] + n_p * (kb["pressure"] + kb["correct"])


def _make_cell3(args):
    r, hmin, seed, n_l = args
    import synth
    c = synth.refined_cell(r=r, h_min=hmin, h_max=0.04, ramp=0.2, seed=seed)
    return c, n_l


def config3_jobs(ncells, seed=3, rank=0):
    """(r, h_min, node seed, N_L) of config 3's cells: radii U[0.15, 0.62], h_min
    U[0.006, 0.012], N_L U{20..45}.  Rank r takes the cells r*ncells ..
    (r+1)*ncells - 1 of one seeded sequence, so the ranks of a multi-GPU run hold
    disjoint cells (rank 0: the same cells as a one-GPU run)."""
    rng = np.random.default_rng(seed)
    draws = [(float(rng.uniform(0.15, 0.62)), float(rng.uniform(0.006, 0.012)), int(rng.integers(20, 46)))
             for _ in range((rank + 1) * ncells)]
    return [(r_, h_, 1000 + i, nl_) for i, (r_, h_, nl_) in enumerate(draws) if i >= rank * ncells]


def config3_cells(ncells, seed=3, rank=0):
    """Config 3's cells (h_max 0.04, the config-2 ramp), generated in a spawn pool
    before any GPU use."""
    import multiprocessing as mp
    jobs = config3_jobs(ncells, seed, rank)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        return pool.map(_make_cell3, jobs)


def _timed(fn, local, dist):
    import torch
    with Clocks(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dist is not None:
            dist.barrier()
    return wall, clk.summary()


def run_workload(args):
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        return _reference_workload(args)
    cells3 = config3_cells(args.cells, rank=rank) if args.workload == "batch-config3" else None
    import torch
    import paper_2404_14195_gb300 as rbf
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    rbf._build.build()
    peaks = measured_peaks()
    if args.workload == "acm-config4":
        line = _acm_config4(args, rbf, local, dist, ws, peaks)
    elif args.workload == "batch-config3":
        line = _batch_config3(args, rbf, local, dist, ws, peaks, cells3)
    elif args.workload == "tts-config1":
        line = _tts_config1(args, rbf, local)
    elif args.workload == "tts-config4-family":
        line = _tts_config4_family(args, rbf, local)
    elif args.workload == "warmstart-config5":
        line = _warmstart_config5(args, rbf, local)
    else:
        line = _mlp_train(args, rbf, local, dist, ws, peaks)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _max_over_ranks(x, dist):
    """The largest x over all ranks (the whole job's time is its slowest rank's);
    the reduction runs on the GPU under NCCL, on the host under gloo."""
    import torch
    dev = "cuda" if dist is None or dist.get_backend() == "nccl" else "cpu"
    if dist is None and not torch.cuda.is_available():
        dev = "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x, dist):
    """The sum of x over all ranks (units of disjoint per-rank work)."""
    import torch
    if dist is None:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_per_rank, world_size, seconds_max):
    """Weak-scaling throughput: every rank processes units_per_rank units (its own
    replica), the job takes the slowest rank's time."""
    return world_size * units_per_rank / seconds_max


def _acm_config4(args, rbf, local, dist, ws, peaks):
    import synth
    import torch
    c = CFG4
    case = synth.refined_cell(r=c["r"], h_min=c["h_min"], h_max=c["h_max"], ramp=args.cfg4_ramp, seed=c["seed"])
    n, nb = case.n, int((case["type"] == 1).sum())
    s = rbf.Solver(local)
    s.set_case(case)
    s.build_stencils(c["n_l"])
    t0 = time.perf_counter()
    rep = s.compute_weights(k=c["k"], m=c["m"], solver=rbf.RBF_SOLVER_ACM)
    t_w = time.perf_counter() - t0
    s.init(precision=prec_code(rbf, args.precision), v_ref=0.01)
    tune, chosen = s.autotune(10)
    s.step(args.warmup)
    l0 = s.launch_count()
    holder = {}

    def work():
        s.step(args.steps)
        holder["ms"] = s.last_step_timing()[0]

    wall, clk = _timed(work, local, dist)
    launches = s.launch_count() - l0
    tmax = _max_over_ranks(holder["ms"], dist)
    prof = s.profile_steps(10)  # predictor, pressure, wall pressure, correction
    L = c["n_l"]
    kb = {nm: b * (nb if nm == "wall_pressure" else n) for nm, b in acm_kernel_bytes(L, args.precision).items()}
    names = list(kb)
    share = {nm: prof[i] * (1 if i == 0 else 3) for i, nm in enumerate(names)}
    dom = max(share, key=share.get)
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    per_kernel = {nm: {"ms": float(prof[i]), "GB/s": kb[nm] / (prof[i] / 1e3) / 1e9} for i, nm in enumerate(names)}
    ach = per_kernel[dom]["GB/s"]
    step_gbs = acm_bytes(L, args.precision) * n / (tmax / args.steps / 1e3) / 1e9
    tname = "double" if args.precision == "fp64" else "float"
    cp = ", true" if args.precision == "fp32c" else ", false"
    # e2e: host fields in, one step, fields out, every step
    f_host = torch.empty((n, 4), dtype=torch.float64, pin_memory=True).numpy()
    f_host[:] = s.get_fields()
    out = torch.empty((n, 4), dtype=torch.float64, pin_memory=True).numpy()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        s.set_fields(f_host)
        s.step(1)
        s.get_fields(out)  # the device-to-host copy writes the pinned buffer
    e2e = _max_over_ranks(time.perf_counter() - t0, dist)
    k_perm, _ = s.permeability(32)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = _oracle_acm_baseline(case, c)
    return {
        "metric": "node-steps/s (ACM steps, config 4)", "value": whole_job_rate(n * args.steps, ws, tmax / 1e3), "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp32c": "f32 (compensated state)", "fp64": "f64"}[args.precision],
        "data": "synthetic (seeded node cloud)",
        "config": {"workload": f"ACM {args.precision.upper()} steps, periodic SC cell r={c['r']}, h(d)={c['h_min']}..{c['h_max']} "
                               f"ramp {args.cfg4_ramp}, N={n} ({nb} wall), N_L={L}, PHS r^{c['k']} + m={c['m']}",
                   "nodes": n, "wall_nodes": nb, "l2": "inputs larger than L2", "parallelism": f"replicas x{ws}",
                   "weights_solve_s": t_w, "h_min": rep["h_min"], "acm_schedule": chosen, "autotune": tune},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": None, "kernel": f"k_acm_{dom}<{tname}{cp}>", "per_kernel": per_kernel,
                     "step_GBs": step_gbs, "step_frac": step_gbs / peak},
        "cpu_baseline": cpu, "e2e": {"value": ws * n * args.e2e_steps / e2e, "unit": UNIT,
                                     "h2d_bytes_per_step": 32 * n, "d2h_bytes_per_step": 32 * n},
        "gpu_launches": int(launches), "clocks": clk, "k_over_d2_after_run": k_perm, "wall_s_timed": wall,
    }


def _oracle_acm_baseline(case, c, budget_s=15.0, max_steps=100):
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    idx = oracle.knn(case["xyz"], case["xyz"], c["n_l"], grid=True)
    w4 = oracle.acm_weights(case["xyz"], idx, c["k"], c["m"])
    wl, idxb = oracle.neumann_stencils(case, c["n_l"])
    wgb = oracle.neumann_weights(case, idxb, c["k"], c["m"])
    t_setup = time.perf_counter() - t0
    dmin = np.linalg.norm(oracle.min_image(case["xyz"][idx[:, 1]] - case["xyz"]), axis=1).min()
    dt = oracle.acm_dt(dmin, 1.0)
    f = np.zeros((case.n, 4))
    t0 = time.perf_counter()
    f, _ = oracle.acm_run(case, idx, w4, idxb, wgb, f, 1, dt=dt, v_ref=0.01)
    t1 = time.perf_counter() - t0
    steps = int(max(1, min(max_steps, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    oracle.acm_run(case, idx, w4, idxb, wgb, f, steps, dt=dt, v_ref=0.01)
    dt_run = time.perf_counter() - t0
    return {"value": case.n * steps / dt_run, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} FP64 oracle ACM steps of the full {case.n}-node cell "
                      f"(stencils and weights untimed: {t_setup:.0f} s)"}


def _cpu_sample_config4():
    """Bounded CPU baseline for the config-4 block of the default line: the oracle
    on a cell of the same family at a coarser resolution (the full cell's FP64
    stencil and weight setup alone takes minutes on the host)."""
    import synth
    c = CFG4
    small = synth.refined_cell(r=c["r"], h_min=0.02, h_max=0.03, ramp=0.32, seed=c["seed"])
    b = _oracle_acm_baseline(small, c, budget_s=15.0, max_steps=5000)
    b["sample"] = (f"config-4 family at h 0.02..0.03 (r={c['r']}, N_L={c['n_l']}, PHS r^{c['k']} + m={c['m']}): "
                   + b["sample"].replace("of the full", "of a"))
    return {k: b[k] for k in ("value", "unit", "cores", "kind", "sample")}


def _cpu_sample_config3(cells):
    """Bounded CPU baseline for the config-3 block: the oracle on the smallest of
    the batch's cells, in node-steps/s."""
    case, n_l = min(cells, key=lambda cn: cn[0].n)
    b = _oracle_acm_baseline(case, dict(n_l=n_l, k=3, m=2), budget_s=15.0, max_steps=5000)
    b["sample"] = f"the smallest of the {len(cells)} cells (N_L={n_l}): " + b["sample"].replace("of the full", "of its")
    return {k: b[k] for k in ("value", "unit", "cores", "kind", "sample")}


def _batch_config3(args, rbf, local, dist, ws, peaks, cells):
    b = rbf.Batch(local)
    n_tot = 0
    for case, n_l in cells:
        b.add_cell(case, n_l)
        n_tot += case.n
    t0 = time.perf_counter()
    rep = b.build(3, 2)
    t_build = time.perf_counter() - t0
    b.init(precision=prec_code(rbf, args.precision), v_ref=0.01)
    tune, chosen = b.autotune(20)  # threads per block of the persistent driver
    b.solve(args.warmup, 1e-300, check_every=args.warmup)
    holder = {}

    def work():
        holder["res"] = b.solve(args.steps, 1e-300, check_every=max(1, args.steps // 4))

    wall, clk = _timed(work, local, dist)
    tmax = _max_over_ranks(wall, dist)
    n_job = _sum_over_ranks(n_tot, dist)  # the ranks hold disjoint cells
    nl = [n_l for _, n_l in cells]
    byts = sum(acm_bytes(n_l, args.precision) * case.n for case, n_l in cells)
    gbs = byts * args.steps / tmax / 1e9
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    return {
        "metric": "node-steps/s (batched ACM steps, config 3)", "value": n_job * args.steps / tmax,
        "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp32c": "f32 (compensated state)", "fp64": "f64"}[args.precision],
        "data": "synthetic (seeded node clouds)",
        "config": {"workload": f"{len(cells)} periodic SC cells, r~U[0.15,0.62], h_min~U[0.006,0.012], h_max 0.04, "
                               f"N_L~U{{20..45}}, one persistent launch (wall-clock timed, includes launch and "
                               f"the per-cell FP64 residual checks)",
                   "cells": len(cells), "nodes_total": n_tot, "nodes_min": min(c.n for c, _ in cells),
                   "nodes_max": max(c.n for c, _ in cells), "n_l_range": [min(nl), max(nl)],
                   "build_s (stencils, one weight launch for all cells, packing)": t_build,
                   "weight_systems": rep["n_systems"],
                   "parallelism": f"disjoint cells per rank x{ws}" + (f" ({n_job:.0f} nodes in all)" if ws > 1 else ""),
                   "persistent_block": chosen, "autotune_ms_per_step": tune},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                     "traffic": None,
                     "kernel": f"k_acm_persistent<{'double' if args.precision == 'fp64' else 'float'}> "
                               f"(whole step, all cells)"},
        "cpu_baseline": None, "e2e": None, "gpu_launches": 1, "clocks": clk, "wall_s_timed": wall,
    }


def _mlp_flops_per_sample():
    # forward 2 * sum(fan_in * fan_out) over the five layers; backward twice that
    return 3 * 2 * (64 * 128 + 3 * 128 * 128 + 128 * 16)


def _mlp_train(args, rbf, local, dist, ws, peaks):
    B = args.mlp_batch
    rng = np.random.default_rng(0)
    n = 1 << 20
    xyz = rng.random((n, 3))
    r = rng.uniform(0.15, 0.62, n).astype(np.float32)
    sdf = rng.uniform(0.0, 0.4, n).astype(np.float32)
    tgt = (0.1 * rng.standard_normal((n, 4))).astype(np.float32)
    from paper_2404_14195_gb300 import warmstart as wsm
    m = rbf.Mlp(local)
    m.set_params(wsm.init_params(1))
    m.set_data(xyz, r, sdf, tgt)
    m.train(args.warmup, B, 1e-3, 1)
    holder = {}
    l0 = m.launch_count()

    def work():
        holder["loss"] = m.train(args.steps, B, 1e-3, 1)

    wall, clk = _timed(work, local, dist)
    tmax = _max_over_ranks(wall, dist)
    launches = m.launch_count() - l0
    fl = _mlp_flops_per_sample() * B * args.steps / tmax / 1e12
    peak = peaks["bf16_tflops_sustained"] if peaks else 1700.0
    # the per-layer schedule (one GEMM launch per layer and pass) on the same work, for comparison
    m.set_fused(False)
    m.train(args.warmup, B, 1e-3, 1)
    holder2 = {}

    def work2():
        holder2["loss"] = m.train(args.steps, B, 1e-3, 1)

    wall2, _ = _timed(work2, local, dist)
    m.set_fused(True)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        from oracle import mlp as om  # the CPU baseline leg: the oracle network
        th = om.init_params(1)
        X = om.features(xyz[:B], r[:B], sdf[:B])
        t0 = time.perf_counter()
        steps = 0
        while time.perf_counter() - t0 < 10.0:
            om.loss_and_grad(th, X, tgt[:B])
            steps += 1
        cpu = {"value": steps * B / (time.perf_counter() - t0), "unit": "samples/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": f"{steps} FP64 numpy forward+backward passes of {B} samples"}
    return {
        "metric": "samples/s (warm-start MLP training steps)", "value": ws * B * args.steps / tmax,
        "unit": "samples/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (fp32 accumulate, fp32 Adam)", "data": "synthetic random samples",
        "config": {"workload": f"MLP 64-128x4-16 GELU, batch {B}, forward + backward + Adam per step (CUDA graph): "
                               f"fused tcgen05 forward and backward kernels",
                   "batch": B, "parallelism": f"replicas x{ws}",
                   "per_layer_schedule": {"samples_per_s": ws * B * args.steps / wall2,
                                          "ms_per_step": 1e3 * wall2 / args.steps}},
        "roofline": {"bound": "tensor", "achieved": fl, "peak": peak, "unit": "TFLOP/s", "frac": fl / peak,
                     "traffic": None, "kernel": "k_mlp_fwd + k_mlp_bwd (tcgen05), whole training step",
                     "flops_per_sample": _mlp_flops_per_sample(),
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained"},
        "cpu_baseline": cpu, "e2e": None, "gpu_launches": int(launches), "clocks": clk,
        "final_loss": float(holder["loss"][-1]), "wall_s_timed": wall,
    }


def _tts_config1(args, rbf, local):
    """The time-to-steady block of the default line on its own (config-1 MNS arms
    and config-2 MLBM arms), as one JSON line whose value is the compensated FP32
    warm-started MNS run's seconds to 1e-4 of the oracle's steady k/d^2."""
    refs = golden_references()
    acm = _tts_acm_config1(rbf, local, refs.get("mns_config1_vref2"))
    lbm = _tts_mlbm_config2(rbf, local, workload(), refs.get("mlbm_config2"))
    v = acm.get("runs", {}).get("fp32c_warm", {}).get("seconds")
    return {"metric": "time-to-steady-permeability (1e-4 rel) vs plain FP64 on same GPU", "value": v, "unit": "s",
            "n_gpus": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 compensated (+ bf16 network)", "data": "synthetic (seeded cells)",
            "config": {"workload": "time to 1e-4 of the FP64 oracle's steady permeability: config-1 MNS cell "
                                   "(five arms) and config-2 MLBM cell (two arms)"},
            "tts": {"acm_config1": acm, "mlbm_config2": lbm}}


def _tts_config4_family(args, rbf, local):
    """The config-4-family arms of the time-to-steady block on their own, as one
    JSON line whose value is the compensated FP32 run's seconds to residual 1e-7."""
    blk = _tts_acm_config4_family(rbf, local, golden_references().get("mns_config4_family"))
    at = blk.get("runs", {}).get("fp32c", {}).get("at_residual") or {}
    return {"metric": "time to residual 1e-7 (config 4 family), error against the FP64 GPU path and the oracle",
            "value": at.get("seconds"), "unit": "s", "n_gpus": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 compensated", "data": "synthetic (seeded cell)",
            "config": {"workload": blk.get("workload")}, "tts": {"acm_config4_family": blk}}


def golden_references():
    """The FP64 oracle's steady k/d^2 and K on the time-to-steady cells, written by
    tests/golden/make_steady_references.py (oracle only, run once on the CPU)."""
    try:
        return json.load(open(os.path.join(ROOT, "tests", "golden", "steady_references.json")))
    except Exception:
        return {}


def _first_within(hist, k_ref, rel=1e-4):
    for i in range(len(hist)):
        if all(abs(h[1] - k_ref) <= rel * abs(k_ref) for h in hist[i:]):
            return hist[i]
    return None


def _tts_acm_config1(rbf, local, ref, chunk=500, max_steps=24000, m_p=32, v_ref=2.0, train_cells=24):
    """Time to a permeability within 1e-4 of the FP64 oracle's steady k/d^2 on the
    config-1 cell (6,857 nodes, r = 0.35, N_L = 25, v_ref = 2): FP64, plain FP32 and
    compensated FP32 from rest, compensated FP32 and FP64 from the network.  The
    network is trained on steady fields of other config-1-family cells (radii
    U[0.2, 0.5], other seeds) that the batched persistent driver solves.  Each run
    steps in chunks through the persistent driver (tuned schedule) and reads k/d^2
    after each chunk; its time counts the stepping and the warm start, not the
    reads or the network's training; it reaches the target at the first chunk
    after which k stays within 1e-4 until the end (max_steps)."""
    import synth
    from paper_2404_14195_gb300 import warmstart as wsm
    case = synth.jittered_cell()
    if not ref or ref.get("nodes") != case.n:
        return {"unavailable": "no oracle reference for this cell in tests/golden/steady_references.json"}
    k_ref = ref["k_over_d2"]
    rng = np.random.default_rng(11)
    train = [synth.jittered_cell(r=float(r), seed=200 + i) for i, r in enumerate(rng.uniform(0.2, 0.5, train_cells))]
    data, res3, t_data = wsm.steady_training_set(train, tol=5e-8, max_steps=200_000, check_every=500, v_ref=v_ref)
    mlp, hist, t_train = wsm.train(data, wsm.init_params(1), steps=12000, batch=4096, lr=2e-3,
                                   decay=((6000, 6e-4), (6000, 2e-4)))
    clk = Clocks(local)
    clk.__enter__()
    runs, sched = {}, {}
    for name, prec, m in (("fp64_zero", rbf.RBF_FP64, None), ("fp32_zero", rbf.RBF_FP32, None),
                          ("fp32c_zero", rbf.RBF_FP32C, None), ("fp32c_warm", rbf.RBF_FP32C, mlp),
                          ("fp64_warm", rbf.RBF_FP64, mlp)):
        h, code = wsm.permeability_history(case, m, chunk=chunk, max_steps=max_steps, precision=prec, m_p=m_p,
                                           v_ref=v_ref, tune_steps=0 if prec in sched else 500,
                                           schedule=sched.get(prec))
        sched[prec] = code
        hit = _first_within(h, k_ref)
        runs[name] = {"steps": None if hit is None else hit[0], "seconds": None if hit is None else hit[2],
                      "s_per_step": h[-1][2] / h[-1][0], "k_start_rel_err": abs(h[0][1] - k_ref) / k_ref,
                      "k_end_rel_err": abs(h[-1][1] - k_ref) / k_ref, "persistent_schedule": code}
    clk.__exit__(None, None, None)
    base = runs["fp64_zero"]["seconds"]
    for v in runs.values():
        v["speedup_vs_fp64_zero"] = (base / v["seconds"]) if (base and v["seconds"]) else None
    return {"workload": f"config-1 MNS cell ({case.n} nodes, jittered grid h=1/20, r=0.35, N_L=25, PHS r^3 + m=2), "
                        f"v_ref={v_ref}, steps in chunks of {chunk} up to {max_steps}",
            "k_ref": k_ref, "k_ref_source": f"FP64 oracle, {ref['steps']} steps (tests/golden/steady_references.json)",
            "target": "first chunk after which |k - k_ref| <= 1e-4 k_ref for the rest of the run",
            "runs": runs,
            "network": {"train_cells": len(train), "train_samples": int(len(data[0])), "train_data_s": t_data,
                        "train_cells_converged": sum(r["status"] == 0 for r in res3), "train_s": t_train,
                        "final_train_loss": float(hist[-1])},
            "clocks": clk.summary()}


CFG4_FAMILY = dict(r=0.45, h_min=0.02, h_max=0.03, ramp=0.32, seed=4)  # 52,941 nodes


def _tts_acm_config4_family(rbf, local, ref, chunk=2000, max_steps=40000, m_p=32, v_ref=2.0, res_tol=1e-7):
    """Config 4's report (run to residual 1e-7; error against the FP64 GPU path and
    the oracle on a 1e-4 permeability target) on a cell of its family that the
    oracle can take to its steady state: r = 0.45, PHS r^5 + order-3 monomials,
    N_L = 40, h 0.02 at the wall to 0.03 (52,941 nodes; the 3.0M-node cell at h
    0.003..0.02 would need ~1e6 steps), v_ref = 2.  FP64, compensated FP32 and
    plain FP32 from rest through the persistent driver (schedule tuned per
    precision), in chunks; after each chunk the residual of the last step, k/d^2 and
    K.  Per run: the first chunk whose residual is below res_tol (steps, seconds, k
    and K errors there), and the first chunk after which k stays within 1e-4 of the
    oracle's k (time to steady); seconds count the stepping, not the reads."""
    import synth
    case = synth.refined_cell(**CFG4_FAMILY)
    if not ref or ref.get("nodes") != case.n:
        return {"unavailable": "no oracle reference for this cell in tests/golden/steady_references.json"}
    k_ref, K_ref = ref["k_over_d2"], ref["K"]
    clk = Clocks(local)
    clk.__enter__()
    runs = {}
    for name, prec in (("fp64", rbf.RBF_FP64), ("fp32c", rbf.RBF_FP32C), ("fp32", rbf.RBF_FP32)):
        s = rbf.Solver(local)
        s.set_case(case)
        s.build_stencils(CFG4["n_l"])
        s.compute_weights(k=CFG4["k"], m=CFG4["m"], solver=rbf.RBF_SOLVER_ACM)
        s.init(precision=prec, v_ref=v_ref)
        code = s.autotune_persistent(500)[1]
        hist, t_run, steps = [], 0.0, 0
        while steps < max_steps:
            t1 = time.perf_counter()
            r = s.solve(chunk, 1e-300, check_every=chunk, m_p=m_p)
            t_run += time.perf_counter() - t1
            steps += chunk
            k = s.permeability(m_p)[0]
            K = s.drag(m_p)[1]
            hist.append((steps, k, t_run, r["residual"], K))
        s.close()
        hit = _first_within(hist, k_ref)
        at = next((h for h in hist if h[3] <= res_tol), None)
        runs[name] = {
            "persistent_schedule": code, "s_per_step": hist[-1][2] / hist[-1][0],
            "residual_end": hist[-1][3],
            "at_residual": None if at is None else {
                "steps": at[0], "seconds": at[2], "residual": at[3],
                "k_rel_err_vs_oracle": abs(at[1] - k_ref) / k_ref, "K_rel_err_vs_oracle": abs(at[4] - K_ref) / K_ref,
                "k": at[1], "K": at[4]},
            "to_1e-4_of_oracle_k": None if hit is None else {"steps": hit[0], "seconds": hit[2]},
            "k_end_rel_err_vs_oracle": abs(hist[-1][1] - k_ref) / k_ref,
            "K_end_rel_err_vs_oracle": abs(hist[-1][4] - K_ref) / K_ref,
            "k_end": hist[-1][1], "K_end": hist[-1][4]}
    clk.__exit__(None, None, None)
    base = runs["fp64"]
    for v in runs.values():
        a, b = v["at_residual"], base["at_residual"]
        if a and b:
            a["k_rel_err_vs_gpu_fp64"] = abs(a["k"] - b["k"]) / abs(b["k"])
            a["K_rel_err_vs_gpu_fp64"] = abs(a["K"] - b["K"]) / abs(b["K"])
        t, t0 = v["to_1e-4_of_oracle_k"], base["to_1e-4_of_oracle_k"]
        v["speedup_vs_fp64"] = (t0["seconds"] / t["seconds"]) if (t and t0) else None
    return {"workload": f"config-4 family MNS cell ({case.n} nodes, r=0.45, h 0.02..0.03, N_L={CFG4['n_l']}, "
                        f"PHS r^{CFG4['k']} + m={CFG4['m']}), v_ref={v_ref}, chunks of {chunk} steps up to {max_steps}",
            "k_ref": k_ref, "K_ref": K_ref,
            "ref_source": f"FP64 oracle, {ref['steps']} steps (tests/golden/steady_references.json)",
            "residual_criterion": res_tol, "runs": runs, "clocks": clk.summary()}


def _tts_mlbm_config2(rbf, local, case, ref, chunk=5000, max_steps=250000, m_p=32):
    """Time to a permeability within 1e-4 of the FP64 oracle's steady k/d^2 on the
    config-2 MLBM cell: FP64, shifted FP32 and refined FP32 (RBF_FP32R: FP32
    correction steps on an FP64 base, one FP64 refresh every 64 steps)
    populations, each on its autotuned schedule, from f_eq(1, 0); device time of
    the stepping (permeability reads excluded)."""
    if not ref or ref.get("nodes") != case.n:
        return {"unavailable": "no oracle reference for this cell in tests/golden/steady_references.json"}
    k_ref = ref["k_over_d2"]
    s = rbf.Solver(local)
    s.set_case(case)
    s.build_stencils(N_L)
    s.compute_weights(k=3, m=2, solver=rbf.RBF_SOLVER_LBM, q=Q, dx=DX)
    clk = Clocks(local)
    clk.__enter__()
    runs = {}
    for name, prec in (("fp64", rbf.RBF_FP64), ("fp32", rbf.RBF_FP32), ("fp32r", rbf.RBF_FP32R)):
        s.init(precision=prec, nu=1.0, g=(1.0, 0.0, 0.0), tau_plus=TAU_P, magic=MAGIC)
        _, chosen = s.autotune(20)
        h = [(0, s.permeability(m_p)[0], 0.0)]
        dev_s = 0.0
        while h[-1][0] < max_steps:
            s.step(chunk)
            dev_s += s.last_step_timing()[0] / 1e3
            h.append((h[-1][0] + chunk, s.permeability(m_p)[0], dev_s))
        hit = _first_within(h, k_ref)
        F, K = s.drag(m_p)
        runs[name] = {"steps": None if hit is None else hit[0], "seconds": None if hit is None else hit[2],
                      "s_per_step": h[-1][2] / h[-1][0], "k_end_rel_err": abs(h[-1][1] - k_ref) / k_ref,
                      "K_end_rel_err": abs(K - ref["K"]) / ref["K"], "schedule": chosen}
    clk.__exit__(None, None, None)
    s.close()
    base = runs["fp64"]["seconds"]
    for v in runs.values():
        v["speedup_vs_fp64"] = (base / v["seconds"]) if (base and v["seconds"]) else None
    return {"workload": f"config-2 MLBM cell ({case.n} nodes), D3Q19 TRT, dx={DX}, steps in chunks of {chunk} "
                        f"up to {max_steps}",
            "k_ref": k_ref, "k_ref_source": f"FP64 oracle, {ref['steps']} steps (tests/golden/steady_references.json)",
            "target": "first chunk after which |k - k_ref| <= 1e-4 k_ref for the rest of the run",
            "runs": runs, "clocks": clk.summary()}


C5_HELDOUT_RADII = (0.29, 0.33, 0.37, 0.41, 0.45)


def _warmstart_config5(args, rbf, local, chunk=1000, max_steps=100000, m_p=32, v_ref=2.0, n_axis=40):
    """What the trained network gains at the configured node counts.  Training:
    steady compensated FP32 fields (v_ref = 2, residual 5e-8) of --cells jittered
    cells (h = 1/40, radii U[0.25, 0.47], seeds 300+) solved in one batched
    persistent launch, then 20,000 Adam steps of 8,192 samples.  Evaluation: five
    held-out radii (other seeds), each solved from rest in FP64 and in compensated
    FP32 and from the network in compensated FP32, in chunks of 1,000 steps; the
    target is the first chunk after which k/d^2 stays within 1e-4 of the FP64
    oracle's steady value (tests/golden/steady_references.json) up to max_steps."""
    import synth
    from paper_2404_14195_gb300 import warmstart as wsm
    refs = golden_references()
    rng = np.random.default_rng(5)
    train = [synth.jittered_cell(r=float(r), n_axis=n_axis, seed=300 + i)
             for i, r in enumerate(rng.uniform(0.25, 0.47, args.cells))]
    data, res, t_data = wsm.steady_training_set(train, tol=5e-8, max_steps=400_000, check_every=1000, v_ref=v_ref)
    mlp, hist, t_train = wsm.train(data, wsm.init_params(1), steps=20000, batch=8192, lr=2e-3,
                                   decay=((10000, 6e-4), (10000, 2e-4)))
    clk = Clocks(local)
    clk.__enter__()
    rows, tot = [], {"fp64_zero": [0, 0.0], "fp32c_zero": [0, 0.0], "fp32c_warm": [0, 0.0]}
    for i, r in enumerate(C5_HELDOUT_RADII):
        ref = refs.get(f"mns_c5_heldout_{i}")
        case = synth.jittered_cell(r=r, n_axis=n_axis, seed=900 + i)
        if not ref or ref.get("nodes") != case.n:
            rows.append({"r": r, "unavailable": "no oracle reference"})
            continue
        k_ref = ref["k_over_d2"]
        row = {"r": r, "nodes": case.n, "k_ref": k_ref}
        sched = {}
        for name, prec, m in (("fp64_zero", rbf.RBF_FP64, None), ("fp32c_zero", rbf.RBF_FP32C, None),
                              ("fp32c_warm", rbf.RBF_FP32C, mlp)):
            h, code = wsm.permeability_history(case, m, chunk=chunk, max_steps=max_steps, precision=prec, m_p=m_p,
                                               v_ref=v_ref, tune_steps=0 if prec in sched else 200,
                                               schedule=sched.get(prec))
            sched[prec] = code
            hit = _first_within(h, k_ref)
            row[name] = {"steps": None if hit is None else hit[0], "seconds": None if hit is None else hit[2],
                         "k_start_rel_err": abs(h[0][1] - k_ref) / k_ref,
                         "k_end_rel_err": abs(h[-1][1] - k_ref) / k_ref}
            if hit is not None and tot[name] is not None:
                tot[name][0] += hit[0]
                tot[name][1] += hit[2]
            else:
                tot[name] = None
        rows.append(row)
    clk.__exit__(None, None, None)
    summ = {k: (None if v is None else {"steps": v[0], "seconds": v[1]}) for k, v in tot.items()}
    gain = None
    if summ["fp32c_zero"] and summ["fp32c_warm"]:
        gain = {"steps_warm_over_zero": summ["fp32c_warm"]["steps"] / summ["fp32c_zero"]["steps"],
                "speedup_warm_fp32c_vs_fp64_zero": (summ["fp64_zero"]["seconds"] / summ["fp32c_warm"]["seconds"]
                                                    if summ["fp64_zero"] else None)}
    return {"metric": "time-to-steady-permeability (1e-4 rel) of held-out cells: network start vs rest",
            "value": None if not summ["fp32c_warm"] else summ["fp32c_warm"]["seconds"], "unit": "s",
            "n_gpus": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 compensated (+ bf16 network)", "data": "synthetic (seeded cells)",
            "config": {"workload": f"{len(train)} training cells and {len(C5_HELDOUT_RADII)} held-out cells, jittered "
                                   f"grid h=1/{n_axis} ({min(c.n for c in train)}-{max(c.n for c in train)} nodes), "
                                   f"N_L=25, v_ref={v_ref}",
                       "train_samples": int(len(data[0])), "train_data_s": t_data,
                       "train_cells_converged": sum(x["status"] == 0 for x in res), "train_s": t_train,
                       "final_train_loss": float(hist[-1]), "chunk": chunk, "max_steps": max_steps},
            "totals": summ, "gain": gain, "heldout": rows, "clocks": clk.summary()}


def _reference_workload(args):
    if args.workload == "acm-config4":
        import synth
        c = CFG4
        case = synth.refined_cell(r=c["r"], h_min=c["h_min"], h_max=c["h_max"], ramp=args.cfg4_ramp, seed=c["seed"])
        base = _oracle_acm_baseline(case, c, budget_s=60.0)
        metric = "node-steps/s (ACM steps, config 4)"
    else:
        print(json.dumps({"impl": "reference", "unavailable": f"no CPU reference leg for {args.workload}"}))
        return 0
    print(json.dumps({"metric": metric, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus, "impl": "reference",
                      "higher_is_better": True, "dtype": "f64", "cpu_baseline": base,
                      "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
