"""Benchmark: certified dual bounds per second at a 1e-6 relative gap.

Workload (default): one branch-and-bound root node of least squares with
FP32 X, n=20000, p=50000, k=20, lambda2=0.1, M=1.5, Toeplitz 0.9 rows, 20 x +-1
ground truth, SNR 5 -- the single-node configuration of the HBM roofline.
One step = one certified bound: problem setup on the resident X (column norms,
power iteration for L), restarted FISTA to a 1e-6 gap, FP64 certificate.
X (4 GB) is larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed.run, one rank per GPU; every rank solves its
own replica (nodes are independent: no data-path collective), value = all
bounds / max rank time ("scaling": "weak").  --impl reference times the FP64
CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "certified dual bounds/sec at 1e-6 rel gap"
UNIT = "bounds/s"
WORKLOAD = dict(workload="single-node least squares FP32 X n=20000 p=50000 k=20 lambda2=0.1 "
                         "M=1.5 toeplitz 0.9, root node, rel gap 1e-6",
                n=20000, p=50000, k=20, lambda2=0.1, M=1.5, r=0.9, x_dtype="f32",
                loss="least_squares", rel_gap=1e-6, l2="X (4 GB) larger than L2; no flush")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "gradient_pass_traffic.json")
KERNEL_SRC = os.path.join(ROOT, "paper_2502_09502_gb300", "csrc", "k_matvec.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--x-dtype", default="f32", choices=["f32", "fp8"],
                    help="single workload: X in FP32 (default) or FP8 e4m3 with per-column power-of-two "
                         "scales quantized from the same FP32 instance (the experiment of the precision pattern); "
                         "batched and bnb workloads: fp8 replaces their BF16 X the same way")
    ap.add_argument("--no-batched", action="store_true",
                    help="single workload: leave out the batched comparison object")
    ap.add_argument("--small", action="store_true",
                    help="8000 x 20000 instance of the same generator (640 MB X, still larger "
                         "than L2) for profiler captures; not a benchmark line")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "serving", "prox", "bnb", "eig"],
                    help="single: the single-node FP32 line (default); batched: 512 nodes of "
                         "the batched logistic BF16 workload in one ksc_solve_batch call; eig: the "
                         "eigen-perspective relaxation on a least-squares instance of the batched shape")
    ap.add_argument("--loss", default="logistic", choices=["logistic", "sqhinge"],
                    help="batched workload: logistic (the configuration) or the squared hinge on the "
                         "same labels")
    ap.add_argument("--nodes", type=int, default=512, help="batched: nodes per call")
    ap.add_argument("--pool", type=int, default=4, help="serving: resident problems drawn from the mix")
    ap.add_argument("--requests", type=int, default=2048, help="serving: distinct requests (reused cyclically)")
    ap.add_argument("--burst", type=int, default=256, help="serving: requests of the saturation burst")
    ap.add_argument("--rates", type=float, nargs="+", default=[0.3, 0.6, 0.9],
                    help="serving: Poisson rates as fractions of the saturation throughput")
    ap.add_argument("--window", type=float, default=8.0, help="serving: seconds of arrivals per rate")
    ap.add_argument("--slots", type=int, default=256, help="serving: slots per problem session")
    ap.add_argument("--max-iter", type=int, default=20000, help="serving: iteration cap per request")
    ap.add_argument("--root-max-iter", type=int, default=0,
                    help="serving: iteration cap of the pool's root solves (warm starts; 0: --max-iter)")
    ap.add_argument("--no-serving", action="store_true",
                    help="default line: leave out the compact serving leg")
    ap.add_argument("--bnb-seconds", type=float, default=90.0, help="bnb: time limit")
    ap.add_argument("--bnb-batch", type=int, default=1024, help="bnb: nodes in flight (per launch)")
    ap.add_argument("--bnb-gap", type=float, default=1e-4, help="bnb: relative gap to certify")
    ap.add_argument("--bnb-n", type=int, default=20000, help="bnb: rows")
    ap.add_argument("--bnb-p", type=int, default=200000, help="bnb: columns")
    ap.add_argument("--eig-bnb-seconds", type=float, default=0.0,
                    help="eig: also run branch and bound on a 4000 x 2000 least-squares instance with "
                         "perspective and with eigen-perspective node bounds, each within this time "
                         "limit (0: skip)")
    ap.add_argument("--plain-nodes", type=int, default=64,
                    help="batched: nodes of the same batch (spread over k') solved one at a time by "
                         "the single-node solver for the comparison")
    ap.add_argument("--oracle-nodes", type=int, default=32,
                    help="batched: nodes of the batch also solved by the FP64 oracle on the host "
                         "cores (per-node rate and parity; 0: skip)")
    return ap.parse_args()


def make_problem(args):
    import ksc_inputs as G
    if args.small:
        P = G.make_problem(8000, 20000, r=0.9, seed=args.seed, loss=G.LSQ, k_true=20, snr=5.0,
                           x_dtype=G.F32, lambda2=0.1, M=1.5, k=20)
    else:
        P = G.cfg_single_node_f32(seed=args.seed)
    return P


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (SM clock, limits and throttle reasons) during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline

def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic(n, p):
    """DRAM bytes per gradient-pass launch from the committed ncu summary, scaled to
    this workload by the X bytes it streams -- null unless the summary was taken
    on the current kernel source."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        src = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
        if t.get("kernel_sha256") != src:
            return None
        return float(t["dram_bytes_per_launch"]) * (n * p) / float(t["n"] * t["p"])
    except Exception:
        return None


# ------------------------------------------------------------------ ranks

def max_over_ranks(x, dist, device="cuda"):
    """The largest of every rank's x (the job's wall time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(items, rank, world):
    """Rank r's share of independent work units (nodes, requests): r, r + world, ..."""
    return items[rank::world]


def whole_job_rate(units_per_rank, world, ms_max):
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world, dist):
    import torch
    from paper_2502_09502_gb300 import ksc as K
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    P = make_problem(args)
    n, p = P.n, P.p
    fp8 = args.x_dtype == "fp8"
    scales = None
    if fp8:
        import ksc_inputs as G
        bits, scales = G.quantize_fp8(P.X)
        Xd = torch.from_numpy(bits).cuda().view(torch.float8_e4m3fn)
    else:
        Xd = torch.from_numpy(P.X).cuda()
    xbytes = 1 if fp8 else 4
    stream = torch.cuda.Stream()
    node = K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-6, max_iter=100000)

    def step(profile=False, stats=None):
        prob = K.Problem(Xd, P.y, K.KSC_LOSS_LSQ, stream=stream, col_scale=scales)
        if profile:
            K.ksc_problem_profile(prob.h, True)
        t0 = time.perf_counter()
        r = prob.solve(node, want_beta=False, want_z=False)
        if stats is not None:
            stats["launches"] += K.ksc_problem_launch_count(prob.h)
            st = K.ksc_problem_solve_stats(prob.h)
            stats["sparse"].append(st["sparse_forward"])
            stats["fallback"].append(st["prox_fallback"])
            stats["pfast"].append(st["prox_predicted"])
            stats["dfast"].append(st["dual_predicted"])
            stats["pow"].append(prob.power_iters)
            stats["iters"].append(r.iters)
            for kid in range(3):
                nl, ms = K.ksc_problem_kernel_time(prob.h, kid)
                stats["k"][kid][0] += nl
                stats["k"][kid][1] += ms
            for key, kid in (("sel", K.KSC_KERNEL_PROX_SELECT), ("app", K.KSC_KERNEL_PROX_APPLY)):
                nl, ms = K.ksc_problem_kernel_time(prob.h, kid)
                stats[key][0] += nl
                stats[key][1] += ms
        prob.close()
        return r, t0

    for _ in range(args.warmup):
        r, _ = step()
        assert r.status == "ok" and r.rel_gap <= 1e-6, r
    stats = {"launches": 0, "pow": [], "iters": [], "sparse": [], "fallback": [], "pfast": [],
             "dfast": [],
             "k": [[0, 0.0], [0, 0.0], [0, 0.0]], "sel": [0, 0.0], "app": [0, 0.0]}
    lat = []
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[dev] if vis and len(vis.split(",")) > dev else str(dev)
    clocks = ClockSampler(smi_index)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r, _ = step(profile=True, stats=stats)
        lat.append(time.perf_counter() - t0)
        assert r.status == "ok" and r.rel_gap <= 1e-6, r
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist)
    value = whole_job_rate(args.steps, world, ms)

    # roofline of the dominant kernel (the gradient pass over X)
    nl, kms = stats["k"][0]
    grad_ms = kms / max(nl, 1)
    alg_bytes = n * p * xbytes + 3 * n * 8 + p * 8    # X (FP32 or FP8) + u_t, u_{t-1}, y + grad
    achieved = alg_bytes / (grad_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    shares = {name: round(stats["k"][i][1] / max(1e-9, sum(x[1] for x in stats["k"])), 4)
              for i, name in enumerate(["gradient", "prox", "forward"])}

    # end to end through the C ABI with host buffers: H2D of X and y inside the
    # timed region, D2H of beta and z
    e2e = None
    if args.e2e_steps > 0:
        Xh = torch.from_numpy(bits if fp8 else P.X).pin_memory()
        e_lat = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            prob = K.Problem(Xh.numpy(), P.y, K.KSC_LOSS_LSQ, stream=stream,
                             x_dtype=K.KSC_FP8 if fp8 else None, col_scale=scales)
            r = prob.solve(node, want_beta=True, want_z=True)
            prob.close()
            assert r.status == "ok"
        e_s = time.perf_counter() - t0
        e2e = {"value": args.e2e_steps * world / e_s if not dist else None, "unit": UNIT,
               "h2d_bytes_per_step": int(Xh.numpy().nbytes + P.y.nbytes),
               "d2h_bytes_per_step": int(2 * p * 8 + 64)}
        if dist:
            e2e["value"] = args.e2e_steps * world / max_over_ranks(e_s, dist)

    out = None
    if rank == 0:
        lat_ms = sorted(1e3 * x for x in lat)
        out = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp8" if fp8 else "f32",
            "data": "synthetic (seeded Toeplitz AR(1) rows, standardised columns)",
            "config": dict(WORKLOAD, parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                           **({"x_dtype": "fp8 e4m3, per-column power-of-two scales, quantized from the FP32 "
                                          "instance (the solved matrix is the quantized one)",
                               "l2": "X (1 GB) larger than L2; no flush"} if fp8 else {}),
                           **({"workload": "profiler case: single-node least squares FP32 X n=8000 p=20000 "
                                           "k=20 lambda2=0.1 M=1.5 toeplitz 0.9 (not a benchmark line)",
                               "n": 8000, "p": 20000, "l2": "X (640 MB) larger than L2; no flush"}
                              if args.small else {})),
            "latency_ms": {"p50": round(float(np.percentile(lat_ms, 50)), 3),
                           "p99": round(float(np.percentile(lat_ms, 99)), 3)},
            "iters_per_bound": float(np.mean(stats["iters"])),
            "lanczos_steps_per_bound": float(np.mean(stats["pow"])),
            "sparse_forward_steps_per_bound": float(np.mean(stats["sparse"])),
            "prox_fallback_steps_per_bound": float(np.mean(stats["fallback"])),
            "prox_predicted_steps_per_bound": float(np.mean(stats["pfast"])),
            "dual_predicted_steps_per_bound": float(np.mean(stats["dfast"])),
            "clocks": clk, "e2e": e2e, "gpu_launches": int(stats["launches"]),
            "kernel_time_share": shares,
            "us_per_step": {name: round(1e3 * stats[key][1] / max(stats[key][0], 1), 2)
                            for name, key in (("prox_select", "sel"), ("prox_apply", "app"))}
                           | {"gradient": round(1e3 * grad_ms, 2),
                              "forward": round(1e3 * stats["k"][2][1] / max(stats["k"][2][0], 1), 2)},
            "roofline": {"bound": "hbm", "kernel": "gradient pass X^T r (k_grad)",
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "peak_kind": peak_kind, "frac": round(achieved / peak, 4),
                         "traffic": None if fp8 else _traffic(n, p), "bytes_per_launch": alg_bytes,
                         "avg_launch_ms": round(grad_ms, 5), "launches": nl},
        }
    return out, P, stats


# ------------------------------------------------------------------ small FP64 configuration

SMALL = dict(workload="single-node least squares FP64 X n=500 p=100 k=5 lambda2=1 M=2 toeplitz 0.5, "
                      "5 x +-1, SNR 5, root node, rel gap 1e-6 (X fits in L2: latency-bound)",
             n=500, p=100, k=5, lambda2=1.0, M=2.0, r=0.5, x_dtype="f64", loss="least_squares")


def run_small(args, reps=20, samples=5):
    """The FP64 parity configuration: time per certified bound on the GPU (problem
    resident, L computed once), iterations, and the oracle's full solve on the same
    inputs (median of `samples`), with the two bounds compared."""
    import torch
    import ksc_inputs as G
    from oracle import oracle as O
    from paper_2502_09502_gb300 import ksc as K
    P = G.cfg_small_lsq(seed=args.seed)
    stream = torch.cuda.Stream()
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_LSQ, stream=stream)
    node = K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-6, max_iter=100000)
    for _ in range(3):
        r = prob.solve(node, want_z=False)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(reps):
        r = prob.solve(node, want_z=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall_ms = 1e3 * (time.perf_counter() - t0) / reps
    dev_ms = ev0.elapsed_time(ev1) / reps
    prob.close()
    times = []
    for _ in range(samples):
        t0 = time.perf_counter()
        ref = O.solve(P.X, P.y, O.LOSS_LSQ, P.lambda2, P.M, P.k, tol=1e-6, max_iter=100000)
        times.append(time.perf_counter() - t0)
    tight = O.solve(P.X, P.y, O.LOSS_LSQ, P.lambda2, P.M, P.k, tol=1e-12, max_iter=200000)
    return {"config": SMALL, "ms_per_bound": round(wall_ms, 3), "device_ms_per_bound": round(dev_ms, 3),
            "bounds_per_s": round(1e3 / wall_ms, 1), "iters": r.iters, "rel_gap": r.rel_gap,
            "oracle": {"ms_per_bound": round(1e3 * statistics.median(times), 2), "iters": ref.iters,
                       "cores": 1, "samples": samples},
            "dual_rel_diff_vs_oracle_1e-12": abs(r.dual_bound - tight.dual) / abs(tight.dual),
            "bound_below_oracle_primal": bool(r.dual_bound <= tight.primal)}


# ------------------------------------------------------------------ branch and bound

BNB = dict(workload="best-first branch and bound, least squares X n=20000 p=200000 k=15 lambda2=0.1 M=2 "
                    "toeplitz 0.7, 15 x +-1, SNR 3 (X drawn on the device in BF16; --x-dtype fp8: FP8 e4m3 "
                    "with power-of-two column scales), node bounds from the batched solver with continuous "
                    "batching")


def run_bnb(args):
    """ksc_bnb_solve on the full branch-and-bound workload within a time limit:
    node relaxations per second, the certified gap reached, and the time to
    certify when it is reached."""
    import torch
    import ksc_inputs as G
    from paper_2502_09502_gb300 import ksc as K
    torch.cuda.set_device(0)
    n, p, k = args.bnb_n, args.bnb_p, 15
    t0 = time.perf_counter()
    X, y, bstar = G.device_problem(n, p, r=0.7, seed=args.seed, loss=G.LSQ, k_true=15, snr=3.0)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    fp8 = args.x_dtype == "fp8"
    if fp8:
        # E4M3 with one power-of-two scale per column: s_j = 2^ceil(log2(max_i |X_ij| / 448))
        amax = X.float().abs().amax(dim=0).clamp_min(1e-30)
        s = torch.exp2(torch.ceil(torch.log2(amax / 448.0)))
        X8 = torch.empty((n, p), dtype=torch.float8_e4m3fn, device="cuda")
        for j0 in range(0, n, 2048):    # in row blocks: no FP32 copy of the whole matrix
            X8[j0:j0 + 2048] = (X[j0:j0 + 2048].float() / s).to(torch.float8_e4m3fn)
        del X
        torch.cuda.synchronize()
        prob = K.Problem(X8, y, K.KSC_LOSS_LSQ, stream=stream, col_scale=s.cpu().numpy().astype(np.float32))
        del X8
    else:
        prob = K.Problem(X, y, K.KSC_LOSS_LSQ, stream=stream)
    setup = time.perf_counter() - t0
    beta, res = prob.bnb(0.1, 2.0, k, opt_gap=args.bnb_gap, time_limit_s=args.bnb_seconds, batch=args.bnb_batch,
                         node_rel_gap=1e-6, node_max_iter=20000)
    supp = set(np.nonzero(beta)[0].tolist())
    truth = set(np.nonzero(bstar)[0].tolist())
    return {
        "metric": "branch-and-bound nodes/s", "value": round(res["nodes"] / max(res["seconds"], 1e-9), 2),
        "unit": "nodes/s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp8-e4m3" if fp8 else "bf16",
        "data": "synthetic (seeded Toeplitz AR(1) rows drawn on the device)",
        "config": dict(BNB, n=n, p=p, k=k, x_dtype="fp8-e4m3" if fp8 else "bf16", opt_gap=args.bnb_gap,
                       time_limit_s=args.bnb_seconds,
                       batch=args.bnb_batch, parallelism="single GPU"),
        "setup_s": round(setup, 1), "result": {kk: (float(f"{v:.10g}") if isinstance(v, float) else v)
                                                for kk, v in res.items()},
        "time_to_certify_s": round(res["seconds"], 2) if res["certified"] else None,
        "incumbent_support_size": len(supp), "true_support_recovered": len(supp & truth),
    }


# ------------------------------------------------------------------ prox micro-benchmark

PROX = dict(workload="prox of g (and g itself, of the prox outputs) on many vectors (Sec. 5.1 / Fig. 1 shapes): gamma ~ N(0, I), k=10, M=1, "
                     "rho=1, p = 100 * 2^i for i = 0..10, >= 2^24 elements per launch (>= 608 rows), "
                     "inputs larger than L2 from p = 100 on")


def run_prox(args, reps=10):
    """Elements per second of ksc_prox_g_batch (one CTA per vector) over the prox
    timing experiment's sizes; 16 algorithmic bytes per element (read w, write beta)."""
    import torch
    from paper_2502_09502_gb300 import ksc as K
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    g = torch.Generator(device="cuda")
    g.manual_seed(int(args.seed))
    try:
        hbm = float(json.load(open(PEAKS_FILE))["hbm_gbs"])
    except Exception:
        hbm = 6800.0
    sweep = []
    for i in range(11):
        p = 100 * 2 ** i
        count = max(4 * 152, -(-(1 << 24) // p))
        W = torch.randn((count, p), generator=g, device="cuda", dtype=torch.float64)
        out = torch.empty_like(W)
        torch.cuda.synchronize()

        def launch():
            K._check(K.ksc_prox_g_batch(W.data_ptr(), p, out.data_ptr(), p, p, count, 10, 1.0, 1.0, stream))

        for _ in range(3):
            launch()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        elems = count * p
        # g (Algorithm 2) of the prox outputs, one CTA per vector: 8 algorithmic
        # bytes per element (read b)
        gout = torch.empty(count, dtype=torch.float64, device="cuda")

        def glaunch():
            K._check(K.ksc_g_value_batch(out.data_ptr(), p, p, count, 10, 1.0, gout.data_ptr(), stream))

        for _ in range(3):
            glaunch()
        e0.record(stream)
        for _ in range(reps):
            glaunch()
        e1.record(stream)
        torch.cuda.synchronize()
        gms = e0.elapsed_time(e1) / reps
        sweep.append({"p": p, "vectors": count, "ms_per_launch": round(ms, 4),
                      "elements_per_s": round(elems / (ms / 1e3), 1),
                      "algorithmic_gbs": round(16.0 * elems / (ms / 1e3) / 1e9, 1),
                      "g_ms_per_launch": round(gms, 4), "g_elements_per_s": round(elems / (gms / 1e3), 1),
                      "g_algorithmic_gbs": round(8.0 * elems / (gms / 1e3) / 1e9, 1)})
        del W, out, gout
    # the oracle (sort + PAVA merge) on a bounded sample of the same shapes
    from oracle import oracle as O
    rng = np.random.default_rng(args.seed)
    t0, elems = time.perf_counter(), 0
    bs = []
    for p in (1600, 12800, 102400):
        for _ in range(3):
            bs.append(O.prox_g(rng.standard_normal(p), 10, 1.0, 1.0)[0])
            elems += p
    cpu_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for b in bs:
        O.g_value(b, 10, 1.0)
    cpu_g_s = time.perf_counter() - t0
    big = sweep[-1]
    return {
        "metric": "prox elements/s", "value": big["elements_per_s"], "unit": "elements/s", "n_gpus": 1,
        "steps": reps, "warmup": 3, "ms_per_step": big["ms_per_launch"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (torch Philox normals)",
        "config": dict(PROX, parallelism="single GPU"), "sweep": sweep,
        "roofline": {"bound": "hbm", "kernel": "k_prox_rows (p = 102400)", "achieved": big["algorithmic_gbs"],
                     "peak": hbm, "unit": "GB/s", "frac": round(big["algorithmic_gbs"] / hbm, 4),
                     "traffic": None, "bytes_per_element": 16},
        "cpu_baseline": {"value": round(elems / cpu_s, 1), "unit": "elements/s", "cores": 1, "kind": "oracle",
                         "sample": "3 vectors each of p = 1600, 12800, 102400 (same distribution and k, M, rho)",
                         "g_value": round(elems / max(cpu_g_s, 1e-9), 1)},
        "g_value": {"kernel": "k_gvalue_rows (ksc_g_value_batch, Algorithm 2 per vector)",
                    "elements_per_s": big["g_elements_per_s"], "algorithmic_gbs": big["g_algorithmic_gbs"],
                    "frac_of_hbm": round(big["g_algorithmic_gbs"] / hbm, 4), "p": big["p"]},
    }


# ------------------------------------------------------------------ serving workload

SERVING = dict(workload="serving stream: Poisson arrivals of single-node requests over a resident pool "
                        "drawn from the mix (least squares or logistic, n~U{2000..40000}, "
                        "p~U{1000..100000}, k~U{5..50}, lambda2 in {1e-3,1e-2,1e-1}, M~U[1,5], "
                        "Toeplitz r in {0.1,0.5,0.9}, 5 x +-1, SNR 5, BF16 X), nodes as in the batched "
                        "workload (|S0|~U{0..200}, |S1|~U{0..min(9,k)}, warm start = the problem's root "
                        "iterate + N(0,1e-2)), rel gap 1e-6, HBM admission budget 120 GB")


def run_serving(args):
    """Continuous batching through ksc_server_*: a pool of resident problems, a
    burst of requests for the saturation throughput, then Poisson streams at
    fractions of it with the latency of every request (submission to completion,
    as the server records it)."""
    import torch
    import ksc_inputs as G
    from paper_2502_09502_gb300 import ksc as K
    torch.cuda.set_device(0)
    budget = 120e9
    stream = torch.cuda.Stream()
    t_setup = time.perf_counter()
    pool, used = [], 0
    for sp in G.serving_mix(args.pool, seed=args.seed):
        X, y, _ = G.device_problem(sp["n"], sp["p"], r=sp["r"], seed=sp["seed"], loss=sp["loss"],
                                   k_true=5, snr=5.0)
        torch.cuda.synchronize()
        prob = K.Problem(X, y, sp["loss"], stream=stream)
        del X
        used += prob.bytes
        root = prob.solve(K.Node(sp["lambda2"], sp["M"], sp["k"], rel_gap_tol=1e-6,
                                 max_iter=args.root_max_iter or args.max_iter), want_z=False)
        pool.append(dict(spec=sp, prob=prob, root=root.beta, root_iters=root.iters))
    setup_s = time.perf_counter() - t_setup
    u = G.uniform(args.seed, 11, 4 * args.requests)

    def request(i):
        e = pool[min(int(u[4 * i] * len(pool)), len(pool) - 1)]
        sp, p = e["spec"], e["prob"].p
        z, o = G.node_sets(p, 1, seed=1000003 * args.seed + i, max_zero=200, max_one=min(9, sp["k"]))[0]
        warm = e["root"] + G.warm_perturbation(p, 1, seed=1000003 * args.seed + i)[0]
        return e, K.Node(sp["lambda2"], sp["M"], sp["k"], fixed_zero=z, fixed_one=o, warm_beta=warm,
                         rel_gap_tol=1e-6, max_iter=args.max_iter)

    memo = {}

    def req(i):
        i %= args.requests
        if i not in memo:
            memo[i] = request(i)
        return memo[i]

    server = K.Server(budget - used, max_slots=args.slots)

    def drive(times, first):
        """Submit request first+j at times[j] (seconds from now); poll until all finish."""
        for j in range(len(times)):
            req(first + j)            # built before the clock starts
        t0 = time.perf_counter()
        pending, done, j = {}, [], 0
        while j < len(times) or pending:
            now = time.perf_counter() - t0
            while j < len(times) and times[j] <= now:
                e, nd = req(first + j)
                pending[server.submit(e["prob"], nd)] = (e, nd, first + j)
                j += 1
            for tk in list(pending):
                r = server.poll(tk, timeout_ms=0, want_beta=False)
                if r is not None:
                    e, nd, idx = pending.pop(tk)
                    done.append((idx, e, r, server.latency(tk), time.perf_counter() - t0))
            if pending:
                time.sleep(0.0005)
        return done, time.perf_counter() - t0

    def summary(done, span, offered):
        lat = np.array([d[3] for d in done]) * 1e3
        ok = [d for d in done if (d[2].status == "ok" and d[2].rel_gap <= 1e-6) or d[2].pruned]
        flops = sum(12.0 * d[1]["prob"].n * d[1]["prob"].p * d[2].iters for d in done)
        return {"offered_per_s": None if offered is None else round(offered, 3),
                "achieved_per_s": round(len(ok) / span, 3), "requests": len(done), "certified": len(ok),
                "certified_fraction": round(len(ok) / max(len(done), 1), 4),
                "p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
                "span_s": round(span, 3), "tensor_tflops_executed": round(flops / span / 1e12, 1)}

    def per_problem(done):
        out = []
        for j, e in enumerate(pool):
            mine = [d for d in done if d[1] is e]
            if not mine:
                continue
            out.append({"problem": j, "requests": len(mine),
                        "certified": sum((d[2].status == "ok" and d[2].rel_gap <= 1e-6) or d[2].pruned for d in mine),
                        "mean_iters": round(float(np.mean([d[2].iters for d in mine])), 1),
                        "p50_ms": round(float(np.percentile([1e3 * d[3] for d in mine], 50)), 1)})
        return out

    # saturation: every request of a burst at once
    burst = min(args.burst, args.requests)
    done, span = drive(np.zeros(burst), 0)
    sat = summary(done, span, None)
    sat["per_problem"] = per_problem(done)
    cap = max(sat["achieved_per_s"], 1e-3)
    curve, nxt = [], burst
    for frac in args.rates:
        arr = G.poisson_arrivals(frac * cap, args.window, seed=args.seed + int(frac * 1000))
        done, span = drive(arr, nxt)
        nxt += len(arr)
        curve.append(dict(summary(done, span, frac * cap), fraction_of_saturation=frac))
    st = server.stats()
    # the same requests alone: each result is the same alone and in the mix
    inv = []
    for (idx, e, r, _, _) in done[:4]:
        alone = e["prob"].solve_batch([req(idx)[1]], want_beta=False)[0]
        inv.append(abs(alone.dual_bound - r.dual_bound) / max(abs(r.dual_bound), 1e-300))
    server.close()
    try:
        peak = float(json.load(open(PEAKS_FILE))["bf16_tflops_sustained"])
    except Exception:
        peak = 1700.0
    return {
        "metric": METRIC, "value": sat["achieved_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1 + len(args.rates),
        "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded Toeplitz AR(1) rows drawn on the device, standardised columns)",
        "config": dict(SERVING, pool=[dict({k: e["spec"][k] for k in ("loss", "n", "p", "k", "lambda2", "M", "r")},
                                           root_iters=e["root_iters"]) for e in pool],
                       pool_bytes=int(used), max_slots=args.slots, max_iter=args.max_iter,
                       parallelism="single GPU"),
        "setup_s": round(setup_s, 1),
        "saturation": sat, "latency_vs_throughput": curve,
        "tensor_frac_of_sustained_peak": round(sat["tensor_tflops_executed"] / peak, 4),
        "server": st, "alone_vs_mix_max_rel_dual_diff": float(max(inv)) if inv else None,
    }


def serving_leg(args):
    """The compact serving leg of the default line: a pool of 8 problems from the
    mix, a burst of 64 requests (saturation) and one Poisson stream at half of it,
    with p50/p99 latency and the certified fraction of each.  Requests (and the
    pool's root solves) are capped at 4000 iterations here so that the leg ends in
    a few minutes; the serving workload's own default cap is 20000."""
    a = argparse.Namespace(**vars(args))
    a.pool, a.burst, a.rates, a.window, a.requests = 8, 64, [0.5], 10.0, 256
    a.max_iter, a.root_max_iter, a.slots = 4000, 4000, 256
    r = run_serving(a)
    keep = ("metric", "value", "unit", "config", "setup_s", "saturation", "latency_vs_throughput",
            "tensor_frac_of_sustained_peak", "alone_vs_mix_max_rel_dual_diff")
    out = {k: r[k] for k in keep if k in r}
    out["config"] = {k: v for k, v in out["config"].items() if k != "pool"}
    out["config"]["pool_problems"] = a.pool
    return out


# ------------------------------------------------------------------ batched workload

BATCHED = dict(workload="batched logistic BF16 X n=10000 p=5000 k=10 lambda2=0.01 M=3 toeplitz 0.5, "
                        "512 nodes per call (|S0|~U{0..200}, |S1|~U{0..9}), warm start = root "
                        "iterate + N(0,1e-2), rel gap 1e-6",
               n=10000, p=5000, k=10, lambda2=0.01, M=3.0, r=0.5, x_dtype="bf16", loss="logistic",
               rel_gap=1e-6, l2="X (100 MB) and its column-major copy read by every step; no flush")


_ORACLE_CASE = {}


def _oracle_worker_init(seed, warm, L):
    """Spawned worker: regenerate the batched workload from its seed (no GPU data)."""
    import ksc_inputs as G
    P = G.cfg_batched_logistic(seed=seed)
    _ORACLE_CASE.update(P=P, X=P.X64(), warm=warm, L=L,
                        sets=G.node_sets(P.p, 512, seed=seed, max_zero=200, max_one=9),
                        pert=G.warm_perturbation(P.p, 512, seed=seed))


def _oracle_node(b):
    """One node of the batched workload solved by the FP64 oracle to a 1e-6 gap."""
    from oracle import oracle as O
    c = _ORACLE_CASE
    P, (zero, one) = c["P"], c["sets"][b]
    st = np.zeros(P.p, np.int8)
    st[zero] = O.ZERO
    st[one] = O.ONE
    t0 = time.perf_counter()
    r = O.solve(c["X"], P.y, P.loss, P.lambda2, P.M, P.k, state=st, warm=c["warm"] + c["pert"][b],
                L=c["L"], tol=1e-6, max_iter=100000)
    return b, r.dual, r.primal, r.iters, r.status, time.perf_counter() - t0


def oracle_subsample(seed, count, gpu_res):
    """The FP64 oracle on a seeded subsample of the batched workload's nodes: its own
    root solve (all cores) for the warm starts, then the nodes in parallel worker
    processes (one core each), giving a per-node rate on the host and the parity of
    the GPU's certified bounds on those nodes."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import ksc_inputs as G
    from oracle import oracle as O
    P = G.cfg_batched_logistic(seed=seed)
    idx = np.sort(np.argsort(G.uniform(seed, 12, len(gpu_res)))[:count])
    t0 = time.perf_counter()
    X = P.X64()
    # L (any valid step constant; it only changes the path): power iteration to 1e-8
    # with the 1.01 factor of the GPU path, c_f = 1/4 for logistic
    L = 0.25 * O.power_iteration(X, tol=1e-8, openmp=True)[0] * 1.01
    root = O.solve(X, P.y, P.loss, P.lambda2, P.M, P.k, L=L, tol=1e-6, max_iter=100000, openmp=True)
    del X
    t_root = time.perf_counter() - t0
    workers = max(1, min(count, os.cpu_count() or 1))
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                initializer=_oracle_worker_init, initargs=(seed, root.beta, L)) as pool:
        out = list(pool.map(_oracle_node, [int(b) for b in idx]))
    wall = time.perf_counter() - t0
    rel = [abs(gpu_res[b].dual_bound - d) / abs(d) for b, d, _, _, _, _ in out]
    return {"nodes": int(count), "indices": [int(b) for b in idx], "workers": workers,
            "cpu": host_cpu()["model"],
            "bounds_per_s_all_cores": round(count / wall, 4),
            "s_per_node_one_core_mean": round(float(np.mean([x[5] for x in out])), 2),
            "oracle_iters_mean": round(float(np.mean([x[3] for x in out])), 1),
            "oracle_root_s": round(t_root, 1),
            "converged": sum(x[4] == "converged" for x in out),
            "max_rel_dual_diff": float(max(rel)),
            "gpu_bound_le_oracle_primal": bool(all(gpu_res[b].dual_bound <= pr for b, _, pr, _, _, _ in out)),
            "note": "oracle and GPU both at a 1e-6 gap from their own root solutions + the same perturbations"}


def run_batched(args):
    """One step = one ksc_solve_batch call over `nodes` nodes of the batched logistic
    workload (X resident; L computed once at problem creation)."""
    import torch
    import ksc_inputs as G
    from paper_2502_09502_gb300 import ksc as K
    torch.cuda.set_device(0)
    P = G.cfg_batched_logistic(seed=args.seed)
    sq = getattr(args, "loss", "logistic") == "sqhinge"
    loss = K.KSC_LOSS_SQHINGE if sq else K.KSC_LOSS_LOGISTIC
    n, p, B = P.n, P.p, args.nodes
    fp8 = getattr(args, "x_dtype", "f32") == "fp8"
    Xd = torch.from_numpy(P.X.view(np.int16)).cuda().view(torch.bfloat16)
    stream = torch.cuda.Stream()
    if fp8:
        # FP8 e4m3 with power-of-two column scales, quantized from the BF16 instance;
        # the solved problem is the represented matrix X_ij s_j
        bits, sc = G.quantize_fp8(G.bf16_to_f32(P.X))
        Xd = torch.from_numpy(bits).cuda().view(torch.float8_e4m3fn)
        prob = K.Problem(Xd, P.y, loss, stream=stream, col_scale=sc)
    else:
        prob = K.Problem(Xd, P.y, loss, stream=stream)
    root = prob.solve(K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-6))
    sets = G.node_sets(p, B, seed=args.seed, max_zero=200, max_one=9)
    pert = G.warm_perturbation(p, B, seed=args.seed)
    nodes = [K.Node(P.lambda2, P.M, P.k, fixed_zero=z, fixed_one=o, warm_beta=root.beta + pert[b],
                    rel_gap_tol=1e-6, max_iter=100000) for b, (z, o) in enumerate(sets)]

    def check(res):
        bad = [r for r in res if not (r.status == "ok" and r.rel_gap <= 1e-6) and not r.pruned]
        assert not bad, bad[:2]

    for _ in range(args.warmup):
        check(prob.solve_batch(nodes, want_beta=False))
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    clocks = ClockSampler(vis.split(",")[0] if vis else "0")
    l0 = K.ksc_problem_launch_count(prob.h)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat, iters = [], []
    ev0.record(stream)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = prob.solve_batch(nodes, want_beta=False)
        lat.append(time.perf_counter() - t0)
        check(res)
        iters.append(float(np.mean([r.iters for r in res])))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = K.ksc_problem_launch_count(prob.h) - l0
    value = B * args.steps / (ms / 1e3)
    # per-phase device time: one more call with events around every kernel of the
    # lock-step graph and around the certificate and anchor phases (not timed above)
    K.ksc_problem_profile(prob.h, True)
    K.ksc_problem_kernel_time(prob.h, 0, reset=True)
    pres = prob.solve_batch(nodes, want_beta=False)
    check(pres)
    kt = {name: K.ksc_problem_kernel_time(prob.h, kid)
          for name, kid in [("residual", K.KSC_KERNEL_B_RESID), ("xt_r", K.KSC_KERNEL_B_GRAD),
                            ("prox", K.KSC_KERNEL_B_PROX), ("x_dbeta", K.KSC_KERNEL_B_FWD),
                            ("step", K.KSC_KERNEL_B_STEP), ("certificates", K.KSC_KERNEL_B_CERT),
                            ("anchors", K.KSC_KERNEL_B_ANCHOR)]}
    bstats = K.ksc_problem_solve_stats(prob.h)
    K.ksc_problem_profile(prob.h, False)
    tot = sum(v[1] for v in kt.values())
    shares = {k: round(v[1] / max(tot, 1e-9), 4) for k, v in kt.items()}
    # rooflines.  Tensor products: algorithmic flops 2 n p per running node per
    # step (tiles whose nodes have all stopped are skipped) over the product's
    # device time, against the sustained BF16 peak (the products run inside a long
    # call).  Exact products of anchors and certificates: two per anchor (X b_ref,
    # X^T r_ref) and two per certificate (X b^, X^T zeta), n p multiply-adds each.
    # On the tensor cores (k_tcx, the default) each is executed as 18 BF16 slice
    # products (3 slices of X times 6 of the FP64 vector), 36 n p flops, against the
    # sustained BF16 peak; with KSC_EXACT_PRODUCT=stream (k_dfprod, double-float
    # FP32 arithmetic) against the FP32 FMA rate 152 SMs x 128 lanes x the median
    # SM clock sampled during the timed calls.  Both over the anchor and
    # certificate phases' device time (slicing, products, residuals, epilogues).
    node_steps = float(sum(r.iters for r in pres))
    alg = 2.0 * n * p * node_steps
    try:
        pk = json.load(open(PEAKS_FILE))
        peak, peak_kind = float(pk["bf16_tflops_sustained"]), "measured (sustained)"
    except Exception:
        peak, peak_kind = 1700.0, "fallback (sustained)"
    bf16_peak = peak
    if fp8:
        # E4M3 products: the BF16 peak times the nominal FP8 / BF16 ratio (4.5 / 2.25)
        peak, peak_kind = 2.0 * peak, peak_kind + " BF16 x 2 (nominal FP8/BF16 ratio)"
    pieces_label = "4 E4M3 pieces" if fp8 else "3 BF16 pieces"

    def tensor_line(key, label):
        nl_, ms_ = kt[key]
        ach = alg / (ms_ / 1e3) / 1e12
        return {"bound": "tensor", "kernel": label, "achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s",
                "peak_kind": peak_kind, "frac": round(ach / peak, 4), "traffic": None,
                "flops_per_launch": alg / max(nl_, 1), "pieces": 4 if fp8 else 3, "node_steps": node_steps,
                "avg_launch_ms": round(ms_ / max(nl_, 1), 5), "launches": nl_}

    exact_products = 2.0 * (bstats["batch_certificates"] + bstats["batch_anchors"])
    macs = exact_products * n * p
    ex_ms = kt["certificates"][1] + kt["anchors"][1]
    fp64_rate = macs / (ex_ms / 1e3) / 1e12
    if os.environ.get("KSC_EXACT_PRODUCT", "") == "stream":
        sm_mhz = clk.get("sm_mhz") or 2070.0
        fma_peak = 152 * 128 * sm_mhz * 1e6 / 1e12          # T multiply-adds/s
        exact_line = {"bound": "alu", "kernel": "exact double-float products of anchors and certificates "
                                                "(k_dfprod; the anchor and certificate phases' device time)",
                      "achieved": round(fp64_rate, 3), "peak": round(fma_peak, 2), "unit": "T multiply-adds/s",
                      "peak_kind": f"derived: 152 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (median sampled)",
                      "frac": round(fp64_rate / fma_peak, 4)}
    else:
        ex_flops = 36.0 * macs
        ex_ach = ex_flops / (ex_ms / 1e3) / 1e12
        exact_line = {"bound": "tensor", "kernel": "exact products of anchors and certificates on the tensor "
                                                   "cores (k_tcx, 18 BF16 slice products each; the anchor and "
                                                   "certificate phases' device time)",
                      "achieved": round(ex_ach, 1), "peak": bf16_peak, "unit": "TFLOP/s",
                      "peak_kind": "measured (sustained)" if "measured" in peak_kind else "fallback (sustained)",
                      "frac": round(ex_ach / bf16_peak, 4), "executed_flops": ex_flops}
    exact_line.update({"traffic": None, "products": exact_products, "multiply_adds": macs,
                       "exact_fp64_multiply_adds_per_s": round(fp64_rate * 1e12, 1), "device_ms": round(ex_ms, 2)})
    rooflines = {"xt_r": tensor_line("xt_r", f"X^T r for the running nodes (k_tcgemm, {pieces_label})"),
                 "x_dbeta": tensor_line("x_dbeta", f"X (beta - beta_ref) for the running nodes (k_tcgemm, "
                                                   f"{pieces_label})"),
                 "exact_products": exact_line}
    phase_ms = {"exact_products": ex_ms, "xt_r": kt["xt_r"][1], "x_dbeta": kt["x_dbeta"][1]}
    dominant = max(phase_ms, key=phase_ms.get)

    # the plain single-node solver on a sample of the same nodes spread over the
    # budgets k' (every (B / plain)-th node in order of k'), one at a time: on an
    # FP32 copy of X (the same represented matrix: BF16 widens exactly), the solver
    # the metric compares against, and on the BF16 X itself
    order = sorted(range(B), key=lambda b: (len(sets[b][1]), b))
    take = max(1, min(args.plain_nodes, B))
    sample = [order[int(i * B / take)] for i in range(take)]

    def plain_rate(pr):
        pr.solve(nodes[sample[0]], want_beta=False, want_z=False)   # untimed: graph and buffers
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for b in sample:
            r = pr.solve(nodes[b], want_beta=False, want_z=False)
            assert r.status == "ok" or r.pruned, r
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return len(sample) / (e0.elapsed_time(e1) / 1e3), len(sample) / wall

    if fp8:
        X32 = (torch.from_numpy(G.fp8_values(bits)) * torch.from_numpy(sc)[None, :]).cuda()
    else:
        X32 = Xd.float()
    prob32 = K.Problem(X32, P.y, loss, stream=stream)
    plain32, plain32_wall = plain_rate(prob32)
    prob32.close()
    del X32
    plain16, plain16_wall = plain_rate(prob)
    plain = plain32
    # end to end: X from pinned host memory into a new problem, the batched call, results back
    if fp8:
        Xh = torch.from_numpy(bits).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob2 = K.Problem(Xh.numpy(), P.y, loss, stream=stream, x_dtype=K.KSC_FP8, col_scale=sc)
    else:
        Xh = torch.from_numpy(P.X.view(np.int16)).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob2 = K.Problem(Xh.numpy().view(np.uint16), P.y, loss, stream=stream, x_dtype=K.KSC_BF16)
    res = prob2.solve_batch(nodes, want_beta=True)
    e_s = time.perf_counter() - t0
    prob2.close()
    check(res)
    lat_ms = sorted(1e3 * x for x in lat)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp8-e4m3" if fp8 else "bf16",
        "data": "synthetic (seeded Toeplitz AR(1) rows, standardised columns)",
        "config": dict(BATCHED, nodes=B, parallelism="single GPU",
                       **({"x_dtype": "fp8-e4m3 (power-of-two column scales, quantized from the BF16 instance)",
                           "workload": BATCHED["workload"].replace("BF16 X", "FP8 e4m3 X")} if fp8 else {}),
                       **({"workload": BATCHED["workload"].replace("batched logistic", "batched squared hinge"),
                           "loss": "squared_hinge"} if sq else {})),
        "latency_ms": {"p50": round(float(np.percentile(lat_ms, 50)), 3),
                       "p99": round(float(np.percentile(lat_ms, 99)), 3)},
        "iters_per_bound": float(np.mean(iters)),
        "lockstep_steps_per_call": kt["xt_r"][0],
        "certificates_per_call": bstats["batch_certificates"],
        "anchors_per_call": bstats["batch_anchors"],
        "prox_fallbacks_per_call": bstats["prox_fallback"],
        "product_tiles": {"x_dbeta": [bstats["tile_fwd"], "stream-K" if bstats["stream_k_fwd"] else "tiled"],
                          "xt_r": [bstats["tile_grad"], "stream-K" if bstats["stream_k_grad"] else "tiled"]},
        "device_ms_per_call": {k: round(v[1], 2) for k, v in kt.items()},
        "plain_single_node": {"value": round(plain32, 3), "unit": UNIT, "x_dtype": "f32", "nodes": len(sample),
                              "ratio": round(value / plain32, 2), "wall_value": round(plain32_wall, 3),
                              "sample": "every (512/nodes)-th node in order of k' = k - |S1|, CUDA events"},
        "plain_single_node_bf16" if not fp8 else "plain_single_node_fp8":
            {"value": round(plain16, 3), "unit": UNIT, "x_dtype": "fp8-e4m3" if fp8 else "bf16",
                                   "nodes": len(sample), "ratio": round(value / plain16, 2),
                                   "wall_value": round(plain16_wall, 3)},
        "clocks": clk, "gpu_launches": int(launches), "kernel_time_share": shares,
        "e2e": {"value": round(B / e_s, 3), "unit": UNIT,
                "h2d_bytes_per_step": int((bits.nbytes if fp8 else P.X.nbytes) + P.y.nbytes),
                "d2h_bytes_per_step": int(B * (p * 8 + 64))},
        "roofline": dict(rooflines[dominant], dominant_of=sorted(phase_ms)),
        "rooflines": rooflines,
    }
    if args.oracle_nodes > 0 and not fp8:
        line["oracle_subsample"] = oracle_subsample(args.seed, args.oracle_nodes, res)
    return line


EIG = dict(workload="eigen-perspective relaxation (App. D.2), least squares BF16 X n=10000 p=5000 k=10 "
                    "lambda2=0.01 M=3 toeplitz 0.5, 10 x +-1, SNR 5, 512 nodes per call as in the batched "
                    "workload (|S0|~U{0..200}, |S1|~U{0..9}, warm start = root iterate + N(0,1e-2)), "
                    "rel gap 1e-6",
           n=10000, p=5000, k=10, lambda2=0.01, M=3.0, r=0.5, x_dtype="bf16", loss="least_squares",
           rel_gap=1e-6)


def run_eig(args):
    """The certified shift (Gram matrix and Cholesky bisection), then one step = one
    ksc_solve_batch call over the nodes with KSC_FLAG_EIG, beside the same call with
    perspective nodes: throughput and how much the bounds rise."""
    import torch
    import ksc_inputs as G
    from paper_2502_09502_gb300 import ksc as K
    torch.cuda.set_device(0)
    P = G.make_problem(10000, 5000, r=0.5, seed=args.seed, loss=G.LSQ, k_true=10, snr=5.0, x_dtype=G.BF16,
                       lambda2=0.01, M=3.0, k=10)
    n, p, B = P.n, P.p, args.nodes
    Xd = torch.from_numpy(P.X.view(np.int16)).cuda().view(torch.bfloat16)
    stream = torch.cuda.Stream()
    prob = K.Problem(Xd, P.y, K.KSC_LOSS_LSQ, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam = prob.eig_lambda()
    t_lam = time.perf_counter() - t0
    root = prob.solve(K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-6))
    sets = G.node_sets(p, B, seed=args.seed, max_zero=200, max_one=9)
    pert = G.warm_perturbation(p, B, seed=args.seed)
    mk = lambda fl: [K.Node(P.lambda2, P.M, P.k, fixed_zero=z, fixed_one=o, warm_beta=root.beta + pert[b],
                            rel_gap_tol=1e-6, max_iter=100000, flags=fl) for b, (z, o) in enumerate(sets)]
    out = {}
    for name, fl in (("perspective", 0), ("eigen_perspective", K.KSC_FLAG_EIG)):
        nodes = mk(fl)
        for _ in range(args.warmup):
            prob.solve_batch(nodes, want_beta=False)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            res = prob.solve_batch(nodes, want_beta=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        assert all((r.status == "ok" and r.rel_gap <= 1e-6) or r.pruned for r in res)
        out[name] = dict(value=round(B * args.steps / (ms / 1e3), 3), ms_per_step=round(ms / args.steps, 3),
                         iters_per_bound=float(np.mean([r.iters for r in res])),
                         bounds=np.array([r.dual_bound for r in res]))
    bp, be = out["perspective"].pop("bounds"), out["eigen_perspective"].pop("bounds")
    rise = (be - bp) / np.abs(bp)
    # the root relaxation on the single-node path (one ksc_solve_node call), both bounds
    single = {}
    for name, fl in (("perspective", 0), ("eigen_perspective", K.KSC_FLAG_EIG)):
        nd = K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-6, max_iter=100000, flags=fl)
        prob.solve(nd)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            r = prob.solve(nd)
        ev1.record(stream)
        torch.cuda.synchronize()
        assert r.status == "ok" and r.rel_gap <= 1e-6
        single[name] = dict(ms_per_solve=round(ev0.elapsed_time(ev1) / args.steps, 3), iters=int(r.iters),
                            dual_bound=float(r.dual_bound), primal=float(r.primal))
    single["bound_rise_rel"] = ((single["eigen_perspective"]["dual_bound"] - single["perspective"]["dual_bound"])
                                / abs(single["perspective"]["dual_bound"]))
    bnb = None
    if args.eig_bnb_seconds > 0:
        # branch and bound on a smaller instance of the config-4 generator with n > p
        Pb = G.make_problem(4000, 2000, r=0.7, seed=args.seed, loss=G.LSQ, k_true=10, snr=3.0,
                            x_dtype=G.BF16, lambda2=0.1, M=2.0, k=10)
        pb = K.Problem(torch.from_numpy(Pb.X.view(np.int16)).cuda().view(torch.bfloat16), Pb.y,
                       K.KSC_LOSS_LSQ, stream=stream)
        bnb = {"config": "least squares BF16 X n=4000 p=2000 k=10 lambda2=0.1 M=2 toeplitz 0.7, "
                         "10 x +-1, SNR 3, opt gap 1e-4, 256 nodes in flight",
               "time_limit_s": args.eig_bnb_seconds}
        for name, fl in (("perspective", 0), ("eigen_perspective", K.KSC_FLAG_EIG)):
            _, r = pb.bnb(0.1, 2.0, 10, opt_gap=1e-4, time_limit_s=args.eig_bnb_seconds, batch=256,
                          node_rel_gap=1e-6, node_max_iter=20000, node_flags=fl)
            bnb[name] = {kk: r[kk] for kk in ("certified", "gap", "seconds", "nodes", "pruned",
                                              "heuristic_solves", "incumbent", "lower_bound")}
    return {
        "metric": METRIC, "value": out["eigen_perspective"]["value"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["eigen_perspective"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded Toeplitz AR(1) rows, standardised columns)",
        "config": dict(EIG, nodes=B, parallelism="single GPU"),
        "eig_lambda": lam, "eig_lambda_seconds": round(t_lam, 3),
        "perspective": out["perspective"], "eigen_perspective": out["eigen_perspective"],
        "bound_rise": {"mean_rel": float(rise.mean()), "max_rel": float(rise.max()),
                       "nodes_higher": int((rise > 1e-9).sum()), "nodes_lower": int((rise < -1e-9).sum())},
        "single_node_root": single,
        "branch_and_bound": bnb,
    }


# ------------------------------------------------------------------ oracle timing

def host_cpu():
    """The host's CPU model and logical core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"model": model, "nproc": os.cpu_count()}


def time_oracle_sample(P, openmp=False):
    """The FP64 oracle on the same workload, on a bounded sample: one power-iteration
    step (2 passes over X) and one step of Algorithm 3 including its set-up (oracle:
    the initial X beta, then X gamma, X^T r, X beta and the bound's X^T zeta)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.power_iteration(P.X, tol=0.0, max_iter=1, openmp=openmp)
    t_pow = time.perf_counter() - t0
    L = 2.0 * float(np.sum(P.X.astype(np.float64) ** 2))   # cheap valid step for timing only
    t0 = time.perf_counter()
    O.solve(P.X, P.y, O.LOSS_LSQ, P.lambda2, P.M, P.k, L=L, tol=0.0, max_iter=1, openmp=openmp)
    t_iter = time.perf_counter() - t0
    return t_pow, t_iter


def oracle_rate(P, iters, pows, samples=5, openmp=False):
    """Median over `samples` bounded samples of the seconds per bound, extrapolated
    to `pows` power-iteration steps and `iters` steps of Algorithm 3."""
    from oracle import oracle as O
    per = []
    for _ in range(samples):
        t_pow, t_iter = time_oracle_sample(P, openmp=openmp)
        per.append((pows * t_pow + iters * t_iter, t_pow, t_iter))
    per.sort()
    med = per[len(per) // 2]
    return {"bounds_per_s": 1.0 / med[0], "s_per_bound": med[0], "power_step_s": med[1],
            "fista_step_s": med[2], "threads": O.threads(openmp), "samples": samples}


def cpu_baseline(P, iters, pows, samples=5):
    """The oracle as it stands on the host cores: single-threaded and with its
    matrix-vector products on every core (OpenMP build, identical results), each the
    median of `samples` bounded samples extrapolated to a full bound."""
    one = oracle_rate(P, iters, pows, samples, openmp=False)
    try:
        allc = oracle_rate(P, iters, pows, samples, openmp=True)
    except Exception as e:          # no OpenMP runtime on the host
        allc = None
        err = str(e)
    best = allc if allc else one
    cpu = host_cpu()
    out = {"value": best["bounds_per_s"], "unit": UNIT, "cores": best["threads"], "kind": "oracle",
           "cpu": cpu["model"], "nproc": cpu["nproc"],
           "single_thread": {"value": one["bounds_per_s"], "power_step_s": round(one["power_step_s"], 3),
                             "fista_step_s": round(one["fista_step_s"], 3)},
           "all_cores": None if allc is None else {
               "value": allc["bounds_per_s"], "threads": allc["threads"],
               "power_step_s": round(allc["power_step_s"], 3), "fista_step_s": round(allc["fista_step_s"], 3)},
           "sample": (f"median of {samples} samples, each 1 power-iteration step and 1 step of Algorithm 3 "
                      f"(with its set-up) of the FP64 oracle on the full workload, extrapolated to "
                      f"{pows:.0f} matrix-vector pairs for L + {iters:.0f} steps per bound (the counts "
                      f"of the full GPU solve); value = the all-cores figure")}
    if allc is None:
        out["all_cores_error"] = err
    return out


# iteration counts of a full solve of this workload (matrix-vector pairs for L, FISTA
# steps), as the GPU solve reports them; they extrapolate the oracle's bounded sample
# when it runs on its own
FULL_SOLVE_COUNTS = {"pow": 32, "iters": 344}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (all-cores build), each
    step one bounded sample of the same workload, extrapolated to a full bound."""
    from oracle import oracle as O
    P = make_problem(args)
    cnt = FULL_SOLVE_COUNTS
    try:
        O.build(openmp=True)
        openmp = True
    except Exception:
        openmp = False
    per_step, wall = [], 0.0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t_pow, t_iter = time_oracle_sample(P, openmp=openmp)
        if s >= args.warmup:
            wall += time.perf_counter() - t0
            per_step.append(cnt["pow"] * t_pow + cnt["iters"] * t_iter)
    per_bound = statistics.median(per_step)
    value = 1.0 / per_bound
    cpu = host_cpu()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * wall / args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism="host cores"),
        "cpu_baseline": {"value": round(value, 8), "unit": UNIT, "cores": O.threads(openmp), "kind": "oracle",
                         "cpu": cpu["model"], "nproc": cpu["nproc"],
                         "s_per_bound_extrapolated": round(per_bound, 1),
                         "sample": f"each step: 1 power-iteration step + 1 step of Algorithm 3 of the FP64 "
                                   f"oracle on the full workload ({'all cores' if openmp else '1 core'}); "
                                   f"value = 1 / the median over steps of the time extrapolated to "
                                   f"{cnt['pow']} power iterations + {cnt['iters']} steps per bound; "
                                   f"ms_per_step is the measured time of one sampled step"},
        "e2e": {"value": round(value, 8), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as D
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        D.init_process_group("nccl")
        dist = D
    if args.workload in ("batched", "serving", "prox", "bnb", "eig"):
        if world > 1:
            raise SystemExit(f"the {args.workload} workload runs on one GPU")
        run = {"batched": run_batched, "serving": run_serving, "prox": run_prox, "bnb": run_bnb,
               "eig": run_eig}[args.workload]
        print(json.dumps(run(args)), flush=True)
        return
    out, P, stats = run_ours(args, rank, world, dist)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(P, float(np.mean(stats["iters"])),
                                               float(np.mean(stats["pow"])))
        if world == 1 and not args.small:
            out["small_fp64"] = run_small(args)
        if not args.no_batched and world == 1 and not args.small:
            # the batched mixed-precision form on its own workload, timed the same
            # way, beside the plain single-node solver on the same nodes
            del P
            b = run_batched(args)
            out["batched"] = {k: b[k] for k in (
                "value", "unit", "steps", "warmup", "ms_per_step", "dtype", "config", "latency_ms",
                "iters_per_bound", "plain_single_node", "plain_single_node_bf16", "e2e", "roofline",
                "rooflines", "device_ms_per_call", "clocks", "gpu_launches", "certificates_per_call",
                "anchors_per_call", "prox_fallbacks_per_call", "lockstep_steps_per_call", "product_tiles")
                if k in b}
            if "oracle_subsample" in b:
                out["batched"]["oracle_subsample"] = b["oracle_subsample"]
        if not args.no_serving and world == 1 and not args.small:
            out["serving"] = serving_leg(args)
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
