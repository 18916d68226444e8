#!/usr/bin/env python
"""Benchmark of the randomized SVD hot path on GB300 (one JSON line on rank 0).

Workload (default): the 16384 x 16384 matrix A = U diag(j^-1.5) V^T with Haar
U, V, rank k = 100, oversampling p = 10, q = 1 power step (four passes over
A), compared with the plain FP32 CUDA-core path on the float32 A at matched
reconstruction error.  The headline tensor-core configuration stores A as bfloat16
hi + bfloat16 lo (A - hi) and reads both in every pass, which keeps the error within
1e-4 of the float32 path's; the bfloat16-only storage and the residual in the final
pass alone are timed as variants with their own error excess.

One step = one full rank-k randomized SVD (test-matrix draw, the four passes,
every orthonormalisation, the small SVD and the lift) through the C ABI with
A resident in HBM.  `value` is milliseconds per rank-k SVD (lower is better);
with N GPUs each rank runs its own replica and value = elapsed / (N * steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the float64 CPU oracle on the host cores instead (the
reference arm); under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rank-k rSVD ms & HBM roofline frac, BF16-TC vs FP32 GPU at matched error"
WORKLOAD = ("c2: A = U diag(j^-1.5) V^T, 16384 x 16384, Haar U,V (float32 QR of seeded "
            "Gaussians), A stored as bf16 hi + bf16 lo and read in full by every pass; "
            "k=100, p=10, q=1 (4 passes over A)")
PASS_KERNEL_SRC = [os.path.join(ROOT, "paper_0909_4061_gb300", "csrc", f)
                   for f in ("k_sketch_tc.cu", "tc_ptx.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sketch_tc_pass_c2.md")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# ----------------------------------------------------------------------------
# distributed plumbing (replicas: no collective on the data path)
# ----------------------------------------------------------------------------


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(backend: str, local_rank: int):
    import torch
    import torch.distributed as dist

    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and not dist.is_initialized():
        kw = {}
        if backend == "nccl":
            kw["device_id"] = torch.device("cuda", local_rank)
        dist.init_process_group(backend=backend, **kw)
    return dist.is_initialized()


def barrier():
    import torch.distributed as dist

    if dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float) -> float:
    """Largest value of x over all ranks (the slowest replica sets the job time)."""
    import torch
    import torch.distributed as dist

    if not dist.is_initialized():
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_unit(max_elapsed_ms: float, steps: int, world: int) -> float:
    """Whole-job time per rank-k SVD: `world` replicas each ran `steps` SVDs in the max elapsed time."""
    return max_elapsed_ms / (steps * world)


# ----------------------------------------------------------------------------
# clocks, peaks, ncu traffic
# ----------------------------------------------------------------------------


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, power = [], [], []
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
                power.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "last ~0.5 s of warm-up load + the timed region"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return dict(FALLBACK_PEAKS)


def file_sha(paths) -> str:
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch of the pass kernel from the committed ncu summary, or None
    when the summary is missing or was taken on a different version of the kernel."""
    try:
        with open(TRAFFIC_FILE) as f:
            text = f.read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            key, _, v = line.strip()[2:].partition(":")
            vals[key.strip()] = v.strip().strip("`")
    try:
        if vals.get("kernel_source_sha") != file_sha(PASS_KERNEL_SRC):
            return None
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------
# the workload
# ----------------------------------------------------------------------------


CACHE = "/tmp/rsvd_bench_c2_{seed}.pt"


def make_inputs(rank: int, pkg, cached: bool = False):
    """The C2 matrix: float32, its bfloat16 copy, and its bfloat16 hi + lo split (2m x n).
    With `cached` (the profile runs), the split is kept in /tmp so that the same command
    under ncu -- where torch's dense linear algebra library cannot be loaded -- reads it
    instead of rebuilding the matrix."""
    import torch

    import synth

    w = synth.C2
    seed = w.matrix_seed + 7919 * rank
    path = CACHE.format(seed=seed)
    if cached and os.path.exists(path):
        Ahl = torch.load(path, map_location="cuda")
        return w, None, Ahl[: w.m], Ahl
    A = synth.device_lowrank(w.m, w.n, w.sigma(), seed)
    Ab = A.to(torch.bfloat16)
    Ahl = pkg.split_bf16(A)
    torch.cuda.synchronize()
    if cached:
        torch.save(Ahl, path)
    return w, A, Ab, Ahl


def bench_config(w, world: int) -> dict:
    """The `config` object of both arms (the same workload, so the same dict)."""
    return {"workload": WORKLOAD, "m": w.m, "n": w.n, "k": w.k, "p": w.p, "q": w.q,
            "precision": "bf16 tensor cores on A stored as bf16 hi + bf16 lo (every pass "
                         "reads both: about 16 significant bits), f32 accumulate, f32 "
                         "re-orthonormalisation",
            "l2": "A is 1.07 GB as hi + lo (> 129 MB L2); no flush needed between steps",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def pass_bytes(m: int, n: int, l: int, a_copies: int = 1) -> int:
    """Bytes one pass Y = A X over an m x n A moves at minimum: A as bfloat16 (a_copies
    times: 2 for hi + lo), the bfloat16 operand (n x l_p) and the float32 output (m x l_p),
    with l_p = l rounded up to 16 (the tile width of the pass)."""
    lp = -(-l // 16) * 16
    return a_copies * 2 * m * n + 2 * n * lp + 4 * m * lp


def oracle_errors(res, ref, k: int) -> dict:
    """Error of a rank-k result (U, S, V) against the float64 oracle's (same A, same Omega):
    singular values relative to sigma_1, and each singular vector's distance (after sign
    alignment) times its spectral gap over sigma_1 -- the size of the perturbation that
    Wedin's theorem would need to explain it."""
    import numpy as np

    u, s, v = (np.asarray(x, dtype=np.float64) for x in res)
    ur, sr, vr, s_next = ref
    gaps = np.empty(k)
    for j in range(k):
        g = sr[j - 1] - sr[j] if j > 0 else np.inf
        g = min(g, (sr[j] - sr[j + 1]) if j + 1 < k else (sr[j] - s_next))
        gaps[j] = g
    d = np.sign(np.sum(u * ur, axis=0))
    d[d == 0] = 1.0
    du = np.linalg.norm(u * d - ur, axis=0)
    dv = np.linalg.norm(v * d - vr, axis=0)
    return {"max_abs_sigma_err_over_sigma1": float(np.max(np.abs(s - sr)) / sr[0]),
            "max_gap_scaled_u_err_over_sigma1": float(np.max(du * gaps) / sr[0]),
            "max_gap_scaled_v_err_over_sigma1": float(np.max(dv * gaps) / sr[0])}


def recon_error(A, U, S, V) -> float:
    """||A - U diag(S) V^T||_F in float64 (on the device)."""
    import torch

    R = A.double()
    R.addmm_(U.double() * S.double(), V.double().T, alpha=-1.0)
    return float(torch.linalg.norm(R).item())


def time_steps(pkg, plan, A, U, S, V, steps: int, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(steps):
        pkg.rsvd_svd(plan.handle, A, U, S, V)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1)


def cpu_baseline(A, w, budget_s: float = 12.0):
    """The float64 oracle on the host cores (bounded number of full rank-k SVDs)."""
    import numpy as np

    from oracle import philox, rsvd64

    a64 = A.cpu().numpy().astype(np.float64)
    om = philox.gaussian(w.omega_seed, philox.STREAM_OMEGA, w.n, w.l)
    times = []
    t_start = time.perf_counter()
    while not times or (time.perf_counter() - t_start < budget_s and len(times) < 5):
        t0 = time.perf_counter()
        u, s, v, _ = rsvd64.rsvd(a64, w.k + w.p, 0, w.q, om)     # untruncated: sigma_{k+1} too
        times.append((time.perf_counter() - t0) * 1e3)
    k = w.k
    r = a64 - (u[:, :k] * s[:k]) @ v[:, :k].T
    e_f = float(np.sqrt(np.sum(r * r)))
    base = {"value": statistics.median(times), "unit": "ms", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{len(times)} full rank-{w.k} SVDs of the same 16384x16384 A in float64 "
                      "(numpy/LAPACK, default BLAS threads), median"}
    return base, (u[:, :k], s[:k], v[:, :k], s[k]), e_f


def run_ours(args):
    import torch

    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    dist_init("nccl", local_rank)
    import __graft_entry__

    __graft_entry__.build()
    import paper_0909_4061_gb300 as pkg

    w, A, Ab, Ahl = make_inputs(rank, pkg, cached=args.profile_run)
    stream = torch.cuda.current_stream()
    dev = Ab.device
    U = torch.empty(w.m, w.k, device=dev)
    S = torch.empty(w.k, device=dev)
    V = torch.empty(w.n, w.k, device=dev)
    out = {}

    # The headline configuration is the one at matched error: A stored as bf16 hi + bf16 lo
    # and every pass reading both (about 16 significant bits of A); the bf16-only storage
    # and the residual in the final pass alone are timed below as variants.
    with pkg.Plan(w.m, w.n, w.k, w.p, w.q, w.omega_seed, pkg.RSVD_BF16_TC, dtype=pkg.RSVD_BF16X2,
                  residual_passes=1, host_f32=1) as pl:
        for _ in range(max(args.warmup, 3)):
            pkg.rsvd_svd(pl.handle, Ahl, U, S, V)
        if pkg.rsvd_sync(pl.handle) != pkg.RSVD_OK:
            raise RuntimeError("device error during warm-up")
        clocks = ClockSampler(local_rank)
        clocks.start()
        t_end = time.perf_counter() + (0.0 if args.profile_run else 0.5)
        while time.perf_counter() < t_end:       # keep the GPU loaded while sampling starts
            pkg.rsvd_svd(pl.handle, Ahl, U, S, V)
            torch.cuda.synchronize()
        # timed region: graph replays of the whole SVD (launch counters on, no per-step events)
        pkg.rsvd_profile(pl.handle, 0)
        elapsed = time_steps(pkg, pl, Ahl, U, S, V, args.steps, stream)
        clk = clocks.stop()
        _, launches = pkg.rsvd_profile_read(pl.handle)
        status = pkg.rsvd_sync(pl.handle)
        if status != pkg.RSVD_OK:
            raise RuntimeError(f"device status {pkg.status_string(status)}")
        # the same K steps again with a CUDA event pair around every pass over A, on the
        # plan's stream (direct launches: events cannot sit inside a replayed graph)
        pkg.rsvd_profile(pl.handle, 1 << pkg.RSVD_STEP_PASS)
        elapsed_ev = time_steps(pkg, pl, Ahl, U, S, V, args.steps, stream)
        pass_ms, pass_launches = pkg.rsvd_profile_read(pl.handle)
        pkg.rsvd_profile(pl.handle, 0)
        e_main = recon_error(A, U, S, V) if A is not None else float("nan")
        s_main = S.double().cpu()
        res_main = (U.double().cpu().numpy(), S.double().cpu().numpy(), V.double().cpu().numpy())
        # per-step breakdown (diagnostic, separate short loop, every step kind timed)
        pkg.rsvd_profile(pl.handle, (1 << pkg.RSVD_NUM_STEPS) - 1)
        for _ in range(5):
            pkg.rsvd_svd(pl.handle, Ahl, U, S, V)
        stage_ms, _ = pkg.rsvd_profile_read(pl.handle)
        pkg.rsvd_profile(pl.handle, 0)
        out["stages_ms_per_svd"] = {k: round(v / 5, 4) for k, v in stage_ms.items()}
        out["jacobi_sweeps_max"] = pkg.rsvd_diagnostics(pl.handle)[1]
        # end to end through the host-buffer entry point
        # (the caller's float32 A is copied in and split into hi + lo on the device by the
        # library -- the host_f32 option -- inside the timed region)
        e2e = None
        if not args.no_e2e and A is not None:
            a_host = A.cpu().pin_memory()
            uh = torch.empty(w.m, w.k).pin_memory()
            sh = torch.empty(w.k).pin_memory()
            vh = torch.empty(w.n, w.k).pin_memory()
            pkg.rsvd_svd_host(pl.handle, a_host, uh, sh, vh)
            k_e2e = max(3, min(args.steps, 10))
            barrier()
            t0 = time.perf_counter()
            for _ in range(k_e2e):
                pkg.rsvd_svd_host(pl.handle, a_host, uh, sh, vh)
            t_e2e = max_over_ranks((time.perf_counter() - t0) * 1e3)
            e2e = {"value": job_ms_per_unit(t_e2e, k_e2e, world), "unit": "ms",
                   "h2d_bytes_per_step": int(w.m * w.n * 4),
                   "d2h_bytes_per_step": int((w.m * w.k + w.k + w.n * w.k) * 4),
                   "steps": k_e2e,
                   "api": "rsvd_svd_host with host_f32 = 1: float32 A from pinned host memory, "
                          "split into bf16 hi + lo on the device, U/S/V back to pinned host memory"}

    # variants: bf16 storage only (every pass reads bf16(A)); hi + lo storage with only the
    # final pass B^T = A^T Q reading the residual; hi + lo with the residual in the passes
    # that make the final bases
    variants = {}
    if A is not None and not args.profile_run:
        for name, kw, Ain, desc in (
                ("bf16_only", {}, Ab, "A as bf16; every pass reads bf16(A)"),
                ("residual_final_pass_only", {"dtype": pkg.RSVD_BF16X2}, Ahl,
                 "A as bf16 hi + bf16 lo (A - hi); Stage A reads hi, the final pass both"),
                ("residual_final_bases", {"dtype": pkg.RSVD_BF16X2, "residual_passes": 2}, Ahl,
                 "A as bf16 hi + bf16 lo (A - hi); the passes whose samples become final bases "
                 "(the last of Stage A and the final pass) read both, the earlier ones hi")):
            with pkg.Plan(w.m, w.n, w.k, w.p, w.q, w.omega_seed, pkg.RSVD_BF16_TC, **kw) as plx:
                for _ in range(max(args.warmup, 3)):
                    pkg.rsvd_svd(plx.handle, Ain, U, S, V)
                kx = max(3, min(args.steps, 20))
                elx = time_steps(pkg, plx, Ain, U, S, V, kx, stream)
                if pkg.rsvd_sync(plx.handle) != pkg.RSVD_OK:
                    raise RuntimeError(f"device error on the {name} variant")
                variants[name] = {"ms": round(elx / kx, 4), "steps": kx,
                                  "recon_err": recon_error(A, U, S, V), "storage": desc}

    # the plain FP32 CUDA-core path on the float32 A, same Omega seed
    k32 = 0
    el32, e_f32, s_f32, res_f32 = float("nan"), float("nan"), s_main, None
    if not args.profile_run:
        with pkg.Plan(w.m, w.n, w.k, w.p, w.q, w.omega_seed, pkg.RSVD_PLAIN_FP32) as pl32:
            pkg.rsvd_svd(pl32.handle, A, U, S, V)
            k32 = max(3, min(args.steps, 10))
            el32 = time_steps(pkg, pl32, A, U, S, V, k32, stream)
            if pkg.rsvd_sync(pl32.handle) != pkg.RSVD_OK:
                raise RuntimeError("device error on the FP32 path")
            e_f32 = recon_error(A, U, S, V)
            s_f32 = S.double().cpu()
            res_f32 = (U.double().cpu().numpy(), S.double().cpu().numpy(), V.double().cpu().numpy())

    elapsed_max = max_over_ranks(elapsed)
    ms_step = elapsed_max / args.steps
    value = job_ms_per_unit(elapsed_max, args.steps, world)
    peaks = measured_peaks()
    n_pass = pass_launches["pass"]
    avg_pass_ms = pass_ms["pass"] / max(n_pass, 1)
    # the pass's algorithmic bytes: A once as bfloat16 + the bf16 operand + the f32 output
    # (the headline kernel reads A as hi + lo, twice those bytes of A: reported beside)
    bytes_per_pass = pass_bytes(w.m, w.n, w.l)
    bytes_moved = pass_bytes(w.m, w.n, w.l, a_copies=2)
    achieved = bytes_per_pass / (avg_pass_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded Haar factors on the device; the paper's datasets are not used)",
        "config": bench_config(w, world),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                     "traffic": ncu_traffic(),
                     "kernel": "sketch_tc_kernel (one pass over A read as hi + lo)",
                     "bytes_per_launch": bytes_per_pass,
                     "bytes_definition": "2mn (A as bf16) + 2 n l_p (operand) + 4 m l_p (output)",
                     "bytes_moved_per_launch": bytes_moved,
                     "frac_of_bytes_moved": round(bytes_moved / (avg_pass_ms * 1e-3) / 1e9
                                                  / peaks["hbm_gbs"], 4),
                     "traffic_note": "DRAM bytes per launch of the hi + lo kernel (ncu): about "
                                     "bytes_moved_per_launch, twice the algorithmic bytes of A "
                                     "because every pass also reads the residual lo",
                     "avg_launch_ms": round(avg_pass_ms, 5),
                     "peak_source": peaks["source"],
                     "timing": f"CUDA events around each of the {n_pass} pass launches of a second "
                               f"{args.steps}-step loop on the plan stream (direct launches, "
                               f"{elapsed_ev / args.steps:.4f} ms/step)"},
        "gpu_launches": int(sum(launches.values())),
        "clocks": clk,
        "fp32_path": {"ms": round(el32 / max(k32, 1), 4), "steps": k32,
                      "speedup_bf16_tc": round((el32 / max(k32, 1)) / ms_step, 3)},
        "accuracy": {"recon_err": e_main, "recon_err_fp32": e_f32,
                     "rel_excess": (e_main - e_f32) / e_f32 if e_f32 == e_f32 else None,
                     "target_rel_excess": 1e-4,
                     "max_sigma_diff_vs_fp32_over_sigma1":
                         float(((s_main - s_f32).abs().max() / s_f32[0]).item())},
    }
    for name, v in variants.items():
        v["rel_excess"] = (v["recon_err"] - e_f32) / e_f32 if e_f32 == e_f32 else None
        line[name] = v
    line.update(out)
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu:
        base, ref, e_oracle = cpu_baseline(A, w)
        line["cpu_baseline"] = base
        acc = {"oracle": "float64 Algorithm 4.4 + 5.1 on the float32 A with the same Omega",
               "recon_err_oracle": e_oracle,
               "headline": oracle_errors(res_main, ref, w.k)}
        acc["headline"]["rel_recon_excess"] = (e_main - e_oracle) / e_oracle
        if res_f32 is not None:
            acc["fp32_path"] = oracle_errors(res_f32, ref, w.k)
            acc["fp32_path"]["rel_recon_excess"] = (e_f32 - e_oracle) / e_oracle
        line["error_vs_fp64_oracle"] = acc
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_pass_probe(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_0909_4061_gb300 as pkg

    m, n, k, p = 8192, 16384, 100, 10
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    X = torch.randn(n, k + p, device="cuda")
    Y = torch.empty(m, k + p, device="cuda")
    if args.pass_probe_bf16:
        # A as bf16 alone (the kernel of the bf16-only storage and of the C3/C4/C5 passes;
        # 16384 x 16384, 537 MB)
        m = 16384
        A = torch.randn(m, n, generator=gen, device="cuda").to(torch.bfloat16)
        Y = torch.empty(m, k + p, device="cuda")
        kw = {}
    else:
        # A as bf16 hi + bf16 lo, every pass reading both: the passes of the bench's headline
        A = pkg.split_bf16(torch.randn(m, n, generator=gen, device="cuda"))
        kw = {"dtype": pkg.RSVD_BF16X2, "residual_passes": 1}
    with pkg.Plan(m, n, k, p, 1, 1, pkg.RSVD_BF16_TC, **kw) as pl:
        for trans in (0, 1):
            for _ in range(3):
                if trans:
                    pkg.rsvd_sketch(pl.handle, A, 1, Y, X)
                else:
                    pkg.rsvd_sketch(pl.handle, A, 0, X, Y)
        if pkg.rsvd_sync(pl.handle) != pkg.RSVD_OK:
            raise RuntimeError("device error in the pass probe")
    print(json.dumps({"pass_probe": "ok", "m": m, "n": n, "l": k + p,
                      "storage": "bf16" if args.pass_probe_bf16 else "bf16 hi + lo"}))


def run_small_probe(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_0909_4061_gb300 as pkg

    m = n = 8192
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    # decaying spectrum without a QR: Gaussian times a graded diagonal
    A = (torch.randn(m, n, generator=gen, device="cuda")
         * torch.arange(1, n + 1, device="cuda").pow(-1.5)).to(torch.bfloat16)
    with pkg.Plan(m, n, 100, 10, 1, 3, pkg.RSVD_BF16_TC) as pl:
        for _ in range(2):
            pl.svd(A)
        bits, sweeps = pkg.rsvd_diagnostics(pl.handle)
    print(json.dumps({"small_probe": "ok", "m": m, "n": n, "l": 110, "jacobi_sweeps": sweeps}))


def _events_ms(fn, steps, warmup):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _rel_err(A, U, S, V):
    """||A - U diag(S) V^T||_F / ||A||_F in float64, by 16384-row blocks (on the device)."""
    import torch

    num, den = 0.0, 0.0
    for r0 in range(0, A.shape[0], 16384):
        a = A[r0:r0 + 16384].double()
        den += float((a * a).sum())
        a.addmm_(U[r0:r0 + 16384].double() * S.double(), V.double().T, alpha=-1.0)
        num += float((a * a).sum())
    return (num / den) ** 0.5


# Table 7.1 of the paper (seconds on its 2009 desktop, double precision, one execution):
# the gauss (Algorithm 4.1, Gaussian Omega, then Algorithm 5.1) and srft (Algorithm 4.1
# with the modified SRFT, then Algorithm 5.2) columns, by n and l.  Context only.
PAPER_TABLE_7_1_S = {
    1024: {10: (5.63e-2, 9.06e-2), 20: (9.69e-2, 1.03e-1), 40: (1.84e-1, 1.27e-1),
           80: (4.00e-1, 2.19e-1), 160: (9.92e-1, 6.92e-1)},
    2048: {10: (2.16e-1, 3.56e-1), 20: (3.69e-1, 3.89e-1), 40: (6.69e-1, 4.33e-1),
           80: (1.43e0, 6.64e-1), 160: (3.36e0, 1.61e0)},
    4096: {10: (8.94e-1, 1.45e0), 20: (1.44e0, 1.53e0), 40: (2.64e0, 1.63e0),
           80: (5.43e0, 2.08e0), 160: (1.16e1, 3.94e0)},
}


def run_table_7_1(pkg, steps, warmup):
    """The timing experiment of Section 7.4 on this GPU: the l leading singular triplets
    of an n x n Gaussian matrix (k = l, p = 0, q = 0), gauss = Gaussian Omega + Algorithm
    5.1 (rsvd_svd), srft = the modified SRFT + Algorithm 5.2 (rsvd_svd_row_extraction),
    each on the float32 path and the bfloat16 tensor-core path.  The library takes
    l <= 256: the table's l = 320, 640, 1280 rows are outside it; l = 256 is added."""
    import torch

    rows = []
    g = torch.Generator(device="cuda")
    for n in (1024, 2048, 4096):
        g.manual_seed(7100 + n)
        A32 = torch.randn(n, n, device="cuda", generator=g)
        Ab = A32.to(torch.bfloat16)
        nrm = float(torch.linalg.matrix_norm(A32.double()))
        for l in (10, 20, 40, 80, 160, 256):
            row = {"n": n, "l": l}
            for prec, A in ((pkg.RSVD_PLAIN_FP32, A32), (pkg.RSVD_BF16_TC, Ab)):
                tag = "fp32" if prec == pkg.RSVD_PLAIN_FP32 else "bf16_tc"
                for method, tm in (("gauss", pkg.RSVD_GAUSSIAN), ("srft", pkg.RSVD_GSRFT)):
                    with pkg.Plan(n, n, l, 0, 0, 7200 + l, prec, test_matrix=tm) as pl:
                        U = torch.empty(n, l, device="cuda")
                        S = torch.empty(l, device="cuda")
                        V = torch.empty(n, l, device="cuda")
                        fn = ((lambda: pkg.rsvd_svd(pl.handle, A, U, S, V)) if method == "gauss" else
                              (lambda: pkg.rsvd_svd_row_extraction(pl.handle, A, U, S, V)))
                        ms = _events_ms(fn, steps, warmup)
                        pkg._check(pkg.rsvd_sync(pl.handle), "table 7.1 run")
                        if tag == "bf16_tc":
                            pkg.rsvd_profile(pl.handle, (1 << pkg.RSVD_NUM_STEPS) - 1)
                            fn()
                            torch.cuda.synchronize()
                            stage_ms, _ = pkg.rsvd_profile_read(pl.handle)
                            pkg.rsvd_profile(pl.handle, 0)
                            row[f"{method}_{tag}_stages_ms"] = {k2: round(v, 3) for k2, v in stage_ms.items() if v > 0}
                        err = float(torch.linalg.matrix_norm(A32.double() - (U.double() * S.double()) @ V.double().T))
                    row[f"{method}_{tag}_ms"] = round(ms, 4)
                    row[f"{method}_{tag}_rel_err_F"] = round(err / nrm, 5)
            paper = PAPER_TABLE_7_1_S.get(n, {}).get(l)
            if paper:
                row["paper_gauss_s"], row["paper_srft_s"] = paper
            rows.append(row)
        del A32, Ab
    return {"metric": "l leading singular triplets of an n x n Gaussian matrix, ms per execution",
            "config": {"k": "l", "p": 0, "q": 0, "matrix": "iid N(0, 1), seeded on the device"},
            "results": rows}


def _spec_norm(apply, n, iters=30, seed=5):
    """Largest eigenvalue of the symmetric positive semidefinite operator x -> apply(x) (n
    columns in), by power iteration on the device in float32."""
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    x = torch.randn(n, 1, generator=g, device="cuda")
    s = 0.0
    for _ in range(iters):
        y = apply(x)
        s = float(torch.linalg.vector_norm(y))
        x = y / max(s, 1e-30)
    return s


def run_algorithms(pkg, steps, warmup):
    """The paper's other algorithms at the C2 size (16384 x 16384, bfloat16 A, sigma_j = j^-1.5):
    the adaptive range finder (Algorithm 4.2 blocked, eps = 0.1 ||A||, blocks of 16), the
    Hermitian Stage B (Algorithms 5.3 and 5.5 on the psd A = V diag(j^-1.5) V^T), and Stage B
    by row extraction (Algorithm 5.2) beside Algorithm 5.1 on the same basis; per call the
    passes over A and the bytes of A they read (2mn each) over the time."""
    import numpy as np
    import torch

    import synth

    w = synth.C2
    n = w.m
    out = {}
    A32 = synth.device_lowrank(n, n, w.sigma(), w.matrix_seed)
    Ab = A32.to(torch.bfloat16)
    a_bytes = 2.0 * n * n
    # adaptive range finder
    eps, block, cap = 0.2 * float(w.sigma()[0]), 16, 128
    with pkg.Plan(n, n, 112, 16, 0, w.omega_seed, pkg.RSVD_BF16_TC) as pl:
        Q = torch.zeros(n, cap, device="cuda")
        res = {}
        ms = _events_ms(lambda: res.update(r=pkg.rsvd_range_finder_adaptive(pl.handle, Ab, eps, block, Q, cap)),
                        steps, warmup)
        rank, est = res["r"]
        passes = rank // block + 1
        qk = Q[:, :rank]
        # ||(I - Q Q^T) A||_2 = sqrt(lambda_max(A^T (I - Q Q^T) A))
        err = _spec_norm(lambda x: A32.T @ (lambda y: y - qk @ (qk.T @ y))(A32 @ x), n) ** 0.5
    out["adaptive_range_finder"] = {
        "ms": round(ms, 4), "eps": eps, "block": block, "rank": rank, "estimate": est,
        "error_spectral": round(err, 6), "guarantee_met": err <= eps, "passes_over_A": passes,
        "A_bytes_per_ms": round(passes * a_bytes / ms / 1e6, 1),
        "note": "the stopping test reads one float per block on the host (it steers the loop)"}
    # Hermitian Stage B
    g = torch.Generator(device="cuda")
    g.manual_seed(w.matrix_seed + 7)
    V = synth.device_haar(n, 1024, g, "cuda")
    lam = torch.as_tensor(w.sigma()[:1024].astype(np.float32), device="cuda")
    S32 = (V * lam) @ V.T
    S32 = 0.5 * (S32 + S32.T)
    Sb = S32.to(torch.bfloat16)
    del V
    for name, method in (("eig_direct", pkg.RSVD_EIG_DIRECT), ("eig_nystrom", pkg.RSVD_EIG_NYSTROM)):
        with pkg.Plan(n, n, w.k, w.p, w.q, w.omega_seed, pkg.RSVD_BF16_TC) as pl:
            U = torch.zeros(n, w.k, device="cuda")
            L = torch.zeros(w.k, device="cuda")
            ms = _events_ms(lambda: pkg.rsvd_eig(pl.handle, Sb, method, U, L), steps, warmup)
            pkg._check(pkg.rsvd_sync(pl.handle), name)
        e = float(torch.linalg.matrix_norm(S32.double() - (U.double() * L.double()) @ U.double().T))
        passes = 2 * w.q + 2
        out[name] = {"ms": round(ms, 4), "rel_err_F": round(e / float(torch.linalg.matrix_norm(S32.double())), 6),
                     "lambda_1": round(float(L[0]), 6), "passes_over_A": passes,
                     "A_bytes_per_ms": round(passes * a_bytes / ms / 1e6, 1)}
    del S32, Sb
    # row extraction beside Algorithm 5.1
    for name, fn, passes in (("svd_alg_5_1", pkg.rsvd_svd, 2 * w.q + 2),
                             ("svd_row_extraction_alg_5_2", pkg.rsvd_svd_row_extraction, 2 * w.q + 1)):
        with pkg.Plan(n, n, w.k, w.p, w.q, w.omega_seed, pkg.RSVD_BF16_TC) as pl:
            U = torch.zeros(n, w.k, device="cuda")
            S = torch.zeros(w.k, device="cuda")
            Vv = torch.zeros(n, w.k, device="cuda")
            ms = _events_ms(lambda: fn(pl.handle, Ab, U, S, Vv), steps, warmup)
            pkg._check(pkg.rsvd_sync(pl.handle), name)
            pkg.rsvd_profile(pl.handle, (1 << pkg.RSVD_NUM_STEPS) - 1)
            fn(pl.handle, Ab, U, S, Vv)
            torch.cuda.synchronize()
            stage_ms, _ = pkg.rsvd_profile_read(pl.handle)
            pkg.rsvd_profile(pl.handle, 0)
        out[name] = {"ms": round(ms, 4), "rel_err_vs_fp32_A": round(_rel_err(A32, U, S, Vv), 6),
                     "passes_over_A": passes, "stages_ms": {k2: round(v, 4) for k2, v in stage_ms.items() if v > 0}}
    return {"metric": "the paper's other algorithms at 16384 x 16384 (bf16 tensor cores), ms per call",
            "config": {"m": n, "n": n, "k": w.k, "p": w.p, "q": w.q, "spectrum": "j^-1.5"},
            "results": out}


def run_workload(args):
    """Secondary workloads (one JSON line each; not the headline metric):
    c3 -- 262144 x 4096, single-pass (Section 5.5) vs q = 2 multi-pass, k = 64, p = 16;
    c4 -- 32768 x 32768, SRFT (Section 4.6) vs Gaussian test matrix, k = 236, p = 20, q = 1;
    c5 -- 512 matrices m ~ U[128, 2048], n ~ U[64, 1024], batched forward and backward;
    t71 -- the Section 7.4 timing sweep (Table 7.1) with gauss and the modified SRFT;
    algos -- the adaptive range finder, Hermitian Stage B and row extraction at 16384^2."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_0909_4061_gb300 as pkg
    import synth

    torch.cuda.set_device(0)
    steps, warmup = max(args.steps, 1), max(args.warmup, 3)
    out = {"workload": args.workload, "unit": "ms", "steps": steps, "warmup": warmup,
           "data": "synthetic (seeded Haar factors on the device)", "higher_is_better": False}
    cache = f"/tmp/rsvd_bench_{args.workload}.pt"
    if args.workload in ("c3", "c4"):
        w = synth.C3 if args.workload == "c3" else synth.C4
        noise = 1e-4 if args.workload == "c3" else 0.0
        if args.profile_run and os.path.exists(cache):
            A = torch.load(cache, map_location="cuda")   # ncu cannot load torch's dense linear algebra
        else:
            A = synth.device_lowrank(w.m, w.n, w.sigma(), w.matrix_seed, noise_std=noise)
            if args.profile_run:
                torch.save(A, cache)
        Ab = A.to(torch.bfloat16)
        torch.cuda.synchronize()
        variants = ([("single_pass", dict(single_pass=1, q=0)), ("multi_pass_q2", dict(q=2))]
                    if args.workload == "c3" else
                    [("srft", dict(test_matrix=pkg.RSVD_SRFT, q=w.q)),
                     ("srft_row_transform", dict(test_matrix=pkg.RSVD_SRFT, srft_fft=1, q=w.q)),
                     ("gaussian", dict(q=w.q))])
        res = {}
        for name, kw in variants:
            q = kw.pop("q")
            torch.cuda.synchronize()
            t_plan = time.perf_counter()
            pl = pkg.Plan(w.m, w.n, w.k, w.p, q, w.omega_seed, pkg.RSVD_BF16_TC, **kw)
            pkg.rsvd_sync(pl.handle)
            plan_ms = (time.perf_counter() - t_plan) * 1e3
            with pl:
                U = torch.empty(w.m, w.k, device="cuda")
                S = torch.empty(w.k, device="cuda")
                V = torch.empty(w.n, w.k, device="cuda")
                ms = _events_ms(lambda: pkg.rsvd_svd(pl.handle, Ab, U, S, V), steps, warmup)
                pkg.rsvd_sync(pl.handle)
                pkg.rsvd_profile(pl.handle, (1 << pkg.RSVD_NUM_STEPS) - 1)
                pkg.rsvd_svd(pl.handle, Ab, U, S, V)
                torch.cuda.synchronize()
                stage_ms, _ = pkg.rsvd_profile_read(pl.handle)
                pkg.rsvd_profile(pl.handle, 0)
                res[name] = {"ms": round(ms, 4), "rel_err_vs_fp32_A": round(_rel_err(A, U, S, V), 6),
                             "plan_create_ms": round(plan_ms, 3),
                             "jacobi_sweeps_max": pkg.rsvd_diagnostics(pl.handle)[1],
                             "passes_over_A": (2 if kw.get("single_pass") else 2 * q + 2),
                             "stages_ms": {k2: round(v, 4) for k2, v in stage_ms.items()}}
        out.update({"metric": "rank-k rSVD ms per matrix (bf16 tensor cores)",
                    "config": {"m": w.m, "n": w.n, "k": w.k, "p": w.p}, "results": res})
    elif args.workload == "t71":
        out.update(run_table_7_1(pkg, steps, warmup))
    elif args.workload == "algos":
        out.update(run_algorithms(pkg, steps, warmup))
    elif args.workload == "c5":
        shapes = synth.c5_shapes()
        if args.profile_run and os.path.exists(cache):
            mats = [t.cuda() for t in torch.load(cache)]
        else:
            mats = []
            for b, (m, n) in enumerate(shapes):
                a = synth.device_lowrank(m, n, synth.spectrum_exp(min(m, n), 4.0),
                                         synth.C5_MATRIX_SEED * 100003 + b)
                lda = -(-n // 8) * 8
                t = torch.zeros(m, lda, dtype=torch.bfloat16, device="cuda")
                t[:, :n] = a.to(torch.bfloat16)
                mats.append(t)
            if args.profile_run:
                torch.save([t.cpu() for t in mats], cache)
        torch.cuda.synchronize()
        with pkg.BatchedPlan(shapes, synth.C5_K, synth.C5_P, synth.C5_Q, seed=synth.C5_OMEGA_SEED) as pl:
            U, S, V = pl.svd(mats)
            grads = pl.backward(mats)
            fwd = _events_ms(lambda: pl.svd(mats, U, S, V), steps, warmup)
            bwd = _events_ms(lambda: pl.backward(mats, grads), steps, warmup)
            sweeps = pl.sync()
            tuning = pl.tuning()
        elems = sum(m * n for m, n in shapes)
        out.update({"metric": "batched rank-16 rSVD forward / backward ms for the whole batch",
                    "config": {"batch": len(shapes), "k": synth.C5_K, "p": synth.C5_P, "q": synth.C5_Q,
                               "elements": elems},
                    "results": {"forward_ms": round(fwd, 4), "backward_ms": round(bwd, 4),
                                "forward_A_bytes_per_ms": round(elems * 2 * 4 / fwd / 1e6, 1),
                                "jacobi_sweeps_max": sweeps,
                                "pass_config": tuning,
                                "launch": "one CUDA graph per call (forward, backward)"}})
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import synth
    from oracle import philox, rsvd64

    w = synth.C2
    try:
        import torch

        if torch.cuda.is_available():
            a64 = synth.device_lowrank(w.m, w.n, w.sigma(), w.matrix_seed).cpu().numpy().astype(np.float64)
        else:
            raise RuntimeError
    except Exception:
        a64, *_ = synth.lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    om = philox.gaussian(w.omega_seed, philox.STREAM_OMEGA, w.n, w.l)
    for _ in range(args.warmup):
        rsvd64.rsvd(a64, w.k, w.p, w.q, om)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rsvd64.rsvd(a64, w.k, w.p, w.q, om)
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    sample = f"{args.steps} full rank-{w.k} SVDs of the 16384x16384 A in float64 (numpy/LAPACK)"
    line = {"impl": "reference", "metric": METRIC, "value": round(ms, 3), "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(w, world),
            "cpu_baseline": {"value": round(ms, 3), "unit": "ms", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(ms, 3), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-run", action="store_true",
                    help="timed pipeline only (no clock-load loop, e2e, FP32 leg or CPU baseline): "
                         "the command the ncu launch list is taken on")
    ap.add_argument("--small-probe", action="store_true",
                    help="two rank-100 SVDs (l = 110) of an 8192 x 8192 bf16 matrix: the small case "
                         "for full ncu captures of the orthonormalisation and small-SVD kernels")
    ap.add_argument("--pass-probe-bf16", action="store_true",
                    help="with --pass-probe: A stored as bf16 alone, 16384 x 16384 (537 MB)")
    ap.add_argument("--pass-probe", action="store_true",
                    help="three launches of the tensor-core pass kernel (each mode) on an 8192 x 16384 "
                         "A stored as bf16 hi + lo (537 MB, larger than L2): the small case for "
                         "full ncu captures")
    ap.add_argument("--workload", choices=("c2", "c3", "c4", "c5", "t71", "algos"), default="c2",
                    help="c2 (default) is the headline line; c3/c4/c5 print one secondary line "
                         "each; t71 is the timing experiment of Section 7.4 (Table 7.1); algos "
                         "times the adaptive range finder, the Hermitian Stage B and row extraction")
    args = ap.parse_args()
    if args.workload != "c2" and args.impl == "ours":
        run_workload(args)
        return
    if args.pass_probe:
        run_pass_probe(args)
        return
    if args.small_probe:
        run_small_probe(args)
        return
    if args.profile_run:
        args.no_e2e = args.no_cpu = True
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
