"""Benchmark of the sigma_min grid engine on one GB300 (or N replicas).

One step = one full-grid evaluation of sigma_min(zI - A) and its eight
epsilon masks for the mid-size workload: a random non-normal banded Toeplitz
matrix (n = 2000, kl = 2, ku = 5, complex coefficients Re, Im ~ N(0,1), seed 0,
superdiagonals scaled by 4) on a 512 x 512 grid over the bounding box of its
symbol curve widened by 20 %, eps = 1e-1 ... 1e-8, Lanczos to convergence
(tol 1e-13). Inputs are synthetic and seeded.

Printed JSON line (rank 0): points/s of the whole job, the roofline of the
dominant kernel (FP64-ALU bound; algorithmic flops / CUDA-event time), the
end-to-end rate through the public API with host buffers, the CPU oracle on a
bounded sample, the restricted-versus-full-grid time on the 5 x 5-dilated
sensitive zone (paper Sec. 4), and the SM clocks seen during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 it runs under torch.distributed.run, one process per GPU;
each rank evaluates the full workload on its own GPU (replicas: the method has
no exchange step) and the timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2605_04550_gb300 import inputs  # noqa: E402

METRIC = "σ_min grid points/s (FP64); restricted vs full-grid time at ≥99% sensitive recall"
UNIT = "grid points/s"
N, KL, KU, SEED, NX, NY = 2000, 2, 5, 0, 512, 512
EPS = inputs.EPS_LEVELS_8
EPS_RESTRICT = 1e-2
TOL, KMAX = 1e-13, 1000
WORKLOAD = (f"random banded Toeplitz n={N} kl={KL} ku={KU} (complex N(0,1) coefficients, seed {SEED}, "
            f"superdiagonals x4), {NX}x{NY} grid over the symbol-curve bounding box +20%, "
            f"8 eps levels 1e-1..1e-8, Lanczos to convergence (tol {TOL:g})")
# nominal FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) per Lanczos row-step of k_sigma_min<2,5>: ncu's
# dram__bytes_read.sum + dram__bytes_write.sum of one main-pass launch of this workload
# itself (--case grid2000, application replay: 9.99 TB for 1.83e10 row-steps). Factor
# rows and Lanczos vectors are streamed once per sweep, so traffic scales with row-steps.
DRAM_BYTES_PER_ROW_STEP = 546.0


# the classifiers trained by `bench.py --workload restriction --save-model ...`
MODEL_PATHS = {net: os.path.join(ROOT, "paper_2605_04550_gb300", "data", f"restriction_{net}.npz")
               for net in ("mlp", "dual")}

# reduced case for profiler captures: same matrix family, n = 256, 384 x 384 grid
# (about 2.5 waves of points in flight), k_max 300 -> about 3.5 GB of workspace
SMALL = dict(n=256, nx=384, ny=384, kmax=300)


def workload(case: str = "mid"):
    if case == "grcar100":  # the first workload: Grcar n = 100 on its 100 x 100 grid
        bands, kl, ku = inputs.grcar(100)
        return bands, kl, ku, inputs.grcar_grid_100()
    n, nx, ny = (N, NX, NY) if case in ("mid", "grid2000") else (SMALL["n"], SMALL["nx"], SMALL["ny"])
    bands, kl, ku, a = inputs.random_toeplitz(n, KL, KU, seed=SEED)
    grid = inputs.toeplitz_symbol_grid(a, kl, ku, nx, ny)
    return bands, kl, ku, grid


def algorithmic_flops(steps: np.ndarray, n: int, kl: int, ku: int) -> float:
    """n (8 kl (kl+ku) + 6 kl + 8) per banded LU + n (16 (2kl+ku) + 30) per Lanczos step."""
    steps = np.asarray(steps, dtype=np.float64)
    lu = n * (8 * kl * (kl + ku) + 6 * kl + 8)
    per_step = n * (16 * (2 * kl + ku) + 30)
    return float(steps.size * lu + steps.sum() * per_step)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over the ranks of the process group (the job's time is the
    slowest replica's); the value itself when no group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = device if (device is not None and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world_size: int, units_per_rank_step: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput of replicas: every rank does the same units per step;
    the job takes the slowest rank's time."""
    return world_size * units_per_rank_step * steps / (max_ms * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(bands, kl, ku, grid, seconds: float = 12.0, seed: int = 1):
    """The CPU oracle (as it stands, OpenMP over points, all host cores) on random
    points of the same grid with the library's stopping settings, until `seconds`."""
    import oracle
    z = oracle.grid_points(grid).ravel()
    rng = np.random.default_rng(seed)
    order = rng.permutation(z.size)
    done, t0, batch = 0, time.perf_counter(), 256
    while True:
        sel = order[done:done + batch]
        oracle.sigma_min_banded(bands, kl, ku, z[sel], k_min=2, k_max=KMAX, tol=TOL)
        done += sel.size
        el = time.perf_counter() - t0
        if el >= seconds or done >= z.size:
            break
        batch = min(4096, batch * 2)
    cores = os.cpu_count() or 1
    return {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} uniformly random points of the {NX}x{NY} grid (same matrix, tol {TOL:g}, "
                      f"k_max {KMAX}), {el:.1f} s on {cores} host threads (OpenMP)"}


def oracle_one_thread_rate(bands, kl, ku, grid, seconds: float = 6.0, seed: int = 3):
    """The CPU oracle on ONE host thread (the paper's protocol, Sec. 5.1) on random
    points of the same grid with the library's stopping settings, until `seconds`."""
    import oracle
    z = oracle.grid_points(grid).ravel()
    order = np.random.default_rng(seed).permutation(z.size)
    done, t0, batch = 0, time.perf_counter(), 16
    while True:
        sel = order[done:done + batch]
        oracle.sigma_min_banded(bands, kl, ku, z[sel], k_min=2, k_max=KMAX, tol=TOL, nthreads=1)
        done += sel.size
        el = time.perf_counter() - t0
        if el >= seconds or done >= z.size:
            break
        batch = min(256, batch * 2)
    return {"value": done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} uniformly random points of the {NX}x{NY} grid, {el:.1f} s on one host thread"}


# The paper's own method on its own class (Sec. 5.1, Table main_results): a dense SVD
# per point of a 100 x 100 grid over [-4, 4]^2 for an n = 64 matrix, on one CPU thread.
# Run in a child process whose BLAS/OpenMP pools are limited to one thread.
_DENSE_SVD_LEG = r"""
import json, sys, time, numpy as np
sys.path.insert(0, ROOT_DIR)
import oracle
from paper_2605_04550_gb300 import inputs
bands, kl, ku, A = inputs.paper_class(0)
grid = inputs.paper_grid_100()
z = oracle.grid_points(grid).ravel()
oracle.sigma_min_dense(A, z[:50])
t0 = time.perf_counter()
s = oracle.sigma_min_dense(A, z)
el = time.perf_counter() - t0
print(json.dumps({"seconds": el, "points": int(z.size), "beta": int(kl),
                  "sensitive_fraction": float(np.mean(s <= 0.01))}))
"""


def paper_method_baselines(psa, dev, opts):
    """Dense SVD on the paper class (one host thread) beside the library on the same grid,
    and the paper's reported time for that method."""
    import torch
    from paper_2605_04550_gb300 import inputs
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _DENSE_SVD_LEG.replace("ROOT_DIR", repr(ROOT))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    dense = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else {"error": r.stderr[-300:]}
    bands, kl, ku, _ = inputs.paper_class(0)
    grid = inputs.paper_grid_100()
    b = torch.as_tensor(bands, device=dev)
    psa.sigma_min(b, kl, ku, grid, eps=(0.01,), opts=opts)
    torch.cuda.synchronize(dev)
    e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    e[0].record()
    for _ in range(5):
        psa.sigma_min(b, kl, ku, grid, eps=(0.01,), opts=opts)
    e[1].record()
    torch.cuda.synchronize(dev)
    gpu_s = e[0].elapsed_time(e[1]) / 5 / 1e3
    out = {"workload": "paper class (Sec. 3.3): n = 64 real banded {-1,0,1} matrix, seed 0, 100x100 grid on "
                       "[-4,4]^2, eps 0.01",
           "paper_dense_svd_s_per_grid": 3.73, "paper_hardware": "one CPU thread, model unstated (Sec. 5.1)",
           "gpu_s_per_grid": gpu_s, "gpu_points_per_s": grid.npoints / gpu_s}
    if "seconds" in dense:
        out.update({"dense_svd_s_per_grid": dense["seconds"], "dense_svd_points_per_s": dense["points"] / dense["seconds"],
                    "dense_svd_cores": 1, "beta": dense["beta"], "gpu_vs_dense_svd": dense["seconds"] / gpu_s})
    else:
        out["dense_svd_error"] = dense["error"]
    return out


def grcar_fixed_step_baseline(psa, dev):
    """The first workload: Grcar n = 100 on its 100 x 100 grid with 20-step inverse Lanczos
    (the workload's own setting) and to convergence, both timed on the GPU, and the
    20-step error against the converged tier."""
    import torch
    from paper_2605_04550_gb300 import inputs
    bands, kl, ku = inputs.grcar(100)
    grid = inputs.grcar_grid_100()
    b = torch.as_tensor(bands, device=dev)
    res = {}
    for name, o in (("fixed20", psa.LanczosOpts.fixed(20)), ("converged", psa.LanczosOpts())):
        out = psa.sigma_min(b, kl, ku, grid, eps=EPS, opts=o)
        torch.cuda.synchronize(dev)
        e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        e[0].record()
        for _ in range(10):
            psa.sigma_min(b, kl, ku, grid, eps=EPS, opts=o, out=out)
        e[1].record()
        torch.cuda.synchronize(dev)
        res[name] = (e[0].elapsed_time(e[1]) / 10, out.sigma.cpu().numpy().ravel(),
                     out.mask.cpu().numpy().view(np.uint32).ravel(), out.steps.cpu().numpy().ravel())
    (t20, s20, m20, _), (tc, sc, mc, kc) = res["fixed20"], res["converged"]
    well = sc > 1e-8 * np.abs(sc).max()
    rel = np.abs(s20 - sc)[well] / sc[well]
    return {"workload": "Grcar n = 100, 100x100 grid over [-1,3]x[-3.5,3.5], eps 1e-1..1e-8",
            "fixed20_points_per_s": grid.npoints / (t20 * 1e-3), "fixed20_ms": t20,
            "converged_points_per_s": grid.npoints / (tc * 1e-3), "converged_ms": tc,
            "converged_mean_steps": float(kc.mean()),
            "fixed20_max_rel_err_vs_converged": float(rel.max()),
            "fixed20_median_rel_err_vs_converged": float(np.median(rel)),
            "fixed20_mask_points_differing": int(np.sum(m20 != mc))}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    bands, kl, ku, grid = workload()
    import oracle
    oracle.build()
    z = oracle.grid_points(grid).ravel()
    rng = np.random.default_rng(7)
    per_step = 512
    order = rng.permutation(z.size)
    for w in range(args.warmup):
        oracle.sigma_min_banded(bands, kl, ku, z[order[:64]], k_min=2, k_max=KMAX, tol=TOL)
    t0 = time.perf_counter()
    for s in range(args.steps):
        sel = order[(s * per_step) % z.size:][:per_step]
        oracle.sigma_min_banded(bands, kl, ku, z[sel], k_min=2, k_max=KMAX, tol=TOL)
    el = time.perf_counter() - t0
    value = args.steps * per_step / el
    cores = os.cpu_count() or 1
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_step": per_step,
                   "note": "CPU oracle (banded LU + inverse Lanczos in C, OpenMP); each step a random "
                           f"{per_step}-point sample of the grid"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} x {per_step} random grid points"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def dilate(mask2d: np.ndarray, k: int) -> np.ndarray:
    """Binary dilation with a k x k square (paper Sec. 3.6 / Sec. 4: 5 x 5 for R, 3 x 3 for truth)."""
    r = k // 2
    m = np.pad(mask2d, r)
    out = np.zeros_like(mask2d)
    for di in range(k):
        for dj in range(k):
            out |= m[di:di + mask2d.shape[0], dj:dj + mask2d.shape[1]]
    return out


def run_gpu(args):
    import torch
    import paper_2605_04550_gb300 as psa

    ws_, rank, local = dist_env()
    if ws_ > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bands, kl, ku, grid = workload(args.case)
    n = bands.shape[1]
    npts = grid.npoints
    b_dev = torch.as_tensor(bands, device=dev)
    opts = psa.LanczosOpts(k_min=2, k_max=SMALL["kmax"] if args.case == "small" else KMAX, tol=TOL, seed=0)
    pif = psa.default_points_in_flight(n, kl, ku, npts)
    wsp = psa.Workspace(n, kl, ku, pif, opts, device=dev, npoints=npts)
    out = psa.sigma_min(b_dev, kl, ku, grid, eps=EPS, opts=opts, workspace=wsp)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def barrier():
        if ws_ > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        psa.sigma_min(b_dev, kl, ku, grid, eps=EPS, opts=opts, workspace=wsp, out=out)
    torch.cuda.synchronize(dev)

    # ---------------- timed region: K full-grid steps, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for s in range(args.steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            psa.sigma_min(b_dev, kl, ku, grid, eps=EPS, opts=opts, workspace=wsp, out=out)
            ev[s][1].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_ms = max_over_ranks(float(np.sum(step_ms)), dev)
    value = job_rate(ws_, npts, args.steps, dev_ms)

    steps = out.steps.cpu().numpy().ravel()
    status = out.status.cpu().numpy().ravel()
    sig = out.sigma.cpu().numpy()
    mask = out.mask.cpu().numpy().view(np.uint32)
    flops = algorithmic_flops(steps, n, kl, ku)
    mean_ms = dev_ms / args.steps if ws_ == 1 else float(np.mean(step_ms))
    achieved = flops / (mean_ms * 1e-3) / 1e12
    # lanes busy inside a warp: a warp holds an 8 x 4 tile of the grid and runs
    # until its slowest point stops
    k2 = steps.reshape(grid.ny, grid.nx)
    ty, tx = -(-grid.ny // 4), -(-grid.nx // 8)
    kp = np.zeros((ty * 4, tx * 8), dtype=np.int64)
    kp[:grid.ny, :grid.nx] = k2
    tiles = kp.reshape(ty, 4, tx, 8).transpose(0, 2, 1, 3).reshape(-1, 32)
    lane_util = float(tiles.sum() / (tiles.max(axis=1).sum() * 32))

    if args.case != "mid":
        if rank == 0:
            print(json.dumps({"case": args.case, "n": n, "points": npts, "ms_per_step": mean_ms,
                              "points_per_s": npts / (mean_ms * 1e-3), "achieved_tflops": achieved,
                              "mean_lanczos_steps": float(steps.mean()), "lane_utilisation": lane_util}),
                  flush=True)
        return 0

    # ---------------- end to end through the public API with host buffers
    pinned_b = torch.as_tensor(bands).pin_memory()
    h_sigma = torch.empty((grid.ny, grid.nx), dtype=torch.float64).pin_memory()
    h_mask = torch.empty((grid.ny, grid.nx), dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        bd = pinned_b.to(dev, non_blocking=True)
        o2 = psa.sigma_min(bd, kl, ku, grid, eps=EPS, opts=opts, workspace=wsp)
        h_sigma.copy_(o2.sigma, non_blocking=True)
        h_mask.copy_(o2.mask, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": npts / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(bands.nbytes),
           "d2h_bytes_per_step": int(h_sigma.numel() * 8 + h_mask.numel() * 4)}

    # ---------------- restricted (paper Sec. 4) vs full grid, region = 5x5-dilated S_eps
    lvl = EPS.index(EPS_RESTRICT)
    s_true = ((mask >> lvl) & 1).astype(bool)
    region = dilate(s_true, 5)
    idx = torch.as_tensor(psa.tile_order(np.flatnonzero(region.ravel()), grid.nx), device=dev)
    psa.sigma_min(b_dev, kl, ku, grid, eps=EPS, idx=idx, opts=opts, workspace=wsp)
    torch.cuda.synchronize(dev)
    r_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    flush.fill_(-1.0)
    r_ev[0].record(stream)
    out_r = psa.sigma_min(b_dev, kl, ku, grid, eps=EPS, idx=idx, opts=opts, workspace=wsp)
    r_ev[1].record(stream)
    torch.cuda.synchronize(dev)
    r_ms = r_ev[0].elapsed_time(r_ev[1])
    mask_r = out_r.mask.cpu().numpy().view(np.uint32)
    s_pred = ((mask_r >> lvl) & 1).astype(bool)
    truth_d = dilate(s_true, 3)
    recall = float((truth_d & region).sum() / max(truth_d.sum(), 1))
    coverage = float((s_true & s_pred).sum() / max(s_true.sum(), 1))
    same = bool(np.array_equal(out_r.sigma.cpu().numpy()[region], sig[region]))
    restricted = {"eps": EPS_RESTRICT, "region": "5x5 dilation of the full-grid sensitive zone",
                  "grid_fraction": float(region.mean()), "recall_dilated_truth": recall,
                  "coverage": coverage, "full_ms": mean_ms, "restricted_ms": r_ms,
                  "speedup": mean_ms / r_ms if r_ms > 0 else None, "sigma_bitwise_equal_on_region": same}

    # ---------------- the same with the learned classifiers' regions (trained weights shipped
    # with the package: bench.py --workload restriction --save-model ...): the MLP and the
    # paper's dual-path network
    restricted_learned = {}
    from paper_2605_04550_gb300 import restriction as rst
    for net, path in MODEL_PATHS.items():
        if not os.path.exists(path):
            continue
        model = rst.Restriction.load(path, dev)
        # one untimed pass loads every kernel and library routine the path uses
        ctx = rst.matrix_contexts([(b_dev, kl, ku)], model.eps)[0]
        model.restricted(ctx, grid, EPS, opts=opts, workspace=wsp)
        flush.fill_(-2.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx = rst.matrix_contexts([(b_dev, kl, ku)], model.eps)[0]
        torch.cuda.synchronize(dev)
        feat_ms = (time.perf_counter() - t0) * 1e3
        out_l, mask_l, idx_l, tm = model.restricted(ctx, grid, EPS, opts=opts, workspace=wsp)
        m_l = mask_l.cpu().numpy().astype(bool)
        met = rst.recall_metrics(sig <= model.eps, m_l)
        hyb = feat_ms + tm["nn_ms"] + tm["restricted_ms"]
        cal = model.calibration
        restricted_learned[net] = {
            "eps": model.eps, "tau": model.tau, "paper_rule_tau": cal.get("paper_rule_tau"),
            "validation_min_recall": cal.get("row", {}).get("min_recall"),
            "model": os.path.relpath(path, ROOT), "features_ms": feat_ms, "nn_ms": tm["nn_ms"],
            "restricted_ms": tm["restricted_ms"], "full_ms": mean_ms, "speedup_actual": mean_ms / hyb,
            "speedup_best": mean_ms / tm["restricted_ms"], "region_points": int(idx_l.numel()), **met,
            "sigma_bitwise_equal_on_region": bool(np.array_equal(out_l.sigma.cpu().numpy()[m_l], sig[m_l]))}

    probe = psa.probe_dfma_rate(4096)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_step": npts, "points_in_flight": pif,
                   "workspace_gb": wsp.nbytes / 1e9,
                   "l2": "L2 flushed (256 MB write) between timed steps; per-step workspace (factors, "
                         "Lanczos vectors) of tens of GB also exceeds L2",
                   "parallelism": "replicas" if ws_ > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": DRAM_BYTES_PER_ROW_STEP * float(steps.sum()) * n,
                     "traffic_source": "ncu dram bytes per Lanczos row-step of one main-pass launch of this "
                                       "workload (bench.py --case grid2000), scaled by this launch's row-steps",
                     "peak_source": "FP64 from unit counts and clocks: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                     "peak_probe_tflops": 2 * probe / 1e12,
                     "frac_of_probe": achieved / (2 * probe / 1e12),
                     "algorithmic_flops_per_launch": flops,
                     "kernel": "k_sigma_min<2,5> main pass (events also cover its estimate pass and four set-up kernels)"},
        "cpu_baseline": None,
        "e2e": e2e,
        "gpu_launches": 6 * args.steps,
        "clocks": clk.summary(),
        "mean_lanczos_steps": float(steps.mean()),
        "max_lanczos_steps": int(steps.max()),
        "lane_utilisation": lane_util,
        "status_counts": {str(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))},
        "restricted": restricted,
        "restricted_learned": restricted_learned,
        "wall_s_timed": wall,
    }
    if rank == 0:
        line["grcar100"] = grcar_fixed_step_baseline(psa, dev)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(bands, kl, ku, grid, seconds=args.cpu_seconds)
        line["cpu_baseline_one_thread"] = oracle_one_thread_rate(bands, kl, ku, grid)
        line["paper_method"] = paper_method_baselines(psa, dev, opts)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws_ > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_differentiation(args):
    """Adjoint workload: Grcar-type n = 4000 (kl = 1, ku = 3) with N(0, 1e-2) band noise;
    ~1e5 grid points with d sigma / dz and the band gradient (unit weights), a
    central-difference check (h = 1e-6) at sampled points, and Newton refinement of
    the eps = 1e-4 contour along grid rows."""
    import torch
    import paper_2605_04550_gb300 as psa
    from paper_2605_04550_gb300 import contour
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    b, kl, ku = inputs.grcar_perturbed(4000, seed=0)
    grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 320, 313)
    bt = torch.as_tensor(b, device=dev)
    xs = grid.re_min + np.arange(grid.nx) * ((grid.re_max - grid.re_min) / (grid.nx - 1))
    ys = grid.im_min + np.arange(grid.ny) * ((grid.im_max - grid.im_min) / (grid.ny - 1))
    # the points in 8 x 4 tile order: a warp's 32 points are a compact patch of the grid with
    # similar Lanczos step counts (9 % faster than row-major order on this workload)
    order = psa.tile_order(np.arange(grid.npoints), grid.nx).astype(np.int64)
    z = torch.as_tensor((xs[None, :] + 1j * ys[:, None]).ravel()[order], device=dev)
    w = torch.ones(z.numel(), dtype=torch.float64, device=dev)
    opts = psa.LanczosOpts()
    for _ in range(args.warmup):
        r = psa.sigma_min_grad(bt, kl, ku, z, weight=w, opts=opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        r = psa.sigma_min_grad(bt, kl, ku, z, weight=w, opts=opts)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    sig = r.sigma.cpu().numpy()
    st = r.status.cpu().numpy()
    steps = r.steps.cpu().numpy()
    sig_grid = np.empty_like(sig)
    sig_grid[order] = sig
    n = b.shape[1]
    two_pass = 2 * algorithmic_flops(steps, n, kl, ku) - steps.size * n * (8 * kl * (kl + ku) + 6 * kl + 8)
    # central differences at resolvable sampled points
    rng = np.random.default_rng(0)
    cand = np.flatnonzero(sig > 1e-3)
    pick = rng.choice(cand, min(64, cand.size), replace=False)
    zc = z.cpu().numpy()[pick]
    h = 1e-6
    tight = psa.LanczosOpts(tol=1e-15, k_max=4000)
    zz = torch.as_tensor(np.concatenate([zc, zc + h, zc - h, zc + 1j * h, zc - 1j * h]), device=dev)
    rf = psa.sigma_min_grad(bt, kl, ku, zz, opts=tight)
    sf = rf.sigma.cpu().numpy().reshape(5, -1)
    fd = (sf[1] - sf[2]) / (2 * h) + 1j * (sf[3] - sf[4]) / (2 * h)
    gz = rf.grad_z.cpu().numpy()[: pick.size]
    fd_err = float(np.max(np.abs(gz - fd) / np.abs(fd)))
    # Newton refinement of the eps = 1e-4 contour along grid rows
    t0 = time.perf_counter()
    ref = contour.refine_rows(bt, kl, ku, grid, sig_grid.reshape(grid.ny, grid.nx), 1e-4)
    newton_s = time.perf_counter() - t0
    npts = z.numel()
    line = {"workload": "differentiation", "metric": "sigma_min + adjoint gradient points/s (FP64)",
            "value": npts / (ms * 1e-3), "unit": "grid points/s", "ms_per_step": ms, "steps": args.steps,
            "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Grcar-type n=4000 kl=1 ku=3, band entries + N(0,1e-2) (seed 0), "
                                   f"{grid.nx}x{grid.ny} grid over [-1,3]x[-3.5,3.5] (points in 8x4 tile order), "
                                   "grad_z and band gradient (unit weights), Lanczos tol 1e-13"},
            "mean_lanczos_steps": float(steps.mean()), "max_lanczos_steps": int(steps.max()),
            "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                         "achieved_two_pass": two_pass / (ms * 1e-3) / 1e12,
                         "frac_two_pass": two_pass / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "flops": "banded LU + 2 x (Lanczos steps) x n x (16 (2 kl + ku) + 30): the forward pass "
                                  "and the replay that forms the Ritz vector"},
            "status_counts": {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
            "fd_check": {"points": int(pick.size), "h": h, "max_rel_err": fd_err},
            "newton_contour": {"eps": 1e-4, "crossings": int(ref.x.size), "converged": int(ref.converged.sum()),
                               "gpu_calls": ref.iterations, "max_rel_residual": float(ref.residual.max()),
                               "seconds": newton_s}}
    print(json.dumps(line), flush=True)
    return 0


def run_grad_case(args):
    """Small case for profiler captures of the gradient kernel: sigma_min on a grid and then
    sigma_min_grad (with unit weights) on the same points in tile order, one call each.
    Grcar-type n = 300 + N(0, 1e-2) band noise (seed 0), 200 x 200 grid over
    [-1, 3] x [-3.5, 3.5]; about 3 GB of workspace, freed between the two calls."""
    import torch
    import paper_2605_04550_gb300 as psa
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    b, kl, ku = inputs.grcar_perturbed(300, seed=0)
    grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 200, 200)
    n, N = b.shape[1], grid.npoints
    bt = torch.as_tensor(b, device=dev)
    xs = grid.re_min + np.arange(grid.nx) * ((grid.re_max - grid.re_min) / (grid.nx - 1))
    ys = grid.im_min + np.arange(grid.ny) * ((grid.im_max - grid.im_min) / (grid.ny - 1))
    order = psa.tile_order(np.arange(N), grid.nx).astype(np.int64)
    z = torch.as_tensor((xs[None, :] + 1j * ys[:, None]).ravel()[order], device=dev)
    w = torch.ones(N, dtype=torch.float64, device=dev)
    opts = psa.LanczosOpts()
    pif = psa.default_points_in_flight(n, kl, ku, N)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ws = psa.Workspace(n, kl, ku, pif, opts, device=dev, npoints=N)
    e[0].record()
    o = psa.sigma_min(bt, kl, ku, grid, opts=opts, workspace=ws)
    e[1].record()
    torch.cuda.synchronize(dev)
    del ws
    torch.cuda.empty_cache()
    gws = psa.GradWorkspace(n, kl, ku, pif, opts, device=dev)
    e[2].record()
    r = psa.sigma_min_grad(bt, kl, ku, z, weight=w, opts=opts, workspace=gws)
    e[3].record()
    torch.cuda.synchronize(dev)
    print(json.dumps({"case": "grad300", "n": n, "points": N, "sigma_min_ms": e[0].elapsed_time(e[1]),
                      "sigma_min_grad_ms": e[2].elapsed_time(e[3]), "mean_lanczos_steps": float(o.steps.float().mean()),
                      "grad_mean_lanczos_steps": float(r.steps.float().mean())}), flush=True)
    return 0


def run_fp64_probe(args):
    """The FP64 unit's rates (psa_probe_fp64): DFMA against warps per SM, dependent chains
    and active lanes, and DADD, DMUL, division and square root at full occupancy. Rates
    are lane-operations per clock per SM at the sampled SM clock."""
    import ctypes
    import torch
    from paper_2605_04550_gb300 import _native
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lib = _native.load()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    st = torch.cuda.current_stream(dev).cuda_stream
    names = ["dfma", "dadd", "dmul", "div", "sqrt"]
    cases = [(0, w, 32, c) for w in (1, 2, 4, 8, 16) for c in (1, 8)]
    cases += [(0, w, 1, 8) for w in (4, 16)] + [(0, 4, 1, 1)]
    cases += [(op, 16, 32, 8) for op in (1, 2, 3, 4)]
    rows = []
    with ClockSampler(0) as clk:
        for op, w, a, c in cases:
            # about 2e9 lane-operations at 32 active lanes (a few ms at the peak); the same
            # iterations with one active lane
            iters = max(64, int(2e9 / (sms * w * 32 * c)) // (8 if op >= 3 else 1))
            r = ctypes.c_double(0.0)
            _native.check(lib.psa_probe_fp64(op, w, a, c, iters, ctypes.byref(r), st), "psa_probe_fp64")
            rows.append({"op": names[op], "warps_per_sm": w, "active_lanes": a, "chains": c,
                         "lane_ops_per_s": r.value})
    mhz = clk.summary().get("sm_mhz") or 2070.0
    for row in rows:
        row["lane_ops_per_clock_per_sm"] = row["lane_ops_per_s"] / (sms * mhz * 1e6)
        # warp instructions per clock per SM: what an instruction costs whatever its active lanes
        row["warp_inst_per_clock_per_sm"] = row["lane_ops_per_clock_per_sm"] / row["active_lanes"]
    print(json.dumps({"case": "fp64probe", "sms": sms, "clocks": clk.summary(), "rows": rows}), flush=True)
    return 0


def run_batched(args):
    """Batch workload: 256 seeded matrices (n log-uniform in [200, 8000], kl 1..4, ku 1..8,
    Grcar-type or random Toeplitz with 1e-3 band noise), each on its own 128 x 128 grid,
    8 eps levels, Lanczos to convergence. Launch controls from the autotuner (timed on
    every 32nd matrix of the batch); the timed step is one replay of the CUDA graph
    that holds the whole batch."""
    import torch
    import paper_2605_04550_gb300 as psa
    from paper_2605_04550_gb300 import batch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = inputs.batch_workload(args.batch_size)
    mats = [(torch.as_tensor(b, device=dev), kl, ku, g) for b, kl, ku, g, _ in w]
    plan = batch.BatchPlan(mats)
    opts = psa.LanczosOpts(k_min=2, k_max=KMAX, tol=TOL, seed=0)
    ws = batch.BatchWorkspace(plan, opts)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    t0 = time.perf_counter()
    if args.no_tune:
        best, tune = batch.BatchConfig(streams=args.batch_streams), {}
    else:
        sub = batch.BatchPlan(mats[::32]) if len(mats) >= 64 else plan
        cands = [batch.BatchConfig(0, order, streams) for streams in (2, 4, 8)
                 for order in (batch.ORDER_AUTO, batch.ORDER_ESTIMATE)]
        best, tune = batch.autotune(sub, EPS, opts, candidates=cands, workspace=ws)
    tune_s = time.perf_counter() - t0
    g = batch.BatchGraph(plan, EPS, opts, best, workspace=ws)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        for s_ in range(args.steps):
            flush.fill_(float(s_))
            ev[s_][0].record(stream)
            g.replay()
            ev[s_][1].record(stream)
        torch.cuda.synchronize(dev)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    mean_ms = float(np.mean(step_ms))
    npts = plan.npoints
    steps = g.out.steps.cpu().numpy()
    status = g.out.status.cpu().numpy()
    flops = 0.0
    for (b, kl, ku, grid, _), o in zip(w, plan.offsets):
        flops += algorithmic_flops(steps[o:o + grid.npoints], b.shape[1], kl, ku)
    achieved = flops / (mean_ms * 1e-3) / 1e12

    # end to end: bands from pinned host memory into the plan's device tensors, the
    # graph, sigma and masks back to pinned host memory
    e2e = None
    pinned = [] if args.no_e2e else [torch.as_tensor(b).pin_memory() for b, *_ in w]
    h_sigma = torch.empty(npts, dtype=torch.float64).pin_memory()
    h_mask = torch.empty(npts, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize(dev)
    if not args.no_e2e:
        t1 = time.perf_counter()
        for hb, (db, *_r) in zip(pinned, mats):
            db.copy_(hb, non_blocking=True)
        out = g.replay()
        h_sigma.copy_(out.sigma, non_blocking=True)
        h_mask.copy_(out.mask, non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t1
        e2e = {"value": npts / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(sum(b.nbytes for b, *_ in w)),
               "d2h_bytes_per_step": int(npts * 12)}
    ns = np.array([b.shape[1] for b, *_ in w])
    line = {"workload": "batched", "metric": METRIC, "value": npts / (mean_ms * 1e-3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{len(w)} seeded banded matrices, n log-uniform in [200, 8000], kl 1..4, "
                                   "ku 1..8, Grcar-type or random Toeplitz + 1e-3 complex band noise, each on its "
                                   "own 128x128 grid over its symbol box +20%, 8 eps levels, Lanczos tol 1e-13",
                       "matrices": len(w), "classes": len(plan.classes()), "points_per_step": npts,
                       "n_min": int(ns.min()), "n_max": int(ns.max()), "n_mean": float(ns.mean()),
                       "workspace_gb": ws.nbytes / 1e9,
                       "autotuned": {"points_in_flight": best.points_in_flight, "order": best.order,
                                     "streams": best.streams,
                                     "candidates_ms": {f"pif{c.points_in_flight}/order{c.order}/streams{c.streams}": t
                                                       for c, t in tune.items()},
                                     "tune_seconds": tune_s, "tuned_on": "every 32nd matrix of the batch"},
                       "l2": "L2 flushed (256 MB write) between timed steps",
                       "graph": "whole batch captured in one CUDA graph, one replay per step"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "algorithmic_flops_per_step": flops,
                         "kernel": "k_sigma_min<kl,ku> over all classes (events cover the whole replay)"},
            "e2e": e2e, "clocks": clk.summary(),
            "mean_lanczos_steps": float(steps.mean()),
            "status_counts": {str(k): int(v) for k, v in zip(*np.unique(status, return_counts=True))}}
    print(json.dumps(line), flush=True)
    return 0


def _worst_matrix_report(model, va, vg, truth, vctx):
    """Where the calibrated region misses sensitive points of the validation matrix with
    the smallest recall: its shape and family, and the sigma and probability there."""
    import torch
    from paper_2605_04550_gb300 import restriction
    w = model.calibration["worst_matrix"]
    b, kl, ku, g, kind = va[w]
    p = model.predict(vctx[w], g)
    r = restriction.region_mask(p.reshape(-1).contiguous(), g, model.tau).cpu().numpy().astype(bool)
    t = truth[w] <= model.eps
    miss = restriction.dilate_np(t, 1) & ~r
    pf = model.predict(vctx[w], g, hierarchical=False).cpu().numpy()
    return {"index": w, "n": int(b.shape[1]), "kl": kl, "ku": ku, "kind": kind,
            "recall": model.calibration["per_matrix_recall"][w], "sensitive_points": int(t.sum()),
            "missed_dilated_points": int(miss.sum()), "missed_truly_sensitive": int((t & ~r).sum()),
            "max_prob_at_missed": float(pf[miss].max()) if miss.any() else None,
            "missed_in_hierarchy_only": int((miss & (pf >= model.tau)).sum())}


def run_restriction(args):
    """Learned restriction (paper Sec. 3-4): train the classifiers (the MLP and the
    paper's dual-path network, on the same labels) on sigma_min labels of seeded
    banded matrices, calibrate their thresholds for >= 99 % recall on validation
    matrices, then compare each restricted run with the full-grid run on the test
    matrix (random banded Toeplitz + 1e-3 noise, n = 20000, kl = 3, ku = 6,
    1024 x 1024 grid over its symbol box +20 %)."""
    import torch
    import paper_2605_04550_gb300 as psa
    from paper_2605_04550_gb300 import inputs as inp, restriction
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nets = ["mlp", "dual"] if args.net == "both" else [args.net]
    eps = restriction.EPS
    t_all = time.perf_counter()
    timing = {}
    models = {}
    if args.load_models:
        for net, path in zip(nets, args.load_models.split(",")):
            models[net] = restriction.Restriction.load(path, dev)
            assert models[net].net == net, (path, models[net].net)
    else:
        # ---- training set: labels from the plain GPU method, shared by the networks
        t0 = time.perf_counter()
        tr = inp.restriction_matrices(args.restrict_train, seed=1, nx=32, ny=32)
        mats = [(torch.as_tensor(b, device=dev), kl, ku) for b, kl, ku, _, _ in tr]
        first = restriction.Restriction(dev, seed=0, net=nets[0])
        x, y, _ = first.build_training_set(mats, [g for *_, g, _ in tr], np.random.default_rng(0))
        torch.cuda.synchronize(dev)
        timing["labels_and_features"] = time.perf_counter() - t0
        timing["training_set"] = first.timing
        for net in nets:
            m = first if net == nets[0] else restriction.Restriction(dev, seed=0, net=net)
            t0 = time.perf_counter()
            m.train(x, y, np.random.default_rng(1))  # the same held-out split and batches for each network
            torch.cuda.synchronize(dev)
            timing[f"training_{net}"] = time.perf_counter() - t0
            models[net] = m
        del x, y, mats
    # ---- calibration on validation matrices (both networks, the same truth); loaded
    # classifiers keep the threshold they were shipped with
    cal, worst = {}, {}
    if args.load_models:
        for net, m in models.items():
            cal[net], worst[net] = m.calibration, None
    else:
        t0 = time.perf_counter()
        va = inp.restriction_matrices(args.restrict_val, seed=2, nx=args.restrict_val_grid, ny=args.restrict_val_grid)
        vm = [(torch.as_tensor(b, device=dev), kl, ku) for b, kl, ku, _, _ in va]
        vg = [g for *_, g, _ in va]
        vctx = restriction.matrix_contexts(vm, eps)
        plan, vs = restriction.labels_batched(vm, vg, eps, opts=psa.LanczosOpts(k_min=2, k_max=KMAX, tol=TOL))
        vs = vs.cpu().numpy()
        truth = [vs[o:o + g.npoints].reshape(g.ny, g.nx) for o, g in zip(plan.offsets, vg)]
        for net, m in models.items():
            cal[net] = m.calibrate(vctx, vg, truth)
            worst[net] = _worst_matrix_report(m, va, vg, truth, vctx)
        timing["calibration"] = time.perf_counter() - t0
        del vm, vctx, plan
        torch.cuda.empty_cache()
    # ---- test matrix: full grid vs restricted
    b, kl, ku, grid = inp.restriction_test_matrix(n=args.restrict_test_n, nx=args.restrict_grid, ny=args.restrict_grid)
    bt = torch.as_tensor(b, device=dev)
    opts = psa.LanczosOpts(k_min=2, k_max=KMAX, tol=TOL)
    pif = psa.default_points_in_flight(bt.shape[1], kl, ku, grid.npoints)
    free, _ = torch.cuda.mem_get_info(dev)
    while pif > 32 * 4 and psa.workspace_bytes(bt.shape[1], kl, ku, pif, opts, grid.npoints) > 0.75 * free:
        pif //= 2  # a large order: fewer points in flight so that the workspace fits with room to spare
    wsp = psa.Workspace(bt.shape[1], kl, ku, pif, opts, device=dev, npoints=grid.npoints)
    small = inp.Grid(grid.re_min, grid.re_max, grid.im_min, grid.im_max, 64, 64)
    psa.sigma_min(bt, kl, ku, small, eps=EPS, opts=opts, workspace=wsp)  # warm-up: modules and workspace
    ctx = restriction.matrix_contexts([(bt, kl, ku)], eps)[0]
    for m in models.values():
        m.restricted(ctx, small, EPS, opts=opts, workspace=wsp)
    torch.cuda.synchronize(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush.fill_(1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_net = {}
    with ClockSampler(0) as clk:
        e0.record()
        full = psa.sigma_min(bt, kl, ku, grid, eps=EPS, opts=opts, workspace=wsp)
        e1.record()
        torch.cuda.synchronize(dev)
        full_ms = e0.elapsed_time(e1)
        s_full = full.sigma.cpu().numpy()
        for net, model in models.items():
            flush.fill_(2.0)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            fctx = restriction.matrix_contexts([(bt, kl, ku)], eps)[0]
            torch.cuda.synchronize(dev)
            feat_ms = (time.perf_counter() - t0) * 1e3
            out, mask, idx, tm = model.restricted(fctx, grid, EPS, opts=opts, workspace=wsp)
            m_ = mask.cpu().numpy().astype(bool)
            hybrid_ms = feat_ms + tm["nn_ms"] + tm["restricted_ms"]
            per_net[net] = {"features_ms": feat_ms, "nn_ms": tm["nn_ms"], "restricted_ms": tm["restricted_ms"],
                            "hybrid_ms": hybrid_ms, "speedup_actual": full_ms / hybrid_ms,
                            "speedup_best": full_ms / tm["restricted_ms"], "region_points": int(idx.numel()),
                            **restriction.recall_metrics(s_full <= eps, m_),
                            "sigma_bitwise_equal_on_region": bool(np.array_equal(out.sigma.cpu().numpy()[m_],
                                                                                 s_full[m_])),
                            "hierarchical": getattr(model, "last_counts", None),
                            "tau": cal[net]["tau"], "paper_rule_tau": cal[net]["paper_rule_tau"],
                            "calibration_row": cal[net]["row"],
                            "validation_recall_min_median": [min(cal[net]["per_matrix_recall"]),
                                                             float(np.median(cal[net]["per_matrix_recall"]))],
                            "worst_validation_matrix": worst[net],
                            "trainable_parameters": (mlp_nparams("mlp") if net == "mlp" else mlp_nparams("dual"))}
            if model.history:
                per_net[net].update({"epochs": len(model.history), "final_val_loss": model.history[-1]["val_loss"],
                                     "final_val_acc": model.history[-1]["val_acc"]})
    steps = full.steps.cpu().numpy()
    flops = algorithmic_flops(steps, bt.shape[1], kl, ku)
    achieved = flops / (full_ms * 1e-3) / 1e12
    N = grid.npoints
    best = min(per_net.values(), key=lambda r: r["hybrid_ms"])
    line = {"workload": "learned restriction", "metric": METRIC, "value": N / (best["hybrid_ms"] * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": best["hybrid_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"test matrix: random banded Toeplitz + 1e-3 complex noise, n={bt.shape[1]}, "
                                   f"kl={kl}, ku={ku}, {grid.nx}x{grid.ny} grid over the symbol box +20%, "
                                   f"eps={eps}; classifiers {', '.join(nets)} (BF16 on tensor cores), "
                                   + ("loaded from " + args.load_models if args.load_models else
                                      f"trained on {args.restrict_train} matrices (n log-uniform [500, 5000], kl "
                                      f"1..4, ku 1..8, 32x32 label grids)")
                                   + f", calibrated on {args.restrict_val} matrices "
                                     f"({args.restrict_val_grid}x{args.restrict_val_grid}) for >= 99% recall",
                       "points_per_step": N, "points_in_flight": pif, "workspace_gb": wsp.nbytes / 1e9,
                       "warmup": "one 64x64 run of the same kernels (the full-grid run takes minutes)",
                       "l2": "256 MB flush before each timed run"},
            "full_grid": {"full_ms": full_ms, "points_per_s": N / (full_ms * 1e-3), "achieved_tflops": achieved,
                          "frac_of_fp64_peak": achieved / FP64_PEAK_TFLOPS, "mean_lanczos_steps": float(steps.mean()),
                          "status_counts": {str(k): int(v) for k, v in zip(*np.unique(full.status.cpu().numpy(),
                                                                                      return_counts=True))}},
            "classifiers": per_net,
            "pipeline_seconds": {**timing, "total": time.perf_counter() - t_all},
            "clocks": clk.summary(), "gpu_launches": None}
    if args.save_model:
        for net, path in zip(nets, args.save_model.split(",")):
            models[net].save(path, meta={"training_matrices": args.restrict_train,
                                         "validation_matrices": args.restrict_val,
                                         "validation_grid": args.restrict_val_grid, "seed_train": 1,
                                         "seed_val": 2, "label_tol": restriction.LABEL_OPTS.tol})
    print(json.dumps(line), flush=True)
    return 0


def _banded_eigvals(item):
    """Eigenvalues of a band (LAPACK zgeev through numpy on the dense matrix): the
    paper's own input to its spectrum features. Runs in a worker process."""
    b, kl, ku = item
    n = b.shape[1]
    A = np.zeros((n, n), dtype=np.complex128)
    for d in range(-kl, ku + 1):
        i = np.arange(max(0, -d), min(n, n - d))
        A[i, i + d] = b[d + kl, i]
    t0 = time.perf_counter()
    lam = np.linalg.eigvals(A)
    return lam, time.perf_counter() - t0


def _eigvals_pool(items, workers: int):
    """Eigenvalues of many bands on single-threaded worker processes (spawned)."""
    import multiprocessing as mp
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            out = pool.map(_banded_eigvals, items, chunksize=1)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return [o[0] for o in out], float(sum(o[1] for o in out))


def run_feature_ablation(args):
    """The paper's eigenvalue features (Sec. 3.1, Tables "matrix" and "matrixAdd"; Eq.
    (dist) over the eigenvalues) against the symbol-curve features that the library
    uses by default: the same network, labels, sampled points, training batches and
    validation truth, at orders where a dense eigensolve is affordable (n log-uniform
    in [300, 1500]); then recall and grid fraction on held-out test matrices and on
    the benchmark matrix (n = 2000, 512 x 512) at each calibrated threshold."""
    import torch
    import paper_2605_04550_gb300 as psa
    from paper_2605_04550_gb300 import inputs as inp, restriction
    workers = max(1, min(os.cpu_count() or 1, 32))
    n_min, n_max = 300, 1500
    tr = inp.restriction_matrices(args.ablation_train, seed=1, n_min=n_min, n_max=n_max, nx=32, ny=32)
    va = inp.restriction_matrices(args.restrict_val, seed=2, n_min=n_min, n_max=n_max, nx=args.restrict_val_grid,
                                  ny=args.restrict_val_grid)
    te = inp.restriction_matrices(args.restrict_val, seed=3, n_min=n_min, n_max=n_max, nx=args.restrict_val_grid,
                                  ny=args.restrict_val_grid)
    bb, bkl, bku, bgrid = workload("mid")
    t0 = time.perf_counter()
    lam_all, eig_cpu_s = _eigvals_pool([(b, kl, ku) for b, kl, ku, *_ in tr + va + te] + [(bb, bkl, bku)], workers)
    eig_wall = time.perf_counter() - t0
    lam_tr, lam_va = lam_all[:len(tr)], lam_all[len(tr):len(tr) + len(va)]
    lam_te, lam_b = lam_all[len(tr) + len(va):-1], lam_all[-1]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    eps = restriction.EPS
    opts_truth = psa.LanczosOpts(k_min=2, k_max=KMAX, tol=TOL)

    def truth_of(mats, grids):
        plan, sg = restriction.labels_batched(mats, grids, eps, opts=opts_truth)
        sg = sg.cpu().numpy()
        return [sg[o:o + g.npoints].reshape(g.ny, g.nx) for o, g in zip(plan.offsets, grids)]

    t0 = time.perf_counter()
    mats = [(torch.as_tensor(b, device=dev), kl, ku) for b, kl, ku, _, _ in tr]
    grids = [g for *_, g, _ in tr]
    vm = [(torch.as_tensor(b, device=dev), kl, ku) for b, kl, ku, _, _ in va]
    vg = [g for *_, g, _ in va]
    tm_ = [(torch.as_tensor(b, device=dev), kl, ku) for b, kl, ku, _, _ in te]
    tg = [g for *_, g, _ in te]
    vtruth, ttruth = truth_of(vm, vg), truth_of(tm_, tg)
    bt = torch.as_tensor(bb, device=dev)
    btruth = psa.sigma_min(bt, bkl, bku, bgrid, eps=(eps,), opts=opts_truth).sigma.cpu().numpy()
    truth_s = time.perf_counter() - t0
    nets = ["mlp", "dual"] if args.net == "both" else [args.net]
    labels = None
    result = {}
    for feat in ("symbol", "eigen"):
        sp = (lambda lst: lst) if feat == "eigen" else (lambda lst: None)
        for net in nets:
            m = restriction.Restriction(dev, seed=0, net=net, features=feat)
            t0 = time.perf_counter()
            x, y, _ = m.build_training_set(mats, grids, np.random.default_rng(0), spectra=sp(lam_tr), labels=labels)
            labels = m.last_labels
            m.train(x, y, np.random.default_rng(1))
            torch.cuda.synchronize(dev)
            train_s = time.perf_counter() - t0
            del x, y
            vctx = restriction.matrix_contexts(vm, eps, spectra=sp(lam_va))
            cal = m.calibrate(vctx, vg, vtruth)
            tctx = restriction.matrix_contexts(tm_, eps, spectra=sp(lam_te))
            recs, fracs, precs = [], [], []
            for c, g, s in zip(tctx, tg, ttruth):
                p = m.predict(c, g)
                r = restriction.region_mask(p.reshape(-1).contiguous(), g, m.tau).cpu().numpy().astype(bool)
                met = restriction.recall_metrics(s <= eps, r)
                recs.append(met["recall"])
                fracs.append(met["grid_fraction"])
                precs.append(met["precision"])
            bctx = restriction.matrix_contexts([(bt, bkl, bku)], eps, spectra=sp([lam_b]))[0]
            pb = m.predict(bctx, bgrid)
            rb = restriction.region_mask(pb.reshape(-1).contiguous(), bgrid, m.tau).cpu().numpy().astype(bool)
            result[f"{net}/{feat}"] = {
                "tau": m.tau, "paper_rule_tau": cal["paper_rule_tau"],
                "validation_min_recall": cal["row"]["min_recall"],
                "validation_mean_grid_fraction": cal["row"]["mean_grid_fraction"],
                "test_min_recall": float(np.min(recs)), "test_median_recall": float(np.median(recs)),
                "test_p10_recall": float(np.percentile(recs, 10)),
                "test_mean_grid_fraction": float(np.mean(fracs)), "test_mean_precision": float(np.mean(precs)),
                "test_true_sensitive_fraction": float(np.mean([(s <= eps).mean() for s in ttruth])),
                "bench_matrix": restriction.recall_metrics(btruth <= eps, rb),
                "epochs": len(m.history), "final_val_loss": m.history[-1]["val_loss"], "train_s": train_s}
    line = {"workload": "feature ablation: eigenvalue features (paper Sec. 3.1) vs symbol-curve features",
            "config": {"training": f"{len(tr)} matrices, n log-uniform [{n_min}, {n_max}], 32x32 label grids "
                                   f"(seed 1)",
                       "validation": f"{len(va)} matrices (seed 2), {args.restrict_val_grid}^2 grids",
                       "test": f"{len(te)} matrices (seed 3), {args.restrict_val_grid}^2 grids; and the benchmark "
                               f"matrix (n={N}, kl={KL}, ku={KU}, {NX}x{NY})",
                       "eps": eps, "truth": f"sigma_min to tol {TOL:g}",
                       "same": "labels, sampled points, held-out split, batches, seeds, validation truth"},
            "eigensolve": {"method": "numpy.linalg.eigvals (LAPACK zgeev) of the dense matrix, one thread per "
                                     "matrix", "workers": workers, "cpu_s": eig_cpu_s, "wall_s": eig_wall,
                           "matrices": len(lam_all)},
            "truth_s": truth_s, "results": result}
    print(json.dumps(line), flush=True)
    return 0


def mlp_nparams(net: str) -> int:
    from paper_2605_04550_gb300 import _native
    return _native.MLP_PARAMS if net == "mlp" else _native.DUAL_TRAINABLE


def run_classifier(args):
    """The classifier's tensor-core kernels: the MLP forward over the 1024 x 1024
    grid's feature rows, and one large BF16 GEMM (8192^3) for the kernel alone."""
    import torch
    from paper_2605_04550_gb300 import mlp
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    peak = float(peaks.get("bf16_tflops", 1900.0))
    g = torch.Generator(device=dev).manual_seed(0)
    rows = 1 << 20
    x = (torch.randn(rows, mlp.IN, device=dev, generator=g) * 0.5).to(torch.bfloat16)
    theta = mlp.init_theta(0, dev)
    nb = mlp.workspace_bytes(rows, False)
    buf, ptr = mlp._aligned_buffer(nb, dev)
    prob = torch.empty(rows, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        mlp.forward(theta, x, out=prob, workspace=(buf, ptr, nb))
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        mlp.forward(theta, x, out=prob, workspace=(buf, ptr, nb))
    e1.record()
    torch.cuda.synchronize(dev)
    fwd_ms = e0.elapsed_time(e1) / args.steps
    fwd_flops = 2.0 * rows * (mlp.IN * mlp.HIDDEN + 2 * mlp.HIDDEN * mlp.HIDDEN + mlp.HIDDEN)
    # the paper's dual-path network on the same rows: its fused, padded GEMMs (128 -> 256,
    # 256 -> 128, three 128 -> 128) as the tensor cores run them
    theta_d = mlp.init_theta(0, dev, "dual")
    nbd = mlp.workspace_bytes(rows, False, "dual")
    bufd, ptrd = mlp._aligned_buffer(nbd, dev)
    for _ in range(args.warmup):
        mlp.forward(theta_d, x, out=prob, workspace=(bufd, ptrd, nbd), net="dual")
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(args.steps):
        mlp.forward(theta_d, x, out=prob, workspace=(bufd, ptrd, nbd), net="dual")
    e1.record()
    torch.cuda.synchronize(dev)
    dual_ms = e0.elapsed_time(e1) / args.steps
    dual_flops = 2.0 * rows * (256 * 128 + 128 * 256 + 3 * 128 * 128 + 128)
    del bufd
    M = N = K = 8192
    A = (torch.randn(M, K, device=dev, generator=g)).to(torch.bfloat16)
    B = (torch.randn(N, K, device=dev, generator=g)).to(torch.bfloat16)
    for _ in range(args.warmup):
        C = mlp.gemm_bf16(A, B)
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(args.steps):
        C = mlp.gemm_bf16(A, B)
    e1.record()
    torch.cuda.synchronize(dev)
    gemm_ms = e0.elapsed_time(e1) / args.steps
    ref = (A[:64].float() @ B.float().T)
    err = float((C[:64] - ref).abs().max().item() / ref.abs().max().item())
    gemm_tf = 2.0 * M * N * K / (gemm_ms * 1e-3) / 1e12
    line = {"workload": "classifier", "metric": "MLP forward rows/s (BF16 tensor cores, FP32 accumulate)",
            "value": rows / (fwd_ms * 1e-3), "unit": "rows/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": fwd_ms, "higher_is_better": True, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": f"MLP {mlp_desc()} over {rows} feature rows (one 1024x1024 grid)"},
            "roofline": {"bound": "tensor", "achieved": fwd_flops / (fwd_ms * 1e-3) / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "frac": fwd_flops / (fwd_ms * 1e-3) / 1e12 / peak, "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)"},
            "dual_path": {"ms": dual_ms, "rows_per_s": rows / (dual_ms * 1e-3),
                          "tflops_padded": dual_flops / (dual_ms * 1e-3) / 1e12,
                          "trainable_parameters": mlp._native.DUAL_TRAINABLE},
            "gemm_8192": {"ms": gemm_ms, "tflops": gemm_tf, "frac_of_bf16_peak": gemm_tf / peak,
                          "max_rel_err_vs_fp32": err}}
    print(json.dumps(line), flush=True)
    return 0


def mlp_desc():
    return "128->256->256->256->1 (SiLU)"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--case", default="mid",
                    choices=["mid", "small", "grcar100", "grid2000", "grad300", "fp64probe"],
                    help="mid: the benchmark workload; small: reduced case for profiler captures; "
                         "grcar100: the Grcar n = 100 workload (small-order profile); grid2000: the "
                         "benchmark workload's grid timing alone (full-size profiles); grad300: sigma_min "
                         "and the gradient kernel on the same 40 000 points (gradient profiles); "
                         "fp64probe: the FP64 unit's rates (psa_probe_fp64)")
    ap.add_argument("--workload", default="grid",
                    choices=["grid", "differentiation", "batched", "restriction", "classifier", "features"],
                    help="grid: the benchmark line; differentiation: the adjoint workload; "
                         "batched: 256 matrices on their own grids; restriction: the learned restriction; "
                         "features: eigenvalue against symbol-curve features (ablation)")
    ap.add_argument("--batch-size", type=int, default=256, help="batched: number of matrices")
    ap.add_argument("--restrict-train", type=int, default=2000, help="restriction: training matrices")
    ap.add_argument("--restrict-val", type=int, default=30, help="restriction: validation matrices")
    ap.add_argument("--ablation-train", type=int, default=600, help="features: training matrices")
    ap.add_argument("--restrict-val-grid", type=int, default=128, help="restriction: validation grid side")
    ap.add_argument("--restrict-test-n", type=int, default=20000, help="restriction: order of the test matrix")
    ap.add_argument("--restrict-grid", type=int, default=1024, help="restriction: test grid side")
    ap.add_argument("--save-model", default=None,
                    help="restriction: write the trained classifier(s) (.npz; comma-separated, one per network)")
    ap.add_argument("--net", default="both", choices=["mlp", "dual", "both"], help="restriction: classifier(s)")
    ap.add_argument("--load-models", default=None,
                    help="restriction: load trained classifier(s) (comma-separated .npz, one per network) "
                         "instead of training")
    ap.add_argument("--no-tune", action="store_true", help="batched: default launch controls")
    ap.add_argument("--no-e2e", action="store_true", help="batched: skip the end-to-end replay")
    ap.add_argument("--batch-streams", type=int, default=8, help="batched with --no-tune: streams")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "grad300":
        return run_grad_case(args)
    if args.case == "fp64probe":
        return run_fp64_probe(args)
    if args.workload == "differentiation":
        return run_differentiation(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "restriction":
        return run_restriction(args)
    if args.workload == "classifier":
        return run_classifier(args)
    if args.workload == "features":
        return run_feature_ablation(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
