"""Benchmark: log p + gradient evaluations per second of the strong-lens
log-posterior on B300.

Workload: the ground-based system (100x100 px at 0.262"/px, 3x3
supersampling, 11x11 Moffat PSF, one lens-light and one source Sersic), 4096
parameter vectors per step drawn from the priors; synthetic data rendered by
the library itself with seeded noise. A step is one fused forward + adjoint
launch over the whole batch. L2 is flushed (a 256 MB write) before every timed
step; each step is timed with CUDA events on its stream.

The same line also carries, as the sub-objects "space" and "uneven", a few
timed steps of the space-telescope workload (200x200 px at 0.05"/px, s = 5,
21x21 PSF, two sources, 16384 HMC chains; a step is one CUDA graph of 10
leapfrogs plus a Metropolis-Hastings test) and of the uneven multi-system
batch (100 systems of 40-200 px, s = 2-5, 256 rows each), each with its own
clocks and roofline (--no-extra-workloads leaves them out).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has) on the host cores, on a bounded sample of the same workload. Under
torchrun every rank runs its own replica (the evaluations are independent):
value is the sum of ranks' evaluations over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "logp+grad evals/s (100x100 px, 3x SS) on 1 B300, learned vs plain; % roofline"
SM_COUNT_B300 = 148
FP32_LANES_PER_SM = 128
MUFU_PER_SM_CLK = 16
# DRAM bytes (read + write) of one k_grad launch of the ground-based workload
# (4096 rows), from one ncu capture of this bench's own launch:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
#       -k regex:k_grad -s 3 -c 1 python bench.py --steps 5 --warmup 3 --no-cpu-baseline
#       --no-extra-workloads
# (763,392 read + 0 written; the outputs are still in L2 when the launch ends).
# Reported only while KGRAD_SOURCES still hash to the value recorded with the
# capture (kgrad_source_hash()); a changed kernel reports traffic null.
TRAFFIC_GROUND_4096 = 763392
# DRAM bytes of one k_grad launch of the space-telescope workload per row,
# from one capture of a 512-row launch inside the HMC leg
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
#       -k regex:k_grad -s 5 -c 1 python bench.py --workload space200-leapfrog
#       --batch 512 --steps 2 --warmup 3
# (26,013,952 read + 179,414,784 written); the traffic is the per-row scratch
# images, so it grows in proportion to the rows.
TRAFFIC_SPACE_PER_ROW = (26013952 + 179414784) / 512
# kgrad_source_hash() of the sources the two captures above were taken with
# (None: no capture of the current kernel yet)
TRAFFIC_SOURCE_HASH = "327c8f8ebcb9f907"
KGRAD_SOURCES = ["gl_internal.cuh", "gl_model.cuh", "gl_subpixel.cuh", "gl_kernels.cuh",
                 "gl_grad.cu", "gl_grad_impl.cuh", "gl_grad_l0_series.cu", "gl_grad_l1_series.cu",
                 "gl_grad_l2_series.cu"]


def kgrad_source_hash() -> str:
    """SHA-256 (first 16 hex digits) of the fused gradient kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for name in KGRAD_SOURCES:
        with open(os.path.join(ROOT, "paper_2606_30633_b300", "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def captured_traffic(value):
    """value if the kernel is the one the ncu capture measured, else None."""
    return value if TRAFFIC_SOURCE_HASH == kgrad_source_hash() else None


# ------------------------------------------------------------ op counts ----
def series_terms(f: float, t: float) -> int:
    """EPL series length the kernels use for |e| = f and slope t = gamma - 1
    (before rounding up to a multiple of 2): the smallest N >= 1 whose next
    coefficient |e_{N+1}| = prod_{k<=N+1} |rho_k| (rho_1 = r_1, rho_k = f r_k,
    r_k = (2k-2+t)/(2k+2-t)) is at most 2^-24 (1-f)^2 / 2."""
    tol = 2.0 ** -24 * (1 - f) ** 2 * 0.5
    e = t / (4.0 - t)
    n = 1
    while n < 128:
        k = n + 1
        e *= f * (2 * k - 2 + t) / (2 * k + 2 - t)
        if e <= tol:
            break
        n += 1
    return n


def algorithmic_ops(theta: np.ndarray, ny: int, nx: int, s: int, k: int, n_light: int,
                    n_src: int) -> tuple:
    """FP32 operations (an FMA counts once, per lane) and MUFU operations of
    one log p + gradient evaluation per row, summed over rows, counted term
    by term from the formulation the kernels evaluate (negations fold into
    the consuming operation and are not counted; max/select are ALU work):
      forward sub-pixel  2 (grid) + 14 (EPL frame, w) + 1 + 2N (series)
                         + 4 (F) + 16 (deflection, shear, lens equation)
                         + 11 per Sersic + (components - 1) (sum) + 1 (bin)
                         ... 3 MUFU for the EPL, 3 per Sersic
      adjoint sub-pixel  2 + 15 + 1 + 4N (both series) + 10 (E, F, dF/dt)
                         + 16 + 24 per Sersic + 8 per source (amplitude and
                         position gradient) + 74 (EPL and shear adjoint)
                         ... 4 MUFU for the EPL, 4 per Sersic
      per pixel          2 k^2 (PSF convolution and its adjoint) + 8
    with N the row's series length (Clenshaw's recurrence: two operations
    per term)."""
    nsub = ny * nx * s * s
    npix = ny * nx
    ncomp = n_light + n_src
    f = np.hypot(theta[:, 2], theta[:, 3])
    N = np.array([series_terms(float(v), float(g) - 1.0) for v, g in zip(f, theta[:, 1])])
    fwd = 2 + 14 + 1 + 2 * N + 4 + 16 + 11 * ncomp + (ncomp - 1) + 1
    adj = 2 + 15 + 1 + 4 * N + 10 + 16 + 24 * ncomp + 8 * n_src + 74
    ops = nsub * (fwd + adj) + npix * (2 * k * k + 8)
    mufu = nsub * (3 + 3 * ncomp + 4 + 4 * ncomp)
    return float(ops.sum()), float(mufu * theta.shape[0])


def unit_rate_roofline(gl, mufu_ops: float, step_s: float, clocks: dict) -> tuple:
    """The pipe rates measured on this GPU (gl_unit_rates, operations per SM
    per SM clock) and the MUFU side of the roofline: MUFU operations per step
    over the step time against n_SM x r_MUFU x the sampled SM clock."""
    r = gl.unit_rates()
    rates = {k: round(v, 2) for k, v in r.items()}
    rates["unit"] = "ops per SM per SM clock"
    mhz = clocks.get("sm_mhz") or 2032.0
    peak = SM_COUNT_B300 * r["mufu"] * mhz * 1e6 / 1e12
    achieved = mufu_ops / step_s / 1e12
    return rates, {"achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                   "clock_mhz": mhz}


# ------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[4:8]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- arms ----
def host_cores() -> int:
    """The host cores this process may run on: the oracle's thread count is
    set from them explicitly, since launchers such as torchrun set
    OMP_NUM_THREADS=1 for every rank."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t_ms: float, world: int, device) -> float:
    """The job's timed total: the slowest rank's (an all-reduce MAX over the
    process group; each rank's own total when there is one rank)."""
    if world == 1:
        return t_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, t_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (ranks hold equal shares of the work: weak scaling)."""
    return world * units_per_rank / (t_ms / 1e3)


def run_reference(args) -> dict | None:
    """The FP64 oracle (value + dual-number gradient, OpenMP over rows) on the
    host cores, on a bounded sample of the same workload."""
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    W = synth.ground_100()
    spec = W.prior()
    cores = host_cores()
    S0 = oracle.System(W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
                       np.ones((W.ny, W.nx)), W.psf, 1, 1, spec)
    m = S0.model_image(W.truth())[0]
    d, sig = synth.noisy_data(m, W.noise())
    S = oracle.System(W.ny, W.nx, W.pixel_scale, W.supersample, d, sig, W.psf, 1, 1, spec)
    theta = W.samples()
    rows = max(cores, 1)
    per_step = []
    for step in range(args.warmup + args.steps):
        th = theta[(step * rows) % W.batch:(step * rows) % W.batch + rows]
        t0 = time.perf_counter()
        S.logp_grad(th, nthreads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            per_step.append(dt)
    total = sum(per_step)
    value = rows * len(per_step) / total
    sample = (f"{rows} rows per step (one per core) of the 4096-row ground-based batch, "
              f"{len(per_step)} timed steps")
    return {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(per_step),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": W.name, "batch_per_step": rows, "ny": W.ny, "nx": W.nx,
                   "supersample": W.supersample, "psf": 11, "params": W.P},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def timed_steps(fn, steps, warmup, stream, flush):
    import torch
    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def learned_leg(args, S, W, theta, theta_np, logp, grad, stream, flush, world) -> dict:
    """The learned deflection surrogate on the same workload: trained here with
    the library's kernels (1e7 exact-series tuples, 120 epochs), then the same
    timed steps with GL_DEFL_SURROGATE (per-row angular tables from the network,
    interpolated per sub-pixel; rows outside its q/gamma domain use the series).
    |d log p| is measured against the exact-series path of the same kernels,
    near the mode (truth + small steps) and at the benchmark's prior draws."""
    import torch
    import paper_2606_30633_b300 as gl
    t0 = time.perf_counter()
    sur = gl.Surrogate.train(n_samples=10_000_000, epochs=120, batch=16384, lr=2e-3, lr_min=1e-5,
                             seed_data=401, seed_init=402)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    S.set_surrogate(sur)
    out = {}
    for name, defl in (("surrogate", gl.GL_DEFL_SURROGATE),
                       ("surrogate_fused", gl.GL_DEFL_SURROGATE_FUSED),
                       ("exact_tables", gl.GL_DEFL_TABLE), ("exact_tables_fp32", gl.GL_DEFL_TABLE32)):
        ms = timed_steps(lambda: S.logp_grad(theta, defl=defl, out=logp, grad=grad, stream=stream),
                         args.steps, args.warmup, stream, flush)
        out[name] = world * W.batch / (statistics.mean(ms) / 1e3)
    near = synth.jitter(W.truth(), W.prior(), 64, 7, rel=0.01).astype(np.float32)
    near[0] = W.truth()
    tn = torch.tensor(near, device=theta.device)
    d_near = (S.logp(tn, defl=gl.GL_DEFL_SURROGATE) - S.logp(tn)).abs().cpu().numpy()
    d_prior = (S.logp(theta, defl=gl.GL_DEFL_SURROGATE) - S.logp(theta)).abs().cpu().numpy()
    t_near = (S.logp(tn, defl=gl.GL_DEFL_TABLE32) - S.logp(tn)).abs().cpu().numpy()
    t_prior = (S.logp(theta, defl=gl.GL_DEFL_TABLE32) - S.logp(theta)).abs().cpu().numpy()
    e = np.hypot(theta_np[:, 2], theta_np[:, 3])
    in_dom = float(np.mean(((1 - e) / (1 + e) >= 0.5) & (e >= 0.01)))
    # deflection error against the library's FP64 series on 2e5 held-out tuples
    # of the training distribution, in arcsec at theta_E = 1.25"
    r = np.random.default_rng(403)
    n = 200_000
    X = np.stack([r.uniform(0.5, 1, n), r.uniform(1.7, 2.3, n),
                  r.uniform(np.log(0.05), np.log(5), n), r.uniform(0, 2 * np.pi, n)],
                 1).astype(np.float32)
    Xt = torch.tensor(X, device=theta.device)
    dF = (sur.infer(Xt) - gl.series_F(Xt)).double().cpu().numpy()
    q, t, thE = X[:, 0].astype(np.float64), X[:, 1] - 1.0, 1.25
    b = thE * np.sqrt(q)
    dal = 2 * b / (1 + q) * (b / (np.exp(X[:, 2]) * thE)) ** (t - 1) * np.hypot(dF[:, 0], dF[:, 1])
    return sur, {"value": out["surrogate"], "unit": "evals/s",
            "deflection": "learned surrogate (4-64x4-2 SiLU MLP, BF16 tensor cores), tables per row",
            "dlogp_abs_max_near_mode": float(d_near.max()),
            "dlogp_abs_prior_draws": {"p50": float(np.median(d_prior)),
                                      "p90": float(np.percentile(d_prior, 90)),
                                      "p99": float(np.percentile(d_prior, 99)),
                                      "max": float(d_prior.max())},
            "deflection_err_arcsec": {"rms": float(np.sqrt(np.mean(dal ** 2))),
                                      "max": float(dal.max()), "theta_E": thE,
                                      "tuples": n},
            "rows_in_surrogate_domain": in_dom,
            "train_seconds": train_s, "train_final_loss": sur.final_loss,
            "surrogate_in_ray_shoot_cta_evals_per_s": out["surrogate_fused"],
            "exact_series_tables_evals_per_s": out["exact_tables"],
            "exact_series_tables_fp32": {
                "value": out["exact_tables_fp32"], "unit": "evals/s",
                "dlogp_abs_max_near_mode": float(t_near.max()),
                "dlogp_abs_prior_draws": {"p50": float(np.median(t_prior)),
                                          "p90": float(np.percentile(t_prior, 90)),
                                          "p99": float(np.percentile(t_prior, 99)),
                                          "max": float(t_prior.max())}},
            "note": "the speed-up over the per-sub-pixel series comes from tabulating F per "
                    "row; exact_series_tables(_fp32) tabulate the exact series the same way "
                    "(FP64 / FP32 build): what the network adds over tabulation is the "
                    "difference between those figures and the surrogate's"}


def cpu_baseline_leg(budget_s: float = 12.0) -> dict:
    import oracle
    W = synth.ground_100()
    spec = W.prior()
    cores = host_cores()
    S0 = oracle.System(W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
                       np.ones((W.ny, W.nx)), W.psf, 1, 1, spec)
    m = S0.model_image(W.truth())[0]
    d, sig = synth.noisy_data(m, W.noise())
    S = oracle.System(W.ny, W.nx, W.pixel_scale, W.supersample, d, sig, W.psf, 1, 1, spec)
    theta = W.samples(8 * cores)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s and done + cores <= theta.shape[0]:
        S.logp_grad(theta[done:done + cores], nthreads=cores)
        done += cores
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} rows of the ground-based batch (value + dual-number gradient), "
                      f"{dt:.1f} s on {cores} threads"}


def run_ours(args) -> dict | None:
    import torch
    import paper_2606_30633_b300 as gl
    from paper_2606_30633_b300 import build as glbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    glbuild.build()
    dev = torch.device("cuda", local)

    W = synth.ground_100()
    if args.batch:
        W.batch = args.batch
    spec = W.prior()
    B = W.batch
    # synthetic data: the library renders the truth; seeded noise on the host
    blank = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
                      np.ones((W.ny, W.nx)), W.psf, 1, 1, spec)
    truth = torch.tensor(W.truth()[None], dtype=torch.float32, device=dev)
    m = blank.model_image(truth)[0].double().cpu().numpy()
    blank.close()
    d, sig = synth.noisy_data(m, W.noise())
    S = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, d, sig, W.psf, 1, 1, spec)
    theta_np = W.samples().astype(np.float32)
    theta = torch.tensor(theta_np, device=dev)
    logp = torch.empty(B, device=dev)
    grad = torch.empty_like(theta)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step():
        S.logp_grad(theta, out=logp, grad=grad, stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = sum(step_ms)
    t_ms = max_over_ranks(t_ms, world, dev)
    value = job_rate(B * args.steps, world, t_ms)
    assert torch.isfinite(logp).all(), "non-finite log p in the benchmark batch"

    # end to end through the public API with host buffers: theta in pinned host
    # memory, log p and the gradient back into pinned host memory
    h_theta = gl.pinned_array(theta_np.shape)
    h_theta[:] = theta_np
    h_out = (gl.pinned_array((B,)), gl.pinned_array(theta_np.shape))
    e2e_ms = []
    for k in range(args.warmup + max(3, args.steps // 5)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.logp_grad_host(h_theta, out=h_out)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            e2e_ms.append(dt * 1e3)
    e2e_value = world * B / (statistics.mean(e2e_ms) / 1e3)

    sur, learned = learned_leg(args, S, W, theta, theta_np, logp, grad, stream, flush, world)

    ops, mufu = algorithmic_ops(theta_np.astype(np.float64), W.ny, W.nx, W.supersample,
                                W.psf.shape[0], 1, 1)
    mean_s = statistics.mean(step_ms) / 1e3
    peak = SM_COUNT_B300 * FP32_LANES_PER_SM * 2.032e9 / 1e12
    achieved = ops / mean_s / 1e12
    clocks = clk.summary()
    rates, mufu_roof = unit_rate_roofline(gl, mufu, mean_s, clocks)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded priors, library-rendered truth, seeded noise)",
            "config": {"workload": W.name, "batch_per_step": B, "ny": W.ny, "nx": W.nx,
                       "supersample": W.supersample, "psf": int(W.psf.shape[0]),
                       "params": W.P, "deflection": "series (plain)",
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}"},
            "learned": learned,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak,
                         "traffic": captured_traffic(TRAFFIC_GROUND_4096) if B == 4096 else None,
                         "kernel_source_hash": kgrad_source_hash(),
                         "algorithmic_bytes": B * (2 * W.P + 1) * 4 + 2 * W.ny * W.nx * 4,
                         "note": "FP32 lane-operations (FMA = 1) of the formulation's op "
                                 "count per evaluation / mean step time; peak = 148 SM x 128 "
                                 "lanes x 2032 MHz; traffic = ncu DRAM bytes of the k_grad "
                                 "launch (one pass, captured on this bench's launch)",
                         "mufu_ops_per_step": mufu,
                         "measured_unit_rates": rates,
                         "mufu": mufu_roof},
            "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": B * W.P * 4,
                    "d2h_bytes_per_step": B * (W.P + 1) * 4},
            "gpu_launches": args.steps,
            "clocks": clocks,
        }
    if not args.no_extra_workloads:
        # the space-telescope HMC graph and the uneven multi-system batch, each
        # timed on its own (a few steps; their own clocks and rooflines)
        space = space_leg(args.extra_steps, 3, world, local, e2e_reps=1)
        uneven = uneven_leg(max(args.extra_steps, 5), 3, world, local, sur=sur)
        if out is not None:
            out["space"] = space
            out["uneven"] = uneven
    if out is not None and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_leg()
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def space_leg(steps: int, warmup: int, world: int, local: int, e2e_reps: int = 2,
              batch: int | None = None) -> dict:
    """Space-telescope-like system under the batched gradient loop: 200x200 px
    at 0.05"/px, s = 5, 21x21 Gaussian-core PSF, two source components, 16384
    chains started near the truth; a step is one HMC transition: a CUDA graph of
    10 leapfrogs (each a fused forward + adjoint over all chains) in the
    unconstrained space of the prior's bijection, then a Metropolis-Hastings
    test, with the step size from dual averaging on 512 of the chains.
    Returns the leg's figures (rank 0's copy is the one reported)."""
    import torch
    import paper_2606_30633_b300 as gl
    dev = torch.device("cuda", local)
    W = synth.space_200()
    if batch:
        W.batch = batch
    spec = W.prior()
    B, L = W.batch, 10
    blank = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
                      np.ones((W.ny, W.nx)), W.psf, W.n_lens_light, W.n_source, spec)
    truth = W.truth()
    m = blank.model_image(torch.tensor(truth[None], dtype=torch.float32, device=dev))[0]
    m = m.double().cpu().numpy()
    blank.close()
    d, sig = synth.noisy_data(m, W.noise())
    S = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, d, sig, W.psf, W.n_lens_light,
                  W.n_source, spec)
    # chains start near the truth; they move in the unconstrained space of the
    # prior's bijection, so no trajectory can leave the support, and every
    # block ends with a Metropolis-Hastings test (divergent proposals are
    # rejected). The step size comes from dual averaging on 512 of the chains.
    th_np = synth.jitter(truth, spec, B, W.seed_samples, rel=0.002).astype(np.float32)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    u0 = S.bijector_inverse(torch.tensor(th_np, device=dev))
    ha = gl.Hmc(S, u0[:512].clone(), L, 1e-3, 0.8, seed=W.seed_samples + 2)
    ha.run(40, gl.GL_HMC_ADAPT_STEP, stream=stream)
    ha.end_adaptation(set_inv_mass=False, stream=stream)
    eps = ha.state()[3]
    ha.close()
    h = gl.Hmc(S, u0, L, eps, 0.8, seed=W.seed_samples + 3)
    acc = torch.empty(warmup + steps, device=dev)
    for k in range(warmup):
        flush.zero_()
        h.run(1, 0, None, acc[k:k + 1], stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with ClockSampler(local) as clk:
        for k, (a, b) in enumerate(ev):
            flush.zero_()
            a.record(stream)
            h.run(1, 0, None, acc[warmup + k:warmup + k + 1], stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = sum(step_ms)
    t_ms = max_over_ranks(t_ms, world, dev)
    value = job_rate(B * L * steps, world, t_ms)
    u_end, lp_end, _, _ = h.state()
    h.close()
    finite = float(torch.isfinite(lp_end).float().mean())
    th_end = S.bijector_forward(u_end)[0].double().cpu().numpy()
    # end to end: chain starts from pinned host memory, one transition, the
    # chains' log p back to the host
    h_u = u0.cpu().pin_memory()
    h_lp = torch.empty(B).pin_memory()
    e2e_ms = []
    for _ in range(e2e_reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ud = h_u.to(dev, non_blocking=True)
        h2 = gl.Hmc(S, ud, L, eps, 0.8, seed=W.seed_samples + 4)
        h2.run(1, 0, stream=stream)
        _, lp2, _, _ = h2.state()
        h_lp.copy_(lp2, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        h2.close()
    S.close()
    e2e_value = world * B * (L + 1) / (min(e2e_ms) / 1e3)
    ops, _ = algorithmic_ops(th_end, W.ny, W.nx, W.supersample,
                             W.psf.shape[0], W.n_lens_light, W.n_source)
    mean_s = statistics.mean(step_ms) / 1e3
    peak = SM_COUNT_B300 * FP32_LANES_PER_SM * 2.032e9 / 1e12
    achieved = ops * L / mean_s / 1e12
    return {
        "metric": "logp+grad evals/s (200x200 px, 5x SS, 16384 chains, 10-leapfrog graph "
                  "blocks, one Metropolis-Hastings test per block) on 1 B300",
        "value": value, "unit": "evals/s", "steps": steps, "warmup": warmup,
        "ms_per_step": t_ms / steps,
        "config": {"workload": W.name, "chains": B, "leapfrogs_per_step": L,
                   "step_size_unconstrained": eps,
                   "mean_accept": float(acc[warmup:].mean()),
                   "ny": W.ny, "nx": W.nx, "supersample": W.supersample,
                   "psf": int(W.psf.shape[0]), "params": W.P,
                   "l2": "flushed (256 MB write) before every timed step",
                   "finite_chains_at_end": finite},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak,
                     "traffic": captured_traffic(TRAFFIC_SPACE_PER_ROW * B),
                     "traffic_note": "ncu DRAM bytes of a 512-row launch scaled to the "
                                     "launch's rows (per-row scratch images)"},
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": B * W.P * 4,
                "d2h_bytes_per_step": B * 4},
        "gpu_launches": (2 * L + 4) * steps,
        "clocks": clk.summary(),
    }


def run_leapfrog(args) -> dict | None:
    """The space-telescope workload on its own (see space_leg)."""
    import torch
    from paper_2606_30633_b300 import build as glbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    glbuild.build()
    leg = space_leg(args.steps, args.warmup, world, local, batch=args.batch)
    out = None
    if rank == 0:
        out = {"metric": leg.pop("metric"), "value": leg.pop("value"), "unit": "evals/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": leg.pop("ms_per_step"), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded priors, library-rendered truth, seeded noise)", **leg}
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def uneven_leg(steps: int, warmup: int, world: int, local: int, sur=None,
               batch: int | None = None, shape: str | None = None,
               policy: str | None = None) -> dict:
    """Uneven-batch persistent run: 100 synthetic systems (sides 40-200 px,
    s = 2-5, 1-3 source components, 0.262"/px, 11x11 Moffat), 256 rows each,
    all evaluated per step by gl_multi_logp_grad (persistent launches per
    group); the launch shapes are picked by the autotuner; the exact series
    and the learned surrogate (sur, trained here when None) side by side."""
    import torch
    import paper_2606_30633_b300 as gl
    from paper_2606_30633_b300 import autotune
    dev = torch.device("cuda", local)
    Ws = synth.uneven_systems()
    systems, thetas, rows = [], [], []
    for W in Ws:
        if batch:
            W.batch = batch  # rows per system (profiling runs)
        spec = W.prior()
        blank = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
                          np.ones((W.ny, W.nx)), W.psf, W.n_lens_light, W.n_source, spec)
        m = blank.model_image(torch.tensor(W.truth()[None], dtype=torch.float32, device=dev))[0]
        m = m.double().cpu().numpy()
        blank.close()
        d, sig = synth.noisy_data(m, W.noise())
        systems.append(gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, d, sig, W.psf,
                                 W.n_lens_light, W.n_source, spec))
        thetas.append(torch.tensor(W.samples().astype(np.float32), device=dev))
        rows.append(W.batch)
    n_rows = sum(rows)
    if shape:
        # a fixed launch shape for every system, no tuning (profiling runs)
        t, p = (int(v) for v in shape.split("x"))
        pol = policy or "two_ctas"
        plan = gl.Multi(systems, rows, autotune.POLICIES[pol], threads=[t] * len(systems),
                        pairs=[p] * len(systems))
        tune = {"assignment": f"fixed {t}x{p}", "policy": pol, "batch_ms": {}, "classes": {}}
    else:
        plan, tune = autotune.tune_multi(systems, rows, thetas, reps=2)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    logps, grads = plan.logp_grad(thetas)
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        ms = timed_steps(lambda: plan.logp_grad(thetas, logps, grads, stream=stream), steps,
                         warmup, stream, flush)
    if sur is None:
        sur = gl.Surrogate.train(n_samples=10_000_000, epochs=120, batch=16384, lr=2e-3,
                                 lr_min=1e-5, seed_data=401, seed_init=402)
    for s_ in systems:
        s_.set_surrogate(sur)
    lps_s = [t.clone() for t in logps]
    ms_sur = timed_steps(lambda: plan.logp_grad(thetas, logps, grads, defl=gl.GL_DEFL_SURROGATE,
                                                stream=stream), steps, warmup, stream, flush)
    dl = torch.cat([(a - b).abs() for a, b in zip(logps, lps_s)]).cpu().numpy()
    # end to end: every system's rows from pinned host memory, one multi-system
    # evaluation (exact series), log p and gradients back to pinned host memory
    h_th = [t.cpu().pin_memory() for t in thetas]
    h_lp = [torch.empty(t.shape[0]).pin_memory() for t in thetas]
    h_g = [torch.empty(t.shape).pin_memory() for t in thetas]
    e2e_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d_, h_ in zip(thetas, h_th):
            d_.copy_(h_, non_blocking=True)
        plan.logp_grad(thetas, logps, grads, stream=stream)
        for a_, b_, c_, d_ in zip(h_lp, logps, h_g, grads):
            a_.copy_(b_, non_blocking=True)
            c_.copy_(d_, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = sum(t.numel() * 4 for t in thetas)
    d2h = sum(t.numel() * 4 + t.shape[0] * 4 for t in thetas)
    t_ms = sum(ms)
    t_ms = max_over_ranks(t_ms, world, dev)
    value = job_rate(n_rows * steps, world, t_ms)
    ops = 0.0
    for W, th in zip(Ws, thetas):
        o, _ = algorithmic_ops(th.double().cpu().numpy(), W.ny, W.nx, W.supersample,
                               W.psf.shape[0], W.n_lens_light, W.n_source)
        ops += o
    peak = SM_COUNT_B300 * FP32_LANES_PER_SM * 2.032e9 / 1e12
    achieved = ops / (statistics.mean(ms) / 1e3) / 1e12
    # one launch per group of (component counts, launch shape)
    launches = len({(W.n_lens_light, W.n_source, sh) for W, sh in zip(Ws, plan.shapes())})
    shapes = {"assignment": tune["assignment"], "smem_policy": tune["policy"],
              "batch_ms": {a: {k: round(v, 3) for k, v in d.items()}
                           for a, d in tune["batch_ms"].items()},
              "per_class": {name: {"threads_per_cta": c["shape"][0], "pixel_pairs": c["shape"][1],
                                   "systems": c["systems"],
                                   "ms": {f"{t}x{p}": round(v, 4) for (t, p), v in c["ms"].items()}}
                            for name, c in tune["classes"].items()}}
    plan.close()
    for s_ in systems:
        s_.close()
    return {
        "metric": "logp+grad evals/s (100 uneven systems: 40-200 px, 2-5x SS, 1-3 sources, "
                  "256 rows each) on 1 B300",
        "value": value, "unit": "evals/s", "steps": steps, "warmup": warmup,
        "ms_per_step": t_ms / steps,
        "config": {"workload": "uneven-100-systems", "systems": len(Ws), "rows": n_rows,
                   "launch_shapes": shapes,
                   "l2": "flushed (256 MB write) before every timed step"},
        "learned": {"value": world * n_rows / (statistics.mean(ms_sur) / 1e3), "unit": "evals/s",
                    "dlogp_abs_median": float(np.median(dl)),
                    "dlogp_abs_p90": float(np.quantile(dl, 0.9))},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": None},
        "e2e": {"value": world * n_rows / (min(e2e_ms) / 1e3), "unit": "evals/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * steps,
        "clocks": clk.summary(),
    }


def run_uneven(args) -> dict | None:
    """The uneven multi-system workload on its own (see uneven_leg)."""
    import torch
    from paper_2606_30633_b300 import build as glbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    glbuild.build()
    leg = uneven_leg(args.steps, args.warmup, world, local, batch=args.batch,
                     shape=args.uneven_shape, policy=args.uneven_policy)
    out = None
    if rank == 0:
        out = {"metric": leg.pop("metric"), "value": leg.pop("value"), "unit": "evals/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": leg.pop("ms_per_step"), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded priors, library-rendered truths, seeded noise)", **leg}
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def run_pipeline(args) -> dict | None:
    """The inference stages of the paper's pipeline (Sec. 3) on the
    ground-based system (100x100 px, s = 3), 4096 rows each, through the
    library's device-resident drivers: multi-start MAP (Adam, one logp+grad
    evaluation per row and step), SVI (AdaBelief, 4096 log p~ samples per
    step, score-function gradient), backward intensity modelling (4096 rows,
    intensities by linear inversion) and HMC (4096 chains, 10-leapfrog
    transitions with Metropolis-Hastings). The line's value is the HMC
    throughput in logp+grad evaluations/s; the other figures ride along."""
    import torch
    import paper_2606_30633_b300 as gl
    from paper_2606_30633_b300 import build as glbuild, infer

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    glbuild.build()
    dev = torch.device("cuda", local)
    W = synth.ground_100()
    if args.batch:
        W.batch = args.batch
    spec = W.prior()
    B, L = W.batch, 10
    blank = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
                      np.ones((W.ny, W.nx)), W.psf, 1, 1, spec)
    truth = W.truth()
    m = blank.model_image(torch.tensor(truth[None], dtype=torch.float32, device=dev))[0]
    blank.close()
    d, sig = synth.noisy_data(m.double().cpu().numpy(), W.noise())
    S = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, d, sig, W.psf, 1, 1, spec)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    # MAP from the prior draws
    u_map = S.bijector_inverse(torch.tensor(W.samples().astype(np.float32), device=dev))
    mm, vv = torch.zeros_like(u_map), torch.zeros_like(u_map)
    state = {"t": 0}
    K = 10

    def map_step():
        S.map_adam(u_map, mm, vv, K, t0=state["t"], lr=1e-2, stream=stream)
        state["t"] += K

    map_ms = timed_steps(map_step, max(2, args.steps // 5), args.warmup, stream, flush)
    map_value = world * B * K / (statistics.mean(map_ms) / 1e3)
    # SVI around the truth
    u_true = S.bijector_inverse(torch.tensor(truth[None].astype(np.float32), device=dev))[0]
    phi, opt = infer.svi_init(S, u_true, scale=1e-3)
    sv = {"t": 0}

    def svi_step():
        S.svi_adabelief(phi, opt, B, K, t0=sv["t"], seed=11, stream=stream)
        sv["t"] += K

    svi_ms = timed_steps(svi_step, max(2, args.steps // 5), args.warmup, stream, flush)
    svi_value = world * B * K / (statistics.mean(svi_ms) / 1e3)
    # backward intensities (linear inversion) on the prior draws
    th_b = torch.tensor(W.samples().astype(np.float32), device=dev)
    bwd_ms = timed_steps(lambda: S.logp_grad_backward(th_b, stream=stream),
                         max(2, args.steps // 5), args.warmup, stream, flush)
    bwd_value = world * B / (statistics.mean(bwd_ms) / 1e3)
    # HMC: chains near the truth, step tuned by a short adaptation first
    th0 = synth.jitter(truth, spec, B, W.seed_samples, rel=0.002).astype(np.float32)
    u0 = S.bijector_inverse(torch.tensor(th0, device=dev))
    h = gl.Hmc(S, u0, L, 1e-3, 0.75, seed=21)
    h.run(30, gl.GL_HMC_ADAPT_STEP, stream=stream)
    h.end_adaptation(set_inv_mass=False, stream=stream)
    acc = torch.empty(args.warmup + args.steps, device=dev)
    for k in range(args.warmup):
        flush.zero_()
        h.run(1, 0, None, acc[k:k + 1], stream=stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k, (a, b) in enumerate(ev):
            flush.zero_()
            a.record(stream)
            h.run(1, 0, None, acc[args.warmup + k:args.warmup + k + 1], stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = sum(step_ms)
    t_ms = max_over_ranks(t_ms, world, dev)
    value = job_rate(B * L * args.steps, world, t_ms)
    u_end, lp_end, _, eps = h.state()
    h.close()
    # end to end: chain starts from pinned host memory, one transition, the
    # chains' log p~ back to the host
    h_u = u0.cpu().pin_memory()
    h_lp = torch.empty(B).pin_memory()
    e2e_ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ud = h_u.to(dev, non_blocking=True)
        h2 = gl.Hmc(S, ud, L, eps, 0.75, seed=22)
        h2.run(1, 0, stream=stream)
        _, lp2, _, _ = h2.state()
        h_lp.copy_(lp2, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        h2.close()
    e2e_value = world * B * (L + 1) / (min(e2e_ms) / 1e3)
    th_end, _ = S.bijector_forward(u_end)
    ops, _ = algorithmic_ops(th_end.double().cpu().numpy(), W.ny, W.nx, W.supersample,
                             W.psf.shape[0], 1, 1)
    peak = SM_COUNT_B300 * FP32_LANES_PER_SM * 2.032e9 / 1e12
    achieved = ops * L / (statistics.mean(step_ms) / 1e3) / 1e12
    out = None
    if rank == 0:
        out = {
            "metric": "HMC logp+grad evals/s (100x100 px, 3x SS, 4096 chains, 10-leapfrog "
                      "transitions with Metropolis-Hastings) on 1 B300",
            "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded priors, library-rendered truth, seeded noise)",
            "config": {"workload": "pipeline-" + W.name, "chains": B, "leapfrogs": L,
                       "step_size": eps, "mean_accept": float(acc[args.warmup:].mean()),
                       "l2": "flushed (256 MB write) before every timed step"},
            "map": {"value": map_value, "unit": "logp+grad evals/s",
                    "ms_per_10_steps": statistics.mean(map_ms), "starts": B},
            "svi": {"value": svi_value, "unit": "logp evals/s",
                    "ms_per_10_steps": statistics.mean(svi_ms), "samples_per_step": B},
            "backward": {"value": bwd_value, "unit": "logp+grad evals/s (intensities solved)",
                         "ms_per_step": statistics.mean(bwd_ms), "rows": B},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None},
            "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": B * W.P * 4,
                    "d2h_bytes_per_step": B * 4},
            "gpu_launches": (2 * L + 4) * args.steps,
            "clocks": clk.summary(),
        }
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def run_fit(args) -> dict | None:
    """The whole inference pipeline of Sec. 3 with the hyperparameter table of
    the hundred simulated systems (Sec. 4.2) on the ground-based system
    (100x100 px, s = 3): multi-start MAP from 2000 prior draws for 1000 Adam
    steps, SVI with 1000 draws for 5000 AdaBelief steps, then HMC with 64
    chains (500 burn-in transitions with step-size and mass adaptation, the
    step-size retune, 1500 samples, 10 leapfrogs each). A step is one whole
    fit (infer.fit); warm-up steps are fits with 1 % of the iterations. The
    value is whole-job fits per hour; each rank fits its own copy."""
    import torch
    import paper_2606_30633_b300 as gl
    from paper_2606_30633_b300 import build as glbuild, infer

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    glbuild.build()
    dev = torch.device("cuda", local)
    W = synth.ground_100()
    spec = W.prior()
    blank = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
                      np.ones((W.ny, W.nx)), W.psf, 1, 1, spec)
    truth = W.truth()
    m = blank.model_image(torch.tensor(truth[None], dtype=torch.float32, device=dev))[0]
    blank.close()
    d, sig = synth.noisy_data(m.double().cpu().numpy(), W.noise())
    S = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, d, sig, W.psf, 1, 1, spec)
    n_map = 2000
    starts_np = synth.draw(spec, n_map, W.seed_samples, 1, 1).astype(np.float32)
    starts = torch.tensor(starts_np, device=dev)
    hp = dict(map_steps=1000, n_vi=1000, svi_steps=5000, n_chains=64, n_burnin=500,
              n_samples=1500, n_leapfrog=10)
    small = dict(map_steps=10, n_vi=1000, svi_steps=50, n_chains=64, n_burnin=5,
                 n_samples=15, n_leapfrog=10)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for k in range(args.warmup):
        infer.fit(S, starts, seed=100 + k, **small)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    secs, stages, results = [], [], []
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = infer.fit(S, starts, seed=k, **hp)
            torch.cuda.synchronize()
            secs.append(time.perf_counter() - t0)
            stages.append(r.seconds)
            results.append(r)
    t_s = max_over_ranks(sum(secs) * 1e3, world, dev) / 1e3
    value = world * args.steps / t_s * 3600.0
    # end to end: the starts from pinned host memory, the draws back to host memory
    h_starts = starts.cpu().pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r_e = infer.fit(S, h_starts.to(dev, non_blocking=True), seed=999, **hp)
    draws_host = r_e.hmc.draws.cpu()
    e2e_s = time.perf_counter() - t0
    last = results[-1]
    th_mean = last.hmc.draws.double().mean((0, 1)).cpu().numpy()
    th_sd = last.hmc.draws.double().std((0, 1)).cpu().numpy()
    evals = {"map": n_map * hp["map_steps"], "svi": hp["n_vi"] * hp["svi_steps"],
             "hmc": hp["n_chains"] * hp["n_leapfrog"]
             * (hp["n_burnin"] + hp["n_burnin"] // 2 + hp["n_samples"])}
    mean_stage = {k: statistics.mean(s[k] for s in stages) for k in stages[0]}
    out = None
    if rank == 0:
        out = {
            "metric": "whole fits per hour (MAP 2000 starts x 1000 steps, SVI 1000 draws x "
                      "5000 steps, HMC 64 chains x (500 + 250 retune + 1500) transitions of 10 "
                      "leapfrogs; 100x100 px, 3x SS) on 1 B300",
            "value": value, "unit": "fits/h", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded priors, library-rendered truth, seeded noise)",
            "config": {"workload": "fit-" + W.name, **hp, "n_map": n_map,
                       "l2": "flushed (256 MB write) before every timed fit"},
            "stages_s": mean_stage,
            "stage_evals_per_s": {k: evals[k] / mean_stage[k] for k in evals},
            "map_best_logp": last.map_logp,
            "hmc": {"rhat_max": float(np.max(last.hmc.rhat)),
                    "ess_min": float(np.min(last.hmc.ess)),
                    "mean_accept": float(np.mean(last.hmc.accept)),
                    "step_size": last.hmc.step_size,
                    "truth_within_sd": float(np.max(np.abs(th_mean - truth) / th_sd))},
            "e2e": {"value": 3600.0 / e2e_s * world, "unit": "fits/h",
                    "h2d_bytes_per_step": n_map * W.P * 4,
                    "d2h_bytes_per_step": int(draws_host.numel() * 4)},
            "gpu_launches": args.steps * (2 * hp["map_steps"] + 5 * hp["svi_steps"]
                                          + (2 * hp["n_leapfrog"] + 4)
                                          * (hp["n_burnin"] + hp["n_burnin"] // 2
                                             + hp["n_samples"])),
            "clocks": clk.summary(),
        }
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 50; 20 for space200-leapfrog, about 40 s; "
                         "1 whole fit for fit)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="ground100 only: skip the space-telescope and uneven-batch legs")
    ap.add_argument("--uneven-shape", default=None,
                    help="uneven workload: one launch shape THREADSxPAIRS for every system "
                         "instead of the autotuner's (profiling runs)")
    ap.add_argument("--uneven-policy", default=None, choices=["global", "two_ctas", "one_cta"],
                    help="shared-memory policy with --uneven-shape (default two_ctas)")
    ap.add_argument("--extra-steps", type=int, default=3,
                    help="timed steps of the space-telescope leg (the uneven leg takes at "
                         "least 5) in the default run")
    ap.add_argument("--batch", type=int, default=None,
                    help="rows per step (rows per system for uneven; default: the "
                         "workload's); for profiling runs")
    ap.add_argument("--workload", choices=["ground100", "space200-leapfrog", "uneven", "pipeline",
                                           "fit"],
                    default="ground100")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"space200-leapfrog": 20, "fit": 1}.get(args.workload, 50)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        res = run_reference(args)
    elif args.workload == "space200-leapfrog":
        res = run_leapfrog(args)
    elif args.workload == "uneven":
        res = run_uneven(args)
    elif args.workload == "pipeline":
        res = run_pipeline(args)
    elif args.workload == "fit":
        res = run_fit(args)
    else:
        res = run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
