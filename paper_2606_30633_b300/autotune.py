"""Autotuner for uneven multi-system batches.

The launch shape of the multi-system kernel is tuned per image class, a class
being the systems that share (image size, supersampling, PSF size). For each
class it times every candidate shape (threads per CTA 128 or 256, phase-1
pixel pairs per thread 2 or 3) on a plan of that class's own systems and rows,
and keeps the fastest; then it times the whole batch with those per-class
shapes and with each shape for all systems, under each shared-memory policy
(all buffers in global scratch / shared memory while the shape's full
occupancy fits / up to one CTA per SM), and keeps the fastest plan. Times are
CUDA events after warm-up, median of the repetitions. The results depend on the
mix of image sizes and supersampling, which is why they are measured on the
device rather than predicted.
"""
from __future__ import annotations

import statistics
from typing import Dict, List, Sequence, Tuple

from . import (GL_DEFL_SERIES, GL_MULTI_SMEM_GLOBAL, GL_MULTI_SMEM_ONE_CTA,
               GL_MULTI_SMEM_TWO_CTAS, Multi)

POLICIES = {"global": GL_MULTI_SMEM_GLOBAL, "two_ctas": GL_MULTI_SMEM_TWO_CTAS,
            "one_cta": GL_MULTI_SMEM_ONE_CTA}
# (threads per CTA, phase-1 pixel pairs per thread)
SHAPES = [(256, 2), (256, 3), (128, 2), (128, 3)]


def time_plan(plan: Multi, thetas, defl: int, warmup: int = 2, reps: int = 3, stream=None) -> float:
    """Median milliseconds of one plan.logp_grad call (CUDA events)."""
    import torch
    logps, grads = plan.logp_grad(thetas, defl=defl, stream=stream)
    for _ in range(warmup):
        plan.logp_grad(thetas, logps, grads, defl=defl, stream=stream)
    torch.cuda.synchronize()
    ms = []
    s = torch.cuda.current_stream() if stream is None else stream
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        plan.logp_grad(thetas, logps, grads, defl=defl, stream=stream)
        b.record(s)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def image_class(system) -> str:
    """The class key of a system: image size, supersampling and PSF size."""
    return f"{system.ny}x{system.nx}-s{system.s}-k{system.psf_size}"


def tune_shapes(systems: Sequence, rows: Sequence[int], thetas: List, defl: int = GL_DEFL_SERIES,
                warmup: int = 2, reps: int = 3,
                shapes: Sequence[Tuple[int, int]] = SHAPES) -> Dict[str, dict]:
    """{class: {"shape": (threads, pairs) of the fastest, "ms": {shape: median ms}}}
    from timing every shape on a plan of the class's own systems and rows."""
    classes: Dict[str, List[int]] = {}
    for k, s in enumerate(systems):
        if rows[k] > 0:
            classes.setdefault(image_class(s), []).append(k)
    out: Dict[str, dict] = {}
    for name, ks in classes.items():
        ms = {}
        for shape in shapes:
            n = len(ks)
            plan = Multi([systems[k] for k in ks], [rows[k] for k in ks], GL_MULTI_SMEM_TWO_CTAS,
                         threads=[shape[0]] * n, pairs=[shape[1]] * n)
            ms[shape] = time_plan(plan, [thetas[k] for k in ks], defl, warmup, reps)
            plan.close()
        out[name] = {"shape": min(ms, key=ms.get), "ms": ms, "systems": len(ks)}
    return out


def tune_multi(systems: Sequence, rows: Sequence[int], thetas: List, defl: int = GL_DEFL_SERIES,
               warmup: int = 2, reps: int = 3, shapes: Sequence[Tuple[int, int]] = SHAPES
               ) -> Tuple[Multi, dict]:
    """Returns (fastest plan, report). The whole batch is timed under every
    shared-memory policy for each assignment of shapes: the per-class picks of
    tune_shapes ("per_class") and every shape for all systems ("uniform TxN"),
    since shapes that win per class can lose on the whole batch when they split
    it into more launch groups. report["classes"] is tune_shapes' result,
    report["batch_ms"] the median ms per (assignment, policy), and
    report["assignment"] / report["policy"] the kept choice."""
    classes = tune_shapes(systems, rows, thetas, defl, warmup, reps, shapes)
    per_class = [classes.get(image_class(s), {"shape": (256, 2)})["shape"] for s in systems]
    assignments = {"per_class": per_class}
    for t, p in shapes:
        assignments[f"uniform {t}x{p}"] = [(t, p)] * len(systems)
    times: Dict[str, Dict[str, float]] = {}
    best, best_ms, choice = None, float("inf"), None
    for aname, shp in assignments.items():
        times[aname] = {}
        for pname, pol in POLICIES.items():
            plan = Multi(systems, rows, pol, threads=[x[0] for x in shp], pairs=[x[1] for x in shp])
            ms = time_plan(plan, thetas, defl, warmup, reps)
            times[aname][pname] = ms
            if ms < best_ms:
                if best is not None:
                    best.close()
                best, best_ms, choice = plan, ms, (aname, pname)
            else:
                plan.close()
    return best, {"classes": classes, "batch_ms": times, "assignment": choice[0],
                  "policy": choice[1]}
