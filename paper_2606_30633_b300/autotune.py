"""Autotuner for uneven multi-system batches.

Times gl_multi_logp_grad under each shared-memory policy (all buffers in
global scratch / shared memory while two CTAs fit per SM / up to one CTA per
SM) on the caller's own systems and rows, with CUDA events after warm-up, and
returns the fastest plan. Results depend on the mix of image sizes and
supersampling, which is why they are measured on the device rather than
predicted.
"""
from __future__ import annotations

import statistics
from typing import Dict, List, Sequence, Tuple

from . import (GL_DEFL_SERIES, GL_MULTI_SMEM_GLOBAL, GL_MULTI_SMEM_ONE_CTA,
               GL_MULTI_SMEM_TWO_CTAS, Multi)

POLICIES = {"global": GL_MULTI_SMEM_GLOBAL, "two_ctas": GL_MULTI_SMEM_TWO_CTAS,
            "one_cta": GL_MULTI_SMEM_ONE_CTA}


def time_plan(plan: Multi, thetas, defl: int, warmup: int = 2, reps: int = 3, stream=None) -> float:
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


def tune_multi(systems: Sequence, rows: Sequence[int], thetas: List, defl: int = GL_DEFL_SERIES,
               warmup: int = 2, reps: int = 3) -> Tuple[Multi, Dict[str, float]]:
    """Returns (fastest plan, {policy name: median ms per call})."""
    times: Dict[str, float] = {}
    best, best_ms = None, float("inf")
    for name, pol in POLICIES.items():
        plan = Multi(systems, rows, pol)
        ms = time_plan(plan, thetas, defl, warmup, reps)
        times[name] = ms
        if ms < best_ms:
            if best is not None:
                best.close()
            best, best_ms = plan, ms
        else:
            plan.close()
    return best, times
