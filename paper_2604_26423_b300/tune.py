"""Autotuner for the kernel configuration choices.

Forward path: the cost mode (C(x) recomputed in each tile from the weight
matrix, or streamed from a precomputed int32 diagonal), the tile shape (qubits
per shared-memory tile and CTAs per SM), the super-tile size, the group order
of the pass plan and the floating coalescing bits are timed on the caller's
instance and the fastest is kept. Each candidate runs on its own context with
its configuration set through ``qaoa_set_opts`` (no process-wide state), and
the winning cost mode is recorded with ``qaoa_set_cost_choice`` so that
QAOA_COST_AUTO contexts of that size and precision use it. Batched path: the
scheduling knobs of ``qaoa_batch_create`` (which instances run all their
passes in one CTA, items per pass, CTAs per SM) are timed on the caller's
batch.

Every candidate runs the full computation (same plan semantics, same results
up to FP32 summation order); timing is by CUDA events on the launching stream
after a warm-up run. Choices are cached in memory per workload key.
"""
from __future__ import annotations

import itertools

_cache: dict = {}

# tile shape of the forward kernel: 2^R registers x 2^WB warps (complex128:
# 4x3 or 5x3)
FWD_SHAPES = ("5x3", "4x4", "5x2", "4x3", "5x4")
# largest super-tile (index bits kept together through L2 by one CTA)
SUPER_TILES = (12, 13, 14, 15)
# group order of the pass plans: the last layer ending on the low group (its
# final pass also writes the sampling block sums), or the low group away from
# the fused passes
GROUP_ORDERS = ("last", "middle")
# coalescing bits applied in a plain high-group pass of each layer (1) or
# with the low group (0)
FLOAT_LANES = (1, 0)


# the CTA's next tile prefetched into L2 (measured faster with the one-CTA-per-SM
# 5x4 tile at 30 qubits, slower at 33)
L2_PREFETCH = (0, 1)


def forward_candidates(n: int, precision: str = "c64", modes=("recompute", "stream"), shapes=None,
                       super_tiles=SUPER_TILES, orders=GROUP_ORDERS, float_lanes=FLOAT_LANES,
                       prefetch=L2_PREFETCH):
    """Configurations to time for one instance: cost mode x tile shape x super-tile bits x group order x
    floating lane bits x L2 prefetch (a super-tile below the shape's tile means one tile)."""
    if shapes is None:
        shapes = FWD_SHAPES if precision == "c64" else ("4x3", "5x3")
    out = []
    for mode, shape, st, order, fl, pf in itertools.product(modes, shapes, super_tiles, orders, float_lanes,
                                                            prefetch):
        if st > n:
            continue
        out.append({"cost_mode": mode, "shape": shape, "super_tile": st, "order": order, "float_lanes": fl,
                    "l2_prefetch": pf})
    return out


def config_opts(cfg: dict) -> dict:
    """``qaoa.make_opts`` arguments that select a forward configuration."""
    return {"shape": cfg["shape"], "super_tile": cfg.get("super_tile"), "order": cfg.get("order", "last"),
            "float_lanes": bool(cfg.get("float_lanes", 1)), "l2_prefetch": bool(cfg.get("l2_prefetch", 0))}


def _time_ms(fn, stream, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_forward(n, u, v, w, p, dgamma, dbeta, scale=0.1, precision="c64", candidates=None, reps=1, key=None):
    """Times qaoa_run (p LR layers) under each candidate; returns (best, timings)."""
    import torch
    from .qaoa import Simulator, set_cost_choice
    key = key or ("fwd", n, precision, p, len(u))
    if key in _cache:
        return _cache[key]
    cands = candidates or forward_candidates(n, precision)
    stream = torch.cuda.current_stream()
    timings = []
    state = None
    for cfg in cands:
        s = Simulator(n, u, v, w, scale, precision, cost_mode=cfg["cost_mode"], state=state, opts=config_opts(cfg))
        try:
            state = s._state_t
            ms = _time_ms(lambda: s.run(p, dgamma, dbeta), stream, reps)
        finally:
            s.close()
        timings.append(dict(cfg, ms=ms))
    best = min(timings, key=lambda t: t["ms"])
    if len({t["cost_mode"] for t in timings}) > 1:
        set_cost_choice(n, precision, best["cost_mode"])
    _cache[key] = (best, timings)
    return best, timings


def batch_candidates(solo=(13, 16, 20, 25), units=(1, 2, 4), ctas=(2,), shapes=("5x3", "4x3"),
                     modes=("recompute", "stream")):
    """Batch configurations to time: scheduling knobs x forward tile shape x cost mode."""
    return [dict(solo_max_n=a, max_units=b, ctas_per_sm=c, fwd_shape=sh, cost_mode=m)
            for a, b, c, sh, m in itertools.product(solo, units, ctas, shapes, modes)]


def tune_batch(instances, with_grad=False, scale=0.1, candidates=None, reps=1, key=None):
    """Times one replay of the batch graph under each scheduling candidate; returns (best, timings)."""
    import torch
    from .qaoa import Batch
    key = key or ("batch", len(instances), bool(with_grad),
                  tuple(int(d["n"]) for d in instances[:64]), tuple(int(d["p"]) for d in instances[:64]))
    if key in _cache:
        return _cache[key]
    stream = torch.cuda.current_stream()
    timings = []
    for opts in candidates or batch_candidates():
        b = Batch(instances, scale=scale, with_grad=with_grad, opts=opts)
        try:
            ms = _time_ms(b.run, stream, reps)
        finally:
            b.close()
        timings.append(dict(opts=opts, ms=ms))
    best = min(timings, key=lambda t: t["ms"])
    _cache[key] = (best, timings)
    return best, timings
