"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only draws numbers: graphs, integer edge weights, schedule
parameters and the uniforms that decide measurement shots. It holds none of
the simulation arithmetic, so both the CUDA path and the oracle can be fed from
it without sharing any of the method.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), used
as a counter-based generator: the k-th draw of stream ``seed`` is
``mix(seed + (k + 1) * 0x9E3779B97F4A7C15)``. A draw becomes a double in
[0, 1) as ``(x >> 11) * 2**-53``.

The instances stand in for the paper's problem set (Sec. II-G: fully connected
weighted MaxCut, weights uniform on [0, 1]), which is not shipped with the
paper. Weights here are integers in {1..10}; the phases scale them by 1/10.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of the SplitMix64 stream ``seed``."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` doubles in [0, 1) from stream ``seed`` (53-bit mantissa draw)."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _weights(seed: int, m: int, wmax: int = 10) -> np.ndarray:
    return (1 + np.floor(uniforms(seed, m) * wmax)).astype(np.int32)


def complete_graph(n: int, seed: int, wmax: int = 10):
    """K_n with edges (i, j), i < j, in lexicographic order; weights in {1..wmax}."""
    iu, ju = np.triu_indices(n, k=1)
    u = iu.astype(np.int32)
    v = ju.astype(np.int32)
    return u, v, _weights(seed, len(u), wmax)


def chain_graph(n: int, seed: int, wmax: int = 10):
    """Path 0-1-...-(n-1); weights in {1..wmax}."""
    u = np.arange(n - 1, dtype=np.int32)
    v = u + 1
    return u, v, _weights(seed, n - 1, wmax)


def regular3_graph(n: int, seed: int, wmax: int = 10, max_tries: int = 10000):
    """Random 3-regular graph on an even number of vertices by the pairing model.

    Three stubs per vertex are shuffled and paired; a draw with a self loop or a
    repeated edge is rejected and redrawn. Edges are returned in lexicographic
    order. Weights are drawn from stream ``seed + 1``.
    """
    if n % 2 or n < 4:
        raise ValueError("3-regular graphs need an even n >= 4")
    stubs = np.repeat(np.arange(n, dtype=np.int64), 3)
    for t in range(max_tries):
        keys = splitmix64(seed, len(stubs), offset=t * len(stubs))
        perm = stubs[np.argsort(keys, kind="stable")]
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        code = lo * n + hi
        if len(np.unique(code)) != len(code):
            continue
        order = np.argsort(code)
        u, v = lo[order].astype(np.int32), hi[order].astype(np.int32)
        return u, v, _weights(seed + 1, len(u), wmax)
    raise RuntimeError("pairing model did not produce a simple graph")


def batch_instances(count: int, seed: int, n_lo: int = 10, n_hi: int = 22,
                    p_lo: int = 1, p_hi: int = 10,
                    dgamma_range=(0.2, 1.2), dbeta_range=(0.1, 0.6)):
    """Mixed batch: 1/3 complete, 1/3 chain, 1/3 random 3-regular graphs.

    Per instance: n uniform in [n_lo, n_hi], p uniform in [p_lo, p_hi], graph
    class by index mod 3, dgamma and dbeta uniform in the given ranges. The
    3-regular class rounds an odd n up to the next even value (n_hi if that
    would exceed it), since 3-regular graphs need an even vertex count.
    """
    d = uniforms(seed, 4 * count).reshape(count, 4)
    out = []
    for i in range(count):
        n = n_lo + int(d[i, 0] * (n_hi - n_lo + 1))
        p = p_lo + int(d[i, 1] * (p_hi - p_lo + 1))
        dg = dgamma_range[0] + d[i, 2] * (dgamma_range[1] - dgamma_range[0])
        db = dbeta_range[0] + d[i, 3] * (dbeta_range[1] - dbeta_range[0])
        kind = i % 3
        gseed = seed * 1_000_003 + i
        if kind == 0:
            u, v, w = complete_graph(n, gseed)
        elif kind == 1:
            u, v, w = chain_graph(n, gseed)
        else:
            if n % 2:
                n = n + 1 if n + 1 <= n_hi else n - 1
            u, v, w = regular3_graph(n, gseed)
        out.append(dict(n=n, p=p, dgamma=float(dg), dbeta=float(db), kind=("complete", "chain", "3-regular")[kind],
                        u=u, v=v, w=w))
    return out
