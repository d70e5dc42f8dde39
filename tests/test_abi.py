"""CPU tests of the C ABI library: it loads, exports every declared symbol,
rejects invalid arguments before touching a GPU, and plans validly."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2604_26423_b300 import build, qaoa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return qaoa.load()


def declared_symbols():
    syms = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            syms |= set(re.findall(r"\b(qaoa_\w+)\s*\(", text))
    return syms


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert "qaoa_init_graph" in syms and "qaoa_run" in syms
    for s in syms:
        assert hasattr(lib, s), s
    assert set(qaoa.EXPORTS) <= syms


def test_sizes(lib):
    assert qaoa.state_bytes(33, "c64") == 64 << 30          # 2^(N+3) bytes in FP32 (Sec. II-E)
    assert qaoa.state_bytes(32, "c128") == 64 << 30
    assert qaoa.state_bytes(35, "c64") == 0
    assert qaoa.state_bytes(0, "c64") == 0
    assert qaoa.aux_bytes(20, "c64", "stream", False) == 4 << 20
    assert qaoa.aux_bytes(20, "c64", "recompute", True) == 8 << 20


def _init(lib, n, u, v, w, scale=0.1, prec=0, mode=1):
    ctx = ctypes.c_void_p()
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    P = ctypes.POINTER(ctypes.c_int32)
    rc = lib.qaoa_init_graph(ctypes.byref(ctx), n, len(u), u.ctypes.data_as(P), v.ctypes.data_as(P),
                             w.ctypes.data_as(P), scale, prec, mode, None, 0, None, 0, None)
    return rc, ctx, lib.qaoa_last_error(None).decode()


@pytest.mark.parametrize("n,u,v,w,scale,prec,mode,word", [
    (5, [0], [0], [1], 0.1, 0, 1, "self loop"),
    (5, [0], [5], [1], 0.1, 0, 1, "out of range"),
    (5, [0, 1], [1, 0], [1, 2], 0.1, 0, 1, "repeated"),
    (5, [0], [1], [0], 0.1, 0, 1, "zero weight"),
    (5, [0], [1], [1], -1.0, 0, 1, "weight_scale"),
    (0, [], [], [], 0.1, 0, 1, "n out of range"),
    (35, [], [], [], 0.1, 0, 1, "n out of range"),
    (34, [], [], [], 0.1, 1, 1, "n out of range"),
    (5, [0], [1], [1], 0.1, 7, 1, "precision"),
    (5, [0], [1], [1], 0.1, 0, 9, "cost_mode"),
    (5, [0, 1], [1, 2], [1 << 20, 1], 0.1, 0, 1, "exceeds"),
])
def test_invalid_graphs_rejected(lib, n, u, v, w, scale, prec, mode, word):
    rc, ctx, msg = _init(lib, n, u, v, w, scale, prec, mode)
    assert rc == qaoa.QAOA_EINVAL
    assert not ctx.value
    assert word in msg


def test_null_context_calls(lib):
    assert lib.qaoa_run(None, 1, 0.1, 0.1) == qaoa.QAOA_EINVAL
    lib.qaoa_free(None)


@pytest.mark.parametrize("n", [13, 16, 24, 28, 30, 33, 34])
@pytest.mark.parametrize("p", [0, 1, 3, 10])
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_plans_valid(lib, n, p, prec):
    text = qaoa.describe_plan(n, p, prec)
    assert "INVALID" not in text and not text.startswith("error"), text[:500]
    passes = int(re.search(r"passes=(\d+)", text).group(1))
    groups = int(re.search(r"groups=(\d+)", text).group(1))
    if p == 0:
        assert passes == 1
    elif groups > 1:
        assert passes == 1 + p * (groups - 1)   # cross-layer fusion
    else:
        assert passes == p


def test_n33_groups(lib, monkeypatch):
    # default complex64 tile at 33 qubits: 5x4 (2^14 amplitudes, 128-byte runs)
    # -> 3 qubit groups and 7 HBM passes at p = 3; the 4x3 tile (2^12
    # amplitudes, 256-byte runs) -> 4 groups and 10 passes, or with 2^15
    # super-tiles through L2 3 groups and 7 passes
    assert "T=14" in qaoa.describe_plan(33, 3, "c64") and "groups=3 passes=7" in qaoa.describe_plan(33, 3, "c64")
    monkeypatch.setenv("QAOA_FWD_SHAPE", "4x3")
    assert "groups=4 passes=10" in qaoa.describe_plan(33, 3, "c64")
    monkeypatch.setenv("QAOA_SMAX", "15")
    assert "groups=3 passes=7" in qaoa.describe_plan(33, 3, "c64")


def test_default_tile_by_size(lib):
    # 5x4 only where it takes fewer mixer groups than 4x3 (29..34 qubits)
    for n in range(16, 35):
        t = qaoa.describe_plan(n, 3, "c64").splitlines()[0]
        assert ("T=14" in t) == (29 <= n <= 34), t
    assert "T=12" in qaoa.describe_plan(33, 3, "c128").splitlines()[0]


@pytest.mark.parametrize("n", [12, 16, 24, 28, 33])
@pytest.mark.parametrize("p", [1, 3, 5, 20])
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_adjoint_plans_valid(lib, n, p, prec):
    text = qaoa.describe_plan(n, p, prec, adjoint=True)
    assert "INVALID" not in text and not text.startswith("error"), text[:800]
    assert " lambda" in text.splitlines()[2 + text.count("group ")] or "lambda" in text
    assert "nostore" in text.splitlines()[-1] or "nostore" in text
    passes = int(re.search(r"passes=(\d+)", text).group(1))
    groups = int(re.search(r"groups=(\d+)", text).group(1))
    assert passes == (1 + p * (groups - 1) if groups > 1 else p)


def test_adjoint_group_counts(lib, monkeypatch):
    # one tile of psi and lambda per CTA (2^12 amplitudes): 3 groups at 24 and
    # 28 qubits, 4 at 33; with 2^14 super-tiles through L2: 2, 3 and 3
    got = [int(re.search(r"groups=(\d+)", qaoa.describe_plan(n, 5, "c64", adjoint=True)).group(1))
           for n in (24, 28, 33)]
    assert got == [3, 3, 4]
    monkeypatch.setenv("QAOA_SMAX_ADJ", "14")
    got = [int(re.search(r"groups=(\d+)", qaoa.describe_plan(n, 5, "c64", adjoint=True)).group(1))
           for n in (24, 28, 33)]
    assert got == [2, 3, 3]


def test_classify_regime_matches_oracle(lib):
    # host-only entry point: the regime rule on a grid of observations
    import oracle
    for r_obs in np.linspace(0.6, 1.0, 81):
        for rs in (0.0, 0.004, 0.02):
            for ideal in ((None, None), (0.88, 0.01), (0.81, 0.03)):
                a = qaoa.classify_regime(r_obs, 0.79, rs, *ideal)
                b = oracle.classify_regime(float(r_obs), 0.79, rs, *ideal)
                assert a == b, (r_obs, rs, ideal)
    assert qaoa.classify_regime(0.9, 0.79, float("nan")) == -1


def test_mean_of_means_rejects_bad_sizes(lib):
    # argument checks come before any device work
    vp = ctypes.c_void_p
    one = vp(16)
    assert lib.qaoa_mean_of_means(None, 10, 2, 2, 0, one, one, None) == qaoa.QAOA_EINVAL
    assert lib.qaoa_mean_of_means(one, 10, 11, 2, 0, one, one, None) == qaoa.QAOA_EINVAL
    assert lib.qaoa_mean_of_means(one, 10, 0, 2, 0, one, one, None) == qaoa.QAOA_EINVAL
    assert lib.qaoa_mean_of_means(one, 10000, 4097, 2, 0, one, one, None) == qaoa.QAOA_EINVAL
    assert lib.qaoa_mean_of_means(one, 10, 2, 0, 0, one, one, None) == qaoa.QAOA_EINVAL
    assert lib.qaoa_mean_of_means(one, 1 << 32, 2, 2, 0, one, one, None) == qaoa.QAOA_EINVAL
    assert lib.qaoa_sample_cuts(None, 1, None, 0, None, None, None) == qaoa.QAOA_EINVAL


def test_overlap_and_k0_match_oracle(lib):
    import oracle
    assert qaoa.overlap_ratio(0.85, 0.9, 0.8) == oracle.overlap_ratio(0.85, 0.9, 0.8)
    a = np.array([0.05, 0.3, 0.7, 1.1, 2.5])
    r = np.array([0.97, 0.8, 0.61, 0.4, -0.02])
    assert abs(qaoa.fit_k0(a, r) - oracle.fit_k0(a, r)) < 1e-14
    assert np.isnan(qaoa.fit_k0([1.0], [-1.0]))


def test_weight_limits_and_quantisation(lib):
    assert qaoa.max_weight_sum(33, "c64") == (1 << 30) - 1
    assert qaoa.max_weight_sum(12, "c64") == 1 << 20
    assert qaoa.max_weight_sum(20, "c128") == 1 << 20
    w = np.concatenate([inputs_uniforms(3, 500), [1e-3, -0.7]])
    for limit in ((1 << 30) - 1, 1 << 20):
        wi, unit = qaoa.quantize_weights(w, limit)
        assert np.abs(wi).sum() <= limit
        assert np.max(np.abs(wi * unit - w)) <= 0.5 * unit * (1 + 1e-12)
        assert np.all(np.sign(wi) == np.sign(w))
    with pytest.raises(qaoa.QaoaError):
        qaoa.quantize_weights([1.0, 0.0], 1 << 20)
    with pytest.raises(qaoa.QaoaError):
        qaoa.quantize_weights([1.0, float("nan")], 1 << 20)
    with pytest.raises(qaoa.QaoaError):
        qaoa.quantize_weights([1.0, 1e-9], 1 << 20)   # below half a unit
    # the limit is enforced at init: 2^20 + 1 on a table path
    rc, ctx, msg = _init(lib, 5, [0, 1], [1, 2], [1 << 20, 1], 0.1, 0, 1)
    assert rc == qaoa.QAOA_EINVAL and "exceeds" in msg


def inputs_uniforms(seed, count):
    from paper_2604_26423_b300 import inputs
    return inputs.uniforms(seed, count)


@pytest.mark.parametrize("shape", ["4x3", "5x4"])
def test_paired_global_layout(lib, monkeypatch, shape):
    # complex64 forward plans load and store through the paired layout
    # (register bit 0 on index bit 0, lanes on bits 1..5) where a shortest
    # round sequence allows it; every plan stays valid; QAOA_PAIRED=0 and the
    # adjoint plans keep 8-byte accesses
    monkeypatch.setenv("QAOA_FWD_SHAPE", shape)
    paired_round = re.compile(r"round src=\d dst=\d reg=0,[^ ]* lane=1,2,3,4,5 ")
    for n in (29, 30, 33):
        text = qaoa.describe_plan(n, 3, "c64")
        assert "INVALID" not in text and paired_round.search(text), n
        assert not paired_round.search(qaoa.describe_plan(n, 3, "c64", adjoint=True))
        assert not paired_round.search(qaoa.describe_plan(n, 3, "c128"))
    monkeypatch.setenv("QAOA_PAIRED", "0")
    assert not paired_round.search(qaoa.describe_plan(33, 3, "c64"))
