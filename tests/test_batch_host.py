"""CPU tests of qaoa_batch_create's argument checks (they run before any CUDA
call) and of the batch workload generator."""
import ctypes

import numpy as np
import pytest

from paper_2604_26423_b300 import build, inputs, qaoa


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return qaoa.load()


def _create(lib, n, p, edges, dg=None, db=None, scale=0.1):
    count = len(n)
    n = np.asarray(n, dtype=np.int32)
    p = np.asarray(p, dtype=np.int32)
    off = np.zeros(count + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(e) for e in edges])
    flat = [x for e in edges for x in e] or [(0, 1, 1)]
    u = np.array([x[0] for x in flat], dtype=np.int32)
    v = np.array([x[1] for x in flat], dtype=np.int32)
    w = np.array([x[2] for x in flat], dtype=np.int32)
    dg = np.full(count, 0.6) if dg is None else np.asarray(dg, dtype=np.float64)
    db = np.full(count, 0.3) if db is None else np.asarray(db, dtype=np.float64)
    P = ctypes.POINTER
    ip = lambda a: a.ctypes.data_as(P(ctypes.c_int32))
    h = ctypes.c_void_p()
    rc = lib.qaoa_batch_create(ctypes.byref(h), count, ip(n), ip(p), off.ctypes.data_as(P(ctypes.c_int64)),
                               ip(u), ip(v), ip(w), dg.ctypes.data_as(P(ctypes.c_double)),
                               db.ctypes.data_as(P(ctypes.c_double)), scale, 0, None, None)
    return rc, lib.qaoa_batch_last_error(None).decode()


@pytest.mark.parametrize("case,expect", [
    (dict(n=[1], p=[1], edges=[[]]), "n out of"),
    (dict(n=[25], p=[1], edges=[[(0, 1, 1)]]), "n out of"),
    (dict(n=[4], p=[0], edges=[[(0, 1, 1)]]), "p out of"),
    (dict(n=[4], p=[65], edges=[[(0, 1, 1)]]), "p out of"),
    (dict(n=[4, 4], p=[1, 1], edges=[[(0, 1, 1)], [(2, 2, 1)]]), "self loop"),
    (dict(n=[4], p=[1], edges=[[(0, 4, 1)]]), "out of range"),
    (dict(n=[4], p=[1], edges=[[(0, 1, 1), (1, 0, 2)]]), "repeated edge"),
    (dict(n=[4], p=[1], edges=[[(0, 1, 0)]]), "zero weight"),
    (dict(n=[4], p=[1], edges=[[(0, 1, 1)]], dg=[np.nan]), "finite"),
    (dict(n=[4], p=[1], edges=[[(0, 1, 1)]], scale=0.0), "weight_scale"),
])
def test_create_rejects(lib, case, expect):
    rc, msg = _create(lib, **case)
    assert rc == qaoa.QAOA_EINVAL
    assert expect in msg


def test_create_rejects_null_output(lib):
    n = np.array([4], dtype=np.int32)
    rc = lib.qaoa_batch_create(None, 1, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, None, None, None,
                               None, None, None, 0.1, 0, None, None)
    assert rc == qaoa.QAOA_EINVAL


def test_batch_instances_shape():
    b = inputs.batch_instances(300, 7)
    assert len(b) == 300
    kinds = [d["kind"] for d in b]
    assert kinds.count("complete") == kinds.count("chain") == kinds.count("3-regular") == 100
    for d in b:
        assert 10 <= d["n"] <= 22 and 1 <= d["p"] <= 10
        assert 0.2 <= d["dgamma"] <= 1.2 and 0.1 <= d["dbeta"] <= 0.6
        m = len(d["u"])
        if d["kind"] == "complete":
            assert m == d["n"] * (d["n"] - 1) // 2
        elif d["kind"] == "chain":
            assert m == d["n"] - 1
        else:
            assert d["n"] % 2 == 0 and m == 3 * d["n"] // 2
            deg = np.bincount(np.concatenate([d["u"], d["v"]]), minlength=d["n"])
            assert (deg == 3).all()
        assert ((np.asarray(d["w"]) >= 1) & (np.asarray(d["w"]) <= 10)).all()


def test_tuner_candidates():
    from paper_2604_26423_b300 import tune
    c = tune.forward_candidates(33, "c64")
    assert {"cost_mode": "recompute", "shape": "5x3", "super_tile": 13, "order": "last", "float_lanes": 1,
            "l2_prefetch": 0} in c
    assert {"cost_mode": "recompute", "shape": "5x3", "super_tile": 13, "order": "last", "float_lanes": 0,
            "l2_prefetch": 1} in c
    assert all(x["super_tile"] <= 33 for x in c)
    assert {x["shape"] for x in tune.forward_candidates(30, "c128")} == {"4x3", "5x3"}
    assert "5x4" in {x["shape"] for x in c}
    opts = tune.config_opts({"cost_mode": "stream", "shape": "4x4", "super_tile": 14, "order": "middle",
                             "float_lanes": 0})
    assert opts == {"shape": "4x4", "super_tile": 14, "order": "middle", "float_lanes": False, "l2_prefetch": False}
    o = qaoa.make_opts(**opts)
    assert (o.fwd_shape, o.super_tile, o.group_order, o.float_lanes) == (qaoa.SHAPES["4x4"], 14, 2, qaoa.OFF)
    assert qaoa.make_opts().fwd_shape == 0 and qaoa.make_opts(specialised=True).specialised == qaoa.ON
    b = tune.batch_candidates(solo=(16,), units=(1, 2), ctas=(2,), shapes=("5x3",), modes=("recompute",))
    assert b == [dict(solo_max_n=16, max_units=1, ctas_per_sm=2, fwd_shape="5x3", cost_mode="recompute"),
                 dict(solo_max_n=16, max_units=2, ctas_per_sm=2, fwd_shape="5x3", cost_mode="recompute")]
    assert len(tune.batch_candidates(solo=(16,), units=(1,))) == 4


def test_group_orders_give_valid_plans():
    # both group orders, with and without floating lane bits, both main tile
    # shapes, plan every size validly (checked by the planner's validator)
    import itertools
    import os
    from paper_2604_26423_b300 import qaoa
    for order, fl, shape in itertools.product(("last", "middle"), ("0", "1"), ("4x3", "5x3")):
        if True:
            os.environ["QAOA_GROUP_ORDER"] = order
            os.environ["QAOA_FLOAT_LANES"] = fl
            os.environ["QAOA_FWD_SHAPE"] = shape
            try:
                for n in (13, 14, 20, 22, 26, 30, 33, 34):
                    for p in (1, 2, 3, 4):
                        for adj in (False, True):
                            for prec in ("c64", "c128"):
                                d = qaoa.describe_plan(n, p, prec, adjoint=adj)
                                assert "passes=" in d and "INVALID" not in d and "error" not in d, d
            finally:
                os.environ.pop("QAOA_GROUP_ORDER", None)
                os.environ.pop("QAOA_FLOAT_LANES", None)
                os.environ.pop("QAOA_FWD_SHAPE", None)


def test_float_lanes_plan_shape():
    # n = 33, p = 3: the coalescing bits 0..4 leave the low group; each layer
    # applies them once in a plain pass on a high group; the fused low-group pass
    # and the final pass lose a shared-memory round trip each; the pass count
    # is unchanged
    # (5x3 tile shape: T = 13, 2^5 registers per thread)
    import os
    import re
    from paper_2604_26423_b300 import qaoa
    os.environ["QAOA_FWD_SHAPE"] = "5x3"
    try:
        os.environ["QAOA_FLOAT_LANES"] = "1"
        d = qaoa.describe_plan(33, 3, "c64")
        os.environ["QAOA_FLOAT_LANES"] = "0"
        d0 = qaoa.describe_plan(33, 3, "c64")
    finally:
        os.environ.pop("QAOA_FLOAT_LANES", None)
        os.environ.pop("QAOA_FWD_SHAPE", None)
    assert "float_lanes=5" in d and "float_lanes" not in d0
    assert "group 0: 5 6 7 8 9 10 11 12\n" in d
    assert "passes=10" in d and "passes=10" in d0

    def rounds(desc):
        out, cur = [], None
        for line in desc.splitlines():
            if line.startswith("pass "):
                cur = [line, 0, 0]
                out.append(cur)
            m = re.match(r"  sub \d+ tile=.* nA=(\d+) nB=(\d+)", line)
            if m:
                cur[2] += int(m.group(1)) + int(m.group(2))
            if line.startswith("    round"):
                cur[1] += 1
        return out
    r1, r0 = rounds(d), rounds(d0)
    # total butterflies per amplitude and layer count unchanged: 33 qubits x 3 layers
    assert sum(x[2] for x in r1) == sum(x[2] for x in r0) == 99
    fused = [i for i, x in enumerate(r1) if " c=" in x[0] and " c=-1" not in x[0] and "init" not in x[0]]
    for i in fused + [len(r1) - 1]:
        assert r1[i][1] <= r0[i][1]
    assert r1[3][1] == 3 and r0[3][1] == 5 and r1[9][1] == 2 and r0[9][1] == 3
