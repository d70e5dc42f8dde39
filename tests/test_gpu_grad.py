"""Adjoint gradient on the GPU vs the oracle's exact parameter-shift gradient
and central finite differences.

Tolerances: complex128 adjoint vs oracle parameter shift (exact up to
rounding): 1e-8 relative to the largest component; vs central differences of
the oracle's complex128 <C> (h = 1e-5, K_24) or, at K_28, of the GPU's own
complex128 forward: 1e-6 relative. complex64 adjoint
vs the complex128 adjoint: 2e-3 relative (single-precision state, gradient
components are sums of ~2^n terms of mixed sign).
"""
import numpy as np
import pytest

import oracle
from paper_2604_26423_b300 import inputs

pytestmark = pytest.mark.gpu
S = 0.1


def sim(*a, **k):
    from paper_2604_26423_b300.qaoa import Simulator
    return Simulator(*a, **k)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / max(1e-30, np.max(np.abs(b)))


@pytest.mark.parametrize("n,p,density", [(4, 1, 1.0), (7, 2, 0.6), (9, 3, 1.0), (10, 2, 0.5)])
def test_grad_small_vs_param_shift(n, p, density):
    u, v, w = inputs.complete_graph(n, 900 + n)
    if density < 1:
        keep = inputs.uniforms(901 + n, len(u)) < density
        keep[0] = True
        u, v, w = u[keep], v[keep], w[keep]
    g, b = oracle.lr_schedule(p, 0.6, 0.3)
    ps_g, ps_b = oracle.grad_param_shift(n, u, v, w, S, g, b)
    with sim(n, u, v, w, S, "c128") as s:
        out = s.grad_angles(g, b)
    scale = max(np.max(np.abs(ps_g)), np.max(np.abs(ps_b)))
    assert np.max(np.abs(out["g_gamma"] - ps_g)) <= 1e-8 * scale
    assert np.max(np.abs(out["g_beta"] - ps_b)) <= 1e-8 * scale


@pytest.mark.parametrize("n,p,prec", [(12, 2, "c128"), (13, 3, "c128"), (15, 2, "c128"), (16, 3, "c128"),
                                      (17, 2, "c128"), (20, 3, "c128")])
def test_grad_pass_kernel_vs_oracle_fd(n, p, prec):
    u, v, w = inputs.complete_graph(n, 950 + n)
    g, b = oracle.lr_schedule(p, 0.6, 0.3)
    fd_g, fd_b = oracle.grad_fd(n, u, v, w, S, g, b)
    with sim(n, u, v, w, S, prec) as s:
        out = s.grad_angles(g, b)
        ref = oracle.run(n, u, v, w, S, g, b)
    scale = max(np.max(np.abs(fd_g)), np.max(np.abs(fd_b)))
    assert np.max(np.abs(out["g_gamma"] - fd_g)) <= 1e-6 * scale
    assert np.max(np.abs(out["g_beta"] - fd_b)) <= 1e-6 * scale
    assert abs(out["exp_c"] - ref["exp_c"]) <= 1e-10 * ref["exp_c"]


@pytest.mark.parametrize("n", [14, 18])
def test_grad_wide_angles_and_stream_mode(n):
    # |beta| > pi/4 takes the plain butterfly form; stream mode reads the diagonal
    u, v, w = inputs.complete_graph(n, 960 + n)
    gamma = np.array([0.4, -0.9, 1.7])
    beta = np.array([1.1, 0.3, -2.4])
    fd_g, fd_b = oracle.grad_fd(n, u, v, w, S, gamma, beta)
    scale = max(np.max(np.abs(fd_g)), np.max(np.abs(fd_b)))
    for mode in ("recompute", "stream"):
        with sim(n, u, v, w, S, "c128", cost_mode=mode) as s:
            out = s.grad_angles(gamma, beta)
        assert np.max(np.abs(out["g_gamma"] - fd_g)) <= 1e-6 * scale, mode
        assert np.max(np.abs(out["g_beta"] - fd_b)) <= 1e-6 * scale, mode


def test_grad_k24_vs_oracle_fd():
    # n = 24, K_24, p = 5 (the gradient workload's smaller size): the
    # complex128 adjoint's d<C>/d(dgamma, dbeta) against central differences
    # (h = 1e-5) of the oracle's gate-by-gate complex128 <C> (four oracle runs)
    n, p = 24, 5
    u, v, w = inputs.complete_graph(n, 970 + n)
    dg, db, h = 0.6, 0.3, 1e-5
    cut = oracle.cut_values(n, u, v, w)

    def f(a, bb):
        return oracle.expectation(oracle.simulate(n, u, v, w, S, *oracle.lr_schedule(p, a, bb)), cut)[0]

    fdg = (f(dg + h, db) - f(dg - h, db)) / (2 * h)
    fdb = (f(dg, db + h) - f(dg, db - h)) / (2 * h)
    with sim(n, u, v, w, S, "c128", with_grad=True) as s:
        out = s.grad(p, dg, db)
    scale = max(abs(fdg), abs(fdb))
    err = max(abs(out["d_dgamma"] - fdg), abs(out["d_dbeta"] - fdb)) / scale
    print(f"\nK_24 p=5 c128 adjoint vs oracle FD: relative error {err:.2e}")
    assert err <= 1e-6


def test_grad_k28_vs_gpu_fd():
    # n = 28, K_28, p = 5: against central differences of the GPU's own
    # complex128 forward (a self-consistency check between the adjoint and the
    # forward kernels; the oracle would take minutes per evaluation here)
    n, p = 28, 5
    u, v, w = inputs.complete_graph(n, 970 + n)
    dg, db, h = 0.6, 0.3, 1e-5
    with sim(n, u, v, w, S, "c128", with_grad=True) as s:
        out = s.grad(p, dg, db)

        def f(a, bb):
            s.run(p, a, bb)
            return s.expect()["exp_c"]

        fdg = (f(dg + h, db) - f(dg - h, db)) / (2 * h)
        fdb = (f(dg, db + h) - f(dg, db - h)) / (2 * h)
    assert abs(out["d_dgamma"] - fdg) <= 1e-6 * max(abs(fdg), abs(fdb))
    assert abs(out["d_dbeta"] - fdb) <= 1e-6 * max(abs(fdg), abs(fdb))


@pytest.mark.parametrize("n,p", [(16, 3), (22, 5)])
def test_grad_c64_vs_c128(n, p):
    u, v, w = inputs.complete_graph(n, 980 + n)
    outs = {}
    for prec in ("c128", "c64"):
        with sim(n, u, v, w, S, prec) as s:
            outs[prec] = s.grad(p, 0.6, 0.3)
    ref = np.concatenate([outs["c128"]["g_gamma"], outs["c128"]["g_beta"]])
    got = np.concatenate([outs["c64"]["g_gamma"], outs["c64"]["g_beta"]])
    d_ref = np.array([outs["c128"]["d_dgamma"], outs["c128"]["d_dbeta"]])
    d_got = np.array([outs["c64"]["d_dgamma"], outs["c64"]["d_dbeta"]])
    print(f"\nK_{n} p={p} c64 gradient vs c128: per-layer {rel(got, ref):.2e}, "
          f"d/d(dgamma, dbeta) {rel(d_got, d_ref):.2e} (relative to the largest component)")
    assert rel(got, ref) <= 2e-3
    assert abs(outs["c64"]["exp_c"] - outs["c128"]["exp_c"]) <= 2e-5 * outs["c128"]["exp_c"]


def test_lr_chain_rule_matches_oracle():
    n, p = 8, 3
    u, v, w = inputs.complete_graph(n, 990)
    gg, gb = oracle.grad_param_shift(n, u, v, w, S, *oracle.lr_schedule(p, 0.6, 0.3))
    cdg, cdb = oracle.lr_chain(gg, gb)
    with sim(n, u, v, w, S, "c128") as s:
        out = s.grad(p, 0.6, 0.3)
    assert abs(out["d_dgamma"] - cdg) <= 1e-8 * abs(cdg)
    assert abs(out["d_dbeta"] - cdb) <= 1e-8 * abs(cdb)


def test_state_after_grad_needs_rerun():
    from paper_2604_26423_b300.qaoa import QaoaError
    n = 14
    u, v, w = inputs.complete_graph(n, 995)
    with sim(n, u, v, w, S, "c64") as s:
        s.grad(2, 0.6, 0.3)
        with pytest.raises(QaoaError):
            s.sample(8)
        s.run(2, 0.6, 0.3)
        assert len(s.sample(8)) == 8


def test_autograd_function_matches_adjoint_and_fd():
    import torch
    from paper_2604_26423_b300.autograd import lr_expectation, expectation
    n, p = 14, 4
    u, v, w = inputs.complete_graph(n, 1414)
    with sim(n, u, v, w, 0.1, "c128", with_grad=True) as s:
        dg = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
        db = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
        e = lr_expectation(s, p, dg, db)
        e.backward()
        ref = s.grad(p, 0.6, 0.3)
        assert abs(e.item() - ref["exp_c"]) <= 1e-9 * abs(ref["exp_c"])
        assert abs(dg.grad.item() - ref["d_dgamma"]) <= 1e-9 * max(1.0, abs(ref["d_dgamma"]))
        assert abs(db.grad.item() - ref["d_dbeta"]) <= 1e-9 * max(1.0, abs(ref["d_dbeta"]))
        # FP64 central differences of the oracle in (dgamma, dbeta)
        h = 1e-5
        cut = oracle.cut_values(n, u, v, w)
        f = lambda a, b: oracle.expectation(oracle.simulate(n, u, v, w, 0.1, *oracle.lr_schedule(p, a, b)), cut)[0]
        fd_g = (f(0.6 + h, 0.3) - f(0.6 - h, 0.3)) / (2 * h)
        fd_b = (f(0.6, 0.3 + h) - f(0.6, 0.3 - h)) / (2 * h)
        assert abs(dg.grad.item() - fd_g) <= 1e-6 * max(1.0, abs(fd_g))
        assert abs(db.grad.item() - fd_b) <= 1e-6 * max(1.0, abs(fd_b))
        # explicit angles: gradient per layer
        g = torch.tensor([0.1, 0.2, 0.35, 0.5], dtype=torch.float64, requires_grad=True)
        b = torch.tensor([0.4, 0.3, 0.2, 0.1], dtype=torch.float64, requires_grad=True)
        expectation(s, g, b).backward()
        r2 = s.grad_angles(g.detach().numpy(), b.detach().numpy())
        assert np.allclose(g.grad.numpy(), r2["g_gamma"], rtol=1e-12, atol=1e-12)
        assert np.allclose(b.grad.numpy(), r2["g_beta"], rtol=1e-12, atol=1e-12)
        # no gradient requested: plain forward
        with torch.no_grad():
            e2 = lr_expectation(s, p, torch.tensor(0.6, dtype=torch.float64), torch.tensor(0.3, dtype=torch.float64))
        assert abs(e2.item() - ref["exp_c"]) <= 1e-9 * abs(ref["exp_c"])


def test_grad_exp_c_matches_forward_and_expect_needs_rerun():
    from paper_2604_26423_b300.qaoa import QaoaError
    n, p = 20, 3
    u, v, w = inputs.complete_graph(n, 2020)
    with sim(n, u, v, w, S, "c64", with_grad=True) as s:
        s.run(p, 0.6, 0.3)
        e = s.expect()["exp_c"]
        g = s.grad(p, 0.6, 0.3)
        assert abs(g["exp_c"] - e) <= 2e-6 * e
        with pytest.raises(QaoaError):
            s.expect()


@pytest.mark.gpu
@pytest.mark.parametrize("n,p", [(20, 3), (24, 5)])
def test_specialised_adjoint_kernels_identical(n, p, monkeypatch):
    # the specialised adjoint kernels do the generic kernel's arithmetic:
    # identical gradients
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import Simulator
    u, v, w = inputs.complete_graph(n, 900 + n)
    res = []
    for spec in ("1", "0"):
        monkeypatch.setenv("QAOA_SPEC", spec)
        with Simulator(n, u, v, w, 0.1, "c64", with_grad=True) as s:
            res.append(s.grad(p, 0.6, 0.3))
    a, b = res
    assert np.array_equal(a["g_gamma"], b["g_gamma"]) and np.array_equal(a["g_beta"], b["g_beta"])
    assert a["exp_c"] == b["exp_c"]


@pytest.mark.gpu
def test_adjoint_tile_prefetch_identical(monkeypatch):
    # asynchronous copies of the next tile (optional) give the same gradients
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import Simulator
    n, p = 22, 3
    u, v, w = inputs.complete_graph(n, 922)
    res = []
    for pf in ("1", "0"):
        monkeypatch.setenv("QAOA_ADJ_PREFETCH", pf)
        with Simulator(n, u, v, w, 0.1, "c64", with_grad=True) as s:
            res.append(s.grad(p, 0.6, 0.3))
    a, b = res
    assert np.array_equal(a["g_gamma"], b["g_gamma"]) and np.array_equal(a["g_beta"], b["g_beta"])


@pytest.mark.gpu
@pytest.mark.parametrize("ckpt", [True, False])
@pytest.mark.parametrize("n,p", [(22, 3), (26, 2)])
def test_adjoint_tma_tile_loads_identical(n, p, ckpt, monkeypatch):
    # psi and lambda tiles loaded into shared memory by tensor loads (issued
    # from the previous tile's last round) carry the same amplitudes as the
    # global loads: bitwise identical gradients and <C>, with stored forward
    # states and with psi uncomputed
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import Simulator
    u, v, w = inputs.complete_graph(n, 940 + n)
    res = []
    for tl in ("1", "0"):
        monkeypatch.setenv("QAOA_ADJ_TMA_LOAD", tl)
        with Simulator(n, u, v, w, 0.1, "c64", with_grad=True, opts=dict(grad_checkpoint=ckpt)) as s:
            res.append(s.grad(p, 0.6, 0.3))
    a, b = res
    assert np.array_equal(a["g_gamma"], b["g_gamma"]) and np.array_equal(a["g_beta"], b["g_beta"])
    assert a["exp_c"] == b["exp_c"]


@pytest.mark.gpu
def test_adjoint_tma_wait_limit_gives_etimeout_then_recovers(monkeypatch):
    # a 1 ns limit makes the adjoint's tensor-load waits give up: qaoa_grad
    # reports ETIMEOUT, and the next gradient on the same device is correct
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import QAOA_ETIMEOUT, QaoaError, Simulator
    n, p = 24, 3
    u, v, w = inputs.complete_graph(n, 1124)
    with Simulator(n, u, v, w, 0.1, "c64", with_grad=True) as s:
        ref = s.grad(p, 0.6, 0.3)
        monkeypatch.setenv("QAOA_TMA_WAIT_NS", "1")
        with pytest.raises(QaoaError) as ei:
            s.grad(p, 0.6, 0.3)
        assert ei.value.code == QAOA_ETIMEOUT
        monkeypatch.delenv("QAOA_TMA_WAIT_NS")
        again = s.grad(p, 0.6, 0.3)
    assert np.array_equal(ref["g_gamma"], again["g_gamma"]) and np.array_equal(ref["g_beta"], again["g_beta"])


@pytest.mark.gpu
@pytest.mark.parametrize("ckpt", [True, False])
@pytest.mark.parametrize("n,p", [(22, 3), (26, 2)])
def test_adjoint_l2_prefetch_identical(n, p, ckpt):
    # tensor prefetches of the next tile of psi and lambda into L2 move no
    # data into the kernel: bitwise identical gradients and <C>, with stored
    # forward states and with psi uncomputed
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import Simulator
    u, v, w = inputs.complete_graph(n, 960 + n)
    res = []
    for pf in (True, False):
        with Simulator(n, u, v, w, 0.1, "c64", with_grad=True,
                       opts=dict(adj_l2_prefetch=pf, grad_checkpoint=ckpt)) as s:
            assert s.get_opts()["adj_l2_prefetch"] == (1 if pf else 2)
            res.append(s.grad(p, 0.6, 0.3))
    a, b = res
    assert np.array_equal(a["g_gamma"], b["g_gamma"]) and np.array_equal(a["g_beta"], b["g_beta"])
    assert a["exp_c"] == b["exp_c"]


@pytest.mark.gpu
@pytest.mark.parametrize("n,p,prec", [(14, 3, "c128"), (21, 1, "c64"), (22, 4, "c64"), (20, 3, "c128"),
                                      (29, 2, "c64")])
def test_grad_stored_forward_states(n, p, prec, monkeypatch):
    # the adjoint reading psi from the forward's stored pass outputs gives the
    # gradients of the adjoint that uncomputes psi, up to rounding, with one
    # state write fewer per adjoint pass (the algorithmic bytes show which
    # path ran); n = 21, p = 1 and n = 29 take the forward plan without
    # floating lane bits so that the adjoint retraces it
    u, v, w = inputs.complete_graph(n, 990 + n)
    res, adj_bytes = [], []
    for ck in ("1", "0"):
        monkeypatch.setenv("QAOA_GRAD_CHECKPOINT", ck)
        with sim(n, u, v, w, S, prec, with_grad=True) as s:
            s.profile(True)
            res.append(s.grad(p, 0.6, 0.3))
            adj_bytes.append(s.profile_read("adjoint")["bytes"])
    a, b = res
    tol = 1e-11 if prec == "c128" else 2e-4
    scale = max(np.max(np.abs(b["g_gamma"])), np.max(np.abs(b["g_beta"])))
    assert np.max(np.abs(a["g_gamma"] - b["g_gamma"])) <= tol * scale
    assert np.max(np.abs(a["g_beta"] - b["g_beta"])) <= tol * scale
    assert abs(a["exp_c"] - b["exp_c"]) <= tol * abs(b["exp_c"])
    # passes - 1 adjoint passes store lambda only (the last one stores nothing)
    sb = (8 if prec == "c64" else 16) << n
    npass = round((adj_bytes[1] - adj_bytes[0]) / sb) + 1
    assert npass >= 2 and adj_bytes[1] - adj_bytes[0] == (npass - 1) * sb


@pytest.mark.gpu
@pytest.mark.parametrize("n,p,prec", [(16, 3, "c128"), (22, 4, "c64"), (26, 2, "c64")])
def test_grad_two_vectors_forward_last_pass_out_of_place(n, p, prec, monkeypatch):
    # with two vectors, the forward's last pass writes psi_p into the adjoint
    # vector's buffer and the adjoint's first pass (its mirror) reads it there
    # and does not write psi back: the gradients of the in-place forward up
    # to rounding, one state write fewer (the adjoint's counted bytes)
    u, v, w = inputs.complete_graph(n, 1060 + n)
    monkeypatch.setenv("QAOA_GRAD_CHECKPOINT", "0")
    res, adj_bytes = [], []
    for hy in ("1", "0"):
        monkeypatch.setenv("QAOA_GRAD_HYBRID", hy)
        with sim(n, u, v, w, S, prec, with_grad=True) as s:
            s.profile(True)
            res.append(s.grad(p, 0.6, 0.3))
            adj_bytes.append(s.profile_read("adjoint")["bytes"])
    a, b = res
    tol = 1e-11 if prec == "c128" else 2e-4
    scale = max(np.max(np.abs(b["g_gamma"])), np.max(np.abs(b["g_beta"])))
    assert np.max(np.abs(a["g_gamma"] - b["g_gamma"])) <= tol * scale
    assert np.max(np.abs(a["g_beta"] - b["g_beta"])) <= tol * scale
    assert abs(a["exp_c"] - b["exp_c"]) <= tol * abs(b["exp_c"])
    sb = (8 if prec == "c64" else 16) << n
    assert adj_bytes[1] - adj_bytes[0] == sb


@pytest.mark.gpu
def test_grad_stored_states_vs_oracle_fd():
    # complex128 with stored forward states against the oracle's central
    # differences (the default path when memory allows)
    n, p = 16, 4
    u, v, w = inputs.complete_graph(n, 1016)
    g, b = oracle.lr_schedule(p, 0.6, 0.3)
    fd_g, fd_b = oracle.grad_fd(n, u, v, w, S, g, b)
    with sim(n, u, v, w, S, "c128", with_grad=True) as s:
        s.profile(True)
        out = s.grad_angles(g, b)
        by = s.profile_read("adjoint")["bytes"]
    scale = max(np.max(np.abs(fd_g)), np.max(np.abs(fd_b)))
    assert np.max(np.abs(out["g_gamma"] - fd_g)) <= 1e-6 * scale
    assert np.max(np.abs(out["g_beta"] - fd_b)) <= 1e-6 * scale
    # first pass reads psi, writes lambda; middle passes read both, write lambda;
    # the last reads both: 2 + 3 (P - 2) + 2 states
    sb = 16 << n
    npass = (by / sb - 4) / 3 + 2
    assert npass == round(npass) and npass >= 3
