"""Noisy LR-QAOA (Sec. II-C) on the GPU: each trajectory's <C> against the
oracle's gate-by-gate trajectory with the same error draws (complex128:
1e-10 relative, the operation order differs; complex64 trajectories, FP32
phases and butterflies: 1e-4 relative), the trajectory mean against the
oracle's exact density-matrix result (statistical, 5 standard errors), and the
overlap ratio / k0 fit of Eq. noise on a depth sweep."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_26423_b300 import inputs

pytestmark = pytest.mark.gpu
S = 0.1


def sim(*a, **k):
    from paper_2604_26423_b300.qaoa import Simulator
    return Simulator(*a, **k)


@pytest.mark.parametrize("n,p,eps,kind,prec", [(4, 1, 0.05, "complete", "c128"), (6, 3, 0.2, "complete", "c128"),
                                               (9, 2, 0.5, "signed", "c128"), (12, 3, 0.02, "complete", "c128"),
                                               (10, 2, 1.0, "sparse", "c128"), (7, 0, 0.3, "complete", "c128"),
                                               (12, 3, 0.02, "complete", "c64"), (9, 4, 0.3, "signed", "c64")])
def test_trajectories_vs_oracle(n, p, eps, kind, prec):
    # complex64: FP32 phases (angles up to ~10 rad) and butterflies, 1e-4 relative
    u, v, w = inputs.complete_graph(n, 60 + n)
    if kind == "signed":
        w = np.where(inputs.uniforms(61 + n, len(w)) < 0.3, -w, w).astype(np.int32)
    if kind == "sparse":
        keep = inputs.uniforms(62 + n, len(u)) < 0.4
        keep[0] = True
        u, v, w = u[keep], v[keep], w[keep]
    g, b = oracle.lr_schedule(max(p, 1), 0.6, 0.3)
    g, b = g[:p], b[:p]
    T, seed = 37, 1000 + n
    cut = oracle.cut_values(n, u, v, w)
    with sim(n, u, v, w, S, prec) as s:
        out = s.noisy_expect(g, b, eps, T, seed)
        per = out["per_trajectory"].cpu().numpy()
    want = np.array([np.sum(np.abs(oracle.noisy_trajectory(n, u, v, w, S, g, b, eps, seed, t)) ** 2 * cut)
                     for t in range(T)])
    scale = max(1.0, float(np.max(np.abs(want))))
    assert np.max(np.abs(per - want)) <= (1e-10 if prec == "c128" else 1e-4) * scale
    assert abs(out["exp_c"] - per.sum() / T) <= 1e-12 * scale
    cmin, cmax, _, _ = oracle.extremes(n, cut)
    assert abs(out["r"] - (out["exp_c"] - cmin) / (cmax - cmin)) < 1e-12


@pytest.mark.parametrize("eps", [0.0, 0.1, 1.0])
def test_trajectory_mean_vs_density_matrix(eps):
    n, p, T = 4, 2, 20000
    u, v, w = inputs.complete_graph(n, 5)
    g, b = oracle.lr_schedule(p, 0.6, 0.3)
    exact = oracle.noisy_density(n, u, v, w, S, g, b, eps)
    with sim(n, u, v, w, S, "c64") as s:
        out = s.noisy_expect(g, b, eps, T, seed=3)
        per = out["per_trajectory"].cpu().numpy()
    se = per.std() / math.sqrt(T)
    # complex64 trajectories: FP32 rounding of the state, ~1e-6 relative
    assert abs(out["exp_c"] - exact) <= 5 * se + 2e-5 * abs(exact)


def test_noisy_rejects_bad_arguments():
    from paper_2604_26423_b300.qaoa import QaoaError
    u, v, w = inputs.complete_graph(13, 1)
    with sim(13, u, v, w, S, "c64") as s:
        with pytest.raises(QaoaError):
            s.noisy_expect([0.1], [0.1], 0.1, 4)
    u, v, w = inputs.complete_graph(5, 1)
    with sim(5, u, v, w, S, "c64") as s:
        for eps, T in ((-0.1, 4), (1.5, 4), (0.1, 0)):
            with pytest.raises(QaoaError):
                s.noisy_expect([0.1], [0.1], eps, T)


def test_overlap_decay_and_k0():
    # Sec. II-C on K_8: r against p for several eps, r_ovl against
    # eps_acc = N_2q eps, and the fit of Eq. noise; r_ovl is 1 without noise
    # and falls toward 0 as the accumulated error grows
    from paper_2604_26423_b300.qaoa import fit_k0, overlap_ratio
    n = 8
    u, v, w = inputs.complete_graph(n, 808)
    cut = oracle.cut_values(n, u, v, w)
    cmin, cmax, _, _ = oracle.extremes(n, cut)
    r_rand = (np.sum(w) / 2 - cmin) / (cmax - cmin)
    pts_a, pts_r = [], []
    with sim(n, u, v, w, S, "c128") as s:
        for p in (3, 6):
            g, b = oracle.lr_schedule(p, 0.6, 0.3)
            ideal = s.noisy_expect(g, b, 0.0, 1, seed=1)["r"]
            assert abs(ideal - oracle.run(n, u, v, w, S, g, b)["r"]) < 1e-10
            prev = 1.0
            for eps in (0.002, 0.01, 0.05):
                rn = s.noisy_expect(g, b, eps, 4000, seed=p)["r"]
                ro = overlap_ratio(rn, ideal, r_rand)
                assert ro < prev + 0.05 and -0.2 < ro < 1.05
                prev = ro
                pts_a.append(p * len(u) * eps)
                pts_r.append(ro)
    # (the fit itself is checked against the oracle's on synthetic points in
    # the CPU tests; here its input comes from the GPU)
    k0 = fit_k0(pts_a, pts_r)
    assert k0 > 0
