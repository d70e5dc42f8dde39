"""Sampling methodology (Sec. II-D) on the GPU against the oracle: cut values
and ratios of shots and of the uniform random sampler (bit-exact: integer cut
values, the same FP64 division), the subsample means drawn without
replacement (the same draws, the same FP64 summation order: bit-exact), and
the regime classification of a full LR-QAOA run."""
import numpy as np
import pytest

import oracle
from paper_2604_26423_b300 import inputs

pytestmark = pytest.mark.gpu
S = 0.1


def sim(*a, **k):
    from paper_2604_26423_b300.qaoa import Simulator
    return Simulator(*a, **k)


def signed_graph(n, seed):
    u, v, w = inputs.complete_graph(n, seed)
    flip = inputs.uniforms(seed + 1, len(w)) < 0.3
    return u, v, np.where(flip, -w, w).astype(np.int32)


@pytest.mark.parametrize("n,kind", [(5, "complete"), (16, "complete"), (18, "signed"), (21, "sparse")])
def test_sample_cuts_of_given_bitstrings(n, kind):
    if kind == "signed":
        u, v, w = signed_graph(n, 300 + n)
    elif kind == "sparse":
        u, v, w = inputs.complete_graph(n, 300 + n)
        keep = inputs.uniforms(301 + n, len(u)) < 0.2
        u, v, w = u[keep], v[keep], w[keep]
    else:
        u, v, w = inputs.complete_graph(n, 300 + n)
    cut = oracle.cut_values(n, u, v, w)
    cmin, cmax, _, _ = oracle.extremes(n, cut)
    count = 3001  # ragged against the 256-thread blocks
    xs = inputs.splitmix64(77 + n, count) >> np.uint64(64 - n)
    xs[:2] = [0, (1 << n) - 1]
    with sim(n, u, v, w, S, "c64") as s:
        out = s.sample_cuts(xs)
        gx, gc, gr = (t.cpu().numpy() for t in (out["x"], out["c"], out["r"]))
    want_c = cut[xs.astype(np.int64)]
    assert np.array_equal(gx.view(np.uint64), xs)
    assert np.array_equal(gc.astype(np.int64), want_c)
    assert np.array_equal(gr, oracle.sample_ratios(want_c, cmin, cmax))


@pytest.mark.parametrize("n,seed,count", [(12, 1, 1), (20, 9, 100003), (24, 3, 65536)])
def test_random_sampler_vs_oracle(n, seed, count):
    u, v, w = signed_graph(n, 400 + n)
    cut = oracle.cut_values(n, u, v, w)
    cmin, cmax, _, _ = oracle.extremes(n, cut)
    with sim(n, u, v, w, S, "c64") as s:
        out = s.sample_cuts(count=count, seed=seed)
        gx, gc, gr = (t.cpu().numpy() for t in (out["x"], out["c"], out["r"]))
    xs = oracle.random_bitstrings(n, count, seed)
    want_c = cut[xs.astype(np.int64)]
    assert np.array_equal(gx.view(np.uint64), xs)
    assert np.array_equal(gc.astype(np.int64), want_c)
    assert np.array_equal(gr, oracle.sample_ratios(want_c, cmin, cmax))


def test_random_sampler_k33_sampled():
    # the full 33-qubit graph: the first draws' cut values against the oracle's
    # literal edge sum, the ratios against the extremes qaoa_expect reports
    n, count = 33, 1 << 22
    u, v, w = inputs.complete_graph(n, 33)
    with sim(n, u, v, w, S, "c64") as s:
        ext = s.extremes()
        out = s.sample_cuts(count=count, seed=12)
        gx = out["x"][:400].cpu().numpy().view(np.uint64)
        gc = out["c"][:400].cpu().numpy().astype(np.int64)
        gr = out["r"].cpu().numpy()
        cfull = out["c"].cpu().numpy().astype(np.int64)
    xs = oracle.random_bitstrings(n, 400, 12)
    assert np.array_equal(gx, xs)
    assert np.array_equal(gc, oracle.sample_cuts(n, u, v, w, xs))
    assert np.array_equal(gr, (cfull - ext["c_min"]) / float(ext["c_max"] - ext["c_min"]))
    # uniform bitstrings: mean cut W/2 within 5 standard errors
    W, Q = float(np.sum(w)), float(np.sum(np.asarray(w, dtype=np.float64) ** 2))
    assert abs(cfull.mean() - W / 2) < 5 * np.sqrt(Q / 4 / count)


def test_sample_cuts_rejects_out_of_range():
    from paper_2604_26423_b300.qaoa import QaoaError
    n = 14
    u, v, w = inputs.complete_graph(n, 14)
    with sim(n, u, v, w, S, "c64") as s:
        with pytest.raises(QaoaError):
            s.sample_cuts(np.array([3, 1 << n], dtype=np.uint64))
        assert s.sample_cuts(np.zeros(0, dtype=np.uint64))["c"].numel() == 0


@pytest.mark.parametrize("m,ns,reps", [(1, 1, 1), (10, 10, 7), (5000, 1, 33), (5000, 10, 100), (5000, 100, 100),
                                       (4096, 4096, 3), (1 << 20, 100, 100), (300, 299, 65)])
def test_mean_of_means_vs_oracle(m, ns, reps):
    import torch
    from paper_2604_26423_b300.qaoa import mean_of_means
    pool = inputs.uniforms(500 + m, m)
    g = mean_of_means(torch.tensor(pool, device="cuda"), ns, reps, seed=m + ns)
    want = oracle.mean_of_means(pool, ns, reps, seed=m + ns)
    assert np.array_equal(g["means"].cpu().numpy(), want["means"])
    assert g["grand_mean"] == want["grand_mean"]
    assert g["sigma"] == want["sigma"]
    assert g["threshold"] == want["threshold"]


def test_regime_pipeline_vs_oracle():
    # Sec. II-D end to end on K_16 (complex128, so shots match the oracle's
    # exactly): noiseless shots and the random sampler, their mean-of-means
    # distributions at 10 and 100 shots, and the regime of a further set of
    # noiseless shots: noise-tolerant and far above the random threshold
    import torch
    from paper_2604_26423_b300.qaoa import classify_regime, mean_of_means
    n, p = 16, 5
    u, v, w = inputs.complete_graph(n, 1616)
    g, b = oracle.lr_schedule(p, 0.6, 0.3)
    ref = oracle.run(n, u, v, w, S, g, b)
    uni = inputs.uniforms(1617, 4096)
    uni_obs = inputs.uniforms(1618, 10)
    shots_o = oracle.sample(ref["psi"], uni)
    obs_o = oracle.sample(ref["psi"], uni_obs)
    rand_o = oracle.random_bitstrings(n, 4096, 1619)
    r_ideal_o = oracle.sample_ratios(ref["cut"][shots_o.astype(np.int64)], ref["c_min"], ref["c_max"])
    r_rand_o = oracle.sample_ratios(ref["cut"][rand_o.astype(np.int64)], ref["c_min"], ref["c_max"])
    r_obs_o = float(np.mean(oracle.sample_ratios(ref["cut"][obs_o.astype(np.int64)], ref["c_min"], ref["c_max"])))
    with sim(n, u, v, w, S, "c128") as s:
        s.run_angles(g, b)
        shots = s.sample(4096, uniforms=uni)
        obs = s.sample(10, uniforms=uni_obs)
        assert np.array_equal(shots, shots_o) and np.array_equal(obs, obs_o)
        r_ideal = s.sample_cuts(shots)["r"]
        r_rand = s.sample_cuts(count=4096, seed=1619)["r"]
        r_obs = float(s.sample_cuts(obs)["r"].mean().item())
    assert np.array_equal(r_ideal.cpu().numpy(), r_ideal_o)
    assert np.array_equal(r_rand.cpu().numpy(), r_rand_o)
    for ns in (10, 100):
        gi = mean_of_means(r_ideal, ns, 100, seed=ns)
        gr = mean_of_means(r_rand, ns, 100, seed=ns + 1)
        oi = oracle.mean_of_means(r_ideal_o, ns, 100, seed=ns)
        orr = oracle.mean_of_means(r_rand_o, ns, 100, seed=ns + 1)
        assert (gi["grand_mean"], gi["sigma"]) == (oi["grand_mean"], oi["sigma"])
        assert (gr["grand_mean"], gr["sigma"]) == (orr["grand_mean"], orr["sigma"])
        if ns == 10:
            reg = classify_regime(r_obs, gr["grand_mean"], gr["sigma"], gi["grand_mean"], gi["sigma"])
            assert reg == oracle.classify_regime(r_obs_o, orr["grand_mean"], orr["sigma"], oi["grand_mean"],
                                                 oi["sigma"])
            assert reg == oracle.REGIME_NOISE_TOLERANT
            assert gi["grand_mean"] > gr["threshold"]
