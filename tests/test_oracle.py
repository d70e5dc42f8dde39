"""Pins that tie the oracle to the paper and to mathematics, not to itself.

Each test checks the oracle against something computed a different way:
dense matrix exponentials, closed forms, invariants, hand-enumerated tiny
cases, or numbers the paper prints. A plausible slip in the oracle (a dropped
term, a wrong sign, a swapped qubit index, a transposed operand) breaks at
least one of them:

* a sign error in the cost or mixer rotation breaks the dense-expm check and
  the closed-form single-layer check;
* a wrong qubit/edge index breaks the dense-expm check on sparse graphs with
  distinct weights, and the hand-enumerated cut tables;
* a dropped term in C(x) breaks the per-edge identity sum_x C(x) = W 2^(n-1);
* a sampling off-by-one breaks the hand-computed CDF cases.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2604_26423_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- independent references
def dense_state(n, u, v, w, s, gamma, beta):
    """prod_k expm(i beta_k sum X_q) diag(exp(-i gamma_k s h)) |+> with dense matrices."""
    N = 1 << n
    z = np.arange(N)
    spin = 1 - 2 * ((z[:, None] >> np.arange(n)[None, :]) & 1)       # s_q = +-1
    h = np.zeros(N)
    for a, b, wt in zip(u, v, w):
        h += wt * spin[:, a] * spin[:, b]                               # Eq. H_C
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    I2 = np.eye(2, dtype=complex)
    B = np.zeros((N, N), dtype=complex)
    for q in range(n):
        op = np.array([[1.0 + 0j]])
        for k in reversed(range(n)):                                    # qubit 0 = least significant
            op = np.kron(op, X if k == q else I2)
        B += op
    psi = np.full(N, 2.0 ** (-n / 2), dtype=complex)
    for g, bt in zip(gamma, beta):
        psi = np.exp(-1j * g * s * h) * psi                             # Eq. UC
        psi = expm(1j * bt * B) @ psi                                   # Eq. UB
    return psi


analytic_p1_zz = oracle.analytic_p1_zz


def random_graph(n, seed, density=1.0):
    u, v, w = inputs.complete_graph(n, seed)
    if density < 1.0:
        keep = inputs.uniforms(seed + 7, len(u)) < density
        u, v, w = u[keep], v[keep], w[keep]
    return u, v, w


# ---------------------------------------------------------------- pins
@pytest.mark.parametrize("n,p,density,seed", [(3, 1, 1.0, 1), (5, 2, 1.0, 2), (6, 3, 0.5, 3),
                                              (8, 3, 1.0, 4), (9, 2, 0.4, 5)])
def test_dense_expm(n, p, density, seed):
    u, v, w = random_graph(n, seed, density)
    gamma, beta = oracle.lr_schedule(p, 0.6, 0.3)
    ref = dense_state(n, u, v, w, 0.1, gamma, beta)
    got = oracle.simulate(n, u, v, w, 0.1, gamma, beta)
    assert np.linalg.norm(got - ref) <= 1e-12


def test_dense_expm_large_angles():
    # angles outside the ramp (|beta| > pi/4, negative gamma) pin both rotation signs
    n = 5
    u, v, w = random_graph(n, 11, 0.7)
    gamma = np.array([-0.9, 2.3])
    beta = np.array([1.1, -2.0])
    ref = dense_state(n, u, v, w, 0.1, gamma, beta)
    got = oracle.simulate(n, u, v, w, 0.1, gamma, beta)
    assert np.linalg.norm(got - ref) <= 1e-12


@pytest.mark.parametrize("n", [2, 5, 11])
def test_uniform_state_identity(n):
    # p = 0: every edge is cut by exactly half of all bitstrings, so
    # sum_x C(x) = W 2^(n-1) exactly and <C> = W/2 (random-sampler baseline, Sec. II-D)
    u, v, w = random_graph(n, 20 + n)
    cut = oracle.cut_values(n, u, v, w)
    W = int(np.sum(w))
    assert int(cut.sum()) == W * (1 << (n - 1))
    psi = oracle.simulate(n, u, v, w, 0.1, [], [])
    e, nrm = oracle.expectation(psi, cut)
    assert abs(e - W / 2) <= 1e-12 * W
    assert abs(nrm - 1) <= 1e-14


@pytest.mark.parametrize("n,density,gamma,beta", [(4, 1.0, 0.37, 0.21), (6, 1.0, 0.6, 0.3),
                                                  (7, 0.5, 1.3, -0.4), (10, 1.0, 0.2, 0.2)])
def test_analytic_single_layer(n, density, gamma, beta):
    u, v, w = random_graph(n, 40 + n, density)
    s = 0.1
    J = np.zeros((n, n))
    for a, b, wt in zip(u, v, w):
        J[a, b] = J[b, a] = s * wt
    cut = oracle.cut_values(n, u, v, w)
    psi = oracle.simulate(n, u, v, w, s, [gamma], [beta])
    e, _ = oracle.expectation(psi, cut)
    ref = sum(wt * (1 - analytic_p1_zz(n, J, gamma, beta, a, b)) / 2 for a, b, wt in zip(u, v, w))
    assert abs(e - ref) <= 1e-11 * max(1.0, abs(ref))


def test_single_edge_hand_derivation():
    # n = 2, one edge: <C> = w (1 + sin(4 beta) sin(2 gamma s w)) / 2, derived by hand
    # in the {|00>+|11>, |01>+|10>} basis where X_0 + X_1 acts as 2 sigma_x.
    for wt, g, b in [(3, 0.4, 0.2), (7, 1.1, -0.35), (1, -0.5, 0.9)]:
        u, v, w = np.array([0]), np.array([1]), np.array([wt])
        cut = oracle.cut_values(2, u, v, w)
        e, _ = oracle.expectation(oracle.simulate(2, u, v, w, 0.1, [g], [b]), cut)
        assert abs(e - wt * (1 + math.sin(4 * b) * math.sin(2 * g * 0.1 * wt)) / 2) <= 1e-13


def test_cut_table_triangle():
    # hand enumeration: triangle 0-1 (w=2), 0-2 (w=3), 1-2 (w=5)
    u, v, w = np.array([0, 0, 1]), np.array([1, 2, 2]), np.array([2, 3, 5])
    cut = oracle.cut_values(3, u, v, w)
    # x = 0b000 .. 0b111, bit q = vertex q
    expect = [0, 2 + 3, 2 + 5, 3 + 5, 3 + 5, 2 + 5, 2 + 3, 0]
    assert cut.tolist() == expect


def test_cut_table_sparse_indices():
    # a path 0-3 (w=4), 3-1 (w=1) on 4 vertices: vertex 2 isolated; checks u/v indexing
    u, v, w = np.array([0, 3]), np.array([3, 1]), np.array([4, 1])
    cut = oracle.cut_values(4, u, v, w)
    for x in range(16):
        b = [(x >> q) & 1 for q in range(4)]
        assert cut[x] == 4 * (b[0] != b[3]) + 1 * (b[3] != b[1])


@pytest.mark.parametrize("n", [4, 7, 10])
def test_extremes_unit_complete(n):
    # K_n with unit weights: max cut = floor(n/2) ceil(n/2), min cut 0 at x = 0;
    # smallest maximiser is the lowest index with floor(n/2) or ceil(n/2) ones.
    u, v, _ = inputs.complete_graph(n, 1)
    w = np.ones(len(u), dtype=np.int32)
    cut = oracle.cut_values(n, u, v, w)
    cmin, cmax, amin, amax = oracle.extremes(n, cut)
    assert (cmin, amin) == (0, 0)
    assert cmax == (n // 2) * ((n + 1) // 2)
    assert amax == (1 << (n // 2)) - 1


@pytest.mark.parametrize("n,p", [(4, 2), (9, 3)])
def test_norm_and_gate_count(n, p):
    u, v, w = random_graph(n, 60 + n)
    gamma, beta = oracle.lr_schedule(p, 0.6, 0.3)
    zz, xx = oracle.gate_angles(n, w, 0.1, gamma, beta)
    psi, count = oracle.circuit(n, u, v, zz, xx, return_count=True)
    assert abs(np.vdot(psi, psi).real - 1) <= 1e-13
    # one RZZ per edge and one RX per qubit per layer; the paper's N_1q = (p+1) n
    # also counts the initial Hadamard layer, which the oracle replaces by |+>^n
    assert count == p * len(u) + p * n
    n2q, n1q = oracle.gate_counts(n, p)
    assert n2q == p * len(u) and n1q == (p + 1) * n


def test_paper_gate_counts_and_memory():
    with open(os.path.join(GOLDEN, "paper_counts.json")) as f:
        g = json.load(f)
    for c in g["two_qubit_gates"]:
        assert oracle.gate_counts(c["n"], c["p"])[0] == c["n2q"]
    # FP32 complex state of N qubits takes 2^(N+3) bytes (Sec. II-E)
    for c in g["fp32_state_bytes"]:
        nbytes = (1 << c["n"]) * 8
        if "gib" in c:
            assert nbytes == c["gib"] << 30
        else:
            assert nbytes == c["tib"] << 40


def test_conjugation_symmetry():
    # exp(+i gamma s H_C) and exp(-i beta B) give the complex conjugate state
    n = 7
    u, v, w = random_graph(n, 70)
    gamma, beta = oracle.lr_schedule(3, 0.6, 0.3)
    a = oracle.simulate(n, u, v, w, 0.1, gamma, beta)
    b = oracle.simulate(n, u, v, w, 0.1, -gamma, -beta)
    assert np.max(np.abs(a - np.conj(b))) <= 1e-15


def test_schedule_endpoints():
    # gamma_0 = dgamma/p, gamma_{p-1} = dgamma; beta_0 = dbeta, beta_{p-1} = dbeta/p
    g, b = oracle.lr_schedule(5, 0.6, 0.3)
    assert abs(g[0] - 0.6 / 5) < 1e-15 and abs(g[-1] - 0.6) < 1e-15
    assert abs(b[0] - 0.3) < 1e-15 and abs(b[-1] - 0.3 / 5) < 1e-15


def test_ratio_grows_with_depth():
    # noiseless LR-QAOA approaches r = 1 as p grows (Sec. II-C); the sign
    # convention of Eqs. UC/UB is what makes r rise rather than fall
    n = 8
    u, v, w = inputs.complete_graph(n, 5)
    rs = []
    for p in (1, 3, 10):
        g, b = oracle.lr_schedule(p, 0.6, 0.3)
        rs.append(oracle.run(n, u, v, w, 0.1, g, b)["r"])
    assert rs[0] < rs[1] < rs[2] and rs[2] > 0.9


def test_sampling_hand_cases():
    # |+>^3: F(x) = (x+1)/8; shot = smallest x with F(x) > u
    psi = np.full(8, 8 ** -0.5, dtype=complex)
    u = np.array([0.0, 0.1249, 0.1251, 0.3, 0.5, 0.99999])
    assert oracle.sample(psi, u).tolist() == [0, 0, 1, 2, 4, 7]
    # a state with zeros: probability only on x = 2 and x = 5 (1/4 and 3/4)
    psi = np.zeros(8, dtype=complex)
    psi[2] = 0.5
    psi[5] = math.sqrt(0.75) * 1j
    assert oracle.sample(psi, np.array([0.0, 0.2, 0.26, 0.9])).tolist() == [2, 2, 5, 5]


def test_sampling_frequencies():
    n = 6
    u, v, w = random_graph(n, 80)
    g, b = oracle.lr_schedule(3, 0.6, 0.3)
    psi = oracle.simulate(n, u, v, w, 0.1, g, b)
    prob = np.abs(psi) ** 2
    shots = oracle.sample(psi, inputs.uniforms(123, 200000))
    freq = np.bincount(shots.astype(np.int64), minlength=1 << n) / len(shots)
    # 5 sigma per bin
    sigma = np.sqrt(prob * (1 - prob) / len(shots))
    assert np.all(np.abs(freq - prob) <= 5 * sigma + 1e-12)


def test_gradients_shift_vs_fd():
    n = 5
    u, v, w = random_graph(n, 90, 0.8)
    g, b = oracle.lr_schedule(3, 0.6, 0.3)
    ps_g, ps_b = oracle.grad_param_shift(n, u, v, w, 0.1, g, b)
    fd_g, fd_b = oracle.grad_fd(n, u, v, w, 0.1, g, b)
    scale = max(np.max(np.abs(ps_g)), np.max(np.abs(ps_b)))
    assert np.max(np.abs(ps_g - fd_g)) <= 1e-7 * scale
    assert np.max(np.abs(ps_b - fd_b)) <= 1e-7 * scale


def test_gradient_vs_analytic_single_layer():
    # derivative of the closed form (by central differences on the formula,
    # which shares nothing with the oracle) against the exact shift rule
    n, s, h = 6, 0.1, 1e-5
    u, v, w = random_graph(n, 95)
    J = np.zeros((n, n))
    for a, b, wt in zip(u, v, w):
        J[a, b] = J[b, a] = s * wt

    def f(gm, bt):
        return sum(wt * (1 - analytic_p1_zz(n, J, gm, bt, a, b)) / 2 for a, b, wt in zip(u, v, w))

    gm, bt = 0.45, 0.25
    ps_g, ps_b = oracle.grad_param_shift(n, u, v, w, s, [gm], [bt])
    dg = (f(gm + h, bt) - f(gm - h, bt)) / (2 * h)
    db = (f(gm, bt + h) - f(gm, bt - h)) / (2 * h)
    assert abs(ps_g[0] - dg) <= 1e-6 * max(1, abs(dg))
    assert abs(ps_b[0] - db) <= 1e-6 * max(1, abs(db))


def test_lr_chain_rule():
    # d/d dgamma through gamma_k = (k+1)/p dgamma, checked by differencing the schedule
    n = 5
    u, v, w = random_graph(n, 99)
    p, dg, db, h = 3, 0.6, 0.3, 1e-5
    gg, gb = oracle.grad_param_shift(n, u, v, w, 0.1, *oracle.lr_schedule(p, dg, db))
    cdg, cdb = oracle.lr_chain(gg, gb)
    cut = oracle.cut_values(n, u, v, w)

    def f(a, b):
        return oracle.expectation(oracle.simulate(n, u, v, w, 0.1, *oracle.lr_schedule(p, a, b)), cut)[0]

    assert abs(cdg - (f(dg + h, db) - f(dg - h, db)) / (2 * h)) <= 1e-6 * max(1, abs(cdg))
    assert abs(cdb - (f(dg, db + h) - f(dg, db - h)) / (2 * h)) <= 1e-6 * max(1, abs(cdb))


def test_inputs_splitmix_reference_values():
    # SplitMix64 with seed 0: published first outputs of the reference generator
    # (state advanced by the golden gamma before mixing)
    x = inputs.splitmix64(0, 3)
    assert [int(t) for t in x] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_analytic_p1_expectation_matches_simulation():
    # the edge sum of the closed form equals the simulated single-layer <C>
    n = 7
    u, v, w = random_graph(n, 77, 0.6)
    for gamma, beta in [(0.3, 0.2), (1.1, -0.4)]:
        cut = oracle.cut_values(n, u, v, w)
        e = oracle.expectation(oracle.simulate(n, u, v, w, 0.1, [gamma], [beta]), cut)[0]
        assert abs(oracle.analytic_p1_expectation(n, u, v, w, 0.1, gamma, beta) - e) <= 1e-10 * abs(e)


# ---------------------------------------------------------------- Sec. II-D
def test_sample_cuts_hand_and_moments():
    # triangle 0-1 (w 2), 1-2 (w 3), 0-2 (w -1): hand values of C(x)
    u, v, w = [0, 1, 0], [1, 2, 2], [2, 3, -1]
    hand = {0: 0, 1: 2 - 1, 2: 2 + 3, 3: 3 - 1, 4: 3 - 1, 5: 2 + 3, 6: 2 - 1, 7: 0}
    got = oracle.sample_cuts(3, u, v, w, list(hand))
    assert list(got) == [hand[x] for x in hand]
    # over all 2^n bitstrings every edge is cut exactly half the time and the
    # cut indicators of distinct edges are pairwise independent: mean W/2,
    # variance sum w^2 / 4; C(x) = C(~x)
    n = 9
    u, v, w = inputs.complete_graph(n, 4242)
    xs = np.arange(1 << n, dtype=np.uint64)
    c = oracle.sample_cuts(n, u, v, w, xs).astype(np.int64)
    W, Q = int(np.sum(w)), int(np.sum(np.asarray(w, dtype=np.int64) ** 2))
    assert 2 * int(c.sum()) == W * (1 << n)
    assert 4 * int(((2 * c - W) ** 2).sum()) == 4 * Q * (1 << n)
    assert np.array_equal(c, c[::-1])
    with pytest.raises(ValueError):
        oracle.sample_cuts(3, [0], [1], [1], [8])


def test_random_sampler_moments():
    n = 12
    u, v, w = inputs.complete_graph(n, 77)
    xs = oracle.random_bitstrings(n, 20000, seed=5)
    assert int(xs.max()) < (1 << n)
    bits = (xs[:, None] >> np.arange(n, dtype=np.uint64)) & np.uint64(1)
    freq = bits.mean(axis=0)
    assert np.all(np.abs(freq - 0.5) < 5 * 0.5 / math.sqrt(len(xs)))
    c = oracle.sample_cuts(n, u, v, w, xs[:4000]).astype(np.float64)
    W, Q = float(np.sum(w)), float(np.sum(np.asarray(w, dtype=np.float64) ** 2))
    assert abs(c.mean() - W / 2) < 5 * math.sqrt(Q / 4 / len(c))
    # ratios: (C - C_min) / (C_max - C_min), exact per sample
    cut = oracle.cut_values(n, u, v, w)
    cmin, cmax, _, _ = oracle.extremes(n, cut)
    r = oracle.sample_ratios(cut[xs[:50].astype(np.int64)], cmin, cmax)
    assert np.all((r >= 0) & (r <= 1))
    assert np.array_equal(oracle.sample_ratios([cmin, cmax], cmin, cmax), [0.0, 1.0])
    assert np.array_equal(oracle.sample_ratios([5, 5], 5, 5), [1.0, 1.0])


def test_subsample_without_replacement():
    idx = oracle.subsample_indices(50, 20, 30, seed=9)
    assert idx.shape == (30, 20)
    for row in idx:
        assert len(set(row.tolist())) == 20 and row.min() >= 0 and row.max() < 50
    full = oracle.subsample_indices(17, 17, 5, seed=1)
    for row in full:
        assert sorted(row.tolist()) == list(range(17))
    # every ordered pair of distinct positions is equally likely
    reps = 12000
    idx = oracle.subsample_indices(4, 2, reps, seed=3)
    counts = {}
    for a, b in idx.tolist():
        counts[(a, b)] = counts.get((a, b), 0) + 1
    assert len(counts) == 12
    mu = reps / 12
    sd = math.sqrt(reps * (1 / 12) * (11 / 12))
    assert all(abs(k - mu) < 5 * sd for k in counts.values())
    with pytest.raises(ValueError):
        oracle.subsample_indices(5, 6, 1, seed=0)


def test_mean_of_means_closed_forms():
    pool = inputs.uniforms(11, 400)
    # ns = m: every subsample is the whole pool
    mm = oracle.mean_of_means(pool, 400, 20, seed=2)
    assert np.all(np.abs(mm["means"] - pool.mean()) < 1e-14)
    assert mm["sigma"] < 1e-14 and abs(mm["threshold"] - mm["grand_mean"]) < 1e-13
    # ns = 1: the means are pool entries
    mm = oracle.mean_of_means(pool, 1, 50, seed=2)
    assert set(mm["means"].tolist()) <= set(pool.tolist())
    # without replacement: Var(mean) = S^2 / ns * (m - ns) / (m - 1) with S^2
    # the pool's variance (1/m); 4000 subsamples put the estimate within ~5%
    m, ns, reps = 400, 40, 4000
    mm = oracle.mean_of_means(pool, ns, reps, seed=4)
    want = pool.var() / ns * (m - ns) / (m - 1)
    assert abs(mm["sigma"] ** 2 / want - 1) < 0.15
    assert abs(mm["grand_mean"] - pool.mean()) < 5 * math.sqrt(want / reps)
    assert mm["threshold"] == mm["grand_mean"] + 3.0 * mm["sigma"]


def test_mean_of_means_shot_scaling_matches_paper():
    # Sec. II-D: going from 100 to 10 shots widens the random sampler's
    # mean-of-means distribution by about 3.5 (100 subsamples each); sampling
    # without replacement from a large pool predicts sqrt(10) ~ 3.2, and the
    # 100-subsample estimates scatter by ~10%
    n = 14
    u, v, w = inputs.complete_graph(n, 140)
    cut = oracle.cut_values(n, u, v, w)
    cmin, cmax, _, _ = oracle.extremes(n, cut)
    xs = oracle.random_bitstrings(n, 5000, seed=8)
    r = oracle.sample_ratios(cut[xs.astype(np.int64)], cmin, cmax)
    s10 = oracle.mean_of_means(r, 10, 100, seed=1)["sigma"]
    s100 = oracle.mean_of_means(r, 100, 100, seed=1)["sigma"]
    assert abs(s10 / s100 / 3.5 - 1) < 0.25


def test_classify_regime_cases():
    R, T, N, A = (oracle.REGIME_RANDOM, oracle.REGIME_TRANSITION, oracle.REGIME_NOISE_TOLERANT,
                  oracle.REGIME_ABOVE_RANDOM)
    # random interval 0.79 +- 0.03 (threshold 0.82), noiseless 0.88 +- 0.03 (from 0.85)
    assert oracle.classify_regime(0.70, 0.79, 0.01) == R          # below the random interval
    assert oracle.classify_regime(0.80, 0.79, 0.01, 0.88, 0.01) == R
    assert oracle.classify_regime(0.83, 0.79, 0.01, 0.88, 0.01) == T
    assert oracle.classify_regime(0.87, 0.79, 0.01, 0.88, 0.01) == N
    assert oracle.classify_regime(0.95, 0.79, 0.01, 0.88, 0.01) == N  # above the noiseless interval
    assert oracle.classify_regime(0.83, 0.79, 0.01) == A
    assert oracle.classify_regime(0.83, 0.79, float("nan")) == -1
    assert oracle.classify_regime(0.83, 0.79, 0.01, 0.88, -1.0) == -1


# ---------------------------------------------------------------- Sec. II-C
def test_noisy_density_closed_forms():
    # one edge, p = 1: the channel after the only ZZ gate mixes the ideal state
    # with I/4, which the mixer leaves alone: <C> = (1 - eps) <C>_ideal + eps w / 2
    u, v, w = [0], [1], [3]
    g, b = oracle.lr_schedule(1, 0.6, 0.3)
    ideal = oracle.run(2, u, v, w, 0.1, g, b)["exp_c"]
    for eps in (0.0, 0.3, 1.0):
        assert abs(oracle.noisy_density(2, u, v, w, 0.1, g, b, eps) - ((1 - eps) * ideal + eps * 1.5)) < 1e-12
    # eps = 0 is the pure-state circuit; eps = 1 on K_n ends maximally mixed (<C> = W/2)
    n = 4
    u, v, w = inputs.complete_graph(n, 9)
    g, b = oracle.lr_schedule(2, 0.6, 0.3)
    assert abs(oracle.noisy_density(n, u, v, w, 0.1, g, b, 0.0) - oracle.run(n, u, v, w, 0.1, g, b)["exp_c"]) < 1e-11
    assert abs(oracle.noisy_density(n, u, v, w, 0.1, g, b, 1.0) - np.sum(w) / 2) < 1e-11


def test_depolarizing_pauli_sum_is_partial_trace():
    # (1/16) sum_P P rho P over the Paulis on (i, j) = I/4 (x) Tr_ij rho
    n, i, j = 3, 0, 2
    rng = inputs.uniforms(31, 2 * 64).reshape(2, 8, 8)
    a = rng[0] + 1j * rng[1]
    rho = a @ a.conj().T
    rho /= np.trace(rho)
    acc = np.zeros_like(rho)
    for pa in range(4):
        for pb in range(4):
            P = oracle._pauli_matrix(n, i, pa) @ oracle._pauli_matrix(n, j, pb)
            acc += P @ rho @ P.conj().T
    # index bits (b2 b1 b0) = qubits (2, 1, 0); reshape as [q2, q1, q0] x [q2, q1, q0]
    t = rho.reshape(2, 2, 2, 2, 2, 2)
    red = np.einsum("abcadc->bd", t)        # trace over qubits 2 and 0, keep qubit 1
    want = np.einsum("ac,bd,ef->abecdf", np.eye(2) / 2, red, np.eye(2) / 2).reshape(8, 8)
    assert np.allclose(acc / 16, want, atol=1e-14)


def test_noisy_trajectories_average_to_density():
    n, p, eps = 4, 2, 0.08
    u, v, w = inputs.complete_graph(n, 5)
    g, b = oracle.lr_schedule(p, 0.6, 0.3)
    exact = oracle.noisy_density(n, u, v, w, 0.1, g, b, eps)
    cut = oracle.cut_values(n, u, v, w)
    vals = np.array([np.sum(np.abs(oracle.noisy_trajectory(n, u, v, w, 0.1, g, b, eps, 7, t)) ** 2 * cut)
                     for t in range(3000)])
    assert abs(vals.mean() - exact) < 5 * vals.std() / math.sqrt(len(vals))
    # no error at eps = 0: the noiseless state
    psi = oracle.noisy_trajectory(n, u, v, w, 0.1, g, b, 0.0, 7, 0)
    assert np.max(np.abs(psi - oracle.simulate(n, u, v, w, 0.1, g, b))) < 1e-12


def test_overlap_and_k0_fit():
    assert oracle.overlap_ratio(0.85, 0.9, 0.8) == (0.85 - 0.8) / (0.9 - 0.8)
    a = np.array([0.1, 0.5, 1.0, 2.0])
    assert abs(oracle.fit_k0(a, 2.0 ** (-1.7 * a)) - 1.7) < 1e-12
    # points at or below zero (random or worse) are left out
    assert abs(oracle.fit_k0(np.append(a, 3.0), np.append(2.0 ** (-0.4 * a), -0.01)) - 0.4) < 1e-12


def test_cut_values_real():
    # integer weights: the integer table; a real-weight triangle by hand
    n = 6
    u, v, w = inputs.complete_graph(n, 66)
    assert np.array_equal(oracle.cut_values_real(n, u, v, w), oracle.cut_values(n, u, v, w).astype(float))
    c = oracle.cut_values_real(3, [0, 1, 0], [1, 2, 2], [0.25, 0.5, 0.125])
    assert np.allclose(c, [0, 0.375, 0.75, 0.625, 0.625, 0.75, 0.375, 0])
