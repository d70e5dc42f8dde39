"""Oracle for the LR-QAOA state-vector hot path: plain, slow, obviously correct.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
never calls it and shares no code with it.

The C part (``oracle.c``) applies gates one at a time in complex128; this file
builds the per-gate angles from the paper's schedule and wraps the results.
Every function names the passage of the paper it follows:

* ``lr_schedule``      -- Sec. II-B, linear schedules for beta_i and gamma_i.
* ``cut_values``       -- Sec. II-B, Eq. for C(x) (literal double sum);
  ``cut_values_real`` the same with real weights (Sec. II-G).
* ``extremes``         -- Sec. II-B, C(x*) = max cut; here by exhaustive search.
* ``simulate``         -- Sec. II-B Eqs. H_C, UC, UB; gates as in Sec. II-E.
* ``expectation``      -- <C> = sum |psi_x|^2 C(x); r as in Eq. r with the
                          exact mean in place of the sample mean.
* ``sample``           -- Sec. II-B, repeated preparation and measurement.
* ``grad_fd``          -- central finite differences of <C> (h = 1e-5).
* ``grad_param_shift`` -- exact two-term shift rule per gate (each gate is
                          exp(-i theta/2 P) with a Pauli product P).
* ``gate_counts``      -- Sec. II-B, N_2q = p N(N-1)/2 and N_1q = (p+1) N.
* ``noisy_trajectory``, ``noisy_density`` -- Sec. II-C: LR-QAOA with a
  two-qubit depolarizing channel after every ZZ gate, as one stochastic
  trajectory (explicit Pauli errors, gate by gate) and exactly (density matrix,
  tiny n); ``overlap_ratio`` and ``fit_k0`` -- Eq. noise, r_ovl = 2^(-k0 eps_acc).
* ``sample_cuts``, ``sample_ratios``, ``random_bitstrings``, ``subsample_indices``,
  ``mean_of_means``, ``classify_regime`` -- Sec. II-D (sampling methodology):
  approximation ratio of individual bitstrings, the uniform random sampler,
  repeated subsampling without replacement, the mean of subsample means with its
  standard deviation, the random threshold and the three performance regimes.

Pins that tie this oracle to the paper and to mathematics (dense matrix
exponentials, the uniform-state identity, the closed-form single-layer
expectation, norm, conjugation symmetry, brute force on tiny graphs and the
paper's printed gate counts) live in ``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles ``oracle.c`` with gcc -O2 -fopenmp into ``liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        i32p, i64p, u64p, f64p = P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_uint64), P(ctypes.c_double)
        lib.oracle_cut_values.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i64p]
        lib.oracle_extremes.argtypes = [ctypes.c_int, i64p, i64p, i64p, u64p, u64p]
        lib.oracle_circuit.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, ctypes.c_int,
                                       f64p, f64p, f64p, i64p]
        lib.oracle_expectation.argtypes = [ctypes.c_int, f64p, i64p, f64p]
        lib.oracle_expectation.restype = ctypes.c_double
        lib.oracle_sample.argtypes = [ctypes.c_int, f64p, ctypes.c_int, f64p, u64p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def lr_schedule(p: int, dgamma: float, dbeta: float):
    """beta_i = (1 - i/p) dbeta and gamma_i = (i + 1)/p dgamma, i = 0..p-1 (Sec. II-B)."""
    i = np.arange(p, dtype=np.float64)
    beta = (1.0 - i / p) * dbeta
    gamma = (i + 1.0) / p * dgamma
    return gamma, beta


def gate_counts(n: int, p: int):
    """N_2q = p n(n-1)/2 and N_1q = (p + 1) n for a fully connected graph (Sec. II-B)."""
    return p * n * (n - 1) // 2, (p + 1) * n


def _edges(u, v, w):
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    return u, v, w


def cut_values(n: int, u, v, w) -> np.ndarray:
    """C(x) = sum_{k<l} w_kl (x_k + x_l - 2 x_k x_l) for all 2^n bitstrings, int64."""
    u, v, w = _edges(u, v, w)
    out = np.empty(1 << n, dtype=np.int64)
    rc = _load().oracle_cut_values(n, len(u), _ptr(u, ctypes.c_int32), _ptr(v, ctypes.c_int32),
                                   _ptr(w, ctypes.c_int32), _ptr(out, ctypes.c_int64))
    if rc:
        raise ValueError("oracle_cut_values rejected its arguments")
    return out


def cut_values_real(n: int, u, v, w) -> np.ndarray:
    """C(x) with real weights (Sec. II-G: U[0, 1] in the paper), float64, all x:
    sum over edges of w_e [x_u != x_v], edge by edge."""
    x = np.arange(1 << n, dtype=np.int64)
    out = np.zeros(1 << n)
    for a, b, we in zip(u, v, w):
        out += float(we) * (((x >> int(a)) ^ (x >> int(b))) & 1)
    return out


def extremes(n: int, cut: np.ndarray):
    """(C_min, C_max, argmin, argmax) by exhaustive search; ties -> smallest index."""
    cmin, cmax = ctypes.c_int64(), ctypes.c_int64()
    amin, amax = ctypes.c_uint64(), ctypes.c_uint64()
    cut = np.ascontiguousarray(cut, dtype=np.int64)
    _load().oracle_extremes(n, _ptr(cut, ctypes.c_int64), ctypes.byref(cmin), ctypes.byref(cmax),
                            ctypes.byref(amin), ctypes.byref(amax))
    return cmin.value, cmax.value, amin.value, amax.value


def gate_angles(n: int, w, scale: float, gamma, beta):
    """Per-gate angles: RZZ(2 gamma_k s w_e) per edge and RX(-2 beta_k) per qubit."""
    w = np.asarray(w, dtype=np.float64)
    gamma = np.asarray(gamma, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    zz = 2.0 * gamma[:, None] * scale * w[None, :]
    xx = np.repeat((-2.0 * beta)[:, None], n, axis=1)
    return np.ascontiguousarray(zz), np.ascontiguousarray(xx)


def circuit(n: int, u, v, zz_theta, x_phi, return_count: bool = False):
    """Applies the gate list with explicit per-gate angles; returns complex128 psi."""
    u, v, _ = _edges(u, v, np.zeros(len(u)))
    zz_theta = np.ascontiguousarray(zz_theta, dtype=np.float64)
    x_phi = np.ascontiguousarray(x_phi, dtype=np.float64)
    p = zz_theta.shape[0] if zz_theta.ndim == 2 else 0
    if p == 0:
        p = x_phi.shape[0] if x_phi.ndim == 2 else 0
    psi = np.empty(1 << n, dtype=np.complex128)
    cnt = ctypes.c_int64()
    rc = _load().oracle_circuit(n, len(u), _ptr(u, ctypes.c_int32), _ptr(v, ctypes.c_int32), p,
                                _ptr(zz_theta, ctypes.c_double), _ptr(x_phi, ctypes.c_double),
                                psi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cnt))
    if rc:
        raise ValueError("oracle_circuit rejected its arguments")
    return (psi, cnt.value) if return_count else psi


def simulate(n: int, u, v, w, scale: float, gamma, beta) -> np.ndarray:
    """prod_k exp(+i beta_k H_B) exp(-i gamma_k s H_C) |+>^n, gate by gate, complex128."""
    gamma = np.atleast_1d(np.asarray(gamma, dtype=np.float64))
    beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
    zz, xx = gate_angles(n, w, scale, gamma, beta)
    return circuit(n, u, v, zz, xx)


def expectation(psi: np.ndarray, cut: np.ndarray):
    """(<C>, norm) with <C> = sum_x |psi_x|^2 C(x), accumulated in index order."""
    n = int(round(math.log2(len(psi))))
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    cut = np.ascontiguousarray(cut, dtype=np.int64)
    norm = ctypes.c_double()
    e = _load().oracle_expectation(n, psi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   _ptr(cut, ctypes.c_int64), ctypes.byref(norm))
    return float(e), norm.value


def approximation_ratio(exp_c: float, cmin: int, cmax: int) -> float:
    """r = (<C> - C_min) / (C_max - C_min); equals <C>/C(x*) when C_min = 0 (Eq. r)."""
    return (exp_c - cmin) / (cmax - cmin) if cmax != cmin else 1.0


def sample(psi: np.ndarray, uni) -> np.ndarray:
    """Shot i = smallest x with F(x) > u_i * total, F the sequential CDF of |psi|^2."""
    n = int(round(math.log2(len(psi))))
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    uni = np.ascontiguousarray(uni, dtype=np.float64)
    out = np.empty(len(uni), dtype=np.uint64)
    rc = _load().oracle_sample(n, psi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(uni),
                               _ptr(uni, ctypes.c_double), _ptr(out, ctypes.c_uint64))
    if rc:
        raise MemoryError("oracle_sample could not allocate the CDF")
    return out


def run(n: int, u, v, w, scale: float, gamma, beta):
    """Full forward result: dict with psi, <C>, norm, C_min, C_max, argmin, argmax, r."""
    cut = cut_values(n, u, v, w)
    psi = simulate(n, u, v, w, scale, gamma, beta)
    e, nrm = expectation(psi, cut)
    cmin, cmax, amin, amax = extremes(n, cut)
    return dict(psi=psi, cut=cut, exp_c=e, norm=nrm, c_min=cmin, c_max=cmax, argmin=amin,
                argmax=amax, r=approximation_ratio(e, cmin, cmax))


def _expect_angles(n, u, v, cut, zz, xx):
    return expectation(circuit(n, u, v, zz, xx), cut)[0]


def grad_fd(n: int, u, v, w, scale: float, gamma, beta, h: float = 1e-5):
    """Central differences of <C> in each gamma_k and beta_k (complex128)."""
    gamma = np.asarray(gamma, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    cut = cut_values(n, u, v, w)

    def f(g, b):
        return expectation(simulate(n, u, v, w, scale, g, b), cut)[0]

    gg = np.zeros(len(gamma))
    gb = np.zeros(len(beta))
    for k in range(len(gamma)):
        e = np.zeros(len(gamma)); e[k] = h
        gg[k] = (f(gamma + e, beta) - f(gamma - e, beta)) / (2 * h)
        gb[k] = (f(gamma, beta + e) - f(gamma, beta - e)) / (2 * h)
    return gg, gb


def grad_param_shift(n: int, u, v, w, scale: float, gamma, beta):
    """Exact gradient by shifting one gate angle at a time by +-pi/2.

    Every gate is exp(-i theta/2 P) with P a Pauli product, so
    d<C>/d theta = (f(theta + pi/2) - f(theta - pi/2)) / 2. RZZ on edge e in
    layer k has theta = 2 gamma_k s w_e, so it contributes 2 s w_e times its
    shift difference to d/d gamma_k; RX on qubit q in layer k has
    phi = -2 beta_k and contributes -2 times its shift difference to d/d beta_k.
    """
    gamma = np.asarray(gamma, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    cut = cut_values(n, u, v, w)
    zz, xx = gate_angles(n, w, scale, gamma, beta)
    wf = np.asarray(w, dtype=np.float64)
    gg = np.zeros(len(gamma))
    gb = np.zeros(len(beta))
    s2 = math.pi / 2
    for k in range(len(gamma)):
        for e in range(len(wf)):
            zp = zz.copy(); zp[k, e] += s2
            zm = zz.copy(); zm[k, e] -= s2
            d = 0.5 * (_expect_angles(n, u, v, cut, zp, xx) - _expect_angles(n, u, v, cut, zm, xx))
            gg[k] += 2.0 * scale * wf[e] * d
        for q in range(n):
            xp = xx.copy(); xp[k, q] += s2
            xm = xx.copy(); xm[k, q] -= s2
            d = 0.5 * (_expect_angles(n, u, v, cut, zz, xp) - _expect_angles(n, u, v, cut, zz, xm))
            gb[k] += -2.0 * d
    return gg, gb


def analytic_p1_zz(n: int, J, gamma: float, beta: float, a: int, b: int) -> float:
    """<Z_a Z_b> after one layer exp(+i beta B) exp(-i gamma sum J ZZ) on |+>^n.

    Closed form for single-layer QAOA on ZZ Ising models without fields
    (Ozaeta, van Dam and McMahon 2022; Wang et al. 2018), in the sign
    convention of the paper's Eqs. UC and UB; J is the n x n coupling matrix
    (the weights times the phase scale s).
    """
    others = [c for c in range(n) if c not in (a, b)]
    pa = np.prod([math.cos(2 * gamma * J[a, c]) for c in others]) if others else 1.0
    pb = np.prod([math.cos(2 * gamma * J[b, c]) for c in others]) if others else 1.0
    pplus = np.prod([math.cos(2 * gamma * (J[a, c] + J[b, c])) for c in others]) if others else 1.0
    pminus = np.prod([math.cos(2 * gamma * (J[a, c] - J[b, c])) for c in others]) if others else 1.0
    return (-0.5 * math.sin(4 * beta) * math.sin(2 * gamma * J[a, b]) * (pa + pb)
            - 0.5 * math.sin(2 * beta) ** 2 * (pplus - pminus))


def analytic_p1_expectation(n: int, u, v, w, scale: float, gamma: float, beta: float) -> float:
    """<C> after one layer, from the closed-form <Z_u Z_v> of every edge:
    <C> = sum_e w_e (1 - <Z_u Z_v>) / 2 (C(x) counts w_e when x_u != x_v)."""
    J = np.zeros((n, n))
    for a, b, wt in zip(u, v, w):
        J[a, b] = J[b, a] = scale * wt
    return float(sum(wt * (1 - analytic_p1_zz(n, J, gamma, beta, a, b)) / 2 for a, b, wt in zip(u, v, w)))


def lr_chain(g_gamma, g_beta):
    """d<C>/d dgamma = sum_k (k+1)/p g_gamma[k]; d<C>/d dbeta = sum_k (1 - k/p) g_beta[k]."""
    p = len(g_gamma)
    k = np.arange(p, dtype=np.float64)
    return float(np.sum((k + 1) / p * np.asarray(g_gamma))), float(np.sum((1 - k / p) * np.asarray(g_beta)))


# ------------------------------------------------------------- Sec. II-D
# The random numbers of the sampling methodology are draws of the SplitMix64
# stream of ``inputs`` (draw k of stream ``seed``); the CUDA path generates the
# same draws on the device from the generator's published definition.

def sample_cuts(n: int, u, v, w, xs) -> np.ndarray:
    """C(x) of each given bitstring, literally sum over edges of w [x_k != x_l] (Sec. II-B)."""
    xs = [int(x) for x in np.asarray(xs, dtype=np.uint64)]
    out = np.empty(len(xs), dtype=np.int64)
    for i, x in enumerate(xs):
        if x >> n:
            raise ValueError("bitstring index out of range")
        out[i] = sum(int(we) for a, b, we in zip(u, v, w) if (x >> int(a) & 1) != (x >> int(b) & 1))
    return out


def sample_ratios(cuts, cmin: int, cmax: int) -> np.ndarray:
    """Approximation ratio of each sample, (C(x) - C_min) / (C_max - C_min) (Eq. r
    with a single bitstring in place of the mean; 1 when C_max = C_min)."""
    cuts = np.asarray(cuts, dtype=np.int64)
    if cmax == cmin:
        return np.ones(len(cuts))
    return np.array([float(c - cmin) / float(cmax - cmin) for c in cuts])


def random_bitstrings(n: int, count: int, seed: int) -> np.ndarray:
    """The random sampler (Sec. II-D): bitstring i is the top n bits of draw i."""
    from paper_2604_26423_b300 import inputs
    return inputs.splitmix64(seed, count) >> np.uint64(64 - n)


def subsample_indices(m: int, ns: int, reps: int, seed: int) -> np.ndarray:
    """reps subsets of ns distinct positions of a pool of m samples, each drawn
    uniformly without replacement (Sec. II-D) by a partial Fisher-Yates shuffle:
    step j of subset i takes draw k = i*ns + j, swaps position j with position
    j + floor(z_k (m - j) / 2^64) and keeps the value moved to position j.
    Returns an (reps, ns) array of pool positions in draw order."""
    from paper_2604_26423_b300 import inputs
    if not (1 <= ns <= m):
        raise ValueError("need 1 <= ns <= m")
    z = inputs.splitmix64(seed, reps * ns)
    out = np.empty((reps, ns), dtype=np.int64)
    for i in range(reps):
        pool = {}  # positions whose content differs from the identity
        for j in range(ns):
            k = j + (int(z[i * ns + j]) * (m - j) >> 64)
            vj, vk = pool.get(j, j), pool.get(k, k)
            pool[k] = vj
            pool[j] = vk
            out[i, j] = vk
    return out


def mean_of_means(r, ns: int, reps: int, seed: int):
    """Sec. II-D: the mean ratio of each subsample (summed in draw order), their
    grand mean <r_bar> and standard deviation sigma (over the reps means, 1/reps
    normalisation), and the random threshold <r_bar> + 3 sigma."""
    r = np.asarray(r, dtype=np.float64)
    idx = subsample_indices(len(r), ns, reps, seed)
    means = np.empty(reps)
    for i in range(reps):
        acc = 0.0
        for k in idx[i]:
            acc += float(r[k])
        means[i] = acc / ns
    g = 0.0
    for mu in means:
        g += float(mu)
    g /= reps
    var = 0.0
    for mu in means:
        d = float(mu) - g
        var += d * d
    sigma = math.sqrt(var / reps)
    return dict(means=means, grand_mean=g, sigma=sigma, threshold=g + 3.0 * sigma)


REGIME_RANDOM, REGIME_TRANSITION, REGIME_NOISE_TOLERANT, REGIME_ABOVE_RANDOM = 0, 1, 2, 3


def classify_regime(r_obs: float, rand_mean: float, rand_sigma: float, ideal_mean=None, ideal_sigma=None) -> int:
    """Sec. II-D: random when r_obs lies within or below the random sampler's 3-sigma
    interval (not above its threshold); otherwise noise-tolerant when r_obs reaches
    the noiseless interval (r_obs >= ideal_mean - 3 ideal_sigma), else transition.
    Without a noiseless reference a result above the threshold is only
    'statistically meaningful' (REGIME_ABOVE_RANDOM). -1 for a NaN or negative sigma."""
    if math.isnan(rand_sigma) or rand_sigma < 0:
        return -1
    if ideal_mean is not None and (math.isnan(ideal_sigma) or ideal_sigma < 0):
        return -1
    if not r_obs > rand_mean + 3.0 * rand_sigma:
        return REGIME_RANDOM
    if ideal_mean is None:
        return REGIME_ABOVE_RANDOM
    if r_obs >= ideal_mean - 3.0 * ideal_sigma:
        return REGIME_NOISE_TOLERANT
    return REGIME_TRANSITION


# ------------------------------------------------------------- Sec. II-C
# Depolarizing channel on the two qubits (i, j) of every ZZ gate, applied right
# after the gate: E(rho) = (1 - eps) rho + eps (I/4 (x) Tr_ij rho), i.e. with
# probability eps one of the 16 two-qubit Paulis (identity included), uniformly.
# Trajectory t draws, for gate g = k m + e (layer k, edge e in input order),
# draw t (p m) + g of stream `seed`: an error when its top 53 bits times 2^-53
# are below eps, the Pauli from its low 4 bits (bits 0-1 on i, 2-3 on j;
# 0 I, 1 X, 2 Y, 3 Z).

def _apply_pauli(psi, x, q, kind):
    if kind == 0:
        return psi
    b = (x >> q) & 1
    if kind == 1:
        return psi[x ^ (1 << q)]
    if kind == 3:
        return psi * (1 - 2 * b)
    return 1j * (2 * b - 1) * psi[x ^ (1 << q)]  # Y = [[0, -i], [i, 0]]


def noisy_trajectory(n: int, u, v, w, scale: float, gamma, beta, eps: float, seed: int, t: int) -> np.ndarray:
    """State of trajectory t: |+>, then per layer every ZZ gate exp(-i gamma_k s w_e Z_i Z_j)
    followed by its sampled Pauli error, then exp(+i beta_k X_q) on every qubit."""
    from paper_2604_26423_b300 import inputs
    gamma = np.atleast_1d(np.asarray(gamma, dtype=np.float64))
    beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
    p, m = len(gamma), len(u)
    x = np.arange(1 << n, dtype=np.int64)
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    draws = inputs.splitmix64(seed, p * m, offset=t * p * m)
    for k in range(p):
        for e in range(m):
            i, j = int(u[e]), int(v[e])
            zz = (1 - 2 * ((x >> i) & 1)) * (1 - 2 * ((x >> j) & 1))
            psi = psi * np.exp(-1j * gamma[k] * scale * float(w[e]) * zz)
            d = int(draws[k * m + e])
            if (d >> 11) * 2.0 ** -53 < eps:
                psi = _apply_pauli(psi, x, i, d & 3)
                psi = _apply_pauli(psi, x, j, (d >> 2) & 3)
        c, s_ = math.cos(beta[k]), math.sin(beta[k])
        for q in range(n):
            flip = psi[x ^ (1 << q)]
            psi = c * psi + 1j * s_ * flip
    return psi


def _pauli_matrix(n, q, kind):
    one = {0: np.eye(2), 1: np.array([[0, 1], [1, 0]]), 2: np.array([[0, -1j], [1j, 0]]),
           3: np.array([[1, 0], [0, -1]])}[kind]
    mat = np.array([[1.0]])
    for b in range(n - 1, -1, -1):  # bit q of the index is qubit q
        mat = np.kron(mat, one if b == q else np.eye(2))
    return mat


def noisy_density(n: int, u, v, w, scale: float, gamma, beta, eps: float) -> float:
    """Exact noisy <C> by density-matrix evolution (n <= 6): after every ZZ gate
    rho -> (1 - eps) rho + eps/16 sum_P P rho P over the 16 Paulis on (i, j)."""
    gamma = np.atleast_1d(np.asarray(gamma, dtype=np.float64))
    beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
    N = 1 << n
    x = np.arange(N)
    plus = np.full(N, 2.0 ** (-n / 2), dtype=np.complex128)
    rho = np.outer(plus, plus.conj())
    X = [_pauli_matrix(n, q, 1) for q in range(n)]
    for k in range(len(gamma)):
        for e in range(len(u)):
            i, j = int(u[e]), int(v[e])
            zz = (1 - 2 * ((x >> i) & 1)) * (1 - 2 * ((x >> j) & 1))
            d = np.exp(-1j * gamma[k] * scale * float(w[e]) * zz)
            rho = d[:, None] * rho * d.conj()[None, :]
            acc = np.zeros_like(rho)
            for a in range(4):
                for b in range(4):
                    P = _pauli_matrix(n, i, a) @ _pauli_matrix(n, j, b)
                    acc += P @ rho @ P.conj().T
            rho = (1 - eps) * rho + eps / 16 * acc
        for q in range(n):
            U = math.cos(beta[k]) * np.eye(N) + 1j * math.sin(beta[k]) * X[q]
            rho = U @ rho @ U.conj().T
    cut = cut_values(n, u, v, w)
    return float(np.real(np.sum(np.diag(rho) * cut)))


def overlap_ratio(r_noisy: float, r_ideal: float, r_random: float) -> float:
    """r_ovl = (r_QPU - r_random) / (r_ideal - r_random) (Sec. II-C)."""
    return (r_noisy - r_random) / (r_ideal - r_random)


def fit_k0(eps_acc, r_ovl) -> float:
    """k0 of Eq. noise, r_ovl = 2^(-k0 eps_acc): least squares on log2 r_ovl = -k0 eps_acc
    (a line through the origin); points with r_ovl <= 0 are left out."""
    a = np.asarray(eps_acc, dtype=np.float64)
    r = np.asarray(r_ovl, dtype=np.float64)
    keep = r > 0
    a, r = a[keep], r[keep]
    num = 0.0
    den = 0.0
    for ai, ri in zip(a, r):
        num += ai * math.log2(ri)
        den += ai * ai
    return -num / den if den > 0 else float("nan")
