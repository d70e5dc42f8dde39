"""Benchmark: LR-QAOA layers/s at n = 33 qubits (complex64 state, 64 GiB) on one B300.

Workload (the n = 33 single-GPU configuration): fully connected weighted MaxCut
K_33 (528 edges), integer weights uniform in {1..10} (SplitMix64 seed 33),
phases scaled by 1/10, LR-QAOA p = 3 with dgamma = 0.6, dbeta = 0.3.

* step (``value``): one preparation of |psi_3> (all fused HBM passes), the FP64
  <C> / norm reduction and r, and 4096 measurement shots, on a context whose
  per-graph preprocessing (weight matrix, exhaustive C_min / C_max) is done
  before the timed region. The state (64 GiB) is far larger than L2, so no
  flush is needed between steps.
* ``e2e``: the same job through the public C ABI from host arrays: per step
  qaoa_init_graph (edge arrays from pinned host memory, exhaustive extremes),
  qaoa_run, qaoa_expect and qaoa_sample back to host memory, qaoa_free.
* ``roofline``: bytes over the event-timed duration of the fused forward pass
  kernels, against the measured HBM copy bandwidth. ``achieved`` / ``frac``
  (= ``frac_alg``) count the algorithmic bytes of the method's pass schedule
  with three mixer groups per layer at n = 33: N b (2 (1 + 2p) - 1) per step
  (7 passes, the first write-only; 893 GB at K_33, p = 3); ``frac_floor``
  counts one read and one write per layer (2 N b p); ``frac_pass`` the bytes
  the library's own passes move (its plan's pass count).
* ``grad``: the adjoint gradient's cost relative to the forward run on the
  gradient workload (K_28, complex64, p = 10): t(qaoa_grad: forward, <C>,
  backward, all 2p layer derivatives) / t(qaoa_run + qaoa_expect), with the
  forward's pass outputs stored (``ratio``, the default) and with two state
  vectors only, psi uncomputed (``ratio_two_vectors``).
* ``batch``: the batched workload (4096 seeded instances, n uniform in 10..22,
  p in 1..10, 1/3 K_n, 1/3 chains, 1/3 random 3-regular graphs, complex64,
  forward with <C>, r and extremes, and forward + adjoint gradients): instances/s
  of one CUDA-graph replay of the persistent batch kernels, scheduling knobs
  picked by the autotuner; ``--batch-reps`` replays are timed.
* ``configs``: qaoa_run + qaoa_expect (event-timed, after one untimed run) on
  K_30 for p = 1..10 in complex128 and complex64 with 4096 shots each, K_32
  complex128 with recomputed and streamed cut values, K_32 complex64 with its
  state error against the complex128 run (also in ``result.c64_err_vs_c128``),
  K_33 complex64 with the streamed cost diagonal, and K_34 complex64.
* ``stats``: the sampling methodology of Sec. II-D on the workload's graph and
  final state: cut values and ratios of 2^26 uniform random bitstrings (the
  random sampler; kernel time, bitstrings/s), the ratios of the step's 4096
  shots, the mean of 100 subsample means at 10 and 100 shots for both, and the
  regime of the first 10 shots.
* ``noise``: noisy LR-QAOA (Sec. II-C) on K_12, p = 10, complex64 (one rate
  also in complex128): 4096 depolarizing-channel trajectories per rate, trajectories/s of the kernel, the
  noisy r, r_ovl and the k0 fit of Eq. noise.
* ``--qubits n`` runs the same step on K_n (smaller cases for profiling; the
  JSON line then names that workload).
* ``cpu_baseline`` / ``--impl reference``: the gate-by-gate complex128 oracle on
  the host cores, timed on one LR-QAOA layer of K_nc (nc chosen so the sample
  takes seconds), scaled to one layer of K_33 by amplitude count times gate
  count.

Multi-GPU (torchrun, N > 1): independent replicas (the method's one-GPU path
does not shard); each rank runs the same workload on its own GPU, timing is the
max over ranks, and ``value`` counts the layers of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS, P, DGAMMA, DBETA, SCALE, SEED, SHOTS = 33, 3, 0.6, 0.3, 0.1, 33, 4096
METRIC = "LR-QAOA layers/s at n=33 (complex64, K_33, p=3)"
GRAD_N, GRAD_P, GRAD_DGAMMA, GRAD_DBETA = 28, 10, 0.6, 0.3
BATCH_COUNT, BATCH_SEED = 4096, 2604
PROFILE_JSON = os.path.join(ROOT, "profiles", "fwd_pass_kernel_traffic.json")
# sources that determine the forward pass kernels' DRAM traffic (kernels, plans, descriptors, dispatch)
KERNEL_SOURCES = ["paper_2604_26423_b300/csrc/pass_kernel.cuh", "paper_2604_26423_b300/csrc/device.cuh",
                  "paper_2604_26423_b300/csrc/plan.cpp", "paper_2604_26423_b300/csrc/desc.cu",
                  "paper_2604_26423_b300/csrc/spec_fwd.cu", "paper_2604_26423_b300/csrc/api.cu"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int):
    """Max over ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle baseline
def oracle_layer_time(budget_s: float = 12.0):
    """Times one LR-QAOA layer of the oracle on K_nc; returns (seconds, nc, threads)."""
    import oracle
    from paper_2604_26423_b300 import inputs
    nc = 20
    t = 0.0
    while True:
        u, v, w = inputs.complete_graph(nc, SEED)
        g, b = oracle.lr_schedule(P, DGAMMA, DBETA)
        zz, xx = oracle.gate_angles(nc, w, SCALE, g[:1], b[:1])
        t0 = time.perf_counter()
        oracle.circuit(nc, u, v, zz, xx)
        t = time.perf_counter() - t0
        # grow the sample while it stays inside the budget (state doubles, gates grow)
        grow = 2.0 * ((nc + 1) * nc / 2 + nc + 1) / (nc * (nc - 1) / 2 + nc)
        if t * grow > budget_s or nc >= 26:
            return t, nc, oracle.num_threads()
        nc += 1


def cpu_baseline(budget_s: float = 12.0):
    t, nc, thr = oracle_layer_time(budget_s)
    gates_c = nc * (nc - 1) / 2 + nc
    gates_33 = N_QUBITS * (N_QUBITS - 1) / 2 + N_QUBITS
    t33 = t * 2 ** (N_QUBITS - nc) * gates_33 / gates_c
    return {"value": 1.0 / t33, "unit": "layers/s", "cores": thr, "kind": "oracle",
            "sample": f"one LR-QAOA layer of K_{nc} ({nc*(nc-1)//2} RZZ + {nc} RX gates, complex128, "
                      f"{(16 << nc) >> 20} MiB state) in {t:.2f} s, scaled to K_{N_QUBITS} by 2^{N_QUBITS-nc} "
                      f"amplitudes x {gates_33:.0f}/{gates_c:.0f} gates"}


# ------------------------------------------------------------------ GPU arm
def grad_ratio(args, stream, reps: int = 3):
    """Adjoint gradient time over forward time (by default K_28, complex64, p = 10)."""
    import torch
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import Simulator

    gn, gp = args.grad_n, args.grad_p
    u, v, w = inputs.complete_graph(gn, SEED)
    with Simulator(gn, u, v, w, SCALE, "c64", cost_mode=args.cost_mode, with_grad=True) as s:
        def fwd():
            s.run(gp, GRAD_DGAMMA, GRAD_DBETA)
            return s.expect()

        def bwd():
            return s.grad(gp, GRAD_DGAMMA, GRAD_DBETA)

        def timed(f):
            for _ in range(3):
                f()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                out = f()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps, out

        t_fwd, _ = timed(fwd)
        # the adjoint with the forward's pass outputs stored (one state sweep
        # fewer per adjoint pass; the library's default when memory allows)
        t_grad, r = timed(bwd)
        # the adjoint that holds two vectors only: psi uncomputed with the
        # inverse gates and written back in every pass
        s.set_opts(dict(grad_checkpoint=False))
        t_grad2, r2 = timed(bwd)
        s.set_opts(dict())
    # the same ratios counted in state sweeps (one read or write of 2^n
    # amplitudes) of the plan's P passes: the forward moves 2P - 1 (its first
    # pass only writes); the adjoint with stored states 3P - 2 (read psi and
    # lambda, write lambda; the first reads psi only, the last writes
    # nothing), with two vectors 4P - 4 (psi written back as well, except by
    # the first pass, whose input the forward's last pass left in place)
    from paper_2604_26423_b300.qaoa import describe_plan
    npass = int(re.search(r"passes=(\d+)", describe_plan(gn, gp, "c64")).group(1))
    sw_f, sw_c, sw_2 = 2 * npass - 1, 3 * npass - 2, 4 * npass - 4
    return {"workload": f"K_{gn} complex64, p={gp}, dgamma={GRAD_DGAMMA}, dbeta={GRAD_DBETA}",
            "forward_ms": t_fwd, "grad_ms": t_grad, "ratio": t_grad / t_fwd,
            "grad_ms_two_vectors": t_grad2, "ratio_two_vectors": t_grad2 / t_fwd,
            "sweeps": {"passes": npass, "forward": sw_f, "adjoint": sw_c, "adjoint_two_vectors": sw_2,
                       "ratio_bound": round(1 + sw_c / sw_f, 3),
                       "ratio_two_vectors_bound": round(1 + sw_2 / sw_f, 3)},
            "two_vectors_rel_diff": abs(r2["d_dgamma"] - r["d_dgamma"]) / max(1e-30, abs(r["d_dgamma"])),
            "exp_c": r["exp_c"], "d_dgamma": r["d_dgamma"], "d_dbeta": r["d_dbeta"]}


def _l2_dev(a, b, chunk=1 << 27):
    """L2 distance of two device state vectors (complex64 / complex128), chunked."""
    import torch
    acc = 0.0
    for i in range(0, a.numel(), chunk):
        d = a[i:i + chunk].to(torch.complex128) - b[i:i + chunk].to(torch.complex128)
        acc += float(torch.sum(d.real ** 2 + d.imag ** 2))
    return acc ** 0.5


def config_bench(args, stream):
    """The other workloads of the method (qaoa_run + qaoa_expect, event-timed
    after one untimed run):
    * K_30, p = 1..10, complex128 and complex64 (16 GB / 8 GB states), each
      with 4096 shots (the single-GPU 30-qubit depth sweep of Sec. III-A);
    * K_32 complex128 (64 GiB, FP64-ALU-bound) with recomputed and with
      streamed cut values, and K_32 complex64 against it: the stated error of
      the precision path where the oracle cannot run (state L2, |r64 - r128|);
    * K_33 complex64 with the streamed int32 cost diagonal;
    * K_34 complex64 (128 GiB), p = 3;
    * sparse graphs: random 3-regular on 32 vertices, a chain on 33."""
    import torch
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import Simulator

    def timed(s, p):
        s.run(p, DGAMMA, DBETA)
        s.expect()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.run(p, DGAMMA, DBETA)
        r = s.expect()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    def row(n, prec, mode, p, ms, r, **kw):
        d = {"n": n, "precision": prec, "cost_mode": mode, "p": p, "ms": ms, "layers_per_s": p / ms * 1e3,
             "r": r["r"], "exp_c": r["exp_c"]}
        d.update(kw)
        return d

    out = {"k30_depth_sweep": [], "runs": []}
    u, v, w = inputs.complete_graph(30, SEED)
    for prec in ("c128", "c64"):
        with Simulator(30, u, v, w, SCALE, prec) as s:
            for p in range(1, 11):
                ms, r = timed(s, p)
                t0 = time.perf_counter()
                shots = s.sample(SHOTS, seed=SEED + p)
                out["k30_depth_sweep"].append(row(30, prec, "recompute", p, ms, r,
                                                  shots=len(shots), sample_ms=(time.perf_counter() - t0) * 1e3))
        torch.cuda.empty_cache()
    u, v, w = inputs.complete_graph(32, SEED)
    with Simulator(32, u, v, w, SCALE, "c128") as s128:
        ms, r128 = timed(s128, P)
        out["runs"].append(row(32, "c128", "recompute", P, ms, r128))
        with Simulator(32, u, v, w, SCALE, "c64") as s64:
            ms, r64 = timed(s64, P)
            out["runs"].append(row(32, "c64", "recompute", P, ms, r64))
            out["c64_err_vs_c128"] = {
                "workload": "K_32 (seed 33), p=3, dgamma=0.6, dbeta=0.3: complex64 vs complex128 on this GPU",
                "state_l2": _l2_dev(s64.state(), s128.state()), "r_abs": abs(r64["r"] - r128["r"]),
                "exp_c_rel": abs(r64["exp_c"] - r128["exp_c"]) / abs(r128["exp_c"])}
    torch.cuda.empty_cache()
    with Simulator(32, u, v, w, SCALE, "c128", cost_mode="stream") as s:
        ms, r = timed(s, P)
        out["runs"].append(row(32, "c128", "stream", P, ms, r))
    torch.cuda.empty_cache()
    u, v, w = inputs.complete_graph(33, SEED)
    with Simulator(33, u, v, w, SCALE, "c64", cost_mode="stream") as s:
        ms, r = timed(s, P)
        out["runs"].append(row(33, "c64", "stream", P, ms, r))
    torch.cuda.empty_cache()
    u, v, w = inputs.complete_graph(34, SEED)
    with Simulator(34, u, v, w, SCALE, "c64") as s:
        ms, r = timed(s, P)
        out["runs"].append(row(34, "c64", "recompute", P, ms, r))
    torch.cuda.empty_cache()
    # sparse instances at large n: a random 3-regular graph (48 edges) and a
    # chain (32 edges) on 32 and 33 vertices
    for n, kind, make in ((32, "regular3", inputs.regular3_graph), (33, "chain", inputs.chain_graph)):
        u, v, w = make(n, SEED)
        with Simulator(n, u, v, w, SCALE, "c64") as s:
            ms, r = timed(s, P)
            out["runs"].append(row(n, "c64", "recompute", P, ms, r, graph=kind, edges=len(u)))
        torch.cuda.empty_cache()
    return out


def batch_bench(args, stream):
    """Instances/s of the 4096-instance batch (forward, and forward + adjoint)."""
    import torch
    from paper_2604_26423_b300 import inputs, tune
    from paper_2604_26423_b300.qaoa import Batch

    count = args.batch_count
    batch = inputs.batch_instances(count, BATCH_SEED)
    out = {"workload": f"{count} instances, n in 10..22, p in 1..10, K_n / chain / 3-regular, complex64"}
    for grad in (False, True):
        best, timings = tune.tune_batch(batch, with_grad=grad,
                                        candidates=tune.batch_candidates(solo=(25,), units=(1, 2), ctas=(2,)))
        b = Batch(batch, with_grad=grad, opts=best["opts"])
        try:
            for _ in range(2):
                b.run()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.batch_reps):
                b.run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.batch_reps
            res = b.results()
            key = "grad" if grad else "forward"
            out[key] = {"instances_per_s": count / ms * 1e3, "ms": ms, "opts": best["opts"],
                        "state_gbytes": b.bytes() / 1e9, "state_gbps": b.bytes() / ms / 1e6,
                        "mean_r": float(res["r"].mean()), "describe": b.describe()}
        finally:
            b.close()
    return out


def stats_bench(sim, shots, stream, pool: int = 1 << 26):
    """Sampling methodology (Sec. II-D) on the workload's graph and state: cut
    values and ratios of a pool of uniform random bitstrings (the random
    sampler, kernel timed with CUDA events), the ratios of the step's shots, the
    mean of 100 subsample means at 10 and 100 shots for both pools, and the
    regime of the first 10 shots against the two distributions."""
    import torch
    from paper_2604_26423_b300.qaoa import REGIMES, classify_regime, mean_of_means

    sim.sample_cuts(count=1024, seed=1)  # weight planes built, extremes known
    sim.profile(True)
    t0 = time.perf_counter()
    rand = sim.sample_cuts(count=pool, seed=SEED + 2)
    wall = time.perf_counter() - t0
    kern = sim.profile_read("sample")
    sim.profile(False)
    r_rand = rand["r"]
    r_shots = sim.sample_cuts(shots)["r"]
    n = sim.n
    out = {"random_sampler": {"bitstrings": pool, "kernel_ms": kern["ms"], "wall_ms": wall * 1e3,
                              "bitstrings_per_s": pool / (kern["ms"] * 1e-3),
                              "edge_terms_per_s": pool * n * (n - 1) / 2 / (kern["ms"] * 1e-3),
                              "mean_r": float(r_rand.mean())},
           "shots": {"count": int(r_shots.numel()), "mean_r": float(r_shots.mean())}}
    for ns in (10, 100):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mr = mean_of_means(r_rand, ns, 100, seed=ns)
        mi = mean_of_means(r_shots, ns, 100, seed=ns + 1)
        t = time.perf_counter() - t0
        out[f"ns{ns}"] = {"random": {k: mr[k] for k in ("grand_mean", "sigma", "threshold")},
                          "noiseless": {k: mi[k] for k in ("grand_mean", "sigma", "threshold")},
                          "ms_both": t * 1e3}
    r_obs = float(r_shots[:10].mean())
    m10 = out["ns10"]
    reg = classify_regime(r_obs, m10["random"]["grand_mean"], m10["random"]["sigma"],
                          m10["noiseless"]["grand_mean"], m10["noiseless"]["sigma"])
    out["regime_first_10_shots"] = {"r_obs": r_obs, "regime": REGIMES.get(reg, reg)}
    return out


def noise_bench(args, trajectories: int = 4096):
    """Noisy LR-QAOA (Sec. II-C) on K_12, p = 10: `trajectories` Monte Carlo
    trajectories per depolarizing rate (complex64, one CTA each, kernel timed
    with CUDA events), the noisy r, the overlap ratio r_ovl against the
    noiseless r and the random sampler's, and the fit of Eq. noise; the same
    trajectories of one rate also in complex128."""
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import Simulator, fit_k0, lr_angles, overlap_ratio

    n, p = 12, 10
    u, v, w = inputs.complete_graph(n, SEED)
    g, b = lr_angles(p, DGAMMA, DBETA)
    out = {"workload": f"K_{n} (seed {SEED}), p={p}, dgamma={DGAMMA}, dbeta={DBETA}, complex64, "
                       f"{trajectories} trajectories per rate", "rates": []}
    with Simulator(n, u, v, w, SCALE, "c128") as s:
        s.noisy_expect(g, b, 0.002, 64, seed=1)  # warm-up
        s.profile(True)
        res = s.noisy_expect(g, b, 0.002, trajectories, seed=SEED)
        k = s.profile_read("small")
        s.profile(False)
        out["complex128_eps_0.002"] = {"r_noisy": res["r"], "kernel_ms": k["ms"],
                                       "trajectories_per_s": trajectories / (k["ms"] * 1e-3)}
    with Simulator(n, u, v, w, SCALE, "c64") as s:
        ext = s.extremes()
        r_rand = (float(np.sum(w)) / 2 - ext["c_min"]) / (ext["c_max"] - ext["c_min"])
        s.noisy_expect(g, b, 0.0, 64, seed=1)  # warm-up
        ideal = s.noisy_expect(g, b, 0.0, 1, seed=1)["r"]
        a_list, o_list = [], []
        for eps in (0.0005, 0.002, 0.005, 0.01):
            s.profile(True)
            res = s.noisy_expect(g, b, eps, trajectories, seed=SEED)
            k = s.profile_read("small")
            s.profile(False)
            ro = overlap_ratio(res["r"], ideal, r_rand)
            acc = p * len(u) * eps
            a_list.append(acc)
            o_list.append(ro)
            out["rates"].append({"eps": eps, "eps_acc": acc, "r_noisy": res["r"], "r_ovl": ro,
                                 "kernel_ms": k["ms"], "trajectories_per_s": trajectories / (k["ms"] * 1e-3)})
    out.update({"r_ideal": ideal, "r_random": r_rand, "k0": fit_k0(a_list, o_list)})
    return out


def run_gpu(args):
    import torch
    from paper_2604_26423_b300 import inputs
    from paper_2604_26423_b300.qaoa import Simulator

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    nq = args.qubits
    u, v, w = inputs.complete_graph(nq, SEED)
    stream = torch.cuda.current_stream()
    fwd_opts = {}
    if args.fwd_shape:
        fwd_opts["shape"] = args.fwd_shape
    if args.l2_prefetch:
        fwd_opts["l2_prefetch"] = True
    sim = Simulator(nq, u, v, w, SCALE, "c64", cost_mode=args.cost_mode, opts=fwd_opts or None)
    state_buf = sim._state_t

    def step():
        sim.run(P, DGAMMA, DBETA)
        res = sim.expect()
        shots = sim.sample(SHOTS, seed=SEED + 1)
        return res, shots

    for _ in range(args.warmup):
        res, shots = step()
    sim.profile(True)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            res, shots = step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms_local = e0.elapsed_time(e1)
    prof = sim.profile_read("pass")
    launches = sum(sim.profile_read(k)["launches"] for k in ("pass", "adjoint", "cost", "sample", "small"))
    launches_all = sim.profile_read(5)["launches"]
    sim.profile(False)
    ms = reduce_max(ms_local, world)

    # end to end through the C ABI from host arrays (per step: init, run, expect, sample, free)
    uh = torch.from_numpy(u).pin_memory().numpy()
    vh = torch.from_numpy(v).pin_memory().numpy()
    wh = torch.from_numpy(w).pin_memory().numpy()
    stats = None if args.no_stats else stats_bench(sim, shots, stream)
    sim.close()
    noise = None if args.no_noise else noise_bench(args)

    def e2e_step():
        s2 = Simulator(nq, uh, vh, wh, SCALE, "c64", cost_mode=args.cost_mode, state=state_buf,
                       opts=fwd_opts or None)
        s2.run(P, DGAMMA, DBETA)
        r2 = s2.expect()
        sh = s2.sample(SHOTS, seed=SEED + 1)
        s2.close()
        return r2, sh

    e2e_s = float("nan")
    if args.e2e_steps > 0:
        e2e_step()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = reduce_max(time.perf_counter() - t0, world)
        barrier(world)
    del state_buf
    torch.cuda.empty_cache()
    grad = None if args.no_grad else grad_ratio(args, stream)
    batch = None if args.no_batch else batch_bench(args, stream)
    configs = None if args.no_configs else config_bench(args, stream)

    peak, peak_kind = measured_peak()
    # three byte counts over the same event-timed forward pass kernels:
    #   algorithmic (the headline): N b (2 passes - 1) for the pass schedule
    #     with three mixer groups per layer at n = 33 (1 + 2p passes, the
    #     first write-only), whatever plan the library runs;
    #   floor: one read and one write of the state per layer (2 N b p);
    #   pass: the bytes the plan's passes actually move (its own pass count)
    nb_state = 8.0 * (1 << nq)
    alg_passes = 1 + P * (3 - 1)
    alg_bytes = nb_state * (2 * alg_passes - 1) * args.steps
    floor_bytes = 2.0 * nb_state * P * args.steps
    kern_s = prof["ms"] * 1e-3
    achieved = alg_bytes / kern_s / 1e9 if kern_s > 0 else 0.0
    achieved_pass = prof["bytes"] / kern_s / 1e9 if kern_s > 0 else 0.0
    achieved_floor = floor_bytes / kern_s / 1e9 if kern_s > 0 else 0.0
    traffic = None
    try:
        with open(PROFILE_JSON) as f:
            pj = json.load(f)
        # the counters were scaled to the K_33 recompute-mode step: other workloads get null
        if pj.get("kernel_hash") == kernel_hash() and nq == N_QUBITS and args.cost_mode == "recompute":
            traffic = pj.get("dram_bytes_per_launch_n33")
    except Exception:
        pass
    layers = P * args.steps * world
    metric = METRIC if nq == N_QUBITS else METRIC.replace("33", str(nq))
    out = {
        "metric": metric, "value": layers / (ms * 1e-3), "unit": "layers/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32 pairs), fp64 reductions",
        "data": f"synthetic: SplitMix64 K_{nq} weights in {{1..10}}",
        "config": {"workload": f"LR-QAOA K_{nq} weighted MaxCut, complex64 ({(8 << nq) >> 20} MiB state), p=3, "
                               "dgamma=0.6, dbeta=0.3, <C>, r and 4096 shots per step",
                   "n": nq, "p": P, "precision": "complex64", "cost_mode": args.cost_mode,
                   "fwd_opts": fwd_opts,
                   "state_bytes": 8 << nq,
                   "l2": f"state {(8 << nq) >> 20} MiB vs 126 MB L2" + (" (no flush needed)" if nq >= 25 else ""),
                   "parallelism": f"replicas x{world}"},
        "e2e": None if args.e2e_steps <= 0 else {"value": P * args.e2e_steps * world / e2e_s, "unit": "layers/s",
                "h2d_bytes_per_step": int(u.nbytes + v.nbytes + w.nbytes + 16),
                "d2h_bytes_per_step": int(SHOTS * 8 + 7 * 8)},
        "gpu_launches": int(launches_all) if launches_all else int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "frac_alg": achieved / peak, "frac_floor": achieved_floor / peak,
                     "frac_pass": achieved_pass / peak, "achieved_pass": achieved_pass,
                     "alg_bytes_per_step": alg_bytes / args.steps, "floor_bytes_per_step": floor_bytes / args.steps,
                     "pass_bytes_per_step": prof["bytes"] / args.steps,
                     "passes_per_step": prof["launches"] / args.steps, "alg_passes_per_step": alg_passes,
                     "kernel_ms_per_step": prof["ms"] / args.steps,
                     "kernel": "forward pass kernels (fwd_spec_kernel, fwd_pass_kernel)", "launches": prof["launches"],
                     "bytes_per_launch": prof["bytes"] / max(1, prof["launches"]),
                     "ms_per_launch": prof["ms"] / max(1, prof["launches"])},
        "result": {"exp_c": res["exp_c"], "r": res["r"], "norm": res["norm"], "c_max": res["c_max"]},
        "clocks": clk.summary(),
    }
    if grad is not None:
        out["grad"] = grad
    if batch is not None:
        out["batch"] = batch
    if configs is not None:
        out["configs"] = configs
        if "c64_err_vs_c128" in configs:
            out["result"]["c64_err_vs_c128"] = configs["c64_err_vs_c128"]
    if stats is not None:
        out["stats"] = stats
    if noise is not None:
        out["noise"] = noise
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_budget)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_layer_time(min(args.cpu_budget, 4.0))
    t0 = time.perf_counter()
    samples = []
    for _ in range(args.steps):
        samples.append(cpu_baseline(min(args.cpu_budget, 4.0)))
    wall = time.perf_counter() - t0
    v = statistics.median(s["value"] for s in samples)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "layers/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (oracle)",
           "data": "synthetic: SplitMix64 K_n weights in {1..10}",
           "config": {"workload": "LR-QAOA K_33 weighted MaxCut, p=3 (bounded oracle sample, scaled)",
                      "n": N_QUBITS, "p": P},
           "cpu_baseline": {"value": v, "unit": "layers/s", "cores": samples[-1]["cores"], "kind": "oracle",
                            "sample": samples[-1]["sample"]},
           "e2e": {"value": v, "unit": "layers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cost-mode", default="recompute", choices=["recompute", "stream"])
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--no-stats", action="store_true")
    ap.add_argument("--no-noise", action="store_true")
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT)
    ap.add_argument("--qubits", type=int, default=N_QUBITS)
    ap.add_argument("--grad-n", type=int, default=GRAD_N, help="qubits of the gradient leg (profiling)")
    ap.add_argument("--grad-p", type=int, default=GRAD_P, help="depth of the gradient leg (profiling)")
    ap.add_argument("--fwd-shape", default=None, choices=["4x3", "5x3", "4x4", "5x2", "5x4"],
                    help="forward tile shape of the step (profiling; default: the library's)")
    ap.add_argument("--l2-prefetch", action="store_true", help="prefetch each CTA's next tile into L2 (profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
