"""Thin ctypes binding of libqaoa.so (C ABI in include/qaoa.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels. PyTorch supplies device memory (the state and auxiliary buffers
are torch tensors handed over by pointer) and the CUDA stream. There is no CPU
fallback: without the built library or a CUDA device, constructing a
``Simulator`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

QAOA_OK, QAOA_EINVAL, QAOA_ENOMEM, QAOA_ECUDA, QAOA_ETIMEOUT, QAOA_ESTATE = range(6)
C64, C128 = 0, 1
COST_AUTO, COST_RECOMPUTE, COST_STREAM = 0, 1, 2
_PREC = {"c64": C64, "complex64": C64, C64: C64, "c128": C128, "complex128": C128, C128: C128}
_COST = {"auto": COST_AUTO, "recompute": COST_RECOMPUTE, "stream": COST_STREAM,
         COST_AUTO: COST_AUTO, COST_RECOMPUTE: COST_RECOMPUTE, COST_STREAM: COST_STREAM}
_ERRNAME = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ESTATE"}

# every entry point declared in include/qaoa.h
EXPORTS = ("qaoa_state_bytes", "qaoa_aux_bytes", "qaoa_init_graph", "qaoa_run", "qaoa_run_angles",
           "qaoa_expect", "qaoa_sample", "qaoa_grad", "qaoa_grad_angles", "qaoa_cost_diag",
           "qaoa_state_ptr", "qaoa_describe_plan", "qaoa_profile_enable", "qaoa_profile_read",
           "qaoa_last_error", "qaoa_free", "qaoa_sample_state_noalloc",
           "qaoa_batch_create", "qaoa_batch_run", "qaoa_batch_results", "qaoa_batch_state",
           "qaoa_batch_describe", "qaoa_batch_bytes", "qaoa_batch_last_error", "qaoa_batch_free",
           "qaoa_sample_cuts", "qaoa_mean_of_means", "qaoa_classify_regime", "qaoa_noisy_expect",
           "qaoa_overlap_ratio", "qaoa_fit_k0", "qaoa_max_weight_sum", "qaoa_quantize_weights",
           "qaoa_set_opts", "qaoa_get_opts", "qaoa_set_cost_choice")
PROFILE_KINDS = {"pass": 0, "adjoint": 1, "cost": 2, "sample": 3, "small": 4}

_lib = None


class QaoaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAME.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load():
    """Loads libqaoa.so (it must have been built; see ``paper_2604_26423_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2604_26423_b300.build`")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    i32p, f64p, u64p, i64p = P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_uint64), P(ctypes.c_int64)
    vp = ctypes.c_void_p
    lib.qaoa_state_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.qaoa_state_bytes.restype = ctypes.c_size_t
    lib.qaoa_aux_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.qaoa_aux_bytes.restype = ctypes.c_size_t
    lib.qaoa_init_graph.argtypes = [P(vp), ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, vp, ctypes.c_size_t, vp]
    lib.qaoa_run.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.qaoa_run_angles.argtypes = [vp, ctypes.c_int, f64p, f64p]
    lib.qaoa_expect.argtypes = [vp, f64p, f64p, f64p, i64p, i64p, u64p, u64p]
    lib.qaoa_sample.argtypes = [vp, ctypes.c_int, f64p, ctypes.c_uint64, u64p]
    lib.qaoa_grad.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, f64p, f64p, f64p, f64p, f64p]
    lib.qaoa_grad_angles.argtypes = [vp, ctypes.c_int, f64p, f64p, f64p, f64p, f64p]
    lib.qaoa_cost_diag.argtypes = [vp, vp]
    lib.qaoa_state_ptr.argtypes = [vp]
    lib.qaoa_state_ptr.restype = vp
    lib.qaoa_describe_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_char_p,
                                       ctypes.c_int]
    lib.qaoa_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.qaoa_profile_read.argtypes = [vp, ctypes.c_int, i64p, f64p, f64p]
    lib.qaoa_last_error.argtypes = [vp]
    lib.qaoa_last_error.restype = ctypes.c_char_p
    lib.qaoa_free.argtypes = [vp]
    lib.qaoa_free.restype = None
    lib.qaoa_batch_create.argtypes = [P(vp), ctypes.c_int, i32p, i32p, i64p, i32p, i32p, i32p, f64p, f64p,
                                      ctypes.c_double, ctypes.c_int, vp, vp]
    lib.qaoa_batch_run.argtypes = [vp]
    lib.qaoa_batch_results.argtypes = [vp, f64p, f64p]
    lib.qaoa_batch_state.argtypes = [vp, ctypes.c_int, P(vp)]
    lib.qaoa_batch_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.qaoa_batch_bytes.argtypes = [vp]
    lib.qaoa_batch_bytes.restype = ctypes.c_double
    lib.qaoa_batch_last_error.argtypes = [vp]
    lib.qaoa_batch_last_error.restype = ctypes.c_char_p
    lib.qaoa_batch_free.argtypes = [vp]
    lib.qaoa_batch_free.restype = None
    lib.qaoa_sample_cuts.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_uint64, vp, vp, vp]
    lib.qaoa_mean_of_means.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, vp, vp, vp]
    lib.qaoa_max_weight_sum.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.qaoa_max_weight_sum.restype = ctypes.c_int64
    lib.qaoa_quantize_weights.argtypes = [ctypes.c_int, f64p, ctypes.c_int64, i32p, f64p]
    lib.qaoa_noisy_expect.argtypes = [vp, ctypes.c_int, f64p, f64p, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
                                      vp, f64p, f64p]
    lib.qaoa_overlap_ratio.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.qaoa_overlap_ratio.restype = ctypes.c_double
    lib.qaoa_fit_k0.argtypes = [ctypes.c_int, f64p, f64p]
    lib.qaoa_fit_k0.restype = ctypes.c_double
    lib.qaoa_classify_regime.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double]
    lib.qaoa_set_opts.argtypes = [vp, P(Opts)]
    lib.qaoa_get_opts.argtypes = [vp, P(Opts)]
    lib.qaoa_set_cost_choice.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    _lib = lib
    return lib


ON, OFF = 1, 2
ORDERS = {"last": 1, "middle": 2}
SHAPES = {"5x3": 1, "4x4": 2, "5x2": 3, "4x3": 4, "5x4": 5}


class Opts(ctypes.Structure):
    """Kernel configuration of one context (``qaoa_opts``; 0 = library default)."""
    _fields_ = [("fwd_shape", ctypes.c_int), ("super_tile", ctypes.c_int), ("group_order", ctypes.c_int),
                ("float_lanes", ctypes.c_int), ("specialised", ctypes.c_int), ("tile_tables", ctypes.c_int),
                ("l2_prefetch", ctypes.c_int), ("grad_order", ctypes.c_int), ("grad_checkpoint", ctypes.c_int),
                ("adj_l2_prefetch", ctypes.c_int), ("tma_load", ctypes.c_int)]


def make_opts(shape=None, super_tile=None, order=None, float_lanes=None, specialised=None, tile_tables=None,
              l2_prefetch=None, grad_order=None, grad_checkpoint=None, adj_l2_prefetch=None,
              tma_load=None) -> Opts:
    """``Opts`` from readable values: shape "4x3" / "5x4" / ..., order "last" /
    "middle", booleans for the on/off fields; None keeps the default."""
    b = lambda x: 0 if x is None else (ON if x else OFF)  # noqa: E731
    return Opts(fwd_shape=SHAPES[shape] if shape else 0, super_tile=int(super_tile or 0),
                group_order=ORDERS[order] if order else 0, float_lanes=b(float_lanes), specialised=b(specialised),
                tile_tables=b(tile_tables), l2_prefetch=b(l2_prefetch),
                grad_order=ORDERS[grad_order] if grad_order else 0, grad_checkpoint=b(grad_checkpoint),
                adj_l2_prefetch=b(adj_l2_prefetch), tma_load=b(tma_load))


def set_cost_choice(n: int, precision, cost_mode) -> None:
    """Records the cost mode that QAOA_COST_AUTO selects for (n, precision)."""
    rc = load().qaoa_set_cost_choice(int(n), _PREC[precision], _COST[cost_mode])
    if rc != QAOA_OK:
        raise QaoaError(rc, "qaoa_set_cost_choice")


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def state_bytes(n: int, precision="c64") -> int:
    return int(load().qaoa_state_bytes(n, _PREC[precision]))


def aux_bytes(n: int, precision="c64", cost_mode="recompute", with_grad=False) -> int:
    return int(load().qaoa_aux_bytes(n, _PREC[precision], _COST[cost_mode], int(bool(with_grad))))


def describe_plan(n: int, p: int, precision="c64", adjoint=False) -> str:
    lib = load()
    need = lib.qaoa_describe_plan(n, _PREC[precision], p, int(adjoint), None, 0)
    buf = ctypes.create_string_buffer(need + 1)
    lib.qaoa_describe_plan(n, _PREC[precision], p, int(adjoint), buf, need + 1)
    return buf.value.decode()


def max_weight_sum(n: int, precision="c64") -> int:
    return int(load().qaoa_max_weight_sum(int(n), _PREC[precision]))


def quantize_weights(w, max_abs_sum: int):
    """Real weights as integers (``qaoa_quantize_weights``): returns (w_int, unit)."""
    wa, wp = _f64(w)
    out = np.empty(len(wa), dtype=np.int32)
    unit = ctypes.c_double()
    rc = load().qaoa_quantize_weights(len(wa), wp, int(max_abs_sum),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(unit))
    if rc:
        raise QaoaError(rc, "weights cannot be quantised (zero, non-finite or too small against their sum)")
    return out, unit.value


def lr_angles(p: int, dgamma: float, dbeta: float):
    """Linear-ramp angles gamma_k = (k+1)/p dgamma, beta_k = (1 - k/p) dbeta (Sec. II-B)."""
    k = np.arange(p, dtype=np.float64)
    return (k + 1) / p * dgamma, (1 - k / p) * dbeta


class Simulator:
    """One weighted MaxCut instance on one GPU (``qaoa_init_graph``).

    ``state`` / ``aux``: optional caller-owned torch CUDA tensors of exactly
    ``state_bytes(n, precision)`` / at least ``aux_bytes(...)`` bytes; by
    default they are allocated here with torch.
    """

    def __init__(self, n, u, v, w, scale=0.1, precision="c64", cost_mode="recompute", with_grad=False,
                 state=None, aux=None, stream=None, opts=None):
        import torch
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("libqaoa needs a CUDA device")
        self.n = int(n)
        self.precision = _PREC[precision]
        self.cost_mode = _COST[cost_mode]
        self.with_grad = bool(with_grad)
        self.unit = 1.0  # real weight per integer weight unit (from_real_weights)
        u = np.ascontiguousarray(u, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int32)
        self.m = len(u)
        sb = state_bytes(self.n, self.precision)
        if sb == 0:
            raise QaoaError(QAOA_EINVAL, "n out of range")
        cdt = torch.complex128 if self.precision == C128 else torch.complex64
        if state is None:
            state = torch.empty(1 << self.n, dtype=cdt, device="cuda")
        ab = aux_bytes(self.n, self.precision, self.cost_mode, self.with_grad)
        if aux is None and ab > 0:
            aux = torch.empty(ab, dtype=torch.uint8, device="cuda")
        self._state_t = state
        self._aux_t = aux
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p()
        rc = lib.qaoa_init_graph(ctypes.byref(ctx), self.n, self.m,
                                 u.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 float(scale), self.precision, self.cost_mode,
                                 ctypes.c_void_p(state.data_ptr()), state.numel() * state.element_size(),
                                 ctypes.c_void_p(aux.data_ptr() if aux is not None else None),
                                 (aux.numel() * aux.element_size()) if aux is not None else 0,
                                 ctypes.c_void_p(self.stream.cuda_stream))
        if rc != QAOA_OK:
            raise QaoaError(rc, lib.qaoa_last_error(None).decode())
        self._ctx = ctx
        self._lib = lib
        if opts is not None:
            self.set_opts(opts)

    # -- helpers
    @classmethod
    def from_real_weights(cls, n, u, v, w_real, scale=1.0, precision="c64", **kw):
        """An instance with real weights (Sec. II-G, U[0, 1] in the paper): the
        weights are quantised with the largest integer sum the path accepts,
        the phase scale absorbs the unit, and ``unit`` converts cut values and
        <C> back (real = integer x unit). Each weight is off by at most unit / 2."""
        w_int, unit = quantize_weights(w_real, max_weight_sum(n, precision))
        sim = cls(n, u, v, w_int, scale * unit, precision, **kw)
        sim.unit = unit
        return sim

    def _check(self, rc):
        if rc != QAOA_OK:
            raise QaoaError(rc, self._lib.qaoa_last_error(self._ctx).decode())

    @property
    def handle(self):
        """The qaoa_ctx pointer, for direct calls into the C ABI."""
        return self._ctx

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.qaoa_free(self._ctx)
            self._ctx = None
        # the device buffers this object allocated (or was given) are released
        # with it, not kept alive by a closed simulator
        self._state_t = None
        self._aux_t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- API
    def set_opts(self, opts):
        """Kernel configuration (``Opts``, or a dict of ``make_opts`` arguments)."""
        o = opts if isinstance(opts, Opts) else make_opts(**opts)
        self._check(self._lib.qaoa_set_opts(self._ctx, ctypes.byref(o)))

    def get_opts(self) -> dict:
        """The configuration in effect, every field resolved."""
        o = Opts()
        self._check(self._lib.qaoa_get_opts(self._ctx, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in Opts._fields_}

    def run(self, p: int, dgamma: float, dbeta: float):
        self._check(self._lib.qaoa_run(self._ctx, int(p), float(dgamma), float(dbeta)))

    def run_angles(self, gamma, beta):
        g, gp = _f64(gamma)
        b, bp = _f64(beta)
        if len(g) != len(b):
            raise ValueError("gamma and beta need the same length")
        self._check(self._lib.qaoa_run_angles(self._ctx, len(g), gp, bp))

    def expect(self) -> dict:
        e, r, nrm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        cmin, cmax = ctypes.c_int64(), ctypes.c_int64()
        amin, amax = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._lib.qaoa_expect(self._ctx, ctypes.byref(e), ctypes.byref(r), ctypes.byref(nrm),
                                          ctypes.byref(cmin), ctypes.byref(cmax), ctypes.byref(amin),
                                          ctypes.byref(amax)))
        return dict(exp_c=e.value, r=r.value, norm=nrm.value, c_min=cmin.value, c_max=cmax.value,
                    argmin=amin.value, argmax=amax.value)

    def extremes(self) -> dict:
        cmin, cmax = ctypes.c_int64(), ctypes.c_int64()
        amin, amax = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._lib.qaoa_expect(self._ctx, None, None, None, ctypes.byref(cmin), ctypes.byref(cmax),
                                          ctypes.byref(amin), ctypes.byref(amax)))
        return dict(c_min=cmin.value, c_max=cmax.value, argmin=amin.value, argmax=amax.value)

    def sample(self, shots: int, uniforms=None, seed: int = 0) -> np.ndarray:
        out = np.empty(int(shots), dtype=np.uint64)
        up = None
        if uniforms is not None:
            uarr, up = _f64(uniforms)
            if len(uarr) != shots:
                raise ValueError("uniforms must have `shots` entries")
        self._check(self._lib.qaoa_sample(self._ctx, int(shots), up, ctypes.c_uint64(seed),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out

    def grad(self, p: int, dgamma: float, dbeta: float) -> dict:
        gg = np.zeros(p)
        gb = np.zeros(p)
        ddg, ddb, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.qaoa_grad(self._ctx, int(p), float(dgamma), float(dbeta),
                                        gg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        gb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.byref(ddg), ctypes.byref(ddb), ctypes.byref(e)))
        return dict(g_gamma=gg, g_beta=gb, d_dgamma=ddg.value, d_dbeta=ddb.value, exp_c=e.value)

    def grad_angles(self, gamma, beta) -> dict:
        g, gp = _f64(gamma)
        b, bp = _f64(beta)
        gg = np.zeros(len(g))
        gb = np.zeros(len(g))
        e = ctypes.c_double()
        self._check(self._lib.qaoa_grad_angles(self._ctx, len(g), gp, bp,
                                               gg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               gb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               ctypes.byref(e)))
        return dict(g_gamma=gg, g_beta=gb, exp_c=e.value)

    def profile(self, enable: bool = True):
        """Starts (clearing the counters) or stops per-kernel event timing."""
        self._check(self._lib.qaoa_profile_enable(self._ctx, int(bool(enable))))

    def profile_read(self, kind="pass") -> dict:
        """Launch count, summed device ms and algorithmic bytes of one kernel kind."""
        k = PROFILE_KINDS.get(kind, kind)
        n, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.qaoa_profile_read(self._ctx, int(k), ctypes.byref(n), ctypes.byref(ms),
                                                ctypes.byref(by)))
        return dict(launches=n.value, ms=ms.value, bytes=by.value)

    def cost_diag(self):
        import torch
        out = torch.empty(1 << self.n, dtype=torch.int32, device="cuda")
        self._check(self._lib.qaoa_cost_diag(self._ctx, ctypes.c_void_p(out.data_ptr())))
        self.stream.synchronize()
        return out

    def state(self):
        """The state vector (torch complex tensor on the GPU, shares memory)."""
        self.stream.synchronize()
        return self._state_t

    def sample_cuts(self, xs=None, count: int = 0, seed: int = 0) -> dict:
        """C(x) and r(x) of bitstrings (Sec. II-D): `xs` (uint64, host or device),
        or `count` draws of the random sampler from stream `seed`. Returns torch
        device tensors x (int64 view of the uint64 indices), c (int32), r (float64)."""
        import torch
        xp = None
        if xs is not None:
            xt = torch.as_tensor(np.asarray(xs, dtype=np.uint64).view(np.int64)) if not torch.is_tensor(xs) else xs
            xt = xt.to(device="cuda", dtype=torch.int64).contiguous()
            count = xt.numel()
            xp = ctypes.c_void_p(xt.data_ptr())
        count = int(count)
        x = torch.empty(count, dtype=torch.int64, device="cuda")
        c = torch.empty(count, dtype=torch.int32, device="cuda")
        r = torch.empty(count, dtype=torch.float64, device="cuda")
        self._check(self._lib.qaoa_sample_cuts(self._ctx, count, xp, ctypes.c_uint64(seed),
                                               ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                               ctypes.c_void_p(r.data_ptr())))
        return dict(x=x, c=c, r=r)

    def noisy_expect(self, gamma, beta, eps: float, trajectories: int, seed: int = 0) -> dict:
        """Noisy LR-QAOA (Sec. II-C) by `trajectories` Monte Carlo trajectories with
        explicit angles: the mean <C>, r, and each trajectory's <C> (CUDA tensor)."""
        import torch
        g, gp = _f64(gamma)
        b, bp = _f64(beta)
        if len(g) != len(b):
            raise ValueError("gamma and beta must have the same length")
        per = torch.empty(int(trajectories), dtype=torch.float64, device="cuda")
        mean, r = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.qaoa_noisy_expect(self._ctx, len(g), gp, bp, float(eps), int(trajectories),
                                                ctypes.c_uint64(seed), ctypes.c_void_p(per.data_ptr()),
                                                ctypes.byref(mean), ctypes.byref(r)))
        return dict(exp_c=mean.value, r=r.value, per_trajectory=per)


def overlap_ratio(r_noisy: float, r_ideal: float, r_random: float) -> float:
    """r_ovl = (r_noisy - r_random) / (r_ideal - r_random) (Sec. II-C)."""
    return float(load().qaoa_overlap_ratio(float(r_noisy), float(r_ideal), float(r_random)))


def fit_k0(eps_acc, r_ovl) -> float:
    """k0 of Eq. noise (r_ovl = 2^(-k0 eps_acc)), least squares through the origin on log2 r_ovl."""
    a, ap = _f64(eps_acc)
    r, rp = _f64(r_ovl)
    if len(a) != len(r):
        raise ValueError("eps_acc and r_ovl must have the same length")
    return float(load().qaoa_fit_k0(len(a), ap, rp))


def mean_of_means(r, ns: int, reps: int = 100, seed: int = 0, stream=None) -> dict:
    """Mean of subsample means of a pool of ratios (Sec. II-D): `r` a float64
    CUDA tensor; returns the reps subsample means (CUDA tensor) and the grand
    mean, sigma and random threshold (host floats)."""
    import torch
    lib = load()
    if not (torch.is_tensor(r) and r.is_cuda and r.dtype == torch.float64):
        raise TypeError("r must be a float64 CUDA tensor")
    r = r.contiguous()
    st = stream if stream is not None else torch.cuda.current_stream()
    means = torch.empty(int(reps), dtype=torch.float64, device=r.device)
    stats = torch.empty(3, dtype=torch.float64, device=r.device)
    rc = lib.qaoa_mean_of_means(ctypes.c_void_p(r.data_ptr()), r.numel(), int(ns), int(reps), ctypes.c_uint64(seed),
                                ctypes.c_void_p(means.data_ptr()), ctypes.c_void_p(stats.data_ptr()),
                                ctypes.c_void_p(st.cuda_stream))
    if rc:
        raise QaoaError(rc, "qaoa_mean_of_means rejected its arguments or failed")
    h = stats.cpu().numpy()
    return dict(means=means, grand_mean=float(h[0]), sigma=float(h[1]), threshold=float(h[2]))


REGIMES = {0: "random", 1: "transition", 2: "noise-tolerant", 3: "above random"}


def classify_regime(r_obs: float, rand_mean: float, rand_sigma: float, ideal_mean=None, ideal_sigma=None) -> int:
    """Performance regime of an observed mean ratio (Sec. II-D); see REGIMES."""
    have = ideal_mean is not None
    return int(load().qaoa_classify_regime(float(r_obs), float(rand_mean), float(rand_sigma), int(have),
                                           float(ideal_mean) if have else 0.0,
                                           float(ideal_sigma) if have else 0.0))


class BatchOpts(ctypes.Structure):
    """Scheduling knobs of ``qaoa_batch_create`` (0 = library default)."""
    _fields_ = [("solo_max_n", ctypes.c_int), ("window_items", ctypes.c_int), ("window_mb", ctypes.c_int),
                ("max_units", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("wait_ns", ctypes.c_int64),
                ("cost_mode", ctypes.c_int), ("fwd_shape", ctypes.c_int)]


BATCH_FIELDS = ("exp_c", "r", "norm", "c_min", "c_max", "argmin", "argmax", "d_dgamma", "d_dbeta")


class Batch:
    """Many independent LR-QAOA instances (complex64) run by one persistent
    kernel per phase, replayed from a CUDA graph (``qaoa_batch_*``).

    ``instances``: dicts with keys n, p, dgamma, dbeta, u, v, w (the shape
    ``inputs.batch_instances`` returns). ``opts``: dict of ``BatchOpts`` fields
    (``cost_mode`` may be "recompute" / "stream", ``fwd_shape`` "5x3" / "4x3").
    """

    def __init__(self, instances, scale=0.1, with_grad=False, opts=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise QaoaError(QAOA_ECUDA, "no CUDA device")
        self._lib = load()
        self.count = len(instances)
        self.with_grad = bool(with_grad)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.n = np.array([d["n"] for d in instances], dtype=np.int32)
        self.p = np.array([d["p"] for d in instances], dtype=np.int32)
        off = np.zeros(self.count + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(d["u"]) for d in instances])
        cat = lambda k: (np.ascontiguousarray(np.concatenate([np.asarray(d[k], dtype=np.int32) for d in instances]))
                         if off[-1] else np.zeros(1, dtype=np.int32))
        u, v, w = cat("u"), cat("v"), cat("w")
        dg = np.array([d["dgamma"] for d in instances], dtype=np.float64)
        db = np.array([d["dbeta"] for d in instances], dtype=np.float64)
        o = dict(opts or {})
        if isinstance(o.get("cost_mode"), str):
            o["cost_mode"] = _COST[o["cost_mode"]]
        if isinstance(o.get("fwd_shape"), str):
            o["fwd_shape"] = SHAPES[o["fwd_shape"]]
        o = BatchOpts(**o)
        P = ctypes.POINTER
        ip = lambda a: a.ctypes.data_as(P(ctypes.c_int32))
        h = ctypes.c_void_p()
        rc = self._lib.qaoa_batch_create(ctypes.byref(h), self.count, ip(self.n), ip(self.p),
                                         off.ctypes.data_as(P(ctypes.c_int64)), ip(u), ip(v), ip(w),
                                         dg.ctypes.data_as(P(ctypes.c_double)), db.ctypes.data_as(P(ctypes.c_double)),
                                         float(scale), int(self.with_grad), ctypes.byref(o),
                                         ctypes.c_void_p(self.stream.cuda_stream))
        if rc != QAOA_OK:
            raise QaoaError(rc, self._lib.qaoa_batch_last_error(None).decode())
        self._h = h
        self._gsz = int(2 * self.p.sum())

    def _check(self, rc):
        if rc != QAOA_OK:
            raise QaoaError(rc, self._lib.qaoa_batch_last_error(self._h).decode())

    def run(self):
        self._check(self._lib.qaoa_batch_run(self._h))

    def results(self) -> dict:
        out = np.zeros(9 * self.count)
        g = np.zeros(max(1, self._gsz))
        self._check(self._lib.qaoa_batch_results(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        out = out.reshape(self.count, 9)
        res = {k: out[:, i].copy() for i, k in enumerate(BATCH_FIELDS)}
        splits = np.cumsum(2 * self.p)[:-1]
        res["grads"] = [(a[:len(a) // 2], a[len(a) // 2:]) for a in np.split(g[:self._gsz], splits)]
        return res

    def state(self, i: int):
        """Copy of instance i's final state as a torch complex64 tensor (forward batches)."""
        import torch
        ptr = ctypes.c_void_p()
        self._check(self._lib.qaoa_batch_state(self._h, int(i), ctypes.byref(ptr)))
        n = int(self.n[i])

        class _View:  # the library's buffer, seen through the CUDA array interface
            __cuda_array_interface__ = {"shape": (1 << n,), "typestr": "<c8", "data": (ptr.value, False),
                                        "version": 2, "strides": None}

        self.stream.synchronize()
        return torch.as_tensor(_View(), device="cuda").clone()

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(512)
        self._lib.qaoa_batch_describe(self._h, buf, 512)
        return buf.value.decode()

    def bytes(self) -> float:
        return float(self._lib.qaoa_batch_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.qaoa_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
