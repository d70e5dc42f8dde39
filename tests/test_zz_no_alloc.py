"""qaoa_sample_state_noalloc: shots without any device allocation.

Some callers cannot call cudaMalloc while they run (a plugin inside a host
framework that owns all device memory, a serving loop with a fixed memory
budget). This entry point keeps its scratch in a fixed device array. Its shots
must match those of qaoa_sample on the same state, under the tolerance the
other sampling tests use (identical indices except where u * total lies within
1e-9 of a CDF step), on two calls in a row. From 29 qubits the entry point
takes blocks larger than qaoa_sample's 2^12 amplitudes (the scratch holds at
most QAOA_NOALLOC_MAX_BLOCKS block sums); the 30-qubit case runs that branch.
"""
import ctypes

import numpy as np
import pytest

from paper_2604_26423_b300 import inputs, qaoa

pytestmark = pytest.mark.gpu


def _boundary(psi, uni, tol=1e-9):
    pr = np.abs(psi) ** 2
    F = np.cumsum(pr)
    t = uni * F[-1]
    idx = np.searchsorted(F, t, side="right")
    near = np.zeros(len(uni), dtype=bool)
    for k, (i, tt) in enumerate(zip(idx, t)):
        for j in (i - 1, i):
            if 0 <= j < len(F) and abs(F[j] - tt) <= tol * F[-1]:
                near[k] = True
    return near


def _noalloc(lib, state_ptr, n, prec, uni_dev, seed, out_dev, stream):
    fn = lib.qaoa_sample_state_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    return fn(ctypes.c_void_p(state_ptr), n, prec, out_dev.numel(),
              ctypes.c_void_p(uni_dev.data_ptr() if uni_dev is not None else None), ctypes.c_uint64(seed),
              ctypes.c_void_p(out_dev.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def _boundary_dev(state, uni, tol=1e-9):
    """_boundary on the device (FP64 CDF of the state with torch), for states
    too large for a host copy."""
    import torch
    pr = state.real.double() ** 2 + state.imag.double() ** 2
    F = torch.cumsum(pr, 0)
    del pr
    total = F[-1]
    t = torch.from_numpy(uni).to(F.device) * total
    idx = torch.searchsorted(F, t, right=True)
    near = torch.zeros(len(uni), dtype=torch.bool, device=F.device)
    for j in (idx - 1, idx):
        ok = (j >= 0) & (j < len(F))
        fj = F[j.clamp(0, len(F) - 1)]
        near |= ok & ((fj - t).abs() <= tol * total)
    return near.cpu().numpy()


@pytest.mark.parametrize("n,prec", [(14, "c128"), (18, "c64"), (30, "c64")])
def test_noalloc_matches_qaoa_sample_two_calls(n, prec):
    import torch
    from paper_2604_26423_b300.qaoa import Simulator
    lib = qaoa.load()
    u, v, w = inputs.complete_graph(n, 1200 + n)
    shots = 2048
    with Simulator(n, u, v, w, 0.1, prec) as s:
        s.run(3, 0.6, 0.3)
        if n <= 20:
            psi = s.state().cpu().numpy().astype(np.complex128)
            boundary = lambda uni: _boundary(psi, uni)  # noqa: E731
        else:
            boundary = lambda uni: _boundary_dev(s.state(), uni)  # noqa: E731
        state_ptr = lib.qaoa_state_ptr(s.handle)
        stream = s.stream
        for call, seed in enumerate((1300 + n, 1400 + n)):
            uni = inputs.uniforms(seed, shots)
            ref = s.sample(shots, uniforms=uni)
            uni_dev = torch.from_numpy(uni).cuda()
            out_dev = torch.zeros(shots, dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            rc = _noalloc(lib, state_ptr, n, qaoa._PREC[prec], uni_dev, 0, out_dev, stream)
            assert rc == qaoa.QAOA_OK, call
            stream.synchronize()
            got = out_dev.cpu().numpy().astype(np.uint64)
            ok = (got == ref) | boundary(uni)
            assert ok.all(), f"call {call}: {(~ok).sum()} shots differ"
            # the seeded path draws the same uniforms on the device
            out2 = torch.zeros(shots, dtype=torch.int64, device="cuda")
            assert _noalloc(lib, state_ptr, n, qaoa._PREC[prec], None, seed, out2, stream) == qaoa.QAOA_OK
            stream.synchronize()
            assert np.array_equal(out2.cpu().numpy().astype(np.uint64), got)


def test_noalloc_rejects_sizes_beyond_limit():
    import torch
    lib = qaoa.load()
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    dummy = torch.zeros(2, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    fn = lib.qaoa_sample_state_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    big = 35  # above QAOA_NOALLOC_MAX_QUBITS
    assert fn(ctypes.c_void_p(dummy.data_ptr()), big, 0, 4, None, 1, ctypes.c_void_p(out.data_ptr()),
              ctypes.c_void_p(stream.cuda_stream)) == qaoa.QAOA_EINVAL
    assert fn(ctypes.c_void_p(dummy.data_ptr()), 1, 0, -1, None, 1, ctypes.c_void_p(out.data_ptr()),
              ctypes.c_void_p(stream.cuda_stream)) == qaoa.QAOA_EINVAL
