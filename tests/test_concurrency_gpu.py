"""Several solvers at once: handles used from different host threads, each on
its own stream (the library keeps no shared mutable state besides the one-time
kernel attribute set-up), give bit for bit the results of the same runs made
one after the other; and a handle closed by its context manager is released."""
import threading

import numpy as np
import pytest

import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ((40, 34, 20), (0, 0, 1, 1, 0, 0), T.FP32, T.KERNEL_FACTORED),
    ((33, 18, 12), (0, 0, 5, 5, 0, 0), T.BF16, T.KERNEL_FACTORED),
    ((20, 20, 20), (0,) * 6, T.FP16, T.KERNEL_AUTO),
    ((16, 12, 10), (2, 2, 2, 2, 0, 0), T.FP32, T.KERNEL_DIRECT),
]


def _run(case, seed, out, key):
    dims, bc, prec, kernel = case
    state = W.random_state(dims, seed=seed)
    with T.Solver(dims, 0.6, force=(1e-5, 0.0, 0.0), bc=bc, precision=prec, kernel=kernel, pi_ref=2e-3) as s:
        s.init_moments(*state)
        s.step(25)
        out[key] = np.concatenate([a.reshape(-1) for a in s.get_moments()])


def test_threads_match_sequential_runs(cuda_ok):
    seq = {}
    for i, case in enumerate(CASES):
        _run(case, 60 + i, seq, i)
    par = {}
    threads = [threading.Thread(target=_run, args=(case, 60 + i, par, i)) for i, case in enumerate(CASES)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert sorted(par) == sorted(seq)
    for i in seq:
        assert np.array_equal(par[i], seq[i]), i


def test_context_manager_releases_the_handle(cuda_ok):
    with T.Solver((8, 8, 8), 0.6) as s:
        s.init_moments(*W.rest_state((8, 8, 8)))
        s.step(2)
    assert s.handle is None


def test_device_inputs_are_ordered_after_the_torch_stream(cuda_ok):
    """CUDA tensors handed to a solver on its own stream are read only after
    the work queued on PyTorch's current stream has run: the inputs below are
    NaN until a fill that waits behind a 25 ms spin on that stream, so an
    unordered read would find NaNs (and the force field would not be the
    one filled)."""
    import torch
    dims = (64, 32, 16)
    N = dims[0] * dims[1] * dims[2]
    st = torch.cuda.Stream()
    with T.Solver(dims, 0.6, stream=st.cuda_stream) as s:
        drho = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
        u = torch.full((3, N), float("nan"), dtype=torch.float32, device="cuda")
        F = torch.full((3 * N,), float("nan"), dtype=torch.float32, device="cuda")
        # one ordered call first, so the library's first-call set-up cannot
        # stand in for the wait below
        s.init_moments_f32(torch.zeros_like(drho), torch.zeros_like(u))
        torch.cuda.synchronize()
        torch.cuda._sleep(50_000_000)  # a bounded spin of 5e7 clock cycles on the current stream
        drho.fill_(0.0)
        u.fill_(0.01)
        F.fill_(0.0)
        s.init_moments_f32(drho, u)
        torch.cuda._sleep(50_000_000)
        F.fill_(1e-6)
        s.set_force_field(F)
        s.step(3)
        d, code = s.diagnostics()
        assert code == T.TSLB_OK and d["nonfinite"] == 0
        _, uu, _ = s.get_moments()
        assert np.allclose(uu[0], 0.01 + 3e-6, rtol=0, atol=1e-8)
