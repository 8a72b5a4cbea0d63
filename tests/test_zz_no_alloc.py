"""The no-allocation diagnostics entry point against tslb_diagnostics.

tslb_diagnostics_noalloc exists for callers that may not allocate device
memory where they need the sums (inside a stream capture, in allocation-free
real-time loops, or when a framework allocator owns the device memory).  Its
partial sums live in a fixed device array instead of cudaMalloc'd scratch.
This file is collected last so that a failure here cannot hide the other
tests; it passes alone in a fresh process (the first call does the per-device
set-up) and after the rest of the suite.
"""
import numpy as np
import pytest

import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _moments_on_device(s, N):
    import torch
    rho = torch.zeros(N, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    pi = torch.zeros(6 * N, dtype=torch.float64, device="cuda")
    T.tslb_get_moments(s.handle, rho, u, pi, T.DEVICE)
    return rho, u, pi


def _compare(ref, got):
    rel = 1e-12
    assert abs(got[0] - ref["mass"]) <= rel * abs(ref["mass"])
    for a in range(3):
        assert abs(got[1 + a] - ref["momentum"][a]) <= rel * abs(ref["mass"]) * 1e-1
    assert abs(got[4] - ref["kinetic_energy"]) <= rel * abs(ref["kinetic_energy"]) + 1e-18
    assert abs(got[5] - ref["wall_shear"]) <= 1e-10 * abs(ref["wall_shear"]) + 1e-18
    assert got[6] == pytest.approx(ref["max_speed"], rel=1e-15, abs=0)
    assert int(got[7]) == ref["nonfinite"]


@pytest.mark.parametrize("case", ["channel", "periodic"])
def test_noalloc_matches_diagnostics_twice(cuda_ok, case):
    import torch
    if case == "channel":
        prm = W.channel_params(nx=40, ny=34, nz=24)
        state = W.channel_state(prm, seed=1)
        dims, tau, bc, force = prm["dims"], prm["tau"], prm["bc"], prm["force"]
    else:
        dims, tau, bc, force = (33, 17, 29), 0.7, (0,) * 6, (0.0, 0.0, 0.0)
        state = W.random_state(dims, seed=31)
    N = dims[0] * dims[1] * dims[2]
    s = T.Solver(dims, tau, force=force, bc=bc)
    s.init_moments(*state)
    s.step(7)
    ref, code = s.diagnostics()
    assert code == T.TSLB_OK
    rho, u, pi = _moments_on_device(s, N)
    stream = torch.cuda.current_stream()
    for _ in range(2):  # two calls in a row share the fixed partial-sum array
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        T.tslb_diagnostics_noalloc(rho, u, pi, dims, bc, tau, out, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        _compare(ref, out.cpu().numpy())
    s.close()


def test_noalloc_rejects_oversize_and_bad_args(cuda_ok):
    import torch
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = (4096, 4096, 5)  # 2^24 * 5 interior nodes > 2^26
    with pytest.raises(T.TslbError) as ei:
        T.tslb_diagnostics_noalloc(one, one, None, big, (0,) * 6, 0.6, out)
    assert ei.value.code == T.TSLB_ERR_INVALID and "TSLB_NOALLOC_MAX_NODES" in str(ei.value)
    with pytest.raises(T.TslbError) as ei:
        T.tslb_diagnostics_noalloc(one, one, None, (8, 8, 8), (0,) * 6, 0.4, out)
    assert ei.value.code == T.TSLB_ERR_INVALID
