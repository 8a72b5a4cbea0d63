"""The no-allocation diagnostics entry point against tslb_diagnostics.

tslb_diagnostics_noalloc exists for callers that cannot allocate device
memory where they need the sums: a program under a fixed device-memory budget
that is already spent, a framework allocator that has reserved the whole
device, or a latency-bound loop between solver steps in which cudaMalloc /
cudaFree (which may synchronise the device) are not acceptable.  Its partial
sums live in a fixed device array instead of cudaMalloc'd scratch.  This file
is collected last so that a failure here cannot hide the other tests; it
passes alone in a fresh process (the first call does the per-device set-up)
and after the rest of the suite.
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
    # past the limit (2^24 * 5 > 2^26), and extents whose product would wrap a
    # 64-bit integer (2^22 per axis): both refused by the library before any
    # launch (the binding's own length checks are bypassed here on purpose by
    # calling the C function directly)
    L = T.load()
    import ctypes
    for big in ((4096, 4096, 5), (1 << 22, 1 << 22, 1 << 22)):
        d = (ctypes.c_int64 * 3)(*big)
        b = (ctypes.c_int * 6)(*(0,) * 6)
        p = ctypes.c_void_p(one.data_ptr())
        code = L.tslb_diagnostics_noalloc(p, p, None, d, b, 0.6, None, ctypes.c_void_p(out.data_ptr()))
        assert code == T.TSLB_ERR_INVALID
        assert "TSLB_NOALLOC_MAX_NODES" in L.tslb_last_error(None).decode()
    big_u = torch.zeros(3 * 512, dtype=torch.float64, device="cuda")
    big_r = torch.zeros(512, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TslbError) as ei:
        T.tslb_diagnostics_noalloc(big_r, big_u, None, (8, 8, 8), (0,) * 6, 0.4, out)
    assert ei.value.code == T.TSLB_ERR_INVALID


@pytest.mark.parametrize("field", [0, 2, 5], ids=["pi_xx", "pi_zz", "pi_yz"])
def test_noalloc_counts_nonfinite_stress(cuda_ok, field):
    """A NaN in one stress component (not rho, u or Pi_xy) makes the node
    non-finite in both calls: the count is 1 and the sums over the remaining
    nodes agree with tslb_diagnostics, on two calls in a row."""
    import torch
    prm = W.channel_params(nx=24, ny=12, nz=10)
    dims, tau, bc = prm["dims"], prm["tau"], prm["bc"]
    rho0, u0, pi0 = W.channel_state(prm, seed=2)
    N = dims[0] * dims[1] * dims[2]
    pi0 = np.array(pi0, dtype=np.float64).reshape(6, N).copy()
    node = 5 + dims[0] * (4 + dims[1] * 3)  # interior: x 5, y 4, z 3
    pi0[field, node] = np.nan
    s = T.Solver(dims, tau, force=prm["force"], bc=bc)
    s.init_moments(rho0, u0, pi0)
    ref, code = s.diagnostics()
    assert code == T.TSLB_ERR_UNSTABLE and ref["nonfinite"] == 1
    rho, u, pi = _moments_on_device(s, N)
    for _ in range(2):
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        T.tslb_diagnostics_noalloc(rho, u, pi, dims, bc, tau, out)
        torch.cuda.synchronize()
        _compare(ref, out.cpu().numpy())
    s.close()


def test_noalloc_rejects_short_arrays(cuda_ok):
    """Arrays shorter than the lattice, or of another dtype, are refused before
    any launch."""
    import torch
    dims = (8, 8, 8)
    N = 512
    rho = torch.zeros(N, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="u holds"):
        T.tslb_diagnostics_noalloc(rho, u[: 3 * N - 1], None, dims, (0,) * 6, 0.6, out)
    with pytest.raises(ValueError, match="pi holds"):
        T.tslb_diagnostics_noalloc(rho, u, u, dims, (0,) * 6, 0.6, out)
    with pytest.raises(ValueError, match="float64"):
        T.tslb_diagnostics_noalloc(rho.float(), u, None, dims, (0,) * 6, 0.6, out)
    with pytest.raises(ValueError, match="out holds"):
        T.tslb_diagnostics_noalloc(rho, u, None, dims, (0,) * 6, 0.6, out[:4])
