"""FP32 host interface of the moments (tslb_init_moments_f32 / _get_moments_f32).

The density travels as its deviation drho = rho - 1, the stored quantity, so
no precision is lost in FP32: with FP32 storage a read-back is bit-identical
to what was loaded; loading the same values through the FP64 interface (rho =
1 + drho in FP64, exact) gives the same stored state, hence bit-identical runs;
and an FP32 read equals the FP64 read cast to FP32 (rho - 1 is exact in FP64).
"""
import numpy as np
import pytest

import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _state32(dims, seed):
    r, u, p = W.random_state(dims, seed=seed)
    return (r - 1.0).astype(np.float32), u.astype(np.float32), p.astype(np.float32)


def _interior(dims, bc):
    nx, ny, nz = dims
    m = np.ones((nz, ny, nx), bool)
    if bc[2] != 0:
        m[:, 0, :] = m[:, -1, :] = False
    return m.reshape(-1)


def test_fp32_round_trip_is_exact(cuda_ok):
    dims, bc = (21, 14, 9), (0, 0, 1, 1, 0, 0)
    d, u, p = _state32(dims, 51)
    s = T.Solver(dims, 0.6, bc=bc)
    s.init_moments_f32(d, u, p)
    d2, u2, p2 = s.get_moments_f32()
    s.close()
    m = _interior(dims, bc)
    assert np.array_equal(d2[m], d[m]) and np.array_equal(u2[:, m], u[:, m]) and np.array_equal(p2[:, m], p[:, m])
    assert np.all(d2[~m] == 0) and np.all(u2[:, ~m] == 0)  # boundary layers read as the rest state


@pytest.mark.parametrize("prec", [T.FP32, T.BF16], ids=["fp32", "bf16"])
def test_fp32_and_fp64_interfaces_agree(cuda_ok, prec):
    dims, bc = (21, 14, 9), (0, 0, 1, 1, 0, 0)
    d, u, p = _state32(dims, 52)
    kw = dict(force=(1e-5, 0.0, 0.0), bc=bc, precision=prec, pi_ref=2e-3)
    a = T.Solver(dims, 0.6, **kw)
    a.init_moments_f32(d, u, p)
    b = T.Solver(dims, 0.6, **kw)
    b.init_moments(1.0 + d.astype(np.float64), u.astype(np.float64), p.astype(np.float64))
    a.step(5)
    b.step(5)
    da, ua, pa = a.get_moments_f32()
    rb, ub, pb = b.get_moments()
    db, ub32, pb32 = b.get_moments_f32()
    a.close()
    b.close()
    assert np.array_equal(da, db) and np.array_equal(ua, ub32) and np.array_equal(pa, pb32)
    assert np.array_equal(da, (rb - 1.0).astype(np.float32))
    assert np.array_equal(ua, ub.astype(np.float32)) and np.array_equal(pa, pb.astype(np.float32))


def test_fp32_interface_with_device_tensors(cuda_ok):
    import torch
    dims = (12, 10, 8)
    d, u, p = _state32(dims, 53)
    s = T.Solver(dims, 0.7)
    s.init_moments_f32(torch.from_numpy(d).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(p).cuda())
    N = d.size
    dd = torch.empty(N, dtype=torch.float32, device="cuda")
    uu = torch.empty((3, N), dtype=torch.float32, device="cuda")
    pp = torch.empty((6, N), dtype=torch.float32, device="cuda")
    T.tslb_get_moments_f32(s.handle, dd, uu, pp, T.DEVICE)
    s.close()
    assert np.array_equal(dd.cpu().numpy(), d) and np.array_equal(uu.cpu().numpy(), u)
    assert np.array_equal(pp.cpu().numpy(), p)


def test_fp32_interface_d3q27_only(cuda_ok):
    prm = W.channel2d_params(nx=32, ny=10)
    s = T.Solver(prm["dims"], prm["tau"], force=prm["force"], bc=prm["bc"], lattice=T.TSLB_D2Q9)
    N = 32 * 10
    with pytest.raises(T.TslbError) as ei:
        s.init_moments_f32(np.zeros(N, np.float32), np.zeros((3, N), np.float32))
    assert ei.value.code == T.TSLB_ERR_UNSUPPORTED
    s.close()
