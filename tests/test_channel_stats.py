"""Channel statistics (mean and Reynolds-stress profiles) on fields with known
averages: x-harmonics average to a^2/2 over a whole period, and two time
samples offset by +-c give a variance of c^2."""
import math

import numpy as np
import torch

from paper_2401_17074_b300.channel_stats import ChannelStats, profile_errors


def _field(dims, shift):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = 0.01 * y * (ny - 1 - y)
    cx = np.cos(2 * math.pi * x / nx)
    u = np.stack([f + 0.003 * cx + shift, 0.002 * cx, 0.001 * np.sin(2 * math.pi * z / nz)])
    return u.reshape(3, -1), f[0, 1:ny - 1, 0]


def _check(res, f, c):
    assert np.allclose(res["U"], f, rtol=0, atol=1e-15)
    assert np.allclose(res["V"], 0.0, atol=1e-15) and np.allclose(res["W"], 0.0, atol=1e-15)
    assert np.allclose(res["uu"], 0.003 ** 2 / 2 + c * c, rtol=1e-12, atol=1e-18)
    assert np.allclose(res["vv"], 0.002 ** 2 / 2, rtol=1e-12, atol=1e-18)
    assert np.allclose(res["ww"], 0.001 ** 2 / 2, rtol=1e-12, atol=1e-18)
    assert np.allclose(res["uv"], 0.003 * 0.002 / 2, rtol=1e-12, atol=1e-18)


def test_stats_numpy_two_samples():
    dims = (12, 9, 8)
    st = ChannelStats(dims)
    for c in (+0.004, -0.004):
        u, f = _field(dims, c)
        st.add(u)
    _check(st.result(), f, 0.004)


def test_stats_torch_matches_numpy():
    dims = (10, 7, 6)
    a, b = ChannelStats(dims), ChannelStats(dims)
    for c in (0.001, -0.001):
        u, f = _field(dims, c)
        a.add(u)
        b.add(torch.from_numpy(u))
    ra, rb = a.result(), b.result()
    _check(rb, f, 0.001)
    for k in ra:
        assert np.allclose(ra[k], rb[k], rtol=1e-13, atol=1e-17)  # zero-mean profiles: summation order
    assert max(profile_errors(rb, ra).values()) < 1e-12
