"""16-bit moment storage (BF16 / FP16 scaled deviations) against the FP64 oracle.

Storage keeps rho - 1, u / u_ref and Pi^neq / pi_ref in 16 bits with FP32
arithmetic.  Each stored value is rounded to nearest even once per step with
relative error eps = 2^-9 (BF16) or 2^-12 (FP16); the rounding noise is
damped by the viscous relaxation, so the field error stays a small multiple of
eps.  The bounds below are 4 eps for u and Pi (taken against the size of the
field) and are checked on the Taylor-Green vortex; the channel set-up compares
the plane-averaged profile u_x(y) that the turbulence statistics are built on.
Pi^neq is quantised against pi_ref = 2 max|Pi| and the Taylor-Green Pi field
has rms max/sqrt(2), so its quantisation step relative to the field is about
2 sqrt(2) times that of u (stored against u_ref = max|u|): its bound is 16 eps.
"""
import numpy as np
import pytest

import oracle
import paper_2401_17074_b300 as T
from paper_2401_17074_b300 import workloads as W

pytestmark = pytest.mark.gpu

EPS = {T.BF16: 2.0 ** -9, T.FP16: 2.0 ** -12}


def _stack(r, u, p):
    return np.concatenate([(r - 1.0)[None], u, p])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [T.BF16, T.FP16], ids=["bf16", "fp16"])
def test_taylor_green_16bit_storage(cuda_ok, prec):
    dims, state = W.taylor_green(n=32, u0=0.05, tau=0.6)
    o = oracle.OracleSim(dims, 0.6)
    o.init_moments(*state)
    o.step(200)
    ref = _stack(*o.get_moments())
    s = T.Solver(dims, 0.6, precision=prec, u_ref=0.05, pi_ref=W.pi_reference(state))
    s.init_moments(*state)
    s.step(200)
    got = _stack(*s.get_moments())
    s.close()
    eps = EPS[prec]
    for k in (1, 2):
        assert _rel(got[k], ref[k]) <= 4 * eps, (k, _rel(got[k], ref[k]))
    for k in (4, 5):
        assert _rel(got[k], ref[k]) <= 16 * eps, (k, _rel(got[k], ref[k]))


@pytest.mark.parametrize("prec", [T.FP32, T.BF16, T.FP16], ids=["fp32", "bf16", "fp16"])
def test_channel_mean_profile(cuda_ok, prec):
    """Plane-averaged u_x(y) of the forced channel after 300 steps (tau = 0.503)."""
    prm = W.channel_params(nx=48, ny=34, nz=32)
    state = W.channel_state(prm, seed=1)
    nsteps = 300
    o = oracle.OracleSim(prm["dims"], prm["tau"], force=prm["force"], bc=prm["bc"])
    o.init_moments(*state)
    o.step(nsteps)
    _, uo, _ = o.get_moments()
    s = T.Solver(prm["dims"], prm["tau"], force=prm["force"], bc=prm["bc"], precision=prec, u_ref=0.05,
                 pi_ref=W.pi_reference(state))
    s.init_moments(*state)
    s.step(nsteps)
    _, ug, _ = s.get_moments()
    s.close()
    nx, ny, nz = prm["dims"]
    prof = lambda u: u[0].reshape(nz, ny, nx)[:, 1:ny - 1, :].mean(axis=(0, 2))
    err = _rel(prof(ug), prof(uo))
    bound = 1e-5 if prec == T.FP32 else 4 * EPS[prec]
    assert err <= bound, err


def test_channel_statistics_against_oracle(cuda_ok):
    """Mean velocity and Reynolds-stress profiles of the forced channel,
    averaged over x, z and the samples at steps 10, 20 and 30 (FP32 storage),
    against the same statistics of the oracle run.

    Bounds: U(y) inherits the 1e-5 relative bound of u_x over these steps (the
    small forced-channel parity test).  A stress <u'_i u'_j> changes by about
    2 <u' du> for a field error du, so its relative error is at most about
    2 |du| / |u'|; with |du| <= 1e-5 |u| and fluctuations of 2 % of the
    centreline velocity (the initial noise) that is 1e-3.
    """
    from paper_2401_17074_b300.channel_stats import ChannelStats, profile_errors
    prm = W.channel_params(nx=20, ny=18, nz=12, u_tau=0.0035, tau=0.503)
    state = W.channel_state(prm, seed=1)
    dims = prm["dims"]
    o = oracle.OracleSim(dims, prm["tau"], force=prm["force"], bc=prm["bc"])
    o.init_moments(*state)
    s = T.Solver(dims, prm["tau"], force=prm["force"], bc=prm["bc"])
    s.init_moments(*state)
    so, sg = ChannelStats(dims), ChannelStats(dims)
    for _ in range(3):
        o.step(10)
        s.step(10)
        so.add(o.get_moments()[1])
        sg.add(s.get_moments()[1])
    s.close()
    ref, got = so.result(), sg.result()
    assert min(np.abs(ref["uu"]).max(), ref["vv"].max(), ref["ww"].max()) > 0.0
    errs = profile_errors(got, ref)
    assert errs["U"] <= 1e-5, errs
    for k in ("uu", "vv", "ww", "uv"):
        assert errs[k] <= 1e-3, errs
