"""The refined reciprocal used by the step's finish (u = J / (216 + D0)).

rcp_refined is the hardware approximate reciprocal followed by one
Newton-Raphson step.  Over a sweep of r = 216 + D0 (D0 from -200 to +1000,
every FP32 value in a dense band around 216 and random values elsewhere) the
result must be within one ulp of 1/r computed in FP64 and rounded, and
correctly rounded for at least 99 % of the inputs."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def probe():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "librcp_probe.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           "-Xcompiler", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2401_17074_b300", "csrc"),
                           os.path.join(HERE, "kernels", "rcp_probe.cu"), "-o", so])
    L = ctypes.CDLL(so)
    L.rcp_probe.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return L


def test_rcp_refined_within_one_ulp(cuda_ok, probe):
    import torch
    band = np.arange(np.float32(215.0).view(np.int32), np.float32(217.0).view(np.int32), dtype=np.int32)
    band = band.view(np.float32)
    rng = np.random.default_rng(5)
    wide = (16.0 + 1200.0 * rng.random(2_000_000)).astype(np.float32)
    r = np.concatenate([band, wide])
    rt = torch.from_numpy(r).cuda()
    out = torch.empty_like(rt)
    assert probe.rcp_probe(ctypes.c_void_p(rt.data_ptr()), ctypes.c_void_p(out.data_ptr()), r.size) == 0
    got = out.cpu().numpy()
    exact = (1.0 / r.astype(np.float64)).astype(np.float32)  # correctly rounded 1/r
    ulps = np.abs(got.view(np.int32).astype(np.int64) - exact.view(np.int32).astype(np.int64))
    print("inputs %d, max %d ulp, correctly rounded %.4f" % (r.size, ulps.max(), np.mean(ulps == 0)))
    assert ulps.max() <= 1
    assert np.mean(ulps == 0) >= 0.99
