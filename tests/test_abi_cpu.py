"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol declared in include/tslb.h, and argument validation rejects bad
requests before any CUDA call (so these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2401_17074_b300 as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "tslb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(tslb_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = _declared_functions()
    assert set(names) == set(T.EXPORTED), names


def test_library_exports_every_declared_symbol():
    path = T._build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared_functions():
        assert name in exported, name
    L = T.load()
    for name in _declared_functions():
        assert hasattr(L, name)


def test_library_targets_sm_103a():
    path = T._build.build()
    out = subprocess.run(["cuobjdump", "--list-elf", path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_options_default():
    o = T.tslb_options_default()
    assert o.precision == T.FP32 and abs(o.u_ref - 0.05) < 1e-15 and o.kernel == T.KERNEL_AUTO


def _create_code(dims=(8, 8, 8), tau=0.6, bc=(0,) * 6, lattice=T.TSLB_D3Q27, opt=None):
    L = T.load()
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 3)(*dims)
    b = (ctypes.c_int * 6)(*bc)
    code = L.tslb_create(ctypes.byref(h), lattice, d, tau, None, b, ctypes.byref(opt) if opt else None)
    return code, h


@pytest.mark.parametrize("kw,code", [
    (dict(tau=0.5), T.TSLB_ERR_INVALID),
    (dict(tau=0.3), T.TSLB_ERR_INVALID),
    (dict(tau=float("nan")), T.TSLB_ERR_INVALID),
    (dict(lattice=19), T.TSLB_ERR_UNSUPPORTED),
    (dict(dims=(2, 8, 8)), T.TSLB_ERR_INVALID),
    (dict(dims=(8, 3, 8), bc=(0, 0, 1, 1, 0, 0)), T.TSLB_ERR_INVALID),
    (dict(bc=(0, 0, 1, 0, 0, 0)), T.TSLB_ERR_INVALID),
    (dict(bc=(1, 1, 0, 0, 0, 0)), T.TSLB_ERR_UNSUPPORTED),
    (dict(bc=(0, 0, 0, 0, 4, 3)), T.TSLB_ERR_UNSUPPORTED),
    (dict(bc=(0, 0, 1, 1, 3, 4)), T.TSLB_ERR_UNSUPPORTED),
    (dict(bc=(0, 0, 9, 9, 0, 0)), T.TSLB_ERR_INVALID),
    (dict(bc=(5, 5, 0, 0, 0, 0)), T.TSLB_ERR_UNSUPPORTED),
    (dict(bc=(2, 2, 5, 5, 0, 0)), T.TSLB_ERR_UNSUPPORTED),
    (dict(bc=(0, 0, 5, 5, 3, 4)), T.TSLB_ERR_UNSUPPORTED),
    (dict(bc=(0, 0, 0, 0, 5, 5)), T.TSLB_ERR_UNSUPPORTED),
])
def test_create_rejects_bad_arguments(kw, code):
    c, h = _create_code(**kw)
    assert c == code
    assert not h.value  # *out untouched
    assert len(T.tslb_last_error(None)) > 0


def test_bad_option_values_rejected():
    o = T.tslb_options_default()
    o.precision = 7
    c, h = _create_code(opt=o)
    assert c == T.TSLB_ERR_INVALID
    o = T.tslb_options_default()
    o.precision = T.BF16
    o.u_ref = 0.0
    c, h = _create_code(opt=o)
    assert c == T.TSLB_ERR_INVALID


def test_rounding_rules():
    o = T.tslb_options_default()
    assert o.rounding == T.TSLB_ROUND_NEAREST and o.rounding_seed == 0
    o.rounding = 5
    assert _create_code(opt=o)[0] == T.TSLB_ERR_INVALID
    o = T.tslb_options_default()
    o.rounding = T.TSLB_ROUND_STOCHASTIC  # FP32 storage has nothing to round
    assert _create_code(opt=o)[0] == T.TSLB_ERR_INVALID


def test_bad_sponge_and_noise_rejected():
    for width, k in ((-1, 10.0), (8, 10.0), (3, -1.0), (3, float("nan"))):  # dims z = 8
        o = T.tslb_options_default()
        o.sponge_width = width
        o.sponge_k = k
        c, h = _create_code(opt=o)
        assert c == T.TSLB_ERR_INVALID, (width, k)
        assert not h.value
    o = T.tslb_options_default()
    o.inflow.noise_kind = 5
    c, h = _create_code(opt=o)
    assert c == T.TSLB_ERR_INVALID


def test_d2q9_create_rules():
    # nz must be 1 with periodic z faces; x periodic; y periodic or bounce-back
    for dims, bc, code in (((8, 8, 2), (0,) * 6, T.TSLB_ERR_INVALID),
                           ((8, 8, 1), (0, 0, 0, 0, 3, 4), T.TSLB_ERR_INVALID),
                           ((8, 8, 1), (2, 2, 0, 0, 0, 0), T.TSLB_ERR_UNSUPPORTED),
                           ((8, 8, 1), (0, 0, 2, 2, 0, 0), T.TSLB_ERR_UNSUPPORTED)):
        c, h = _create_code(dims=dims, bc=bc, lattice=T.TSLB_D2Q9)
        assert c == code, (dims, bc, c)
        assert not h.value
    o = T.tslb_options_default()
    o.precision = T.BF16
    c, h = _create_code(dims=(8, 8, 1), lattice=T.TSLB_D2Q9, opt=o)
    assert c == T.TSLB_ERR_UNSUPPORTED


def test_guo_forcing_rules():
    for kw in (dict(bc=(2, 2, 0, 0, 0, 0)), dict(bc=(0, 0, 5, 5, 0, 0)), dict(bc=(0, 0, 0, 0, 3, 4), dims=(8, 8, 8)),
               dict(dims=(8, 8, 1), lattice=T.TSLB_D2Q9)):
        o = T.tslb_options_default()
        o.forcing = T.TSLB_FORCING_GUO
        c, h = _create_code(opt=o, **kw)
        assert c == T.TSLB_ERR_UNSUPPORTED, kw
    o = T.tslb_options_default()
    o.forcing = T.TSLB_FORCING_GUO
    o.sponge_width = 3
    o.sponge_k = 1.0
    assert _create_code(opt=o)[0] == T.TSLB_ERR_UNSUPPORTED
    o = T.tslb_options_default()
    o.forcing = 7
    assert _create_code(opt=o)[0] == T.TSLB_ERR_INVALID


def test_null_handle_calls_fail_cleanly():
    L = T.load()
    assert L.tslb_step(None, 1) == T.TSLB_ERR_INVALID
    assert L.tslb_synchronize(None) == T.TSLB_ERR_INVALID
    assert L.tslb_interior_nodes(None) == 0
    L.tslb_destroy(None)
    assert L.tslb_adjoint(None, None, 4, 0, None, T.HOST) == T.TSLB_ERR_INVALID
    assert L.tslb_adjoint_force_gradient(None, 4, None, T.HOST) == T.TSLB_ERR_INVALID


def test_noalloc_wrapper_rejects_bad_arrays_before_launch():
    """The binding checks the device, dtype, layout and length of every array
    the no-allocation kernels read or write before it calls the library, so a
    short, CPU or float32 array never reaches a launch (these run without a
    GPU: each case is rejected in Python)."""
    import torch
    dims, bc = (4, 4, 4), (0,) * 6
    N = 64
    cpu = torch.zeros(N, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        T.tslb_diagnostics_noalloc(cpu, torch.zeros(3 * N, dtype=torch.float64), None, dims, bc, 0.6,
                                   torch.zeros(8, dtype=torch.float64))
    with pytest.raises(ValueError, match="dims"):
        T.tslb_diagnostics_noalloc(cpu, cpu, None, (4, 4), bc, 0.6, cpu)
    with pytest.raises(ValueError, match="out must be given"):
        T.tslb_diagnostics_noalloc(cpu, cpu, None, dims, bc, 0.6, None)


def test_halo_face_rules():
    """Halo faces (the z-slab decomposition) are z faces on both sides, with
    periodic x, periodic or bounce-back y, the factored kernel, no sponge and
    no checkpoints; the rejections come before any CUDA call."""
    H = T.HALO
    for dims, bc, code in (((8, 8, 8), (H, H, 0, 0, 0, 0), T.TSLB_ERR_UNSUPPORTED),   # x faces
                           ((8, 8, 8), (0, 0, 0, 0, H, 0), T.TSLB_ERR_INVALID),       # mixed with periodic
                           ((8, 8, 8), (0, 0, 0, 0, H, 4), T.TSLB_ERR_UNSUPPORTED),   # halo + outflow
                           ((8, 8, 8), (2, 2, 0, 0, H, H), T.TSLB_ERR_UNSUPPORTED),   # free-slip x
                           ((8, 8, 8), (0, 0, 5, 5, H, H), T.TSLB_ERR_UNSUPPORTED),   # NEE walls
                           ((8, 8, 2), (0, 0, 0, 0, H, H), T.TSLB_ERR_INVALID),       # fewer than 3 layers
                           ((8, 8, 8), (0, 0, 0, 0, 7, 7), T.TSLB_ERR_INVALID)):      # unknown code
        c, h = _create_code(dims=dims, bc=bc)
        assert c == code, (bc, c)
        assert not h.value
    for attr, val in (("kernel", T.KERNEL_DIRECT), ("checkpoint_every", 4), ("forcing", T.TSLB_FORCING_GUO)):
        o = T.tslb_options_default()
        setattr(o, attr, val)
        assert _create_code(bc=(0, 0, 0, 0, H, H), opt=o)[0] == T.TSLB_ERR_UNSUPPORTED, attr
    o = T.tslb_options_default()
    o.sponge_width, o.sponge_k = 3, 1.0
    assert _create_code(bc=(0, 0, 0, 0, H, H), opt=o)[0] == T.TSLB_ERR_UNSUPPORTED
    L = T.load()
    b = ctypes.c_int64(0)
    assert L.tslb_halo_plane_bytes(None, ctypes.byref(b)) == T.TSLB_ERR_INVALID
    assert L.tslb_halo_export(None, 0, None, T.HOST) == T.TSLB_ERR_INVALID
    assert L.tslb_halo_import(None, 0, None, T.HOST) == T.TSLB_ERR_INVALID
