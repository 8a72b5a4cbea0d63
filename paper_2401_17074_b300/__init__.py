"""Python binding of the B300 high-order thread-safe lattice Boltzmann library.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libtslb.so`` (built from ``csrc/`` by ``build.py``).  The functions keep
the C names of ``include/tslb.h``; ``Solver`` is a small convenience wrapper
that accepts numpy arrays or CUDA torch tensors.  Loading fails loudly when
the shared library is missing -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

TSLB_OK = 0
TSLB_ERR_INVALID = -1
TSLB_ERR_UNSUPPORTED = -2
TSLB_ERR_CUDA = -3
TSLB_ERR_ALLOC = -4
TSLB_ERR_UNSTABLE = -5
TSLB_ERR_STATE = -6

TSLB_D3Q27 = 27
TSLB_D2Q9 = 9
PERIODIC, BOUNCEBACK, FREESLIP, INFLOW, OUTFLOW, NEE_WALL, HALO = 0, 1, 2, 3, 4, 5, 6
FP32, BF16, FP16 = 0, 1, 2
HOST, DEVICE = 0, 1
KERNEL_AUTO, KERNEL_DIRECT, KERNEL_FACTORED = 0, 1, 2
TSLB_NOISE_UNIFORM, TSLB_NOISE_GAUSSIAN = 0, 1
TSLB_FORCING_LUO, TSLB_FORCING_GUO = 0, 1
TSLB_ROUND_NEAREST, TSLB_ROUND_STOCHASTIC = 0, 1

EXPORTED = [
    "tslb_options_default", "tslb_create", "tslb_init_moments", "tslb_init_moments_f32", "tslb_set_force_field",
    "tslb_step", "tslb_get_moments", "tslb_get_moments_f32", "tslb_diagnostics", "tslb_adjoint_force_gradient",
    "tslb_adjoint", "tslb_interior_nodes", "tslb_synchronize", "tslb_destroy", "tslb_last_error",
    "tslb_diagnostics_noalloc", "tslb_halo_plane_bytes", "tslb_halo_export", "tslb_halo_import", "tslb_step_part",
]
TSLB_PART_EDGES, TSLB_PART_INTERIOR = 1, 2
HALO_EDGE_LAYERS = 4
NOALLOC_MAX_NODES = 1 << 26


class tslb_inflow(ctypes.Structure):
    _fields_ = [("center2", ctypes.c_int64 * 2), ("diameter", ctypes.c_int64), ("u_jet", ctypes.c_double),
                ("noise_amp", ctypes.c_double), ("seed", ctypes.c_uint64), ("noise_kind", ctypes.c_int)]


class tslb_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("u_ref", ctypes.c_double), ("pi_ref", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("device", ctypes.c_int), ("kernel", ctypes.c_int),
                ("checkpoint_every", ctypes.c_int), ("inflow", tslb_inflow), ("sponge_width", ctypes.c_int),
                ("sponge_k", ctypes.c_double), ("forcing", ctypes.c_int), ("rounding", ctypes.c_int),
                ("rounding_seed", ctypes.c_uint64), ("halo_stream", ctypes.c_void_p)]


class tslb_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3), ("kinetic_energy", ctypes.c_double),
                ("wall_shear", ctypes.c_double), ("max_speed", ctypes.c_double), ("nonfinite", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("nodes", ctypes.c_int64)]

    def as_dict(self):
        return {"mass": self.mass, "momentum": list(self.momentum), "kinetic_energy": self.kinetic_energy,
                "wall_shear": self.wall_shear, "max_speed": self.max_speed, "nonfinite": self.nonfinite,
                "steps": self.steps, "nodes": self.nodes}


_lib = None


def lib_path():
    """libtslb.so; with TSLB_CHECKED=1 its index-checked build libtslb_checked.so,
    with TSLB_HOSTSAN=1 its host-sanitized build libtslb_hostsan.so."""
    if os.environ.get("TSLB_HOSTSAN") == "1":
        return _build.LIB_HOSTSAN
    return _build.LIB_CHECKED if os.environ.get("TSLB_CHECKED") == "1" else _build.LIB


def load(build_if_missing=True):
    """Load the library (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("%s is missing; run paper_2401_17074_b300.build.build()" % os.path.basename(path))
    L = ctypes.CDLL(path)
    vp, i64, dp, fp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
    L.tslb_options_default.argtypes = [ctypes.POINTER(tslb_options)]
    L.tslb_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(i64), ctypes.c_double, dp,
                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(tslb_options)]
    L.tslb_init_moments.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    L.tslb_init_moments_f32.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    L.tslb_set_force_field.argtypes = [vp, fp, ctypes.c_int]
    L.tslb_step.argtypes = [vp, i64]
    L.tslb_get_moments.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    L.tslb_get_moments_f32.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    L.tslb_diagnostics.argtypes = [vp, ctypes.POINTER(tslb_diag)]
    L.tslb_adjoint_force_gradient.argtypes = [vp, i64, fp, ctypes.c_int]
    L.tslb_adjoint.argtypes = [vp, vp, i64, ctypes.c_int, fp, ctypes.c_int]
    L.tslb_interior_nodes.argtypes = [vp]
    L.tslb_interior_nodes.restype = i64
    L.tslb_synchronize.argtypes = [vp]
    L.tslb_destroy.argtypes = [vp]
    L.tslb_destroy.restype = None
    L.tslb_last_error.argtypes = [vp]
    L.tslb_last_error.restype = ctypes.c_char_p
    L.tslb_diagnostics_noalloc.argtypes = [vp, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int),
                                           ctypes.c_double, vp, vp]
    L.tslb_halo_plane_bytes.argtypes = [vp, ctypes.POINTER(i64)]
    L.tslb_halo_export.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.tslb_halo_import.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
    L.tslb_step_part.argtypes = [vp, ctypes.c_int]
    _lib = L
    return L


class TslbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("tslb error %d: %s" % (code, msg))
        self.code = code


def _check(code, h=None):
    if code != TSLB_OK:
        msg = load().tslb_last_error(h).decode(errors="replace")
        raise TslbError(code, msg)
    return code


# ---- C-named thin wrappers --------------------------------------------------

def tslb_options_default():
    o = tslb_options()
    _check(load().tslb_options_default(ctypes.byref(o)))
    return o


def tslb_create(dims, tau, force=None, bc=(0,) * 6, opt=None, lattice=TSLB_D3Q27):
    L = load()
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 3)(*[int(v) for v in dims])
    b = (ctypes.c_int * 6)(*[int(v) for v in bc])
    f = (ctypes.c_double * 3)(*[float(v) for v in force]) if force is not None else None
    code = L.tslb_create(ctypes.byref(h), int(lattice), d, float(tau), f, b,
                         ctypes.byref(opt) if opt is not None else None)
    _check(code, None)
    return h


def _device_ptr(t):
    """Pointer of a CUDA tensor for a call that reads or writes it on the
    handle's own stream.  Work queued on PyTorch's current stream may still be
    producing the tensor (or, for freshly allocated memory, still reading what
    the allocator handed back), so that stream is drained first."""
    import torch
    torch.cuda.current_stream(t.device).synchronize()
    return ctypes.c_void_p(t.data_ptr())


def _out_ptr(a):
    """Pointer of an output array: numpy, CPU tensor or CUDA tensor."""
    if a is None:
        return None
    if hasattr(a, "is_cuda") and a.is_cuda:
        return _device_ptr(a)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _ptr(a, dtype):
    """Return (pointer, where, keepalive) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, HOST, None
    if hasattr(a, "is_cuda") and a.is_cuda:
        import torch
        want = torch.float64 if dtype == np.float64 else torch.float32
        t = a.contiguous()
        if t.dtype != want:
            raise TypeError("expected %s tensor" % want)
        return _device_ptr(t), DEVICE, t
    if hasattr(a, "numpy"):  # CPU torch tensor (pinned or pageable)
        t = a.contiguous()
        return ctypes.c_void_p(t.data_ptr()), HOST, t
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), HOST, arr


def tslb_init_moments(h, rho, u, pi=None):
    pr, w, k1 = _ptr(rho, np.float64)
    pu, w2, k2 = _ptr(u, np.float64)
    pp, w3, k3 = _ptr(pi, np.float64)
    if pi is not None and not (w == w2 == w3):
        raise ValueError("rho, u, pi must all be host or all device")
    _check(load().tslb_init_moments(h, pr, pu, pp, w), h)


def tslb_set_force_field(h, F):
    if F is None:
        _check(load().tslb_set_force_field(h, None, HOST), h)
        return
    p, w, k = _ptr(F, np.float32)
    _check(load().tslb_set_force_field(h, p, w), h)


def tslb_step(h, nsteps=1):
    _check(load().tslb_step(h, int(nsteps)), h)


def tslb_init_moments_f32(h, drho, u, pi=None):
    """FP32 moments with the density as drho = rho - 1 (numpy float32 or CUDA float32 tensors)."""
    pr, w, k1 = _ptr(drho, np.float32)
    pu, w2, k2 = _ptr(u, np.float32)
    pp, w3, k3 = _ptr(pi, np.float32)
    if pi is not None and not (w == w2 == w3):
        raise ValueError("drho, u, pi must all be host or all device")
    _check(load().tslb_init_moments_f32(h, pr, pu, pp, w), h)


def tslb_get_moments_f32(h, drho=None, u=None, pi=None, where=HOST):
    p = _out_ptr
    _check(load().tslb_get_moments_f32(h, p(drho), p(u), p(pi), int(where)), h)


def tslb_get_moments(h, rho=None, u=None, pi=None, where=HOST):
    p = _out_ptr
    _check(load().tslb_get_moments(h, p(rho), p(u), p(pi), int(where)), h)


def tslb_diagnostics(h):
    d = tslb_diag()
    code = load().tslb_diagnostics(h, ctypes.byref(d))
    if code not in (TSLB_OK, TSLB_ERR_UNSTABLE):
        _check(code, h)
    return d, code


def tslb_adjoint_force_gradient(h, nsteps, dJdF, where=HOST):
    _check(load().tslb_adjoint_force_gradient(h, int(nsteps), _out_ptr(dJdF), int(where)), h)


def tslb_adjoint(h, lambda_T, nsteps, ckpt_every, dJdF, where=HOST):
    """dJ/dF for the cotangent lambda_T ([10][N] FP64: rho, u, Pi rows, full lattice).

    lambda_T and dJdF are both host arrays (where=HOST: numpy or CPU tensors) or
    both CUDA tensors (where=DEVICE)."""
    if where == DEVICE:
        lp, lw, keep = _ptr(lambda_T, np.float64)
        if lw != DEVICE:
            raise TypeError("lambda_T must be a CUDA float64 tensor with where=DEVICE")
    else:
        keep = np.ascontiguousarray(lambda_T, dtype=np.float64)
        lp = ctypes.c_void_p(keep.ctypes.data)
    _check(load().tslb_adjoint(h, lp, int(nsteps), int(ckpt_every), _out_ptr(dJdF), int(where)), h)


def tslb_diagnostics_noalloc(rho, u, pi, dims, bc, tau, out, stream=None):
    """FP64 diagnostics of caller-owned device moment arrays without any allocation.

    rho, u, pi: CUDA float64 tensors in the full-lattice layout of
    tslb_get_moments; out: CUDA float64 tensor of 8 entries.  Asynchronous on
    `stream` (a raw cudaStream_t value, None = default stream).
    """
    import torch
    dims = [int(v) for v in dims]
    if len(dims) != 3 or min(dims) < 1:
        raise ValueError("dims must be three positive extents")
    N = dims[0] * dims[1] * dims[2]
    # every array is checked before the launch: the kernels read N, 3N and 6N
    # doubles and write 8, with no bounds of their own
    arrays = (("rho", rho, N), ("u", u, 3 * N), ("pi", pi, 6 * N), ("out", out, 8))
    for name, a, need in arrays:
        if a is None and name != "pi":
            raise ValueError("%s must be given" % name)
    for name, a, need in arrays:
        if a is None:
            continue
        if not (hasattr(a, "is_cuda") and a.is_cuda):
            raise ValueError("%s must be a CUDA tensor" % name)
        if a.dtype != torch.float64:
            raise ValueError("%s must be float64" % name)
        if not a.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if a.numel() < need:
            raise ValueError("%s holds %d values, %d needed" % (name, a.numel(), need))

    def p(a):
        return None if a is None else ctypes.c_void_p(a.data_ptr())
    d = (ctypes.c_int64 * 3)(*dims)
    b = (ctypes.c_int * 6)(*[int(v) for v in bc])
    s = ctypes.c_void_p(int(stream)) if stream else None
    _check(load().tslb_diagnostics_noalloc(p(rho), p(u), p(pi), d, b, float(tau), s, p(out)), None)


def tslb_halo_plane_bytes(h):
    b = ctypes.c_int64(0)
    _check(load().tslb_halo_plane_bytes(h, ctypes.byref(b)), h)
    return b.value


def _buf_ptr(a):
    """(pointer, where) of a contiguous buffer: CUDA tensor, CPU tensor or numpy array.
    A CUDA buffer is passed as it is, without draining PyTorch's stream: halo
    buffers are ordered by the caller on the handle's halo stream."""
    if hasattr(a, "is_cuda") and a.is_cuda:
        if not a.is_contiguous():
            raise ValueError("halo buffers must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), DEVICE
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr()), HOST
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("halo buffers must be contiguous")
    return ctypes.c_void_p(a.ctypes.data), HOST


def _halo_buf(h, a):
    nbytes = a.numel() * a.element_size() if hasattr(a, "element_size") else a.nbytes
    need = tslb_halo_plane_bytes(h)
    if nbytes < need:
        raise ValueError("halo buffer holds %d bytes, %d needed" % (nbytes, need))
    return _buf_ptr(a)


def tslb_halo_export(h, side, dst):
    """Pack this slab's layer z = 0 (side 0) or z = nz - 1 (side 1) into dst."""
    p, where = _halo_buf(h, dst)
    _check(load().tslb_halo_export(h, int(side), p, where), h)


def tslb_halo_import(h, side, src):
    """Load a packed plane into the ghost layer below (side 0) or above (side 1) the slab."""
    p, where = _halo_buf(h, src)
    _check(load().tslb_halo_import(h, int(side), p, where), h)


def tslb_step_part(h, part):
    """One part of a split step of a halo slab: TSLB_PART_EDGES, then TSLB_PART_INTERIOR."""
    _check(load().tslb_step_part(h, int(part)), h)


def tslb_interior_nodes(h):
    return load().tslb_interior_nodes(h)


def tslb_synchronize(h):
    _check(load().tslb_synchronize(h), h)


def tslb_destroy(h):
    load().tslb_destroy(h)


def tslb_last_error(h=None):
    return load().tslb_last_error(h).decode(errors="replace")


# ---- convenience wrapper ----------------------------------------------------

class Solver:
    """Owns one TSLB handle.  Arrays follow the C ABI layouts (full lattice, x fastest)."""

    def __init__(self, dims, tau, force=(0.0, 0.0, 0.0), bc=(0,) * 6, precision=FP32, u_ref=0.05, pi_ref=1e-3,
                 kernel=KERNEL_AUTO, stream=None, device=0, checkpoint_every=0, inflow=None, sponge=None,
                 lattice=None, forcing="luo", rounding="nearest", rounding_seed=0, halo_stream=None):
        """inflow: dict(center2, diameter, u_jet, noise_amp, seed[, noise="uniform" | "gaussian"]);
        sponge: (width, K) viscosity layer towards the z+ face (tslb_options.sponge_width / sponge_k);
        rounding: "nearest" or "stochastic" (16-bit storage; tslb_options.rounding / rounding_seed)."""
        o = tslb_options_default()
        o.precision = int(precision)
        o.u_ref = float(u_ref)
        o.pi_ref = float(pi_ref)
        o.kernel = int(kernel)
        o.device = int(device)
        o.checkpoint_every = int(checkpoint_every)
        if stream is not None:
            o.stream = ctypes.c_void_p(int(stream))
        if inflow is not None:
            o.inflow.center2[0] = int(inflow["center2"][0])
            o.inflow.center2[1] = int(inflow["center2"][1])
            o.inflow.diameter = int(inflow["diameter"])
            o.inflow.u_jet = float(inflow["u_jet"])
            o.inflow.noise_amp = float(inflow["noise_amp"])
            o.inflow.seed = int(inflow["seed"])
            o.inflow.noise_kind = {"uniform": TSLB_NOISE_UNIFORM,
                                   "gaussian": TSLB_NOISE_GAUSSIAN}[inflow.get("noise", "uniform")]
        o.forcing = {"luo": TSLB_FORCING_LUO, "guo": TSLB_FORCING_GUO}[forcing]
        o.rounding = {"nearest": TSLB_ROUND_NEAREST, "stochastic": TSLB_ROUND_STOCHASTIC}[rounding]
        o.rounding_seed = int(rounding_seed)
        if halo_stream is not None:
            o.halo_stream = ctypes.c_void_p(int(halo_stream))
        if sponge is not None:
            o.sponge_width = int(sponge[0])
            o.sponge_k = float(sponge[1])
        self.dims = tuple(int(d) for d in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        # the stream the halo copies run on, where the caller chose it (None: the
        # handle's own stream, which PyTorch cannot see)
        self.halo_copy_stream = halo_stream if halo_stream is not None else stream
        self._h = tslb_create(self.dims, tau, force, bc, o, lattice=TSLB_D3Q27 if lattice is None else lattice)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            tslb_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_moments(self, rho, u, pi=None):
        tslb_init_moments(self._h, rho, u, pi)

    def set_force_field(self, F):
        tslb_set_force_field(self._h, F)

    def step(self, n=1):
        tslb_step(self._h, n)

    def init_moments_f32(self, drho, u, pi=None):
        """FP32 moments; the density given as drho = rho - 1 (tslb_init_moments_f32)."""
        tslb_init_moments_f32(self._h, drho, u, pi)

    def get_moments_f32(self):
        """(drho, u, pi) as FP32 arrays, drho = rho - 1 (tslb_get_moments_f32)."""
        drho = np.zeros(self.N, dtype=np.float32)
        u = np.zeros(3 * self.N, dtype=np.float32)
        pi = np.zeros(6 * self.N, dtype=np.float32)
        tslb_get_moments_f32(self._h, drho, u, pi, HOST)
        return drho, u.reshape(3, self.N), pi.reshape(6, self.N)

    def get_moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        pi = np.zeros(6 * self.N)
        tslb_get_moments(self._h, rho, u, pi, HOST)
        return rho, u.reshape(3, self.N), pi.reshape(6, self.N)

    def diagnostics(self):
        d, code = tslb_diagnostics(self._h)
        return d.as_dict(), code

    def interior_nodes(self):
        return tslb_interior_nodes(self._h)

    def synchronize(self):
        tslb_synchronize(self._h)

    def adjoint_force_gradient(self, nsteps):
        g = np.zeros(3 * self.N, dtype=np.float32)
        tslb_adjoint_force_gradient(self._h, nsteps, g, HOST)
        return g.reshape(3, self.N)

    def halo_plane_bytes(self):
        return tslb_halo_plane_bytes(self._h)

    def halo_export(self, side, dst):
        tslb_halo_export(self._h, side, dst)

    def halo_import(self, side, src):
        tslb_halo_import(self._h, side, src)

    def step_part(self, part):
        tslb_step_part(self._h, part)

    def adjoint(self, lam, nsteps):
        """dJ/dF ([3, N] FP32) for the cotangent lam = dJ/dm of the current moments,
        given as (lam_rho [N], lam_u [3, N], lam_pi [6, N]) or one [10, N] array."""
        if isinstance(lam, (tuple, list)):
            lam = np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in lam])
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
        if lam.size != 10 * self.N:
            raise ValueError("the cotangent needs 10 N values")
        g = np.zeros(3 * self.N, dtype=np.float32)
        tslb_adjoint(self._h, lam, nsteps, 0, g, HOST)
        return g.reshape(3, self.N)
