"""FP64 CPU oracle for the high-order thread-safe lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
(``paper_2401_17074_b300``) never imports this package, and this package
shares no code with it.

The numerics live in ``tslb_oracle.cpp`` (population-based, direct
per-direction sums of Eq. eqts / Eq. noneqts / Eq. pushLB of arXiv 2401.17074);
this module only compiles it with g++/OpenMP and marshals numpy arrays.
Array conventions match the C ABI: full-lattice arrays of N = nx*ny*nz nodes,
x fastest; ``u`` is [3][N]; ``pi`` is [6][N] in the order xx, yy, zz, xy, xz, yz.
"""
import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tslb_oracle.cpp")
_SRC2 = os.path.join(_HERE, "tslb_oracle2d.cpp")
# ORACLE_SANITIZE=1 selects a build with AddressSanitizer and
# UndefinedBehaviorSanitizer (the process must preload the ASan runtime).
_SANITIZE = os.environ.get("ORACLE_SANITIZE") == "1"
_LIB = os.path.join(_HERE, "liboracle_san.so" if _SANITIZE else "liboracle.so")

PERIODIC, BOUNCEBACK, FREESLIP, INFLOW, OUTFLOW, NEE_WALL = 0, 1, 2, 3, 4, 5

_lib = None


def build(force=False):
    """Compile the oracle shared library with g++ -O3 -fopenmp (sanitized: -O1 with ASan and UBSan)."""
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(p) for p in (_SRC, _SRC2))
    if force or stale:
        opt = (["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                "-fno-sanitize-recover=undefined"] if _SANITIZE else ["-O3"])
        subprocess.check_call(["g++"] + opt + ["-fopenmp", "-fPIC", "-shared", "-std=c++17",
                                               "-o", _LIB, _SRC, _SRC2])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ip = ctypes.POINTER(ctypes.c_int)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_lattice.argtypes = [ip, dp]
        L.orc_feq3.argtypes = [ctypes.c_double, dp, dp]
        L.orc_fneq3.argtypes = [dp, dp, dp]
        L.orc_post.argtypes = [ctypes.c_double, dp, dp, ctypes.c_double, dp, dp]
        L.orc_moments.argtypes = [dp, dp, dp, dp]
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_inflow_noise.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        L.orc_inflow_noise.restype = ctypes.c_double
        L.orc_inflow_noise_gauss.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        L.orc_inflow_noise_gauss.restype = ctypes.c_double
        L.orc_set_sponge.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double]
        L.orc_set_forcing.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_create.argtypes = [i64p, ctypes.c_double, dp, ip, i64p, dp, ctypes.c_uint64, ip]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_init_moments.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc_set_force_field.argtypes = [ctypes.c_void_p, dp]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc_get_moments.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc_get_populations.argtypes = [ctypes.c_void_p, dp]
        L.orc_time.argtypes = [ctypes.c_void_p]
        L.orc_time.restype = ctypes.c_int64
        L.orc2_lattice.argtypes = [ip, dp]
        L.orc2_feq3.argtypes = [ctypes.c_double, dp, dp]
        L.orc2_fneq3.argtypes = [dp, dp, dp]
        L.orc2_moments.argtypes = [dp, dp, dp, dp]
        L.orc2_create.argtypes = [i64p, ctypes.c_double, dp, ip, ip]
        L.orc2_create.restype = ctypes.c_void_p
        L.orc2_destroy.argtypes = [ctypes.c_void_p]
        L.orc2_init_moments.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc2_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc2_get_moments.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc_complex_run.argtypes = [i64p, ctypes.c_double, ip, dp, dp, dp, dp, dp, ctypes.c_int64, dp, dp]
        L.orc_complex_run_moments.argtypes = [i64p, ctypes.c_double, ip, dp, dp, dp, dp, dp, ctypes.c_int64, dp,
                                              dp]
        L.orc_threads.argtypes = []
        L.orc_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice():
    """Return (c [27,3] int, w [27]) in the oracle's direction order."""
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().orc_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(w))
    return c, w


def feq3(rho, u):
    out = np.zeros(27)
    u = _f64(u)
    lib().orc_feq3(float(rho), _d(u), _d(out))
    return out


def fneq3(pi6, u):
    out = np.zeros(27)
    pi6, u = _f64(pi6), _f64(u)
    lib().orc_fneq3(_d(pi6), _d(u), _d(out))
    return out


def post_collision(rho, u, pi6, omega, F=(0.0, 0.0, 0.0)):
    out = np.zeros(27)
    u, pi6, F = _f64(u), _f64(pi6), _f64(F)
    lib().orc_post(float(rho), _d(u), _d(pi6), float(omega), _d(F), _d(out))
    return out


def moments(f):
    f = _f64(f)
    rho = np.zeros(1)
    u = np.zeros(3)
    pi6 = np.zeros(6)
    lib().orc_moments(_d(f), _d(rho), _d(u), _d(pi6))
    return rho[0], u, pi6


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    p = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def inflow_noise(seed, x, y, t):
    return lib().orc_inflow_noise(int(seed), int(x), int(y), int(t))


def inflow_noise_gauss(seed, x, y, t):
    return lib().orc_inflow_noise_gauss(int(seed), int(x), int(y), int(t))


class OracleSim:
    """Population-based FP64 TSLB simulation on a full nx*ny*nz lattice.

    bc = (x-, x+, y-, y+, z-, z+) face codes.  A non-periodic face makes the
    outermost node layer a boundary layer (solid for BOUNCEBACK / FREESLIP,
    ghost for INFLOW / OUTFLOW); only interior nodes are updated.
    inflow = dict(center2=(cx2, cy2), diameter=D, u_jet=U, noise_amp=a, seed=s[, origin=(ox, oy)]
    [, noise="uniform" | "gaussian"]); origin places this box inside a larger lattice for the nozzle
    mask and the noise counter (a sub-box that reproduces part of a full-size run).
    sponge = (W, K): viscosity raised over the last W layers towards z+ (jet exit).
    forcing = "luo" (default) or "guo"; with Guo forcing and a force field, set the
    field before init_moments (the initial populations depend on it).
    """

    def __init__(self, dims, tau, force=(0.0, 0.0, 0.0), bc=(0,) * 6, inflow=None, sponge=None, forcing="luo"):
        self.dims = tuple(int(d) for d in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        d = np.array(self.dims, dtype=np.int64)
        F = _f64(force)
        b = np.array(bc, dtype=np.int32)
        ii = np.zeros(6, dtype=np.int64)
        dd = np.zeros(2)
        seed = 0
        if inflow is not None:
            org = inflow.get("origin", (0, 0))
            kind = {"uniform": 0, "gaussian": 1}[inflow.get("noise", "uniform")]
            ii[:] = [inflow["center2"][0], inflow["center2"][1], inflow["diameter"], org[0], org[1], kind]
            dd[:] = [inflow["u_jet"], inflow["noise_amp"]]
            seed = int(inflow["seed"])
        st = ctypes.c_int(0)
        self._h = lib().orc_create(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(tau), _d(F),
                                   b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   ii.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _d(dd),
                                   seed, ctypes.byref(st))
        if not self._h:
            raise ValueError("oracle rejected the configuration (status %d)" % st.value)
        if sponge is not None:
            if lib().orc_set_sponge(self._h, int(sponge[0]), float(sponge[1])) != 0:
                raise ValueError("oracle rejected the sponge layer")
        if forcing != "luo":
            if lib().orc_set_forcing(self._h, {"guo": 1}[forcing]) != 0:
                raise ValueError("oracle rejected Guo forcing for these faces")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def init_moments(self, rho, u, pi=None):
        rho = _f64(rho).reshape(-1)
        u = _f64(u).reshape(-1)
        pi_p = None
        if pi is not None:
            pi = _f64(pi).reshape(-1)
            pi_p = _d(pi)
        assert rho.size == self.N and u.size == 3 * self.N
        lib().orc_init_moments(self._h, _d(rho), _d(u), pi_p)

    def set_force_field(self, F):
        if F is None:
            lib().orc_set_force_field(self._h, None)
            return
        F = _f64(F).reshape(-1)
        assert F.size == 3 * self.N
        lib().orc_set_force_field(self._h, _d(F))

    def step(self, n=1):
        st = lib().orc_step(self._h, int(n))
        if st != 0:
            raise RuntimeError("oracle step failed (%d)" % st)

    @property
    def t(self):
        return lib().orc_time(self._h)

    def get_moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        pi = np.zeros(6 * self.N)
        lib().orc_get_moments(self._h, _d(rho), _d(u), _d(pi))
        return rho, u.reshape(3, self.N), pi.reshape(6, self.N)

    def get_populations(self):
        f = np.zeros(27 * self.N)
        lib().orc_get_populations(self._h, _d(f))
        return f.reshape(self.N, 27)


def complex_step_energy(dims, tau, bc, rho, u, pi, F_re, F_im, nsteps):
    """J = 1/2 sum rho u.u after nsteps, with a complex force field (F_re + i F_im).

    Returns the complex J as a Python complex; Im(J)/h for F_im = h v is the
    directional derivative of J along v (complex-step differentiation).
    """
    d = np.array(dims, dtype=np.int64)
    b = np.array(bc, dtype=np.int32)
    rho, u = _f64(rho).reshape(-1), _f64(u).reshape(-1)
    pi = _f64(pi).reshape(-1) if pi is not None else np.zeros(6 * rho.size)
    F_re, F_im = _f64(F_re).reshape(-1), _f64(F_im).reshape(-1)
    jr = ctypes.c_double(0.0)
    ji = ctypes.c_double(0.0)
    st = lib().orc_complex_run(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(tau),
                               b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(rho), _d(u), _d(pi),
                               _d(F_re), _d(F_im), int(nsteps), ctypes.byref(jr), ctypes.byref(ji))
    if st != 0:
        raise ValueError("oracle rejected the configuration (status %d)" % st)
    return complex(jr.value, ji.value)


def complex_step_moments(dims, tau, bc, rho, u, pi, F_re, F_im, nsteps):
    """Complex final moments after nsteps with the force field F_re + i F_im.

    Returns (rho [N], u [3, N], pi [6, N]) as complex arrays (full lattice,
    boundary layers at the rest state).  For F_im = h v, Im J(m)/h of any
    holomorphic objective J is its directional derivative along v.
    """
    d = np.array(dims, dtype=np.int64)
    b = np.array(bc, dtype=np.int32)
    rho, u = _f64(rho).reshape(-1), _f64(u).reshape(-1)
    N = rho.size
    pi = _f64(pi).reshape(-1) if pi is not None else np.zeros(6 * N)
    F_re, F_im = _f64(F_re).reshape(-1), _f64(F_im).reshape(-1)
    m_re = np.zeros(10 * N)
    m_im = np.zeros(10 * N)
    st = lib().orc_complex_run_moments(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(tau),
                                       b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(rho), _d(u), _d(pi),
                                       _d(F_re), _d(F_im), int(nsteps), _d(m_re), _d(m_im))
    if st != 0:
        raise ValueError("oracle rejected the configuration (status %d)" % st)
    m = m_re + 1j * m_im
    return m[:N], m[N:4 * N].reshape(3, N), m[4 * N:].reshape(6, N)


def threads():
    """OpenMP threads of the oracle's parallel loops in this process."""
    return int(lib().orc_threads())


# ---- D2Q9 ------------------------------------------------------------------------

def lattice2d():
    """Return (c [9,2] int, w [9]) of the D2Q9 oracle."""
    c = np.zeros((9, 2), dtype=np.int32)
    w = np.zeros(9)
    lib().orc2_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(w))
    return c, w


def feq3_2d(rho, u):
    out = np.zeros(9)
    lib().orc2_feq3(float(rho), _d(_f64(u)), _d(out))
    return out


def fneq3_2d(pi3, u):
    """pi3 = (xx, yy, xy)."""
    out = np.zeros(9)
    lib().orc2_fneq3(_d(_f64(pi3)), _d(_f64(u)), _d(out))
    return out


def moments2d(f):
    rho = np.zeros(1)
    u = np.zeros(2)
    pi3 = np.zeros(3)
    lib().orc2_moments(_d(_f64(f)), _d(rho), _d(u), _d(pi3))
    return rho[0], u, pi3


class OracleSim2D:
    """Population-based FP64 D2Q9 TSLB simulation on a full nx*ny lattice.

    bc = (x-, x+, y-, y+): PERIODIC, or BOUNCEBACK on the y faces (solid
    layers y = 0 and y = ny-1).  Moments: rho[N], u[2][N], pi[3][N] (xx, yy, xy).
    """

    def __init__(self, dims, tau, force=(0.0, 0.0), bc=(0, 0, 0, 0)):
        self.dims = (int(dims[0]), int(dims[1]))
        self.N = self.dims[0] * self.dims[1]
        d = np.array(self.dims, dtype=np.int64)
        b = np.array(bc, dtype=np.int32)
        st = ctypes.c_int(0)
        self._h = lib().orc2_create(d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(tau), _d(_f64(force)),
                                    b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(st))
        if not self._h:
            raise ValueError("oracle rejected the configuration (status %d)" % st.value)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc2_destroy(self._h)
            self._h = None

    def init_moments(self, rho, u, pi=None):
        rho = _f64(rho).reshape(-1)
        u = _f64(u).reshape(-1)
        keep = _f64(pi).reshape(-1) if pi is not None else None
        pi_p = _d(keep) if keep is not None else None
        assert rho.size == self.N and u.size == 2 * self.N
        lib().orc2_init_moments(self._h, _d(rho), _d(u), pi_p)

    def step(self, n=1):
        st = lib().orc2_step(self._h, int(n))
        if st != 0:
            raise RuntimeError("oracle step failed (%d)" % st)

    def get_moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(2 * self.N)
        pi = np.zeros(3 * self.N)
        lib().orc2_get_moments(self._h, _d(rho), _d(u), _d(pi))
        return rho, u.reshape(2, self.N), pi.reshape(3, self.N)
