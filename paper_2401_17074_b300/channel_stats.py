"""Wall-normal statistics of a channel run: the mean velocity U(y) and the
Reynolds stresses <u'_i u'_j>(y), averaged over the periodic x and z
directions and over samples in time.  These are the quantities the channel
results of Sec. 3.1 are compared on, and the measures of the 16-bit storage
study.

Analysis of outputs only (none of the step's arithmetic).  Works on numpy
arrays and on torch tensors alike (host or device); sums accumulate in FP64.
Fields use the C ABI layout: full lattice, x fastest, u [3][N]; the wall
rows y = 0 and y = ny - 1 are excluded.
"""
import numpy as np

PAIRS = (("uu", 0, 0), ("vv", 1, 1), ("ww", 2, 2), ("uv", 0, 1))


class ChannelStats:
    def __init__(self, dims):
        self.nx, self.ny, self.nz = (int(d) for d in dims)
        self.count = 0
        self.s1 = None  # [3][ny - 2] sums of u_i
        self.s2 = None  # [4][ny - 2] sums of u_i u_j for PAIRS

    def add(self, u):
        """Add one sample of the velocity field u [3][N]."""
        nx, ny, nz = self.nx, self.ny, self.nz
        comp = [u[i].reshape(nz, ny, nx)[:, 1:ny - 1, :] for i in range(3)]
        s1 = [c.sum(axis=(0, 2)) for c in comp]
        s2 = [(comp[a] * comp[b]).sum(axis=(0, 2)) for _, a, b in PAIRS]
        s1 = np.stack([_host(v) for v in s1])
        s2 = np.stack([_host(v) for v in s2])
        if self.s1 is None:
            self.s1, self.s2 = s1, s2
        else:
            self.s1 += s1
            self.s2 += s2
        self.count += nx * nz

    def result(self):
        """Mean profiles U, V, W and stresses uu, vv, ww, uv (each an array over the ny - 2 fluid rows)."""
        m = self.s1 / self.count
        out = {"U": m[0], "V": m[1], "W": m[2]}
        for k, (name, a, b) in enumerate(PAIRS):
            out[name] = self.s2[k] / self.count - m[a] * m[b]
        return out


def _host(v):
    if hasattr(v, "detach"):  # torch tensor
        return v.detach().double().cpu().numpy()
    return np.asarray(v, dtype=np.float64)


def profile_errors(got, ref):
    """Relative L2 errors over y of U and of each Reynolds-stress profile of `got` against `ref`."""
    out = {}
    for k in ("U", "uu", "vv", "ww", "uv"):
        out[k] = float(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k]))
    return out
