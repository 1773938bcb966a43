"""FP64 CPU oracle for the FIt-SNE gradient (arXiv 1712.09005).

TEST INFRASTRUCTURE. This package is the checker, not the product: only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the CUDA library
(``paper_1712_09005_gb300``) and never consumes anything that library
produced.

The arithmetic lives in ``fitsne_oracle.c`` (built here with gcc,
``-O2 -ffp-contract=off -fopenmp``); this module only marshals numpy arrays.
``affinities.py`` holds the oracle's own input-affinity builder (Sec. 1.1,
Eq. p_ij); ``heatmap.py`` the t-SNE heatmaps of Sec. 5; ``oocpca.py`` the
out-of-core randomized PCA of Sec. 6 (Algorithm oocPCA).

Parity status of each function (what pins it is in tests/test_oracle_*.py):
  exact_gradient      pinned: finite differences of KL, closed forms, invariants
  kl                  pinned: closed form for two points, finite differences
  interp_gradient     pinned: Lagrange exactness, nodes-on-grid exactness,
                      convergence to exact_gradient, error bound of Sec. 2.1
  fft                 pinned: numpy.fft and the direct DFT
  step / run          pinned: special cases (plain gradient descent, gain rule)
  affinities.build_P  pinned: perplexity, symmetry, normalisation, brute force
  heatmap.bins        pinned: hand-worked bins, the FP32 decision at a bin edge
  heatmap.gene_bin_sums  pinned: one-hot sparse product, column totals
  heatmap.nearest     pinned: scipy cdist, a planted tie, brute force
  oocpca.oocpca       pinned: planted rank and spectrum, dense SVD (LAPACK),
                      blocking invariance, centring, power-iteration gain
  oocpca.lu_renormalize  pinned: L U = Y, |L| <= 1, permuted unit trapezoid
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fitsne_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP32 decisions need -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Box(ctypes.Structure):
    _fields_ = [("y_min", ctypes.c_float), ("width", ctypes.c_float),
                ("b", ctypes.c_float), ("inv_b", ctypes.c_float),
                ("n_int", ctypes.c_int32), ("p", ctypes.c_int32),
                ("delta", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("n_int_fixed", ctypes.c_int32),
                ("n_min", ctypes.c_int32), ("n_int_max", ctypes.c_int32),
                ("use_fft", ctypes.c_int32), ("force_box", ctypes.c_int32),
                ("box_y_min", ctypes.c_float), ("box_width", ctypes.c_float)]


class _Sched(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int32), ("early_iters", ctypes.c_int32),
                ("late_iters", ctypes.c_int32), ("mom_switch_iter", ctypes.c_int32),
                ("early_alpha", ctypes.c_double), ("late_alpha", ctypes.c_double),
                ("lr", ctypes.c_double), ("momentum_early", ctypes.c_double),
                ("momentum_late", ctypes.c_double), ("min_gain", ctypes.c_double),
                ("gain_inc", ctypes.c_double), ("gain_dec", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.orc_exact_gradient.argtypes = [i64, i32, P, P, P, P, f64, P, P, P, P]
            lib.orc_exact_gradient.restype = i32
            lib.orc_kl.argtypes = [i64, i32, P, P, P, P, f64]
            lib.orc_kl.restype = f64
            lib.orc_box.argtypes = [i64, i32, P, P, P]
            lib.orc_box.restype = i32
            lib.orc_interp_gradient.argtypes = [i64, i32, P, P, P, P, f64, P, P, P, P, P,
                                                P, P, P]
            lib.orc_interp_gradient.restype = i32
            lib.orc_fft.argtypes = [i64, P, P, i32]
            lib.orc_fft.restype = i32
            lib.orc_alpha.argtypes = [P, i32]
            lib.orc_alpha.restype = f64
            lib.orc_step.argtypes = [i64, i32, P, P, P, P, P, i32]
            lib.orc_step.restype = i32
            lib.orc_run.argtypes = [i64, i32, P, P, P, P, P, P, P]
            lib.orc_run.restype = i32
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(P):
    row_ptr, col, val = P
    return (np.ascontiguousarray(row_ptr, dtype=np.int32),
            np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float32))


def _Y(Y):
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    return Y


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def num_threads() -> int:
    return int(_load().orc_num_threads())


@dataclass
class Box:
    y_min: float
    width: float
    b: float
    inv_b: float
    n_int: int
    p: int
    delta: float


@dataclass
class InterpOptions:
    """Interval rule and evaluation mode of the interpolated gradient."""
    p: int = 3
    n_int_fixed: int = 0       # > 0: fixed intervals per dimension
    n_min: int = 50            # floor of max(n_min, ceil(width))
    n_int_max: int = 1000      # cap of the rule
    use_fft: bool = True       # False: literal Toeplitz sum
    force_box: tuple | None = None  # (y_min, width) with n_int_fixed

    def _c(self):
        o = _Opts(self.p, self.n_int_fixed, self.n_min, self.n_int_max, int(self.use_fft),
                  0, 0.0, 0.0)
        if self.force_box is not None:
            o.force_box = 1
            o.box_y_min, o.box_width = float(self.force_box[0]), float(self.force_box[1])
        return o


@dataclass
class Schedule:
    """Exaggeration schedule (Sec. 1.2, Sec. 4) and the optimizer constants."""
    n_iter: int = 1000
    early_iters: int = 250
    late_iters: int = 0
    mom_switch_iter: int = 250
    early_alpha: float = 12.0
    late_alpha: float = 1.0
    lr: float = 200.0
    momentum_early: float = 0.5
    momentum_late: float = 0.8
    min_gain: float = 0.01
    gain_inc: float = 0.2
    gain_dec: float = 0.8

    def _c(self):
        return _Sched(self.n_iter, self.early_iters, self.late_iters, self.mom_switch_iter,
                      self.early_alpha, self.late_alpha, self.lr, self.momentum_early,
                      self.momentum_late, self.min_gain, self.gain_inc, self.gain_dec)


def exact_gradient(Y, P, alpha: float = 1.0):
    """Exact O(N^2) gradient (Sec. 1.1). Returns dict dY, Z, attr, rep."""
    lib = _load()
    Y = _Y(Y)
    N, s = Y.shape
    rp, col, val = _csr(P)
    dY = np.zeros((N, s)); attr = np.zeros((N, s)); rep = np.zeros((N, s))
    Z = ctypes.c_double()
    _check(lib.orc_exact_gradient(N, s, _ptr(Y), _ptr(rp), _ptr(col), _ptr(val), alpha,
                                  _ptr(dY), ctypes.byref(Z), _ptr(attr), _ptr(rep)),
           "exact_gradient")
    return {"dY": dY, "Z": Z.value, "attr": attr, "rep": rep}


def kl(Y, P, Z: float) -> float:
    """KL(P||Q) over the stored entries of P (Sec. 1.1), for a given Z."""
    lib = _load()
    Y = _Y(Y)
    N, s = Y.shape
    rp, col, val = _csr(P)
    return float(lib.orc_kl(N, s, _ptr(Y), _ptr(rp), _ptr(col), _ptr(val), Z))


def box(Y, opts: InterpOptions = InterpOptions()) -> Box:
    lib = _load()
    Y = _Y(Y)
    N, s = Y.shape
    b = _Box()
    o = opts._c()
    _check(lib.orc_box(N, s, _ptr(Y), ctypes.byref(o), ctypes.byref(b)), "box")
    return Box(b.y_min, b.width, b.b, b.inv_b, b.n_int, b.p, b.delta)


def interp_gradient(Y, P, alpha: float = 1.0, opts: InterpOptions = InterpOptions(),
                    want_grids: bool = False):
    """Interpolated gradient (Sec. 2 + Appendix).

    Returns dict with dY (N x s), Z, h (N x (s+2) potentials at the points),
    attr, rep (N x s), box, and with want_grids the spread grids w
    ((s+1) x n^s, node-major as (g1, g2)).
    """
    lib = _load()
    Y = _Y(Y)
    N, s = Y.shape
    rp, col, val = _csr(P)
    o = opts._c()
    bx = box(Y, opts)
    n = bx.n_int * bx.p
    G = n if s == 1 else n * n
    dY = np.zeros((N, s)); attr = np.zeros((N, s)); rep = np.zeros((N, s))
    h = np.zeros((N, s + 2))
    w = np.zeros((s + 1, G)) if want_grids else None
    Z = ctypes.c_double()
    b = _Box()
    _check(lib.orc_interp_gradient(N, s, _ptr(Y), _ptr(rp), _ptr(col), _ptr(val), alpha,
                                   ctypes.byref(o), _ptr(dY), ctypes.byref(Z), _ptr(h),
                                   _ptr(w), _ptr(attr), _ptr(rep), ctypes.byref(b)),
           "interp_gradient")
    out = {"dY": dY, "Z": Z.value, "h": h, "attr": attr, "rep": rep,
           "box": Box(b.y_min, b.width, b.b, b.inv_b, b.n_int, b.p, b.delta)}
    if want_grids:
        out["w"] = w.reshape((s + 1,) + ((n,) if s == 1 else (n, n)))
    return out


def fft(x, inverse: bool = False):
    """Radix-2 complex FFT of the oracle (forward sign -1, inverse unscaled)."""
    lib = _load()
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real.copy())
    im = np.ascontiguousarray(x.imag.copy())
    _check(lib.orc_fft(len(x), _ptr(re), _ptr(im), 1 if inverse else -1), "fft")
    return re + 1j * im


def alpha_at(sched: Schedule, it: int) -> float:
    s = sched._c()
    return float(_load().orc_alpha(ctypes.byref(s), it))


def step(Y, uY, gains, dY, sched: Schedule, it: int):
    """One optimizer update in place on float64 arrays (Y, uY, gains)."""
    lib = _load()
    for a in (Y, uY, gains):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    dY = np.ascontiguousarray(dY, dtype=np.float64)
    N, s = Y.shape if Y.ndim == 2 else (Y.shape[0], 1)
    sc = sched._c()
    _check(lib.orc_step(N, s, _ptr(Y), _ptr(uY), _ptr(gains), _ptr(dY), ctypes.byref(sc),
                        it), "step")


def run(Y0, P, sched: Schedule = Schedule(), opts: InterpOptions = InterpOptions()):
    """Full optimisation from Y0; returns (Y_final, KL_final)."""
    lib = _load()
    Y = _Y(Y0).copy()
    N, s = Y.shape
    rp, col, val = _csr(P)
    o = opts._c()
    sc = sched._c()
    klv = ctypes.c_double()
    _check(lib.orc_run(N, s, _ptr(Y), _ptr(rp), _ptr(col), _ptr(val), ctypes.byref(o),
                       ctypes.byref(sc), ctypes.byref(klv)), "run")
    return Y, klv.value
