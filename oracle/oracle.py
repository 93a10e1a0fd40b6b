"""FP64 CPU oracle for the joint-acceleration bilateral filter.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product library never loads
it.  This wrapper compiles ``bf_oracle.c`` with gcc into ``oracle/_build`` and
exposes numpy-level functions:

* ``exact_bf``       -- O1, Eq. (1) by brute force;
* ``approx_direct``  -- O2, Eq. (1) with the approximated kernels (Eqs. (30), (33));
* ``approx_fast``    -- O3, the paper's algorithm (Eqs. (34)-(36), App. A boxes);
* ``approx3d_direct`` / ``approx3d_fast`` -- O2 / O3 of the 3-D form (Sec. IV-D: P = T_r, the range box
  applied over Z intensity slices by dimension promotion, Eqs. (2), (28)-(29), (35)-(36));
* ``approx3dh_direct`` / ``approx3dh_fast`` -- the same with a Haar series in range (best N-term Haar
  expansion of the truncated range kernel on the slice axis; each term is boxes along z);
* ``range_coeffs``, ``haar1d``, ``plan_info`` -- coefficient and selection steps.

Every function follows the paper step by step; the C file header lists the
passages and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")

GAUSSIAN, EXPONENTIAL, BOX = 0, 1, 2
TRUNCATED_MIN_PERIOD, UNTRUNCATED_FULL, PAPER_3D, PAPER_TRUNCATED = 0, 1, 2, 3

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        d, i = C.c_double, C.c_int
        pd, pi = C.POINTER(C.c_double), C.POINTER(C.c_int)
        lib.orc_range_coeffs.argtypes = [i, d, d, d, i, pd]
        lib.orc_haar1d.argtypes = [i, d, d, i, pd, pi, pi]
        lib.orc_haar_eval.argtypes = [i, i, d, d]
        lib.orc_haar_eval.restype = d
        lib.orc_haar_levels.argtypes = [d]
        lib.orc_default_tr.argtypes = [i, d]
        lib.orc_default_tr.restype = d
        lib.orc_period.argtypes = [i, d, d]
        lib.orc_period.restype = d
        lib.orc_select_range.argtypes = [pd, i, i, pi, pd]
        lib.orc_plan_info.argtypes = [i, d, i, i, i, d, d, i, i, d, pi, pd, pi, pd, pi, pd, pd, i]
        lib.orc_exact_bf.argtypes = [pd, i, i, i, d, i, i, d, pd, pi, i, i]
        common = [pd, i, i, i, d, i, i, i, d, d, i, i, d, pd, pi, i]
        lib.orc_approx_direct.argtypes = common
        lib.orc_approx_fast.argtypes = common + [pd]
        lib.orc_box_count.argtypes = [i, d, i, i, i, d, d, i, i, d]
        lib.orc_approx_direct_at.argtypes = [pd, i, i, i, d, i, i, i, d, d, i, i, d, pi, i, pd, i]
        lib.orc_exact_bf_lut.argtypes = [pd, i, i, i, d, i, i, d, i, d, pd, i]
        lib.orc_rect_int_exp.argtypes = [d, d, d, d, d]
        lib.orc_rect_int_exp.restype = d
        lib.orc_haar2d_exp.argtypes = [d, d, i, pd, i]
        lib.orc_approx3d_direct.argtypes = [pd, i, i, i, d, i, i, i, d, d, i, i, d, i, pd, pi, i, pd]
        lib.orc_approx3d_direct_at.argtypes = [pd, i, i, i, d, i, i, i, d, d, i, i, d, i, pi, i, pd, pd, i]
        lib.orc_approx3d_fast.argtypes = [pd, i, i, i, d, i, i, i, d, d, i, i, d, i, pd, pi, i, pd]
        lib.orc_z_bins.argtypes = [d, i, d, pd, i, pi, pi]
        lib.orc_zhaar_info.argtypes = [i, d, d, i, i, d, pi, pi, pi, pd, pd, i]
        lib.orc_approx3dh_direct.argtypes = [pd, i, i, i, d, i, i, i, d, d, i, i, d, pi, i, pd, pd, i]
        lib.orc_approx3dh_fast.argtypes = [pd, i, i, i, d, i, i, i, d, d, i, i, d, pd, pi, i]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def max_threads() -> int:
    return int(_load().orc_max_threads())


@dataclass(frozen=True)
class Desc:
    """Filter parameters (mirrors the product's plan descriptor, defined separately)."""
    spatial: int = GAUSSIAN
    sigma_s: float = 4.0
    radius: int = 0          # 0 -> round(3 sigma_s)
    ns_terms: int = 5
    range: int = GAUSSIAN
    sigma_r: float = 0.1
    t_r: float = 0.0         # 0 -> default truncation point
    nr_terms: int = 8
    policy: int = TRUNCATED_MIN_PERIOD
    data_range: float = 1.0

    def args(self):
        return (self.spatial, self.sigma_s, self.radius, self.ns_terms, self.range,
                self.sigma_r, self.t_r, self.nr_terms, self.policy, self.data_range)


def range_coeffs(kind: int, sigma_r: float, t_r: float, period: float, ncand: int) -> np.ndarray:
    a = np.zeros(ncand)
    st = _load().orc_range_coeffs(kind, sigma_r, t_r, period, ncand, _dp(a))
    if st:
        raise ValueError("orc_range_coeffs status %d" % st)
    return a


def haar_levels(T: float) -> int:
    return int(_load().orc_haar_levels(T))


def haar1d(kind: int, sigma_s: float, T: float, J: int | None = None):
    """1-D Haar coefficients in dictionary order; returns (c, level, k)."""
    if J is None:
        J = haar_levels(T)
    n = 1 << (J + 1)
    c = np.zeros(n)
    lev = np.zeros(n, dtype=np.int32)
    kk = np.zeros(n, dtype=np.int32)
    st = _load().orc_haar1d(kind, sigma_s, T, J, _dp(c), _ip(lev), _ip(kk))
    if st:
        raise ValueError("orc_haar1d status %d" % st)
    return c, lev, kk


def rect_int_exp(sigma: float, x0: float, x1: float, y0: float, y1: float) -> float:
    """Integral of exp(-sqrt(x^2 + y^2) / sigma) over [x0, x1] x [y0, y1] (signed triangle fan)."""
    return float(_load().orc_rect_int_exp(sigma, x0, x1, y0, y1))


def haar2d_exp(sigma_s: float, T: float, J: int | None = None, threads: int = 1) -> np.ndarray:
    """2-D Haar coefficients of the radial exponential kernel: c[i2, i1] (i1 along x, i2 along y),
    indices in the 1-D dictionary order of haar1d."""
    if J is None:
        J = haar_levels(T)
    n = 1 << (J + 1)
    c = np.zeros((n, n))
    st = _load().orc_haar2d_exp(sigma_s, T, J, _dp(c), threads)
    if st:
        raise ValueError("orc_haar2d_exp status %d" % st)
    return c


def haar_eval(lev: int, k: int, T: float, x: float) -> float:
    return float(_load().orc_haar_eval(lev, k, T, x))


def default_tr(kind: int, sigma_r: float) -> float:
    return float(_load().orc_default_tr(kind, sigma_r))


def period(policy: int, t_r: float, data_range: float = 1.0) -> float:
    return float(_load().orc_period(policy, t_r, data_range))


def select_range(a: np.ndarray, nr: int):
    a = np.ascontiguousarray(a, dtype=np.float64)
    ks = np.zeros(nr, dtype=np.int32)
    aks = np.zeros(nr)
    n = _load().orc_select_range(_dp(a), len(a), nr, _ip(ks), _dp(aks))
    return ks[:n].copy(), aks[:n].copy()


@dataclass
class PlanInfo:
    R: int
    J: int
    Ts: float
    Tr: float
    P: float
    den_eps: float
    ks: np.ndarray
    ak: np.ndarray
    terms: np.ndarray      # (ns, 4): lev1, k1, lev2, k2  (first factor: column offset)
    term_c: np.ndarray
    tie_split: bool
    Ks: np.ndarray         # (2R+1, 2R+1) indexed [dy+R, dx+R] = K~_s(dx, dy)


def plan_info(desc: Desc) -> PlanInfo:
    lib = _load()
    R = int(np.floor(3.0 * desc.sigma_s + 0.5)) if desc.radius == 0 else desc.radius
    w = 2 * R + 1
    ints = np.zeros(5, dtype=np.int32)
    dbl = np.zeros(4)
    ks = np.zeros(desc.nr_terms, dtype=np.int32)
    ak = np.zeros(desc.nr_terms)
    tid = np.zeros(4 * desc.ns_terms, dtype=np.int32)
    tc = np.zeros(desc.ns_terms)
    Ks = np.zeros(w * w)
    st = lib.orc_plan_info(*desc.args(), _ip(ints), _dp(dbl), _ip(ks), _dp(ak), _ip(tid), _dp(tc), _dp(Ks), w * w)
    if st:
        raise ValueError("orc_plan_info status %d" % st)
    nr, ns = int(ints[2]), int(ints[3])
    return PlanInfo(R=int(ints[0]), J=int(ints[1]), Ts=float(dbl[0]), Tr=float(dbl[1]), P=float(dbl[2]),
                    den_eps=float(dbl[3]), ks=ks[:nr].copy(), ak=ak[:nr].copy(),
                    terms=tid[:4 * ns].reshape(ns, 4).copy(), term_c=tc[:ns].copy(),
                    tie_split=bool(ints[4]), Ks=Ks.reshape(w, w))


def _img(I):
    I = np.ascontiguousarray(I, dtype=np.float64)
    if I.ndim != 2:
        raise ValueError("image must be 2-D")
    return I


def exact_bf(I, desc: Desc, rows=None, threads: int = 1) -> np.ndarray:
    """O1: Eq. (1), Gaussian/box spatial kernel on the (2R+1)^2 square, untruncated range kernel."""
    I = _img(I)
    H, W = I.shape
    if rows is None:
        out = np.zeros((H, W))
        rp, nr = None, 0
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.zeros((len(rows), W))
        rp, nr = _ip(rows), len(rows)
    st = _load().orc_exact_bf(_dp(I), H, W, desc.spatial, desc.sigma_s, desc.radius, desc.range,
                              desc.sigma_r, _dp(out), rp, nr, threads)
    if st:
        raise ValueError("orc_exact_bf status %d" % st)
    return out


def exact_bf_lut(I, desc: Desc, levels: int, data_range: float = 1.0, threads: int = 1) -> np.ndarray:
    """Eq. (1) with the range kernel read from a `levels`-entry table over [0, data_range] (nearest entry,
    chosen in fp32): the look-up-table brute-force baseline."""
    I = _img(I)
    H, W = I.shape
    out = np.zeros((H, W))
    st = _load().orc_exact_bf_lut(_dp(I), H, W, desc.spatial, desc.sigma_s, desc.radius, desc.range, desc.sigma_r,
                                  levels, data_range, _dp(out), threads)
    if st:
        raise ValueError("orc_exact_bf_lut status %d" % st)
    return out


def approx_direct(I, desc: Desc, threads: int = 1):
    """O2: returns (output, number of pixels where the denominator guard fired)."""
    I = _img(I)
    H, W = I.shape
    out = np.zeros((H, W))
    nd = np.zeros(1, dtype=np.int32)
    st = _load().orc_approx_direct(_dp(I), H, W, *desc.args(), _dp(out), _ip(nd), threads)
    if st:
        raise ValueError("orc_approx_direct status %d" % st)
    return out, int(nd[0])


def approx_fast(I, desc: Desc, threads: int = 1, return_den: bool = False):
    """O3: returns (output, number of pixels where the denominator guard fired)
    [, denominator of Eq. (1) per pixel if return_den]."""
    I = _img(I)
    H, W = I.shape
    out = np.zeros((H, W))
    den = np.zeros((H, W)) if return_den else None
    nd = np.zeros(1, dtype=np.int32)
    st = _load().orc_approx_fast(_dp(I), H, W, *desc.args(), _dp(out), _ip(nd), threads,
                                 _dp(den) if return_den else None)
    if st:
        raise ValueError("orc_approx_fast status %d" % st)
    if return_den:
        return out, int(nd[0]), den
    return out, int(nd[0])


def approx_direct_at(I, desc: Desc, pts, threads: int = 1) -> np.ndarray:
    """O2 at the given (row, col) pixels only."""
    I = _img(I)
    H, W = I.shape
    pts = np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(len(pts))
    st = _load().orc_approx_direct_at(_dp(I), H, W, *desc.args(), _ip(pts), len(pts), _dp(out), threads)
    if st:
        raise ValueError("orc_approx_direct_at status %d" % st)
    return out


def box_count(desc: Desc) -> int:
    return int(_load().orc_box_count(*desc.args()))


def approx3d_direct(I, desc: Desc, zbins: int = 256, threads: int = 1, return_den: bool = False):
    """O2-3D (desc.policy must be PAPER_3D): returns (output, guard count)[, denominator]."""
    I = _img(I)
    H, W = I.shape
    out = np.zeros((H, W))
    den = np.zeros((H, W)) if return_den else None
    nd = np.zeros(1, dtype=np.int32)
    st = _load().orc_approx3d_direct(_dp(I), H, W, *desc.args(), zbins, _dp(out), _ip(nd), threads,
                                     _dp(den) if return_den else None)
    if st:
        raise ValueError("orc_approx3d_direct status %d" % st)
    if return_den:
        return out, int(nd[0]), den
    return out, int(nd[0])


def approx3d_direct_at(I, desc: Desc, pts, zbins: int = 256, threads: int = 1):
    """O2-3D at the given (row, col) pixels: (output, denominator) arrays."""
    I = _img(I)
    H, W = I.shape
    pts = np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(len(pts))
    den = np.zeros(len(pts))
    st = _load().orc_approx3d_direct_at(_dp(I), H, W, *desc.args(), zbins, _ip(pts), len(pts), _dp(out), _dp(den),
                                        threads)
    if st:
        raise ValueError("orc_approx3d_direct_at status %d" % st)
    return out, den


def approx3d_fast(I, desc: Desc, zbins: int = 256, threads: int = 1, return_den: bool = False):
    """O3-3D (desc.policy must be PAPER_3D): returns (output, guard count)[, denominator]."""
    I = _img(I)
    H, W = I.shape
    out = np.zeros((H, W))
    den = np.zeros((H, W)) if return_den else None
    nd = np.zeros(1, dtype=np.int32)
    st = _load().orc_approx3d_fast(_dp(I), H, W, *desc.args(), zbins, _dp(out), _ip(nd), threads,
                                   _dp(den) if return_den else None)
    if st:
        raise ValueError("orc_approx3d_fast status %d" % st)
    if return_den:
        return out, int(nd[0]), den
    return out, int(nd[0])


def z_bins(I, t_r: float, zbins: int = 256, data_range: float = 1.0):
    """(slice index of each intensity, R_z) on the z axis of the 3-D form; t_r already resolved."""
    v = np.ascontiguousarray(np.ravel(I), dtype=np.float64)
    out = np.zeros(len(v), dtype=np.int32)
    rz = np.zeros(1, dtype=np.int32)
    st = _load().orc_z_bins(t_r, zbins, data_range, _dp(v), len(v), _ip(out), _ip(rz))
    if st:
        raise ValueError("orc_z_bins status %d" % st)
    return out.reshape(np.shape(I)), int(rz[0])


def _hargs(desc: Desc, zbins: int, data_range: float):
    return (desc.spatial, desc.sigma_s, desc.radius, desc.ns_terms, desc.range, desc.sigma_r, desc.t_r,
            desc.nr_terms, zbins, data_range)


@dataclass
class ZHaarInfo:
    Rz: int
    Jz: int
    lev: np.ndarray
    k: np.ndarray
    c: np.ndarray
    w: np.ndarray          # K~_r at slice offsets d = n(x) - n(y), index d + Rz


def zhaar_info(desc: Desc, zbins: int = 256, data_range: float = 1.0) -> ZHaarInfo:
    lib = _load()
    ints = np.zeros(3, dtype=np.int32)
    n = desc.nr_terms
    lev, kk, c = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32), np.zeros(n)
    w = np.zeros(2 * 4096 + 1)
    st = lib.orc_zhaar_info(desc.range, desc.sigma_r, desc.t_r, n, zbins, data_range, _ip(ints), _ip(lev), _ip(kk),
                            _dp(c), _dp(w), len(w))
    if st:
        raise ValueError("orc_zhaar_info status %d" % st)
    Rz, Jz, m = int(ints[0]), int(ints[1]), int(ints[2])
    return ZHaarInfo(Rz, Jz, lev[:m].copy(), kk[:m].copy(), c[:m].copy(), w[:2 * Rz + 1].copy())


def approx3dh_direct(I, desc: Desc, zbins: int = 256, pts=None, threads: int = 1, data_range: float = 1.0):
    """O2-3D with the Haar range series: (output, denominator), over the image or at (row, col) pts."""
    I = _img(I)
    H, W = I.shape
    if pts is None:
        out, den, pp, n = np.zeros((H, W)), np.zeros((H, W)), None, 0
    else:
        pts = np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 2)
        out, den, pp, n = np.zeros(len(pts)), np.zeros(len(pts)), _ip(pts), len(pts)
    st = _load().orc_approx3dh_direct(_dp(I), H, W, *_hargs(desc, zbins, data_range), pp, n, _dp(out), _dp(den),
                                      threads)
    if st:
        raise ValueError("orc_approx3dh_direct status %d" % st)
    return out, den


def approx3dh_fast(I, desc: Desc, zbins: int = 256, threads: int = 1, data_range: float = 1.0):
    """O3-3D with the Haar range series (per-slice tables, z table, boxes along z): (output, guard count)."""
    I = _img(I)
    H, W = I.shape
    out = np.zeros((H, W))
    nd = np.zeros(1, dtype=np.int32)
    st = _load().orc_approx3dh_fast(_dp(I), H, W, *_hargs(desc, zbins, data_range), _dp(out), _ip(nd), threads)
    if st:
        raise ValueError("orc_approx3dh_fast status %d" % st)
    return out, int(nd[0])
