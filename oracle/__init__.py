"""FP64 CPU oracle for the fastCAT CBCT hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is independent of the CUDA library:
it neither imports nor links it, and the library never calls it.

The numerical work lives in ``fastcat_oracle.c`` (projection, energy sum,
blur, FDK; double precision) and ``noise_oracle.c`` (Poisson noise in binary32,
the precision in which the GPU takes the same integer decision).  This module
compiles them with gcc on first use and wraps them with numpy arrays.  HU and
CNR (Sec. II.G, CNR equation) are plain numpy here.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRCS = [os.path.join(_HERE, f) for f in ("fastcat_oracle.c", "noise_oracle.c")]
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp] + _SRCS + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcGeom(ctypes.Structure):
    _fields_ = [("sad", ctypes.c_double), ("sdd", ctypes.c_double),
                ("n_u", ctypes.c_int32), ("n_v", ctypes.c_int32),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("n_angles", ctypes.c_int32),
                ("theta0", ctypes.c_double), ("arc", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


def _geom(g):
    return OrcGeom(g.sad, g.sdd, g.n_u, g.n_v, g.du, g.dv, g.n_angles, g.theta0,
                   g.arc, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_L = ctypes.c_long


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            gp = ctypes.POINTER(OrcGeom)
            sig = {
                "orc_siddon": (_D, [gp, _P, _I, _P, _P, _P]),
                "orc_ray_lengths": (_D, [gp, _P, _I, _I, _I, _I, _P]),
                "orc_energy_sum": (_D, [_I, _I, _P, _P, _P, _P]),
                "orc_project_T": (None, [gp, _P, _I, _I, _P, _P, _P, _I, _I, _P]),
                "orc_rays": (None, [gp, _P, _I, _I, _P, _P, _P, _L, _P, _P, _P]),
                "orc_gauss_blur": (None, [_P, _I, _I, _I, _D, _P]),
                "orc_intensity": (None, [_P, _I, _I, _I, _D, _D, _D, _D, _P]),
                "orc_fdk_weight": (None, [gp, _P, _I, _D, _P]),
                "orc_ramp_filter": (None, [_P, _I, _I, _D, _P]),
                "orc_backproject": (None, [gp, _P, _P]),
                "orc_fdk": (None, [gp, _P, _D, _P]),
                "orc_omp_threads": (_I, []),
                "orc_philox4x32_10": (None, [_P, _P, _P]),
                "orc_log_f32": (ctypes.c_float, [ctypes.c_float]),
                "orc_exp_f32": (ctypes.c_float, [ctypes.c_float]),
                "orc_poisson_one": (ctypes.c_float, [ctypes.c_float, ctypes.c_uint32,
                                                     ctypes.c_uint32, ctypes.c_uint32,
                                                     ctypes.c_uint64]),
                "orc_poisson": (None, [_P, _I, _I, _I, _I, ctypes.c_uint64, _P]),
                "orc_path_matrix": (ctypes.c_int64, [gp, _I, _I, _P, _P, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def threads():
    """OpenMP threads the oracle's parallel loops use."""
    return lib().orc_omp_threads()


# ---------------------------------------------------------------- projection
def siddon(g, labels, n_mat, S, P):
    """Per-material path lengths (cm) of the segment S -> P (Siddon 1985)."""
    L = np.zeros(n_mat)
    lab = _c(labels, np.uint8)
    tot = lib().orc_siddon(ctypes.byref(_geom(g)), _ptr(lab), n_mat,
                           _ptr(_c(S, np.float64)), _ptr(_c(P, np.float64)), _ptr(L))
    return L, tot


def ray_lengths(g, labels, n_mat, k, iv, iu):
    """Path lengths of pixel ray (k, iv, iu); returns (L[n_mat], total)."""
    L = np.zeros(n_mat)
    lab = _c(labels, np.uint8)
    tot = lib().orc_ray_lengths(ctypes.byref(_geom(g)), _ptr(lab), n_mat, k, iv, iu, _ptr(L))
    return L, tot


def energy_sum(w, D, mu, L):
    """T = sum_E w D exp(-sum_m mu L) / sum_E w D (Sec. II.F, I_f equation)."""
    mu = _c(mu, np.float64)
    n_e, n_mat = mu.shape
    return lib().orc_energy_sum(n_e, n_mat, _ptr(_c(w, np.float64)), _ptr(_c(D, np.float64)),
                                _ptr(mu), _ptr(_c(L, np.float64)))


def project_T(g, labels, w, D, mu, a0=0, na=None):
    """Flood-normalised primary signal T[k][iv][iu] for angles a0 .. a0+na-1."""
    na = g.n_angles - a0 if na is None else na
    mu = _c(mu, np.float64)
    n_e, n_mat = mu.shape
    T = np.empty((na, g.n_v, g.n_u))
    lab = _c(labels, np.uint8)
    lib().orc_project_T(ctypes.byref(_geom(g)), _ptr(lab), n_mat, n_e,
                        _ptr(_c(w, np.float64)), _ptr(_c(D, np.float64)), _ptr(mu),
                        a0, na, _ptr(T))
    return T


def rays(g, labels, w, D, mu, ray_idx):
    """L[n][n_mat] and T[n] of sampled rays ray_idx[n] = (k, iv, iu)."""
    mu = _c(mu, np.float64)
    n_e, n_mat = mu.shape
    r = _c(ray_idx, np.int32).reshape(-1, 3)
    L = np.empty((len(r), n_mat))
    T = np.empty(len(r))
    lab = _c(labels, np.uint8)
    lib().orc_rays(ctypes.byref(_geom(g)), _ptr(lab), n_mat, n_e,
                   _ptr(_c(w, np.float64)), _ptr(_c(D, np.float64)), _ptr(mu),
                   len(r), _ptr(r), _ptr(L), _ptr(T))
    return L, T


def path_matrix(g, a0=0, na=None):
    """CSR (rowptr, col, val) of the ray x voxel path lengths (cm) of angles
    a0 .. a0+na-1; rows in [k][iv][iu] order, columns flat [z][y][x]."""
    na = g.n_angles - a0 if na is None else na
    nrays = na * g.n_v * g.n_u
    cap = g.nx + g.ny + g.nz + 2
    rowptr = np.zeros(nrays + 1, np.int64)
    col = np.zeros(nrays * cap, np.int64)
    val = np.zeros(nrays * cap)
    nnz = lib().orc_path_matrix(ctypes.byref(_geom(g)), a0, na, _ptr(rowptr), _ptr(col), _ptr(val))
    return rowptr, col[:nnz].copy(), val[:nnz].copy()


# ---------------------------------------------------------------- detector
def gauss_blur(img, sigma):
    """Separable sampled-Gaussian blur, clamp-to-edge, over [..., nv, nu]."""
    a = _c(img, np.float64)
    shp = a.shape
    a3 = a.reshape(-1, shp[-2], shp[-1])
    out = np.empty_like(a3)
    lib().orc_gauss_blur(_ptr(a3), a3.shape[0], shp[-2], shp[-1], float(sigma), _ptr(out))
    return out.reshape(shp)


def intensity(T, sig_psf, sig_sc, spr, n0):
    """I = N0 (G_psf (x) T + SPR G_scatter (x) T)."""
    a = _c(T, np.float64)
    shp = a.shape
    a3 = a.reshape(-1, shp[-2], shp[-1])
    out = np.empty_like(a3)
    lib().orc_intensity(_ptr(a3), a3.shape[0], shp[-2], shp[-1], float(sig_psf),
                        float(sig_sc), float(spr), float(n0), _ptr(out))
    return out.reshape(shp)


def counts_noise_before_psf(T, sig_psf, sig_sc, spr, n0, seed=None, k0=0):
    """Sec. II.G order: rate lambda = N0 (T + SPR G_sc (x) T) incident on the
    detector, Poisson counts drawn from it (binary32 rates; skipped when
    seed is None), then the optical spread: K = G_psf (x) counts.
    Returns (lambda, K)."""
    lam = intensity(T, 0.0, sig_sc, spr, n0)
    k = lam if seed is None else poisson(lam, seed, k0).astype(np.float64)
    return lam, gauss_blur(k, sig_psf)


def i_flood(n0, spr):
    """Flood intensity: T = 1 everywhere, both kernels sum to one."""
    return n0 * (1.0 + spr)


# ---------------------------------------------------------------- noise (binary32)
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def log_f32(x):
    return lib().orc_log_f32(float(x))


def exp_f32(x):
    return lib().orc_exp_f32(float(x))


def poisson(lam, seed, k0=0):
    """Counts ~ Poisson(lam[k][iv][iu]) with counters (iu, iv, k0 + k, j)."""
    a = _c(lam, np.float32)
    shp = a.shape
    a3 = a.reshape(-1, shp[-2], shp[-1])
    out = np.empty_like(a3)
    lib().orc_poisson(_ptr(a3), a3.shape[0], shp[-2], shp[-1], int(k0), int(seed), _ptr(out))
    return out.reshape(shp)


# ---------------------------------------------------------------- FDK
def fdk_weight(g, counts, flood):
    c = _c(counts, np.float64)
    q = np.empty_like(c)
    lib().orc_fdk_weight(ctypes.byref(_geom(g)), _ptr(c), c.shape[0], float(flood), _ptr(q))
    return q


def ramp_filter(q, tau):
    a = _c(q, np.float64)
    nu = a.shape[-1]
    out = np.empty_like(a)
    lib().orc_ramp_filter(_ptr(a), a.size // nu, nu, float(tau), _ptr(out))
    return out


def backproject(g, f):
    a = _c(f, np.float64)
    vol = np.empty((g.nz, g.ny, g.nx))
    lib().orc_backproject(ctypes.byref(_geom(g)), _ptr(a), _ptr(vol))
    return vol


def fdk(g, counts, flood):
    """FDK reconstruction mu[z][y][x] (1/cm) of counts[k][iv][iu]."""
    c = _c(counts, np.float64)
    vol = np.empty((g.nz, g.ny, g.nx))
    lib().orc_fdk(ctypes.byref(_geom(g)), _ptr(c), float(flood), _ptr(vol))
    return vol


def hu(vol, water_mask):
    """HU = 1000 (mu - mu_w) / mu_w, mu_w the mean over the water region."""
    mu_w = float(np.mean(vol[water_mask]))
    return 1000.0 * (vol - mu_w) / mu_w, mu_w


def cnr(hu_img, water_mask, roi_mask):
    """CNR = |HU_w - HU_roi| / sqrt(sigma_w^2 + sigma_roi^2) (Sec. II.G)."""
    a, b = hu_img[water_mask], hu_img[roi_mask]
    return abs(a.mean() - b.mean()) / math.sqrt(a.var() + b.var())
