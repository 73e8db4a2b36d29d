"""Thin Python binding of libfastcat (C ABI in include/fastcat.h).

Argument marshalling only: every function forwards to the C entry point of
the same name; all computation happens in the library's CUDA kernels.  There
is no fallback -- if ``lib/libfastcat.so`` is missing, loading raises.

Device buffers are passed as torch CUDA tensors (their data pointers), host
buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libfastcat.so")

FC_OK, FC_EINVAL, FC_ENOMEM, FC_ECUDA, FC_ESTATE, FC_ETIMEOUT = 0, -1, -2, -3, -4, -5
FC_HOST, FC_DEVICE, FC_HOST_ASYNC = 0, 1, 2
FC_OUT_NONE, FC_OUT_PRIMARY, FC_OUT_INTENSITY, FC_OUT_COUNTS = 0, 1, 2, 3
FC_NOISE_AFTER_BLUR, FC_NOISE_BEFORE_PSF = 0, 1
FC_BP_AUTO, FC_BP_CHUNKED, FC_BP_CHUNKED_DENSE, FC_BP_SLAB, FC_BP_SLAB_SYM, FC_BP_CHUNKED_SYM = 0, 1, 2, 3, 4, 5
FC_FAULT_NONE, FC_FAULT_ALLOC, FC_FAULT_BLUR_TIMEOUT = 0, 1, 2
FC_BP_NAMES = {FC_BP_CHUNKED: "chunked", FC_BP_CHUNKED_DENSE: "chunked_dense", FC_BP_SLAB: "slab",
               FC_BP_SLAB_SYM: "slab_sym", FC_BP_CHUNKED_SYM: "chunked_sym"}
FC_MAX_MATERIALS, FC_MAX_BINS = 8, 256

# every entry point declared in include/fastcat.h
ENTRY_POINTS = ("fc_create", "fc_destroy", "fc_last_error", "fc_set_geometry", "fc_set_phantom",
                "fc_set_spectrum_detector", "fc_project", "fc_reconstruct", "fc_set_water_roi",
                "fc_poisson", "fc_project_lengths", "fc_profile_enable", "fc_profile_read",
                "fc_detector_blur_static", "fc_surrogate_init", "fc_surrogate_train",
                "fc_surrogate_grad", "fc_surrogate_get", "fc_surrogate_set", "fc_surrogate_eval",
                "fc_energy_sum_lengths", "fc_cnr_grad", "fc_surrogate_project",
                "fc_dose_estimate", "fc_fluence_for_dose", "fc_set_noise_order",
                "fc_set_energy_groups", "fc_deconvolve_rl", "fc_detector_mtf",
                "fc_set_backprojector", "fc_backprojector_in_use", "fc_inject_fault",
                "fc_surrogate_guard", "fc_surrogate_sigma", "fc_wait_outputs")
FC_STATIC_SCRATCH_FLOATS = 8 << 20
FC_SURROGATE_PARAMS = 34305
FC_SURROGATE_STATE = 34305 + 52 + 2 * 34305 + 1
FC_K_NAMES = ("project", "blur_rows", "blur_cols", "fdk_filter", "backproject", "hu", "lengths",
              "noise", "surrogate_eval", "surrogate_train", "energy_sum", "dose", "group_blur",
              "deconv", "blur_band")


class FastcatError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fastcat error %d: %s" % (code, msg))
        self.code = code


class fc_geometry(ctypes.Structure):
    _fields_ = [("sad_cm", ctypes.c_double), ("sdd_cm", ctypes.c_double),
                ("n_u", ctypes.c_int32), ("n_v", ctypes.c_int32),
                ("du_cm", ctypes.c_double), ("dv_cm", ctypes.c_double),
                ("n_angles", ctypes.c_int32),
                ("theta0_rad", ctypes.c_double), ("arc_rad", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx_cm", ctypes.c_double), ("dy_cm", ctypes.c_double), ("dz_cm", ctypes.c_double)]


class fc_cnr_roi(ctypes.Structure):
    _fields_ = [("cx_cm", ctypes.c_double), ("cy_cm", ctypes.c_double),
                ("radius_cm", ctypes.c_double)]


class fc_spectrum_detector(ctypes.Structure):
    _fields_ = [("n_e", ctypes.c_int32), ("n_mat", ctypes.c_int32),
                ("w", ctypes.c_void_p), ("d", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("psf_sigma_px", ctypes.c_double), ("scatter_sigma_px", ctypes.c_double),
                ("spr", ctypes.c_double), ("n0", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("noise", ctypes.c_int32)]


class fc_energy_groups(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int32), ("bin_end", ctypes.c_void_p),
                ("psf_sigma_px", ctypes.c_void_p), ("scatter_amp", ctypes.c_void_p),
                ("scatter_a_cm", ctypes.c_void_p), ("scatter_b", ctypes.c_void_p)]


_lib = None


def load():
    """Load libfastcat.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfastcat.so not found at %s; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, I = ctypes.c_void_p, ctypes.c_int
    sig = {
        "fc_create": (I, [ctypes.POINTER(P), I]),
        "fc_destroy": (I, [P]),
        "fc_last_error": (ctypes.c_char_p, []),
        "fc_set_geometry": (I, [P, ctypes.POINTER(fc_geometry)]),
        "fc_set_phantom": (I, [P, P, I, I, P]),
        "fc_set_spectrum_detector": (I, [P, ctypes.POINTER(fc_spectrum_detector)]),
        "fc_project": (I, [P, I, I, I, P, I, P]),
        "fc_reconstruct": (I, [P, P, I, P, P, I, P]),
        "fc_wait_outputs": (I, [P]),
        "fc_set_water_roi": (I, [P, ctypes.c_double, ctypes.c_double]),
        "fc_poisson": (I, [P, P, I, I, I, I, ctypes.c_uint64, P]),
        "fc_project_lengths": (I, [P, I, I, P, P]),
        "fc_profile_enable": (I, [P, I]),
        "fc_profile_read": (I, [P, P, P]),
        "fc_detector_blur_static": (I, [P, P, I, I, I, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, P]),
        "fc_surrogate_init": (I, [P, ctypes.c_uint64]),
        "fc_surrogate_train": (I, [P, P, P, ctypes.c_int64, I, I, ctypes.c_float, ctypes.c_uint64,
                                   P, P]),
        "fc_surrogate_grad": (I, [P, P, P, ctypes.c_int64, P, P, P]),
        "fc_surrogate_get": (I, [P, P]),
        "fc_surrogate_set": (I, [P, P]),
        "fc_surrogate_eval": (I, [P, P, ctypes.c_int64, P, P, P]),
        "fc_energy_sum_lengths": (I, [P, P, ctypes.c_int64, P, P]),
        "fc_cnr_grad": (I, [P, P, P, P, P, P, I, P, P, P, P, P, P]),
        "fc_surrogate_project": (I, [P, I, I, P, I, P]),
        "fc_dose_estimate": (I, [P, I, I, P, P, P, P, P, I, P]),
        "fc_fluence_for_dose": (I, [P, ctypes.c_double, ctypes.c_double, P]),
        "fc_set_noise_order": (I, [P, I]),
        "fc_set_energy_groups": (I, [P, ctypes.POINTER(fc_energy_groups)]),
        "fc_deconvolve_rl": (I, [P, I, I, ctypes.c_double, I, P, I, P]),
        "fc_detector_mtf": (I, [P, ctypes.c_double, ctypes.c_double, I, P, P, I, P]),
        "fc_set_backprojector": (I, [P, I]),
        "fc_backprojector_in_use": (I, [P, ctypes.POINTER(I)]),
        "fc_inject_fault": (I, [I, ctypes.c_int64]),
        "fc_surrogate_guard": (I, [P, P, P, ctypes.c_int64, ctypes.c_double, P, P]),
        "fc_surrogate_sigma": (I, [P, P, ctypes.c_int64, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != FC_OK:
        raise FastcatError(rc, load().fc_last_error().decode())
    return rc


def _ptr(x):
    """(pointer, where) of a torch tensor (device) or numpy array (host)."""
    if x is None:
        return None, FC_HOST
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data, FC_HOST
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr(), (FC_DEVICE if x.is_cuda else FC_HOST)
    raise TypeError("expected a numpy array or torch tensor, got %r" % type(x))


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_geometry(g):
    """fc_geometry from any object with the workloads.Geometry fields."""
    return fc_geometry(g.sad, g.sdd, g.n_u, g.n_v, g.du, g.dv, g.n_angles, g.theta0, g.arc,
                       g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)


# ---------------------------------------------------------------- C names
def fc_create(device=0):
    h = ctypes.c_void_p()
    _check(load().fc_create(ctypes.byref(h), device))
    return h


def fc_destroy(h):
    return _check(load().fc_destroy(h))


def fc_last_error():
    return load().fc_last_error().decode()


def fc_set_geometry(h, geom):
    g = geom if isinstance(geom, fc_geometry) else make_geometry(geom)
    return _check(load().fc_set_geometry(h, ctypes.byref(g)))


def fc_set_phantom(h, labels, n_mat, stream=None):
    p, where = _ptr(labels)
    return _check(load().fc_set_phantom(h, p, n_mat, where, _stream(stream)))


def fc_set_spectrum_detector(h, w, d, mu, psf_sigma_px, scatter_sigma_px, spr, n0, seed, noise):
    w = np.ascontiguousarray(w, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    mu = np.ascontiguousarray(mu, np.float64)
    s = fc_spectrum_detector(len(w), mu.shape[1], w.ctypes.data, d.ctypes.data, mu.ctypes.data,
                             psf_sigma_px, scatter_sigma_px, spr, n0, seed, int(bool(noise)))
    return _check(load().fc_set_spectrum_detector(h, ctypes.byref(s)))


def fc_project(h, angle_begin, angle_count, out_kind, out=None, stream=None):
    p, where = _ptr(out)
    return _check(load().fc_project(h, angle_begin, angle_count, out_kind, p, where, _stream(stream)))


def fc_reconstruct(h, counts=None, vol_mu=None, vol_hu=None, stream=None, async_host=False):
    """async_host: host outputs (page-locked) are filled asynchronously
    (FC_HOST_ASYNC); read them after fc_wait_outputs(h)."""
    cp, cw = _ptr(counts)
    mp, mw = _ptr(vol_mu)
    hp, hw = _ptr(vol_hu)
    if mp is not None and hp is not None and mw != hw:
        raise ValueError("vol_mu and vol_hu must both be host or both be device buffers")
    ow = mw if mp is not None else hw
    if async_host:
        if ow != FC_HOST:
            raise ValueError("async_host applies to host outputs")
        ow = FC_HOST_ASYNC
    return _check(load().fc_reconstruct(h, cp, cw, mp, hp, ow, _stream(stream)))


def fc_wait_outputs(h):
    return _check(load().fc_wait_outputs(h))


def fc_set_water_roi(h, radius_cm, z_margin):
    return _check(load().fc_set_water_roi(h, radius_cm, z_margin))


def fc_poisson(lam, counts, n_angles, n_v, n_u, angle0, seed, stream=None):
    lp, lw = _ptr(lam)
    cp, cw = _ptr(counts)
    if lw != FC_DEVICE or cw != FC_DEVICE:
        raise ValueError("fc_poisson takes device tensors")
    return _check(load().fc_poisson(lp, cp, n_angles, n_v, n_u, angle0, seed, _stream(stream)))


def fc_project_lengths(h, angle_begin, angle_count, L, stream=None):
    p, where = _ptr(L)
    if where != FC_DEVICE:
        raise ValueError("fc_project_lengths writes a device tensor")
    return _check(load().fc_project_lengths(h, angle_begin, angle_count, p, _stream(stream)))


def fc_dose_estimate(h, angle_begin, angle_count, e_kev, muen_over_mu, rho, d0=None, dp=None,
                     stream=None):
    """D0(E) and Dp (Gy per particle).  With d0/dp omitted, returns host
    arrays; device tensors d0 [n_e] / dp [1] (float64) receive the results on
    `stream` instead."""
    e = np.ascontiguousarray(e_kev, np.float64)
    m = np.ascontiguousarray(muen_over_mu, np.float64)
    r = np.ascontiguousarray(rho, np.float64)
    if d0 is None:
        d0 = np.zeros(len(e), np.float64)
    if dp is None:
        dp = np.zeros(1, np.float64)
    p0, w0 = _ptr(d0)
    p1, w1 = _ptr(dp)
    if w0 != w1:
        raise ValueError("d0 and dp must both be host or both be device buffers")
    _check(load().fc_dose_estimate(h, angle_begin, angle_count, e.ctypes.data, m.ctypes.data,
                                   r.ctypes.data, p0, p1, w0, _stream(stream)))
    return d0, dp


def fc_set_energy_groups(h, bin_end=(), psf_sigma_px=(), scatter_amp=(), scatter_a_cm=(),
                         scatter_b=()):
    """Energy-group detector model; no groups turns it off."""
    be = np.ascontiguousarray(bin_end, np.int32)
    arr = [np.ascontiguousarray(x, np.float64) for x in
           (psf_sigma_px, scatter_amp, scatter_a_cm, scatter_b)]
    n = len(be)
    if any(len(a) != n for a in arr):
        raise ValueError("all group arrays need n_groups entries")
    gs = fc_energy_groups(n, be.ctypes.data, *[a.ctypes.data for a in arr])
    return _check(load().fc_set_energy_groups(h, ctypes.byref(gs)))


def fc_deconvolve_rl(h, angle_begin, angle_count, psf_sigma_px, n_iter, out=None, stream=None):
    """Richardson-Lucy deconvolution of the handle's counts, in place."""
    p, where = _ptr(out)
    return _check(load().fc_deconvolve_rl(h, angle_begin, angle_count, float(psf_sigma_px),
                                          int(n_iter), p, where, _stream(stream)))


def fc_detector_mtf(h, slit_width_mm=0.3, slit_angle_deg=2.5, oversample=4):
    """(frequencies in 1/mm, MTF) of the handle's detector model."""
    cap = 16 * oversample + 1
    f = np.zeros(cap)
    m = np.zeros(cap)
    n = ctypes.c_int()
    _check(load().fc_detector_mtf(h, slit_width_mm, slit_angle_deg, oversample, f.ctypes.data,
                                  m.ctypes.data, cap, ctypes.byref(n)))
    return f[:n.value], m[:n.value]


def fc_set_backprojector(h, variant):
    return _check(load().fc_set_backprojector(h, variant))


def fc_backprojector_in_use(h):
    v = ctypes.c_int(-1)
    _check(load().fc_backprojector_in_use(h, ctypes.byref(v)))
    return v.value


def fc_inject_fault(kind, arg=0):
    return _check(load().fc_inject_fault(kind, arg))


def fc_set_noise_order(h, order):
    return _check(load().fc_set_noise_order(h, order))


def fc_fluence_for_dose(h, dose_gy, dp_gy):
    n0 = ctypes.c_double()
    _check(load().fc_fluence_for_dose(h, dose_gy, dp_gy, ctypes.byref(n0)))
    return n0.value


def fc_profile_enable(h, enable=True):
    return _check(load().fc_profile_enable(h, int(bool(enable))))


def fc_profile_read(h):
    """{kernel name: (ms, launches)} since the last read; resets the totals."""
    ms = np.zeros(len(FC_K_NAMES), np.float64)
    n = np.zeros(len(FC_K_NAMES), np.int64)
    _check(load().fc_profile_read(h, ms.ctypes.data, n.ctypes.data))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(FC_K_NAMES)}


def check_blur_static_args(T, I, n_img, n_v, n_u):
    """Argument checks of fc_detector_blur_static, raised before any launch:
    T and I float32, contiguous, on the same CUDA device, each holding at
    least n_img * n_v * n_u elements (the kernels read and write that many)."""
    import torch
    for name, x in (("T", T), ("I", I)):
        if not hasattr(x, "data_ptr") or not getattr(x, "is_cuda", False):
            raise ValueError("fc_detector_blur_static takes device tensors (%s)" % name)
        if x.dtype != torch.float32:
            raise ValueError("fc_detector_blur_static: %s must be float32, got %s" % (name, x.dtype))
        if not x.is_contiguous():
            raise ValueError("fc_detector_blur_static: %s must be contiguous" % name)
    if T.device != I.device:
        raise ValueError("fc_detector_blur_static: T on %s, I on %s" % (T.device, I.device))
    if min(n_img, n_v, n_u) <= 0:
        raise ValueError("fc_detector_blur_static: sizes must be positive")
    n = int(n_img) * int(n_v) * int(n_u)
    for name, x in (("T", T), ("I", I)):
        if x.numel() < n:
            raise ValueError("fc_detector_blur_static: %s holds %d elements, n_img * n_v * n_u = %d"
                             % (name, x.numel(), n))


def fc_detector_blur_static(T, I, n_img, n_v, n_u, psf_sigma_px, scatter_sigma_px, spr, n0,
                            stream=None):
    """Allocation-free detector blur on caller-provided device tensors (the
    library runs on T's device)."""
    import torch
    check_blur_static_args(T, I, n_img, n_v, n_u)
    with torch.cuda.device(T.device):
        return _check(load().fc_detector_blur_static(T.data_ptr(), I.data_ptr(), n_img, n_v, n_u,
                                                     psf_sigma_px, scatter_sigma_px, spr, n0,
                                                     _stream(stream)))


def _dev(x, name):
    p, w = _ptr(x)
    if w != FC_DEVICE:
        raise ValueError("%s must be a device tensor" % name)
    return p


def fc_surrogate_init(h, seed=0):
    return _check(load().fc_surrogate_init(h, seed))


def fc_surrogate_train(h, L, lnT, steps, batch, lr, seed=0, stream=None):
    """Train on device tensors L [n][n_mat], lnT [n]; returns the per-step MSE."""
    n = lnT.numel()
    hist = np.zeros(max(steps, 1), np.float32)
    _check(load().fc_surrogate_train(h, _dev(L, "L"), _dev(lnT, "lnT"), n, steps, batch, lr, seed,
                                     hist.ctypes.data, _stream(stream)))
    return hist[:steps]


def fc_surrogate_grad(h, L, lnT, n=None, stream=None):
    """(gradient [FC_SURROGATE_PARAMS], loss) over the first n samples."""
    n = lnT.numel() if n is None else n
    g = np.zeros(FC_SURROGATE_PARAMS, np.float32)
    loss = np.zeros(1, np.float32)
    _check(load().fc_surrogate_grad(h, _dev(L, "L"), _dev(lnT, "lnT"), n, g.ctypes.data,
                                    loss.ctypes.data, _stream(stream)))
    return g, float(loss[0])


def fc_surrogate_get(h):
    st = np.zeros(FC_SURROGATE_STATE, np.float32)
    _check(load().fc_surrogate_get(h, st.ctypes.data))
    return st


def fc_surrogate_set(h, state):
    st = np.ascontiguousarray(state, np.float32)
    if st.size != FC_SURROGATE_STATE:
        raise ValueError("state must hold FC_SURROGATE_STATE floats")
    return _check(load().fc_surrogate_set(h, st.ctypes.data))


def fc_surrogate_eval(h, L, lnT, stream=None, count_fallback=True):
    """ln T by the surrogate into device tensor lnT; returns the fallback count."""
    c = ctypes.c_int64(0)
    _check(load().fc_surrogate_eval(h, _dev(L, "L"), lnT.numel(), _dev(lnT, "lnT"),
                                    ctypes.byref(c) if count_fallback else None, _stream(stream)))
    return c.value


def fc_surrogate_guard(h, L, lnT, tol, stream=None):
    """Set the per-ray guard from data (device L [n][n_mat], exact lnT [n]);
    returns the baseline-attenuation threshold (inf: none)."""
    thr = ctypes.c_double(0.0)
    _check(load().fc_surrogate_guard(h, _dev(L, "L"), _dev(lnT, "lnT"), lnT.numel(), float(tol),
                                     ctypes.byref(thr), _stream(stream)))
    return thr.value


def fc_surrogate_sigma(z, out, stream=None):
    """sigma(z) of device float32 z into out, as the surrogate kernels
    evaluate it (the activations' error is measured through this)."""
    if str(z.dtype) != "torch.float32" or str(out.dtype) != "torch.float32" or out.numel() < z.numel():
        raise ValueError("fc_surrogate_sigma: out must be float32 with at least z.numel() elements")
    return _check(load().fc_surrogate_sigma(_dev(z, "z"), _dev(out, "out"), z.numel(), _stream(stream)))


def fc_surrogate_project(h, angle_begin, angle_count, out, stream=None):
    """T of every ray by projector path lengths + surrogate (instead of the
    energy loop) into out (host array or device tensor)."""
    p, where = _ptr(out)
    return _check(load().fc_surrogate_project(h, angle_begin, angle_count, p, where,
                                              _stream(stream)))


def fc_energy_sum_lengths(h, L, lnT, stream=None):
    return _check(load().fc_energy_sum_lengths(h, _dev(L, "L"), lnT.numel(), _dev(lnT, "lnT"),
                                               _stream(stream)))


def fc_cnr_grad(h, logits, D, rho0, rho, z, rois, grads=True, stream=None):
    """CNR objective J and its gradients.

    logits, D, rho0: host arrays; rho: device float tensor [nz][ny][nx];
    z: device float tensor [n_angles][n_v][n_u] or None; rois: (cx, cy, r)
    tuples in cm.  Returns (J, dJ/dlogits, dJ/dD, dJ/drho) (the last a device
    tensor), or (J, None, None, None) when grads is False."""
    lg = np.ascontiguousarray(logits, np.float64)
    dd = np.ascontiguousarray(D, np.float64)
    r0 = np.ascontiguousarray(rho0, np.float64)
    roi = (fc_cnr_roi * len(rois))(*[fc_cnr_roi(*r) for r in rois])
    J = ctypes.c_double(0.0)
    gl = np.zeros_like(lg) if grads else None
    gd = np.zeros_like(dd) if grads else None
    gr = None
    if grads:
        import torch
        gr = torch.empty_like(rho)
    zp = _dev(z, "z") if z is not None else None
    _check(load().fc_cnr_grad(h, lg.ctypes.data, dd.ctypes.data, r0.ctypes.data, _dev(rho, "rho"),
                              zp, len(rois), roi, ctypes.byref(J),
                              gl.ctypes.data if grads else None, gd.ctypes.data if grads else None,
                              _dev(gr, "g_rho") if grads else None, _stream(stream)))
    return J.value, gl, gd, gr


def cnr_objective(h, rho0, z, rois):
    """torch.autograd.Function-backed J(logits, D, rho) for a configured
    handle: J = apply(logits (cpu f64), D (cpu f64), rho (cuda f32)).  The
    forward call runs the library's adjoint as well and keeps the gradients."""
    import torch

    class _Cnr(torch.autograd.Function):
        @staticmethod
        def forward(ctx, logits, D, rho):
            J, gl, gd, gr = fc_cnr_grad(h, logits.detach().cpu().numpy(),
                                        D.detach().cpu().numpy(), rho0, rho.detach().contiguous(),
                                        z, rois)
            ctx.save_for_backward(torch.from_numpy(gl), torch.from_numpy(gd), gr)
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            gl, gd, gr = ctx.saved_tensors
            return gJ * gl.to(gJ.device), gJ * gd.to(gJ.device), (gJ.to(gr.device) * gr).to(gr.dtype)

    return _Cnr.apply


# ---------------------------------------------------------------- convenience
class Scanner:
    """A handle configured for one workload (geometry + phantom + spectrum)."""

    def __init__(self, workload, labels=None, device=0, noise=None, stream=None):
        self.w = workload
        self.g = workload.geom
        self.h = fc_create(device)
        fc_set_geometry(self.h, self.g)
        lab = workload.make_phantom() if labels is None else labels
        self.n_mat = len(workload.labels)
        fc_set_phantom(self.h, lab, self.n_mat, stream)
        w, d = workload.spectrum()
        fc_set_spectrum_detector(self.h, w, d, workload.mu(), workload.psf_sigma_px,
                                 workload.scatter_sigma_px, workload.spr, workload.n0,
                                 workload.seed, workload.noise if noise is None else noise)

    def dose(self, angle_begin=0, angle_count=1):
        """(D0(E) [n_e], Dp) in Gy per particle for the workload's materials."""
        d0, dp = fc_dose_estimate(self.h, angle_begin, angle_count, self.w.energies(),
                                  self.w.muen_water(), self.w.densities())
        return d0, float(dp[0])

    def close(self):
        if self.h is not None:
            fc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
