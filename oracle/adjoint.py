"""FP64 reference of the CNR objective and its gradient -- TEST INFRASTRUCTURE.

Only the tests may import this module.  The objective follows the simulate-
and-reconstruct path (Sec. II.F-G):

    A_im  = sum_v M_iv rho_v / rho0_{m(v)} [m(v) = m]   (Siddon path lengths M)
    T_i   = sum_E c_E exp(-sum_m mu_m(E) A_im) / sum_E c_E,  c = softmax(logits) D
    I     = N0 (G_psf (x) T + SPR G_sc (x) T)           (separable, clamp-to-edge)
    K     = I + sqrt(I) z                                (fixed standard normals z)
    q     = ln(I_flood / max(K, 1)) SAD / sqrt(SAD^2 + u^2 + v^2)
    f     = Ram-Lak (x) q  (zero padding),   mu = B f  (bilinear backprojection)
    HU    = 1000 (mu - mu_w) / mu_w,   J = sum_r |HU_w - HU_r| / sqrt(s_w^2 + s_r^2)

written with plain PyTorch CPU operations in float64; the gradient is
PyTorch's reverse-mode differentiation of this forward (pinned by central
finite differences in the tests).  M comes from the oracle's Siddon
(``oracle.path_matrix``), B from the same bilinear rule as
``oracle.backproject`` (the two are checked against each other).
"""
from __future__ import annotations

import math

import numpy as np

import oracle


def backprojection_matrix(g):
    """Sparse (COO) B with mu.ravel() = B @ f.ravel() for f [n_angles][n_v][n_u]:
    bilinear taps (zero outside the detector) x (SAD / U)^2 x arc / (2 N)."""
    import torch
    nx, ny, nz = g.nx, g.ny, g.nz
    x = (np.arange(nx) - (nx - 1) / 2) * g.dx
    y = (np.arange(ny) - (ny - 1) / 2) * g.dy
    z = (np.arange(nz) - (nz - 1) / 2) * g.dz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    vox = np.arange(X.size)
    scale = 0.5 * g.arc / g.n_angles
    rows, cols, vals = [], [], []
    for k, th in enumerate(g.angles()):
        c, s = math.cos(th), math.sin(th)
        U = g.sad - (X * c + Y * s)
        ru = -X * s + Y * c
        fu = g.sdd * ru / U / g.du + (g.n_u - 1) / 2
        fv = g.sdd * Z / U / g.dv + (g.n_v - 1) / 2
        wgt = scale * (g.sad / U) ** 2
        u0, v0 = np.floor(fu).astype(np.int64), np.floor(fv).astype(np.int64)
        au, av = fu - u0, fv - v0
        for du_, dv_, ww in ((0, 0, (1 - au) * (1 - av)), (1, 0, au * (1 - av)),
                             (0, 1, (1 - au) * av), (1, 1, au * av)):
            uu, vv = u0 + du_, v0 + dv_
            ok = (uu >= 0) & (uu < g.n_u) & (vv >= 0) & (vv < g.n_v) & (ww != 0)
            rows.append(vox[ok])
            cols.append((k * g.n_v + vv[ok]) * g.n_u + uu[ok])
            vals.append((wgt * ww)[ok])
    idx = torch.from_numpy(np.stack([np.concatenate(rows), np.concatenate(cols)]))
    return torch.sparse_coo_tensor(idx, torch.from_numpy(np.concatenate(vals)),
                                   (g.n_voxels, g.n_rays)).coalesce()


def path_lengths_matrix(g):
    import torch
    rp, col, val = oracle.path_matrix(g)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    idx = torch.from_numpy(np.stack([rows, col]))
    return torch.sparse_coo_tensor(idx, torch.from_numpy(val), (g.n_rays, g.n_voxels)).coalesce()


def _taps(sigma):
    R = int(math.ceil(4 * sigma)) if sigma > 0 else 0
    j = np.arange(-R, R + 1)
    t = np.exp(-j * j / (2 * sigma * sigma)) if R > 0 else np.ones(1)
    return t / t.sum()


def _blur(x, sigma):
    """Separable clamp-to-edge sampled-Gaussian blur over the last two axes."""
    import torch
    import torch.nn.functional as F
    t = torch.from_numpy(_taps(sigma)).view(1, 1, -1)
    R = (t.shape[-1] - 1) // 2
    na, nv, nu = x.shape
    a = F.conv1d(F.pad(x.reshape(na * nv, 1, nu), (R, R), mode="replicate"), t).reshape(na, nv, nu)
    b = a.permute(0, 2, 1).reshape(na * nu, 1, nv)
    b = F.conv1d(F.pad(b, (R, R), mode="replicate"), t).reshape(na, nu, nv).permute(0, 2, 1)
    return b


def _ramp(q, tau):
    """Ram-Lak row filter with zero padding: tau * sum_j h[i - j] q[j]."""
    import torch
    import torch.nn.functional as F
    na, nv, nu = q.shape
    n = np.arange(-(nu - 1), nu)
    h = np.where(n == 0, 1.0 / (4 * tau * tau),
                 np.where(n % 2 != 0, -1.0 / (math.pi**2 * np.maximum(n * n, 1) * tau * tau), 0.0))
    k = torch.from_numpy(tau * h).view(1, 1, -1)
    return F.conv1d(q.reshape(na * nv, 1, nu), k, padding=nu - 1).reshape(na, nv, nu)


def roi_masks(g, water_r, z_margin, rois):
    """Boolean voxel masks [water, roi_1, ...] as the CUDA path defines them."""
    x = (np.arange(g.nx) - (g.nx - 1) / 2) * g.dx
    y = (np.arange(g.ny) - (g.ny - 1) / 2) * g.dy
    X, Y = np.meshgrid(x, y)
    zc = int(math.floor(g.nz * z_margin))
    zc = zc if g.nz > 2 * zc else 0
    zs = np.zeros(g.nz, bool)
    zs[zc:g.nz - zc] = True
    water = X**2 + Y**2 <= water_r**2
    out = [zs[:, None, None] & water[None]]
    taken = water.copy()
    for (cx, cy, r) in rois:
        m = ((X - cx) ** 2 + (Y - cy) ** 2 <= r * r) & ~taken
        taken |= m
        out.append(zs[:, None, None] & m[None])
    return [m.ravel() for m in out]


class Objective:
    """J(logits, D, rho) for one scan; build once, evaluate many times."""

    def __init__(self, wl, labels, rho0, z=None, rois=(), water_r=1.0, z_margin=0.1):
        import torch
        self.wl, self.g = wl, wl.geom
        g = self.g
        self.M = path_lengths_matrix(g)
        self.B = backprojection_matrix(g)
        lab = np.asarray(labels).ravel()
        n_mat = len(wl.labels)
        self.onehot = torch.from_numpy(np.eye(n_mat)[lab])
        self.irho0 = torch.from_numpy((1.0 / np.asarray(rho0, float))[lab])
        self.mu = torch.from_numpy(wl.mu())
        self.z = None if z is None else torch.from_numpy(np.asarray(z, np.float64))
        self.masks = [torch.from_numpy(m) for m in roi_masks(g, water_r, z_margin, rois)]
        u = (np.arange(g.n_u) - (g.n_u - 1) / 2) * g.du * g.sad / g.sdd
        v = (np.arange(g.n_v) - (g.n_v - 1) / 2) * g.dv * g.sad / g.sdd
        self.cosw = torch.from_numpy(g.sad / np.sqrt(g.sad**2 + u[None, :]**2 + v[:, None]**2))

    def __call__(self, logits, D, rho):
        import torch
        g, wl = self.g, self.wl
        c = torch.softmax(logits, 0) * D
        X = (rho * self.irho0)[:, None] * self.onehot
        A = torch.sparse.mm(self.M, X)
        T = (torch.exp(-A @ self.mu.T) @ c / c.sum()).reshape(g.n_angles, g.n_v, g.n_u)
        I = wl.n0 * (_blur(T, wl.psf_sigma_px) + wl.spr * _blur(T, wl.scatter_sigma_px))
        K = I if self.z is None else I + torch.sqrt(I) * self.z
        flood = wl.n0 * (1 + wl.spr)
        q = torch.log(flood / torch.clamp(K, min=1.0)) * self.cosw
        f = _ramp(q, g.du * g.sad / g.sdd)
        mu = torch.sparse.mm(self.B, f.reshape(-1, 1)).reshape(-1)
        w = self.masks[0]
        mu_w = mu[w].mean()
        hu = 1000.0 * (mu - mu_w) / mu_w
        hw = hu[w]
        J = 0.0
        for m in self.masks[1:]:
            hr = hu[m]
            var_w = ((hw - hw.mean()) ** 2).mean()
            var_r = ((hr - hr.mean()) ** 2).mean()
            J = J + torch.abs(hw.mean() - hr.mean()) / torch.sqrt(var_w + var_r)
        return J

    def value_and_grad(self, logits, D, rho):
        import torch
        lt = torch.tensor(np.asarray(logits, np.float64), requires_grad=True)
        dt = torch.tensor(np.asarray(D, np.float64), requires_grad=True)
        rt = torch.tensor(np.asarray(rho, np.float64).ravel(), requires_grad=True)
        J = self(lt, dt, rt)
        J.backward()
        return float(J), lt.grad.numpy(), dt.grad.numpy(), rt.grad.numpy()
