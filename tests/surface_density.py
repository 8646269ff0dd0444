"""The loss of the differentiable run: a 64 x 64 surface-density map of
the x-y plane over [-15, 15]^2 kpc with cloud-in-cell (bilinear) weights,
and its squared difference from a target map.  Test-side application code
(the loss a user would write), in FP64 numpy with its analytic gradient and
in torch for autograd; not part of the tree method."""
import numpy as np

NPIX = 64
HALF = 15.0


def _cic(x, y):
    h = 2.0 * HALF / NPIX
    fx = (x + HALF) / h - 0.5
    fy = (y + HALF) / h - 0.5
    ix = np.floor(fx)
    iy = np.floor(fy)
    return h, ix.astype(np.int64), iy.astype(np.int64), fx - ix, fy - iy


def density_map(pos, mass):
    """Sigma[iy, ix] = sum_i m_i w_i(pixel) / h^2 (pixels outside dropped)."""
    h, ix, iy, tx, ty = _cic(pos[0], pos[1])
    out = np.zeros((NPIX, NPIX))
    for dx, wx in ((0, 1.0 - tx), (1, tx)):
        for dy, wy in ((0, 1.0 - ty), (1, ty)):
            jx, jy = ix + dx, iy + dy
            ok = (jx >= 0) & (jx < NPIX) & (jy >= 0) & (jy < NPIX)
            np.add.at(out, (jy[ok], jx[ok]), (mass * wx * wy)[ok] / (h * h))
    return out


def loss(pos, mass, target):
    return float(((density_map(pos, mass) - target) ** 2).sum())


def loss_grad(pos, mass, target):
    """(dL/dpos (3, N), dL/dmass (N,)) of loss(pos, mass, target)."""
    g = 2.0 * (density_map(pos, mass) - target)
    h, ix, iy, tx, ty = _cic(pos[0], pos[1])
    gx = np.zeros(pos.shape[1])
    gy = np.zeros(pos.shape[1])
    gm = np.zeros(pos.shape[1])
    for dx, wx, dwx in ((0, 1.0 - tx, -1.0), (1, tx, 1.0)):
        for dy, wy, dwy in ((0, 1.0 - ty, -1.0), (1, ty, 1.0)):
            jx, jy = ix + dx, iy + dy
            ok = (jx >= 0) & (jx < NPIX) & (jy >= 0) & (jy < NPIX)
            gp = np.zeros(pos.shape[1])
            gp[ok] = g[jy[ok], jx[ok]] / (h * h)
            gm += gp * wx * wy
            gx += gp * mass * dwx / h * wy
            gy += gp * mass * wx * dwy / h
    return np.stack([gx, gy, np.zeros_like(gx)]), gm


def density_map_torch(pos, mass):
    """The same map as a differentiable torch function of pos and mass."""
    import torch
    h = 2.0 * HALF / NPIX
    fx = (pos[0] + HALF) / h - 0.5
    fy = (pos[1] + HALF) / h - 0.5
    ix = torch.floor(fx).detach()
    iy = torch.floor(fy).detach()
    tx, ty = fx - ix, fy - iy
    ix, iy = ix.long(), iy.long()
    out = torch.zeros(NPIX * NPIX, dtype=pos.dtype, device=pos.device)
    for dx, wx in ((0, 1.0 - tx), (1, tx)):
        for dy, wy in ((0, 1.0 - ty), (1, ty)):
            jx, jy = ix + dx, iy + dy
            ok = (jx >= 0) & (jx < NPIX) & (jy >= 0) & (jy < NPIX)
            out = out.index_add(0, (jy * NPIX + jx)[ok], (mass * wx * wy)[ok] / (h * h))
    return out.view(NPIX, NPIX)
