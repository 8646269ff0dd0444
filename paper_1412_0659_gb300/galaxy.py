"""On-the-fly galaxy initial conditions (Sec. IV): the Milky Way model --
NFW halo, exponential disk, Hernquist bulge -- sampled on the GPU by
``bonsai_galaxy_generate`` (include/bonsai_gb.h) straight into device
memory, ready for ``TreeGravity.build``.

    g = galaxy.sec4(1 << 23, seed=1006)        # the model's parameters
    pos, vel, mass = galaxy.generate(g)         # float64 CUDA tensors
"""
from __future__ import annotations

import torch

from . import capi

RADIAL_ROWS = ("r", "Psi", "M_total", "M_halo", "M_bulge", "P_halo", "P_bulge", "g2_halo",
               "g2_bulge", "f_halo", "f_bulge", "vnorm_halo", "vnorm_bulge", "rho_halo",
               "rho_bulge")
DISK_ROWS = ("cdf", "vc2", "kappa", "sigma_R", "sigma_phi", "sigma_z", "v_phi")


def sec4(n: int, seed: int = 1006, **overrides) -> capi.bonsai_galaxy:
    """Parameters of the Sec. IV model for n particles; keyword arguments
    replace fields (for instance M_bulge=0.0, n_bulge=0)."""
    g = capi.bonsai_galaxy_sec4(n, seed)
    for k, v in overrides.items():
        if not hasattr(g, k):
            raise AttributeError(k)
        setattr(g, k, v)
    return g


def generate(g: capi.bonsai_galaxy, device=None, stream=None):
    """Positions (3, n), velocities (3, n) and masses (n,) as float64 CUDA
    tensors: halo, disk, bulge in that order, centre of mass at rest."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n = int(g.n_halo + g.n_disk + g.n_bulge)
    pos = torch.empty(3, n, dtype=torch.float64, device=dev)
    vel = torch.empty(3, n, dtype=torch.float64, device=dev)
    mass = torch.empty(n, dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        capi.bonsai_galaxy_generate(g, pos, vel, mass, stream)
    return pos, vel, mass


def tables(g: capi.bonsai_galaxy, device=None, with_vcdf: bool = True) -> dict:
    """The generator's tables as a dict of CUDA tensors (rows by name, plus
    'vcdf' of shape (2, K, V): halo, bulge)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    rad = torch.empty(capi.BONSAI_ICS_NRAD_OUT, capi.BONSAI_ICS_K, dtype=torch.float64, device=dev)
    disk = torch.empty(capi.BONSAI_ICS_NDISK_OUT, capi.BONSAI_ICS_KD, dtype=torch.float64, device=dev)
    vc = (torch.empty(2, capi.BONSAI_ICS_K, capi.BONSAI_ICS_V, dtype=torch.float64, device=dev)
          if with_vcdf else None)
    with torch.cuda.device(dev):
        capi.bonsai_galaxy_tables(g, rad, vc, disk)
    out = {k: rad[i] for i, k in enumerate(RADIAL_ROWS)}
    out.update({"disk_" + k: disk[i] for i, k in enumerate(DISK_ROWS)})
    out["vcdf"] = vc
    return out
