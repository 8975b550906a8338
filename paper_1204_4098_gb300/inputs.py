"""Seeded synthetic initial conditions shared by the CUDA path and the oracle.

This module holds none of the lattice Boltzmann arithmetic: it only draws
density (and velocity) fields on the host, as float64 numpy arrays of shape
(ny, nx) with x fastest, from explicit parameters and a seed.  Both the CUDA
library and the oracle receive the same arrays, so neither needs a random
number generator of its own.

Recipes (coexistence densities are passed in by the caller):

* ``slab_step``  -- liquid rows [y_lo, y_hi) at rho_l, vapour elsewhere, then
  multiplicative noise rho (1 + amp U[-1, 1]) (flat-interface start);
* ``slab_tanh``  -- the smooth flat-interface profile of Eq. 36 with
  interfaces at ny/4 and 3 ny/4 (100 x 100 in the paper: 25 and 75);
* ``droplet``    -- the tanh droplet of Eq. 24 centred at (nx/2, ny/2);
* ``spinodal``   -- rho_avg (1 + amp U[-1, 1]) (spinodal decomposition);
* ``shear_wave``, ``taylor_green`` -- uniform density with a decaying
  sinusoidal velocity field (force-free checks);
* ``sweep_instances`` -- the parameter-sweep sampler (grid sizes, T/Tc, tau,
  sigma, scheme) of the batched flat-interface sweep.
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.default_rng(seed)


def slab_step(nx, ny, rho_g, rho_l, y_lo=None, y_hi=None, amp=0.0, seed=1):
    """Step profile: rho_l on rows [y_lo, y_hi), rho_g elsewhere, then noise."""
    y_lo = ny // 4 if y_lo is None else y_lo
    y_hi = 3 * ny // 4 if y_hi is None else y_hi
    rho = np.full((ny, nx), float(rho_g))
    rho[y_lo:y_hi, :] = float(rho_l)
    if amp:
        rho *= 1.0 + amp * _rng(seed).uniform(-1.0, 1.0, size=(ny, nx))
    return rho


def slab_tanh(nx, ny, rho_g, rho_l, W=5.0, y1=None, y2=None):
    """Eq. 36: rho_g + (rho_l - rho_g)/2 [tanh(2(y-y1)/W) - tanh(2(y-y2)/W)]."""
    y1 = ny / 4.0 if y1 is None else y1
    y2 = 3.0 * ny / 4.0 if y2 is None else y2
    y = np.arange(ny, dtype=np.float64)[:, None]
    prof = rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2.0 * (y - y1) / W)
                                             - np.tanh(2.0 * (y - y2) / W))
    return np.broadcast_to(prof, (ny, nx)).copy()


def droplet(nx, ny, rho_g, rho_l, r0, W=5.0, x0=None, y0=None):
    """Eq. 24: (rho_l + rho_g)/2 - (rho_l - rho_g)/2 tanh(2 (r - r0) / W)."""
    x0 = nx / 2.0 if x0 is None else x0
    y0 = ny / 2.0 if y0 is None else y0
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")
    r = np.sqrt((x - x0) ** 2 + (y - y0) ** 2)
    return 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (r - r0) / W)


def spinodal(nx, ny, rho_avg, amp=0.01, seed=3):
    """rho_avg (1 + amp U[-1, 1]) per cell."""
    return rho_avg * (1.0 + amp * _rng(seed).uniform(-1.0, 1.0, size=(ny, nx)))


def shear_wave(nx, ny, u0=1e-3, rho0=1.0, modes=1):
    """Shear wave u_x = u0 sin(k y), u_y = 0 on a uniform density.

    Returns (rho, ux, uy, k).  A single Fourier mode decays as
    exp(-nu k^2 t) under the incompressible Navier-Stokes equations.
    """
    k = 2.0 * np.pi * modes / ny
    y = np.arange(ny, dtype=np.float64)[:, None]
    ux = np.broadcast_to(u0 * np.sin(k * y), (ny, nx)).copy()
    uy = np.zeros((ny, nx))
    rho = np.full((ny, nx), float(rho0))
    return rho, ux, uy, k


def taylor_green(nx, ny, u0=1e-3, rho0=1.0):
    """Taylor-Green vortex u = u0 (sin kx cos ky, -cos kx sin ky), square grid.

    Returns (rho, ux, uy, k) with k = 2 pi / nx; the velocity decays as
    exp(-2 nu k^2 t).
    """
    k = 2.0 * np.pi / nx
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")
    ux = u0 * np.sin(k * x) * np.cos(k * y)
    uy = -u0 * np.cos(k * x) * np.sin(k * y)
    rho = np.full((ny, nx), float(rho0))
    return rho, ux, uy, k


def sweep_instances(count, seed=4, nx_range=(32, 512), ny_range=(128, 512),
                    t_range=(0.45, 0.95), tau_range=(0.6, 1.5),
                    sigma_range=(0.0, 0.2), schemes=(0, 1, 2)):
    """Independent uniform draws of (nx, ny, T/Tc, tau, sigma, scheme)."""
    g = _rng(seed)
    out = []
    for _ in range(count):
        out.append(dict(
            nx=int(g.integers(nx_range[0], nx_range[1] + 1)),
            ny=int(g.integers(ny_range[0], ny_range[1] + 1)),
            T_over_Tc=float(g.uniform(*t_range)),
            tau=float(g.uniform(*tau_range)),
            sigma=float(g.uniform(*sigma_range)),
            scheme=int(g.choice(schemes)),
        ))
    return out
