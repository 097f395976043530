"""Seeded synthetic inputs for the PIC workloads (shared by the tests, the
benchmark and the oracle runs).  This module only draws numbers: it holds none
of the method's arithmetic.

Workloads (all normalised units, c = 1; the paper's own input decks are not
available, so these stand in for them with the shapes and structure of its
runs -- a dense target in vacuum hit by a laser, and boxes of wildly uneven
particle counts):
  uniform32      3D cold electron plasma on fixed ions: 32^3 cells of dx = 0.25
                 in 64 boxes of 8^3, 8 electrons/cell at uniform random
                 positions, u ~ N(0, 0.01^2) per component, w = n0 dx^3 / 8
                 (n0 = 1), linear shape, periodic, dt = 0.99 dx / sqrt(3).
  foil256        3D laser-foil: 256^3 cells of dx = lambda0/32 (lambda0 = 2 pi,
                 omega0 = 1) in 512 boxes of 32^3; hydrogen foil in cell layers
                 z in [128, 136) at n = 30 n_c, 64 electrons + 64 protons per
                 foil cell (each proton at an electron's position: neutral
                 start), electrons u ~ N(0, 0.01^2), protons at rest; Gaussian
                 laser a0 = 20, x-polarised, from an antenna near z-min; z damping
                 layers of 16 cells; linear shape.
  lognormal4096  3D batched uneven boxes: 4096 boxes of 16^3 cells (256^3,
                 dx = 0.25), box particle counts round(exp(N(ln 2000, 2^2))),
                 uniform positions inside the box, u ~ N(0, 0.01^2), weights for
                 a mean density n0 = 1, quadratic shape, periodic.
  foil_at_scale  3D laser-foil at scale: 512 x 512 x 1024 cells in 32^3 boxes,
                 foil 16 cells thick at 64 ppc per species.
  laser_ion_2d   the paper's 2D3V laser-ion setup (Sec. 3.1) at one-GPU scale:
                 (z, x) domain 30 um x 30 um (z in [-10, 20] um, x in [-15, 15]
                 um) in 1920^2 cells (dx = 0.0195 lambda0) and 64^2-cell boxes;
                 hydrogen disk of radius 5 um + 2 um slope (exponential, 50 nm
                 scale length, constant macro-particle number) at 5 n_c;
                 electrons with 0.01 m_e c Gaussian momenta in x and z, protons
                 at rest; laser a0 = 25, lambda0 = 0.8 um, x-polarised, waist
                 4 um, 10 fs amplitude e-folding time, from z = -9 um; cubic
                 shapes; 32 macro-particles per cell per species (the paper:
                 900, which does not fit one GPU); scale = 2 gives the paper's
                 960^2 run.
The ``scale`` argument shrinks a workload for the oracle-sized parity cases
(same recipe, fewer cells / particles).
"""
from __future__ import annotations

import math

import numpy as np

PROTON_MASS = 1836.15267343


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _species(q, m, x, y, z, ux, uy, uz, w, id0=0):
    n = len(x)
    return {"q": float(q), "m": float(m), "x": x, "y": y, "z": z, "ux": ux, "uy": uy, "uz": uz,
            "w": w, "id": np.arange(id0, id0 + n, dtype=np.int64)}


def uniform32(seed=1, n=32, box=8, ppc=8, dx=0.25, uth=0.01, order=1):
    """3D uniform thermal electron plasma on a fixed ion background."""
    r = _rng(seed)
    L = n * dx
    npart = n ** 3 * ppc
    x, y, z = (r.uniform(0.0, L, npart) for _ in range(3))
    ux, uy, uz = (r.normal(0.0, uth, npart) for _ in range(3))
    n0 = 1.0
    w = np.full(npart, n0 * dx ** 3 / ppc)
    return {
        "name": f"uniform{n}", "dim": 3, "ncell": (n, n, n), "box": (box, box, box),
        "dx": (dx, dx, dx), "dt": 0.99 * dx / math.sqrt(3.0), "order": order, "absorb": 0,
        "species": [_species(-1.0, 1.0, x, y, z, ux, uy, uz, w)], "laser": None,
        "rho0": n0, "steps": 50,
    }


def foil(seed=2, n=(256, 256, 256), box=32, foil_z=(128, 136), ppc=64, density=30.0,
         uth=0.01, a0=20.0, absorb=16, order=1):
    """3D laser-foil: a thin overdense hydrogen foil in vacuum hit by a laser."""
    r = _rng(seed)
    lam = 2.0 * math.pi
    dx = lam / 32.0
    nx, ny, nz = n
    z0, z1 = foil_z
    ncell_foil = nx * ny * (z1 - z0)
    npart = ncell_foil * ppc
    x = r.uniform(0.0, nx * dx, npart)
    y = r.uniform(0.0, ny * dx, npart)
    z = r.uniform(z0 * dx, z1 * dx, npart)
    ue = [r.normal(0.0, uth, npart) for _ in range(3)]
    w = np.full(npart, density * dx ** 3 / ppc)
    zeros = np.zeros(npart)
    e = _species(-1.0, 1.0, x, y, z, *ue, w, id0=0)
    p = _species(1.0, PROTON_MASS, x.copy(), y.copy(), z.copy(), zeros, zeros.copy(), zeros.copy(),
                 w.copy(), id0=npart)
    Lx, Ly = nx * dx, ny * dx
    laser = {"a0": a0, "w0": 2.0 * lam, "tau": 3.75 * lam, "t_peak": 3.0 * 3.75 * lam,
             "omega": 1.0, "xc": 0.5 * Lx, "yc": 0.5 * Ly, "k_ant": absorb + 4}
    return {
        "name": f"foil{nx}x{ny}x{nz}", "dim": 3, "ncell": tuple(n), "box": (box, box, box),
        "dx": (dx, dx, dx), "dt": 0.99 * dx / math.sqrt(3.0), "order": order, "absorb": absorb,
        "species": [e, p], "laser": laser, "rho0": 0.0, "steps": 1000, "lb_interval": 10,
    }


def foil_at_scale(seed=5, scale=1):
    """The foil at scale: 512 x 512 x 1024 cells in 32^3 boxes, the foil 16
    cells thick (z in [512, 528)) at 64 ppc per species (536,870,912
    particles); 2000 steps into the expansion, balancing every 20.  scale > 1
    divides every extent (the foil's thickness, the boxes and the damping
    layers too, down to 2 cells, 8 cells and 4 cells)."""
    nx, nz = 512 // scale, 1024 // scale
    t = max(2, 16 // scale)
    wl = foil(seed=seed, n=(nx, nx, nz), box=max(8, 32 // scale), foil_z=(nz // 2, nz // 2 + t), ppc=64,
              absorb=max(4, 16 // scale))
    wl["steps"], wl["lb_interval"] = 2000, 20
    return wl


def foil256(seed=2, scale=1):
    """The 256^3 foil; scale > 1 divides every extent (and the foil) by scale."""
    n = 256 // scale
    t = max(2, 8 // scale)
    return foil(seed=seed, n=(n, n, n), box=max(8, 32 // scale), foil_z=(n // 2, n // 2 + t),
                absorb=max(4, 16 // scale))


def lognormal(seed=3, nbox=(16, 16, 16), box=16, dx=0.25, median=2000.0, sigma=2.0, uth=0.01,
              order=2, max_per_box=None):
    """3D boxes with log-normally distributed particle counts."""
    r = _rng(seed)
    nb = nbox[0] * nbox[1] * nbox[2]
    counts = np.rint(np.exp(r.normal(math.log(median), sigma, nb))).astype(np.int64)
    if max_per_box is not None:
        counts = np.minimum(counts, max_per_box)
    npart = int(counts.sum())
    bidx = np.repeat(np.arange(nb), counts)
    bx = bidx % nbox[0]
    by = (bidx // nbox[0]) % nbox[1]
    bz = bidx // (nbox[0] * nbox[1])
    bl = box * dx
    x = (bx + r.uniform(0.0, 1.0, npart)) * bl
    y = (by + r.uniform(0.0, 1.0, npart)) * bl
    z = (bz + r.uniform(0.0, 1.0, npart)) * bl
    ux, uy, uz = (r.normal(0.0, uth, npart) for _ in range(3))
    ncell = tuple(nbox[a] * box for a in range(3))
    n0 = 1.0
    w = np.full(npart, n0 * dx ** 3 * ncell[0] * ncell[1] * ncell[2] / max(npart, 1))
    return {
        "name": f"lognormal{nb}", "dim": 3, "ncell": ncell, "box": (box, box, box),
        "dx": (dx, dx, dx), "dt": 0.99 * dx / math.sqrt(3.0), "order": order, "absorb": 0,
        "species": [_species(-1.0, 1.0, x, y, z, ux, uy, uz, w)], "laser": None, "rho0": n0,
        "steps": 50, "box_counts": counts,
    }


def random_plasma(seed, dim, ncell, box, dx, order, nspecies=2, npart=2000, umax=0.5,
                  absorb=0, laser=False):
    """Small random multi-species plasma for parity cases: positions uniform,
    momenta with random directions and magnitudes up to umax (electrons) so
    that many particles cross cell boundaries every step."""
    r = _rng(seed)
    L = [ncell[a] * dx[a] for a in range(3)]
    sp = []
    masses = [(-1.0, 1.0), (1.0, PROTON_MASS), (2.0, 4.0 * PROTON_MASS)]
    id0 = 0
    for s in range(nspecies):
        q, m = masses[s % len(masses)]
        x = r.uniform(0.0, L[0], npart)
        y = r.uniform(0.0, L[1], npart) if dim == 3 else np.zeros(npart)
        if absorb > 0:
            z = r.uniform((absorb + 1) * dx[2], (ncell[2] - absorb - 1) * dx[2], npart)
        else:
            z = r.uniform(0.0, L[2], npart)
        u = r.normal(size=(3, npart))
        scale = umax / (1.0 + s * 10.0)
        u *= scale / np.maximum(np.linalg.norm(u, axis=0), 1e-300) * r.uniform(0, 1, npart)
        w = r.uniform(0.5, 1.5, npart) * 0.05 * dx[0] * dx[1] * dx[2]
        sp.append(_species(q, m, x, y, z, u[0], u[1], u[2], w, id0=id0))
        id0 += npart
    inv = sum(1.0 / dx[a] ** 2 for a in range(3) if not (dim == 2 and a == 1))
    las = None
    if laser:
        las = {"a0": 0.5, "w0": 0.3 * L[0], "tau": 2.0, "t_peak": 1.0, "omega": 1.0,
               "xc": 0.5 * L[0], "yc": 0.5 * L[1], "k_ant": absorb + 2}
    return {
        "name": "random", "dim": dim, "ncell": tuple(ncell), "box": tuple(box), "dx": tuple(dx),
        "dt": 0.95 / math.sqrt(inv), "order": order, "absorb": absorb, "species": sp,
        "laser": las, "rho0": 0.0, "steps": 10,
    }


def random_fields(seed, ncell, amp=0.05):
    """Random smooth-ish initial E and B (six components, dense layout)."""
    r = _rng(seed)
    n = ncell[0] * ncell[1] * ncell[2]
    return [amp * r.normal(size=n) for _ in range(6)]


def laser_ion_2d(seed=6, ppc=32, scale=1, absorb=32):
    """The paper's 2D3V laser-ion acceleration setup at one-GPU scale."""
    r = _rng(seed)
    um = 2.0 * math.pi / 0.8  # one micrometre in c/omega0 for lambda0 = 0.8 um
    n = 1920 // scale
    L = 30.0 * um
    dx = L / n
    xc, zc = 15.0 * um, 10.0 * um  # the disk centre (x = z = 0) in domain coordinates
    rcore, rslope, lscale = 5.0 * um, 7.0 * um, 0.05 * um
    ii = np.arange(n)
    cx = (ii + 0.5) * dx - xc
    cz = (ii + 0.5) * dx - zc
    CZ, CX = np.meshgrid(cz, cx, indexing="ij")
    inside = np.sqrt(CX * CX + CZ * CZ) < rslope
    kz, kx = np.nonzero(inside)
    ncell = kz.size
    npart = ncell * ppc
    cell_x = np.repeat(kx, ppc)
    cell_z = np.repeat(kz, ppc)
    x = (cell_x + r.uniform(0.0, 1.0, npart)) * dx
    z = (cell_z + r.uniform(0.0, 1.0, npart)) * dx
    rad = np.sqrt((x - xc) ** 2 + (z - zc) ** 2)
    dens = 5.0 * np.where(rad <= rcore, 1.0, np.exp(-(rad - rcore) / lscale))
    w = dens * dx * dx / ppc
    ux = r.normal(0.0, 0.01, npart)
    uz = r.normal(0.0, 0.01, npart)
    zeros = np.zeros(npart)
    e = _species(-1.0, 1.0, x, zeros, z, ux, zeros.copy(), uz, w, id0=0)
    p = _species(1.0, PROTON_MASS, x.copy(), zeros.copy(), z.copy(), zeros.copy(), zeros.copy(),
                 zeros.copy(), w.copy(), id0=npart)
    fs = 2.0 * math.pi * 0.299792458 / 0.8  # one femtosecond in 1/omega0
    tau = 10.0 * fs
    laser = {"a0": 25.0, "w0": 4.0 * um, "tau": tau, "t_peak": 2.5 * tau, "omega": 1.0,
             "xc": xc, "yc": 0.0, "k_ant": int(round(1.0 * um / dx))}
    dt = 0.999 * dx / math.sqrt(2.0)
    return {
        "name": f"laser_ion_2d_{n}", "dim": 2, "ncell": (n, 1, n), "box": (64 // scale, 1, 64 // scale),
        "dx": (dx, 1.0, dx), "dt": dt, "order": 3, "absorb": absorb, "species": [e, p],
        "laser": laser, "rho0": 0.0, "steps": int(round(150.0 * fs / dt)), "lb_interval": 10,
    }
