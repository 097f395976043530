"""The seeded input recipes (paper_2104_11385_gb300/workloads.py) against the
shapes and sizes they are documented to have: particle counts, the foil's
extent and density, weights that reproduce the stated densities, thermal
spreads, the log-normal box counts and the 2D laser-ion target.  CPU only,
at reduced extents where the full recipe would not fit a test."""
import math

import numpy as np

from paper_2104_11385_gb300 import workloads as W


def _charge_density(sp, volume):
    return sp["q"] * float(np.sum(sp["w"])) / volume


def test_uniform32_recipe():
    wl = W.uniform32(seed=1)
    (e,) = wl["species"]
    n, dx = wl["ncell"][0], wl["dx"][0]
    assert wl["ncell"] == (32, 32, 32) and wl["box"] == (8, 8, 8) and len(e["x"]) == 32 ** 3 * 8
    L = n * dx
    for k in ("x", "y", "z"):
        assert e[k].min() >= 0.0 and e[k].max() < L
    # the electrons neutralise the unit ion background exactly
    assert math.isclose(_charge_density(e, L ** 3), -wl["rho0"], rel_tol=1e-12)
    for k in ("ux", "uy", "uz"):
        assert abs(np.std(e[k]) - 0.01) < 2e-4 and abs(np.mean(e[k])) < 1e-4
    assert math.isclose(wl["dt"], 0.99 * dx / math.sqrt(3.0))


def test_foil_recipe_at_a_quarter_of_the_extents():
    wl = W.foil256(seed=2, scale=4)
    e, p = wl["species"]
    n, dx = wl["ncell"][0], wl["dx"][0]
    assert wl["ncell"] == (64, 64, 64)
    # the foil: 2 cell layers at the domain's middle, 64 particles per cell per species
    assert len(e["x"]) == len(p["x"]) == 64 * 64 * 2 * 64
    assert e["z"].min() >= 32 * dx and e["z"].max() < 34 * dx
    # each proton starts on an electron, at rest; the electrons are thermal
    for k in ("x", "y", "z"):
        assert np.array_equal(e[k], p[k])
    assert not np.any(p["ux"]) and not np.any(p["uy"]) and not np.any(p["uz"])
    assert abs(np.std(e["ux"]) - 0.01) < 3e-4
    # 30 times the critical density (omega_pe^2 = 30 with omega0 = 1) inside the foil
    foil_volume = (n * dx) ** 2 * 2 * dx
    assert math.isclose(-_charge_density(e, foil_volume), 30.0, rel_tol=1e-12)
    assert math.isclose(_charge_density(p, foil_volume), 30.0, rel_tol=1e-12)
    assert math.isclose(dx, 2.0 * math.pi / 32.0)  # lambda0 / 32
    assert len(set(e["id"]) | set(p["id"])) == 2 * len(e["x"])  # ids unique across species


def test_lognormal_box_counts():
    wl = W.lognormal(seed=3, nbox=(8, 8, 8))
    c = wl["box_counts"]
    assert len(c) == 512 and int(c.sum()) == len(wl["species"][0]["x"])
    # round(exp(N(ln 2000, 2^2))): median 2000, and ln(count) spread 2
    assert 1700 < np.median(c) < 2350
    lc = np.log(np.maximum(c, 1))
    assert abs(np.std(lc[c > 0]) - 2.0) < 0.2
    # every particle inside its own box
    e = wl["species"][0]
    bl = wl["box"][0] * wl["dx"][0]
    b = ((e["z"] // bl) * 8 + e["y"] // bl) * 8 + e["x"] // bl
    assert np.array_equal(np.bincount(b.astype(np.int64), minlength=512), c)


def test_laser_ion_2d_target():
    wl = W.laser_ion_2d(seed=6, scale=8)
    e, p = wl["species"]
    n, dx = wl["ncell"][0], wl["dx"][0]
    um = 2.0 * math.pi / 0.8
    assert wl["dim"] == 2 and wl["ncell"] == (240, 1, 240) and wl["order"] == 3
    assert math.isclose(n * dx, 30.0 * um)
    # the disk: density 5 n_c inside r = 5 um, particles only within the 7 um slope
    r = np.hypot(e["x"] - 15.0 * um, e["z"] - 10.0 * um)
    assert r.max() < 7.0 * um + 2 * dx
    dens = e["w"] * 32 / (dx * dx)
    assert math.isclose(dens.max(), 5.0, rel_tol=1e-12)
    assert np.all(dens[r <= 5.0 * um] == 5.0) and np.all(dens[r > 5.0 * um] < 5.0)
    assert np.array_equal(e["x"], p["x"]) and np.array_equal(e["z"], p["z"])
    assert wl["laser"]["a0"] == 25.0 and math.isclose(wl["laser"]["w0"], 4.0 * um)
