"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each expected value comes from a
closed form (discrete dispersion, exact Boris rotation, leapfrog plasma
frequency), a conservation law (Esirkepov continuity, Gauss), a textbook
property (B-spline partition of unity, exact interpolation of linear fields), a
brute-force search on tiny inputs, or a number the paper prints.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- shapes ---
def test_shape_values_and_partition_of_unity():
    # textbook B-spline values
    assert orc.shape(1, 0.0) == 1.0 and orc.shape(1, 0.25) == 0.75 and orc.shape(1, 1.0) == 0.0
    assert orc.shape(2, 0.0) == 0.75 and orc.shape(2, 0.5) == 0.5
    assert orc.shape(2, 1.0) == 0.125 and orc.shape(2, 1.5) == 0.0
    assert orc.shape(3, 0.0) == pytest.approx(2 / 3, abs=1e-16) and orc.shape(3, 1.0) == pytest.approx(1 / 6, abs=1e-16)
    assert orc.shape(3, 2.0) == 0.0 and orc.shape(3, 1.5) == pytest.approx(1 / 48, abs=1e-16)
    # the cubic B-spline is the hat convolved with the hat: S3(0.5) = 23/48
    assert orc.shape(3, 0.5) == pytest.approx(23 / 48, abs=1e-16)
    rng = np.random.default_rng(0)
    for order in (1, 2, 3):
        for x in rng.uniform(-3, 3, 50):
            nodes = np.arange(math.floor(x) - 3, math.floor(x) + 4)
            vals = [orc.shape(order, x - k) for k in nodes]
            assert abs(sum(vals) - 1.0) < 1e-15
            # first moment: shape centred on the particle
            assert abs(sum(v * k for v, k in zip(vals, nodes)) - x) < 1e-13


# ---------------------------------------------------------------- gather ---
STAG = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


@pytest.mark.parametrize("dim,order", [(3, 1), (3, 2), (3, 3), (2, 1), (2, 2), (2, 3)])
def test_gather_reproduces_linear_fields(dim, order):
    """Linear and quadratic B-splines interpolate affine fields exactly, so any
    error in a component's staggering offset shows up as a b*dx/2 bias."""
    n = (12, 12 if dim == 3 else 1, 12)
    d = (0.3, 0.4 if dim == 3 else 1.0, 0.5)
    sim = orc.OracleSim(dim, n, d, 0.1, order)
    rng = np.random.default_rng(1)
    coef = rng.normal(size=(6, 4))
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for c in range(6):
        sx, sy, sz = STAG[c]
        X = (i + sx) * d[0]
        Y = (j + sy) * d[1] if dim == 3 else 0 * X
        Z = (k + sz) * d[2]
        sim.set_field(c, coef[c, 0] + coef[c, 1] * X + coef[c, 2] * Y + coef[c, 3] * Z)
    for _ in range(40):
        x = rng.uniform(3, 8) * d[0]
        y = rng.uniform(3, 8) * d[1] if dim == 3 else 0.0
        z = rng.uniform(3, 8) * d[2]
        got = sim.gather(x, y, z)
        want = coef[:, 0] + coef[:, 1] * x + coef[:, 2] * y + coef[:, 3] * z
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


# ----------------------------------------------------------------- Boris ---
@pytest.mark.parametrize("q", [1.0, -1.0])
def test_boris_exact_gyration(q):
    """E = 0, uniform B along z: every push rotates u about z by exactly
    2*atan(q B dt / (2 m gamma)) (clockwise for q > 0), |u| is conserved."""
    B0, dt, m = 1.7, 0.3, 1.0
    u = np.array([0.8, 0.0, 0.3])
    g = math.sqrt(1 + u @ u)
    theta = 2 * math.atan(q * B0 * dt / (2 * m * g))
    eb = np.array([0, 0, 0, 0, 0, B0])
    uu = u.copy()
    for n in range(1, 1001):
        uu = orc.boris(q, m, dt, eb, uu)
        assert abs(math.sqrt(uu @ uu) - math.sqrt(u @ u)) < 1e-14
    ang = -1000 * theta
    want = np.array([u[0] * math.cos(ang), u[0] * math.sin(ang), u[2]])
    np.testing.assert_allclose(uu, want, atol=2e-12)


def test_boris_parallel_fields_rotate_with_the_half_kicked_gamma():
    """E and B both along z: u_z gains q E dt / m per step exactly (the
    rotation about z leaves it alone), |u_perp| is conserved, and step n
    rotates u_perp by -2 atan(k B / gamma-) with k = q dt / (2 m) and gamma-
    that of u after the first half kick, u_z0 + (2n + 1) k E: the relativistic
    factor belongs to u-, not to u^{n-1/2} (which would turn the orbit by
    0.09 rad more here)."""
    q, m, dt, B, E = -1.0, 1.0, 0.2, 1.3, 0.4
    k = q * dt / (2 * m)
    u0 = np.array([0.7, 0.2, 0.5])
    eb = np.array([0, 0, E, 0, 0, B])
    u, ang, up2 = u0.copy(), 0.0, u0[0] ** 2 + u0[1] ** 2
    N = 200
    for n in range(N):
        u = orc.boris(q, m, dt, eb, u)
        ang -= 2 * math.atan(k * B / math.sqrt(1 + up2 + (u0[2] + (2 * n + 1) * k * E) ** 2))
    want = [u0[0] * math.cos(ang) - u0[1] * math.sin(ang), u0[0] * math.sin(ang) + u0[1] * math.cos(ang),
            u0[2] + 2 * N * k * E]
    np.testing.assert_allclose(u, want, rtol=0, atol=1e-11)


def test_boris_pure_electric_kick():
    """B = 0: the two half kicks add to q E dt / m exactly."""
    E = np.array([0.3, -0.2, 0.5])
    eb = np.concatenate([E, np.zeros(3)])
    u = np.array([0.1, 0.2, -0.3])
    out = orc.boris(-1.0, 2.0, 0.25, eb, u)
    np.testing.assert_allclose(out, u + (-1.0) * E * 0.25 / 2.0, rtol=0, atol=1e-15)


def test_gyration_orbit_in_full_cycle():
    """A single test particle (negligible weight) in a uniform Bz: the
    position after N cycles is the closed-form sum of the rotated velocities."""
    n, d, dt = (8, 8, 8), (0.5, 0.5, 0.5), 0.2
    sim = orc.OracleSim(3, n, d, dt, 1)
    B0 = 0.9
    sim.set_field(orc.BZ, np.full(512, B0))
    u0 = np.array([0.4, 0.1, 0.05])
    x0 = np.array([2.0, 2.0, 2.0])
    q = -1.0
    sim.add_species(q, 1.0, [x0[0]], [x0[1]], [x0[2]], [u0[0]], [u0[1]], [u0[2]], [1e-300])
    N = 37
    sim.step(N)
    g = math.sqrt(1 + u0 @ u0)
    phi = -2 * math.atan(q * B0 * dt / (2 * g))  # rotation angle per step (counter-clockwise)
    zeta = complex(math.cos(phi), math.sin(phi))
    w0 = complex(u0[0], u0[1])
    s = w0 * zeta * (1 - zeta ** N) / (1 - zeta)  # sum_{m=1..N} zeta^m w0
    L = 4.0
    want = np.array([(x0[0] + dt * s.real / g) % L, (x0[1] + dt * s.imag / g) % L,
                     (x0[2] + N * dt * u0[2] / g) % L])
    p = sim.particles(0)
    np.testing.assert_allclose([p["x"][0], p["y"][0], p["z"][0]], want, atol=1e-12)
    uz = u0[2]
    wN = w0 * zeta ** N
    np.testing.assert_allclose([p["ux"][0], p["uy"][0], p["uz"][0]], [wN.real, wN.imag, uz],
                               atol=1e-13)


def test_uniform_E_acceleration_relativistic():
    n, d, dt = (4, 4, 4), (0.5, 0.5, 0.5), 0.1
    sim = orc.OracleSim(3, n, d, dt, 2)
    E0 = 0.7
    sim.set_field(orc.EX, np.full(64, E0))
    q, m = 1.0, 3.0
    sim.add_species(q, m, [1.0], [1.0], [1.0], [0.0], [0.0], [0.0], [1e-300])
    N = 25
    sim.step(N)
    p = sim.particles(0)
    # u^{n+1/2} = n q E dt / m ; x^{n+1} = x^n + dt u / gamma
    us = [(k + 1) * q * E0 * dt / m for k in range(N)]
    x = 1.0 + sum(dt * u / math.sqrt(1 + u * u) for u in us)
    assert abs(p["ux"][0] - us[-1]) < 1e-14
    assert abs(p["x"][0] - (x % 2.0)) < 1e-13


# ------------------------------------------------------------------- Yee ---
def _yee_mode(dim, n, d, dt, kvec_int, a_vec):
    L = np.array([n[0] * d[0], n[1] * d[1], n[2] * d[2]])
    k = 2 * np.pi * np.array(kvec_int) / L
    kap = 2 * np.sin(k * np.array(d) / 2) / np.array(d)
    if dim == 2:
        kap[1] = 0.0
        k[1] = 0.0
    Om = np.linalg.norm(kap)
    w = 2 / dt * math.asin(dt * Om / 2)
    Ehat = np.cross(kap, a_vec)
    Ehat /= np.linalg.norm(Ehat)
    Bhat = np.cross(kap, Ehat) / Om
    return k, w, Ehat, Bhat


def _yee_fields(dim, n, d, k, w, Ehat, Bhat, dt, step):
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    out = []
    for c in range(6):
        sx, sy, sz = STAG[c]
        ph = k[0] * (ii + sx) * d[0] + k[2] * (kk + sz) * d[2] - w * step * dt
        if dim == 3:
            ph = ph + k[1] * (jj + sy) * d[1]
        if c < 3:
            out.append(Ehat[c] * np.cos(ph))
        else:
            out.append(Bhat[c - 3] * math.cos(w * dt / 2) * np.cos(ph))
    return out


@pytest.mark.parametrize("dim", [3, 2])
def test_yee_vacuum_dispersion(dim):
    """Yee eigenmode: after N steps the fields equal the travelling wave whose
    frequency obeys (sin(w dt/2)/dt)^2 = sum_i (sin(k_i dx_i/2)/dx_i)^2."""
    if dim == 3:
        n, d, kint, a = (12, 10, 8), (0.3, 0.35, 0.4), (1, 2, 3), np.array([0.0, 0.0, 1.0])
    else:
        n, d, kint, a = (16, 1, 12), (0.3, 1.0, 0.4), (1, 0, 2), np.array([0.0, 1.0, 0.0])
    dt = 0.9 / math.sqrt(sum(1 / v ** 2 for v, ax in zip(d, range(3)) if not (dim == 2 and ax == 1)))
    k, w, Eh, Bh = _yee_mode(dim, n, d, dt, kint, a)
    sim = orc.OracleSim(dim, n, d, dt, 1)
    for c, f in enumerate(_yee_fields(dim, n, d, k, w, Eh, Bh, dt, 0)):
        sim.set_field(c, f)
    N = 60
    sim.step(N)
    want = _yee_fields(dim, n, d, k, w, Eh, Bh, dt, N)
    for c in range(6):
        np.testing.assert_allclose(sim.field(c), want[c], rtol=0, atol=1e-12)
    # div B stays zero
    Bx, By, Bz = (sim.field(c) for c in (3, 4, 5))
    divB = (np.roll(Bx, -1, 2) - Bx) / d[0] + (np.roll(Bz, -1, 0) - Bz) / d[2]
    if dim == 3:
        divB += (np.roll(By, -1, 1) - By) / d[1]
    assert np.abs(divB).max() < 1e-12


# ------------------------------------------------------- plasma frequency ---
@pytest.mark.parametrize("order", [1, 2, 3])
def test_cold_plasma_oscillation_leapfrog_frequency(order):
    """Uniform cold electrons (lattice loaded) drifting with u0 over fixed
    ions: the k = 0 mode is the leapfrog oscillator with
    sin(w dt / 2) = w_pe dt / 2, so u^{n+1/2} = u0 cos(w (n+1/2) dt) / cos(w dt/2)."""
    n, d, dt = (4, 4, 4), (0.5, 0.5, 0.5), 0.15
    ppc_side = 2
    n0 = 1.0  # w_pe^2 = n0 q^2 / m = 1
    offs = (np.arange(ppc_side) + 0.5) / ppc_side
    pts = []
    for k, j, i in itertools.product(range(n[2]), range(n[1]), range(n[0])):
        for oz, oy, ox in itertools.product(offs, offs, offs):
            pts.append(((i + ox) * d[0], (j + oy) * d[1], (k + oz) * d[2]))
    pts = np.array(pts)
    npart = len(pts)
    w = n0 * d[0] * d[1] * d[2] / ppc_side ** 3
    u0 = 1e-6
    sim = orc.OracleSim(3, n, d, dt, order)
    sim.add_species(-1.0, 1.0, pts[:, 0], pts[:, 1], pts[:, 2], np.full(npart, u0),
                    np.zeros(npart), np.zeros(npart), np.full(npart, w))
    wfreq = 2 / dt * math.asin(dt * math.sqrt(n0) / 2)
    for step in range(1, 60):
        sim.step(1)
        ux = sim.particles(0)["ux"]
        want = u0 * math.cos(wfreq * (step - 0.5) * dt) / math.cos(wfreq * dt / 2)
        assert np.abs(ux - want).max() < 1e-9 * u0


# ------------------------------------------------------ charge continuity ---
def _random_plasma(dim, n, d, rng, npart, umax):
    L = [n[a] * d[a] for a in range(3)]
    x = rng.uniform(0, L[0], npart)
    y = rng.uniform(0, L[1], npart) if dim == 3 else np.zeros(npart)
    z = rng.uniform(0, L[2], npart)
    u = rng.normal(size=(3, npart))
    u *= umax / np.maximum(np.linalg.norm(u, axis=0), 1e-300) * rng.uniform(0, 1, npart)
    w = rng.uniform(0.5, 1.5, npart)
    return x, y, z, u[0], u[1], u[2], w


def _div_nodes(dim, n, d, Fx, Fy, Fz):
    div = (Fx - np.roll(Fx, 1, 2)) / d[0] + (Fz - np.roll(Fz, 1, 0)) / d[2]
    if dim == 3:
        div += (Fy - np.roll(Fy, 1, 1)) / d[1]
    return div


@pytest.mark.parametrize("dim,order", [(3, 1), (3, 2), (3, 3), (2, 1), (2, 2), (2, 3)])
def test_esirkepov_discrete_continuity(dim, order):
    """(rho^{n+1} - rho^n)/dt + div J^{n+1/2} = 0 at every node (Esirkepov
    2001), with rho deposited by S at the nodes; fast particles so that many
    cross cell boundaries."""
    n = (6, 5 if dim == 3 else 1, 7)
    d = (0.4, 0.5 if dim == 3 else 1.0, 0.45)
    inv = sum(1 / d[a] ** 2 for a in range(3) if not (dim == 2 and a == 1))
    dt = 0.99 / math.sqrt(inv)
    rng = np.random.default_rng(10 + dim + order)
    sim = orc.OracleSim(dim, n, d, dt, order)
    parts = _random_plasma(dim, n, d, rng, 300, umax=3.0)
    sim.add_species(-1.0, 1.0, *parts)
    sim.add_species(2.0, 5.0, *_random_plasma(dim, n, d, rng, 200, umax=1.0))
    # random smooth fields to get varied pushes
    for c in range(6):
        sim.set_field(c, 0.3 * rng.normal(size=sim.ncell))
    rho0 = sim.rho()
    sim.step(1)
    rho1 = sim.rho()
    J = [sim.field(c) for c in (orc.JX, orc.JY, orc.JZ)]
    res = (rho1 - rho0) / dt + _div_nodes(dim, n, d, *J)
    scale = np.abs(rho0).max() / dt
    assert np.abs(res).max() < 1e-13 * scale
    assert np.abs(J[0]).max() > 1e-3 * scale * d[0]  # currents are not trivially zero


@pytest.mark.parametrize("dim,order", [(3, 1), (3, 2), (3, 3), (2, 2), (2, 3)])
def test_gauss_law_residual_preserved(dim, order):
    """Charge-conserving deposit + Yee: div E - rho changes by roundoff only."""
    n = (6, 6 if dim == 3 else 1, 6)
    d = (0.5, 0.5 if dim == 3 else 1.0, 0.5)
    inv = sum(1 / d[a] ** 2 for a in range(3) if not (dim == 2 and a == 1))
    dt = 0.95 / math.sqrt(inv)
    rng = np.random.default_rng(20 + dim + order)
    sim = orc.OracleSim(dim, n, d, dt, order)
    sim.add_species(-1.0, 1.0, *_random_plasma(dim, n, d, rng, 400, umax=0.8))
    sim.add_species(1.0, 1836.15267343, *_random_plasma(dim, n, d, rng, 400, umax=0.01))

    def residual():
        E = [sim.field(c) for c in (orc.EX, orc.EY, orc.EZ)]
        return _div_nodes(dim, n, d, *E) - sim.rho()

    r0 = residual()
    scale = np.abs(sim.rho()).max()
    for _ in range(8):
        sim.step(1)
        assert np.abs(residual() - r0).max() < 1e-13 * scale


# --------------------------------------------------------------- antenna ---
def test_antenna_radiates_amplitude_a0():
    """A sheet current Jx = 2 a0 / dz radiates a plane wave of amplitude a0
    (|E| = |K| / 2 for a current sheet K with c = mu0 = 1)."""
    n, d = (4, 1, 256), (0.2, 1.0, 0.2)
    dt = 0.98 * d[2]
    sim = orc.OracleSim(2, n, d, dt, 1, absorb_cells=40)
    a0 = 0.5
    sim.set_laser(a0, 1e9, 1e9, 0.0, 1.0, 0.0, 0.0, 60)
    sim.step(300)
    ex = sim.field(orc.EX)[:, 0, 0]
    # forward wave region ahead of the antenna, away from the absorbing layer
    seg = ex[90:200]
    assert 0.97 * a0 < np.abs(seg).max() < 1.03 * a0


def test_antenna_forward_wave_is_half_the_sheet_current_at_the_retarded_time():
    """A current sheet K(t) x-hat at z0 radiates Ex(z, t) = -K(t - |z - z0|) / 2
    (c = mu0 = 1), here K = 2 a0 env(t) with env(t) = exp(-((t - tp)/tau)^2)
    sin(omega (t - tp)): the pulse's shape, sign, timing and delay one probe
    downstream.  Periodic z, long enough that nothing comes back in time; the
    Yee grid resolves the pulse to 0.1 % (a time offset of half a step already
    costs 2 %)."""
    dz, dt = 0.05, 0.04
    a0, tau, tp, om, kant, D = 0.5, 4.0, 12.0, 1.0, 60, 200
    sim = orc.OracleSim(2, (4, 1, 1400), (0.2, 1.0, dz), dt, 1)
    sim.set_laser(a0, 1e9, tau, tp, om, 0.0, 0.0, kant)
    ts, ex = [], []
    for step in range(int((tp + D * dz + 3 * tau) / dt)):
        sim.step(1)
        ts.append((step + 1) * dt)
        ex.append(sim.field(orc.EX)[kant + D, 0, 0])
    tr = np.array(ts) - D * dz - tp
    want = -a0 * np.exp(-(tr / tau) ** 2) * np.sin(om * tr)
    assert np.abs(np.array(ex) - want).max() < 5e-3 * a0


def test_antenna_transverse_profile_is_gaussian_in_the_waist():
    """Near the antenna (2 cells of 0.1 against a Rayleigh length of 72) the
    wave keeps the sheet's transverse profile exp(-x^2 / w0^2) (w0 the 1/e
    radius of the field): the envelope of |Ex| across x matches it to 1 %;
    reading w0 as the 1/e^2 radius or the Gaussian's sigma is off by 25 %."""
    nx, nz, dx, dz, dt = 512, 260, 0.2, 0.1, 0.06
    a0, w0, tau, tp, om, kant, D = 0.5, 12.0, 4.0, 12.0, 1.0, 30, 20
    xc = nx * dx / 2
    sim = orc.OracleSim(2, (nx, 1, nz), (dx, 1.0, dz), dt, 1)
    sim.set_laser(a0, w0, tau, tp, om, xc, 0.0, kant)
    env = np.zeros(nx)
    for _ in range(int((tp + D * dz + 2.5 * tau) / dt)):
        sim.step(1)
        env = np.maximum(env, np.abs(sim.field(orc.EX)[kant + D, 0, :]))
    x = (np.arange(nx) + 0.5) * dx - xc
    assert np.abs(env / env.max() - np.exp(-x ** 2 / w0 ** 2)).max() < 0.02


def test_damping_layer_absorbs_outgoing_pulse():
    n, d = (4, 1, 200), (0.2, 1.0, 0.2)
    dt = 0.98 * d[2]
    sim = orc.OracleSim(2, n, d, dt, 1, absorb_cells=40)
    sim.set_laser(1.0, 1e9, 2.0, 6.0, 1.0, 0.0, 0.0, 100)
    sim.step(90)
    e_mid = sum(float((sim.field(c) ** 2).sum()) for c in range(6))
    sim.step(260)
    e_end = sum(float((sim.field(c) ** 2).sum()) for c in range(6))
    assert e_mid > 0 and e_end < 0.05 * e_mid


@pytest.mark.parametrize("dim,which", [(3, "A4"), (2, "A4"), (3, "A8")])
def test_damping_profile_exact_on_a_uniform_field(dim, which):
    """The damping profile layer by layer, bit for bit.  A uniform field is
    curl-free, so with no particles and no laser one step leaves E and B
    unchanged exactly until the layers scale them: afterwards every component
    in cell layer k must equal its uniform value times the hand-computed factor
    of the absorbing-layer reading (tests/golden/damping_profile.json: 1/2 in
    the outermost layer of each end, 1 inside the domain).  The values are
    exact binary fractions, so a profile linear in the depth, a dropped 1/2,
    a depth counted from 0 or a layer at the wrong end all fail."""
    g = json.load(open(os.path.join(HERE, "golden", "damping_profile.json")))
    if which == "A4":
        A, nz, fac = g["A"], g["nz"], [Fraction(x) for x in g["factor_by_layer"]]
    else:
        A, nz, fac = 8, g["A8_nz"], [Fraction(x) for x in g["A8_factor_by_layer"]]
    n = (4, 4 if dim == 3 else 1, nz)
    d = (0.5, 0.5 if dim == 3 else 1.0, 0.5)
    sim = orc.OracleSim(dim, n, d, 0.2, 1, absorb_cells=A)
    values = [1.0, -2.0, 0.5, 0.25, -1.5, 3.0]  # Ex Ey Ez Bx By Bz
    for c, v in enumerate(values):
        sim.set_field(c, np.full((n[2], n[1], n[0]), v))
    sim.step(1)
    for c, v in enumerate(values):
        f = sim.field(c)
        for k in range(nz):
            want = float(Fraction(v) * fac[k])
            assert np.all(f[k] == want), (c, k, np.unique(f[k]), want)


def test_absorbed_particles_are_removed_by_id():
    n, d, dt = (4, 4, 16), (0.5, 0.5, 0.5), 0.2
    sim = orc.OracleSim(3, n, d, dt, 1, absorb_cells=2)
    # z layer boundaries at 1.0 and 7.0
    sim.add_species(-1.0, 1.0, [1.0, 1.0, 1.0], [1.0, 1.0, 1.0], [1.02, 4.0, 6.98],
                    [0, 0, 0], [0, 0, 0], [-0.5, 0.0, 0.5], [1e-300] * 3, ids=[7, 8, 9])
    sim.step(1)
    p = sim.particles(0)
    assert list(p["id"]) == [8]


# -------------------------------------------------------- load balancing ---
def test_fig1_efficiency_from_paper():
    g = json.load(open(os.path.join(HERE, "golden", "fig1_lb_example.json")))
    costs = np.array(g["particle_counts"], dtype=float)
    E = orc.lb_efficiency(costs, g["mapping_b"], g["n_ranks"])
    assert E == g["efficiency_mapping_b_particle_cost"]
    # a knapsack mapping of the same costs puts the two loaded boxes on
    # different ranks: E = 15 / 18
    a = orc.knapsack(costs, 2)
    assert a[0] != a[3]
    assert orc.lb_efficiency(costs, a, 2) == pytest.approx(15 / 18, abs=1e-15)
    s = orc.sfc(costs, g["box_ijk"], 2, 2)
    assert orc.lb_efficiency(costs, s, 2) >= 0.5


def test_efficiency_edge_cases():
    assert orc.lb_efficiency([0, 0, 0], [0, 1, 1], 2) == 1.0
    assert orc.lb_efficiency([1, 1, 1, 1], [0, 1, 0, 1], 2) == 1.0
    assert orc.lb_efficiency([4, 0], [0, 0], 4) == 0.25


def _brute_opt(costs, m):
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = [0.0] * m
        for c, a in zip(costs, assign):
            loads[a] += c
        best = min(best, max(loads))
    return best


def test_knapsack_graham_bound_against_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(60):
        nb = int(rng.integers(1, 9))
        m = int(rng.integers(1, 4))
        costs = rng.integers(0, 20, nb).astype(float)
        a = orc.knapsack(costs, m, cap_factor=1e9)  # uncapped: plain LPT
        loads = np.bincount(a, weights=costs, minlength=m)
        opt = _brute_opt(costs, m)
        assert loads.max() >= opt - 1e-12
        assert loads.max() <= (4 / 3 - 1 / (3 * m)) * opt + 1e-12


def test_knapsack_tie_rules_and_cap():
    # equal costs: lower box index first, lowest worker id wins ties
    a = orc.knapsack([1.0, 1.0, 1.0, 1.0], 2)
    assert list(a) == [0, 1, 0, 1]
    # cap: 6 boxes, 3 workers, cap = max(ceil(2), floor(1.5*2)) = 3 boxes per worker
    costs = [100.0, 1.0, 1.0, 1.0, 1.0, 1.0]
    a = orc.knapsack(costs, 3)
    cnt = np.bincount(a, minlength=3)
    assert cnt.max() <= 3 and a[0] == 0
    # with cap_factor 1.0 the cap is 2 boxes per worker
    a = orc.knapsack(costs, 3, cap_factor=1.0)
    assert np.bincount(a, minlength=3).max() <= 2


def test_morton_keys_by_hand():
    assert orc.morton(3, 1, 0, 0) == 1
    assert orc.morton(3, 0, 1, 0) == 2
    assert orc.morton(3, 0, 0, 1) == 4
    assert orc.morton(3, 1, 1, 1) == 7
    assert orc.morton(3, 2, 0, 0) == 8
    assert orc.morton(3, 3, 5, 6) == 427
    assert orc.morton(2, 1, 0, 0) == 1
    assert orc.morton(2, 0, 0, 1) == 2
    assert orc.morton(2, 3, 0, 1) == 7
    # 4x4 2D grid: the Z curve visits (0,0) (1,0) (0,1) (1,1) (2,0) ...
    order = sorted(((x, z) for x in range(4) for z in range(4)), key=lambda p: orc.morton(2, p[0], 0, p[1]))
    assert order[:8] == [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (3, 0), (2, 1), (3, 1)]


def _contiguous_opt(costs, m):
    """min over contiguous partitions of the sequence into m pieces of the max piece sum (DP)."""
    nb = len(costs)
    pre = np.concatenate([[0.0], np.cumsum(costs)])
    INF = float("inf")
    f = [[INF] * (nb + 1) for _ in range(m + 1)]
    f[0][0] = 0.0
    for k in range(1, m + 1):
        for i in range(nb + 1):
            for j in range(i + 1):
                f[k][i] = min(f[k][i], max(f[k - 1][j], pre[i] - pre[j]))
    return f[m][nb]


def test_sfc_contiguous_and_bounded():
    rng = np.random.default_rng(6)
    ijk = np.array([(x, y, z) for z in range(2) for y in range(2) for x in range(4)], dtype=np.int32)
    for trial in range(30):
        costs = rng.lognormal(0, 1.5, len(ijk))
        m = int(rng.integers(1, 6))
        a = orc.sfc(costs, ijk, 3, m)
        keys = [orc.morton(3, *p) for p in ijk]
        seq = np.argsort(keys)
        # worker ids are non-decreasing along the curve (contiguous pieces)
        assert np.all(np.diff(a[seq]) >= 0)
        loads = np.bincount(a, weights=costs, minlength=m)
        opt = _contiguous_opt(list(costs[seq]), m)
        assert loads.max() >= opt - 1e-12
        assert loads.max() <= costs.sum() / m + costs.max() + 1e-12


def test_threshold_meets_or_exceeds():
    assert orc.lb_adopt(0.5, 0.625, 0.25)
    assert not orc.lb_adopt(0.5, 0.62499999, 0.25)
    assert orc.lb_adopt(0.5, 0.5, 0.0)


def test_performance_model_paper_values():
    """Sec. 4: c_max0/c_avg0 = 6.2 with x = 0.91 (2D3V) or 0.88 (3D3V) gives a
    best speedup of about 5x."""
    for x in (0.91, 0.88):
        s = orc.predicted_speedup(1 / 6.2, x)
        assert round(s) == 5
    assert orc.predicted_speedup(1.0, 0.9) == 1.0


# ------------------------------------------- in-cell line-integral current ---
def _gl3(f):
    """3-point Gauss-Legendre on [0, 1]: exact for polynomials of degree <= 5."""
    xs = [0.5 - 0.5 * math.sqrt(0.6), 0.5, 0.5 + 0.5 * math.sqrt(0.6)]
    ws = [5 / 18, 8 / 18, 5 / 18]
    return sum(w * f(x) for w, x in zip(ws, xs))


@pytest.mark.parametrize("dim", [3, 2])
def test_linear_deposit_equals_line_integral_for_in_cell_motion(dim):
    """With linear shapes and a straight move that stays inside one cell, the
    charge-conserving current through each cell face is the exact time
    integral of q v S(y(t)) S(z(t)) along the path (Villasenor-Buneman); this
    pins every Esirkepov weight term, including the 2D out-of-plane Jy."""
    n = (6, 6 if dim == 3 else 1, 6)
    d = (0.5, 0.5 if dim == 3 else 1.0, 0.5)
    dt = 0.1
    rng = np.random.default_rng(40 + dim)
    for trial in range(10):
        sim = orc.OracleSim(dim, n, d, dt, 1)
        X0 = np.array([2.0, 2.0 if dim == 3 else 0.0, 3.0]) + rng.uniform(0.2, 0.8, 3)
        if dim == 2:
            X0[1] = 0.0
        u = rng.uniform(-0.5, 0.5, 3)
        g = math.sqrt(1 + u @ u)
        v = u / g
        dX = v * dt / np.array(d)
        if dim == 2:
            dX[1] = 0.0
        q, w = -1.0, 0.7
        pos = X0 * np.array(d)
        sim.add_species(q, 1.0, [pos[0]], [pos[1]], [pos[2]], [u[0]], [u[1]], [u[2]], [w])
        sim.step(1)  # zero fields: the push leaves u unchanged
        J = [sim.field(c) for c in (orc.JX, orc.JY, orc.JZ)]
        V = d[0] * d[1] * d[2]
        i0 = np.floor(X0).astype(int)

        def hat(t, a, node):
            return max(0.0, 1 - abs(X0[a] + t * dX[a] - node))

        want = [np.zeros_like(J[0]) for _ in range(3)]
        ys = [i0[1], i0[1] + 1] if dim == 3 else [0]
        for kk in (i0[2], i0[2] + 1):
            for jj in ys:
                for ii in (i0[0], i0[0] + 1):
                    hy = (lambda t, jj=jj: hat(t, 1, jj)) if dim == 3 else (lambda t: 1.0)
                    if ii == i0[0]:
                        want[0][kk, jj, ii] = q * w * v[0] / V * _gl3(lambda t: hy(t) * hat(t, 2, kk))
                    if kk == i0[2]:
                        want[2][kk, jj, ii] = q * w * v[2] / V * _gl3(lambda t: hat(t, 0, ii) * hy(t))
                    if dim == 3 and jj == i0[1]:
                        want[1][kk, jj, ii] = q * w * v[1] / V * _gl3(lambda t: hat(t, 0, ii) * hat(t, 2, kk))
                    if dim == 2:
                        want[1][kk, jj, ii] = q * w * v[1] / V * _gl3(lambda t: hat(t, 0, ii) * hat(t, 2, kk))
        for c in range(3):
            np.testing.assert_allclose(J[c], want[c], rtol=0, atol=1e-14)


# ------------------------------------------------------------ box binning ---
def test_bin_particles_by_hand():
    """4 x 2 x 1 cells in boxes of 2 x 1 x 1 (dx = 0.5): boxes (0,0) (1,0) (0,1) (1,1)."""
    x = [0.2, 1.9, 0.7, 1.2, 0.4, -0.1, 2.0]   # -0.1 and 2.0 wrap to cells 3 and 0
    y = [0.1, 0.9, 0.6, 0.2, 0.8, 0.3, 0.7]
    z = [0.0] * 7
    off, perm = orc.bin_particles(3, (4, 2, 1), (0.5, 0.5, 0.5), (2, 1, 1), x, y, z)
    # cells: p0 (0,0) p1 (3,1) p2 (1,1) p3 (2,0) p4 (0,1) p5 (3,0) p6 (0,1)
    # boxes: p0 0, p1 3, p2 2, p3 1, p4 2, p5 1, p6 2
    assert list(off) == [0, 1, 3, 6, 7]
    assert list(perm) == [0, 3, 5, 2, 4, 6, 1]


def test_box_counts_by_hand():
    """The per-box particle counts of a simulation, for the hand case of the
    binning test: 4 x 2 x 1 cells of 0.5 in boxes of 2 x 1 x 1; positions just
    outside the domain count in the periodic image."""
    sim = orc.OracleSim(3, (4, 2, 1), (0.5, 0.5, 0.5), 0.1, 1)
    x = [0.2, 1.9, 0.7, 1.2, 0.4, -0.1, 2.0]
    y = [0.1, 0.9, 0.6, 0.2, 0.8, 0.3, 0.7]
    sim.add_species(-1.0, 1.0, x, y, [0.1] * 7, [0.0] * 7, [0.0] * 7, [0.0] * 7, [1.0] * 7)
    assert list(sim.box_counts((2, 1, 1)).ravel()) == [1, 2, 3, 1]


def test_periodic_positions_stay_in_the_domain():
    """Fast particles (|u| up to 3, several cells per step) in a small periodic
    box: after every step each coordinate lies in [0, L), wrapped at both ends,
    and none is lost."""
    rng = np.random.default_rng(7)
    n, d = (6, 5, 4), (0.3, 0.4, 0.5)
    L = [n[a] * d[a] for a in range(3)]
    npart = 400
    sim = orc.OracleSim(3, n, d, 0.09, 2)
    sim.add_species(-1.0, 1.0, rng.uniform(0, L[0], npart), rng.uniform(0, L[1], npart),
                    rng.uniform(0, L[2], npart), *(rng.uniform(-3, 3, (3, npart))), np.full(npart, 1e-3))
    for _ in range(20):
        sim.step(1)
        p = sim.particles(0)
        assert len(p["x"]) == npart
        for a, k in enumerate(("x", "y", "z")):
            assert p[k].min() >= 0.0 and p[k].max() < L[a]


# ------------------------------------------- energy-conserving gather ---
def _gl3_on(f, a, b):
    """3-point Gauss-Legendre on [a, b] (interior nodes only, so a jump at
    an end does not matter): exact for polynomials of degree <= 5."""
    return (b - a) * _gl3(lambda s: f(a + s * (b - a)))


@pytest.mark.parametrize("dim,order", [(3, 1), (3, 2), (3, 3), (2, 1), (2, 2), (2, 3)])
def test_energy_conserving_gather_is_the_transpose_of_esirkepov(dim, order):
    """For a straight move along one axis a, the Esirkepov current J_a is
    the path integral of the order-(n-1) shape on the half-node grid times the
    order-n transverse shapes (the B-spline derivative identity), so for any
    grid field G on the J_a locations
        sum_cells J_a G dV dt = q w * integral over the path of G gathered with
        order n - 1 along a and order n across it,
    which is the energy-conserving gather of E_a.  The gather is piecewise
    polynomial of degree <= 3 between multiples of half a cell, so Gauss-
    Legendre quadrature on those pieces is exact.  The default gather (order n along a)
    misses the identity, which the last check shows."""
    n = (10, 10 if dim == 3 else 1, 10)
    d = (0.5, 0.6 if dim == 3 else 1.0, 0.7)
    dt = 0.99 / math.sqrt(sum(1 / x ** 2 for x in (d if dim == 3 else (d[0], d[2]))))
    rng = np.random.default_rng(70 + 10 * dim + order)
    axes = (0, 1, 2) if dim == 3 else (0, 2)
    for a in axes:
        for trial in range(4):
            X0 = rng.uniform(4.0, 6.0, 3)
            if dim == 2:
                X0[1] = 0.0
            u = np.zeros(3)
            u[a] = rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 6.0)
            q, w = rng.choice([-1.0, 1.0]), rng.uniform(0.3, 2.0)
            pos = X0 * np.array(d)
            sim = orc.OracleSim(dim, n, d, dt, order)
            sim.add_species(q, 1.0, [pos[0]], [pos[1]], [pos[2]], [u[0]], [u[1]], [u[2]], [w])
            sim.step(1)  # zero fields: the push leaves u unchanged
            J = sim.field(orc.JX + a)
            G = rng.normal(size=J.shape)
            lhs = float((J * G).sum()) * d[0] * d[1] * d[2] * dt
            X1 = X0.copy()
            X1[a] = sim.particles(0)[("x", "y", "z")[a]][0] / d[a]
            rhs = {}
            for ec in (True, False):
                probe = orc.OracleSim(dim, n, d, dt, order)
                probe.set_gather(ec)
                probe.set_field(orc.EX + a, G)

                def field_at(t):
                    P = X0.copy()
                    P[a] = t
                    return probe.gather(*(P * np.array(d)))[a]

                lo, hi = sorted((X0[a], X1[a]))
                cuts = [lo] + [k / 2 for k in range(math.floor(2 * lo) + 1, math.ceil(2 * hi))] + [hi]
                integ = sum(_gl3_on(field_at, cuts[m], cuts[m + 1]) for m in range(len(cuts) - 1))
                rhs[ec] = q * w * d[a] * integ * (1.0 if X1[a] >= X0[a] else -1.0)
            assert abs(lhs - rhs[True]) <= 1e-12 * max(abs(lhs), 1e-300), (a, trial, lhs, rhs[True])
            assert abs(lhs - rhs[False]) > 1e-6 * abs(lhs), (a, trial)


# variance of the centred B-spline of order m (m + 1 unit boxes convolved)
_BSPLINE_VAR = {1: 1 / 6, 2: 1 / 4, 3: 1 / 3}


@pytest.mark.parametrize("dim,order", [(3, 1), (3, 2), (3, 3), (2, 2)])
def test_energy_conserving_gather_orders_per_direction(dim, order):
    """A field equal to the square of a grid coordinate, h^2, gathered with a
    centred B-spline of order m >= 2 gives x^2 + (m + 1)/12 (splines of degree
    >= 2 reproduce quadratics; the constant is the spline's variance), with
    the hat (m = 1) x^2 + t (1 - t), t the fraction of x on that grid.  So each component shows,
    direction by direction, which order it was gathered with: order - 1 along
    the directions where it sits at half nodes (Ex along x; Bx along y and z;
    ...), order n elsewhere; order 0 picks the nearest half node."""
    n = (14, 14 if dim == 3 else 1, 14)
    d = (1.0, 1.0, 1.0)
    sim = orc.OracleSim(dim, n, d, 0.1, order)
    sim.set_gather(True)
    rng = np.random.default_rng(90 + order)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = (i, j, k)
    axes = (0, 1, 2) if dim == 3 else (0, 2)
    for a in axes:
        for c in range(6):
            h = idx[a] + STAG[c][a]
            for comp in range(6):
                sim.set_field(comp, np.zeros(i.shape))
            sim.set_field(c, h.astype(np.float64) ** 2)
            for _ in range(12):
                P = rng.uniform(5.0, 9.0, 3)
                if dim == 2:
                    P[1] = 0.0
                got = sim.gather(*P)[c]
                m = order - 1 if STAG[c][a] == 0.5 else order
                x = P[a]
                if m == 0:  # nearest half node
                    want = (math.floor(x) + 0.5) ** 2
                elif m == 1:  # linear interpolation of h^2: x^2 + t (1 - t)
                    t = (x - STAG[c][a]) - math.floor(x - STAG[c][a])
                    want = x * x + t * (1.0 - t)
                else:
                    want = x * x + _BSPLINE_VAR[m]
                assert abs(got - want) < 1e-12, (a, c, order, got, want)
