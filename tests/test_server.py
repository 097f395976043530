"""Request server (include/pic_server.h): continuous batching of independent
PIC simulations packed into one persistent particle launch per tick.  Each
request's result must be the same alone and in a mix of requests that arrive
and leave while it runs (only the order of atomic current sums may differ),
and an explicit-array request must match the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle as orc
from paper_2104_11385_gb300 import _lib as L
from paper_2104_11385_gb300 import workloads
from paper_2104_11385_gb300.server import Server

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _run_one(srv, rid):
    while srv.poll(rid)["state"] != L.REQ_DONE:
        srv.tick()


def _result(srv, rid, ncell):
    f = [srv.read_field(rid, c, ncell) for c in (L.EX, L.EZ, L.BY, L.JX)]
    p = srv.particles(rid, 0)
    o = np.argsort(p["id"])
    return f, {k: v[o] for k, v in p.items()}


A = dict(ncell=(64, 1, 64), box=(32, 1, 32), dx=(0.2, 1.0, 0.2), nsteps=40,
         plasma=dict(ppc=4, density=1.0, u_th=0.05, ripple=0.05, seed=11))


def test_request_alone_equals_request_in_a_mix():
    alone = Server(dim=2, max_active=8)
    ra = alone.submit(**A)
    _run_one(alone, ra)
    ref = _result(alone, ra, A["ncell"])

    mix = Server(dim=2, max_active=8)
    others = [
        mix.submit((128, 1, 128), (32, 1, 32), (0.2, 1, 0.2), 60, plasma=dict(ppc=8, seed=3)),
        mix.submit((256, 1, 64), (32, 1, 32), (0.3, 1, 0.3), 15, plasma=dict(ppc=2, seed=4)),
    ]
    for _ in range(5):
        mix.tick()
    rb = mix.submit(**A)  # arrives while the others are on the GPU
    late = None
    for t in range(200):
        if t == 7:
            late = mix.submit((64, 1, 128), (32, 1, 32), (0.2, 1, 0.2), 80, plasma=dict(ppc=16, seed=5))
        mix.tick()
        if mix.poll(rb)["state"] == L.REQ_DONE:
            break
    assert mix.poll(rb)["state"] == L.REQ_DONE
    # the mix really overlapped: the first request was still running when A finished
    assert mix.poll(others[0])["state"] == L.REQ_ACTIVE and mix.poll(late)["state"] == L.REQ_ACTIVE
    got = _result(mix, rb, A["ncell"])
    for fg, fr in zip(got[0], ref[0]):
        assert rel(fg, fr) < TOL
    for k in ("x", "z", "ux", "uy", "uz"):
        assert rel(got[1][k], ref[1][k]) < TOL
    assert np.array_equal(got[1]["id"], ref[1]["id"])
    mix.run_until_idle()
    assert mix.stats()["finished"] == 4


def test_explicit_request_in_a_mix_matches_oracle():
    n, box, dx = (48, 1, 64), (16, 1, 32), (0.3, 1.0, 0.3)
    wl = workloads.random_plasma(21, 2, n, box, dx, 1, nspecies=2, npart=3000, umax=1.5)
    srv = Server(dim=2, max_active=4)
    srv.submit((96, 1, 96), (32, 1, 32), (0.25, 1, 0.25), 30, plasma=dict(ppc=4, seed=9))
    rid = srv.submit(n, box, dx, 10, dt=wl["dt"], species=wl["species"])
    _run_one(srv, rid)
    ref = orc.OracleSim(2, n, dx, wl["dt"], 1)
    for sp in wl["species"]:
        ref.add_species(sp["q"], sp["m"], sp["x"], sp["y"], sp["z"], sp["ux"], sp["uy"], sp["uz"], sp["w"], sp["id"])
    ref.step(10)
    for c in (L.EX, L.EY, L.EZ, L.BX, L.BY, L.BZ, L.JX, L.JY, L.JZ):
        assert rel(srv.read_field(rid, c, n), ref.field(c)) < TOL
    for s in range(2):
        g, r = srv.particles(rid, s), ref.particles(s)
        gi, ri = np.argsort(g["id"]), np.argsort(r["id"])
        assert np.array_equal(g["id"][gi], r["id"][ri])
        for k in ("ux", "uz"):
            assert rel(g[k][gi], r[k][ri]) < TOL


def test_admission_by_footprint():
    probe = Server(dim=2, max_active=4, hbm_budget_bytes=1 << 40)
    r0 = probe.submit((128, 1, 128), (32, 1, 32), (0.2, 1, 0.2), 5, plasma=dict(ppc=8))
    est = probe.footprint(r0)
    probe.tick()
    assert probe.footprint(r0) == est  # the estimate is the allocation
    probe.close()

    # budget for one such request at a time: the second waits for memory
    srv = Server(dim=2, max_active=4, hbm_budget_bytes=int(est * 1.5))
    a = srv.submit((128, 1, 128), (32, 1, 32), (0.2, 1, 0.2), 5, plasma=dict(ppc=8, seed=1))
    b = srv.submit((128, 1, 128), (32, 1, 32), (0.2, 1, 0.2), 5, plasma=dict(ppc=8, seed=2))
    for _ in range(8):
        srv.tick()
    assert srv.poll(a)["state"] == L.REQ_DONE
    assert srv.poll(b)["state"] == L.REQ_PENDING  # a's results still hold the memory
    srv.release(a)
    srv.run_until_idle()
    assert srv.poll(b)["state"] == L.REQ_DONE
    # a request that can never fit is refused at submission
    with pytest.raises(L.PicError) as ei:
        srv.submit((512, 1, 512), (32, 1, 32), (0.2, 1, 0.2), 5, plasma=dict(ppc=64))
    assert ei.value.status == L.PIC_ENOMEM
    # results of unfinished requests are not readable
    c = srv.submit((64, 1, 64), (32, 1, 32), (0.2, 1, 0.2), 50, plasma=dict(ppc=1))
    with pytest.raises(L.PicError):
        srv.read_field(c, L.EX, (64, 1, 64))


@pytest.mark.parametrize("order", [1, 2, 3])
def test_footprint_estimate_is_the_allocation(order):
    """The admission estimate equals the bytes the request then allocates, for
    every serving grid side and a spread of ppc (guards widen with the shape
    order), so the HBM budget holds for what is actually allocated."""
    srv = Server(dim=2, shape_order=order, max_active=8, hbm_budget_bytes=1 << 40)
    rids = []
    for side, ppc in ((64, 1), (128, 64), (256, 4), (512, 2)):
        rid = srv.submit((side, 1, side), (32, 1, 32), (0.2, 1, 0.2), 3, plasma=dict(ppc=ppc))
        rids.append((rid, srv.footprint(rid)))
    srv.tick()
    for rid, est in rids:
        assert srv.poll(rid)["state"] in (L.REQ_ACTIVE, L.REQ_DONE)
        assert srv.footprint(rid) == est
    srv.close()


def test_langmuir_ripple_oscillates_at_plasma_frequency():
    """Self-checking request: the k = 2 pi / Lx density ripple of a cold plasma
    oscillates at about omega_pe = 1, so Ex reverses sign after half a period."""
    n, dx = (64, 1, 32), (0.5, 1.0, 0.5)
    srv = Server(dim=2, max_active=2)
    dt = 0.95 / np.sqrt(1 / dx[0] ** 2 + 1 / dx[2] ** 2)
    half = int(round(np.pi / dt))
    r1 = srv.submit(n, (32, 1, 32), dx, half // 2, plasma=dict(ppc=16, u_th=1e-4, ripple=0.02, seed=5))
    r2 = srv.submit(n, (32, 1, 32), dx, half // 2 + half, plasma=dict(ppc=16, u_th=1e-4, ripple=0.02, seed=5))
    srv.run_until_idle()
    e1 = srv.read_field(r1, L.EX, n).mean(axis=(0, 1))
    e2 = srv.read_field(r2, L.EX, n).mean(axis=(0, 1))
    c = float(np.dot(e1, e2) / np.sqrt(np.dot(e1, e1) * np.dot(e2, e2)))
    assert c < -0.8, c


def test_cancel_pending_and_active_requests():
    """A withdrawn request leaves between ticks: a pending one is never
    admitted, an active one frees its slot and memory for the next pending
    request, and a request still running finishes with its result alone."""
    alone = Server(dim=2, max_active=8)
    ra = alone.submit(**A)
    _run_one(alone, ra)
    ref = _result(alone, ra, A["ncell"])
    alone.close()

    srv = Server(dim=2, max_active=2)
    busy = srv.submit((128, 1, 128), (32, 1, 32), (0.2, 1, 0.2), 500, plasma=dict(ppc=8, seed=3))
    rb = srv.submit(**A)
    waiting = srv.submit((64, 1, 64), (32, 1, 32), (0.2, 1, 0.2), 20, plasma=dict(ppc=2, seed=6))
    dropped = srv.submit((64, 1, 64), (32, 1, 32), (0.2, 1, 0.2), 20, plasma=dict(ppc=2, seed=7))
    for _ in range(5):
        srv.tick()
    assert srv.poll(busy)["state"] == L.REQ_ACTIVE and srv.poll(waiting)["state"] == L.REQ_PENDING
    held = srv.stats()["bytes_in_use"]
    srv.cancel(dropped)
    srv.cancel(busy)
    assert srv.stats()["bytes_in_use"] == held - srv.footprint(busy)
    assert srv.poll(busy)["state"] == L.REQ_CANCELLED and srv.poll(busy)["steps"] == 5
    srv.tick()
    assert srv.poll(waiting)["state"] == L.REQ_ACTIVE  # took the freed slot
    srv.run_until_idle()
    assert srv.poll(dropped)["state"] == L.REQ_CANCELLED and srv.poll(dropped)["t_admit"] < 0
    assert srv.poll(waiting)["state"] == L.REQ_DONE and srv.stats()["finished"] == 2
    got = _result(srv, rb, A["ncell"])
    for fg, fr in zip(got[0], ref[0]):
        assert rel(fg, fr) < TOL
    for k in ("x", "z", "ux", "uy", "uz"):
        assert rel(got[1][k], ref[1][k]) < TOL
    assert np.array_equal(got[1]["id"], ref[1]["id"])
    # a cancelled request has no results; finished or cancelled ones cannot be cancelled
    with pytest.raises(L.PicError) as ei:
        srv.read_field(busy, L.EX, (128, 1, 128))
    assert ei.value.status == L.PIC_ESTATE
    for rid in (busy, rb):
        with pytest.raises(L.PicError) as ei:
            srv.cancel(rid)
        assert ei.value.status == L.PIC_ESTATE
    with pytest.raises(L.PicError) as ei:
        srv.cancel(10_000)
    assert ei.value.status == L.PIC_EINVAL


def test_request_rejected_at_admission_fails_alone():
    """A request that passes submission but that the simulation set-up rejects
    (an odd number of cells along x) fails by itself, and the requests behind
    it are admitted and finish."""
    srv = Server(dim=2, max_active=2)
    bad = srv.submit((63, 1, 64), (63, 1, 32), (0.2, 1, 0.2), 5, plasma=dict(ppc=2, seed=1))
    good = srv.submit((64, 1, 64), (32, 1, 32), (0.2, 1, 0.2), 5, plasma=dict(ppc=2, seed=2))
    srv.run_until_idle()
    assert srv.poll(bad)["state"] == L.REQ_FAILED and srv.poll(bad)["t_done"] >= 0
    assert srv.poll(good)["state"] == L.REQ_DONE
    assert srv.stats()["bytes_in_use"] == srv.footprint(good)
    for call in (lambda: srv.cancel(bad), lambda: srv.read_field(bad, L.EX, (63, 1, 64))):
        with pytest.raises(L.PicError) as ei:
            call()
        assert ei.value.status == L.PIC_ESTATE
