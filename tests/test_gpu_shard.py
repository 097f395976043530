"""Box sharding on one GPU: two or three libpic handles, each owning part of
the boxes, stepped together by paper_2104_11385_gb300.shard with direct
device-buffer hand-over (LocalTransport), against the single-handle run of
the same workload: fields (assembled from the owners of their cells) and
particles (matched by id) within 1e-10 relative after 10 steps, also across
a cross-rank load-balancing call that moves boxes in the middle of the run."""
import numpy as np
import pytest

import paper_2104_11385_gb300 as pic
from paper_2104_11385_gb300 import shard as SH
from paper_2104_11385_gb300 import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0


def run_pair(wl, owner, nranks, steps=10, rebalance_at=None, fields=None):
    ref = pic.from_workload(wl)
    ranks = [SH.LibRank(wl, r, owner) for r in range(nranks)]
    if fields is not None:
        for c, f in enumerate(fields):
            ref.set_field(c, f)
            for rk in ranks:
                rk.set_field(c, f)
    sim = SH.ShardedSimulation(wl, ranks, owner, nranks, SH.LocalTransport())
    ref.step(steps)
    if rebalance_at is None:
        sim.step(steps)
    else:
        sim.step(rebalance_at)
        sim.rebalance(policy=pic.POLICY_KNAPSACK, cost=pic.COST_HEURISTIC, theta=0.0)
        sim.step(steps - rebalance_at)
    ref.sync()
    worst = {}
    for c in range(9):
        worst[f"F{c}"] = rel(sim.read_field(c).reshape(-1), ref.read_field(c).reshape(-1))
    L = [wl["ncell"][a] * wl["dx"][a] for a in range(3)]
    for s in range(len(wl["species"])):
        g, r = sim.particles(s), ref.particles(s)
        assert g["id"].size == r["id"].size, (s, g["id"].size, r["id"].size)
        gi, ri = np.argsort(g["id"]), np.argsort(r["id"])
        assert np.array_equal(g["id"][gi], r["id"][ri])
        for a, k in enumerate(("x", "y", "z")):
            if wl["dim"] == 2 and k == "y":
                continue
            d = np.abs(g[k][gi] - r[k][ri])
            d = np.minimum(d, L[a] - d)
            worst[f"s{s}{k}"] = float(d.max() / L[a]) if d.size else 0.0
        for k in ("ux", "uy", "uz", "w"):
            worst[f"s{s}{k}"] = rel(g[k][gi], r[k][ri])
    bad = {k: v for k, v in worst.items() if not v <= TOL}
    assert not bad, f"sharded vs single handle above {TOL}: {bad}"
    log = sim.log
    sim.close()
    ref.close()
    return log


def halves(wl, axis=0):
    ijk = SH.box_ijk(wl)
    nb = wl["ncell"][axis] // wl["box"][axis]
    return (ijk[:, axis] >= nb // 2).astype(np.int32)


def test_uniform32_two_ranks_match_single_handle():
    wl = workloads.uniform32()
    run_pair(wl, halves(wl, 0), 2)


def test_small_foil_two_ranks_match_single_handle():
    """The foil recipe at 1/4 extents (64^3 cells, laser antenna, absorbing z
    layers, electrons and protons), split across the foil."""
    wl = workloads.foil256(seed=2, scale=4)
    run_pair(wl, halves(wl, 1), 2)


def test_three_ranks_checkerboard_and_a_rebalance():
    """Three ranks owning boxes in a scattered pattern (every box borders
    other ranks), relativistic random plasma with random fields, quadratic
    shapes, and a cross-rank load-balancing call after 4 steps that moves
    boxes and their particles."""
    n, box = (24, 16, 16), (8, 8, 8)
    wl = workloads.random_plasma(501, 3, n, box, (0.3, 0.3, 0.3), 2, nspecies=2, npart=5000, umax=1.5)
    fields = workloads.random_fields(9, n, amp=0.1)
    nboxes = 3 * 2 * 2
    owner = (np.arange(nboxes) % 3).astype(np.int32)
    log = run_pair(wl, owner, 3, steps=10, rebalance_at=4, fields=fields)
    assert len(log) == 1 and log[0]["adopted"]


def test_2d_cubic_two_ranks_match_single_handle():
    wl = workloads.random_plasma(502, 2, (64, 1, 64), (16, 1, 16), (0.3, 1.0, 0.3), 3, nspecies=2, npart=6000,
                                 umax=2.0, absorb=6, laser=True)
    owner = halves(wl, 2)
    run_pair(wl, owner, 2)
