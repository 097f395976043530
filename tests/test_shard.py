"""Box sharding across ranks on the CPU (no GPU): the ghost-cell plans of
libpic against brute force, and two or three gloo ranks running the orchestrator of
paper_2104_11385_gb300.shard -- J ghost sum, E/B ghost exchange, particle
migration and the cross-rank load-balancing routine with redistribution --
over torch.distributed, with a numpy model of a rank in place of the GPU
handle (the device side of each call is covered by tests/test_gpu_shard.py)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2104_11385_gb300 import _lib as L
from paper_2104_11385_gb300 import shard as SH
from paper_2104_11385_gb300.sim import shard_halo_cells, shard_moved_cells


def _brute_halo(n, box, owner, own, near, halo, dim):
    """Cells of own's boxes within `halo` (periodic, per axis) of a box of near's."""
    nb = [n[a] // box[a] for a in range(3)]
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    coords = [i.reshape(-1), j.reshape(-1), k.reshape(-1)]
    cell_box = ((coords[2] // box[2]) * nb[1] + coords[1] // box[1]) * nb[0] + coords[0] // box[0]
    mine = owner[cell_box] == own
    hit = np.zeros(coords[0].size, bool)
    for b in np.nonzero(owner == near)[0]:
        bi = (b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1]))
        ok = np.ones(coords[0].size, bool)
        for a in range(3):
            if dim == 2 and a == 1:
                continue
            c0, c1 = bi[a] * box[a], bi[a] * box[a] + box[a]
            x = coords[a]
            d = np.full(x.size, n[a])
            for s in (-n[a], 0, n[a]):
                lo, hi = c0 + s, c1 + s
                d = np.minimum(d, np.where(x < lo, lo - x, np.where(x >= hi, x - hi + 1, 0)))
            ok &= d <= halo
        hit |= ok
    return np.nonzero(mine & hit)[0]


@pytest.mark.parametrize("dim,n,box", [(3, (16, 24, 16), (8, 8, 4)), (3, (8, 8, 16), (4, 8, 8)),
                                       (2, (32, 1, 24), (8, 1, 8)), (3, (24, 8, 8), (8, 4, 4))])
def test_halo_cells_match_brute_force(dim, n, box):
    """The neighbour-box plan equals a search over every box of the other rank
    (periodic distance per axis), for three ranks and halos 1..4; boxes one or
    two per axis exercise the periodic images of a box on both sides."""
    rng = np.random.default_rng(sum(n) + dim)
    nboxes = int(np.prod([n[a] // box[a] for a in range(3)]))
    for trial in range(3):
        owner = rng.integers(0, 3, nboxes).astype(np.int32)
        for halo in (1, 3, min(4, min(box[a] for a in range(3) if not (dim == 2 and a == 1)))):
            for own in range(3):
                for near in range(3):
                    if own == near:
                        continue
                    got = shard_halo_cells(dim, n, box, owner, own, near, halo)
                    want = _brute_halo(n, box, owner, own, near, halo, dim)
                    assert np.array_equal(got, want), (trial, halo, own, near)


def test_moved_cells_and_argument_errors():
    n, box = (8, 8, 8), (4, 4, 4)
    old = np.array([0, 0, 1, 1, 0, 1, 0, 1], np.int32)
    new = np.array([0, 1, 1, 0, 0, 1, 1, 1], np.int32)
    got01 = shard_moved_cells(3, n, box, old, new, 0, 1)
    got10 = shard_moved_cells(3, n, box, old, new, 1, 0)
    assert got01.size == 2 * 64 and got10.size == 64
    cb = _cell_boxes(n, box)
    assert set(np.unique(cb[got01])) == {1, 6} and set(np.unique(cb[got10])) == {3}
    with pytest.raises(L.PicError):
        shard_halo_cells(3, n, box, old, 0, 0, 3)      # own == near
    with pytest.raises(L.PicError):
        shard_halo_cells(3, n, box, old, 0, 1, 5)      # halo above the box extent
    with pytest.raises(L.PicError):
        shard_halo_cells(3, (8, 8, 9), box, old, 0, 1, 2)


def _cell_boxes(n, box):
    nb = [n[a] // box[a] for a in range(3)]
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return (((k // box[2]) * nb[1] + j // box[1]) * nb[0] + i // box[0]).reshape(-1)


# ---------------------------------------------------------------- gloo ranks ---
class HostRank:
    """numpy model of a rank for the CPU test: dense fields (9 components) and
    particle records in cell units, with the semantics of include/pic_shard.h."""

    def __init__(self, wl, rank, owner, fields, parts):
        self.wl, self.rank = wl, rank
        self.F = fields.copy()
        self.parts = [{k: v.copy() for k, v in p.items()} for p in parts]
        self.owner = np.asarray(owner, np.int32)
        self.out = {}

    def set_owner(self, owner):
        self.owner = np.asarray(owner, np.int32)

    def cells(self, c):
        return torch.as_tensor(c, dtype=torch.int64)

    def pack(self, c0, nc, cells):
        return torch.as_tensor(self.F[c0:c0 + nc][:, cells.numpy()].copy())

    def unpack(self, c0, nc, cells, buf, add):
        idx = cells.numpy()
        if add:
            self.F[c0:c0 + nc][:, idx] += buf.numpy()
        else:
            self.F[c0:c0 + nc][:, idx] = buf.numpy()

    def _boxes(self, p):
        wl = self.wl
        n, b = wl["ncell"], wl["box"]
        nb = [n[a] // b[a] for a in range(3)]
        out = np.zeros(p["X"].size, np.int64)
        mul = 1
        for a, key in enumerate(("X", "Y", "Z")):
            c = np.floor(p[key]).astype(np.int64) % n[a]
            out += (c // b[a]) * mul
            mul *= nb[a]
        return out

    def take_leaving(self, sp, nranks):
        p = self.parts[sp]
        dest = self.owner[self._boxes(p)]
        counts = np.zeros(nranks, np.int64)
        self.out = {}
        for d in range(nranks):
            if d == self.rank:
                continue
            m = dest == d
            counts[d] = int(m.sum())
            self.out[d] = {k: v[m] for k, v in p.items()}
        keep = dest == self.rank
        self.parts[sp] = {k: v[keep] for k, v in p.items()}
        return counts

    def read_leaving(self, sp, dst, n):
        g = self.out[dst]
        assert g["id"].size == n
        buf = np.stack([g[k] for k in ("X", "Y", "Z", "ux", "uy", "uz", "w")] + [g["id"].view(np.float64)])
        return torch.as_tensor(buf)

    def add_arriving(self, sp, buf):
        b = buf.numpy()
        new = {k: b[a] for a, k in enumerate(("X", "Y", "Z", "ux", "uy", "uz", "w"))}
        new["id"] = b[7].copy().view(np.int64)
        self.parts[sp] = {k: np.concatenate([self.parts[sp][k], new[k]]) for k in new}

    def finish(self, advance):
        pass

    def rekey(self):
        pass

    def field_stage(self, k):
        pass

    def box_costs(self, cost):
        nb = self.owner.size
        c = np.zeros(nb)
        for p in self.parts:
            np.add.at(c, self._boxes(p), 1.0)
        return np.where(self.owner == self.rank, c, 0.0)


OWNERS = {2: [0, 1, 1, 0, 1, 0, 0, 1, 1, 1, 0, 0],
          3: [0, 1, 2, 2, 0, 1, 1, 2, 0, 0, 1, 2]}  # three ranks: every box borders the other two


def _setup(seed=5, world=2):
    wl = {"dim": 3, "ncell": (16, 16, 24), "box": (8, 8, 8), "dx": (1.0, 1.0, 1.0), "species": [{}]}
    n = wl["ncell"]
    ncell = n[0] * n[1] * n[2]
    nboxes = 2 * 2 * 3
    rng = np.random.default_rng(seed)
    owner = np.array(OWNERS[world], np.int32)
    # global fields; per-rank J contributions that live within 3 cells of the rank's boxes
    E = rng.normal(size=(6, ncell))
    J = [np.zeros((3, ncell)) for _ in range(world)]
    for r in range(world):
        reach = _brute_halo(n, wl["box"], owner, r, r, 0, 3)
        for o in range(world):
            if o != r:
                reach = np.union1d(reach, _brute_halo(n, wl["box"], owner, o, r, 3, 3))
        J[r][:, reach] = rng.normal(size=(3, reach.size))
    npart = 3000
    P = {"X": rng.uniform(0, n[0], npart), "Y": rng.uniform(0, n[1], npart), "Z": rng.uniform(0, n[2], npart),
         "ux": rng.normal(size=npart), "uy": rng.normal(size=npart), "uz": rng.normal(size=npart),
         "w": rng.uniform(0.5, 1.5, npart), "id": np.arange(npart, dtype=np.int64)}
    return wl, owner, E, J, P, nboxes


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, owner, E, J, P, nboxes = _setup(world=world)
        n = wl["ncell"]
        cb = _cell_boxes(n, wl["box"])
        F = np.full((9, E.shape[1]), np.nan)
        mine = owner[cb] == rank
        F[:6, mine] = E[:, mine]                    # E/B valid on own boxes only
        F[6:9] = J[rank]                            # this rank's current contributions
        parts = [{k: v[P["id"] % world == rank] for k, v in P.items()}]   # particles in the wrong place too
        rk = HostRank(wl, rank, owner, F, parts)
        sim = SH.ShardedSimulation(wl, [rk], owner, world, SH.DistTransport("cpu"))
        res = {}
        # J ghost sum: own cells hold every rank's contribution
        sim._fields(6, 3, "J", True)
        res["j_sum"] = bool(np.allclose(rk.F[6:9, mine], sum(J)[:, mine], rtol=0, atol=1e-12))
        # E/B ghosts: own cells and every cell within 3 of own boxes hold the global values
        sim._fields(0, 6, "EB", False)
        near = np.nonzero(mine)[0]
        for o in range(world):
            if o != rank:
                near = np.union1d(near, _brute_halo(n, wl["box"], owner, o, rank, 3, 3))
        res["eb_ghosts"] = bool(np.array_equal(rk.F[:6, near], E[:, near]))
        # migration: every particle ends on the owner of its box, values intact
        sim._migrate()
        p = rk.parts[0]
        res["migrated_ok"] = bool(np.all(owner[rk._boxes(p)] == rank))
        order = np.argsort(p["id"])
        res["values_ok"] = bool(all(np.array_equal(p[k][order], P[k][p["id"][order]]) for k in ("X", "ux", "w")))
        res["ids"] = p["id"].tolist()
        # the cross-rank load-balancing routine: costs summed over ranks, one
        # mapping on both, moved boxes' fields and particles follow
        rec = sim.rebalance(policy=L.POLICY_KNAPSACK, cost=L.COST_HEURISTIC, theta=0.0)
        res["rec"] = rec
        res["owner"] = sim.owner.tolist()
        mine2 = sim.owner[cb] == rank
        res["moved_fields_ok"] = bool(np.array_equal(rk.F[:6, mine2], E[:, mine2]))
        p = rk.parts[0]
        res["migrated2_ok"] = bool(np.all(sim.owner[rk._boxes(p)] == rank))
        res["ids2"] = p["id"].tolist()
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_migrate_and_rebalance(world):
    """world ranks as gloo processes: the J ghost sum, the E/B ghost exchange,
    migration and the cross-rank load-balancing routine (three ranks: every
    box borders both other ranks)."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = [out[r] for r in range(world)]
    for r in res:
        assert r["j_sum"] and r["eb_ghosts"] and r["migrated_ok"] and r["values_ok"]
        assert r["moved_fields_ok"] and r["migrated2_ok"]
    assert sorted(sum((r["ids"] for r in res), [])) == list(range(3000))
    assert sorted(sum((r["ids2"] for r in res), [])) == list(range(3000))
    # every rank computed the same mapping and the same efficiencies
    assert all(r["owner"] == res[0]["owner"] and r["rec"] == res[0]["rec"] for r in res)
    wl, owner, E, J, P, nboxes = _setup(world=world)
    counts = np.bincount(SH.box_of_positions({"dim": 3, "ncell": wl["ncell"], "box": wl["box"], "dx": (1, 1, 1)},
                                             P["X"], P["Y"], P["Z"]), minlength=nboxes).astype(float)
    assert res[0]["rec"]["e_old"] == pytest.approx(SH.lb_efficiency(counts, owner, world))
    assert res[0]["rec"]["adopted"] == (res[0]["rec"]["e_new"] >= res[0]["rec"]["e_old"])
