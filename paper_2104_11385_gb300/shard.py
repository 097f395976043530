"""Box-sharded runs: one simulation split across ranks, the setting of arXiv
2104.11385 (Sec. 2.1: boxes distributed among MPI ranks, each owning the
fields and particles of its boxes, guard cells exchanged; Sec. 2.2, Listing 1:
per-box costs gathered at load-balancing steps, a new box-to-rank mapping
computed and, when it improves E enough, boxes and particles redistributed).

Host orchestration only: every step of the path runs in libpic (the calls of
include/pic_shard.h); this module decides which rank sends which cells and
particles to which, and moves the packed buffers with a transport:
  LocalTransport  every rank in this process (handles on one or more GPUs):
                  buffers are handed over directly (peer copies);
  DistTransport   one rank per process over torch.distributed: point-to-point
                  send/recv (NCCL between GPUs, gloo on the CPU).
The rank objects implement a small interface (push, field_stage, pack, unpack,
take_leaving, read_leaving, add_arriving, finish, set_owner, rekey,
box_costs); LibRank wraps a libpic Simulation.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L
from .sim import Simulation, balance_compute, lb_efficiency, shard_halo_cells, shard_moved_cells

HALO_J = 3    # the current of a particle reaches up to 3 cells beyond its box
HALO_EB = 3   # staged E/B tiles and the Yee stencil read up to 2 cells beyond a box (one spare)


def box_of_positions(wl, x, y, z):
    """Box index of physical positions: floor(x/dx) wrapped into [0, n), over
    the box extent, per direction; (bz*nby + by)*nbx + bx."""
    n, b, d = wl["ncell"], wl["box"], wl["dx"]
    nb = [n[a] // b[a] for a in range(3)]
    out = np.zeros(len(x), np.int64)
    mul = 1
    for a, p in enumerate((x, y, z)):
        if wl["dim"] == 2 and a == 1:
            continue
        c = np.floor(np.asarray(p, np.float64) / d[a]).astype(np.int64) % n[a]
        out += (c // b[a]) * mul
        mul *= nb[a]
    return out


def box_ijk(wl):
    n, b = wl["ncell"], wl["box"]
    nb = [n[a] // b[a] for a in range(3)]
    idx = np.arange(nb[0] * nb[1] * nb[2])
    return np.stack([idx % nb[0], (idx // nb[0]) % nb[1], idx // (nb[0] * nb[1])], axis=1).astype(np.int32)


class LocalTransport:
    """All ranks live in this process: a message is handed to its receiver as is."""

    def exchange(self, sends, recv_specs):
        return {k: sends[k] for k in recv_specs}

    def all_counts(self, local_counts):
        return dict(local_counts)

    def sum_costs(self, local_costs):
        return sum(local_costs.values())


class DistTransport:
    """One rank per process over torch.distributed (NCCL on GPUs, gloo on CPU)."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

    def exchange(self, sends, recv_specs):
        dist = self.torch.distributed
        reqs, out = [], {}
        for (s, d), t in sorted(sends.items()):
            reqs.append(dist.isend(t.contiguous(), d))
        for (s, d), (shape, dtype) in sorted(recv_specs.items()):
            buf = self.torch.empty(shape, dtype=dtype, device=self.device)
            reqs.append(dist.irecv(buf, s))
            out[(s, d)] = buf
        for r in reqs:
            r.wait()
        return out

    def all_counts(self, local_counts):
        """{rank: counts vector} for every rank, from each rank's own vector."""
        dist = self.torch.distributed
        (me, row), = local_counts.items()
        t = self.torch.as_tensor(np.asarray(row, np.int64), device=self.device)
        rows = [self.torch.empty_like(t) for _ in range(dist.get_world_size())]
        dist.all_gather(rows, t)
        return {r: rows[r].cpu().numpy() for r in range(len(rows))}

    def sum_costs(self, local_costs):
        dist = self.torch.distributed
        (me, c), = local_costs.items()
        t = self.torch.as_tensor(np.asarray(c, np.float64), device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.cpu().numpy()


class LibRank:
    """One rank backed by a libpic Simulation (full-size field arrays, the
    particles of its own boxes)."""

    def __init__(self, wl, rank, owner, device="cuda", stream=None, precision=1):
        import torch
        self.torch = torch
        self.rank = rank
        self.device = device
        mine = set(np.nonzero(np.asarray(owner) == rank)[0].tolist())
        sim = Simulation(wl["dim"], wl["ncell"], wl["box"], wl["dx"], dt=wl["dt"], shape_order=wl["order"],
                         absorb_cells=wl.get("absorb", 0), stream=stream)
        for s in wl["species"]:
            keep = np.isin(box_of_positions(wl, s["x"], s["y"], s["z"]), list(mine)) if mine else \
                np.zeros(len(s["x"]), bool)
            sim.add_species(s["q"], s["m"], *(np.ascontiguousarray(s[k][keep]) for k in
                                              ("x", "y", "z", "ux", "uy", "uz", "w")),
                            ids=np.ascontiguousarray(s["id"][keep]))
        if wl.get("laser"):
            Ld = wl["laser"]
            sim.add_laser(Ld["a0"], Ld["w0"], Ld["tau"], Ld["t_peak"], Ld["omega"], Ld["xc"], Ld["yc"],
                          Ld["k_ant"])
        if wl.get("gather") == "energy":
            sim.set_gather(True)
        if precision != 1:
            sim.set_launch(precision=precision)
        self.sim = sim
        self.nspecies = len(wl["species"])
        self.set_owner(owner)

    def set_owner(self, owner):
        self.owner = np.ascontiguousarray(owner, np.int32)
        self.sim.shard_set_owner(self.owner, self.rank)

    def set_field(self, comp, data):
        self.sim.set_field(comp, data)

    def push(self):
        self.sim.shard_push()

    def field_stage(self, k):
        self.sim.shard_field_stage(k)

    def cells(self, cells_np):
        return self.torch.as_tensor(cells_np, dtype=self.torch.int64, device=self.device)

    def pack(self, c0, nc, cells):
        buf = self.torch.empty((nc, cells.numel()), dtype=self.torch.float64, device=self.device)
        self.sim.shard_pack(c0, nc, cells, buf)
        return buf

    def unpack(self, c0, nc, cells, buf, add):
        self.sim.shard_unpack(c0, nc, cells, buf, add)

    def take_leaving(self, sp, nranks):
        return self.sim.shard_take_leaving(sp, nranks)

    def read_leaving(self, sp, dst, n):
        """The records leaving for dst as one (8, n) float64 buffer: X Y Z ux uy
        uz w and the ids (their int64 bits)."""
        buf = self.torch.empty((8, n), dtype=self.torch.float64, device=self.device)
        self.sim.shard_read_leaving(sp, dst, [buf[a] for a in range(7)], buf[7].view(self.torch.int64))
        return buf

    def add_arriving(self, sp, buf):
        buf = buf.contiguous()
        self.sim.shard_add_arriving(sp, [buf[a] for a in range(7)], buf[7].view(self.torch.int64))

    def finish(self, advance):
        self.sim.shard_finish(advance)

    def rekey(self):
        self.sim.shard_rekey()

    def box_costs(self, cost):
        """Costs of this rank's boxes (zero elsewhere: the heuristic's cell term
        counts a box once, on its owner)."""
        c = self.sim.box_costs(cost)[0]
        return np.where(self.owner == self.rank, c, 0.0)

    def rebalance_within(self):
        """The rank's own mapping of its boxes onto its SMs, from particle counts."""
        self.sim.rebalance(mode=L.LB_DYNAMIC, theta=0.0, cost=L.COST_HEURISTIC, sched=L.SCHED_QUEUE)

    def close(self):
        self.sim.close()


class ShardedSimulation:
    """One simulation whose boxes are split over ranks.  `ranks` holds this
    process's rank objects (all of them with LocalTransport, one with
    DistTransport); `owner` maps every box to a rank."""

    def __init__(self, wl, ranks, owner, nranks, transport):
        self.wl = wl
        self.ranks = {r.rank: r for r in ranks}
        self.owner = np.ascontiguousarray(owner, np.int32)
        self.nranks = int(nranks)
        self.t = transport
        self.nspecies = len(wl["species"])
        self.step_count = 0
        self.log = []
        self._plans()

    # ---- cell plans (pure host, libpic) for the current owner map
    def _plans(self):
        g = (self.wl["dim"], self.wl["ncell"], self.wl["box"])
        self.cells = {}
        for own in range(self.nranks):
            for near in range(self.nranks):
                if own == near:
                    continue
                for kind, h in (("J", HALO_J), ("EB", HALO_EB)):
                    c = shard_halo_cells(*g, self.owner, own, near, h)
                    self.cells[(kind, own, near)] = c
        self.dev_cells = {}
        for key, c in self.cells.items():
            _, own, near = key
            for r in (own, near):
                if r in self.ranks and c.size:
                    self.dev_cells[key + (r,)] = self.ranks[r].cells(c)

    def _fields(self, c0, nc, kind, add):
        """J ghost sum (kind "J", add): rank s sends its J at the cells of d's
        boxes near s's boxes; E/B ghosts (kind "EB"): rank s sends its values
        at the cells of its boxes near d's boxes."""
        sends, specs = {}, {}
        for s in range(self.nranks):
            for d in range(self.nranks):
                if s == d:
                    continue
                key = (kind, d, s) if kind == "J" else (kind, s, d)
                n = self.cells[key].size
                if n == 0:
                    continue
                if s in self.ranks:
                    sends[(s, d)] = self.ranks[s].pack(c0, nc, self.dev_cells[key + (s,)])
                if d in self.ranks:
                    specs[(s, d)] = ((nc, n), self._f64())
        got = self.t.exchange(sends, specs)
        for (s, d), buf in sorted(got.items()):
            key = (kind, d, s) if kind == "J" else (kind, s, d)
            self.ranks[d].unpack(c0, nc, self.dev_cells[key + (d,)], buf, add)

    def _f64(self):
        import torch
        return torch.float64

    def _migrate(self):
        """Particles whose box another rank owns go to that rank."""
        for sp in range(self.nspecies):
            local = {r: rk.take_leaving(sp, self.nranks) for r, rk in self.ranks.items()}
            counts = self.t.all_counts(local)
            sends, specs = {}, {}
            for s in range(self.nranks):
                for d in range(self.nranks):
                    n = int(counts[s][d]) if s != d else 0
                    if n == 0:
                        continue
                    if s in self.ranks:
                        sends[(s, d)] = self.ranks[s].read_leaving(sp, d, n)
                    if d in self.ranks:
                        specs[(s, d)] = ((8, n), self._f64())
            got = self.t.exchange(sends, specs)
            for (s, d), buf in sorted(got.items()):
                self.ranks[d].add_arriving(sp, buf)

    def step(self, nsteps=1):
        """nsteps PIC cycles over all ranks (the phases of include/pic_shard.h)."""
        for _ in range(nsteps):
            for rk in self.ranks.values():
                rk.push()
            self._fields(6, 3, "J", True)
            for rk in self.ranks.values():
                rk.field_stage(0)
            self._fields(3, 3, "EB", False)
            for rk in self.ranks.values():
                rk.field_stage(1)
            self._fields(0, 3, "EB", False)
            for rk in self.ranks.values():
                rk.field_stage(2)
            self._fields(0, 6, "EB", False)
            for rk in self.ranks.values():
                rk.field_stage(3)
            self._migrate()
            for rk in self.ranks.values():
                rk.finish(True)
            self.step_count += 1

    def rebalance(self, policy=L.POLICY_KNAPSACK, cost=L.COST_HEURISTIC, theta=0.10, cap_factor=1.5):
        """The load-balancing routine across ranks (Sec. 2.2, Listing 1): per-box
        costs summed over ranks (each measures only its own boxes), a new
        mapping by the knapsack or space-filling-curve policy, E of both, and
        the redistribution when E_new >= (1 + theta) E_old."""
        costs = self.t.sum_costs({r: rk.box_costs(cost) for r, rk in self.ranks.items()})
        e_old = lb_efficiency(costs, self.owner, self.nranks)
        new, e_new = balance_compute(costs, box_ijk(self.wl), self.wl["dim"], self.nranks, policy, cap_factor)
        adopted = e_new >= (1.0 + theta) * e_old
        if adopted:
            self.redistribute(new)
        rec = {"step": self.step_count, "e_old": e_old, "e_new": e_new, "adopted": bool(adopted)}
        self.log.append(rec)
        return rec

    def redistribute(self, new_owner):
        """Moves boxes to new owners: E and B of the moved boxes go from the old
        owner to the new one, then the particles follow their boxes."""
        new_owner = np.ascontiguousarray(new_owner, np.int32)
        old = self.owner
        g = (self.wl["dim"], self.wl["ncell"], self.wl["box"])
        sends, specs, cells = {}, {}, {}
        for s in range(self.nranks):
            for d in range(self.nranks):
                if s == d:
                    continue
                c = shard_moved_cells(*g, old, new_owner, s, d)
                if c.size == 0:
                    continue
                cells[(s, d)] = c
                if s in self.ranks:
                    sends[(s, d)] = self.ranks[s].pack(0, 6, self.ranks[s].cells(c))
                if d in self.ranks:
                    specs[(s, d)] = ((6, c.size), self._f64())
        got = self.t.exchange(sends, specs)
        for (s, d), buf in sorted(got.items()):
            self.ranks[d].unpack(0, 6, self.ranks[d].cells(cells[(s, d)]), buf, False)
        self.owner = new_owner
        for rk in self.ranks.values():
            rk.set_owner(new_owner)
        self._plans()
        for rk in self.ranks.values():
            rk.rekey()
        self._migrate()
        for rk in self.ranks.values():
            rk.finish(False)
        self._fields(0, 6, "EB", False)
        for rk in self.ranks.values():
            rk.field_stage(3)
            if hasattr(rk, "rebalance_within"):
                rk.rebalance_within()

    # ---- results (all ranks local)
    def read_field(self, comp):
        """A field component assembled from the owners of its cells (every
        rank must be in this process)."""
        n = self.wl["ncell"]
        out = None
        bo = self._cell_owner()
        for r, rk in self.ranks.items():
            f = rk.sim.read_field(comp).reshape(-1)
            out = f.copy() if out is None else out
            out[bo == r] = f[bo == r]
        return out.reshape(n[2], n[1], n[0])

    def _cell_owner(self):
        n, b = self.wl["ncell"], self.wl["box"]
        nb = [n[a] // b[a] for a in range(3)]
        k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
        box = ((k // b[2]) * nb[1] + (j // b[1])) * nb[0] + (i // b[0])
        return self.owner[box.reshape(-1)]

    def particles(self, sp=0):
        parts = [rk.sim.particles(sp) for rk in self.ranks.values()]
        return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}

    def close(self):
        for rk in self.ranks.values():
            rk.close()
