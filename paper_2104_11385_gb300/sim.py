"""Thin Python wrapper over libpic's C ABI (same names as include/pic_api.h).

Marshalling only: numpy arrays become host pointers, torch CUDA tensors become
device pointers; every step of the PIC path runs in libpic's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L


def _ptr(a):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, 0, None
    mod = type(a).__module__
    if mod.startswith("torch"):
        if a.dtype.is_floating_point:
            import torch
            assert a.dtype == torch.float64, "particle and field arrays are float64"
        t = a.contiguous()
        return ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0, t
    arr = np.ascontiguousarray(a)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


class Simulation:
    """One libpic simulation (pic_init ... pic_destroy)."""

    def __init__(self, dim, ncell, box, dx, dt=0.0, cfl=0.99, shape_order=1, absorb_cells=0,
                 stream=None):
        self._lib = L.load()
        d = L.GridDesc()
        d.dim = int(dim)
        for a in range(3):
            d.ncell[a] = int(ncell[a])
            d.box[a] = int(box[a])
            d.dx[a] = float(dx[a])
        d.dt = float(dt)
        d.cfl = float(cfl)
        d.shape_order = int(shape_order)
        d.absorb_cells = int(absorb_cells)
        d.stream = ctypes.c_void_p(stream) if stream else None
        h = ctypes.c_void_p()
        L.check(self._lib.pic_init(ctypes.byref(d), ctypes.byref(h)), None)
        self._h = h
        self.dim = int(dim)
        self.ncell = tuple(int(v) for v in ncell)
        self.box = tuple(int(v) for v in box)
        self.dx = tuple(float(v) for v in dx)
        self.nspecies = 0

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.pic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        L.check(st, self._h)

    @property
    def ncells_total(self):
        return self.ncell[0] * self.ncell[1] * self.ncell[2]

    @property
    def nboxes(self):
        return int(np.prod([self.ncell[a] // self.box[a] for a in range(3)]))

    # ------------------------------------------------------------------
    def add_species(self, charge, mass, x, y, z, ux, uy, uz, w, ids=None) -> int:
        arrs = [x, y, z, ux, uy, uz, w]
        n = len(x)
        keep = []
        ptrs = (ctypes.c_void_p * 7)()
        on_dev = 0
        for i, a in enumerate(arrs):
            if a is None:
                ptrs[i] = None
                continue
            p, dev, k = _ptr(a if type(a).__module__.startswith("torch") else np.asarray(a, np.float64))
            ptrs[i] = p
            on_dev = dev
            keep.append(k)
        idp = None
        if ids is not None:
            idp, _, k = _ptr(ids if type(ids).__module__.startswith("torch") else np.asarray(ids, np.int64))
            keep.append(k)
        out = ctypes.c_int()
        self._check(self._lib.pic_add_species(self._h, float(charge), float(mass), int(n), ptrs, idp,
                                              on_dev, ctypes.byref(out)))
        self.nspecies += 1
        return out.value

    def add_background(self, rho0):
        self._check(self._lib.pic_add_background(self._h, float(rho0)))

    def add_laser(self, a0, w0, tau, t_peak, omega, xc, yc, k_ant):
        ld = L.LaserDesc(a0, w0, tau, t_peak, omega, xc, yc, int(k_ant))
        self._check(self._lib.pic_add_laser(self._h, ctypes.byref(ld)))

    def set_field(self, comp, data):
        p, dev, k = _ptr(data if type(data).__module__.startswith("torch") else np.asarray(data, np.float64))
        self._check(self._lib.pic_set_field(self._h, int(comp), p, dev))

    def set_step(self, step: int):
        """Sets the step counter (time t = step * dt), for resuming from saved state."""
        self._check(self._lib.pic_set_step(self._h, int(step)))

    def selftest_bounded_wait(self, limit_ns: int):
        """Runs the device bounded-wait self-test; raises PicError(PIC_ETIMEOUT) as designed."""
        self._check(self._lib.pic_selftest_bounded_wait(self._h, int(limit_ns)))

    def set_gather(self, energy_conserving: bool):
        """Energy-conserving (order - 1 along staggered directions) or default field gather."""
        kind = L.GATHER_ENERGY if energy_conserving else L.GATHER_MOMENTUM
        self._check(self._lib.pic_set_gather(self._h, kind))

    def set_cost_capture(self, clock=True, kernel_time=True):
        """In-kernel cost capture: clock64 (device-clock cost) and %globaltimer (kernel-time cost)."""
        mask = (L.CAPTURE_CLOCK if clock else 0) | (L.CAPTURE_TIME if kernel_time else 0)
        self._check(self._lib.pic_set_cost_capture(self._h, mask))

    def efficiency(self, cost=None, reset_window=False) -> float:
        """E (Eq. 1) of the mapping in force over the current cost window."""
        e = ctypes.c_double()
        self._check(self._lib.pic_get_efficiency(self._h, L.COST_DEVICE_CLOCK if cost is None else int(cost),
                                                 int(bool(reset_window)), ctypes.byref(e)))
        return e.value

    def set_lb_params(self, **kw):
        self._check(self._lib.pic_set_lb_params(self._h, ctypes.byref(lb_params(**kw))))

    def step(self, nsteps=1):
        self._check(self._lib.pic_step(self._h, int(nsteps)))

    def sync(self):
        self._check(self._lib.pic_sync(self._h))

    def box_costs(self, strategy=L.COST_DEVICE_CLOCK):
        c = np.empty(self.nboxes, np.float64)
        n = np.empty(self.nboxes, np.int64)
        self._check(self._lib.pic_get_box_costs(self._h, int(strategy), c.ctypes.data_as(L._pd),
                                                n.ctypes.data_as(L._pi64)))
        return c, n

    def rebalance(self, **kw):
        r = L.LBResult()
        a = np.empty(self.nboxes, np.int32)
        self._check(self._lib.pic_rebalance(self._h, ctypes.byref(lb_params(**kw)), ctypes.byref(r),
                                            a.ctypes.data_as(L._pi32)))
        return {"e_old": r.e_old, "e_new": r.e_new, "adopted": bool(r.adopted), "n_units": r.n_units,
                "predicted_speedup": r.predicted_speedup, "step": r.step, "assign": a}

    def lb_log(self) -> list:
        n = ctypes.c_int64()
        self._check(self._lib.pic_get_lb_log(self._h, None, 0, ctypes.byref(n)))
        buf = (L.LBResult * max(n.value, 1))()
        self._check(self._lib.pic_get_lb_log(self._h, buf, n.value, ctypes.byref(n)))
        return [{"e_old": r.e_old, "e_new": r.e_new, "adopted": bool(r.adopted), "n_units": r.n_units,
                 "predicted_speedup": r.predicted_speedup, "step": r.step} for r in buf[:n.value]]

    def read_field(self, comp, out=None):
        if out is None:
            out = np.empty(self.ncells_total, np.float64)
            self._check(self._lib.pic_read_fields(self._h, int(comp), ctypes.c_void_p(out.ctypes.data), 0))
            return out.reshape(self.ncell[2], self.ncell[1], self.ncell[0])
        p, dev, _ = _ptr(out)
        self._check(self._lib.pic_read_fields(self._h, int(comp), p, dev))
        return out

    def num_particles(self, species=0) -> int:
        n = ctypes.c_int64()
        self._check(self._lib.pic_num_particles(self._h, int(species), ctypes.byref(n)))
        return n.value

    def particles(self, species=0, device=False) -> dict:
        """A species' particles (x, y, z, ux, uy, uz, w, id) in the library's
        order: numpy arrays, or torch tensors on the GPU with device=True."""
        n = self.num_particles(species)
        names = ("x", "y", "z", "ux", "uy", "uz", "w")
        if device:
            import torch
            out = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in names}
            ids = torch.empty(n, dtype=torch.int64, device="cuda")
            addr = {k: out[k].data_ptr() for k in names}
            id_addr = ids.data_ptr()
        else:
            out = {k: np.empty(n, np.float64) for k in names}
            ids = np.empty(n, np.int64)
            addr = {k: out[k].ctypes.data for k in names}
            id_addr = ids.ctypes.data
        ptrs = (ctypes.c_void_p * 7)(*[ctypes.c_void_p(addr[k]) for k in names])
        self._check(self._lib.pic_read_particles(self._h, int(species), ptrs, ctypes.c_void_p(id_addr),
                                                 1 if device else 0))
        out["id"] = ids
        return out

    def set_launch(self, threads=0, ctas_per_sm=0, split=0, precision=0, tile=0, ppt=0):
        c = L.LaunchCfg(int(threads), int(ctas_per_sm), int(split), int(precision), int(tile), int(ppt))
        self._check(self._lib.pic_set_launch(self._h, ctypes.byref(c)))

    def get_launch(self):
        c = L.LaunchCfg()
        self._check(self._lib.pic_get_launch(self._h, ctypes.byref(c)))
        return {"threads": c.threads, "ctas_per_sm": c.ctas_per_sm, "split": c.split, "precision": c.precision,
                "tile": c.tile, "ppt": c.ppt}

    def autotune(self, steps_per_candidate=2):
        c = L.LaunchCfg()
        self._check(self._lib.pic_autotune(self._h, int(steps_per_candidate), ctypes.byref(c)))
        return {"threads": c.threads, "ctas_per_sm": c.ctas_per_sm, "split": c.split, "tile": c.tile, "ppt": c.ppt}

    # ---- box sharding (include/pic_shard.h); device tensors for buffers
    def shard_set_owner(self, owner, rank):
        o = np.ascontiguousarray(owner, np.int32)
        self._check(self._lib.pic_shard_set_owner(self._h, o.ctypes.data_as(L._pi32), int(rank)))

    def shard_pack(self, first_comp, ncomp, cells, buf):
        self._check(self._lib.pic_shard_pack(self._h, int(first_comp), int(ncomp), ctypes.c_void_p(cells.data_ptr()),
                                             int(cells.numel()), ctypes.c_void_p(buf.data_ptr())))

    def shard_unpack(self, first_comp, ncomp, cells, buf, add):
        self._check(self._lib.pic_shard_unpack(self._h, int(first_comp), int(ncomp),
                                               ctypes.c_void_p(cells.data_ptr()), int(cells.numel()),
                                               ctypes.c_void_p(buf.data_ptr()), 1 if add else 0))

    def shard_push(self):
        self._check(self._lib.pic_shard_push(self._h))

    def shard_field_stage(self, stage):
        self._check(self._lib.pic_shard_field_stage(self._h, int(stage)))

    def shard_rekey(self):
        self._check(self._lib.pic_shard_rekey(self._h))

    def shard_take_leaving(self, species, nranks):
        c = np.zeros(int(nranks), np.int64)
        self._check(self._lib.pic_shard_take_leaving(self._h, int(species), int(nranks), c.ctypes.data_as(L._pi64)))
        return c

    def shard_read_leaving(self, species, dst, soa, ids):
        ptrs = (ctypes.c_void_p * 7)(*[ctypes.c_void_p(t.data_ptr()) for t in soa])
        self._check(self._lib.pic_shard_read_leaving(self._h, int(species), int(dst), ptrs,
                                                     ctypes.c_void_p(ids.data_ptr())))

    def shard_add_arriving(self, species, soa, ids):
        ptrs = (ctypes.c_void_p * 7)(*[ctypes.c_void_p(t.data_ptr()) for t in soa])
        self._check(self._lib.pic_shard_add_arriving(self._h, int(species), int(ids.numel()), ptrs,
                                                     ctypes.c_void_p(ids.data_ptr())))

    def shard_finish(self, advance=True):
        self._check(self._lib.pic_shard_finish(self._h, 1 if advance else 0))

    def set_profiling(self, on=True):
        self._check(self._lib.pic_set_profiling(self._h, 1 if on else 0))

    def stats(self) -> dict:
        s = L.Stats()
        self._check(self._lib.pic_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in L.Stats._fields_}


def lb_params(mode=L.LB_DYNAMIC, interval=10, theta=0.10, policy=L.POLICY_KNAPSACK,
              cost=L.COST_DEVICE_CLOCK, w_p=0.75, w_c=0.25, cap_factor=1.5, n_workers=0, split=0,
              sched=L.SCHED_LISTS) -> L.LBParams:
    return L.LBParams(int(mode), int(interval), float(theta), int(policy), int(cost), float(w_p),
                      float(w_c), float(cap_factor), int(n_workers), int(split), int(sched))


def balance_compute(costs, box_ijk, dim, n_workers, policy=L.POLICY_KNAPSACK, cap_factor=1.5):
    """pic_balance_compute: the pure host balancer (no GPU needed)."""
    lib = L.load()
    c = np.ascontiguousarray(costs, np.float64)
    ijk = None if box_ijk is None else np.ascontiguousarray(box_ijk, np.int32).reshape(-1)
    out = np.empty(c.size, np.int32)
    e = ctypes.c_double()
    L.check(lib.pic_balance_compute(c.ctypes.data_as(L._pd), c.size,
                                    None if ijk is None else ijk.ctypes.data_as(L._pi32), int(dim),
                                    int(n_workers), int(policy), float(cap_factor),
                                    out.ctypes.data_as(L._pi32), ctypes.byref(e)))
    return out, e.value


def lb_efficiency(costs, assign, n_workers) -> float:
    lib = L.load()
    c = np.ascontiguousarray(costs, np.float64)
    a = np.ascontiguousarray(assign, np.int32)
    e = ctypes.c_double()
    L.check(lib.pic_lb_efficiency(c.ctypes.data_as(L._pd), a.ctypes.data_as(L._pi32), c.size,
                                  int(n_workers), ctypes.byref(e)))
    return e.value


def shard_halo_cells(dim, ncell, box, owner, own, near, halo) -> np.ndarray:
    """pic_shard_halo_cells: cells of `own`'s boxes within `halo` of `near`'s boxes (host, no GPU)."""
    lib = L.load()
    g = grid_desc(dim, ncell, box, (1.0, 1.0, 1.0))
    o = np.ascontiguousarray(owner, np.int32)
    n = ctypes.c_int64()
    L.check(lib.pic_shard_halo_cells(ctypes.byref(g), o.ctypes.data_as(L._pi32), int(own), int(near), int(halo),
                                     None, ctypes.byref(n)))
    out = np.empty(n.value, np.int64)
    L.check(lib.pic_shard_halo_cells(ctypes.byref(g), o.ctypes.data_as(L._pi32), int(own), int(near), int(halo),
                                     out.ctypes.data_as(L._pi64), ctypes.byref(n)))
    return out


def shard_moved_cells(dim, ncell, box, old_owner, new_owner, src, dst) -> np.ndarray:
    """pic_shard_moved_cells: cells of the boxes moving from rank src to rank dst (host, no GPU)."""
    lib = L.load()
    g = grid_desc(dim, ncell, box, (1.0, 1.0, 1.0))
    a = np.ascontiguousarray(old_owner, np.int32)
    b = np.ascontiguousarray(new_owner, np.int32)
    n = ctypes.c_int64()
    L.check(lib.pic_shard_moved_cells(ctypes.byref(g), a.ctypes.data_as(L._pi32), b.ctypes.data_as(L._pi32),
                                      int(src), int(dst), None, ctypes.byref(n)))
    out = np.empty(n.value, np.int64)
    L.check(lib.pic_shard_moved_cells(ctypes.byref(g), a.ctypes.data_as(L._pi32), b.ctypes.data_as(L._pi32),
                                      int(src), int(dst), out.ctypes.data_as(L._pi64), ctypes.byref(n)))
    return out


def grid_desc(dim, ncell, box, dx, stream=None) -> L.GridDesc:
    d = L.GridDesc()
    d.dim = int(dim)
    for a in range(3):
        d.ncell[a] = int(ncell[a])
        d.box[a] = int(box[a])
        d.dx[a] = float(dx[a])
    d.stream = ctypes.c_void_p(stream) if stream else None
    return d


def bin_particles(dim, ncell, box, dx, x, y, z, box_off, perm, stream=None, fn="pic_bin_particles"):
    """pic_bin_particles on torch CUDA tensors (x, y, z float64; box_off and perm int64)."""
    lib = L.load()
    g = grid_desc(dim, ncell, box, dx, stream)
    yp = ctypes.c_void_p(y.data_ptr()) if y is not None else None
    L.check(getattr(lib, fn)(ctypes.byref(g), ctypes.c_void_p(x.data_ptr()), yp,
                             ctypes.c_void_p(z.data_ptr()), int(x.numel()),
                             ctypes.c_void_p(box_off.data_ptr()), ctypes.c_void_p(perm.data_ptr())))


def probe_fp64_fma(iters=20000) -> float:
    """pic_probe_fp64_fma: measured FP64 FMA throughput of the current device (TFLOP/s)."""
    lib = L.load()
    out = ctypes.c_double()
    L.check(lib.pic_probe_fp64_fma(int(iters), ctypes.byref(out)))
    return out.value
