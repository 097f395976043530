"""Python wrapper of the request server (include/pic_server.h): marshalling only."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L


class Server:
    """Continuous-batching server of independent PIC simulations on one GPU."""

    def __init__(self, dim=2, shape_order=1, max_active=64, hbm_budget_bytes=64 << 30, stream=None):
        self._lib = L.load()
        d = L.ServerDesc(int(dim), int(shape_order), int(max_active), int(hbm_budget_bytes),
                         ctypes.c_void_p(stream) if stream else None)
        h = ctypes.c_void_p()
        L.check(self._lib.pic_server_create(ctypes.byref(d), ctypes.byref(h)), None)
        self._h = h
        self.dim = dim

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pic_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != L.PIC_OK:
            raise L.PicError(st, self._lib.pic_server_last_error(self._h).decode(errors="replace"))

    def submit(self, ncell, box, dx, nsteps, dt=0.0, cfl=0.95, plasma=None, species=None) -> int:
        """plasma: dict(ppc, density, u_th, ripple, seed); or species: list of
        dicts with q, m, x, y, z, ux, uy, uz, w, id (host arrays)."""
        r = L.RequestDesc()
        g = r.grid
        g.dim = self.dim
        for a in range(3):
            g.ncell[a] = int(ncell[a])
            g.box[a] = int(box[a])
            g.dx[a] = float(dx[a])
        g.dt = float(dt)
        g.cfl = float(cfl)
        g.shape_order = 1
        r.nsteps = int(nsteps)
        keep = []
        if species:
            r.nspecies = len(species)
            for i, sp in enumerate(species):
                si = r.species[i]
                si.charge, si.mass = float(sp["q"]), float(sp["m"])
                si.np = len(sp["x"])
                for a, k in enumerate(("x", "y", "z", "ux", "uy", "uz", "w")):
                    arr = np.ascontiguousarray(sp[k], np.float64)
                    keep.append(arr)
                    si.soa[a] = arr.ctypes.data
                ids = np.ascontiguousarray(sp["id"], np.int64)
                keep.append(ids)
                si.ids = ids.ctypes.data
        else:
            p = plasma or {}
            r.nspecies = 0
            r.plasma = L.PlasmaInit(int(p.get("ppc", 4)), float(p.get("density", 1.0)),
                                    float(p.get("u_th", 0.01)), float(p.get("ripple", 0.01)),
                                    int(p.get("seed", 1)))
        rid = ctypes.c_int64()
        self._check(self._lib.pic_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        return rid.value

    def tick(self):
        a, p = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.pic_server_tick(self._h, ctypes.byref(a), ctypes.byref(p)))
        return a.value, p.value

    def poll(self, rid) -> dict:
        st, steps = ctypes.c_int(), ctypes.c_int()
        ts, ta, td = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.pic_server_poll(self._h, int(rid), ctypes.byref(st), ctypes.byref(ts),
                                              ctypes.byref(ta), ctypes.byref(td), ctypes.byref(steps)))
        return {"state": st.value, "t_submit": ts.value, "t_admit": ta.value, "t_done": td.value,
                "steps": steps.value}

    def read_field(self, rid, comp, ncell):
        out = np.empty(int(np.prod(ncell)), np.float64)
        self._check(self._lib.pic_server_read_fields(self._h, int(rid), int(comp), ctypes.c_void_p(out.ctypes.data)))
        return out.reshape(ncell[2], ncell[1], ncell[0])

    def particles(self, rid, species=0) -> dict:
        n = ctypes.c_int64()
        self._check(self._lib.pic_server_num_particles(self._h, int(rid), int(species), ctypes.byref(n)))
        names = ("x", "y", "z", "ux", "uy", "uz", "w")
        out = {k: np.empty(n.value, np.float64) for k in names}
        ids = np.empty(n.value, np.int64)
        ptrs = (ctypes.c_void_p * 7)(*[ctypes.c_void_p(out[k].ctypes.data) for k in names])
        self._check(self._lib.pic_server_read_particles(self._h, int(rid), int(species), ptrs,
                                                        ctypes.c_void_p(ids.ctypes.data)))
        out["id"] = ids
        return out

    def release(self, rid):
        self._check(self._lib.pic_server_release(self._h, int(rid)))

    def cancel(self, rid):
        """Withdraws a pending or active request between ticks (pic_server_cancel)."""
        self._check(self._lib.pic_server_cancel(self._h, int(rid)))

    def footprint(self, rid) -> int:
        b = ctypes.c_int64()
        self._check(self._lib.pic_server_footprint(self._h, int(rid), ctypes.byref(b)))
        return b.value

    def stats(self) -> dict:
        s = L.ServerStats()
        self._check(self._lib.pic_server_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in L.ServerStats._fields_}

    def run_until_idle(self, max_ticks=1_000_000):
        for _ in range(max_ticks):
            a, p = self.tick()
            if a == 0 and p == 0:
                return
        raise RuntimeError("server did not drain")
