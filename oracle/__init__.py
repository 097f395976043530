"""Python view of the FP64 CPU oracle (``pic_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import this
package.  The product library never calls it and shares no code with it.

The oracle restates the per-box PIC cycle of arXiv 2104.11385 Sec. 2.1 (gather,
push, deposit, field solve) with the schemes the paper leaves open fixed as Yee
/ Boris / Esirkepov, and the load-balancing routine of Sec. 2.2 (Eq. 1, the
knapsack and Morton-curve policies, the improvement threshold) plus the
performance model of Sec. 4 (Eq. 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "libpic_oracle.so")
_lock = threading.Lock()
_lib = None

EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)

_d = ctypes.c_double
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)
_pi32 = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # PIC_ORACLE_LIB loads another build of pic_oracle.c (the mutation
            # test uses it to check that the pins catch planted mistakes)
            path = os.environ.get("PIC_ORACLE_LIB")
            if not path:
                path = build()
            L = ctypes.CDLL(path)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.c_int, _pi64, _pd, _d, ctypes.c_int, ctypes.c_int]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_add_species.restype = ctypes.c_int
            L.orc_add_species.argtypes = [ctypes.c_void_p, _d, _d, _i64] + [_pd] * 7 + [_pi64]
            L.orc_set_laser.argtypes = [ctypes.c_void_p] + [_d] * 7 + [_i64]
            L.orc_set_field.argtypes = [ctypes.c_void_p, ctypes.c_int, _pd]
            L.orc_set_gather.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_get_field.argtypes = [ctypes.c_void_p, ctypes.c_int, _pd]
            L.orc_num_particles.restype = _i64
            L.orc_num_particles.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_get_particles.argtypes = [ctypes.c_void_p, ctypes.c_int] + [_pd] * 7 + [_pi64]
            L.orc_step_count.restype = _i64
            L.orc_step_count.argtypes = [ctypes.c_void_p]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_deposit_rho.argtypes = [ctypes.c_void_p, _pd]
            L.orc_box_counts.argtypes = [ctypes.c_void_p, _pi64, _pi64]
            L.orc_shape.restype = _d
            L.orc_shape.argtypes = [ctypes.c_int, _d]
            L.orc_gather.argtypes = [ctypes.c_void_p, _d, _d, _d, _pd]
            L.orc_boris.restype = None
            L.orc_boris.argtypes = [_d, _d, _d, _pd, _pd]
            L.orc_lb_efficiency.restype = _d
            L.orc_lb_efficiency.argtypes = [_pd, _pi32, _i64, ctypes.c_int]
            L.orc_knapsack.argtypes = [_pd, _i64, ctypes.c_int, _d, _pi32]
            L.orc_morton.restype = ctypes.c_uint64
            L.orc_morton.argtypes = [ctypes.c_int, _i64, _i64, _i64]
            L.orc_sfc.argtypes = [_pd, _pi32, _i64, ctypes.c_int, ctypes.c_int, _pi32]
            L.orc_lb_adopt.argtypes = [_d, _d, _d]
            L.orc_bin_particles.argtypes = [ctypes.c_int, _pi64, _pd, _pi64, _pd, _pd, _pd, _i64, _pi64, _pi64]
            L.orc_predicted_speedup.restype = _d
            L.orc_predicted_speedup.argtypes = [_d, _d]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_pd)


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleSim:
    """One oracle simulation (fields periodic, flat index (k*ny+j)*nx+i)."""

    def __init__(self, dim, n, d, dt, order, absorb_cells=0):
        self.dim = int(dim)
        self.n = tuple(int(v) for v in n)
        self.d = tuple(float(v) for v in d)
        self.dt = float(dt)
        self.order = int(order)
        n_arr = np.array(self.n, dtype=np.int64)
        d_arr = np.array(self.d, dtype=np.float64)
        self._h = lib().orc_create(self.dim, n_arr.ctypes.data_as(_pi64), _dp(d_arr), self.dt,
                                   self.order, int(absorb_cells))
        if not self._h:
            raise ValueError("oracle rejected the grid description")
        self.nspecies = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def ncell(self):
        return self.n[0] * self.n[1] * self.n[2]

    def add_species(self, q, m, x, y, z, ux, uy, uz, w, ids=None) -> int:
        arrs = [_c64(a) for a in (x, y, z, ux, uy, uz, w)]
        npart = arrs[0].shape[0]
        ids = np.arange(npart, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, np.int64)
        r = lib().orc_add_species(self._h, float(q), float(m), npart, *[_dp(a) for a in arrs],
                                  ids.ctypes.data_as(_pi64))
        if r < 0:
            raise ValueError("oracle rejected the species")
        self.nspecies += 1
        return r

    def set_laser(self, a0, w0, tau, t_peak, omega, xc, yc, k_ant):
        if lib().orc_set_laser(self._h, a0, w0, tau, t_peak, omega, xc, yc, int(k_ant)) != 0:
            raise ValueError("oracle rejected the laser")

    def set_gather(self, energy_conserving: bool):
        """Field gather: energy-conserving (order - 1 along staggered directions) or not."""
        if lib().orc_set_gather(self._h, int(bool(energy_conserving))) != 0:
            raise ValueError("bad gather kind")

    def set_field(self, comp, data):
        a = _c64(data).reshape(-1)
        assert a.size == self.ncell
        lib().orc_set_field(self._h, comp, _dp(a))

    def field(self, comp) -> np.ndarray:
        out = np.empty(self.ncell, dtype=np.float64)
        lib().orc_get_field(self._h, comp, _dp(out))
        return out.reshape(self.n[2], self.n[1], self.n[0])

    def particles(self, sp=0) -> dict:
        npart = lib().orc_num_particles(self._h, sp)
        out = {k: np.empty(npart, dtype=np.float64) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
        ids = np.empty(npart, dtype=np.int64)
        lib().orc_get_particles(self._h, sp, *[_dp(out[k]) for k in ("x", "y", "z", "ux", "uy", "uz", "w")],
                                ids.ctypes.data_as(_pi64))
        out["id"] = ids
        return out

    def step(self, nsteps=1):
        lib().orc_step(self._h, int(nsteps))

    @property
    def step_count(self) -> int:
        return lib().orc_step_count(self._h)

    def rho(self) -> np.ndarray:
        out = np.empty(self.ncell, dtype=np.float64)
        lib().orc_deposit_rho(self._h, _dp(out))
        return out.reshape(self.n[2], self.n[1], self.n[0])

    def box_counts(self, bsize) -> np.ndarray:
        bs = np.array(bsize, dtype=np.int64)
        nb = [self.n[a] // int(bsize[a]) for a in range(3)]
        out = np.zeros(nb[0] * nb[1] * nb[2], dtype=np.int64)
        if lib().orc_box_counts(self._h, bs.ctypes.data_as(_pi64), out.ctypes.data_as(_pi64)) != 0:
            raise ValueError("box size must divide the grid")
        return out

    def gather(self, x, y, z) -> np.ndarray:
        out = np.empty(6, dtype=np.float64)
        lib().orc_gather(self._h, float(x), float(y), float(z), _dp(out))
        return out


def shape(order: int, dist: float) -> float:
    return lib().orc_shape(int(order), float(dist))


def boris(q, m, dt, eb, u) -> np.ndarray:
    ebv = _c64(eb).copy()
    uv = _c64(u).copy()
    lib().orc_boris(float(q), float(m), float(dt), _dp(ebv), _dp(uv))
    return uv


def lb_efficiency(costs, assign, n_workers) -> float:
    c = _c64(costs)
    a = np.ascontiguousarray(assign, dtype=np.int32)
    return lib().orc_lb_efficiency(_dp(c), a.ctypes.data_as(_pi32), c.size, int(n_workers))


def knapsack(costs, n_workers, cap_factor=1.5) -> np.ndarray:
    c = _c64(costs)
    out = np.empty(c.size, dtype=np.int32)
    if lib().orc_knapsack(_dp(c), c.size, int(n_workers), float(cap_factor), out.ctypes.data_as(_pi32)) != 0:
        raise ValueError("bad knapsack input")
    return out


def morton(dim, bx, by, bz) -> int:
    return int(lib().orc_morton(int(dim), int(bx), int(by), int(bz)))


def sfc(costs, box_ijk, dim, n_workers) -> np.ndarray:
    c = _c64(costs)
    ijk = np.ascontiguousarray(box_ijk, dtype=np.int32).reshape(-1, 3)
    out = np.empty(c.size, dtype=np.int32)
    if lib().orc_sfc(_dp(c), ijk.ctypes.data_as(_pi32), c.size, int(dim), int(n_workers),
                     out.ctypes.data_as(_pi32)) != 0:
        raise ValueError("bad sfc input")
    return out


def bin_particles(dim, n, d, bsize, x, y, z):
    """Stable binning of particles by box: (box_off[nboxes+1], perm[np])."""
    xs, ys, zs = (_c64(a) for a in (x, y if y is not None else np.zeros(len(x)), z))
    nb = int(np.prod([int(n[a]) // int(bsize[a]) for a in range(3)]))
    off = np.zeros(nb + 1, np.int64)
    perm = np.zeros(xs.size, np.int64)
    na, ba = np.array(n, np.int64), np.array(bsize, np.int64)
    da = np.array(d, np.float64)
    if lib().orc_bin_particles(int(dim), na.ctypes.data_as(_pi64), _dp(da), ba.ctypes.data_as(_pi64),
                               _dp(xs), _dp(ys), _dp(zs), xs.size, off.ctypes.data_as(_pi64),
                               perm.ctypes.data_as(_pi64)) != 0:
        raise ValueError("bad binning arguments")
    return off, perm


def lb_adopt(e_old, e_new, theta) -> bool:
    return bool(lib().orc_lb_adopt(float(e_old), float(e_new), float(theta)))


def predicted_speedup(e0, x) -> float:
    return lib().orc_predicted_speedup(float(e0), float(x))
