"""ctypes view of libpic's C ABI (include/pic_api.h): argument marshalling only.

Every step of the PIC path runs in libpic's CUDA kernels; this module converts
Python/numpy/torch arguments into the plain pointers and sizes the ABI takes.
There is no CPU fallback: if libpic.so cannot be loaded the import fails.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ETIMEOUT, PIC_ESTATE, PIC_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "PIC_OK", -1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ECUDA", -4: "PIC_ETIMEOUT",
                -5: "PIC_ESTATE", -6: "PIC_EUNSUPPORTED"}
EX, EY, EZ, BX, BY, BZ, JX, JY, JZ, RHO = range(10)
BIN_NOALLOC_MAX_BOXES = 1 << 20  # PIC_BIN_NOALLOC_MAX_BOXES of include/pic_noalloc.h
POLICY_KNAPSACK, POLICY_SFC, POLICY_BOX_ORDER = 0, 1, 2
COST_HEURISTIC, COST_DEVICE_CLOCK, COST_KERNEL_TIME = 0, 1, 2
LB_NONE, LB_STATIC, LB_DYNAMIC = 0, 1, 2
SCHED_LISTS, SCHED_QUEUE = 0, 1

_d = ctypes.c_double
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_int = ctypes.c_int
_vp = ctypes.c_void_p
_pd = ctypes.POINTER(ctypes.c_double)
_pi32 = ctypes.POINTER(ctypes.c_int32)
_pi64 = ctypes.POINTER(ctypes.c_int64)


class GridDesc(ctypes.Structure):
    _fields_ = [("dim", _int), ("ncell", _i64 * 3), ("box", _i32 * 3), ("dx", _d * 3), ("dt", _d),
                ("cfl", _d), ("shape_order", _int), ("absorb_cells", _int), ("stream", _vp)]


class LaserDesc(ctypes.Structure):
    _fields_ = [("a0", _d), ("w0", _d), ("tau", _d), ("t_peak", _d), ("omega", _d), ("xc", _d),
                ("yc", _d), ("k_ant", _i64)]


class LBParams(ctypes.Structure):
    _fields_ = [("mode", _int), ("interval", _int), ("theta", _d), ("policy", _int), ("cost", _int),
                ("w_p", _d), ("w_c", _d), ("cap_factor", _d), ("n_workers", _int), ("split", _int),
                ("sched", _int)]


class LBResult(ctypes.Structure):
    _fields_ = [("e_old", _d), ("e_new", _d), ("adopted", _int), ("n_units", _i64),
                ("predicted_speedup", _d), ("step", _i64)]


class LaunchCfg(ctypes.Structure):
    _fields_ = [("threads", _int), ("ctas_per_sm", _int), ("split", _int), ("precision", _int), ("tile", _int),
                ("ppt", _int)]


PREC_FP64, PREC_FLOAT_FLOAT, PREC_FP32 = 1, 2, 3
GATHER_MOMENTUM, GATHER_ENERGY = 0, 1
CAPTURE_CLOCK, CAPTURE_TIME = 1, 2


class Stats(ctypes.Structure):
    _fields_ = [("ms_particle", _d), ("ms_fields", _d), ("ms_sort", _d), ("ms_total", _d),
                ("steps", _i64), ("launches", _i64), ("particle_launches", _i64),
                ("particles_pushed", _i64)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("dim", _int), ("shape_order", _int), ("max_active", _int), ("hbm_budget_bytes", _i64),
                ("stream", _vp)]


class PlasmaInit(ctypes.Structure):
    _fields_ = [("ppc", _int), ("density", _d), ("u_th", _d), ("ripple", _d), ("seed", ctypes.c_uint64)]


class SpeciesInit(ctypes.Structure):
    _fields_ = [("charge", _d), ("mass", _d), ("np", _i64), ("soa", _vp * 7), ("ids", _vp)]


class RequestDesc(ctypes.Structure):
    _fields_ = [("grid", GridDesc), ("nsteps", _int), ("plasma", PlasmaInit), ("nspecies", _int),
                ("species", SpeciesInit * 4)]


class ServerStats(ctypes.Structure):
    _fields_ = [("ticks", _i64), ("particle_updates", _i64), ("particle_launches", _i64), ("kernels", _i64),
                ("admitted", _i64), ("finished", _i64), ("bytes_in_use", _i64)]


REQ_PENDING, REQ_ACTIVE, REQ_DONE, REQ_RELEASED, REQ_CANCELLED, REQ_FAILED = range(6)

# (name, restype, argtypes) of every exported function of include/*.h
SIGNATURES = [
    ("pic_init", _int, [ctypes.POINTER(GridDesc), ctypes.POINTER(_vp)]),
    ("pic_add_species", _int, [_vp, _d, _d, _i64, ctypes.POINTER(_vp), _vp, _int, ctypes.POINTER(_int)]),
    ("pic_add_background", _int, [_vp, _d]),
    ("pic_add_laser", _int, [_vp, ctypes.POINTER(LaserDesc)]),
    ("pic_set_field", _int, [_vp, _int, _vp, _int]),
    ("pic_set_gather", _int, [_vp, _int]),
    ("pic_set_step", _int, [_vp, _i64]),
    ("pic_selftest_bounded_wait", _int, [_vp, _i64]),
    ("pic_set_cost_capture", _int, [_vp, _int]),
    ("pic_get_efficiency", _int, [_vp, _int, _int, ctypes.POINTER(ctypes.c_double)]),
    ("pic_set_lb_params", _int, [_vp, ctypes.POINTER(LBParams)]),
    ("pic_step", _int, [_vp, _int]),
    ("pic_sync", _int, [_vp]),
    ("pic_get_box_costs", _int, [_vp, _int, _pd, _pi64]),
    ("pic_rebalance", _int, [_vp, ctypes.POINTER(LBParams), ctypes.POINTER(LBResult), _pi32]),
    ("pic_get_lb_log", _int, [_vp, ctypes.POINTER(LBResult), _i64, _pi64]),
    ("pic_balance_compute", _int, [_pd, _i64, _pi32, _int, _int, _int, _d, _pi32, _pd]),
    ("pic_lb_efficiency", _int, [_pd, _pi32, _i64, _int, _pd]),
    ("pic_read_fields", _int, [_vp, _int, _vp, _int]),
    ("pic_num_particles", _int, [_vp, _int, _pi64]),
    ("pic_read_particles", _int, [_vp, _int, ctypes.POINTER(_vp), _vp, _int]),
    ("pic_bin_particles", _int, [ctypes.POINTER(GridDesc), _vp, _vp, _vp, _i64, _vp, _vp]),
    ("pic_bin_particles_noalloc", _int, [ctypes.POINTER(GridDesc), _vp, _vp, _vp, _i64, _vp, _vp]),
    ("pic_set_launch", _int, [_vp, ctypes.POINTER(LaunchCfg)]),
    ("pic_get_launch", _int, [_vp, ctypes.POINTER(LaunchCfg)]),
    ("pic_autotune", _int, [_vp, _int, ctypes.POINTER(LaunchCfg)]),
    ("pic_set_profiling", _int, [_vp, _int]),
    ("pic_get_stats", _int, [_vp, ctypes.POINTER(Stats)]),
    ("pic_probe_fp64_fma", _int, [_i64, _pd]),
    ("pic_shard_halo_cells", _int, [ctypes.POINTER(GridDesc), _pi32, _int, _int, _int, _pi64, _pi64]),
    ("pic_shard_moved_cells", _int, [ctypes.POINTER(GridDesc), _pi32, _pi32, _int, _int, _pi64, _pi64]),
    ("pic_shard_set_owner", _int, [_vp, _pi32, _int]),
    ("pic_shard_pack", _int, [_vp, _int, _int, _vp, _i64, _vp]),
    ("pic_shard_unpack", _int, [_vp, _int, _int, _vp, _i64, _vp, _int]),
    ("pic_shard_push", _int, [_vp]),
    ("pic_shard_field_stage", _int, [_vp, _int]),
    ("pic_shard_rekey", _int, [_vp]),
    ("pic_shard_take_leaving", _int, [_vp, _int, _int, _pi64]),
    ("pic_shard_read_leaving", _int, [_vp, _int, _int, ctypes.POINTER(_vp), _vp]),
    ("pic_shard_add_arriving", _int, [_vp, _int, _i64, ctypes.POINTER(_vp), _vp]),
    ("pic_shard_finish", _int, [_vp, _int]),
    ("pic_destroy", _int, [_vp]),
    ("pic_last_error", ctypes.c_char_p, [_vp]),
    ("pic_server_create", _int, [ctypes.POINTER(ServerDesc), ctypes.POINTER(_vp)]),
    ("pic_server_submit", _int, [_vp, ctypes.POINTER(RequestDesc), _pi64]),
    ("pic_server_tick", _int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    ("pic_server_poll", _int, [_vp, _i64, ctypes.POINTER(_int), _pd, _pd, _pd, ctypes.POINTER(_int)]),
    ("pic_server_read_fields", _int, [_vp, _i64, _int, _vp]),
    ("pic_server_num_particles", _int, [_vp, _i64, _int, _pi64]),
    ("pic_server_read_particles", _int, [_vp, _i64, _int, ctypes.POINTER(_vp), _vp]),
    ("pic_server_release", _int, [_vp, _i64]),
    ("pic_server_cancel", _int, [_vp, _i64]),
    ("pic_server_footprint", _int, [_vp, _i64, _pi64]),
    ("pic_server_get_stats", _int, [_vp, ctypes.POINTER(ServerStats)]),
    ("pic_server_destroy", _int, [_vp]),
    ("pic_server_last_error", ctypes.c_char_p, [_vp]),
]

_lib = None


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libpic.so (building it with nvcc first when it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libpic.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, handle=None):
    if status != PIC_OK:
        msg = load().pic_last_error(handle).decode(errors="replace")
        raise PicError(status, msg)
