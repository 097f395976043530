"""GB300-native PIC step with in-situ device-side cost measurement and dynamic
load balancing (after arXiv 2104.11385).  The compute path is libpic.so
(hand-written CUDA for sm_103a behind the C ABI in include/pic_api.h); this
package is the thin Python binding over it."""
from . import _lib
from ._lib import (BX, BY, BZ, COST_DEVICE_CLOCK, COST_HEURISTIC, COST_KERNEL_TIME, EX, EY, EZ, GATHER_ENERGY,
                   GATHER_MOMENTUM, JX, JY, JZ, LB_DYNAMIC,
                   LB_NONE, LB_STATIC, POLICY_BOX_ORDER, POLICY_KNAPSACK, POLICY_SFC, RHO, SCHED_LISTS, SCHED_QUEUE,
                   PicError)
from .sim import Simulation, balance_compute, lb_efficiency, lb_params


def from_workload(wl: dict, stream=None, species_on_device=False) -> Simulation:
    """Creates a Simulation holding a workload dict from ``workloads``."""
    sim = Simulation(wl["dim"], wl["ncell"], wl["box"], wl["dx"], dt=wl["dt"],
                     shape_order=wl["order"], absorb_cells=wl.get("absorb", 0), stream=stream)
    for sp in wl["species"]:
        arrs = [sp[k] for k in ("x", "y", "z", "ux", "uy", "uz", "w")]
        ids = sp["id"]
        if species_on_device:
            import torch
            arrs = [torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in arrs]
            ids = torch.as_tensor(ids, dtype=torch.int64, device="cuda")
        sim.add_species(sp["q"], sp["m"], *arrs, ids=ids)
    if wl.get("laser"):
        L = wl["laser"]
        sim.add_laser(L["a0"], L["w0"], L["tau"], L["t_peak"], L["omega"], L["xc"], L["yc"], L["k_ant"])
    if wl.get("rho0"):
        sim.add_background(wl["rho0"])
    if wl.get("gather") == "energy":
        sim.set_gather(True)
    return sim


__all__ = ["Simulation", "from_workload", "balance_compute", "lb_efficiency", "lb_params", "PicError"]
