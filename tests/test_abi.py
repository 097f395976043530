"""CPU-side checks of the C ABI: the library loads and exports every symbol the
header declares, the pure host balancer matches the oracle bit for bit, and bad
arguments come back as status codes (no GPU needed for any of these)."""
import ctypes
import json
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as orc
from paper_2104_11385_gb300 import _lib as L
from paper_2104_11385_gb300 import sim as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pic_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = L.load()
    declared = _declared_functions()
    assert "pic_init" in declared and "pic_balance_compute" in declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    bound = {n for n, _, _ in L.SIGNATURES}
    assert declared <= bound | {"pic_last_error"}, declared - bound


STRUCTS = [("pic_grid_desc", "GridDesc"), ("pic_laser_desc", "LaserDesc"), ("pic_lb_params", "LBParams"),
           ("pic_lb_result", "LBResult"), ("pic_launch_cfg", "LaunchCfg"), ("pic_stats", "Stats"),
           ("pic_server_desc", "ServerDesc"), ("pic_plasma_init", "PlasmaInit"),
           ("pic_species_init", "SpeciesInit"), ("pic_request_desc", "RequestDesc"),
           ("pic_server_stats", "ServerStats")]


def test_struct_layouts_match_the_headers(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the header's struct (gcc on this host)."""
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pic_api.h"', '#include "pic_server.h"',
             "int main(void) {"]
    for cname, pyname in STRUCTS:
        lines.append(f'    printf("{pyname} size %zu\\n", sizeof({cname}));')
        for fname, _ in getattr(L, pyname)._fields_:
            lines.append(f'    printf("{pyname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for cname, pyname in STRUCTS:
        cls = getattr(L, pyname)
        assert got[(pyname, "size")] == ctypes.sizeof(cls), pyname
        for fname, _ in cls._fields_:
            assert got[(pyname, fname)] == getattr(cls, fname).offset, (pyname, fname)


def _random_case(rng, nb, dim):
    costs = rng.lognormal(0.0, 2.0, nb)
    costs[rng.uniform(size=nb) < 0.2] = 0.0
    # exact ties too
    costs[rng.uniform(size=nb) < 0.2] = 3.5
    side = int(np.ceil(nb ** (1 / 3))) + 1
    if dim == 3:
        ijk = np.array([(i % side, (i // side) % side, i // (side * side)) for i in range(nb)], np.int32)
    else:
        ijk = np.array([(i % side, 0, i // side) for i in range(nb)], np.int32)
    rng.shuffle(ijk)
    return costs, ijk


@pytest.mark.parametrize("dim", [2, 3])
def test_balancer_bit_exact_against_oracle(dim):
    rng = np.random.default_rng(123 + dim)
    for trial in range(40):
        nb = int(rng.integers(1, 400))
        nw = int(rng.integers(1, 64))
        costs, ijk = _random_case(rng, nb, dim)
        for cap in (1.5, 1.0, 4.0):
            a, e = S.balance_compute(costs, ijk, dim, nw, L.POLICY_KNAPSACK, cap)
            ra = orc.knapsack(costs, nw, cap)
            assert np.array_equal(a, ra)
            assert e == orc.lb_efficiency(costs, ra, nw)
        a, e = S.balance_compute(costs, ijk, dim, nw, L.POLICY_SFC)
        ra = orc.sfc(costs, ijk, dim, nw)
        assert np.array_equal(a, ra)
        assert e == orc.lb_efficiency(costs, ra, nw)


def test_fig1_through_the_library():
    g = json.load(open(os.path.join(HERE, "golden", "fig1_lb_example.json")))
    costs = np.array(g["particle_counts"], float)
    assert S.lb_efficiency(costs, g["mapping_b"], 2) == 0.5
    a, e = S.balance_compute(costs, g["box_ijk"], 2, 2, L.POLICY_KNAPSACK)
    assert e == pytest.approx(15 / 18, abs=1e-15)


def test_large_balancer_case_matches_oracle():
    # the foil-like shape: few heavy boxes among many empty ones
    rng = np.random.default_rng(7)
    nb = 4096
    costs = np.zeros(nb)
    heavy = rng.choice(nb, 300, replace=False)
    costs[heavy] = rng.lognormal(10, 0.5, 300)
    ijk = np.array([(i % 16, (i // 16) % 16, i // 256) for i in range(nb)], np.int32)
    for nw in (152, 304):
        a, _ = S.balance_compute(costs, ijk, 3, nw, L.POLICY_KNAPSACK, 1.5)
        assert np.array_equal(a, orc.knapsack(costs, nw, 1.5))
        a, _ = S.balance_compute(costs, ijk, 3, nw, L.POLICY_SFC)
        assert np.array_equal(a, orc.sfc(costs, ijk, 3, nw))


def test_bad_arguments_are_status_codes():
    lib = L.load()
    c = np.ones(4)
    out = np.empty(4, np.int32)
    st = lib.pic_balance_compute(c.ctypes.data_as(L._pd), 4, None, 3, 0, L.POLICY_KNAPSACK, 1.5,
                                 out.ctypes.data_as(L._pi32), None)
    assert st == L.PIC_EINVAL
    assert b"bad balancer" in lib.pic_last_error(None)
    c[1] = -1.0
    st = lib.pic_balance_compute(c.ctypes.data_as(L._pd), 4, None, 3, 2, L.POLICY_KNAPSACK, 1.5,
                                 out.ctypes.data_as(L._pi32), None)
    assert st == L.PIC_EINVAL
    c[1] = 1.0
    st = lib.pic_balance_compute(c.ctypes.data_as(L._pd), 4, None, 3, 2, L.POLICY_SFC, 1.5,
                                 out.ctypes.data_as(L._pi32), None)
    assert st == L.PIC_EINVAL  # SFC needs coordinates
    st = lib.pic_balance_compute(c.ctypes.data_as(L._pd), 4, None, 3, 2, 7, 1.5,
                                 out.ctypes.data_as(L._pi32), None)
    assert st == L.PIC_EINVAL
    # a null grid description is rejected before any CUDA call
    h = ctypes.c_void_p()
    assert lib.pic_init(None, ctypes.byref(h)) == L.PIC_EINVAL
    # destroying a null handle is a no-op
    assert lib.pic_destroy(None) == L.PIC_OK
    assert lib.pic_set_gather(None, 1) == L.PIC_EINVAL
    assert lib.pic_set_cost_capture(None, 3) == L.PIC_EINVAL
    e = ctypes.c_double()
    assert lib.pic_get_efficiency(None, 1, 0, ctypes.byref(e)) == L.PIC_EINVAL


def test_grid_validation_without_gpu():
    lib = L.load()
    h = ctypes.c_void_p()
    d = L.GridDesc()
    d.dim = 4
    assert lib.pic_init(ctypes.byref(d), ctypes.byref(h)) == L.PIC_EINVAL
    d.dim = 3
    d.shape_order = 3
    assert lib.pic_init(ctypes.byref(d), ctypes.byref(h)) == L.PIC_EINVAL
    d.shape_order = 1
    for a in range(3):
        d.ncell[a] = 30
        d.box[a] = 8  # does not divide
        d.dx[a] = 0.5
    assert lib.pic_init(ctypes.byref(d), ctypes.byref(h)) == L.PIC_EINVAL
    assert b"divide" in lib.pic_last_error(None)
