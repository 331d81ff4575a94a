"""The C ABI without a GPU: the library builds, loads, exports every symbol
that include/wost.h declares, and rejects malformed scenes on the host."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2302_11815_gb300 import build as libbuild
from paper_2302_11815_gb300 import scenes, wost

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return wost.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wost.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wost_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("wost_scene_create", "wost_scene_destroy", "wost_solve", "wost_poll", "wost_wait",
                 "wost_cancel", "wost_solve_destroy", "wost_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    cdll = C.CDLL(wost.LIBPATH)
    missing = [n for n in declared_functions() if not hasattr(cdll, n)]
    assert not missing, missing
    assert wost.wost_abi_version() == wost.ABI_VERSION == 4


STRUCTS = ("wost_field", "wost_scene_desc", "wost_scene_info", "wost_solve_desc", "wost_progress",
           "wost_engine_desc", "wost_engine_stats", "wost_tune_result")


def test_ctypes_structures_match_the_header(tmp_path):
    """sizeof and every offsetof of the public structures, as a C compiler
    lays them out from include/wost.h, against the binding's ctypes mirrors
    (the version number alone would not catch a drift between them)."""
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "wost.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(wost, name)
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-std=c11", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name in STRUCTS:
        cls = getattr(wost, name)
        assert got[(name, "sizeof")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def _good():
    return scenes.disk_scene(16, "exp_cos", neumann=(np.arange(16) % 2).astype(np.uint8))


@pytest.mark.parametrize("mutate, why", [
    (lambda s: s.update(dim=4), "dim"),
    (lambda s: s["prims"].__setitem__((3, 1), 999), "index out of range"),
    (lambda s: s["prims"].__setitem__((2, 0), -1), "negative index"),
    (lambda s: s["flags"].__setitem__(5, 4), "flag"),
    (lambda s: s["vertices"].__setitem__((1, 0), np.nan), "non-finite"),
    (lambda s: s.update(g={"kind": "per_vertex", "values": None}), "missing values"),
    (lambda s: s.update(g={"kind": "analytic", "fn": "exp_cos", "params": []}, f={"kind": "per_vertex", "values": np.zeros(16)}), "f per vertex"),
    (lambda s: s.update(h={"kind": "grid", "values": np.zeros(4), "origin": [0, 0], "spacing": [1, 1], "dims": [2, 2]}), "h grid"),
])
def test_malformed_scene_rejected_on_host(lib, mutate, why):
    sc = _good()
    sc["prims"] = sc["prims"].copy()
    sc["vertices"] = sc["vertices"].copy()
    sc["flags"] = sc["flags"].copy()
    mutate(sc)
    if sc["g"].get("values", 0) is None:
        # a NULL values pointer with a PER_VERTEX kind
        d = wost.wost_scene_desc()
        V = np.ascontiguousarray(sc["vertices"], np.float32)
        P = np.ascontiguousarray(sc["prims"], np.int32)
        F = np.ascontiguousarray(sc["flags"], np.uint8)
        d.dim, d.n_vertices, d.n_prims = 2, 16, 16
        d.vertices = V.ctypes.data_as(C.POINTER(C.c_float))
        d.prims = P.ctypes.data_as(C.POINTER(C.c_int32))
        d.flags = F.ctypes.data_as(C.POINTER(C.c_uint8))
        d.g.kind = wost.DATA["per_vertex"]
        h = C.c_void_p()
        st = lib.wost_scene_create(C.byref(d), C.byref(h))
        assert st == wost.ERR_INVALID_ARG and not h.value
        return
    with pytest.raises(wost.WostError) as ei:
        wost.wost_scene_create(sc)
    assert ei.value.status == wost.ERR_INVALID_ARG, (why, str(ei.value))
    assert wost.wost_last_error()


def test_null_arguments(lib):
    assert lib.wost_scene_create(None, None) == wost.ERR_INVALID_ARG
    assert lib.wost_solve(None, None, None) == wost.ERR_INVALID_ARG
    assert lib.wost_poll(None, None, None, None, None) == wost.ERR_INVALID_ARG
    assert lib.wost_wait(None, 0.0) == wost.ERR_INVALID_ARG
    assert lib.wost_cancel(None) == wost.ERR_INVALID_ARG
    assert lib.wost_solve_destroy(None) == wost.ERR_INVALID_ARG
    assert lib.wost_scene_destroy(None) == wost.ERR_INVALID_ARG
    assert lib.wost_query_closest_dirichlet(None, 1, None, None, None, None, None) == wost.ERR_INVALID_ARG


@pytest.mark.parametrize("name,leaf", [("config1", 0), ("config1", 1), ("config1", 16), ("koch3_hole", 0),
                                       ("annulus", 0), ("square", 2), ("cube", 0), ("box_sphere", 0),
                                       ("box_sphere", 8), ("torus_small", 0), ("pure_neumann_disk", 0)])
def test_scene_hierarchies_are_well_formed(lib, name, leaf):
    # host-only build and structural check (no GPU): references, coverage of
    # every record by exactly one leaf, nested boxes, silhouette cones that
    # contain the normals below them, depth within the stack sizing
    from paper_2302_11815_gb300 import wost

    if name == "config1":
        sc = scenes.config1()
    elif name == "koch3_hole":
        sc = scenes.config2(grid=8, level=3)
    elif name == "annulus":
        sc = scenes.annulus_scene()
    elif name == "square":
        sc = scenes.square_scene(m=16)
    elif name == "cube":
        sc = scenes.cube_scene(m=8, neumann_faces=(1, 4))
    elif name == "box_sphere":
        sc = scenes.box_sphere_scene()
    elif name == "torus_small":
        sc = scenes.config3(grid=4, nu=60, nv=24, cube_m=4)
    else:
        sc = scenes.disk_scene(64, "exp_plane", (1.0, 0.5, 0.2, 0.0), neumann=np.ones(64, bool))
    info = wost.wost_scene_validate(sc, leaf_size=leaf)
    n = len(sc["prims"])
    assert info["n_dirichlet"] + info["n_neumann"] + info["n_dropped"] == n
    if info["n_dropped"] == 0:
        assert info["n_dirichlet"] == int((sc["flags"] == 0).sum())
    if info["n_dirichlet"]:
        assert info["depth_dirichlet"] >= 1 and info["wide_depth_dirichlet"] >= 1
    assert info["n_silhouette"] >= 1 and info["depth_silhouette"] >= 1


@pytest.mark.parametrize("name", ["slit", "crack", "sheet", "plate", "keyhole"])
@pytest.mark.parametrize("split", [0, 1])
def test_double_sided_and_stress_scenes_are_well_formed(lib, name, split):
    # App. B's double-sided scenes (flags 2 and 3) and the keyhole, with the
    # surface-area x orientation split of the silhouette tree (0) and plain
    # SAH (1): every record counted once, double-sided records kept on their
    # side of the Dirichlet / Neumann split, hierarchies well formed
    from paper_2302_11815_gb300 import wost

    sc = {"slit": scenes.slit_square_scene, "crack": scenes.crack_square_scene,
          "sheet": scenes.sheet_square_scene, "plate": scenes.plate_cube_scene,
          "keyhole": scenes.keyhole_scene}[name]()
    sc = dict(sc, silhouette_split=split)
    info = wost.wost_scene_validate(sc)
    flags = np.asarray(sc["flags"])
    assert info["n_dirichlet"] + info["n_neumann"] + info["n_dropped"] == len(sc["prims"])
    if info["n_dropped"] == 0:
        assert info["n_dirichlet"] == int(np.isin(flags, (0, 2)).sum())
        assert info["n_neumann"] == int(np.isin(flags, (1, 3)).sum())
    assert info["depth_dirichlet"] >= 1
    if info["n_neumann"]:  # (the slit scene is all Dirichlet: no silhouette candidates)
        assert info["n_silhouette"] >= 1 and info["depth_silhouette"] >= 1


def test_batched_workload_scenes_are_well_formed(lib):
    # the batched workload's generator (2D radial polygons with holes, 3D
    # cube + torus), scenes capped at 20k primitives here: every scene
    # builds and passes the structural checks
    from paper_2302_11815_gb300 import wost

    for sc in scenes.config4(n_scenes=12, points=(1, 64), max_scene=20000):
        info = wost.wost_scene_validate(sc)
        assert info["n_dirichlet"] > 0 and info["n_neumann"] > 0
        assert info["n_dirichlet"] + info["n_neumann"] + info["n_dropped"] == len(sc["prims"])
