"""The C-ABI library builds, loads without a GPU, exports every entry point
include/ugkwp.h declares, and its host-only calls (mesh validation, workspace
sizing) behave as documented.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2007_13091_gb300 import ugkwp, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^int\s+(ugkwp_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    L = ugkwp.lib()
    declared = _declared()
    assert {"ugkwp_mesh_load", "ugkwp_init", "ugkwp_step", "ugkwp_moments", "ugkwp_adjoint_wave"} <= declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(ugkwp.EXPORTED) >= declared


def test_struct_layouts_match_header():
    # sizes follow from the header's field order with natural alignment
    assert ctypes.sizeof(ugkwp.Bc) == 80
    assert ctypes.sizeof(ugkwp.Params) == 8 * 8 + 8 * 4 + 8 + 8 + 16 * 80
    assert ctypes.sizeof(ugkwp.MeshDesc) == 16 + 4 * 8
    assert ctypes.sizeof(ugkwp.State) == 8 + 8 + 8 + 20 + 4 + 7 * 8
    assert ctypes.sizeof(ugkwp.StateNative) == 8 + 8 + 8 + 20 + 4 + 7 * 8
    assert ctypes.sizeof(ugkwp.LaunchCfg) == 4 * 4


def test_mesh_load_and_sizes_host_only():
    cfg = wl.shock_tube(nx=10, ny=2, nz=2)
    m = ugkwp.ugkwp_mesh_load(cfg["mesh"])
    s = ugkwp.ugkwp_query_sizes(m, cfg["params"])
    assert s.n_cells == 240 and s.n_bfaces == len(cfg["mesh"]["bfaces"])
    assert s.n_faces == (4 * 240 + s.n_bfaces) // 2
    assert s.workspace_bytes > 0 and s.workspace_bytes % 256 == 0
    p2 = dict(cfg["params"], precision="mixed")
    assert ugkwp.ugkwp_query_sizes(m, p2).workspace_bytes < s.workspace_bytes


def test_mesh_validation_errors():
    cfg = wl.uniform_box(n=(2, 2, 2))
    m = cfg["mesh"]
    bad = m["tets"].copy()
    bad[3] = bad[3][[0, 1, 3, 2]]
    with pytest.raises(ugkwp.UgkwpError, match="volume"):
        ugkwp.ugkwp_mesh_load({**m, "tets": bad})
    with pytest.raises(ugkwp.UgkwpError, match="no boundary tag"):
        ugkwp.ugkwp_mesh_load({**m, "bfaces": m["bfaces"][1:], "btags": m["btags"][1:]})
    oob = m["tets"].copy()
    oob[0, 0] = 10 ** 6
    with pytest.raises(ugkwp.UgkwpError, match="out of range"):
        ugkwp.ugkwp_mesh_load({**m, "tets": oob})


def _raise_sampling(mesh, params):
    """query_sizes with an unknown sampling mode (bypassing the binding's names)."""
    p = ugkwp.make_params(params)
    p.sampling = 7
    s = ugkwp.Sizes()
    ugkwp._check(ugkwp.lib().ugkwp_query_sizes(mesh.handle, ctypes.byref(p), ctypes.byref(s)))


def test_parameter_validation():
    cfg = wl.uniform_box(n=(2, 2, 2))
    mesh = ugkwp.ugkwp_mesh_load(cfg["mesh"])
    for key, val, pat in (("CFL", 1.5, "CFL"), ("N_ref", 0, "N_ref"), ("order", 3, "order must be"),
                          ("particle_capacity", 2 ** 31, "capacity"), ("Pr", -0.5, "Pr must be"),
                          ("Pr", float("nan"), "Pr must be")):
        with pytest.raises(ugkwp.UgkwpError, match=pat):
            ugkwp.ugkwp_query_sizes(mesh, dict(cfg["params"], **{key: val}))
    with pytest.raises(ugkwp.UgkwpError, match="sampling"):
        _raise_sampling(mesh, cfg["params"])
    with pytest.raises(ugkwp.UgkwpError, match="order 2"):
        ugkwp.ugkwp_query_sizes(mesh, dict(cfg["params"], order=1, sampling="gp1"))
    with pytest.raises(ugkwp.UgkwpError, match="venkat_K"):
        ugkwp.ugkwp_query_sizes(mesh, dict(cfg["params"], order=2, venkat_K=-1.0))
    with pytest.raises(ugkwp.UgkwpError, match="no entry"):
        ugkwp.ugkwp_query_sizes(mesh, dict(cfg["params"], bc=[]))


def test_adjoint_rejects_bad_arguments_without_gpu_work():
    with pytest.raises(ugkwp.UgkwpError) as e:
        ugkwp.ugkwp_adjoint_wave(None)
    assert e.value.code == ugkwp.E_ARG
    with pytest.raises(ugkwp.UgkwpError) as e:
        ugkwp.ugkwp_adjoint_query(None, 3)
    assert e.value.code == ugkwp.E_ARG


def test_batch_and_launch_cfg_reject_bad_arguments_without_gpu_work():
    """Argument checks that run before any CUDA call."""
    import ctypes
    L = ugkwp.lib()
    out = ctypes.c_void_p()
    assert L.ugkwp_batch_create(None, 0, None, ctypes.byref(out)) == ugkwp.E_ARG
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.ugkwp_batch_create(arr, 2, None, ctypes.byref(out)) == ugkwp.E_ARG
    assert L.ugkwp_batch_step(None, 1) == ugkwp.E_ARG
    assert L.ugkwp_batch_sync(None) == ugkwp.E_ARG
    assert L.ugkwp_set_launch_cfg(None, None) == ugkwp.E_ARG
    assert L.ugkwp_autotune(None, 2, None) == ugkwp.E_ARG
    assert L.ugkwp_batch_autotune(None, 2, None) == ugkwp.E_ARG
