"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/dgr.h.  No compute calls (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dgr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:(?:long|unsigned)\s+)*\w+\s*\*?\s*(dgr_\w+)\s*\(",
                                 src, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dgr_voxelize", "dgr_voxelize_backward", "dgr_project", "dgr_backproject",
              "dgr_step", "dgr_ws_create", "dgr_ws_destroy", "dgr_status"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2411_04844_b300 import dgr
    L = dgr.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(dgr.EXPORTS) <= set(declared_functions())


def test_host_side_validation_without_gpu():
    """Argument checks run on the host and never touch the device."""
    from paper_2411_04844_b300 import dgr
    L = dgr.lib()
    g = dgr.Grid(0, 4, 4, 1.0, 0.0, 0.0, 0.0)
    t = ctypes.c_int()
    assert L.dgr_tile_count(ctypes.byref(g), ctypes.byref(t)) == dgr.DGR_ERR_ARG
    g = dgr.Grid(64, 64, 64, 1.0, -32.0, -32.0, -32.0)
    assert L.dgr_tile_count(ctypes.byref(g), ctypes.byref(t)) == dgr.DGR_OK
    assert t.value == 8 * 4 * 2
    plan = dgr.WsPlan()
    plan.max_n = 10; plan.max_tiles = 4; plan.max_pairs = 100
    b = ctypes.c_size_t()
    assert L.dgr_ws_bytes(ctypes.byref(plan), ctypes.byref(b)) == dgr.DGR_OK and b.value > 0
    plan.max_pairs = -1
    assert L.dgr_ws_bytes(ctypes.byref(plan), ctypes.byref(b)) == dgr.DGR_ERR_ARG
    # k_trunc must be > 0 or a negative odd integer; a null workspace is refused
    assert L.dgr_voxelize(ctypes.byref(g), 0, None, None, None, None, ctypes.c_float(-4.0),
                          ctypes.c_void_p(1), None, None) == dgr.DGR_ERR_ARG
    assert L.dgr_voxelize(ctypes.byref(g), 0, None, None, None, None, ctypes.c_float(3.0),
                          ctypes.c_void_p(1), None, None) == dgr.DGR_ERR_ARG
    assert L.dgr_strerror(dgr.DGR_ERR_WS_TOO_SMALL).decode().startswith("workspace")


def test_library_is_sm103a_only():
    from paper_2411_04844_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_noalloc_projector_refuses_on_the_host():
    """dgr_project_noalloc validates like dgr_project and sizes its ray tables
    in 64-bit arithmetic: a views x columns product just above 2^32 (which
    would wrap to a small 32-bit count) is refused before anything runs, as
    are more views than any geometry may have.  The pointers are never
    dereferenced on these paths."""
    from paper_2411_04844_b300 import dgr
    L = dgr.lib()
    g = dgr.Grid(16, 16, 16, 1.0, -8.0, -8.0, -8.0)
    fake = ctypes.c_void_p(256)
    # 65536 views x 65538 columns = 2^32 + 2^17 entries (a 17 GB sinogram at one row)
    geo = dgr.Geom(dgr.DGR_PARALLEL, 65536, 65538, 1, 1.0, 1.0, 0.0, 0.0, 256)
    assert (65536 * 65538) % (1 << 32) * 32 <= dgr.NOALLOC_SCRATCH_BYTES
    assert L.dgr_project_noalloc(ctypes.byref(g), ctypes.byref(geo), fake, fake,
                                 None) == dgr.DGR_ERR_WS_TOO_SMALL
    geo = dgr.Geom(dgr.DGR_PARALLEL, (1 << 20) + 1, 1, 1, 1.0, 1.0, 0.0, 0.0, 256)
    assert L.dgr_project_noalloc(ctypes.byref(g), ctypes.byref(geo), fake, fake,
                                 None) == dgr.DGR_ERR_ARG
    # a cone whose source circle does not contain the grid, as dgr_project refuses
    geo = dgr.Geom(dgr.DGR_CONE, 4, 8, 8, 1.0, 1.0, 10.0, 20.0, 256)
    assert L.dgr_project_noalloc(ctypes.byref(g), ctypes.byref(geo), fake, fake,
                                 None) == dgr.DGR_ERR_ARG


def test_slab_grids_are_validated_on_the_host():
    """dgr_grid.z0 must be >= 0; the calls that take whole grids (the fused
    step, the optimiser, densification, seeding) refuse a slab.  The pointers
    are never dereferenced on these paths."""
    from paper_2411_04844_b300 import dgr
    L = dgr.lib()
    t = ctypes.c_int()
    whole = dgr.Grid(64, 64, 64, 1.0, -32.0, -32.0, -32.0)
    assert L.dgr_tile_count(ctypes.byref(whole.slab(32, 32)), ctypes.byref(t)) == dgr.DGR_OK
    bad = dgr.Grid(64, 64, 32, 1.0, -32.0, -32.0, -32.0, -1)
    assert L.dgr_tile_count(ctypes.byref(bad), ctypes.byref(t)) == dgr.DGR_ERR_ARG
    with pytest.raises(dgr.DgrError):
        whole.slab(40, 32)  # past the whole grid's last layer
    fake = ctypes.c_void_p(256)
    geo = dgr.Geom(dgr.DGR_PARALLEL, 4, 8, 8, 1.0, 1.0, 0.0, 0.0, 256)
    prob = dgr.make_problem(whole.slab(0, 32), geo)
    prob.grid.z0 = 8
    p = dgr.Params(4, fake, fake, fake, fake, fake, fake, fake, fake, None)
    assert L.dgr_adam(ctypes.byref(prob), ctypes.byref(p), fake, fake, fake, fake, None) == dgr.DGR_ERR_ARG
    assert L.dgr_params_init(ctypes.byref(prob), ctypes.byref(p), None) == dgr.DGR_ERR_ARG
    prob.grid.z0 = 0
    assert L.dgr_adam(ctypes.byref(prob), ctypes.byref(p), None, fake, fake, fake, None) == dgr.DGR_ERR_ARG
