"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports
every entry point declared in include/nsn.h (no compute calls without a GPU)."""
import ctypes
import re

import pytest

from paper_1907_04587_gb300 import _build, nsn


@pytest.fixture(scope="module")
def libnsn():
    _build.build()
    return nsn.lib()


def test_header_declares_the_boundary():
    names = nsn.exported_names()
    for required in ("nsn_create", "nsn_add_bodies", "nsn_add_constraints", "nsn_step", "nsn_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libnsn):
    for name in nsn.exported_names():
        assert hasattr(libnsn, name), name


def test_record_layouts_match_header():
    src = open(nsn.HEADER).read()
    # field counts of the packed records: 2 ints + 11 floats, 2 ints + 13 floats, 4 ints + 14 floats
    assert nsn.CONTACT_DTYPE.itemsize == 4 * (2 + 11)
    assert nsn.REVOLUTE_DTYPE.itemsize == 4 * (2 + 13)
    assert nsn.TET_DTYPE.itemsize == 4 * (4 + 14)
    assert "nsn_contact" in src and "nsn_revolute" in src and "nsn_tet" in src


def test_config_struct_and_defaults(libnsn):
    cfg = nsn.nsn_default_config()
    assert abs(cfg.h - 1.0 / 60.0) < 1e-15 and cfg.newton_iters == 4 and cfg.cr_iters == 20
    assert cfg.damping == 0.75 and cfg.eps == 1e-6 and cfg.precision == nsn.NSN_FP32
    assert cfg.cone_project == 0 and cfg.island_stop == 0    # the printed method, one system
    assert cfg.line_search == 0 and cfg.best_iterate == 0
    # h, gravity[3], 2 ints, damping, eps, tol_rel, 8 ints
    assert ctypes.sizeof(nsn.nsn_config) == 8 * 4 + 4 * 2 + 8 * 3 + 4 * 12


def test_invalid_arguments_are_rejected_without_gpu(libnsn):
    out = ctypes.c_void_p()
    assert libnsn.nsn_create(None, None, ctypes.byref(out)) == 1
    cfg = nsn.nsn_default_config()
    cfg.h = -1.0
    assert libnsn.nsn_create(ctypes.byref(cfg), None, ctypes.byref(out)) == 1
    cfg = nsn.nsn_default_config()
    cfg.best_iterate = 1                   # island mode required
    assert libnsn.nsn_create(ctypes.byref(cfg), None, ctypes.byref(out)) == 1
    assert libnsn.nsn_destroy(None) == 1


def test_built_for_sm103a():
    assert "compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_collider_rejects_invalid_scenes_without_gpu(libnsn):
    """nsn_collider_create checks its arguments on the host before any CUDA
    call: margin <= 0, environments out of order, excluded ids out of range."""
    base = dict(kind=[0, 0], half=[[.1, .1, .1]] * 2, env=[0, 1], n_envs=2, mu_env=[.5, .5],
                planes=[[0, 0, 1, 0]], exclude=None, margin=0.01, h=1 / 60)
    for bad in (dict(margin=0.0), dict(env=[1, 0]), dict(exclude=[[0, 5]]), dict(n_envs=1), dict(kind=[0, 2])):
        with pytest.raises(nsn.ColliderError) as e:
            nsn.nsn_collider_create(**{**base, **bad})
        assert e.value.status == nsn.NSN_ERR_INVALID_ARG
    assert libnsn.nsn_collider_destroy(None) == nsn.NSN_ERR_INVALID_ARG
    # 17,000 boxes in one environment: 8 x 17,000 x 17,001 pairs overflow the
    # int32 contact count, rejected before any device work
    n = 17000
    with pytest.raises(nsn.ColliderError) as e:
        nsn.nsn_collider_create([0] * n, [[.1, .1, .1]] * n, [0] * n, 1, [.5], [[0, 0, 1, 0]], None, 0.01, 1 / 60)
    assert e.value.status == nsn.NSN_ERR_INVALID_ARG


def test_constraint_counts_beyond_int32_rejected_without_gpu(libnsn):
    """nsn_add_constraints sizes the scene in int64 before storing anything:
    716M contacts (3 rows each, 2.148e9 rows) or 179M tets (12 Jacobian
    entries each, 2.148e9 entries) would overflow the int32 row and entry
    indices of the device layout and are rejected with NSN_ERR_INVALID_ARG.
    The context uses the per-thread default stream handle, so nothing here
    touches a GPU; the records are not read once the count is rejected."""
    cfg = nsn.nsn_default_config()
    ctx = ctypes.c_void_p()
    per_thread_stream = ctypes.c_void_p(2)   # cudaStreamPerThread
    assert libnsn.nsn_create(ctypes.byref(cfg), per_thread_stream, ctypes.byref(ctx)) == nsn.NSN_OK
    try:
        rec = (ctypes.c_char * 256)()
        first = ctypes.c_int32()
        for typ, n in ((nsn.NSN_CONTACT, 716_000_000), (nsn.NSN_TET_NH, 179_000_000)):
            st = libnsn.nsn_add_constraints(ctx, typ, n, rec, ctypes.byref(first))
            assert st == nsn.NSN_ERR_INVALID_ARG
            assert b"limit 2^31 - 1" in libnsn.nsn_last_error(ctx)
        # a count that fits is still validated record by record (zeroed records: bad body ids)
        st = libnsn.nsn_add_constraints(ctx, nsn.NSN_CONTACT, 1, rec, ctypes.byref(first))
        assert st == nsn.NSN_ERR_INVALID_ARG
    finally:
        libnsn.nsn_destroy(ctx)
