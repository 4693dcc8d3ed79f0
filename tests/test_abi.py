"""The C-ABI library loads and exports every symbol include/muser.h declares (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "muser.h")).read()
    return sorted(set(re.findall(r"MUSER_API\s+[\w\s\*]*?\b(muser_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    import paper_1712_06913_b300 as m
    lib = m._lib.load()
    syms = header_symbols()
    assert len(syms) >= 13
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(m._lib.SIGNATURES), "binding declares exactly the header's calls"


def test_record_and_config_layout():
    import paper_1712_06913_b300 as m
    # 10 int32/float fields, a double at offset 40, batch_chunk, clean_kernel, w-projection (3),
    # the CLEAN variant (2) and 1 reserved int32
    assert ctypes.sizeof(m._lib.Config) == 80
    assert m._lib.Config.lat_rad.offset == 40 and m._lib.Config.batch_chunk.offset == 48
    assert m.api.RECORD_FLOATS * 4 == 32


def test_host_pixel_size_and_workspace_queries():
    import paper_1712_06913_b300 as m
    cell = m.pixel_size([0.4e9, 2e9, 15e9], 3000.0, 1024, 60 * np.pi / 180 / 60)
    assert cell[0] == pytest.approx(299792458.0 / 0.4e9 / 3000 / 3, rel=1e-15)
    assert cell[2] == pytest.approx(60 * np.pi / 180 / 60 / 1024, rel=1e-15)
    cfg = m.Config(N=256, G=1024)
    assert m.workspace_size(m.CALL_DIRTY, 4, 0, cfg) > 4 * 512 * 1024 * 8
    assert m.workspace_size(m.CALL_IMAGE, 100, 780, m.Config(N=256, G=1024, batch_chunk=10)) < \
        m.workspace_size(m.CALL_IMAGE, 100, 780, m.Config(N=256, G=1024, batch_chunk=20))
    with pytest.raises(m.MuserError):
        m.workspace_size(m.CALL_DIRTY, 1, 0, m.Config(N=256, G=512))       # imaging needs G = 4N
    with pytest.raises(m.MuserError):
        m.workspace_size(m.CALL_DEGRID, 1, 10, m.Config(N=256, G=1024))    # degridding needs G = 2N


def test_config_validation_of_the_widened_calls():
    """Image sides, w-projection and CLEAN-variant fields are checked on the host (no GPU)."""
    import paper_1712_06913_b300 as m
    ok = [m.Config(N=n, G=4 * n) for n in (16, 1024, 160, 320, 1280, 2560, 5120)]
    for c in ok:
        assert m.workspace_size(m.CALL_DIRTY, 1, 0, c) > 0
    bad = [m.Config(N=n, G=4 * n) for n in (100, 80, 2048, 10240, 96)]
    for c in bad:
        with pytest.raises(m.MuserError):
            m.workspace_size(m.CALL_DIRTY, 1, 0, c)
    with pytest.raises(m.MuserError):                                   # 5 * 2^a sides: imaging only
        m.workspace_size(m.CALL_DEGRID, 1, 10, m.Config(N=320, G=640))
    # w-projection
    assert m.workspace_size(m.CALL_GRID, 2, 100, m.Config(N=64, G=256, w_planes=16, w_max=5.0, w_support=15)) > \
        m.workspace_size(m.CALL_GRID, 2, 100, m.Config(N=64, G=256))
    for kw in (dict(w_planes=1, w_max=5.0), dict(w_planes=16, w_max=0.0), dict(w_planes=16, w_max=5.0, w_support=14),
               dict(w_planes=16, w_max=5.0, w_support=5), dict(w_planes=16, w_max=5.0, w_support=65)):
        with pytest.raises(m.MuserError):
            m.workspace_size(m.CALL_GRID, 1, 10, m.Config(N=64, G=256, **kw))
    with pytest.raises(m.MuserError):                                   # no w-projection in the operator
        m.workspace_size(m.CALL_DEGRID, 1, 10, m.Config(N=64, G=128, w_planes=8, w_max=1.0))
    # uniform weighting: imaging calls only; its scratch (records copy, cell counts) is sized in
    assert m.workspace_size(m.CALL_GRID, 2, 100, m.Config(N=64, G=256, weight_mode=1)) > \
        m.workspace_size(m.CALL_GRID, 2, 100, m.Config(N=64, G=256)) + 2 * (64 * 64 + 64) * 4
    assert m.workspace_size(m.CALL_IMAGE, 2, 100, m.Config(N=64, G=256, weight_mode=1)) > \
        m.workspace_size(m.CALL_IMAGE, 2, 100, m.Config(N=64, G=256))
    with pytest.raises(m.MuserError):
        m.workspace_size(m.CALL_GRID, 1, 10, m.Config(N=64, G=256, weight_mode=2))
    # uniform weighting in the degridding operator's plan: the cell counts on top
    assert m.workspace_size(m.CALL_GRAD, 1, 10, m.Config(N=64, G=128, weight_mode=1)) == \
        m.workspace_size(m.CALL_GRAD, 1, 10, m.Config(N=64, G=128)) + \
        (((64 * 64 + 64 + 1) * 4 + 255) // 256) * 256
    # CLEAN variant
    assert m.workspace_size(m.CALL_IMAGE, 4, 100, m.Config(N=64, G=256, clean_variant=1)) > \
        m.workspace_size(m.CALL_IMAGE, 4, 100, m.Config(N=64, G=256))
    for kw in (dict(clean_variant=2), dict(clean_variant=1, steer_clip=0.0), dict(clean_variant=1, steer_clip=1.5)):
        with pytest.raises(m.MuserError):
            m.workspace_size(m.CALL_IMAGE, 1, 10, m.Config(N=64, G=256, **kw))
    # gradient step workspace holds the operator's
    c = m.Config(N=64, G=128)
    assert m.workspace_size(m.CALL_GRAD, 1, 500, c) > m.workspace_size(m.CALL_DEGRID, 1, 500, c)


def test_call_argument_errors_without_a_gpu():
    """Argument errors are returned before any device work (the library loads without a GPU)."""
    import paper_1712_06913_b300 as m
    lib = m._lib.load()
    c = m.Config(N=64, G=256).c()
    null = ctypes.c_void_p(0)
    # muser_steer: clip outside (0, 1]
    rc = lib.muser_steer(null, null, 1, ctypes.byref(c), null, 1.5, null, null, null, 0, null, null)
    assert rc != 0 and b"clip" in lib.muser_last_error()
    # muser_steer: residual not 16-byte aligned (checked before any device work)
    fake = [ctypes.c_void_p(a) for a in (0x10004, 0x20000, 0x30000, 0x40000)]
    rc = lib.muser_steer(fake[0], fake[1], 1, ctypes.byref(c), null, 0.9, fake[2], fake[3], null, 0, null, null)
    assert rc != 0 and b"aligned" in lib.muser_last_error()
    # muser_grad_step: bad flags, missing pointers
    cd = m.Config(N=64, G=128).c()
    assert lib.muser_grad_step(3, null, null, 10, null, 1.0, 0.1, null, null, ctypes.byref(cd), null, 0, null) != 0
    # a step that consumes a chained forward pass must reuse the plan's workspace
    assert lib.muser_grad_step(m._lib.GRAD_ROWS_READY, null, null, 10, null, 1.0, 0.1, null, null, ctypes.byref(cd),
                               null, 0, null) == m._lib.MUSER_ERR_ARG
    assert lib.muser_grad_step(0, null, null, 10, null, 1.0, 0.1, null, null, ctypes.byref(cd), null, 0, null) != 0
    # muser_image_events: a negative event count, or events missing while announced (checked
    # before any device work)
    args = [null, 2, null, 1, null, null, 1, null, null, 1, null, null, null, ctypes.byref(c), null, null, null, null,
            null, null, null, null, 0, null]
    assert lib.muser_image_events(*args, null, -1, null) == m._lib.MUSER_ERR_ARG
    assert lib.muser_image_events(*args, null, 2, null) == m._lib.MUSER_ERR_ARG
    assert b"chunk_done" in lib.muser_last_error()
    # muser_set_tuning: band rows must divide G; column variant 0 or 1
    assert lib.muser_set_tuning(m.CALL_GRID, ctypes.byref(c), 3) != 0
    assert lib.muser_set_tuning(m.CALL_DIRTY, ctypes.byref(c), 2) != 0
    assert lib.muser_set_tuning(m.CALL_CLEAN, ctypes.byref(c), 0) != 0
    # muser_image's tuned shape: variants 0..3
    assert lib.muser_set_tuning(m.CALL_IMAGE, ctypes.byref(c), 4) != 0
    assert lib.muser_set_tuning(m.CALL_IMAGE, ctypes.byref(c), 2) == 0
    assert lib.muser_set_tuning(m.CALL_IMAGE, ctypes.byref(c), 0) == 0
    # muser_selftest_wait: bound above about one second
    st = ctypes.c_void_p(16)
    assert lib.muser_selftest_wait(1 << 40, st, null) != 0


def test_gradient_imaging_calls_reject_bad_arguments_without_a_gpu():
    """The step-size and update calls check their arguments before any device work."""
    import paper_1712_06913_b300 as m
    lib = m._lib.load()
    cd = m.Config(N=64, G=128).c()
    null = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(0x10000)
    # muser_normalize: n < 1, missing pointers
    assert lib.muser_normalize(fake, 0, fake, fake, null) == m._lib.MUSER_ERR_ARG
    assert lib.muser_normalize(null, 10, fake, fake, null) == m._lib.MUSER_ERR_ARG
    # muser_axpy: non-finite alpha, missing pointers; n = 0 is a no-op
    assert lib.muser_axpy(fake, fake, 10, float("nan"), null, null) == m._lib.MUSER_ERR_ARG
    assert lib.muser_axpy(null, fake, 10, 1.0, null, null) == m._lib.MUSER_ERR_ARG
    assert lib.muser_axpy(null, null, 0, 1.0, null, null) == m._lib.MUSER_OK
    # muser_lipschitz / muser_normal_apply: iterations, sigma, flags, records, workspace
    assert lib.muser_lipschitz(0, fake, fake, 10, 1.0, 0, fake, ctypes.byref(cd), fake, 1 << 30, null) != 0
    assert b"iters" in lib.muser_last_error()
    assert lib.muser_lipschitz(0, fake, fake, 10, -1.0, 5, fake, ctypes.byref(cd), fake, 1 << 30, null) != 0
    assert b"inv_sigma2" in lib.muser_last_error()
    assert lib.muser_normal_apply(2, fake, fake, fake, 10, 1.0, ctypes.byref(cd), fake, 1 << 30, null) != 0
    assert lib.muser_normal_apply(0, fake, fake, null, 10, 1.0, ctypes.byref(cd), fake, 1 << 30, null) != 0
    assert lib.muser_normal_apply(0, fake, fake, fake, 10, 1.0, ctypes.byref(cd), fake, 16, null) == \
        m._lib.MUSER_ERR_WORKSPACE
    # imaging-side configurations are refused by the operator's calls (G = 2N)
    ci = m.Config(N=64, G=256).c()
    assert lib.muser_normal_apply(0, fake, fake, fake, 10, 1.0, ctypes.byref(ci), fake, 1 << 30, null) != 0
