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
    # 10 int32/float fields, a double at offset 40, batch_chunk, clean_kernel and 6 reserved int32
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
