"""The C ABI library builds, loads and exports every entry point of include/gbid.h.

CPU only: no call here reaches the GPU (argument errors return before any
CUDA work, and the size queries are host arithmetic).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gbid():
    from paper_2105_07076_gb300 import _build

    _build.build()
    import paper_2105_07076_gb300 as m

    return m


def _header_functions():
    text = open(os.path.join(ROOT, "include", "gbid.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(id_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(gbid):
    names = _header_functions()
    assert "id_decompose" in names and "id_cpqr" in names and "id_solve" in names
    L = ctypes.CDLL(gbid.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name
    assert set(names) <= set(gbid.exported_symbols())


def test_version(gbid):
    assert "sm_103a" in gbid.version()


def test_workspace_size_rules(gbid):
    import torch

    assert gbid.workspace_size(torch.float64, 200, 400, 20) > 200 * 400 * 8
    assert gbid.workspace_size(torch.float32, 200, 400, 20) < gbid.workspace_size(torch.float64, 200, 400, 20)
    # the m > n route works on the transpose: same working size
    assert gbid.workspace_size(torch.float64, 400, 200, 20) == gbid.workspace_size(torch.float64, 200, 400, 20)
    L = gbid.lib()
    assert L.id_workspace_size(0, 10, 20, 0, None) == 0      # k < 1
    assert L.id_workspace_size(0, 10, 20, 11, None) == 0     # k > min(m, n)
    assert L.id_workspace_size(7, 10, 20, 5, None) == 0      # bad dtype
    assert L.id_cpqr_workspace_size(0, 10, 20, 12, 5, None) == 0   # ldx not a multiple of 8


def test_argument_errors_return_before_any_launch(gbid):
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    ws = ctypes.c_void_p(4096)
    # null pointers
    assert L.id_decompose(None, 0, 10, 20, 20, 5, None, fake, fake, 20, ws, 1 << 20, None, None) == gbid.ID_EINVAL
    # k out of range
    assert L.id_decompose(fake, 0, 10, 20, 20, 11, None, fake, fake, 20, ws, 1 << 20, None, None) == gbid.ID_EINVAL
    # lda < n
    assert L.id_decompose(fake, 0, 10, 20, 19, 5, None, fake, fake, 20, ws, 1 << 20, None, None) == gbid.ID_EINVAL
    # ldz < max(m, n)
    assert L.id_decompose(fake, 0, 30, 20, 20, 5, None, fake, fake, 20, ws, 1 << 20, None, None) == gbid.ID_EINVAL
    # misaligned workspace
    assert L.id_decompose(fake, 0, 10, 20, 20, 5, None, fake, fake, 20, ctypes.c_void_p(4100), 1 << 20, None,
                          None) == gbid.ID_EINVAL
    # bad dtype
    assert L.id_decompose(fake, 5, 10, 20, 20, 5, None, fake, fake, 20, ws, 1 << 20, None, None) == gbid.ID_EINVAL
    # workspace too small
    assert L.id_decompose(fake, 0, 10, 20, 20, 5, None, fake, fake, 20, ws, 64, None, None) == gbid.ID_ENOMEM
    # id_cpqr: m > n and bad ldx
    assert L.id_cpqr(fake, 0, 30, 20, 32, 5, None, fake, fake, ws, 1 << 20, None, None) == gbid.ID_EINVAL
    assert L.id_cpqr(fake, 0, 10, 20, 12, 5, None, fake, fake, ws, 1 << 20, None, None) == gbid.ID_EINVAL
    # id_solve: k > n
    assert L.id_solve(fake, 0, 5, 8, 6, fake, 1, None) == gbid.ID_EINVAL


def test_binding_refuses_cpu_tensors(gbid):
    import torch

    with pytest.raises(ValueError):
        gbid.id_decompose(torch.zeros(4, 8, dtype=torch.float64), 2)
