"""The C ABI library builds, loads and exports every entry point of include/gbid.h.

CPU only: no call here reaches the GPU (argument errors return before any
CUDA work, and the size queries are host arithmetic).
"""
import ctypes
import os
import re

import pytest
import torch

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
    # empty matrices have no ID
    assert L.id_workspace_size(0, 0, 20, 1, None) == 0
    assert L.id_workspace_size(0, 10, 0, 1, None) == 0
    assert L.id_sampled_workspace_size(0, 10, 20, 0, 0, None) == 0
    assert L.id_two_sided_workspace_size(1, 0, 0, 1, None) == 0
    assert L.id_csr_workspace_size(0, 0, 20, 1, None) == 0
    assert L.id_reconstruct_workspace_size(0, 10, 20, 0, 0) == 0
    # the size limits: k <= 16384, the long side <= 2048 * 256, the short side <= 65536
    assert L.id_workspace_size(1, 16, 2048 * 256, 8, None) > 0
    assert L.id_workspace_size(1, 16, 2048 * 256 + 1, 8, None) == 0
    assert L.id_workspace_size(1, 65537, 65537, 8, None) == 0
    assert L.id_workspace_size(1, 20000, 20000, 16385, None) == 0


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
    # id_cpqr_residual_norms: NULL workspace or output, m > n, bad ldx
    assert L.id_cpqr_residual_norms(None, 0, 10, 20, 16, 5, None, fake, None) == gbid.ID_EINVAL
    assert L.id_cpqr_residual_norms(ws, 0, 10, 20, 16, 5, None, None, None) == gbid.ID_EINVAL
    assert L.id_cpqr_residual_norms(ws, 0, 30, 20, 32, 5, None, fake, None) == gbid.ID_EINVAL
    assert L.id_cpqr_residual_norms(ws, 0, 10, 20, 12, 5, None, fake, None) == gbid.ID_EINVAL
    # id_solve: k > n
    assert L.id_solve(fake, 0, 5, 8, 6, fake, 1, None) == gbid.ID_EINVAL
    # id_decompose_batched: count < 0, NULL descriptors, bad dtype, small queue scratch; count 0 is a no-op
    assert L.id_decompose_batched(fake, -1, 1, fake, 256, fake, None) == gbid.ID_EINVAL
    assert L.id_decompose_batched(None, 3, 1, fake, 256, fake, None) == gbid.ID_EINVAL
    assert L.id_decompose_batched(fake, 3, 9, fake, 256, fake, None) == gbid.ID_EINVAL
    assert L.id_decompose_batched(fake, 3, 1, fake, 16, fake, None) == gbid.ID_ENOMEM
    assert L.id_decompose_batched(None, 0, 1, None, 0, None, None) == gbid.ID_OK


def test_batched_instances_and_tuner_rules(gbid):
    """The batched kernel's instance table and the tuner's argument checks
    (nothing here reaches the device)."""
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    n32, n64 = L.id_batched_config_count(1), L.id_batched_config_count(0)
    assert n32 >= 2 and n64 >= 2 and L.id_batched_config_count(5) == 0
    for dt, cnt in ((0, n64), (1, n32)):
        seen = set()
        for i in range(cnt):
            c = gbid.IdBatchedConfig()
            assert L.id_batched_config_get(dt, i, ctypes.byref(c)) == gbid.ID_OK
            d = c.as_dict()
            assert d["threads"] % 32 == 0 and 32 <= d["threads"] <= 512
            assert d["cols_per_warp"] >= 1 and d["rows_per_lane"] >= 1 and d["ctas_per_sm"] >= 1
            # 32-bit registers per CTA within the SM's 65536 at the stated residency
            assert d["threads"] * d["ctas_per_sm"] <= 2048
            seen.add(tuple(d.values()))
        assert len(seen) == cnt                                  # no instance twice
        c = gbid.IdBatchedConfig()
        assert L.id_batched_config_get(dt, cnt, ctypes.byref(c)) == gbid.ID_EINVAL
        assert L.id_batched_config_get(dt, -1, ctypes.byref(c)) == gbid.ID_EINVAL
        assert L.id_batched_config_get(dt, 0, None) == gbid.ID_EINVAL
    assert gbid.batched_configs(torch.float32)[0] == {"threads": 256, "cols_per_warp": 4, "rows_per_lane": 8,
                                                      "ctas_per_sm": 3}
    assert L.id_batched_config_get(7, 0, ctypes.byref(gbid.IdBatchedConfig())) == gbid.ID_EINVAL
    # id_decompose_batched_with: the config index is checked first; count 0 is a no-op
    assert L.id_decompose_batched_with(fake, 3, 1, fake, 256, fake, n32, None) == gbid.ID_EINVAL
    assert L.id_decompose_batched_with(fake, 3, 1, fake, 256, fake, -1, None) == gbid.ID_EINVAL
    assert L.id_decompose_batched_with(fake, 3, 1, fake, 16, fake, 1, None) == gbid.ID_ENOMEM
    assert L.id_decompose_batched_with(None, 0, 1, None, 0, None, 1, None) == gbid.ID_OK
    # id_batched_autotune: NULL best, reps out of range; an empty batch picks 0 and launches nothing
    best = ctypes.c_int(-7)
    ms = (ctypes.c_float * n32)(*([1.0] * n32))
    assert L.id_batched_autotune(fake, 3, 1, fake, 256, fake, 3, ms, None, None) == gbid.ID_EINVAL
    assert L.id_batched_autotune(fake, 3, 1, fake, 256, fake, 0, ms, ctypes.byref(best), None) == gbid.ID_EINVAL
    assert L.id_batched_autotune(fake, 3, 9, fake, 256, fake, 3, ms, ctypes.byref(best), None) == gbid.ID_EINVAL
    assert L.id_batched_autotune(None, 0, 1, None, 0, None, 3, ms, ctypes.byref(best), None) == gbid.ID_OK
    assert best.value == 0 and list(ms) == [0.0] * n32


def test_engine_option(gbid):
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    ws = ctypes.c_void_p(4096)
    bad = gbid._opts(0, engine=3)
    assert L.id_decompose(fake, 0, 10, 20, 20, 5, ctypes.byref(bad), fake, fake, 20, ws, 1 << 20, None,
                          None) == gbid.ID_EINVAL
    cl = gbid._opts(0, engine=gbid.ENGINE_CLUSTER)
    # a small problem fits one cluster (kernel + statistics kernel); a large one does not
    assert L.id_launch_count(0, 200, 400, 20, ctypes.byref(cl)) == 2
    assert L.id_launch_count(0, 4096, 8192, 256, ctypes.byref(cl)) == -1
    grid = gbid._opts(0, engine=gbid.ENGINE_GRID)
    assert L.id_launch_count(0, 200, 400, 20, ctypes.byref(grid)) == 6
    assert L.id_launch_count(1, 200, 400, 20, None) == 2          # FP32: the default takes the cluster


def test_refine_rules(gbid):
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    assert L.id_refine_workspace_size(1, 100, 300, 20) > 100 * 20 * 12
    assert L.id_refine_workspace_size(0, 100, 300, 20) == 0      # FP32 only
    assert L.id_refine_workspace_size(1, 300, 100, 20) == 0      # a column ID (m <= n)
    assert L.id_refine_workspace_size(1, 100, 300, 101) == 0     # k <= m
    assert L.id_refine(None, 1, 100, 300, 300, 20, fake, fake, 300, fake, 1 << 30, None, None) == gbid.ID_EINVAL
    assert L.id_refine(fake, 1, 100, 300, 299, 20, fake, fake, 300, fake, 1 << 30, None, None) == gbid.ID_EINVAL
    assert L.id_refine(fake, 1, 100, 300, 300, 20, fake, fake, 300, fake, 1024, None, None) == gbid.ID_ENOMEM
    # the randomized workspace grows by the refinement's unless it is switched off
    o_on, o_off = gbid._opts(0, True), gbid._opts(0, False)
    on = L.id_rid_workspace_size(1000, 3000, 70, 60, ctypes.byref(o_on))
    off = L.id_rid_workspace_size(1000, 3000, 70, 60, ctypes.byref(o_off))
    assert on > off


def test_sampled_rules(gbid):
    """Optim RID: p sampled columns, k <= p <= n, k <= m; the sample is checked
    on the host (distinct, in range) before anything reaches the device."""
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    o = gbid._opts(0)
    assert L.id_sampled_workspace_size(0, 300, 1000, 228, 190, ctypes.byref(o)) > 300 * 228 * 8
    assert L.id_sampled_workspace_size(1, 1000, 600, 36, 30, ctypes.byref(o)) > 0     # tall A: CPQR of 1000 x 36
    assert L.id_sampled_workspace_size(0, 300, 1000, 1001, 190, None) == 0             # p > n
    assert L.id_sampled_workspace_size(0, 300, 1000, 100, 190, None) == 0              # k > p
    assert L.id_sampled_workspace_size(0, 100, 1000, 228, 190, None) == 0              # k > m
    assert L.id_sampled_workspace_size(3, 300, 1000, 228, 190, None) == 0              # dtype

    def call(idx, p=None, k=2, work_bytes=1 << 30, lda=80):
        arr = (ctypes.c_int32 * len(idx))(*idx)
        return L.id_decompose_sampled(fake, 0, 50, 80, lda, arr, len(idx) if p is None else p, k, None, fake, fake,
                                      80, fake, work_bytes, None, None)

    assert call([1, 1, 2, 3]) == gbid.ID_EINVAL           # repeated column
    assert call([0, 5, 80, 2]) == gbid.ID_EINVAL           # out of range
    assert call([-1, 2, 3, 4]) == gbid.ID_EINVAL
    assert call([0, 1, 2, 3], k=5) == gbid.ID_EINVAL       # k > p
    assert call([0, 1, 2, 3], lda=79) == gbid.ID_EINVAL
    assert call([0, 1, 2, 3], lda=1 << 31) == gbid.ID_EINVAL
    assert call([0, 1, 2, 3], work_bytes=64) == gbid.ID_ENOMEM


def test_normal_equation_route_rules(gbid):
    """opts.zsolve = 1 (the paper's normal-equation Z): column IDs on the grid engine only."""
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    base = L.id_workspace_size(0, 300, 700, 40, None)
    ne = gbid._opts(0, zsolve=1)
    assert L.id_workspace_size(0, 300, 700, 40, ctypes.byref(ne)) > base
    assert L.id_workspace_size(0, 700, 300, 40, ctypes.byref(ne)) == 0       # a row ID
    bad = gbid._opts(0, zsolve=2)
    assert L.id_workspace_size(0, 300, 700, 40, ctypes.byref(bad)) == 0
    cl = gbid._opts(0, engine=gbid.ENGINE_CLUSTER, zsolve=1)
    assert L.id_decompose(fake, 0, 200, 400, 400, 20, ctypes.byref(cl), fake, fake, 400, fake, 1 << 30, None,
                          None) == gbid.ID_EINVAL
    assert L.id_decompose(fake, 0, 400, 200, 200, 20, ctypes.byref(ne), fake, fake, 400, fake, 1 << 30, None,
                          None) == gbid.ID_EINVAL
    assert L.id_launch_count(0, 300, 700, 40, ctypes.byref(ne)) == -1


def test_reconstruct_rules(gbid):
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    assert L.id_reconstruct_workspace_size(0, 300, 700, 40, 0) >= 300 * 40 * 8
    assert L.id_reconstruct_workspace_size(1, 700, 300, 40, 1) >= 40 * 300 * 4
    assert L.id_reconstruct_workspace_size(0, 300, 700, 701, 0) == 0        # k > n
    assert L.id_reconstruct_workspace_size(0, 30, 700, 31, 1) == 0          # k > m for a row ID
    assert L.id_reconstruct_workspace_size(0, 300, 700, 40, 2) == 0
    assert L.id_reconstruct_workspace_size(2, 300, 700, 40, 0) == 0

    def call(lda=700, ldz=700, ldo=700, tr=0, work_bytes=1 << 30, A=fake):
        return L.id_reconstruct(A, 0, 300, 700, lda, 40, fake, fake, ldz, tr, fake, ldo, fake, work_bytes, None, None)

    assert call(A=None) == gbid.ID_EINVAL
    assert call(lda=699) == gbid.ID_EINVAL
    assert call(ldo=699) == gbid.ID_EINVAL
    assert call(ldz=699) == gbid.ID_EINVAL
    assert call(tr=1, ldz=299) == gbid.ID_EINVAL      # a row ID's Z is k x m
    assert call(work_bytes=64) == gbid.ID_ENOMEM


def test_two_sided_rules(gbid):
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    one = L.id_workspace_size(0, 300, 700, 40, None)
    assert L.id_two_sided_workspace_size(0, 300, 700, 40, None) > one + 300 * 40 * 8
    assert L.id_two_sided_workspace_size(1, 700, 300, 40, None) > 0
    assert L.id_two_sided_workspace_size(0, 40, 700, 40, None) > 0          # k = m: the second stage is trivial
    assert L.id_two_sided_workspace_size(0, 300, 700, 301, None) == 0
    ne = gbid._opts(0, zsolve=1)
    assert L.id_two_sided_workspace_size(0, 300, 700, 40, ctypes.byref(ne)) == 0

    def call(ldx=300, ldz=700, lda=700, work_bytes=1 << 30):
        return L.id_decompose_two_sided(fake, 0, 300, 700, lda, 40, None, fake, fake, fake, ldx, fake, ldz, fake,
                                        work_bytes, None, None)

    assert call(ldx=299) == gbid.ID_EINVAL     # X is k x m
    assert call(ldz=699) == gbid.ID_EINVAL     # Z is k x n
    assert call(lda=699) == gbid.ID_EINVAL
    assert call(work_bytes=1024) == gbid.ID_ENOMEM


def test_csr_rules(gbid):
    L = gbid.lib()
    fake = ctypes.c_void_p(256)
    assert L.id_csr_workspace_size(0, 300, 700, 40, None) > L.id_workspace_size(0, 300, 700, 40, None)
    assert L.id_csr_workspace_size(0, 300, 700, 301, None) == 0
    cl = gbid._opts(0, engine=gbid.ENGINE_CLUSTER)
    assert L.id_csr_workspace_size(0, 200, 400, 20, ctypes.byref(cl)) == 0
    ne = gbid._opts(0, zsolve=1)
    assert L.id_csr_workspace_size(0, 200, 400, 20, ctypes.byref(ne)) == 0

    def call(nnz=100, ldz=700, colind=fake, work_bytes=1 << 30):
        return L.id_decompose_csr(fake, colind, fake, 0, 300, 700, nnz, 40, None, fake, fake, ldz, fake, work_bytes,
                                  None, None)

    assert call(nnz=-1) == gbid.ID_EINVAL
    assert call(colind=None) == gbid.ID_EINVAL
    assert call(ldz=699) == gbid.ID_EINVAL
    assert call(work_bytes=1024) == gbid.ID_ENOMEM


def test_batched_workspace_rules(gbid):
    L = gbid.lib()
    assert L.id_batched_problem_workspace_size(1, 100, 300, 20) >= 100 * 300 * 4 + 300 * 4
    assert L.id_batched_problem_workspace_size(0, 100, 300, 20) >= 100 * 300 * 8
    # the m > n route: the same working size
    assert L.id_batched_problem_workspace_size(1, 300, 100, 20) == L.id_batched_problem_workspace_size(1, 100, 300, 20)
    assert L.id_batched_problem_workspace_size(1, 100, 300, gbid.BATCHED_MAX_K + 1) == 0
    assert L.id_batched_problem_workspace_size(1, gbid.BATCHED_MAX_MIN_DIM + 1, 5000, 8) == 0
    assert L.id_batched_problem_workspace_size(1, 10, 20, 11) == 0
    assert L.id_batched_problem_workspace_size(1, 10, 20, 0) == 0


def test_binding_refuses_cpu_tensors(gbid):
    import torch

    with pytest.raises(ValueError):
        gbid.id_decompose(torch.zeros(4, 8, dtype=torch.float64), 2)


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises; there is no CPU fallback."""
    import subprocess
    import sys

    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_2105_07076_gb300 as g\n"
        "g.LIB_PATH = %r\n"
        "g._lib = None\n"
        "try:\n"
        "    g.lib()\n"
        "except RuntimeError as e:\n"
        "    print('raised', e)\n"
        "else:\n"
        "    print('loaded')\n"
    ) % (ROOT, str(tmp_path / "libgbid.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert "raised" in out.stdout, out.stdout + out.stderr


def test_tuning_cache_file(gbid, tmp_path):
    """The persisted tuner choices: keys separate dtype, GPU model, instance
    table and shape multiset (in any order); the file round-trips, keeps other
    entries, survives a malformed file, and leaves no temporary files."""
    cfgs = [{"threads": 256}, {"threads": 128}]
    shapes = [(40, 90, 8), (100, 30, 12)]
    key = gbid.tune_cache_key("torch.float32", "GPU X", cfgs, shapes)
    assert key == gbid.tune_cache_key("torch.float32", "GPU X", cfgs, list(reversed(shapes)))
    others = [gbid.tune_cache_key("torch.float64", "GPU X", cfgs, shapes),
              gbid.tune_cache_key("torch.float32", "GPU Y", cfgs, shapes),
              gbid.tune_cache_key("torch.float32", "GPU X", cfgs[:1], shapes),
              gbid.tune_cache_key("torch.float32", "GPU X", cfgs, shapes[:1])]
    assert len(set(others + [key])) == 5
    path = str(tmp_path / "tune.json")
    assert gbid.tune_cache_get(path, key) is None                    # no file yet
    gbid.tune_cache_put(path, key, 1, [2.5, 1.5])
    gbid.tune_cache_put(path, others[0], 0, [3.0, 4.0])
    assert gbid.tune_cache_get(path, key) == (1, [2.5, 1.5])
    assert gbid.tune_cache_get(path, others[0]) == (0, [3.0, 4.0])
    assert gbid.tune_cache_get(path, others[1]) is None
    assert sorted(os.listdir(tmp_path)) == ["tune.json"]
    with open(path, "w") as f:
        f.write("{not json")
    assert gbid.tune_cache_get(path, key) is None
    gbid.tune_cache_put(path, key, 1, [2.5, 1.5])                    # a malformed file is replaced
    assert gbid.tune_cache_get(path, key) == (1, [2.5, 1.5])
    with open(path, "w") as f:
        f.write('{"%s": {"config": "x"}}' % key)
    assert gbid.tune_cache_get(path, key) is None


C_PROGRAM = r"""
#include <stdio.h>
#include "gbid.h"

#define CHECK(c) do { if (!(c)) { printf("failed: %s\n", #c); return 1; } } while (0)

int main(void) {
    id_opts o = {0};
    CHECK(id_workspace_size(ID_F64, 100, 300, 20, &o) > 0);
    CHECK(id_workspace_size(ID_F64, 100, 300, 20, NULL) == id_workspace_size(ID_F64, 100, 300, 20, &o));
    CHECK(id_workspace_size(ID_F32, 100, 300, 101, NULL) == 0);          /* k > min(m, n) */
    CHECK(id_batched_problem_workspace_size(ID_F32, 100, 300, 20) > 0);
    CHECK(id_batched_config_count(ID_F32) >= 2);
    id_batched_config c;
    CHECK(id_batched_config_get(ID_F32, 0, &c) == ID_OK && c.threads % 32 == 0);
    CHECK(id_decompose(NULL, ID_F64, 100, 300, 300, 20, NULL, NULL, NULL, 300, NULL, 0, NULL, NULL) == ID_EINVAL);
    CHECK(id_launch_count(ID_F64, 100, 300, 400, NULL) == -1);
    CHECK(id_rid_pipe_workspace_size(256, 1024, 74, 64, NULL) > 2 * id_rid_workspace_size(256, 1024, 74, 64, NULL) / 2);
    CHECK(id_rid_pipe_workspace_size(256, 1024, 74, 75, NULL) == 0);   /* k > l */
    id_rid_pipe* pipe = NULL;
    CHECK(id_rid_pipe_create(&pipe, 256, 1024, 74, 64, NULL, NULL, 0) == ID_EINVAL && pipe == NULL);
    CHECK(id_rid_pipe_submit(NULL, NULL, 0, NULL, 0, NULL, NULL, 0, NULL, NULL) == ID_EINVAL);
    CHECK(id_rid_pipe_sync(NULL) == ID_EINVAL);
    id_rid_pipe_destroy(NULL);
    printf("ok\n");
    return 0;
}
"""


def test_header_is_plain_c_and_callable_from_c(gbid, tmp_path):
    """include/gbid.h compiles as strict C99, and a C program linked against
    the library calls it (host-only entry points: sizes, the instance table,
    argument errors)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_gbid.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_gbid"
    libdir = os.path.dirname(gbid.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + os.path.join(ROOT, "include"),
                        str(src), "-L" + libdir, "-lgbid", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_rid_pipe_rules(gbid):
    """The pipelined randomized entry points: sizes and argument errors, all
    decided on the host before any CUDA call."""
    L = gbid.lib()
    one = L.id_rid_workspace_size(256, 1024, 74, 64, None)
    both = L.id_rid_pipe_workspace_size(256, 1024, 74, 64, None)
    # two slots of A (256 x 1024 FP32), Omega (74 x 256 BF16), J, Z (64 x 1024 FP32), status
    assert both >= one + 2 * (256 * 1024 * 4 + 74 * 256 * 2 + 64 * 4 + 64 * 1024 * 4)
    assert L.id_rid_pipe_workspace_size(256, 1024, 74, 75, None) == 0     # k > l
    assert L.id_rid_workspace_size(2048, 4096, 700, 64, None) == 0          # l > 640
    assert L.id_rid_pipe_workspace_size(2048, 4096, 700, 64, None) == 0
    pipe = ctypes.c_void_p()
    assert L.id_rid_pipe_create(ctypes.byref(pipe), 256, 1024, 74, 64, None, None, 0) == gbid.ID_EINVAL
    assert L.id_rid_pipe_create(None, 256, 1024, 74, 64, None, 256, both) == gbid.ID_EINVAL
    assert L.id_rid_pipe_create(ctypes.byref(pipe), 256, 1024, 74, 64, None, 255 * 256 + 8, both) == gbid.ID_EINVAL
    assert L.id_rid_pipe_create(ctypes.byref(pipe), 256, 1024, 74, 64, None, 256 * 256, both - 1) == gbid.ID_ENOMEM
    assert not pipe.value
    assert L.id_rid_pipe_submit(None, None, 0, None, 0, None, None, 0, None, None) == gbid.ID_EINVAL
    assert L.id_rid_pipe_sync(None) == gbid.ID_EINVAL
    L.id_rid_pipe_destroy(None)


def test_cpu_tensors_are_refused_not_computed(gbid):
    """No CPU fallback: every device-side entry point of the binding rejects a
    CPU tensor before any work."""
    A = torch.randn(10, 20, dtype=torch.float64)
    J = torch.arange(5, dtype=torch.int32)
    calls = [
        lambda: gbid.id_decompose(A, 5),
        lambda: gbid.id_decompose_randomized(A.float(), torch.randn(8, 10).to(torch.bfloat16), 5),
        lambda: gbid.id_decompose_batched([A], [5]),
        lambda: gbid.id_refine(A.float(), J, torch.zeros(5, 20)),
        lambda: gbid.id_decompose_two_sided(A, 5),
        lambda: gbid.id_decompose_sampled(A, list(range(8)), 5),
        lambda: gbid.id_reconstruct(A, J, torch.zeros(5, 20, dtype=torch.float64)),
        lambda: gbid.IdFunction.apply(A, 5),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="CUDA"):
            call()


def test_bounded_wait_selftest_argument_rules(gbid):
    """id_selftest_bounded_wait checks its scratch before any CUDA work."""
    L = gbid.lib()
    st = ctypes.c_int(7)
    assert L.id_selftest_bounded_wait(None, 4096, ctypes.byref(st), None) == gbid.ID_EINVAL
    assert L.id_selftest_bounded_wait(ctypes.c_void_p(4096), 4095, ctypes.byref(st), None) == gbid.ID_EINVAL
    assert L.id_selftest_bounded_wait(ctypes.c_void_p(4096 + 16), 4096, ctypes.byref(st), None) == gbid.ID_EINVAL
    assert L.id_selftest_bounded_wait(ctypes.c_void_p(4096), 4096, None, None) == gbid.ID_EINVAL
    assert st.value == 7
    assert gbid.SELFTEST_WORK_BYTES == 4096

