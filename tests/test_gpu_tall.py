"""Tall working matrices and the bounded wait.

Tall working matrices: the k_cpqr configurations that only a large m reaches.

Beyond about 13 400 FP64 rows (27 900 FP32) the reflector's shared-memory
copy leaves room for one CTA per SM instead of two; beyond about 25 000 FP64
rows (50 000 FP32) v no longer fits and the k_cpqr<T, false, false> instance
reads it from global memory. Each case runs a few pivot steps on a Gaussian
matrix with graded column scales and checks the pivots by the oracle's greedy
replay and Z against the oracle's Z for the GPU's pivots (the same bars as the
other parity tests).

Each tall case moves several GB through the oracle on the host.

The bounded wait: the library's wait primitive (behind every grid barrier of
the CPQR kernel), run on a counter that nothing increments, must give up and
report ID_ETIMEOUT, and the context must stay usable afterwards.
"""
import time

import math

import numpy as np
import pytest
import torch

from oracle import id_oracle as orc

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def gbid():
    import __graft_entry__ as g

    g.build()
    import paper_2105_07076_gb300 as m

    return m


@pytest.mark.parametrize("dtype,m,n,k", [(torch.float64, 14000, 14100, 6), (torch.float32, 28500, 28600, 5),
                                         (torch.float64, 26000, 26050, 4)],
                         ids=["f64-one-cta-per-sm", "f32-one-cta-per-sm", "f64-v-in-global-memory"])
def test_tall_working_matrix(gbid, dtype, m, n, k):
    g = torch.Generator(device="cuda").manual_seed(m + k)
    order = torch.randperm(n, generator=g, device="cuda").double()
    A = torch.randn(m, n, generator=g, device="cuda", dtype=torch.float64) * torch.exp(-4.0 * order / n)
    A = A.to(dtype)
    J, Z, info = gbid.id_decompose(A, k, engine=gbid.ENGINE_GRID)
    assert info["status"] == gbid.ID_OK, info
    Ah = A.double().cpu().numpy()
    del A
    Jg = J.cpu().numpy().astype(np.int64)
    tol = 1e-6 if dtype == torch.float64 else 64 * U32 * math.sqrt(m)
    ok, worst = orc.verify_pivots(Ah, Jg, tol)
    assert ok, worst.max()
    Zg = Z.double().cpu().numpy()
    assert np.array_equal(Zg[:, Jg], np.eye(k))
    Zo = orc.interp_decomp(Ah, k, pivots=Jg)[1]
    bar = 1e-10 if dtype == torch.float64 else max(1e-4, 2 * np.linalg.cond(Ah[:, Jg]) * U32)
    assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= bar


def test_bounded_wait_gives_up_and_the_context_survives(gbid):
    t0 = time.monotonic()
    assert gbid.selftest_bounded_wait() == gbid.ID_ETIMEOUT
    assert time.monotonic() - t0 < 60.0
    A = torch.randn(40, 90, dtype=torch.float64, device="cuda")
    J, Z, info = gbid.id_decompose(A, 8)
    assert info["status"] == gbid.ID_OK
    assert torch.equal(Z[torch.arange(8, device="cuda"), J.long()], torch.ones(8, dtype=torch.float64, device="cuda"))
