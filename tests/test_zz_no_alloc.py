"""The allocation-free KKT entry point against the context-based one.

aln_kkt_residual_noalloc serves callers that cannot call cudaMalloc (fixed
memory budgets, callbacks running while their own pool is exhausted, hot
paths that forbid allocation).  It keeps all scratch in a fixed array inside
the library; this test checks, through the C ABI, that two calls in a row
reproduce aln_kkt_residual within the tolerance the parity tests use.  The
file name sorts last so that a stop-at-first-failure run has already run
every other test.
"""
import numpy as np
import pytest

from paper_1502_01645_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10  # same tolerance as the KKT parity test against the oracle


@pytest.fixture(scope="module")
def aln():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_01645_gb300 import build_lib, aln as binding
    build_lib.build()
    binding.load()
    return binding


def test_noalloc_kkt_matches_context_kkt_twice(aln):
    import torch
    p = W.lopsided_single(d=3000, n=700, seed=21)
    d, n = p.A.shape
    r = np.random.default_rng(3)
    xs = [np.where(r.random(n) < 0.6, 0.0, r.random(n)) for _ in range(2)]

    # reference: the existing context-based entry point
    with aln.Solver("split_bf16") as s:
        s.prepare(p.A, np.stack([p.B[0], p.B[0]]))
        rel_ref, obj_ref = s.kkt(np.stack(xs))

    A = torch.from_numpy(np.ascontiguousarray(p.A.T)).cuda().t()
    b = torch.from_numpy(p.B[0].copy()).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for c in range(2):                                  # two calls in a row
        x = torch.from_numpy(xs[c]).cuda()
        aln.aln_kkt_residual_noalloc(A, d, n, d, aln.DTYPE_F32, b, x, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[0], rel_ref[c], rtol=RTOL)
        np.testing.assert_allclose(got[1], obj_ref[c], rtol=RTOL)


def test_noalloc_rejects_sizes_beyond_the_scratch(aln):
    import torch
    A = torch.zeros((8, 4), dtype=torch.float32, device="cuda")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    big_n = (1 << 21)  # 3n alone exceeds ALN_NOALLOC_SCRATCH_DOUBLES
    with pytest.raises(aln.AlnError) as e:
        aln.aln_kkt_residual_noalloc(A, 8, big_n, 8, aln.DTYPE_F32, A, x, out)
    assert e.value.code == aln.ERR_INVALID_ARG
