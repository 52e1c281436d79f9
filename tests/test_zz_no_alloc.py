"""The allocation-free KKT entry point against the oracle and the context path.

aln_kkt_residual_noalloc serves callers that cannot call cudaMalloc (fixed
memory budgets, callbacks running while their own pool is exhausted, hot
paths that forbid allocation).  It keeps all scratch in a fixed array inside
the library.  These tests check, through the C ABI:
  * two calls in a row reproduce aln_kkt_residual within the tolerance the
    parity tests use, for FP32 and FP64 inputs;
  * the same two calls match the FP64 oracle's kkt_residual (1e-10);
  * a NaN in A, b or x gives NaN in both outputs, and the next call on clean
    inputs is right again (the flag word starts at zero every call);
  * host pointers are refused with INVALID_ARG before anything is launched;
  * sizes beyond the scratch are refused with INVALID_ARG.
The file name sorts last so that a stop-at-first-failure run has already run
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


def _points(n, seed):
    r = np.random.default_rng(seed)
    return [np.where(r.random(n) < 0.6, 0.0, r.random(n)) for _ in range(2)]


def _device(aln, A, b, dtype):
    import torch
    tdt = torch.float32 if dtype == aln.DTYPE_F32 else torch.float64
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(tdt).cuda().t()
    bd = torch.from_numpy(np.ascontiguousarray(b)).to(tdt).cuda()
    return Ad, bd


def _call(aln, Ad, bd, x, dtype):
    import torch
    d, n = Ad.shape
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    aln.aln_kkt_residual_noalloc(Ad, d, n, d, dtype, bd, xd, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype_name", ["f32", "f64"])
def test_noalloc_kkt_matches_context_kkt_twice(aln, dtype_name):
    dtype = aln.DTYPE_F32 if dtype_name == "f32" else aln.DTYPE_F64
    p = W.lopsided_single(d=3000, n=700, seed=21)
    A = p.A if dtype == aln.DTYPE_F32 else p.A.astype(np.float64)
    b = p.B[0] if dtype == aln.DTYPE_F32 else p.B[0].astype(np.float64)
    d, n = A.shape
    xs = _points(n, 3)

    # reference: the existing context-based entry point
    prec = "split_bf16" if dtype == aln.DTYPE_F32 else "fp64"
    with aln.Solver(prec) as s:
        s.prepare(A, np.stack([b, b]))
        rel_ref, obj_ref = s.kkt(np.stack(xs))

    Ad, bd = _device(aln, A, b, dtype)
    for c in range(2):                                  # two calls in a row
        got = _call(aln, Ad, bd, xs[c], dtype)
        np.testing.assert_allclose(got[0], rel_ref[c], rtol=RTOL)
        np.testing.assert_allclose(got[1], obj_ref[c], rtol=RTOL)


@pytest.mark.parametrize("dtype_name", ["f32", "f64"])
def test_noalloc_kkt_matches_oracle(aln, dtype_name):
    from oracle import nnls as O
    dtype = aln.DTYPE_F32 if dtype_name == "f32" else aln.DTYPE_F64
    p = W.uniform_small(seed=7) if dtype == aln.DTYPE_F64 else W.lopsided_single(
        d=2500, n=600, seed=22)
    A = np.asarray(p.A, np.float64 if dtype == aln.DTYPE_F64 else np.float32)
    b = np.asarray(p.B[0], A.dtype)
    d, n = A.shape
    # a point on the solution path (the oracle's optimum), then a random one
    x_opt = O.reference_solution(A.astype(np.float64), b.astype(np.float64))[0]
    xs = [x_opt, _points(n, 5)[0]]
    Ad, bd = _device(aln, A, b, dtype)
    for x in xs:
        rel_o, obj_o = O.kkt_residual(A, b, x)
        got = _call(aln, Ad, bd, x, dtype)
        np.testing.assert_allclose(got[0], rel_o, rtol=RTOL, atol=1e-13)
        np.testing.assert_allclose(got[1], obj_o, rtol=RTOL)


@pytest.mark.parametrize("where", ["A", "b", "x"])
def test_noalloc_nonfinite_input_gives_nan_then_recovers(aln, where):
    p = W.lopsided_single(d=1500, n=300, seed=23)
    A, b = p.A.copy(), p.B[0].copy()
    d, n = A.shape
    x = _points(n, 9)[0]
    clean = _call(aln, *_device(aln, A, b, aln.DTYPE_F32), x, aln.DTYPE_F32)
    assert np.all(np.isfinite(clean))
    Ab, bb, xb = A.copy(), b.copy(), x.copy()
    if where == "A":
        Ab[17, 5] = np.nan
    elif where == "b":
        bb[3] = np.inf
    else:
        xb[11] = np.nan
    bad = _call(aln, *_device(aln, Ab, bb, aln.DTYPE_F32), xb, aln.DTYPE_F32)
    assert np.isnan(bad[0]) and np.isnan(bad[1])
    again = _call(aln, *_device(aln, A, b, aln.DTYPE_F32), x, aln.DTYPE_F32)
    np.testing.assert_array_equal(again, clean)


def test_noalloc_rejects_host_pointers(aln):
    import torch
    d, n = 64, 16
    A = torch.rand((n, d), dtype=torch.float32, device="cuda").t()
    b = torch.rand(d, dtype=torch.float32, device="cuda")
    x = torch.rand(n, dtype=torch.float64, device="cuda")
    out = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    host = {"A": np.asfortranarray(A.cpu().numpy()), "b": b.cpu().numpy(),
            "x": x.cpu().numpy(), "out": np.zeros(2)}
    for name in ("A", "b", "x", "out"):
        args = {"A": A, "b": b, "x": x, "out": out}
        args[name] = host[name]
        with pytest.raises(aln.AlnError) as e:
            aln.aln_kkt_residual_noalloc(args["A"], d, n, d, aln.DTYPE_F32, args["b"],
                                         args["x"], args["out"])
        assert e.value.code == aln.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)   # nothing was launched
    assert np.all(host["out"] == 0.0)


def test_noalloc_rejects_sizes_beyond_the_scratch(aln):
    import torch
    A = torch.zeros((8, 4), dtype=torch.float32, device="cuda")
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    big_n = (1 << 21)  # 3n alone exceeds ALN_NOALLOC_SCRATCH_DOUBLES
    with pytest.raises(aln.AlnError) as e:
        aln.aln_kkt_residual_noalloc(A, 8, big_n, 8, aln.DTYPE_F32, A, x, out)
    assert e.value.code == aln.ERR_INVALID_ARG
