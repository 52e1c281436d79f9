"""The sparse input recipe (workloads.banded_tall) and the CSC helpers: the
structure the CSC entry point requires, the window each column lives in, the
stated sizes, and the round trip between the dense and CSC forms."""
import numpy as np

from oracle import sparse as S
from paper_1502_01645_gb300 import workloads as W


def test_banded_tall_structure():
    p = W.banded_tall(d=5000, n=300, band=400, density=0.25, seed=3)
    per = int(round(0.25 * 400))
    assert p.col_ptr.dtype == np.int64 and p.row_idx.dtype == np.int32
    assert p.nnz == 300 * per and p.meta["nnz"] == p.nnz
    S.check_csc(p.d, p.n, p.col_ptr, p.row_idx, p.vals)   # sorted, in range
    for j in (0, 1, 150, 299):
        rows = p.row_idx[p.col_ptr[j]:p.col_ptr[j + 1]]
        r0 = int(round(j * (5000 - 400) / 299))
        assert rows.min() >= r0 and rows.max() < r0 + 400
    assert np.all(p.vals > 0)
    assert p.B.shape == (1, 5000) and p.B.dtype == np.float32


def test_banded_tall_is_seeded():
    a = W.banded_tall(d=2000, n=100, band=200, density=0.1, seed=9)
    b = W.banded_tall(d=2000, n=100, band=200, density=0.1, seed=9)
    c = W.banded_tall(d=2000, n=100, band=200, density=0.1, seed=10)
    np.testing.assert_array_equal(a.row_idx, b.row_idx)
    np.testing.assert_array_equal(a.B, b.B)
    assert not np.array_equal(a.row_idx, c.row_idx)


def test_dense_and_csc_round_trip():
    p = W.banded_tall(d=700, n=90, band=100, density=0.3, seed=4)
    A = p.dense()
    assert A.flags.f_contiguous and A.dtype == np.float32
    np.testing.assert_array_equal(A, S.csc_to_dense(p.d, p.n, p.col_ptr, p.row_idx, p.vals))
    cp, ri, v = W.to_csc(A)
    np.testing.assert_array_equal(cp, p.col_ptr)
    np.testing.assert_array_equal(ri, p.row_idx)
    np.testing.assert_array_equal(v, p.vals)


def test_bench_block_pair_count_matches_brute_force():
    """The block-sparse Gram's algorithmic work in bench.py: occupied
    (64-row block, tile pair) combinations, counted by brute force."""
    import bench
    p = W.banded_tall(d=3000, n=300, band=500, density=0.05, seed=12)
    off, diag = bench.sgram_block_products(p)
    cols = np.repeat(np.arange(p.n), np.diff(p.col_ptr))
    T = (p.n + 127) // 128
    occ = [set() for _ in range(T)]
    for r, c in zip(p.row_idx.tolist(), cols.tolist()):
        occ[c // 128].add(r // 64)
    assert diag == sum(len(o) for o in occ)
    assert off == sum(len(occ[i] & occ[j]) for i in range(T) for j in range(i))
