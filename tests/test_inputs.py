"""The seeded synthetic workloads have the shapes their recipes state.

The bench and the full-size parity tests name their workloads by these
recipes; a generator change that altered a graph would silently change
every measured figure, so the sizes are pinned here (and each graph is a
valid symmetric CSR with no loops or duplicates)."""
import numpy as np
import pytest

from paper_2011_03479_gb300 import inputs


def _valid(rp, ci):
    from paper_2011_03479_gb300 import binding
    binding.gempe_validate_csr(rp, ci)   # raises on an invalid graph


def test_sbm_1000_recipe():
    w = inputs.sbm_1000()
    rp, ci = w["row_ptr"], w["col_idx"]
    assert len(rp) - 1 == 1000 and len(ci) // 2 == 6888
    assert (w["d"], w["k"]) == (2, 5)
    _valid(rp, ci)


def test_rmat_s16_recipe():
    w = inputs.rmat_s16()
    rp, ci = w["row_ptr"], w["col_idx"]
    deg = np.diff(rp)
    assert len(rp) - 1 == 65536 and len(ci) // 2 == 910301
    assert int(deg.max()) == 9763 and int((deg == 0).sum()) == 18792
    assert (w["d"], w["k"], w["epochs"]) == (2, 10, 500)
    _valid(rp, ci)
    w2 = inputs.rmat_s16()
    np.testing.assert_array_equal(w2["col_idx"], ci)   # seeded: the same graph every time


def test_ba_1m_recipe():
    w = inputs.ba_1m()
    rp, ci = w["row_ptr"], w["col_idx"]
    assert len(rp) - 1 == 1_000_000 and len(ci) // 2 == 7_999_964
    assert w["d"] == 64
    assert int(np.diff(rp).min()) >= 8          # every vertex after the seed clique attaches 8 edges
    _valid(rp, ci)


def test_sbm_batch_256_recipe():
    w = inputs.sbm_batch_256()
    gs = w["graphs"]
    assert len(gs) == 256 and w["k"] == 5
    ns = [len(g["row_ptr"]) - 1 for g in gs]
    assert sum(ns) == 2_675_819
    assert sum(len(g["col_idx"]) // 2 for g in gs) == 25_492_493
    dims = [g["d"] for g in gs]
    assert (dims.count(2), dims.count(16), dims.count(64)) == (88, 75, 93)
    assert 500 <= min(ns) and max(ns) <= 50_000
    for g in gs[:8]:
        _valid(g["row_ptr"], g["col_idx"])
