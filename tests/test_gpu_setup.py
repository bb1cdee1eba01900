"""GPU tests of context set-up: the symmetry check runs on the device against
the edge set (the host checks the rows first), and names the same pair the
host-only check names; valid graphs of every size class pass it."""
import numpy as np
import pytest

from conftest import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def B():
    from paper_2011_03479_gb300 import binding
    binding.load()
    return binding


def _drop_reverse(rp, ci, i):
    """Remove slot (j, i) for the first neighbour j > i of i: (i, j) loses its reverse."""
    row = ci[rp[i]:rp[i + 1]]
    j = int(row[row > i][0])
    e = rp[j] + int(np.searchsorted(ci[rp[j]:rp[j + 1]], i))
    ci2 = np.delete(ci, e)
    rp2 = rp.copy()
    rp2[j + 1:] -= 1
    return rp2, ci2, j


@pytest.mark.parametrize("d", [2, 16])
def test_asymmetric_graph_rejected_on_device(B, d):
    from paper_2011_03479_gb300 import inputs
    rp, ci = inputs.rmat(12, 8, seed=41)
    i = int(np.argmax(np.diff(rp) > 3))
    rp2, ci2, j = _drop_reverse(rp, ci, i)
    with pytest.raises(B.GempeError) as ei:
        B.gempe_create(rp2, ci2, d)
    assert ei.value.status == -2
    with pytest.raises(B.GempeError) as eh:
        B.gempe_validate_csr(rp2, ci2)
    assert str(ei.value) == str(eh.value)
    assert "without its reverse" in str(ei.value)
    # the intact graph is accepted
    with B.gempe_create(rp, ci, d) as ctx:
        B.gempe_step(ctx, 1)


def test_tiny_asymmetric_graph(B):
    rp = np.array([0, 1, 1, 1], np.int32)
    ci = np.array([1], np.int32)
    with pytest.raises(B.GempeError) as ei:
        B.gempe_create(rp, ci, 2)
    assert ei.value.status == -2 and "(0,1) without its reverse" in str(ei.value)


def test_batch_asymmetric_graph_named(B):
    """In a batch the device check names the graph by its index."""
    good = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), 2)
    asym = (np.array([0, 1, 1], np.int32), np.array([1], np.int32), 2)
    with pytest.raises(B.GempeError) as ei:
        B.gempe_batch_create([good, good, asym])
    assert ei.value.status == -2 and "graph 2" in str(ei.value) and "without its reverse" in str(ei.value)
