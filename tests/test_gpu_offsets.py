"""gwam_cell_offsets: per-cell segment offsets of a cell-ordered array, against a brute-force count."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _expected(cells, ncell):
    return np.searchsorted(np.sort(cells), np.arange(ncell + 1), side="left").astype(np.int32)


@pytest.mark.parametrize("n,ncell", [(0, 5), (1, 1), (1000, 37), (4097, 2049), (1_000_000, 2_949_120),
                                     (300_000, 2048 * 3 + 1)])
def test_offsets_match_brute_force(gw, n, ncell):
    import torch
    rng = np.random.default_rng(n + ncell)
    cells = np.sort(rng.integers(0, ncell, n)).astype(np.int32)
    got = gw.cell_offsets(torch.from_numpy(cells).cuda(), ncell).cpu().numpy()
    np.testing.assert_array_equal(got, _expected(cells, ncell))


def test_offsets_of_unsorted_input_are_the_count_prefix(gw):
    import torch
    rng = np.random.default_rng(3)
    cells = rng.integers(0, 500, 20000).astype(np.int32)
    got = gw.cell_offsets(torch.from_numpy(cells).cuda(), 500).cpu().numpy()
    np.testing.assert_array_equal(got, _expected(cells, 500))


def test_out_of_range_cells_are_rejected(gw):
    import torch
    cells = torch.tensor([0, 1, 7, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(gw.GwamError) as e:
        gw.cell_offsets(cells, 5)
    assert e.value.code == gw.GWAM_EINVAL
