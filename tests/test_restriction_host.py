"""Host logic of the learned restriction (no GPU): the box dilation and the paper's
metrics (Sec. 5.2) on hand-made masks, and the hierarchical map's cell selection."""
import numpy as np
import pytest

from paper_2605_04550_gb300 import restriction


def test_dilate_matches_brute_force():
    rng = np.random.default_rng(0)
    m = rng.random((23, 31)) < 0.05
    for r in (0, 1, 2, 3):
        ref = np.zeros_like(m)
        for i in range(m.shape[0]):
            for j in range(m.shape[1]):
                ref[i, j] = m[max(i - r, 0):i + r + 1, max(j - r, 0):j + r + 1].any()
        np.testing.assert_array_equal(restriction.dilate_np(m, r), ref)


def test_recall_coverage_precision_definitions():
    truth = np.zeros((10, 10), dtype=bool)
    truth[4:6, 4:6] = True                     # 4 points; 3x3-dilated: 16 points (3:7 x 3:7)
    pred = np.zeros_like(truth)
    pred[3:7, 3:6] = True                      # 12 points, covers 12 of the 16 dilated
    m = restriction.recall_metrics(truth, pred)
    assert m["recall"] == pytest.approx(12 / 16)
    assert m["coverage"] == pytest.approx(1.0)
    assert m["precision"] == pytest.approx(4 / 12)
    assert m["grid_fraction"] == pytest.approx(0.12)
    assert restriction.recall_metrics(np.zeros_like(truth), pred)["recall"] == 1.0


def test_hierarchical_mask_keeps_flagged_cells_and_neighbours():
    torch = pytest.importorskip("torch")
    full = torch.zeros((20, 24))
    full[9, 13] = 0.9                          # one fine point high
    full[8, 12] = 0.95                         # coarse anchor (8, 12) -> cell (2, 3)
    h = restriction.Restriction.hierarchical_mask(full, 0.5)
    keep = h != 0
    # cell (2, 3) and its neighbours (rows 1..3, cols 2..4 in cells) keep their fine values
    assert keep[9, 13] and keep[8, 12]
    assert not keep[0, 0] or full[0, 0] == 0
    kept_cells = set()
    for i in range(20):
        for j in range(24):
            if keep[i, j]:
                kept_cells.add((i // 4, j // 4))
    assert kept_cells <= {(a, b) for a in (1, 2, 3) for b in (2, 3, 4)}
