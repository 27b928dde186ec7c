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


def test_feature_kind_is_checked_and_survives_save_and_load(tmp_path):
    """A classifier remembers whether it takes symbol-curve or eigenvalue features: the
    kind is saved with it, and a context of the other kind is refused before any kernel."""
    pytest.importorskip("torch")
    with pytest.raises(ValueError):
        restriction.Restriction("cpu", features="eigenvalues")
    eig = restriction.Restriction("cpu", net="dual", features="eigen")
    path = str(tmp_path / "eig.npz")
    eig.save(path)
    back = restriction.Restriction.load(path, "cpu")
    assert back.features == "eigen" and back.net == "dual"
    sym = restriction.Restriction("cpu", net="mlp")
    assert sym.features == "symbol"
    ctx_sym = restriction.MatrixContext(None, 1, 1, None, None, None)
    ctx_eig = restriction.MatrixContext(None, 1, 1, None, None, None, spectrum=object())
    with pytest.raises(ValueError):
        sym._check_ctx(ctx_eig)
    with pytest.raises(ValueError):
        eig._check_ctx(ctx_sym)
    sym._check_ctx(ctx_sym)
    eig._check_ctx(ctx_eig)
    with pytest.raises(ValueError):  # spectra exactly for the eigenvalue kind
        sym.build_training_set([(None, 1, 1)], [None], np.random.default_rng(0), spectra=[np.zeros(3)])


@pytest.mark.parametrize("net", ["mlp", "dual"])
def test_shipped_classifiers_take_symbol_features(net):
    import os
    pytest.importorskip("torch")
    path = os.path.join(os.path.dirname(restriction.__file__), "data", f"restriction_{net}.npz")
    r = restriction.Restriction.load(path, "cpu")
    assert r.net == net and r.features == "symbol" and 0.01 < r.tau < 1.0
