"""Host logic of the calibration driver (no GPU): the GA checkpoint format."""
import numpy as np
import pytest

from paper_1701_03549_gb300 import calibrate


def test_checkpoint_round_trip_and_run_identity(tmp_path):
    path = str(tmp_path / "ga.npz")
    rng = np.random.default_rng(0)
    hist = calibrate.History([rng.normal(size=(8, 7)) for _ in range(3)],
                             [rng.random(8) for _ in range(3)],
                             [0.5, 0.25, 0.125])
    genes = rng.normal(size=(8, 7))
    meta = calibrate._meta("ga7", pop=8, reps=2, ga_seed=3, lo=-30.0)
    calibrate.save_checkpoint(path, 3, genes, hist, meta)
    g, genes2, hist2 = calibrate.load_checkpoint(path, meta)
    assert g == 3 and np.array_equal(genes2, genes)
    for a, b in zip(hist.params + hist.fitness, hist2.params + hist2.fitness):
        assert np.array_equal(a, b)
    assert hist2.seconds == hist.seconds
    other = calibrate._meta("ga7", pop=8, reps=2, ga_seed=4, lo=-30.0)
    with pytest.raises(ValueError):
        calibrate.load_checkpoint(path, other)
    assert not (tmp_path / "ga.npz.tmp.npz").exists()


def test_scar_layout_orders_individual_scar_replicate():
    """Simulation j of a multi-scar generation belongs to individual
    j // (K R) and scar (j // R) % K, so that one group mean of size K R per
    individual averages over its scars and replicates."""
    from paper_1701_03549_gb300 import calibrate

    P, K, R = 3, 4, 2
    lay = calibrate.scar_layout(P, K, R)
    assert lay.dtype == np.int32 and lay.shape == (P * K * R,)
    j = np.arange(P * K * R)
    assert np.array_equal(lay, (j // R) % K)
    assert np.array_equal(np.bincount(lay), np.full(K, P * R))
