"""Saving and loading the rank model's weights (host only)."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import rank_model


def test_round_trip(tmp_path):
    th = rank_model.init_theta(5)
    meta = {"train_sets": [dict(s) for s in rank_model.TRAIN_SETS], "loss": [0.5, 0.1]}
    path = tmp_path / "model.npz"
    rank_model.save(path, th, meta)
    th2, meta2 = rank_model.load(path)
    assert th2.dtype == np.float32 and np.array_equal(th2, th)
    assert meta2["loss"] == [0.5, 0.1] and meta2["nparam"] == rank_model.NPARAM
    assert meta2["train_sets"][1]["n"] == rank_model.TRAIN_SETS[1]["n"]


def test_refuses_other_sizes(tmp_path):
    with pytest.raises(ValueError):
        rank_model.save(tmp_path / "x.npz", np.zeros(10, np.float32))
    np.savez(tmp_path / "y.npz", theta=np.zeros(rank_model.NPARAM, np.float32),
             meta=np.frombuffer(b'{"nparam": 3}', np.uint8))
    with pytest.raises(ValueError):
        rank_model.load(tmp_path / "y.npz")
