"""Checkpoint / resume of the CNN trainer (host logic, no GPU): the state
round-trips exactly, and a write that dies half-way leaves the previous
checkpoint as it was."""
import os

import numpy as np
import pytest

from paper_2001_09632_gb300 import train


def _state(seed, step):
    rng = np.random.default_rng(seed)
    return {"params": rng.standard_normal(100).astype(np.float32), "m": rng.random(100).astype(np.float32),
            "v": rng.random(100).astype(np.float32), "gen": rng.integers(0, 256, 16, dtype=np.uint8),
            "step": np.int64(step), "hist": np.array([[1, 0.5], [200, 0.25]])}


def test_round_trip(tmp_path):
    path = str(tmp_path / "ckpt.npz")
    assert train.load_checkpoint(path) is None
    st = _state(0, 700)
    train.save_checkpoint(path, st)
    back = train.load_checkpoint(path)
    assert set(back) == set(st)
    for k in st:
        assert np.array_equal(back[k], st[k]) and back[k].dtype == np.asarray(st[k]).dtype


def test_interrupted_write_keeps_the_previous_checkpoint(tmp_path, monkeypatch):
    path = str(tmp_path / "ckpt.npz")
    train.save_checkpoint(path, _state(1, 500))

    def dying_savez(f, **kw):
        f.write(b"PK\x03\x04 half a zip")                           # some bytes, then the process dies
        raise KeyboardInterrupt

    monkeypatch.setattr(train.np, "savez", dying_savez)
    with pytest.raises(KeyboardInterrupt):
        train.save_checkpoint(path, _state(2, 1000))
    monkeypatch.undo()
    back = train.load_checkpoint(path)
    assert int(back["step"]) == 500
    assert np.array_equal(back["params"], _state(1, 500)["params"])
    # the next save replaces both the stale temporary file and the checkpoint
    train.save_checkpoint(path, _state(3, 1500))
    assert int(train.load_checkpoint(path)["step"]) == 1500
    assert not os.path.exists(path + ".tmp")
