"""Checkpoint / resume of the outer-iteration state (host logic, no GPU)."""
import json
import os

import numpy as np
import pytest

from paper_2012_15662_gb300.checkpoint import CheckpointError, load_state, save_state


def _state(nb=7, ng=6, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nb, nb)), rng.uniform(0.05, 0.3, ng), np.sort(rng.standard_normal(nb))


def test_round_trip_is_bitwise(tmp_path):
    C, g, d = _state()
    C[0, 0] = np.nextafter(1.0, 2.0)  # a value a decimal format would round
    j = save_state(str(tmp_path / "s"), "square4", C, g, d, -11.39, 7, True, "fp64", extra={"seed": 1})
    assert j.endswith("s.json") and os.path.exists(str(tmp_path / "s.bin"))
    r = load_state(str(tmp_path / "s.json"), workload="square4", nbf=7)
    for a, b in ((r["C"], C), (r["gamma"], g), (r["diag"], d)):
        assert a.dtype == np.float64
        np.testing.assert_array_equal(a, b)
    assert (r["E"], r["outer"], r["converged"], r["form"], r["extra"]) == (-11.39, 7, True, "fp64", {"seed": 1})
    # a second write replaces the first and leaves no temporary files
    save_state(str(tmp_path / "s"), "square4", 2 * C, g, d, -11.4, 8, False, "fp64")
    assert load_state(str(tmp_path / "s"))["outer"] == 8
    assert sorted(os.listdir(tmp_path)) == ["s.bin", "s.json"]


def test_damage_and_mismatch_are_reported(tmp_path):
    C, g, d = _state()
    p = str(tmp_path / "s")
    save_state(p, "c6h12", C, g, d, -224.7, 3, False, "slice4")
    with pytest.raises(CheckpointError, match="workload"):
        load_state(p, workload="c10h20")
    with pytest.raises(CheckpointError, match="nbf"):
        load_state(p, nbf=8)
    raw = bytearray(open(p + ".bin", "rb").read())
    raw[17] ^= 1
    open(p + ".bin", "wb").write(bytes(raw))
    with pytest.raises(CheckpointError, match="checksum"):
        load_state(p)
    open(p + ".bin", "wb").write(bytes(raw[:-8]))
    with pytest.raises(CheckpointError, match="bytes"):
        load_state(p)
    meta = json.load(open(p + ".json"))
    meta["version"] = 99
    json.dump(meta, open(p + ".json", "w"))
    with pytest.raises(CheckpointError, match="version"):
        load_state(p)
    with pytest.raises(CheckpointError, match="cannot read"):
        load_state(str(tmp_path / "missing"))


def test_inconsistent_or_non_finite_state_is_not_written(tmp_path):
    C, g, d = _state()
    with pytest.raises(CheckpointError, match="shapes"):
        save_state(str(tmp_path / "a"), "w", C[:, :6], g, d, 0.0, 1, False, "fp64")
    C[2, 3] = np.nan
    with pytest.raises(CheckpointError, match="non-finite"):
        save_state(str(tmp_path / "b"), "w", C, g, d, 0.0, 1, False, "fp64")
    assert os.listdir(tmp_path) == []
