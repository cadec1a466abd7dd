"""Host utilities (no GPU): the autotuner's schedule cache and Davidson checkpoints."""
import json
import os

import numpy as np
import pytest

from paper_2309_03513_b300 import runtime as R


def test_tuning_key_separates_every_identity_field():
    base = dict(n=72, nocc_src=128, nocc_tgt=128, nb=8, precision=1, spin_flip=False, device="NVIDIA B300")
    keys = {R.tuning_key(**base)}
    for field, other in (("n", 64), ("nocc_src", 127), ("nocc_tgt", 126), ("nb", 4), ("precision", 0),
                         ("spin_flip", True), ("device", "other GPU")):
        keys.add(R.tuning_key(**dict(base, **{field: other})))
    assert len(keys) == 8


def test_tuning_cache_round_trip_keeps_other_entries(tmp_path):
    path = str(tmp_path / "tuning.json")
    assert R.load_tuning(path, "a") is None  # no file yet
    t1 = {"targets": 32, "sources": 8, "k1d_block": 16, "accumulate": 1, "graph": 1}
    t2 = {"targets": 16, "sources": 4, "k1d_block": 8, "accumulate": 0}
    R.store_tuning(path, "a", t1)
    R.store_tuning(path, "b", t2)
    assert R.load_tuning(path, "a") == {k: t1[k] for k in R.TUNED_FIELDS}  # only the tuned fields are kept
    assert R.load_tuning(path, "b") == t2
    R.store_tuning(path, "a", t2)  # replaced in place
    assert R.load_tuning(path, "a") == t2 and R.load_tuning(path, "b") == t2
    assert sorted(os.listdir(tmp_path)) == ["tuning.json"]  # no temporary file left behind
    with open(path) as fh:
        table = json.load(fh)
    table["c"] = {"targets": 8}  # an incomplete entry is not a cached schedule
    with open(path, "w") as fh:
        json.dump(table, fh)
    assert R.load_tuning(path, "c") is None
    assert R.load_tuning(path, "missing") is None


def test_davidson_checkpoint_round_trip_and_size_checks(tmp_path):
    rng = np.random.default_rng(5)
    v = rng.standard_normal((3, 4, 17)) + 1j * rng.standard_normal((3, 4, 17))
    theta = np.array([0.1, 0.2, 0.3])
    path = str(tmp_path / "dav.npz")
    R.save_checkpoint(path, v, theta, n=12, npw=17, nocc_src=4, step=9)
    got_v, got_t, step = R.load_checkpoint(path, n=12, npw=17, nocc_src=4)
    assert np.array_equal(got_v, v) and np.array_equal(got_t, theta) and step == 9
    assert sorted(os.listdir(tmp_path)) == ["dav.npz"]
    with pytest.raises(ValueError):
        R.load_checkpoint(path, n=16, npw=17, nocc_src=4)  # another grid
    with pytest.raises(ValueError):
        R.load_checkpoint(path, n=12, npw=17, nocc_src=5)  # another orbital count
    with pytest.raises(ValueError):
        R.save_checkpoint(path, v, theta[:2], n=12, npw=17, nocc_src=4, step=1)  # values do not match
    with pytest.raises(ValueError):
        R.save_checkpoint(path, v, theta, n=12, npw=18, nocc_src=4, step=1)  # rows do not match
