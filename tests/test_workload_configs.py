"""The workload files under ``configs/`` and the JSON form of a workload.

Each file must describe exactly the named workload of the same name that
``workloads.workload`` builds (so ``bench.py --workload configs/<name>.json``
times the same link as ``--workload <index>``), and the JSON form must
round-trip and reject keys it does not know.
"""
import glob
import json
import os

import numpy as np
import pytest

from paper_1101_0086_gb300.workloads import WORKLOADS, Workload, load_workload, save_workload, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "configs", "*.json")))


def test_every_named_workload_has_a_file():
    names = {os.path.basename(f)[:-5] for f in FILES}
    assert names == {WORKLOADS[k]().name for k in WORKLOADS}


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_file_matches_the_built_in_workload(path):
    w = workload(path)
    assert w == workload(os.path.basename(path)[:-5])
    assert w.fiber.length_km == pytest.approx(w.length_km)


def test_round_trip_and_field(tmp_path):
    w = workload("0")
    p = str(tmp_path / "w.json")
    save_workload(w, p, note="round trip")
    w2 = load_workload(p)
    assert w2 == w
    np.testing.assert_array_equal(w2.field(), w.field())


def test_unknown_and_missing_keys_are_rejected():
    d = workload("0").to_dict()
    with pytest.raises(ValueError, match="unknown"):
        Workload.from_dict({**d, "mpa_Mx": 3})
    missing = dict(d)
    del missing["mpa_M"]
    with pytest.raises(ValueError, match="missing"):
        Workload.from_dict(missing)
    bad_fiber = json.loads(json.dumps(d))
    bad_fiber["fiber"]["loss"] = 0.2
    with pytest.raises(ValueError, match="fiber"):
        Workload.from_dict(bad_fiber)
