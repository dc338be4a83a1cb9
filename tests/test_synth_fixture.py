"""The seeded water-box inputs and the parameter table are those the stored
oracle results (tests/golden/<config>_oracle.npz) were computed from: the
generator still reproduces the fingerprints recorded beside them."""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_synth_fixture  # noqa: E402


@pytest.mark.parametrize("config", ["water4096", "water32000"])
def test_inputs_match_recorded_fingerprints(config):
    with open(os.path.join(HERE, "golden", f"synth_{config}.json")) as f:
        rec = json.load(f)
    now = make_synth_fixture.fingerprint(rec["config"])
    assert now["n_mol"] == rec["n_mol"] and now["molecules"] == rec["molecules"]
    assert now["params"] == rec["params"]
    for k in ("box", "pos", "mp_local", "pos_sum", "mp_sum"):
        np.testing.assert_allclose(np.array(now[k]), np.array(rec[k]), rtol=1e-12, atol=1e-12, err_msg=k)
