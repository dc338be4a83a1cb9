"""Write synth_<config>.json: fingerprints of the seeded water-box inputs
that <config>_oracle.npz was computed from (a few molecules' positions and
local multipoles, column sums, and the parameter table), so that a change of
the generator or of the parameters shows up on the host before the stored
oracle results go stale.  Calls only synth/.

    python tests/golden/make_synth_fixture.py [water4096 water32000]
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def fingerprint(name="water4096"):
    s, _ = synth.make_config(name)
    idx = [0, s.n_mol // 3, 2 * s.n_mol // 3, s.n_mol - 1]
    return {"config": name, "n_mol": s.n_mol, "box": s.box.tolist(), "molecules": idx,
            "pos": s.pos[idx].tolist(), "mp_local": s.mp_local[idx].tolist(),
            "pos_sum": s.pos.sum(axis=(0, 1)).tolist(), "mp_sum": s.mp_local.sum(axis=0).tolist(),
            "params": dict(synth.PARAMS)}


def main(names=("water4096", "water32000")):
    for name in names:
        out = os.path.join(HERE, f"synth_{name}.json")
        with open(out, "w") as f:
            json.dump(fingerprint(name), f, indent=1)
        print(out)


if __name__ == "__main__":
    main(sys.argv[1:] or ("water4096", "water32000"))
