"""Write synth_water4096.json: fingerprints of the seeded 4096-water inputs
that water4096_oracle.npz was computed from (a few molecules' positions and
local multipoles, and column sums), so that a change of the generator shows
up on the host before the stored oracle results go stale.  Calls only synth/.

    python tests/golden/make_synth_fixture.py
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
            "pos_sum": s.pos.sum(axis=(0, 1)).tolist(), "mp_sum": s.mp_local.sum(axis=0).tolist()}


def main():
    out = os.path.join(HERE, "synth_water4096.json")
    with open(out, "w") as f:
        json.dump(fingerprint(), f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
