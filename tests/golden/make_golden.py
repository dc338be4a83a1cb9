"""Write the oracle's results for a water-box workload to
<name>_oracle.npz: every energy term, the PCG residual, and the forces and
induced dipoles of a seeded sample of 256 molecules.  Calls only synth/ and
oracle/.

    python tests/golden/make_golden.py [water4096|water32000]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main(name="water4096"):
    s, o = synth.make_config(name)
    t = time.time()
    ref = oracle.evaluate(s, o, tol_D=1e-10, chunk=4096)
    dt = time.time() - t
    sample = np.sort(np.random.default_rng(s.n_mol).choice(s.n_mol, 256, replace=False))
    out = os.path.join(HERE, f"{name}_oracle.npz")
    np.savez_compressed(out, terms=np.array([ref["terms"][k] for k in oracle.TERMS + ("total",)]),
                        term_names=np.array(oracle.TERMS + ("total",)), sample=sample,
                        forces=ref["forces"][sample], mu=ref["mu"][sample], iters=ref["iters"],
                        resid_D=ref["resid_D"], seconds=dt)
    print(out, dt, ref["terms"], ref["iters"], ref["resid_D"])


if __name__ == "__main__":
    main(*sys.argv[1:])
