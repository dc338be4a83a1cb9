"""Write the oracle's results for the 4096-water box (seed 2, rc 9 A, SPME
64^3 order 5, alpha 0.4) to water4096_oracle.npz: every energy term, the PCG
residual, and the forces and induced dipoles of a seeded sample of 256
molecules.  Calls only synth/ and oracle/.

    python tests/golden/make_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "water4096_oracle.npz")


def main():
    s, o = synth.make_config("water4096")
    t = time.time()
    ref = oracle.evaluate(s, o, tol_D=1e-10, chunk=4096)
    dt = time.time() - t
    sample = np.sort(np.random.default_rng(4096).choice(s.n_mol, 256, replace=False))
    np.savez_compressed(OUT, terms=np.array([ref["terms"][k] for k in oracle.TERMS + ("total",)]),
                        term_names=np.array(oracle.TERMS + ("total",)), sample=sample,
                        forces=ref["forces"][sample], mu=ref["mu"][sample], iters=ref["iters"],
                        resid_D=ref["resid_D"], seconds=dt)
    print(OUT, dt, ref["terms"], ref["iters"], ref["resid_D"])


if __name__ == "__main__":
    main()
