"""FP64 CPU oracle for the SIBFA21 intermolecular water potential.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import it; the product package never does,
and the two share no code (only the seeded inputs from `synth`).

Pins (tests/test_oracle_*.py): finite-difference forces per term, rotation
and translation invariance and zero net force/torque in the gas phase,
textbook two-site closed forms, Thole and kernel recurrences, Ewald alpha
independence and agreement with an exact k-space sum and a direct lattice sum,
B-spline partition of unity, symmetry of T, PCG against a dense solve, the
polarization-energy identity at the solution, the penetration b -> infinity
limit, and hand evaluations of the paper's formulas on laid-out geometries:
lone-pair and frame geometry, the rotated multipoles' potential, bond-bond,
bond-lone pair and lone pair-lone pair repulsion, one pair of each
dispersion/exchange-dispersion kind, a donor-acceptor charge-transfer case
and V_int; the gas-phase lone-pair potential against the textbook multipole
potential; and alpha independence of the periodic lone-pair potential,
permanent field, induced dipoles and polarization energy.

Parity with the paper's printed energies (Tables 1-2) is unpinned: the
parameters, lone-pair positions and geometries they need are not in the
paper's text.
"""
from .evaluate import TERMS, energy_only, evaluate  # noqa: F401
