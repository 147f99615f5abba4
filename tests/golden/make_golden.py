"""Write the stored expected values of tests/ from the FP64 oracle alone.

    python tests/golden/make_golden.py

pentacene4_fmo3_gradient.txt: the analytic FMO3 gradient (Eh/bohr, atoms x
3 in the input order) of molecules 0, 2, 93 and 1 of the seeded 660-molecule
pentacene crystal (every pair an SCC dimer, the trimers of n = 348 basis
functions), from oracle.fmo_gradient.fmo3_gradient; about two minutes in
NumPy, too slow to recompute inside the GPU test.  The oracle's FMO3 gradient
is pinned to central finite differences by tests/test_fmo_gradient_oracle.py.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

from oracle import fmo as ofmo  # noqa: E402
from oracle import fmo_gradient as ofg  # noqa: E402
from paper_2606_28022_b300.inputs import geometry as G  # noqa: E402
from paper_2606_28022_b300.inputs.params import synthetic_gfn1_table  # noqa: E402


def main():
    params = synthetic_gfn1_table()
    s, _ = G.pentacene_cluster(660, 4)
    s = s.subsystem([0, 2, 93, 1])
    g = ofg.fmo3_gradient(s, params, ofmo.FMOOptions(level=3))
    np.savetxt(os.path.join(HERE, "pentacene4_fmo3_gradient.txt"), g, fmt="%.17e",
               header="oracle fmo3_gradient, pentacene molecules 0 2 93 1 of pentacene_cluster(660, 4); Eh/bohr")


if __name__ == "__main__":
    main()
