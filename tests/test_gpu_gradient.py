"""GPU analytic gradient (fmo_get_gradient, through the C ABI) of systems that
are one fragment against the oracle's analytic single-system gradient, itself
pinned to finite differences (tests/test_gradient_oracle.py).  Several
fragments: tests/test_gpu_fmo_gradient.py."""
import dataclasses

import numpy as np
import pytest

from oracle import gradient as ograd
from paper_2606_28022_b300.inputs import geometry as G

pytestmark = pytest.mark.gpu

G_TOL = 1e-7     # Eh/bohr: both sides converged to 1e-10 in the charges


@pytest.fixture(scope="module")
def gpu(params):
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo.FMO(params, 0)


def _one_fragment(s):
    return dataclasses.replace(s, frag=np.zeros(len(s.Z), dtype=s.frag.dtype),
                               frag_charge=np.array([float(np.sum(s.frag_charge))]))


@pytest.mark.parametrize("name", ["water_dimer", "alanine", "anthracene"])
def test_gradient_of_one_fragment_system_matches_oracle(gpu, params, water64, name):
    from paper_2606_28022_b300 import fmo
    if name == "water_dimer":
        s = _one_fragment(water64.subsystem([3, 7]))
    elif name == "alanine":
        s = G.polyalanine_helix(1)
    else:
        s = G.anthracene_cluster(8, 2)[0].subsystem([0])
    assert s.n_frag == 1 and len(s.cut_bonds) == 0
    gpu.set_system(s)
    gpu.run(fmo.options(level=1))
    g = gpu.gradient()
    ref = ograd.scc_gradient(s.Z, s.xyz, params)
    assert np.abs(ref).max() > 1e-3
    assert np.max(np.abs(g - ref)) < G_TOL


def test_gradient_refuses_what_it_does_not_cover(gpu, params, water64):
    from paper_2606_28022_b300 import fmo
    gpu.set_system(water64.subsystem([0]))
    gpu.run(fmo.options(precision="mixed"))
    with pytest.raises(fmo.FMOError):
        gpu.gradient()                 # n-mer densities not converged in FP64
    gpu.set_system(G.polyalanine_helix(3))
    gpu.run(fmo.options())
    with pytest.raises(fmo.FMOError):
        gpu.gradient()                 # cut bonds (hybrid orbital projection)


def test_gradient_with_fractional_occupations(params):
    # a high electronic temperature smears the occupations over the frontier
    # orbitals: P and W~ are the Fermi-weighted sums over canonical orbitals
    from paper_2606_28022_b300 import fmo
    hot = dataclasses.replace(params, t_el=20000.0)
    s = G.polyalanine_helix(1)
    g = fmo.FMO(hot, 0)
    g.set_system(s)
    g.run(fmo.options(level=1))
    grad = g.gradient()
    g.close()
    ref = ograd.scc_gradient(s.Z, s.xyz, hot)
    assert np.max(np.abs(grad - ref)) < G_TOL
