"""GPU analytic FMO gradient (fmo_get_gradient through the C ABI) against the
oracle's analytic FMO1/FMO2/FMO3 gradients (oracle/fmo_gradient.py), which
central finite differences of the oracle's FMO energies pin
(tests/test_fmo_gradient_oracle.py).  Bar: 1e-7 Eh/bohr per component, both
sides converged to 1e-10 (GPU) / 1e-12 (oracle) in the charges."""
import dataclasses
import os

import numpy as np
import pytest

from oracle import fmo as ofmo
from oracle import fmo_gradient as ofg
from paper_2606_28022_b300.inputs import geometry as G

pytestmark = pytest.mark.gpu

G_TOL = 1e-7
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def gpu(params):
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo.FMO(params, 0)


def _grad(gpu, system, **kw):
    from paper_2606_28022_b300 import fmo
    gpu.set_system(system)
    gpu.run(fmo.options(**kw))
    return gpu.gradient()


def test_fmo1_gradient_three_waters(gpu, params, water64):
    s = water64.subsystem([0, 1, 2])
    ref = ofg.fmo1_gradient(s, params)
    g = _grad(gpu, s, level=1)
    assert np.abs(ref).max() > 1e-3
    assert np.max(np.abs(g - ref)) < G_TOL


def test_fmo2_gradient_water8_scc_and_esdim(gpu, params, water64):
    s = water64.subsystem(range(8))
    r = ofmo.fmo(s, params, ofmo.FMOOptions())
    assert r.dimer_scc.any() and not r.dimer_scc.all()
    ref = ofg.fmo2_gradient(s, params)
    g = _grad(gpu, s, level=2)
    assert np.max(np.abs(g - ref)) < G_TOL


def test_fmo3_gradient_water4_all_trimers(gpu, params, water64):
    s = water64.subsystem(range(4))
    opts = ofmo.FMOOptions(level=3, all_dimers_scc=True, trimer_cut=1e9)
    ref = ofg.fmo3_gradient(s, params, opts)
    g = _grad(gpu, s, level=3, all_dimers_scc=1, trimer_cut=1e9)
    assert np.max(np.abs(g - ref)) < G_TOL


def test_fmo3_gradient_water6_cut_rule(gpu, params, water64):
    # the 4.0 A rule for dimers and trimers: a mix of SCC dimers, ES-DIM pairs
    # and trimers, coefficients from the inclusion-exclusion of Eq. 16
    s = water64.subsystem(range(6))
    ref = ofg.fmo3_gradient(s, params)
    r = ofmo.fmo(s, params, ofmo.FMOOptions(level=3))
    g = _grad(gpu, s, level=3)
    assert np.max(np.abs(g - ref)) < G_TOL
    assert len(r.trimers) >= 0


def test_fmo2_gradient_anthracene3(gpu, params):
    a, _ = G.anthracene_cluster(128, 2)
    s = a.subsystem([0, 1, 2])
    ref = ofg.fmo2_gradient(s, params, ofmo.FMOOptions(all_dimers_scc=True))
    g = _grad(gpu, s, all_dimers_scc=1)
    assert np.max(np.abs(g - ref)) < G_TOL


def test_fmo3_gradient_pentacene4_golden(gpu, params):
    # the C4-shaped piece of the pentacene crystal (trimers of n = 348); the
    # oracle's gradient (110 s in NumPy) is stored by tests/golden/make_golden.py
    path = os.path.join(GOLDEN, "pentacene4_fmo3_gradient.txt")
    ref = np.loadtxt(path).reshape(-1, 3)
    s, _ = G.pentacene_cluster(660, 4)
    s = s.subsystem([0, 2, 93, 1])
    g = _grad(gpu, s, level=3)
    assert np.max(np.abs(g - ref)) < G_TOL


def test_gradient_mixed_precision_with_want_gradient(gpu, params, water64):
    # mixed precision: the FP32 phase hands over to FP64 iterations that
    # converge every n-mer density; the gradient equals the FP64 run's
    from paper_2606_28022_b300 import fmo
    s = water64.subsystem(range(8))
    g64 = _grad(gpu, s, level=2)
    gpu.run(fmo.options(level=2, precision="mixed"))
    with pytest.raises(fmo.FMOError):
        gpu.gradient()                          # FP32-converged n-mer densities: refused
    gmx = _grad(gpu, s, level=2, precision="mixed", want_gradient=1)
    assert np.max(np.abs(gmx - g64)) < G_TOL


def test_gradient_translation_invariance_anthracene16(gpu, params):
    # a property that holds at any size: the forces of an isolated system sum
    # to zero; and the Z-vector solve converged
    a, _ = G.anthracene_cluster(128, 2)
    s = a.subsystem(range(16))
    g = _grad(gpu, s, level=2)
    assert np.abs(g).max() > 1e-3
    assert np.max(np.abs(g.sum(axis=0))) < 1e-8
    st = gpu.stats()
    assert st["zvector_iterations"] > 0 and st["zvector_residual"] < 1e-10


def test_fmo2_gradient_fractional_occupations(params, water64):
    # a high electronic temperature: every fragment has fractional frontier
    # occupations; the response takes the full Fermi form (M_ij over all
    # orbital pairs and the Fermi-level shift)
    from paper_2606_28022_b300 import fmo
    hot = dataclasses.replace(params, t_el=15000.0)
    s = water64.subsystem([0, 1, 2, 3])
    ref = ofg.fmo2_gradient(s, hot, ofmo.FMOOptions(all_dimers_scc=True))
    g = fmo.FMO(hot, 0)
    g.set_system(s)
    g.run(fmo.options(all_dimers_scc=1))
    grad = g.gradient()
    g.close()
    assert np.max(np.abs(grad - ref)) < G_TOL
