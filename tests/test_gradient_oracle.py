"""Pins of the oracle's analytic GFN1-xTB gradient (oracle/gradient.py) to
facts outside it: central finite differences of the oracle's SCC energy (the
gradient's definition), finite differences of the overlap matrix and of the
coordination numbers (its two hand-differentiated building blocks), and the
translation and rotation invariance of an isolated system's energy."""
import numpy as np
import pytest

from oracle import fmo as ofmo
from oracle import gradient, xtb
from paper_2606_28022_b300.inputs import geometry as G

H = 1e-4            # central differences: error ~ h^2 E''' ~ 1e-9 here
FD_TOL = 2e-8       # Eh/bohr


def _energy(Z, xyz, params):
    cn = xtb.coordination_numbers(Z, xyz, params)
    return xtb.scc(Z, xyz, params, cn, tol=1e-12, e_tol=1e-13).energy


def _fd(f, xyz, k, c):
    xp = xyz.copy(); xp[k, c] += H
    xm = xyz.copy(); xm[k, c] -= H
    return (f(xp) - f(xm)) / (2 * H)


@pytest.fixture(scope="module")
def water_dimer(water64):
    return water64.subsystem([3, 7])


def test_water_dimer_gradient_equals_finite_differences(params, water_dimer):
    Z, xyz = water_dimer.Z, water_dimer.xyz.copy()
    g = gradient.scc_gradient(Z, xyz, params)
    fd = np.array([[_fd(lambda x: _energy(Z, x, params), xyz, k, c) for c in range(3)] for k in range(len(Z))])
    assert np.abs(g).max() > 1e-3
    assert np.max(np.abs(g - fd)) < FD_TOL


def test_alanine_gradient_equals_finite_differences(params):
    # C, N, O and H: p-p blocks, several element pairs, CN terms of all kinds
    s = G.polyalanine_helix(1)
    Z, xyz = s.Z, s.xyz.copy()
    g = gradient.scc_gradient(Z, xyz, params)
    rng = np.random.default_rng(5)
    for k in rng.choice(len(Z), size=4, replace=False):
        for c in range(3):
            assert abs(g[k, c] - _fd(lambda x: _energy(Z, x, params), xyz, k, c)) < FD_TOL


def test_overlap_and_cn_derivatives_equal_finite_differences(params):
    s = G.polyalanine_helix(1)
    Z, xyz = s.Z, s.xyz.copy()
    b = xtb.make_basis(Z, params)
    dS = gradient.overlap_derivative(Z, xyz, params, b)
    dcn = gradient.cn_derivative(Z, xyz, params)
    for k in (0, 4, 9):
        for c in range(3):
            fd_S = _fd(lambda x: xtb.overlap_matrix(Z, x, params, b), xyz, k, c)
            assert np.max(np.abs(dS[k, c] - fd_S)) < 1e-9
            fd_cn = _fd(lambda x: xtb.coordination_numbers(Z, x, params), xyz, k, c)
            assert np.max(np.abs(dcn[:, k, c] - fd_cn)) < 2e-8   # steep counting function: h^2 CN''' ~ 3e-9


def test_gradient_is_translation_and_rotation_invariant(params):
    a, _ = G.anthracene_cluster(8, 2)
    a = a.subsystem([0])
    g = gradient.scc_gradient(a.Z, a.xyz, params)
    assert np.max(np.abs(g.sum(axis=0))) < 1e-12                 # no net force
    assert np.max(np.abs(np.cross(a.xyz, g).sum(axis=0))) < 1e-11  # no net torque
    assert np.abs(g).max() > 1e-3


def test_fmo_gradient_one_fragment_equals_scc_gradient(params, water64):
    s = water64.subsystem([5])
    g_fmo = gradient.fmo_gradient(s, params, ofmo.FMOOptions(level=2))
    assert np.max(np.abs(g_fmo - gradient.scc_gradient(s.Z, s.xyz, params))) < FD_TOL


def test_fmo2_gradient_of_two_fragments_equals_whole_system_gradient(params, water_dimer):
    # FMO2 of two fragments with an SCC dimer is the whole-system energy
    g_fmo = gradient.fmo_gradient(water_dimer, params, ofmo.FMOOptions(level=2, all_dimers_scc=True))
    g_all = gradient.scc_gradient(water_dimer.Z, water_dimer.xyz, params)
    assert np.max(np.abs(g_fmo - g_all)) < FD_TOL


def test_fmo2_gradient_of_three_fragments_has_no_net_force(params, water64):
    s = water64.subsystem([0, 1, 2])
    g = gradient.fmo_gradient(s, params, ofmo.FMOOptions(level=2, all_dimers_scc=True))
    assert np.abs(g).max() > 1e-3
    assert np.max(np.abs(g.sum(axis=0))) < 1e-8
