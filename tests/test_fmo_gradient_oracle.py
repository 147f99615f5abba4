"""Pins of the oracle's analytic FMO1 gradient (explicit terms plus the
self-consistent Z-vector response, oracle/fmo_gradient.py): central
differences of the oracle's FMO1 energy, the one-fragment identity, and a
planted mistake (no response) that the finite differences catch."""
import dataclasses

import numpy as np
import pytest

from oracle import fmo as ofmo
from oracle import fmo_gradient, gradient
from paper_2606_28022_b300.inputs import geometry as G

FD_TOL = 2e-8   # Eh/bohr


@pytest.fixture(scope="module")
def water3(water64):
    return water64.subsystem([0, 1, 2])


@pytest.fixture(scope="module")
def water3_fd(params, water3):
    return gradient.fmo_gradient(water3, params, ofmo.FMOOptions(level=1))


def test_fmo1_gradient_equals_finite_differences(params, water3, water3_fd):
    g = fmo_gradient.fmo1_gradient(water3, params)
    assert np.abs(water3_fd).max() > 1e-3
    assert np.max(np.abs(g - water3_fd)) < FD_TOL
    assert np.max(np.abs(g.sum(axis=0))) < 1e-12


def test_fmo1_gradient_without_response_misses(params, water3, water3_fd, monkeypatch):
    # planted mistake: monomer susceptibilities set to zero (no SCZV response)
    real = fmo_gradient.response.susceptibility
    monkeypatch.setattr(fmo_gradient.response, "susceptibility", lambda prob, res: 0.0 * real(prob, res))
    g = fmo_gradient.fmo1_gradient(water3, params)
    assert np.max(np.abs(g - water3_fd)) > 1e-4


def test_fmo1_gradient_one_fragment_is_scc_gradient(params, water64):
    s = water64.subsystem([4])
    g = fmo_gradient.fmo1_gradient(s, params)
    assert np.max(np.abs(g - gradient.scc_gradient(s.Z, s.xyz, params))) < 1e-9


def test_fmo1_gradient_anthracene_pair_sampled(params):
    a, _ = G.anthracene_cluster(8, 2)
    a = a.subsystem([0, 1])
    g = fmo_gradient.fmo1_gradient(a, params)
    opts = ofmo.FMOOptions(level=1, scc_tol=1e-12, e_tol=1e-13, outer_tol=1e-12)
    energy = lambda x: ofmo.fmo(dataclasses.replace(a, xyz=x), params, opts).e_fmo1
    for k in (0, 17, 30):
        for c in range(3):
            xp = a.xyz.copy(); xp[k, c] += 1e-4
            xm = a.xyz.copy(); xm[k, c] -= 1e-4
            assert abs((energy(xp) - energy(xm)) / 2e-4 - g[k, c]) < FD_TOL


@pytest.mark.parametrize("frags,all_scc", [([0, 1, 2], True), ([0, 1, 2, 3], False)])
def test_fmo2_gradient_equals_finite_differences(params, water64, frags, all_scc):
    # all SCC dimers, and a mix of SCC dimers and ES-DIM pairs (4.0 A rule)
    s = water64.subsystem(frags)
    opts = ofmo.FMOOptions(level=2, all_dimers_scc=all_scc)
    r = ofmo.fmo(s, params, opts)
    assert r.dimer_scc.all() if all_scc else (r.dimer_scc.any() and not r.dimer_scc.all())
    g = fmo_gradient.fmo2_gradient(s, params, opts)
    fd = gradient.fmo_gradient(s, params, opts)
    assert np.max(np.abs(g - fd)) < FD_TOL


def test_fmo3_gradient_of_three_fragments_is_the_whole_system_gradient(params, water3):
    # FMO3 with all dimers and the trimer SCC reproduces the whole system
    opts = ofmo.FMOOptions(level=3, all_dimers_scc=True, trimer_cut=1e9)
    g = fmo_gradient.fmo3_gradient(water3, params, opts)
    assert np.max(np.abs(g - gradient.scc_gradient(water3.Z, water3.xyz, params))) < 1e-10


def test_fmo3_gradient_equals_finite_differences(params, water64):
    s = water64.subsystem([0, 1, 2, 3])
    opts = ofmo.FMOOptions(level=3, all_dimers_scc=True, trimer_cut=1e9)
    assert len(ofmo.fmo(s, params, opts).trimers) == 4
    g = fmo_gradient.fmo3_gradient(s, params, opts)
    assert np.max(np.abs(g - gradient.fmo_gradient(s, params, opts))) < FD_TOL


def test_fmo2_gradient_of_six_waters_rmsd(params, water64):
    # the accuracy bar for the analytic gradient: RMSD against central
    # differences well below 1e-7 Eh/bohr on a (H2O)_6 cluster (4.0 A rule)
    s = water64.subsystem(range(6))
    opts = ofmo.FMOOptions(level=2)
    g = fmo_gradient.fmo2_gradient(s, params, opts)
    fd = gradient.fmo_gradient(s, params, opts)
    assert np.sqrt(np.mean((g - fd) ** 2)) < 1e-8


def test_fmo1_gradient_with_cut_bonds_equals_finite_differences(params, water3):
    # hybrid orbital projection: E'_I leaves Tr(P V^HOP) out, which the
    # monomer density does not make stationary (its own response enters)
    s = G.polyalanine_helix(2)
    assert len(s.cut_bonds) == 1
    g = fmo_gradient.fmo1_gradient_hop(s, params)
    opts = ofmo.FMOOptions(level=1, scc_tol=1e-12, e_tol=1e-13, outer_tol=1e-12)
    energy = lambda x: ofmo.fmo(dataclasses.replace(s, xyz=x), params, opts).e_fmo1
    bda, baa = (int(a) for a in s.cut_bonds[0])
    for k in (bda, baa, 7):
        for c in range(3):
            xp = s.xyz.copy(); xp[k, c] += 1e-4
            xm = s.xyz.copy(); xm[k, c] -= 1e-4
            # the 1e6 Eh projector leaves ~1e-8 of noise in these differences
            assert abs((energy(xp) - energy(xm)) / 2e-4 - g[k, c]) < 2e-7
    assert np.max(np.abs(g.sum(axis=0))) < 1e-12
    # without cut bonds the general form reduces to fmo1_gradient
    assert np.max(np.abs(fmo_gradient.fmo1_gradient_hop(water3, params)
                         - fmo_gradient.fmo1_gradient(water3, params))) < 1e-12


def test_gradient_with_healed_bonds_equals_whole_molecule(params):
    # FMO2 of two and FMO3 of three bonded fragments heal every cut bond and
    # reproduce the whole molecule exactly, so their gradients must too
    a2 = G.polyalanine_helix(2)
    g2 = fmo_gradient.fmo_gradient_records(a2, params, ofmo.FMOOptions(level=2, all_dimers_scc=True))
    assert np.max(np.abs(g2 - gradient.scc_gradient(a2.Z, a2.xyz, params))) < 1e-10
    a3 = G.polyalanine_helix(3)
    g3 = fmo_gradient.fmo_gradient_records(a3, params,
                                           ofmo.FMOOptions(level=3, all_dimers_scc=True, trimer_cut=1e9))
    assert np.max(np.abs(g3 - gradient.scc_gradient(a3.Z, a3.xyz, params))) < 1e-10


def test_fmo2_gradient_with_cut_bonds_equals_finite_differences(params, water64):
    # Ala3: each bonded dimer heals one bond and keeps the other detached
    s = G.polyalanine_helix(3)
    opts = ofmo.FMOOptions(level=2, all_dimers_scc=True)
    g = fmo_gradient.fmo_gradient_records(s, params, opts)
    assert np.abs(g - gradient.scc_gradient(s.Z, s.xyz, params)).max() > 1e-4      # not the whole molecule
    o = dataclasses.replace(opts, scc_tol=1e-12, e_tol=1e-13, outer_tol=1e-12)
    energy = lambda x: ofmo.fmo(dataclasses.replace(s, xyz=x), params, o).e_fmo2
    k = int(s.cut_bonds[0][0])
    for c in range(3):
        xp = s.xyz.copy(); xp[k, c] += 1e-4
        xm = s.xyz.copy(); xm[k, c] -= 1e-4
        assert abs((energy(xp) - energy(xm)) / 2e-4 - g[k, c]) < 2e-7
    # without cut bonds the record form is the plain FMO2 gradient
    w4 = water64.subsystem([0, 1, 2, 3])
    o2 = ofmo.FMOOptions(level=2)
    assert np.max(np.abs(fmo_gradient.fmo_gradient_records(w4, params, o2)
                         - fmo_gradient.fmo2_gradient(w4, params, o2))) < 1e-12
