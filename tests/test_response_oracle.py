"""Pins of the oracle's coupled-perturbed SCC charge response
(oracle/response.py): central differences of the oracle's SCC charges under
a small shell potential, symmetry of the susceptibility, and conservation of
the electron count, for integer and for strongly smeared occupations."""
import dataclasses

import numpy as np
import pytest

from oracle import response, xtb
from paper_2606_28022_b300.inputs import geometry as G

H = 1e-3


def _chi_and_fd(Z, xyz, params, seed):
    cn = xtb.coordination_numbers(Z, xyz, params)
    prob = xtb.SCCProblem(Z, xyz, params, cn)
    res = xtb.solve_problem(prob, tol=1e-12, e_tol=1e-13)
    chi = response.susceptibility(prob, res)
    v = np.random.default_rng(seed).normal(size=prob.basis.n_sh) * 0.01

    def q(sign):
        p = xtb.SCCProblem(Z, xyz, params, cn, esp=sign * H * v)
        return xtb.solve_problem(p, guess=res.dq, tol=1e-13, e_tol=1e-14).dq

    return chi, v, (q(1.0) - q(-1.0)) / (2 * H), res


@pytest.mark.parametrize("name", ["water_dimer", "alanine"])
def test_susceptibility_equals_finite_differences(params, water64, name):
    s = water64.subsystem([3, 7]) if name == "water_dimer" else G.polyalanine_helix(1)
    chi, v, fd, _ = _chi_and_fd(s.Z, s.xyz, params, 1)
    assert np.abs(fd).max() > 1e-3
    assert np.max(np.abs(chi @ v - fd)) < 1e-9
    assert np.max(np.abs(chi - chi.T)) < 1e-12           # second derivative of a free energy
    assert np.max(np.abs(chi.sum(axis=0))) < 1e-12       # the electron count is fixed


def test_susceptibility_with_fractional_occupations(params):
    # a high electronic temperature: the occupation derivatives and the
    # Fermi-level shift of the response carry weight
    hot = dataclasses.replace(params, t_el=20000.0)
    s = G.polyalanine_helix(1)
    chi, v, fd, res = _chi_and_fd(s.Z, s.xyz, hot, 2)
    assert np.sum((res.occ > 1e-6) & (res.occ < 2.0 - 1e-6)) > 10
    assert np.max(np.abs(chi @ v - fd)) < 1e-8
    assert np.max(np.abs(chi.sum(axis=0))) < 1e-12
