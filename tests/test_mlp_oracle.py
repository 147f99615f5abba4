"""Pins of the learned-guess oracle (oracle/mlp.py) against closed forms,
symmetry and finite differences."""
import numpy as np

from oracle import mlp
from paper_2606_28022_b300.inputs import geometry as G
from paper_2606_28022_b300.inputs.params import ANGSTROM


def _tiny():
    s = G.water_cluster(3, seed=5)
    return s


def test_radial_descriptor_of_a_pair_is_the_closed_form():
    r = 2.3
    X = mlp.geometric_features(np.array([8, 1]), np.array([[0, 0, 0], [r, 0, 0]]) * ANGSTROM)
    fc = 0.5 * (np.cos(np.pi * r / mlp.RC) + 1)
    want = np.exp(-mlp.ETA_R * (r - mlp.RS) ** 2) * fc
    assert np.allclose(X[0, 0:8], want, rtol=1e-12, atol=0)       # O sees one H
    assert np.allclose(X[1, 3 * 8:4 * 8], want, rtol=1e-12, atol=0)   # H sees one O
    assert X[0, 8:32].max() == 0.0


def test_angular_descriptor_of_three_atoms_is_the_closed_form():
    r1, r2, th = 1.0, 1.5, np.radians(104.5)
    xyz = np.array([[0, 0, 0], [r1, 0, 0], [r2 * np.cos(th), r2 * np.sin(th), 0]]) * ANGSTROM
    X = mlp.geometric_features(np.array([8, 1, 1]), xyz)
    fc = lambda r: 0.5 * (np.cos(np.pi * r / mlp.RC) + 1)
    w = np.exp(-mlp.ETA_A * (r1 ** 2 + r2 ** 2)) * fc(r1) * fc(r2)
    p = mlp.PAIRS.index((0, 0))                                        # H-H neighbour pair
    for t, (lam, zeta) in enumerate(mlp.ANG_TERMS):
        want = 2 ** (1 - zeta) * (1 + lam * np.cos(th)) ** zeta * w
        assert abs(X[0, 32 + 4 * p + t] - want) < 1e-13


def test_descriptors_are_rotation_and_translation_invariant():
    s = _tiny()
    X = mlp.geometric_features(s.Z, s.xyz)
    a, b, c = 0.3, -1.1, 2.0
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    Y = mlp.geometric_features(s.Z, s.xyz @ (Rz @ Rx).T + c)
    assert np.max(np.abs(X - Y)) < 1e-12


def test_projection_makes_every_fragment_neutral():
    s = _tiny()
    y = np.random.default_rng(1).normal(size=(s.n_atoms, 2))
    q = mlp.project(y, s.frag, np.array([0, 1, -1]))
    for f, c in enumerate([0, 1, -1]):
        assert abs(q[np.repeat(s.frag, 2) == f].sum() + c) < 1e-12


def test_backward_matches_finite_differences(params):
    s = _tiny()
    X = mlp.features(s, params)
    p = mlp.init_params(3)
    p["mean"], p["scale"] = X.mean(0), 1.0 / (X.std(0) + 1.0)
    target = np.random.default_rng(2).normal(size=2 * s.n_atoms) * 0.1
    L, g = mlp.loss_and_grad(p, X, s.frag, s.frag_charge, target)
    rng = np.random.default_rng(4)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(3):
            idx = tuple(rng.integers(0, n) for n in p[k].shape)
            h = 1e-6
            pp, pm = {**p, k: p[k].copy()}, {**p, k: p[k].copy()}
            pp[k][idx] += h
            pm[k][idx] -= h
            fd = (mlp.loss_and_grad(pp, X, s.frag, s.frag_charge, target)[0]
                  - mlp.loss_and_grad(pm, X, s.frag, s.frag_charge, target)[0]) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1e-3, abs(fd))


def test_first_adam_step_moves_by_the_learning_rate():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    mlp.adam_step(p, g, {}, lr=0.01, t=1)
    # bias-corrected first step: -lr g / (|g| + eps)
    assert np.allclose(p["w"], np.array([1.0, -2.0, 0.5]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), atol=1e-15)


def test_esp_feature_is_the_gamma_sum_over_other_fragments(params):
    from oracle import xtb
    s = G.water_cluster(2, seed=3)
    dq = np.random.default_rng(0).normal(size=2 * s.n_atoms) * 0.1
    e = mlp.esp_feature(s, params, dq)
    b = xtb.make_basis(s.Z, params)
    eta = xtb.shell_hardness(s.Z, b, params)
    a, first = 0, 0                                    # atom 0, its first shell
    want = 0.0
    for sh in range(b.n_sh):
        if s.frag[b.sh_atom[sh]] != s.frag[a]:
            r = np.linalg.norm(s.xyz[a] - s.xyz[b.sh_atom[sh]])
            want += dq[sh] / np.sqrt(r ** 2 + (0.5 * (1 / eta[first] + 1 / eta[sh])) ** 2)
    assert abs(e[a] - want) < 1e-12
