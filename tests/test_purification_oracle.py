"""Pins of the occupied-subspace projector oracle against closed forms and
invariants: diagonal matrices, the 2 x 2 rotation, idempotency, trace,
commutation with F, invariance under a shift and positive scaling of F, and
the complement identity D(F, n_occ) + D(-F, n - n_occ) = I."""
import numpy as np
import pytest

from oracle import purification as pu


def _gapped(n, n_occ, seed, gap=0.2):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    e = np.sort(rng.uniform(-1.0, 1.0, n))
    e[n_occ:] += gap
    return (Q * e) @ Q.T


def test_diagonal_matrix_gives_indicator_of_lowest_entries():
    d = np.array([0.3, -1.0, 2.0, -0.5, 0.1])
    D = pu.occupied_projector(np.diag(d), 2)
    assert np.allclose(D, np.diag([0, 1, 0, 1, 0]), atol=1e-15)


def test_two_by_two_closed_form():
    # F = [[a, b], [b, c]]: lower eigenvector (cos t, sin t) with
    # tan(2t) = 2b / (a - c) and the branch giving the smaller eigenvalue
    a, b, c = 0.4, -0.3, 1.1
    t = 0.5 * np.arctan2(2 * b, a - c) + np.pi / 2
    v = np.array([np.cos(t), np.sin(t)])
    lam = v @ np.array([[a, b], [b, c]]) @ v
    assert lam < 0.5 * (a + c)
    D = pu.occupied_projector(np.array([[a, b], [b, c]]), 1)
    assert np.allclose(D, np.outer(v, v), atol=1e-14)


@pytest.mark.parametrize("n,n_occ", [(7, 3), (40, 17), (33, 0), (33, 33)])
def test_projector_invariants(n, n_occ):
    F = _gapped(n, n_occ, seed=n + n_occ)
    D = pu.occupied_projector(F, n_occ)
    assert np.allclose(D @ D, D, atol=1e-12)
    assert abs(np.trace(D) - n_occ) < 1e-12
    assert np.allclose(F @ D, D @ F, atol=1e-12)
    assert np.allclose(pu.occupied_projector(2.5 * F - 0.7 * np.eye(n), n_occ), D, atol=1e-12)
    assert np.allclose(D + pu.occupied_projector(-F, n - n_occ), np.eye(n), atol=1e-12)
    # the occupied energy is the sum of the n_occ lowest eigenvalues
    assert abs(np.trace(D @ F) - np.sort(np.linalg.eigvalsh(F))[:n_occ].sum()) < 1e-12


def test_gap_and_arguments():
    F = np.diag([0.0, 1.0, 3.0])
    assert pu.homo_lumo_gap(F, 2) == 2.0
    assert pu.homo_lumo_gap(F, 0) == float("inf")
    with pytest.raises(ValueError):
        pu.occupied_projector(F, 4)
