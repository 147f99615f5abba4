"""FP64 CPU oracle of the density-matrix purification variant of the SCC step.

TEST INFRASTRUCTURE ONLY (see oracle/xtb.py): nothing in the product path
imports it.

In every SCC iteration of GFN1-xTB the orthogonalised Fock matrix is
diagonalised and the density built from the occupied orbitals; this
diagonalisation is the step that makes the method cubic (Introduction;
Methodology, GFN1-xTB).  Purification computes the same occupied-subspace
projector from matrix products alone.  Its result has a plain definition,
which is what this oracle writes out:

  D = sum_{i < n_occ} c_i c_i^T,   F' c_i = e_i c_i,   e_0 <= e_1 <= ...

the orthogonal projector onto the n_occ lowest eigenvectors of the symmetric
matrix F' (zero electronic temperature; unique when e_{n_occ-1} < e_{n_occ}).
A closed-shell density is 2 D.
"""
from __future__ import annotations

import numpy as np


def occupied_projector(F: np.ndarray, n_occ: int) -> np.ndarray:
    """D for one symmetric n x n matrix F (FP64)."""
    F = np.asarray(F, dtype=np.float64)
    n = F.shape[0]
    if not 0 <= n_occ <= n:
        raise ValueError("n_occ outside 0..n")
    e, C = np.linalg.eigh(0.5 * (F + F.T))
    Co = C[:, :n_occ]
    return Co @ Co.T


def homo_lumo_gap(F: np.ndarray, n_occ: int) -> float:
    """e_{n_occ} - e_{n_occ-1} (inf when every or no orbital is occupied)."""
    e = np.linalg.eigvalsh(0.5 * (np.asarray(F, dtype=np.float64) + np.asarray(F).T))
    if n_occ == 0 or n_occ == len(e):
        return float("inf")
    return float(e[n_occ] - e[n_occ - 1])
