"""FP64 CPU oracle of the linear response of one converged SCC system to a
shell-resolved external potential: the coupled-perturbed SCC equations whose
transpose the self-consistent Z-vector (SCZV) equations of the response
gradient solve (Sec. 2.4, response gradient, Eqs. 39-47).

TEST INFRASTRUCTURE ONLY (see oracle/xtb.py).

A potential v on the shells (the form in which the ESP enters the Fock
matrix, Eq. 21: 1/2 S (v_mu + v_nu)) changes the converged shell charges by
dq = chi v.  At fixed shell shifts the orbital response is first-order
perturbation theory with Fermi occupations f_i = 2 / (1 + exp((e_i - e_F)/kT))
(Eq. 6):
  dP = C [M o (C^T dF C)] C^T,  M_ij = (f_i - f_j) / (e_i - e_j)  (e_i != e_j),
  M_ii (and degenerate pairs) = df/de = -(2/kT) (f/2)(1 - f/2),
plus the shift of e_F that keeps the electron count (sum_i df_i = 0); the
Mulliken charges of dP (Eq. 3) give the bare response chi0 v.  The shell
shifts of the SCC Fock matrix (Eq. 7) respond to the charges through
K = d sigma / d dq = gamma - 2 Gamma_A dq_A (third order, on the shells of
atom A), so dq = chi0 (v + K dq) and chi = (1 - chi0 K)^-1 chi0.

chi is symmetric: it is the second derivative of the SCC free energy plus
v . dq with respect to v.  Central differences of the SCC charges in the
potential pin it (tests/test_response_oracle.py).
"""
from __future__ import annotations

import numpy as np

from . import xtb


def bare_response(prob: xtb.SCCProblem, res: xtb.SCCResult) -> np.ndarray:
    """chi0 (n_sh x n_sh): charge response at fixed shell shifts."""
    b = prob.basis
    C, eps, f = res.C, res.eps, res.occ
    kT = prob.kT
    n = len(eps)
    fp = -2.0 * (f / 2.0) * (1.0 - f / 2.0) / kT                     # df/de
    de = eps[:, None] - eps[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        M = np.where(np.abs(de) > 1e-12, (f[:, None] - f[None, :]) / de, 0.5 * (fp[:, None] + fp[None, :]))
    S = prob.S
    sh = b.ao_shell
    chi0 = np.zeros((b.n_sh, b.n_sh))
    for s in range(b.n_sh):
        v = np.zeros(b.n_sh)
        v[s] = 1.0
        dF = 0.5 * S * (v[sh][:, None] + v[sh][None, :])
        dFm = C.T @ dF @ C
        X = M * dFm
        sfp = fp.sum()
        if abs(sfp) > 0.0:                       # Fermi level keeps the electron count
            def_ = float(fp @ np.diag(dFm)) / sfp
            X = X - np.diag(fp * def_)
        dP = C @ X @ C.T
        chi0[:, s] = np.bincount(sh, weights=(dP * S).sum(axis=1), minlength=b.n_sh)
    return chi0


def charge_kernel(prob: xtb.SCCProblem, res: xtb.SCCResult) -> np.ndarray:
    """K = d sigma / d dq of the SCC shell shifts (Eq. 7)."""
    b = prob.basis
    nat = len(prob.Z)
    dq_at = np.bincount(b.sh_atom, weights=res.dq, minlength=nat)
    same_atom = (b.sh_atom[:, None] == b.sh_atom[None, :]).astype(np.float64)
    return prob.gam - 2.0 * (prob.g3 * dq_at)[b.sh_atom][:, None] * same_atom


def susceptibility(prob: xtb.SCCProblem, res: xtb.SCCResult) -> np.ndarray:
    """chi = d dq / d v (n_sh x n_sh) of the converged SCC solution."""
    chi0 = bare_response(prob, res)
    K = charge_kernel(prob, res)
    return np.linalg.solve(np.eye(len(chi0)) - chi0 @ K, chi0)
