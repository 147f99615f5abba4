"""FP64 CPU oracle of the analytic FMO1 gradient: explicit terms plus the
self-consistent Z-vector (SCZV) response of the monomer charges (Sec. 2.4,
explicit gradient and response gradient).

TEST INFRASTRUCTURE ONLY (see oracle/xtb.py).

E_FMO1 = sum_I E'_I, each monomer I converged in the potential esp_I =
sum_{K != I} Gamma_IK dq_K of the others' shell charges (Eq. 21).  With
L_I = E'_I + esp_I . dq_I, which the monomer density makes stationary,
  dE/dxi = sum_I dL_I/dxi|_(esp_I fixed) - sum_I esp_I . d dq_I/dxi.
The first sum is the single-system gradient of each monomer with the ESP
inside its shell shifts and orbital energies, and the supersystem CN chain
rule (oracle/gradient.explicit_gradient).  The charges obey
dq_I = Q_I(xi, esp_I), so d dq/dxi = (1 - chi Gamma)^-1 (dQ/dxi|_esp +
chi dGamma dq) with chi the block-diagonal monomer susceptibilities
(oracle/response.py).  The Z-vector z = (1 - Gamma chi)^-1 esp (chi and
Gamma symmetric) turns the response into
  - sum_I z_I . dQ_I/dxi|_esp - (chi z)^T dGamma dq.
z_I . dQ_I/dxi at fixed esp is the derivative of monomer I's explicit
gradient along the potential z_I (Q_I = dL_I/d esp_I): the explicit terms
contracted with the first-order changes of P, W~, the shifts and the charges
that the potential z_I causes (coupled-perturbed SCC, as in
oracle/response.py; W~ = sum f_i e_i c_i c_i^T changes by
C [N o (C^T dF C)] C^T with N_ij = (f_i e_i - f_j e_j)/(e_i - e_j), minus
the Fermi-level shift).  Systems without cut bonds.  Central differences of
the oracle's FMO1 energy pin it (tests/test_fmo_gradient_oracle.py).
"""
from __future__ import annotations

import numpy as np

from . import fmo as ofmo
from . import gradient, response, xtb


def _first_order(prob, res, dv):
    """Changes of dq, shifts, P and W~ of a converged SCC system under the
    shell potential dv (coupled-perturbed SCC)."""
    b = prob.basis
    sh = b.ao_shell
    chi = response.susceptibility(prob, res)
    dq = chi @ dv
    dsig = dv + response.charge_kernel(prob, res) @ dq
    dF = 0.5 * prob.S * (dsig[sh][:, None] + dsig[sh][None, :])
    C, eps, f = res.C, res.eps, res.occ
    fp = -2.0 * (f / 2.0) * (1.0 - f / 2.0) / prob.kT
    de = eps[:, None] - eps[None, :]
    fe = f * eps
    with np.errstate(divide="ignore", invalid="ignore"):
        M = np.where(np.abs(de) > 1e-12, (f[:, None] - f[None, :]) / de, 0.5 * (fp[:, None] + fp[None, :]))
        dfe = fp * eps + f
        N = np.where(np.abs(de) > 1e-12, (fe[:, None] - fe[None, :]) / de, 0.5 * (dfe[:, None] + dfe[None, :]))
    dFm = C.T @ dF @ C
    X = M * dFm
    Y = N * dFm
    sfp = fp.sum()
    if abs(sfp) > 0.0:
        def_ = float(fp @ np.diag(dFm)) / sfp
        X = X - np.diag(fp * def_)
        Y = Y - np.diag(fp * eps * def_)
    return dq, dsig, C @ X @ C.T, C @ Y @ C.T


def fmo1_gradient(system, params, tol=1e-12) -> np.ndarray:
    """dE_FMO1/dxyz (n_atoms x 3, Eh/bohr), analytic (explicit + SCZV)."""
    Z = np.asarray(system.Z)
    xyz = np.asarray(system.xyz, dtype=np.float64)
    if len(system.cut_bonds):
        raise ValueError("cut bonds are not covered")
    nf = system.n_frag
    n_all = len(Z)
    atoms = [np.nonzero(system.frag == f)[0] for f in range(nf)]
    cn_all = xtb.coordination_numbers(Z, xyz, params)
    dcn_all = gradient.cn_derivative(Z, xyz, params)
    r = ofmo.fmo(system, params, ofmo.FMOOptions(level=1, scc_tol=tol, e_tol=0.1 * tol, outer_tol=tol))
    q = [np.asarray(d, dtype=np.float64) for d in r.dq_mono]
    bases = [xtb.make_basis(Z[a], params) for a in atoms]
    pos = [xyz[a][b.sh_atom] for a, b in zip(atoms, bases)]
    eta = [xtb.shell_hardness(Z[a], b, params) for a, b in zip(atoms, bases)]
    gam = [[xtb.gamma_between(pos[I], eta[I], pos[K], eta[K], params.k_g) for K in range(nf)] for I in range(nf)]
    esp = [sum(gam[I][K] @ q[K] for K in range(nf) if K != I) if nf > 1 else np.zeros(len(q[I]))
           for I in range(nf)]

    # monomers at the converged potential
    probs, ress = [], []
    for I in range(nf):
        prob = xtb.SCCProblem(Z[atoms[I]], xyz[atoms[I]], params, cn_all[atoms[I]], esp=esp[I],
                              charge=float(system.frag_charge[I]))
        res = xtb.solve_problem(prob, guess=q[I], tol=tol, e_tol=0.1 * tol)
        probs.append(prob)
        ress.append(res)
        q[I] = res.dq

    def explicit(I, P, Wt, sig, Q, with_rep=True, M_extra=None):
        return gradient.explicit_gradient(Z[atoms[I]], xyz[atoms[I]], params, bases[I], P, Wt, sig, Q,
                                          cn_all[atoms[I]], dcn_all[atoms[I]], atoms=atoms[I], n_all=n_all,
                                          with_rep=with_rep, M_extra=M_extra)

    grad = np.zeros((n_all, 3))
    sig = []
    for I in range(nf):
        prob, res = probs[I], ress[I]
        b = bases[I]
        dq_at = np.bincount(b.sh_atom, weights=res.dq, minlength=len(atoms[I]))
        sig.append(prob.gam @ res.dq - prob.g3[b.sh_atom] * dq_at[b.sh_atom] ** 2 + esp[I])
        Wt = (res.C * (res.occ * res.eps)) @ res.C.T
        grad += explicit(I, res.P, Wt, sig[I], np.outer(res.dq, res.dq))
    if nf == 1:
        return grad

    # Z-vector in charge space: z = esp + Gamma chi z
    off = np.cumsum([0] + [len(x) for x in q])
    n_sh = off[-1]
    G = np.zeros((n_sh, n_sh))
    chi = np.zeros((n_sh, n_sh))
    for I in range(nf):
        chi[off[I]:off[I + 1], off[I]:off[I + 1]] = response.susceptibility(probs[I], ress[I])
        for K in range(nf):
            if K != I:
                G[off[I]:off[I + 1], off[K]:off[K + 1]] = gam[I][K]
    e = np.concatenate(esp)
    z = np.linalg.solve(np.eye(n_sh) - G @ chi, e)
    y = chi @ z

    # - sum_I z_I . dQ_I/dxi|_esp
    for I in range(nf):
        prob, res = probs[I], ress[I]
        zI = z[off[I]:off[I + 1]]
        dq1, dsig, dP, dWt = _first_order(prob, res, zI)
        sh = bases[I].ao_shell
        M_extra = 0.5 * (dsig[sh][:, None] + dsig[sh][None, :]) * res.P
        Q = np.outer(res.dq, dq1) + np.outer(dq1, res.dq)
        grad -= explicit(I, dP, dWt, sig[I], Q, with_rep=False, M_extra=M_extra)

    # - (chi z)^T dGamma dq over the shell pairs of different fragments
    sh_atom = [atoms[I][bases[I].sh_atom] for I in range(nf)]
    for I in range(nf):
        for K in range(nf):
            if K == I:
                continue
            yI = y[off[I]:off[I + 1]]
            for s in range(len(yI)):
                for t in range(len(q[K])):
                    a, c = sh_atom[I][s], sh_atom[K][t]
                    rv = xyz[a] - xyz[c]
                    rr = float(np.linalg.norm(rv))
                    ee = 2.0 / (1.0 / eta[I][s] + 1.0 / eta[K][t])
                    gm = (rr ** params.k_g + ee ** (-params.k_g)) ** (-1.0 / params.k_g)
                    dg = -rr ** (params.k_g - 1.0) * gm ** (1.0 + params.k_g)
                    v = yI[s] * q[K][t] * dg * rv / rr
                    grad[a] -= v
                    grad[c] += v
    return grad
