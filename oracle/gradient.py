"""FP64 CPU oracle of the GFN1-xTB nuclear gradient of one SCC system.

TEST INFRASTRUCTURE ONLY (see oracle/xtb.py): the slow, plain reference for
the analytic-gradient rows.  It differentiates the energy that oracle/xtb.py
computes, term by term, at the converged density (Sec. 2.4, GFN1-xTB energy
gradient):
  Eq. 23  the single-system gradient: P dH0 + W dS + 1/2 dq dq dgamma
          + dE_rep
  Eq. 24  W with the energy-weighted density, the shell shifts and the
          third-order term
  Eq. 25  dH0 = H dS + S dH: the S part joins the W term; the rest is the
          derivative of the distance polynomial Pi (Eq. 9) and of the
          CN-dependent levels (Eq. 10)
  Eqs. 26-28  coordination number, its gradient F_A dCN_A, and F_A, the
          sensitivity of the energy to CN_A
(equation numbers as in oracle/fmo.py: the halogen-bond expression is not
counted)
Because the Fermi-smeared SCC energy E - TS is stationary in the orbitals and
occupations at convergence, these explicit terms are the whole gradient of a
system in no external potential; finite differences of xtb.single_point pin
it (tests/test_gradient_oracle.py).  The derivative of the overlap of two
contracted s/p Gaussians is the derivative of the closed form that
xtb.overlap_matrix evaluates: with R = A - B, mu = ab/p, s00 = (pi/p)^1.5
exp(-mu R^2), PA = -(b/p) R and PB = (a/p) R.

READING C-19: the CN counting function is cut at cn_cutoff (READING C-3), so
the gradient is that of the cut sum (no pair within the cut contributes a
derivative at the cut itself).

fmo_gradient is the FMO gradient by its definition: central differences of
the oracle's FMO1/2/3 energy (oracle/fmo.py) in every coordinate.  It is the
reference the analytic FMO gradient (explicit terms plus the self-consistent
Z-vector response of Sec. 2.4) has to reach; slow (6 N_atoms FMO runs), for
small systems.  Two exact identities pin it to the analytic single-system
gradient: one fragment (E_FMO = E), and FMO2 of two fragments with an SCC
dimer (E_FMO2 = E of the whole system).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fmo as ofmo
from . import xtb


def overlap_derivative(Z, xyz, params, basis: xtb.Basis | None = None) -> np.ndarray:
    """dS[k, c] = dS / d xyz[k, c] (n_atoms x 3 x n_ao x n_ao)."""
    if basis is None:
        basis = xtb.make_basis(Z, params)
    n_at = len(Z)
    n = basis.n_ao
    dS = np.zeros((n_at, 3, n, n))
    # primitive expansion, as in xtb.overlap_matrix
    prims = []
    for mu in range(n):
        s = basis.ao_shell[mu]
        el = params.elements[int(Z[basis.sh_atom[s]])]
        k = basis.sh_index[s]
        a = np.asarray(el.alpha[k], dtype=np.float64)
        c = np.asarray(el.coef[k], dtype=np.float64)
        norm = (2.0 * a / np.pi) ** 0.75
        if basis.sh_l[s] == 1:
            norm = norm * 2.0 * np.sqrt(a)
        prims.append((a, c * norm))
    eye = np.eye(3)
    for mu in range(n):
        A_at = basis.ao_atom[mu]
        lu = basis.sh_l[basis.ao_shell[mu]]
        u = basis.ao_comp[mu]
        a, ca = prims[mu]
        for nu in range(n):
            B_at = basis.ao_atom[nu]
            if A_at == B_at:
                continue                       # one-centre overlaps do not move
            lv = basis.sh_l[basis.ao_shell[nu]]
            v = basis.ao_comp[nu]
            b, cb = prims[nu]
            R = xyz[A_at] - xyz[B_at]
            R2 = float(R @ R)
            aa = a[:, None]
            bb = b[None, :]
            p = aa + bb
            m = aa * bb / p
            s00 = (np.pi / p) ** 1.5 * np.exp(-m * R2) * (ca[:, None] * cb[None, :])
            g = np.zeros(3)
            for x in range(3):
                if lu == 0 and lv == 0:
                    val = -2.0 * m * R[x] * s00
                elif lu == 1 and lv == 0:
                    val = -(bb / p) * s00 * (eye[u, x] - 2.0 * m * R[u] * R[x])
                elif lu == 0 and lv == 1:
                    val = (aa / p) * s00 * (eye[v, x] - 2.0 * m * R[v] * R[x])
                else:
                    q = aa * bb / (p * p)
                    val = s00 * (-q * (eye[u, x] * R[v] + R[u] * eye[v, x])
                                 - 2.0 * m * R[x] * (-q * R[u] * R[v] + eye[u, v] / (2.0 * p)))
                g[x] = float(np.sum(val))
            dS[A_at, :, mu, nu] += g          # d/dA = d/dR
            dS[B_at, :, mu, nu] -= g          # d/dB = -d/dR
    return dS


def cn_derivative(Z, xyz, params) -> np.ndarray:
    """dCN[A, k, c] = d CN_A / d xyz[k, c] of xtb.coordination_numbers."""
    rcov = xtb.atom_param(Z, params, "r_cov")
    n = len(Z)
    d = np.zeros((n, n, 3))
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            rv = xyz[a] - xyz[b]
            r = float(np.linalg.norm(rv))
            if r >= params.cn_cutoff:
                continue
            rc = rcov[a] + rcov[b]
            f = 1.0 / (1.0 + np.exp(-params.cn_k1 * (params.cn_k2 * rc / r - 1.0)))
            df = -f * (1.0 - f) * params.cn_k1 * params.cn_k2 * rc / (r * r)
            d[a, a] += df * rv / r
            d[a, b] -= df * rv / r
    return d


def explicit_gradient(Z, xyz, params, basis, P, Wt, sigma, Q, cn, dcn, atoms=None, n_all=None,
                      with_rep=True, M_extra=None, rep_mask=None, hop=None) -> np.ndarray:
    """The explicit terms of Eqs. 23-28 for one system at fixed P, W~, shell
    shifts sigma and charge product Q (n_sh x n_sh, Q = dq dq^T for the
    energy): sum dS (P H + 1/2 (sigma_mu + sigma_nu) P - W~ [+ M_extra])
    + the Pi and CN parts of dH0 + 1/2 sum Q dgamma [+ dE_rep].
    cn: the CN of the system's atoms (in FMO: supersystem values); dcn
    [a, k, c]: their derivatives with respect to every atom k of the
    supersystem (n_all atoms); atoms: the system's atoms in the supersystem
    (default: all; a ghost record of the hybrid orbital projection maps to
    its bond-detachment atom).  rep_mask: records in the repulsion (default
    all); hop: the projected records, [(record, kind "bda"|"ghost", BDA atom,
    BAA atom, unit vector BDA -> BAA, bond length)], whose projector V = sum S[:,A] D_A S[A,:] is in the Fock
    matrix: adds Tr(P dV/dxi).  Returns n_all x 3."""
    Z = np.asarray(Z)
    xyz = np.asarray(xyz, dtype=np.float64)
    b = basis
    n_at = len(Z)
    atoms = np.arange(n_at) if atoms is None else np.asarray(atoms)
    n_all = n_at if n_all is None else n_all
    sh = b.ao_shell
    at = b.ao_atom
    S = xtb.overlap_matrix(Z, xyz, params, b)
    sig_ao = np.asarray(sigma)[sh]
    # pieces of H0 (Eq. 8) per AO pair
    h_l = xtb.shell_param(Z, b, params, "h_l")
    k_cn = xtb.shell_param(Z, b, params, "k_cn_l")
    k_poly = xtb.shell_param(Z, b, params, "k_poly_l")
    h_sh = h_l * (1.0 + k_cn * cn[b.sh_atom])
    en = xtb.atom_param(Z, params, "en")
    rcov = xtb.atom_param(Z, params, "r_cov")
    k_l = np.asarray(params.k_l)[b.sh_l]
    A = at[:, None]
    B = at[None, :]
    off = A != B
    Rv = xyz[A] - xyz[B]
    R = np.linalg.norm(Rv, axis=-1)
    Rcov = rcov[A] + rcov[B]
    x = np.sqrt(np.where(off, R / Rcov, 0.0))
    kp_u = k_poly[sh][:, None]
    kp_v = k_poly[sh][None, :]
    Pi = (1.0 + kp_u * x) * (1.0 + kp_v * x)
    kab = np.vectorize(params.k_ab)(Z[A], Z[B])
    fen = 1.0 + params.k_en * (en[A] - en[B]) ** 2
    kll = 0.5 * (k_l[sh][:, None] + k_l[sh][None, :])
    hbar = 0.5 * (h_sh[sh][:, None] + h_sh[sh][None, :])
    Hpref = np.where(off, kab * kll * hbar * fen * Pi, 0.0)           # H0 = Hpref S off the atom blocks

    grad = np.zeros((n_at, 3))
    # (1) every S-dependence: P Hpref + 1/2 (sigma_mu + sigma_nu) P - W~ (Eqs. 23-25)
    dS = overlap_derivative(Z, xyz, params, b)
    Mw = P * Hpref + 0.5 * (sig_ao[:, None] + sig_ao[None, :]) * P - Wt
    if M_extra is not None:
        Mw = Mw + M_extra
    Mw = np.where(off, Mw, 0.0)
    grad += np.einsum("kcij,ij->kc", dS, Mw)
    # (2) the distance polynomial Pi(R_AB) (Eq. 9)
    with np.errstate(divide="ignore", invalid="ignore"):
        dPi_dx = kp_u * (1.0 + kp_v * x) + kp_v * (1.0 + kp_u * x)
        dx_dR = np.where(off, x / (2.0 * R), 0.0)
        dE_dR = np.where(off, P * S * kab * kll * hbar * fen * dPi_dx * dx_dR, 0.0)
        unit = np.where(off[..., None], Rv / R[..., None], 0.0)
    pair = dE_dR[..., None] * unit                                      # d/dxyz[A(mu)]
    for k in range(n_at):
        grad[k] += pair[at == k].sum(axis=(0, 1))
        grad[k] -= pair[:, at == k].sum(axis=(0, 1))
    # (4) the Coulomb kernel: 1/2 sum Q_st dgamma_st (Eq. 23)
    eta = xtb.shell_hardness(Z, b, params)
    sa = b.sh_atom
    for s_ in range(b.n_sh):
        for t in range(b.n_sh):
            if sa[s_] == sa[t] or Q[s_, t] == 0.0:
                continue
            rv = xyz[sa[s_]] - xyz[sa[t]]
            r = float(np.linalg.norm(rv))
            e = 2.0 / (1.0 / eta[s_] + 1.0 / eta[t])
            gm = (r ** params.k_g + e ** (-params.k_g)) ** (-1.0 / params.k_g)
            dg = -r ** (params.k_g - 1.0) * gm ** (1.0 + params.k_g)
            v = 0.5 * Q[s_, t] * dg * rv / r
            grad[sa[s_]] += v
            grad[sa[t]] -= v
    # (5) repulsion (Eq. 11)
    if with_rep:
        zeff = xtb.atom_param(Z, params, "z_eff")
        arep = xtb.atom_param(Z, params, "alpha_rep")
        rm = np.ones(n_at, dtype=bool) if rep_mask is None else np.asarray(rep_mask, dtype=bool)
        for a in range(n_at):
            for c in range(a):
                if not (rm[a] and rm[c]):
                    continue
                rv = xyz[a] - xyz[c]
                r = float(np.linalg.norm(rv))
                al = np.sqrt(arep[a] * arep[c])
                ex = np.exp(-al * r ** params.k_f)
                de = zeff[a] * zeff[c] * ex * (-1.0 / r ** 2 - al * params.k_f * r ** (params.k_f - 2.0))
                grad[a] += de * rv / r
                grad[c] -= de * rv / r
    out = np.zeros((n_all, 3))
    np.add.at(out, atoms, grad)
    if hop:
        out += _hop_gradient(Z, xyz, params, b, S, dS, P, hop, atoms, n_all)
    # (3) CN-dependent levels (Eqs. 10, 26-28): F_A = dE/dCN_A, then the chain
    # rule over every atom the CN depends on
    dh_ao = (h_l * k_cn)[sh]                                            # dh_l / dCN of the shell's atom
    F = np.zeros(n_at)
    np.add.at(F, at, np.diag(P) * dh_ao)
    Hcn = np.where(off, P * S * kab * kll * fen * Pi * 0.5, 0.0)       # d(hbar)/dh_mu = 1/2
    np.add.at(F, at, (Hcn * dh_ao[:, None]).sum(axis=1))
    np.add.at(F, at, (Hcn * dh_ao[None, :]).sum(axis=0))
    out += np.einsum("a,akc->kc", F, dcn)
    return out


def _hop_gradient(Z, xyz, params, b, S, dS, P, hop, atoms, n_all):
    """Tr(P dV/dxi) of the hybrid-orbital projector V = sum_A S[:,A] D_A S[A,:]
    with D = V_hop h h^T (detached BDA) or V_hop (1 - h h^T) (ghost), h =
    (c_s, c_p b) on the record's s and p functions, b the unit vector from
    the BDA to the BAA (HOP section)."""
    from .fmo import C_P, C_S
    out = np.zeros((n_all, 3))
    X = np.zeros_like(P)
    for rec, kind, bda, baa, bvec, blen in hop:
        sh = np.nonzero(b.sh_atom == rec)[0]
        s_sh = sh[b.sh_l[sh] == 0][0]
        p_sh = sh[b.sh_l[sh] == 1][0]
        idx = np.concatenate([[b.sh_ao0[s_sh]], b.sh_ao0[p_sh] + np.arange(3)])
        h = np.concatenate([[C_S], C_P * bvec])
        sign = 1.0 if kind == "bda" else -1.0
        D = params.v_hop * (np.outer(h, h) if kind == "bda" else np.eye(4) - np.outer(h, h))
        # dS part: 2 sum_{mu, a in A} dS_mu,a (P S[:,A] D)_mu,a
        X[:, idx] += 2.0 * (P @ S[:, idx] @ D)
        # dD part: <S[A,:] P S[:,A], dD>, dD = sign V_hop (dh h^T + h dh^T),
        # dh = c_p (0, db), db = J dx_BAA - J dx_BDA, J = (1 - b b^T) / |b|
        G = S[idx, :] @ P @ S[:, idx]
        gh = (G @ h)[1:]
        J = (np.eye(3) - np.outer(bvec, bvec)) / blen
        v = sign * params.v_hop * 2.0 * C_P * (J @ gh)
        out[baa] += v
        out[bda] -= v
    g = np.einsum("kcij,ij->kc", dS, X)
    np.add.at(out, atoms, g)
    return out


def scc_gradient(Z, xyz, params, res: xtb.SCCResult | None = None, tol=1e-12) -> np.ndarray:
    """Analytic gradient (n_atoms x 3, Eh/bohr) of the GFN1-xTB energy of one
    neutral system without external potential, at its SCC solution."""
    Z = np.asarray(Z)
    xyz = np.asarray(xyz, dtype=np.float64)
    cn = xtb.coordination_numbers(Z, xyz, params)
    if res is None:
        res = xtb.scc(Z, xyz, params, cn, tol=tol, e_tol=tol)
    b = res.basis
    Wt = (res.C * (res.occ * res.eps)) @ res.C.T                  # energy-weighted density (Eq. 24)
    gam = xtb.gamma_matrix(Z, xyz, params, b)
    g3 = xtb.atom_param(Z, params, "gamma3")
    dq = res.dq
    dq_at = np.bincount(b.sh_atom, weights=dq, minlength=len(Z))
    sigma = gam @ dq - g3[b.sh_atom] * dq_at[b.sh_atom] ** 2         # shell shifts
    return explicit_gradient(Z, xyz, params, b, res.P, Wt, sigma, np.outer(dq, dq), cn,
                             cn_derivative(Z, xyz, params))


def fmo_gradient(system, params, opts=None, h=1e-4) -> np.ndarray:
    """dE_FMO/dxyz (n_atoms x 3) by central differences of the oracle's FMO
    energy at the level opts.level, converged to 1e-12."""
    opts = ofmo.FMOOptions() if opts is None else opts
    opts = dataclasses.replace(opts, scc_tol=1e-12, e_tol=1e-13, outer_tol=1e-12)
    key = {1: "e_fmo1", 2: "e_fmo2", 3: "e_fmo3"}[opts.level]

    def energy(xyz):
        return getattr(ofmo.fmo(dataclasses.replace(system, xyz=xyz), params, opts), key)

    xyz0 = np.asarray(system.xyz, dtype=np.float64)
    g = np.zeros_like(xyz0)
    for k in range(len(xyz0)):
        for c in range(3):
            xp = xyz0.copy()
            xp[k, c] += h
            xm = xyz0.copy()
            xm[k, c] -= h
            g[k, c] = (energy(xp) - energy(xm)) / (2.0 * h)
    return g
