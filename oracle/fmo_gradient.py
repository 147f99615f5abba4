"""FP64 CPU oracle of the analytic FMO1, FMO2 and FMO3 gradients: explicit terms
plus the self-consistent Z-vector (SCZV) response of the monomer charges
(Sec. 2.4, explicit gradient and response gradient).

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
the Fermi-level shift).  FMO2 (fmo2_gradient) adds the SCC dimers and the
ES-DIM pairs in the same form, FMO3 (fmo3_gradient) the trimer corrections;
these take systems without cut bonds.  fmo1_gradient_hop covers FMO1 with cut
bonds (hybrid orbital projection, HOP section): ghost records, the projector
term Tr(P dV/dxi), and the derivative of the Tr(P V^HOP) that E'_I leaves
out.  fmo_gradient_records is the general form (FMO1/2/3, cut bonds healed
in the n-mers that hold both of their fragments).  Central differences of the oracle's FMO1, FMO2 and FMO3 energies pin
them, and so does the exact identity of FMO3 of three fragments with the
whole system (tests/test_fmo_gradient_oracle.py).
"""
from __future__ import annotations

import numpy as np

from . import fmo as ofmo
from . import gradient, response, xtb


def _first_order(prob, res, dv):
    """Changes of dq, shifts, P and W~ of a converged SCC system under the
    shell potential dv (coupled-perturbed SCC; _first_order_general)."""
    return _first_order_general(prob, res, dv=dv)


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


def _gamma_pair_grad(xyz, at_a, eta_a, ca, at_b, eta_b, cb, k_g, n_all):
    """Gradient of sum_{s in a, t in b} ca_s cb_t gamma_st over shell sets a
    and b (different atoms)."""
    g = np.zeros((n_all, 3))
    rv = xyz[at_a][:, None, :] - xyz[at_b][None, :, :]
    rr = np.linalg.norm(rv, axis=-1)
    ee = 2.0 / (1.0 / eta_a[:, None] + 1.0 / eta_b[None, :])
    gm = (rr ** k_g + ee ** (-k_g)) ** (-1.0 / k_g)
    dg = -rr ** (k_g - 1.0) * gm ** (1.0 + k_g)
    with np.errstate(divide="ignore", invalid="ignore"):
        # a ghost and its own bond-detachment atom share one position and
        # move together: their distance has no gradient
        v = np.where((rr > 0.0)[..., None], (ca[:, None] * cb[None, :] * dg / rr)[..., None] * rv, 0.0)
    np.add.at(g, at_a, v.sum(axis=1))
    np.add.at(g, at_b, -v.sum(axis=0))
    return g


def fmo2_gradient(system, params, opts=None, tol=1e-12) -> np.ndarray:
    """dE_FMO2/dxyz (n_atoms x 3, Eh/bohr), analytic: explicit terms of the
    monomers, SCC dimers (Eq. 12 with dE^V of Eqs. 13-14) and ES-DIM pairs
    (Eq. 15), plus the SCZV response of the monomer charges.  With
    L_X = E'_X + esp_X . dq_X stationary in each n-mer density,
      E_FMO2 = sum_I c_I E'_I + sum_SCC [L_IJ - esp_IJ . (dq_I + dq_J)]
               + sum_ES dq_I Gamma_IJ dq_J,
    c_I = 1 - (SCC dimers of I); every term linear in the monomer-charge
    derivatives collects into w, and z = (1 - Gamma chi)^-1 w gives the
    response z . dQ/dxi|_esp + (chi z)^T dGamma dq."""
    opts = ofmo.FMOOptions(level=2) if opts is None else opts
    return _nmer_gradient(system, params, opts, 2, tol)


def fmo3_gradient(system, params, opts=None, tol=1e-12) -> np.ndarray:
    """dE_FMO3/dxyz: as fmo2_gradient with the trimer corrections of
    Eqs. 16-19, corr_IJK = dE_IJK - dE_IJ - dE_IK - dE_JK.  Each trimer adds
    L_IJK - esp_IJK . (dq_I + dq_J + dq_K) with coefficient 1, takes one from
    the coefficient of each of its pair terms, and changes c_I by
    -1 + (its SCC pairs holding I)."""
    opts = ofmo.FMOOptions(level=3) if opts is None else opts
    return _nmer_gradient(system, params, opts, 3, tol)


def _nmer_gradient(system, params, opts, level, tol):
    import dataclasses
    Z = np.asarray(system.Z)
    xyz = np.asarray(system.xyz, dtype=np.float64)
    if len(system.cut_bonds):
        raise ValueError("cut bonds are not covered")
    o = dataclasses.replace(opts, level=level, scc_tol=tol, e_tol=0.1 * tol, outer_tol=tol)
    r = ofmo.fmo(system, params, o)
    nf = system.n_frag
    n_all = len(Z)
    kg = params.k_g
    atoms = [np.nonzero(system.frag == f)[0] for f in range(nf)]
    cn_all = xtb.coordination_numbers(Z, xyz, params)
    dcn_all = gradient.cn_derivative(Z, xyz, params)
    bases = [xtb.make_basis(Z[a], params) for a in atoms]
    sh_at = [atoms[I][bases[I].sh_atom] for I in range(nf)]           # supersystem atom of each shell
    eta = [xtb.shell_hardness(Z[a], b, params) for a, b in zip(atoms, bases)]
    gam = [[xtb.gamma_between(xyz[sh_at[I]], eta[I], xyz[sh_at[K]], eta[K], kg) for K in range(nf)]
           for I in range(nf)]
    q = [np.asarray(d, dtype=np.float64) for d in r.dq_mono]

    def esp_of(nmer):
        return [sum((gam[I][K] @ q[K] for K in range(nf) if K not in nmer), np.zeros(len(q[I]))) for I in nmer]

    def solve(nmer):
        at = np.concatenate([atoms[I] for I in nmer])
        esp = np.concatenate(esp_of(nmer))
        prob = xtb.SCCProblem(Z[at], xyz[at], params, cn_all[at], esp=esp,
                              charge=float(sum(system.frag_charge[I] for I in nmer)))
        res = xtb.solve_problem(prob, guess=np.concatenate([q[I] for I in nmer]), tol=tol, e_tol=0.1 * tol)
        return at, esp, prob, res

    def explicit(at, b, prob, res, esp):
        dq_at = np.bincount(b.sh_atom, weights=res.dq, minlength=len(at))
        sig = prob.gam @ res.dq - prob.g3[b.sh_atom] * dq_at[b.sh_atom] ** 2 + esp
        Wt = (res.C * (res.occ * res.eps)) @ res.C.T
        return gradient.explicit_gradient(Z[at], xyz[at], params, b, res.P, Wt, sig, np.outer(res.dq, res.dq),
                                          cn_all[at], dcn_all[at], atoms=at, n_all=n_all), sig

    pairs = [tuple(int(x) for x in pq) for pq in r.dimers]
    scc = [bool(x) for x in r.dimer_scc]
    tris = [tuple(int(x) for x in t) for t in r.trimers] if level >= 3 else []
    pair_k = {pq: k for k, pq in enumerate(pairs)}
    m_pair = np.ones(len(pairs))                  # coefficient of each pair term
    c_mono = np.ones(nf)                          # coefficient of each E'_I
    for (I, J), ok in zip(pairs, scc):
        if ok:
            c_mono[I] -= 1.0
            c_mono[J] -= 1.0
    for t in tris:
        for pq in ((t[0], t[1]), (t[0], t[2]), (t[1], t[2])):
            k = pair_k[pq]
            m_pair[k] -= 1.0
            if scc[k]:                            # -dE_IJ gives +E'_I, +E'_J back
                c_mono[pq[0]] += 1.0
                c_mono[pq[1]] += 1.0
        for I in t:
            c_mono[I] -= 1.0
    off = np.cumsum([0] + [len(x) for x in q])
    w = np.zeros(off[-1])
    grad = np.zeros((n_all, 3))

    # monomers: c_I (dL_I/dxi|_esp - esp_I . dq_I')
    mono = []
    for I in range(nf):
        at, esp, prob, res = solve((I,))
        q[I] = res.dq
        mono.append((prob, res))
    for I in range(nf):
        prob, res = mono[I]
        esp = esp_of((I,))[0]
        gI, sigI = explicit(atoms[I], bases[I], prob, res, esp)
        mono[I] = (prob, res, sigI)
        c = c_mono[I]
        grad += c * gI
        w[off[I]:off[I + 1]] -= c * esp
    # n-mer terms m_X [L_X - esp_X . (sum of its monomer charges)] for SCC
    # dimers and trimers; ES-DIM pairs m_IJ dq_I Gamma_IJ dq_J
    nmers = [(pq, m_pair[k]) for k, (pq, ok) in enumerate(zip(pairs, scc)) if ok] + [(t, 1.0) for t in tris]
    for k, ((I, J), ok) in enumerate(zip(pairs, scc)):
        m = m_pair[k]
        if ok or m == 0.0:
            continue
        grad += m * _gamma_pair_grad(xyz, sh_at[I], eta[I], q[I], sh_at[J], eta[J], q[J], kg, n_all)
        w[off[I]:off[I + 1]] += m * (gam[I][J] @ q[J])
        w[off[J]:off[J + 1]] += m * (gam[J][I] @ q[I])
    for X, m in nmers:
        if m == 0.0:
            continue
        at, esp, prob, res = solve(X)
        b = xtb.make_basis(Z[at], params)
        gX, _ = explicit(at, b, prob, res, esp)
        grad += m * gX
        ddq = res.dq - np.concatenate([q[I] for I in X])
        o0 = np.cumsum([0] + [len(q[I]) for I in X])
        for a, I in enumerate(X):
            w[off[I]:off[I + 1]] -= m * esp[o0[a]:o0[a + 1]]
        for K in range(nf):
            if K in X:
                continue
            # ddq . dGamma_{X,K} dq_K (explicit) and ddq . Gamma_{X,K} dq_K' (into w)
            for a, I in enumerate(X):
                dd = ddq[o0[a]:o0[a + 1]]
                grad += m * _gamma_pair_grad(xyz, sh_at[I], eta[I], dd, sh_at[K], eta[K], q[K], kg, n_all)
                w[off[K]:off[K + 1]] += m * (gam[K][I] @ dd)

    # response: z = (1 - Gamma chi)^-1 w; z . dQ/dxi|_esp + (chi z)^T dGamma dq
    n_sh = off[-1]
    G = np.zeros((n_sh, n_sh))
    chi = np.zeros((n_sh, n_sh))
    for I in range(nf):
        chi[off[I]:off[I + 1], off[I]:off[I + 1]] = response.susceptibility(mono[I][0], mono[I][1])
        for K in range(nf):
            if K != I:
                G[off[I]:off[I + 1], off[K]:off[K + 1]] = gam[I][K]
    z = np.linalg.solve(np.eye(n_sh) - G @ chi, w)
    y = chi @ z
    for I in range(nf):
        prob, res, sigI = mono[I]
        dq1, dsig, dP, dWt = _first_order(prob, res, z[off[I]:off[I + 1]])
        sh = bases[I].ao_shell
        M_extra = 0.5 * (dsig[sh][:, None] + dsig[sh][None, :]) * res.P
        Q = np.outer(res.dq, dq1) + np.outer(dq1, res.dq)
        grad += gradient.explicit_gradient(Z[atoms[I]], xyz[atoms[I]], params, bases[I], dP, dWt, sigI, Q,
                                           cn_all[atoms[I]], dcn_all[atoms[I]], atoms=atoms[I], n_all=n_all,
                                           with_rep=False, M_extra=M_extra)
        for K in range(nf):
            if K != I:
                grad += _gamma_pair_grad(xyz, sh_at[I], eta[I], y[off[I]:off[I + 1]], sh_at[K], eta[K], q[K],
                                         kg, n_all)
    return grad


def _first_order_general(prob, res, dv=None, dF_ext=None):
    """First-order changes of dq, the shell shifts, P and W~ of a converged
    SCC system (coupled-perturbed SCC) under a shell potential dv and/or an
    AO-matrix perturbation dF_ext of the Fock matrix (kept out of the
    shifts): dP = C [M o dF'] C^T and dW~ = C [N o dF'] C^T in the MO basis
    (M, N as in the module notes, minus the Fermi-level shift), with the
    charges self-consistent through dq = (1 - chi0 K)^-1 (bare source)."""
    b = prob.basis
    sh = b.ao_shell
    C, eps, f = res.C, res.eps, res.occ
    fp = -2.0 * (f / 2.0) * (1.0 - f / 2.0) / prob.kT
    de = eps[:, None] - eps[None, :]
    fe = f * eps
    with np.errstate(divide="ignore", invalid="ignore"):
        M = np.where(np.abs(de) > 1e-12, (f[:, None] - f[None, :]) / de, 0.5 * (fp[:, None] + fp[None, :]))
        dfe = fp * eps + f
        N = np.where(np.abs(de) > 1e-12, (fe[:, None] - fe[None, :]) / de, 0.5 * (dfe[:, None] + dfe[None, :]))
    sfp = fp.sum()

    def orbital(dF):
        dFm = C.T @ dF @ C
        X = M * dFm
        Y = N * dFm
        if abs(sfp) > 0.0:
            def_ = float(fp @ np.diag(dFm)) / sfp
            X = X - np.diag(fp * def_)
            Y = Y - np.diag(fp * eps * def_)
        return C @ X @ C.T, C @ Y @ C.T

    chi0 = response.bare_response(prob, res)
    K = response.charge_kernel(prob, res)
    n_sh = b.n_sh
    src = np.zeros(n_sh)
    if dv is not None:
        src = src + chi0 @ dv
    if dF_ext is not None:
        dP0, _ = orbital(dF_ext)
        src = src + np.bincount(sh, weights=(dP0 * prob.S).sum(axis=1), minlength=n_sh)
    dq = np.linalg.solve(np.eye(n_sh) - chi0 @ K, src)
    dsig = K @ dq + (dv if dv is not None else 0.0)
    dF = 0.5 * prob.S * (dsig[sh][:, None] + dsig[sh][None, :])
    if dF_ext is not None:
        dF = dF + dF_ext
    dP, dWt = orbital(dF)
    return dq, dsig, dP, dWt


def _records(fr, nmer):
    """Records of an n-mer (supersystem atom, cut bond or -1), its repulsion
    mask and its projected records for explicit_gradient (as ofmo._Frags.problem)."""
    s = fr.system
    recs = [r for k, f in enumerate(nmer) for r, keep in zip(fr.recs[f], fr.present(nmer)[k]) if keep]
    at = np.array([a for a, _ in recs], dtype=np.int64)
    rep_mask = np.array([bond < 0 for _, bond in recs])
    hop = []
    for i, (a, bond) in enumerate(recs):
        ks = [(bond, "ghost")] if bond >= 0 else \
             [(k, "bda") for k in range(len(fr.cut)) if fr.cut[k, 0] == a and fr.bond_frag[k][1] not in nmer]
        for k, kind in ks:
            bda, baa = int(fr.cut[k, 0]), int(fr.cut[k, 1])
            v = s.xyz[baa] - s.xyz[bda]
            n = float(np.linalg.norm(v))
            hop.append((i, kind, bda, baa, v / n, n))
    return at, rep_mask, hop


def fmo1_gradient_hop(system, params, tol=1e-12) -> np.ndarray:
    """dE_FMO1/dxyz with cut bonds (hybrid orbital projection): as
    fmo1_gradient, with E'_I = L_I - esp_I . dq_I - Tr(P_I V_I^HOP).  The last
    term is not stationary in the monomer density: its derivative is that of
    the explicit gradient along the Fock perturbation V^HOP (the projector
    scaled by 1 + lambda), plus its charge response times d esp_I/dxi.  The
    FMO1 case of fmo_gradient_records."""
    return fmo_gradient_records(system, params, ofmo.FMOOptions(level=1), tol)


def fmo_gradient_records(system, params, opts=None, tol=1e-12) -> np.ndarray:
    """dE_FMO/dxyz at opts.level (1, 2 or 3) for systems with or without cut
    bonds, in one form: every monomer I (coefficient c_I) and every SCC dimer
    and trimer X (coefficient m_X) contributes
        L_X - Tr(P_X V_X^HOP) - esp_X . (monomer charges of X's fragments),
    with L_X = E'_X + esp_X . dq_X + Tr(P_X V_X) stationary in the n-mer
    density, esp_X on every monomer shell of X's fragments (a healed ghost
    keeps its monomer charge there, its n-mer charge is zero: the -dq_mono
    charge transfer of dE^V), and ES-DIM pairs m_IJ dq_I Gamma_IJ dq_J.  The
    coefficients count the FMO2/FMO3 subtractions (fmo3_gradient)."""
    import dataclasses
    opts = ofmo.FMOOptions() if opts is None else opts
    level = opts.level
    Z = np.asarray(system.Z)
    xyz = np.asarray(system.xyz, dtype=np.float64)
    nf = system.n_frag
    n_all = len(Z)
    kg = params.k_g
    fr = ofmo._Frags(system, params)
    dcn_all = gradient.cn_derivative(Z, xyz, params)
    r = ofmo.fmo(system, params, dataclasses.replace(opts, scc_tol=tol, e_tol=0.1 * tol, outer_tol=tol))
    q = [np.asarray(d, dtype=np.float64) for d in r.dq_mono]
    at_f = [np.array([a for a, _ in fr.recs[f]], dtype=np.int64) for f in range(nf)]
    sh_at = [at_f[f][fr.sh_rec[f]] for f in range(nf)]               # global atom of each monomer shell
    off = np.cumsum([0] + [fr.n_sh[f] for f in range(nf)])
    w = np.zeros(off[-1])
    grad = np.zeros((n_all, 3))

    # coefficients (as fmo2/fmo3_gradient)
    pairs = [tuple(int(x) for x in pq) for pq in r.dimers] if level >= 2 else []
    scc = [bool(x) for x in r.dimer_scc] if level >= 2 else []
    tris = [tuple(int(x) for x in t) for t in r.trimers] if level >= 3 else []
    pair_k = {pq: k for k, pq in enumerate(pairs)}
    m_pair = np.ones(len(pairs))
    c_mono = np.ones(nf)
    for (I, J), ok in zip(pairs, scc):
        if ok:
            c_mono[I] -= 1.0
            c_mono[J] -= 1.0
    for t in tris:
        for pq in ((t[0], t[1]), (t[0], t[2]), (t[1], t[2])):
            k = pair_k[pq]
            m_pair[k] -= 1.0
            if scc[k]:
                c_mono[pq[0]] += 1.0
                c_mono[pq[1]] += 1.0
        for I in t:
            c_mono[I] -= 1.0
    terms = [((I,), c_mono[I]) for I in range(nf)]
    terms += [(pq, m_pair[k]) for k, (pq, ok) in enumerate(zip(pairs, scc)) if ok]
    terms += [(t, 1.0) for t in tris]

    mono = {}
    for X, m in terms:
        at, rep_mask, hop = _records(fr, X)
        esp = fr.esp(X, q)                                    # on the n-mer's shells
        esp_full = fr.esp_full(X, q)                          # on every monomer shell of X
        mask = fr.shell_mask(X)
        qmono = np.concatenate([q[f] for f in X])
        prob = fr.problem(X, esp)
        res = xtb.solve_problem(prob, guess=qmono[mask], tol=tol, e_tol=0.1 * tol)
        b = prob.basis
        dq_at = np.bincount(b.sh_atom, weights=res.dq, minlength=len(at))
        sig = prob.gam @ res.dq - prob.g3[b.sh_atom] * dq_at[b.sh_atom] ** 2 + esp
        if len(X) == 1:
            mono[X[0]] = (prob, res, at, rep_mask, hop, sig)
        if m == 0.0:
            continue

        def explicit(P, Wt, Q, with_rep=True, M_extra=None):
            return gradient.explicit_gradient(Z[at], xyz[at], params, b, P, Wt, sig, Q, fr.cn[at], dcn_all[at],
                                              atoms=at, n_all=n_all, with_rep=with_rep, M_extra=M_extra,
                                              rep_mask=rep_mask, hop=hop)

        Wt = (res.C * (res.occ * res.eps)) @ res.C.T
        grad += m * explicit(res.P, Wt, np.outer(res.dq, res.dq))
        coef = -qmono.copy()                                   # - esp_full . q_mono
        qx = np.zeros_like(qmono)
        qx[mask] = res.dq
        coef += qx                                             # + esp . dq_X (from dL/d esp)
        if prob.extra_fock is not None:
            dqv, dsig, dP, dWt = _first_order_general(prob, res, dF_ext=prob.extra_fock)
            sh = b.ao_shell
            M_extra = 0.5 * (dsig[sh][:, None] + dsig[sh][None, :]) * res.P
            Q = np.outer(res.dq, dqv) + np.outer(dqv, res.dq)
            grad -= m * explicit(dP, dWt, Q, with_rep=False, M_extra=M_extra)
            grad -= m * gradient._hop_gradient(Z[at], xyz[at], params, b, prob.S,
                                               gradient.overlap_derivative(Z[at], xyz[at], params, b), res.P,
                                               hop, at, n_all)
            dv_full = np.zeros_like(qmono)
            dv_full[mask] = dqv
            coef -= dv_full                                    # - dq^V . d esp/dxi
        o0 = np.cumsum([0] + [fr.n_sh[f] for f in X])
        for a, I in enumerate(X):
            w[off[I]:off[I + 1]] -= m * esp_full[o0[a]:o0[a + 1]]
        for K in range(nf):
            if K in X:
                continue
            for a, I in enumerate(X):
                cI = coef[o0[a]:o0[a + 1]]
                grad += m * _gamma_pair_grad(xyz, sh_at[I], fr.sh_eta[I], cI, sh_at[K], fr.sh_eta[K], q[K], kg,
                                             n_all)
                w[off[K]:off[K + 1]] += m * (fr.gamma(K, I) @ cI)
    for k, ((I, J), ok) in enumerate(zip(pairs, scc)):
        mm = m_pair[k]
        if ok or mm == 0.0:
            continue
        grad += mm * _gamma_pair_grad(xyz, sh_at[I], fr.sh_eta[I], q[I], sh_at[J], fr.sh_eta[J], q[J], kg, n_all)
        w[off[I]:off[I + 1]] += mm * (fr.gamma(I, J) @ q[J])
        w[off[J]:off[J + 1]] += mm * (fr.gamma(J, I) @ q[I])
    if nf == 1:
        return grad

    # response: z = (1 - Gamma chi)^-1 w
    n_sh = off[-1]
    G = np.zeros((n_sh, n_sh))
    chi = np.zeros((n_sh, n_sh))
    for I in range(nf):
        chi[off[I]:off[I + 1], off[I]:off[I + 1]] = response.susceptibility(mono[I][0], mono[I][1])
        for K in range(nf):
            if K != I:
                G[off[I]:off[I + 1], off[K]:off[K + 1]] = fr.gamma(I, K)
    z = np.linalg.solve(np.eye(n_sh) - G @ chi, w)
    y = chi @ z
    for I in range(nf):
        prob, res, at, rep_mask, hop, sig = mono[I]
        b = prob.basis
        dq1, dsig, dP, dWt = _first_order_general(prob, res, dv=z[off[I]:off[I + 1]])
        sh = b.ao_shell
        M_extra = 0.5 * (dsig[sh][:, None] + dsig[sh][None, :]) * res.P
        Q = np.outer(res.dq, dq1) + np.outer(dq1, res.dq)
        grad += gradient.explicit_gradient(Z[at], xyz[at], params, b, dP, dWt, sig, Q, fr.cn[at], dcn_all[at],
                                           atoms=at, n_all=n_all, with_rep=False, M_extra=M_extra,
                                           rep_mask=rep_mask, hop=hop)
        for K in range(nf):
            if K != I:
                grad += _gamma_pair_grad(xyz, sh_at[I], fr.sh_eta[I], y[off[I]:off[I + 1]], sh_at[K],
                                         fr.sh_eta[K], q[K], kg, n_all)
    return grad
