"""FP64 CPU oracle of the GFN1-xTB self-consistent-charge (SCC) solve.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against; only the tests, the smoke check and the bench's
CPU-baseline leg may import it.  It shares no code with the CUDA path: it reads
the seeded inputs (geometry, parameter table) and nothing else.

Every function follows one passage of the paper (Einsele & Mitric, FMO-xTB):
  Eq. 2   electronic energy E_el
  Eq. 3   shell-resolved Mulliken charges
  Eqs. 4-5 Coulomb kernel gamma and effective hardness eta
  Eq. 6   Fermi-Dirac occupations
  Eq. 7   Fock matrix (second- and third-order shifts)
  Eqs. 8-10 zeroth-order Hamiltonian H0, polynomial factor Pi, CN-dependent
          levels
  Eq. 11  repulsion energy
  Eq. 26 (CN definition, gradient section) coordination number
  Eq. 21 (embedding potential V^I) the ESP term of the Fock matrix
Readings of passages the paper leaves open are marked READING and listed in
the design notes.  Units: bohr, Hartree; charges in electrons
(dq = population - reference occupation, READING C-6).
PARITY UNPINNED: the modifiers of H0 in Eqs. 8-10 (the polynomial factor Pi,
the electronegativity factor and the CN-dependent levels) have no independent
pin: the extended-Hueckel test switches them off and the in-shell
proportionality test cannot see them; the paper prints no parameter table or
worked value to check them against.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# --------------------------------------------------------------------------
# basis bookkeeping


@dataclasses.dataclass
class Basis:
    """Shells and atomic orbitals of a set of atoms, in input atom order."""
    sh_atom: np.ndarray      # (n_sh,) atom of each shell
    sh_l: np.ndarray         # (n_sh,) angular momentum
    sh_index: np.ndarray     # (n_sh,) index of the shell within its element
    sh_ao0: np.ndarray       # (n_sh,) first AO of the shell
    ao_shell: np.ndarray     # (n_ao,) shell of each AO
    ao_atom: np.ndarray      # (n_ao,) atom of each AO
    ao_comp: np.ndarray      # (n_ao,) 0 for s; 0,1,2 = x,y,z for p
    n_ao: int
    n_sh: int


def make_basis(Z, params) -> Basis:
    sh_atom, sh_l, sh_index, sh_ao0, ao_shell, ao_atom, ao_comp = [], [], [], [], [], [], []
    n_ao = 0
    for a, z in enumerate(Z):
        el = params.elements[int(z)]
        for k, l in enumerate(el.shells_l):
            s = len(sh_atom)
            sh_atom.append(a)
            sh_l.append(l)
            sh_index.append(k)
            sh_ao0.append(n_ao)
            for m in range(2 * l + 1):
                ao_shell.append(s)
                ao_atom.append(a)
                ao_comp.append(m)
            n_ao += 2 * l + 1
    as_i = lambda v: np.asarray(v, dtype=np.int64)
    return Basis(as_i(sh_atom), as_i(sh_l), as_i(sh_index), as_i(sh_ao0), as_i(ao_shell),
                 as_i(ao_atom), as_i(ao_comp), n_ao, len(sh_atom))


def shell_param(Z, basis, params, name):
    """Per-shell array of a per-element-shell parameter (e.g. 'h_l')."""
    return np.array([getattr(params.elements[int(Z[a])], name)[k]
                     for a, k in zip(basis.sh_atom, basis.sh_index)], dtype=np.float64)


def atom_param(Z, params, name):
    return np.array([getattr(params.elements[int(z)], name) for z in Z], dtype=np.float64)


# --------------------------------------------------------------------------
# overlap of contracted Gaussian s/p shells (the STO-nG basis of Sec. 2.1)


def overlap_matrix(Z, xyz, params, basis: Basis | None = None) -> np.ndarray:
    """S_mu,nu over contracted, normalised s and p Gaussians.

    Two primitives exp(-a|r-A|^2), exp(-b|r-B|^2) combine into one Gaussian
    of exponent p = a+b centred at P = (aA+bB)/p; with K = exp(-ab/p |A-B|^2)
    the s-s overlap is (pi/p)^(3/2) K.  A Cartesian factor (x-A_x) of a p
    function contributes (P_x - A_x), and a pair of factors contributes
    (P_x-A_x)(P_y-B_y) + delta_xy/(2p) (Gaussian moments about P).
    Primitive normalisation: s (2a/pi)^(3/4), p (2a/pi)^(3/4) 2 sqrt(a).
    """
    if basis is None:
        basis = make_basis(Z, params)
    # expand every AO into its primitives
    p_ao, p_alpha, p_c = [], [], []
    for mu in range(basis.n_ao):
        s = basis.ao_shell[mu]
        el = params.elements[int(Z[basis.sh_atom[s]])]
        k = basis.sh_index[s]
        a = np.asarray(el.alpha[k], dtype=np.float64)
        c = np.asarray(el.coef[k], dtype=np.float64)
        norm = (2.0 * a / np.pi) ** 0.75
        if basis.sh_l[s] == 1:
            norm = norm * 2.0 * np.sqrt(a)
        p_ao.append(np.full(len(a), mu))
        p_alpha.append(a)
        p_c.append(c * norm)
    p_ao = np.concatenate(p_ao)
    p_alpha = np.concatenate(p_alpha)
    p_c = np.concatenate(p_c)
    p_l = basis.sh_l[basis.ao_shell[p_ao]]
    p_comp = basis.ao_comp[p_ao]
    p_cen = xyz[basis.ao_atom[p_ao]]

    n = basis.n_ao
    S = np.zeros(n * n)
    npr = len(p_ao)
    chunk = max(1, 4_000_000 // npr)
    for i0 in range(0, npr, chunk):
        i = slice(i0, min(npr, i0 + chunk))
        a = p_alpha[i][:, None]
        b = p_alpha[None, :]
        p = a + b
        A = p_cen[i][:, None, :]
        B = p_cen[None, :, :]
        P = (a[..., None] * A + b[..., None] * B) / p[..., None]
        r2 = ((A - B) ** 2).sum(-1)
        s00 = (np.pi / p) ** 1.5 * np.exp(-a * b / p * r2)
        li = p_l[i][:, None]
        lj = p_l[None, :]
        ci = p_comp[i]
        cj = p_comp
        PA = np.take_along_axis(P - A, np.broadcast_to(ci[:, None, None], P.shape[:2] + (1,)), axis=2)[..., 0]
        PB = np.take_along_axis(P - B, np.broadcast_to(cj[None, :, None], P.shape[:2] + (1,)), axis=2)[..., 0]
        same = (ci[:, None] == cj[None, :]).astype(np.float64)
        fac = np.where((li == 0) & (lj == 0), 1.0,
              np.where((li == 1) & (lj == 0), PA,
              np.where((li == 0) & (lj == 1), PB,
                       PA * PB + same / (2.0 * p))))
        val = p_c[i][:, None] * p_c[None, :] * s00 * fac
        flat = (p_ao[i][:, None] * n + p_ao[None, :]).ravel()
        S += np.bincount(flat, weights=val.ravel(), minlength=n * n)
    return S.reshape(n, n)


# --------------------------------------------------------------------------
# coordination number (the CN definition of the gradient section)


def coordination_numbers(Z, xyz, params) -> np.ndarray:
    """CN_A = sum_{B != A} 1 / (1 + exp(-k1 (k2 (Rcov_A + Rcov_B)/R_AB - 1))).

    READING C-3: the counting function tends to 1/(1+e^k1), not 0, at large
    R, so pairs at R_AB >= cn_cutoff are not counted.
    """
    rcov = atom_param(Z, params, "r_cov")
    n = len(Z)
    cn = np.zeros(n)
    for a in range(n):
        d = np.linalg.norm(xyz - xyz[a], axis=1)
        mask = (d < params.cn_cutoff) & (np.arange(n) != a)
        r = d[mask]
        arg = -params.cn_k1 * (params.cn_k2 * (rcov[a] + rcov[mask]) / r - 1.0)
        cn[a] = np.sum(1.0 / (1.0 + np.exp(arg)))
    return cn


# --------------------------------------------------------------------------
# zeroth-order Hamiltonian (Eqs. 8-10)


def h0_matrix(Z, xyz, params, S, cn, basis: Basis) -> np.ndarray:
    """H0 of Eq. 8 with Pi of Eq. 9 and CN-dependent levels of Eq. 10.

    READING C-4: on-site blocks are diagonal, H0_mumu = h_A^l; same-atom
    off-diagonal elements are zero.
    """
    h_l = shell_param(Z, basis, params, "h_l")
    k_cn = shell_param(Z, basis, params, "k_cn_l")
    k_poly = shell_param(Z, basis, params, "k_poly_l")
    h_sh = h_l * (1.0 + k_cn * cn[basis.sh_atom])                      # Eq. 10
    en = atom_param(Z, params, "en")
    rcov = atom_param(Z, params, "r_cov")
    k_l = np.asarray(params.k_l)[basis.sh_l]

    sh = basis.ao_shell
    at = basis.ao_atom
    A = at[:, None]
    B = at[None, :]
    R = np.linalg.norm(xyz[A] - xyz[B], axis=-1)
    Rcov = rcov[A] + rcov[B]
    ratio = np.sqrt(np.where(A != B, R / Rcov, 0.0))
    Pi = (1.0 + k_poly[sh][:, None] * ratio) * (1.0 + k_poly[sh][None, :] * ratio)  # Eq. 9
    kab = np.vectorize(params.k_ab)(Z[A], Z[B])
    den = en[A] - en[B]
    H0 = (kab * 0.5 * (k_l[sh][:, None] + k_l[sh][None, :])
          * 0.5 * (h_sh[sh][:, None] + h_sh[sh][None, :]) * S
          * (1.0 + params.k_en * den * den) * Pi)                        # Eq. 8
    onsite = A == B
    H0[onsite] = 0.0
    H0[np.arange(basis.n_ao), np.arange(basis.n_ao)] = h_sh[sh]
    return H0


# --------------------------------------------------------------------------
# Coulomb kernel (Eqs. 4-5)


def shell_hardness(Z, basis, params) -> np.ndarray:
    """(1 + kappa_A^l) eta_A, the shell hardness entering Eq. 5."""
    kappa = shell_param(Z, basis, params, "kappa_l")
    eta = atom_param(Z, params, "eta")[basis.sh_atom]
    return (1.0 + kappa) * eta


def gamma_between(xyz_a, eta_a, xyz_b, eta_b, k_g) -> np.ndarray:
    """gamma_mu,nu = (R^kg + eta^-kg)^(-1/kg), eta = 2 / (1/eta_mu + 1/eta_nu)."""
    R = np.linalg.norm(xyz_a[:, None, :] - xyz_b[None, :, :], axis=-1)
    eta = 2.0 / (1.0 / eta_a[:, None] + 1.0 / eta_b[None, :])
    return (R ** k_g + eta ** (-k_g)) ** (-1.0 / k_g)


def gamma_matrix(Z, xyz, params, basis: Basis) -> np.ndarray:
    eta_sh = shell_hardness(Z, basis, params)
    pos = xyz[basis.sh_atom]
    return gamma_between(pos, eta_sh, pos, eta_sh, params.k_g)


# --------------------------------------------------------------------------
# repulsion (Eq. 11)


def repulsion_energy(Z, xyz, params) -> float:
    """E_rep = sum over unordered atom pairs (READING C-5)."""
    zeff = atom_param(Z, params, "z_eff")
    arep = atom_param(Z, params, "alpha_rep")
    e = 0.0
    for a in range(len(Z)):
        for b in range(a):
            r = np.linalg.norm(xyz[a] - xyz[b])
            e += zeff[a] * zeff[b] / r * np.exp(-np.sqrt(arep[a] * arep[b]) * r ** params.k_f)
    return e


# --------------------------------------------------------------------------
# Fermi smearing (Eq. 6) and electronic entropy


def fermi_occupations(eps, n_el, kT, tol=1e-13):
    """Closed-shell occupations n_i = 2 / (exp((e_i - e_F)/kT) + 1) with the
    Fermi level found by bisection so that sum n_i = n_el (READING C-7).
    Returns (n, e_F, -T S_el) with S_el = -2 k_B sum[f ln f + (1-f) ln(1-f)],
    f = n/2."""
    if kT <= 0.0:
        n = np.zeros_like(eps)
        nocc = int(round(n_el)) // 2
        n[:nocc] = 2.0
        return n, 0.5 * (eps[nocc - 1] + eps[min(nocc, len(eps) - 1)]), 0.0

    def occ(ef):
        x = np.clip((eps - ef) / kT, -700.0, 700.0)
        return 2.0 / (np.exp(x) + 1.0)

    lo, hi = eps.min() - 50.0 * kT - 1.0, eps.max() + 50.0 * kT + 1.0
    ef = 0.5 * (lo + hi)
    for _ in range(400):
        ef = 0.5 * (lo + hi)
        total = occ(ef).sum()
        if abs(total - n_el) < tol or hi - lo < 1e-15:
            break
        if total > n_el:
            hi = ef
        else:
            lo = ef
    n = occ(ef)
    f = n / 2.0
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = np.where(f > 1e-300, f * np.log(f), 0.0)
        t2 = np.where(1.0 - f > 1e-300, (1.0 - f) * np.log(1.0 - f), 0.0)
    minus_ts = 2.0 * kT * np.sum(t1 + t2)
    return n, ef, minus_ts


# --------------------------------------------------------------------------
# charge mixing: modified Broyden (Johnson, Phys. Rev. B 38, 12807 (1988))


class Broyden:
    """Modified Broyden mixing of the shell-charge vector (READING C-8).

    x_in(m+1) = x_in(m) + a F(m) - sum_n w_n g_n u(n) with F = x_out - x_in,
    dF(n), dx(n) the normalised differences of consecutive residuals and
    inputs, u(n) = a dF(n) + dx(n), beta = (w0^2 I + A)^-1 with
    A_kn = w_k w_n dF(k).dF(n), c_k = w_k dF(k).F(m), g_n = sum_k c_k beta_kn.
    """

    def __init__(self, alpha=0.4, history=8, w0=0.01):
        self.alpha, self.history, self.w0 = alpha, history, w0
        self.dF, self.u = [], []
        self.prev_x = self.prev_F = None

    def step(self, x_in, x_out):
        F = x_out - x_in
        if self.prev_x is not None:
            dF = F - self.prev_F
            norm = np.linalg.norm(dF)
            if norm > 0.0:
                dF = dF / norm
                dx = (x_in - self.prev_x) / norm
                self.dF.append(dF)
                self.u.append(self.alpha * dF + dx)
                if len(self.dF) > self.history:
                    self.dF.pop(0)
                    self.u.pop(0)
        self.prev_x, self.prev_F = x_in.copy(), F.copy()
        x_new = x_in + self.alpha * F
        if self.dF:
            dFm = np.array(self.dF)
            a = dFm @ dFm.T
            beta = np.linalg.inv(self.w0 ** 2 * np.eye(len(self.dF)) + a)
            c = dFm @ F
            g = c @ beta
            x_new = x_new - g @ np.array(self.u)
        return x_new


class LinearMixer:
    def __init__(self, alpha=0.4):
        self.alpha = alpha

    def step(self, x_in, x_out):
        return x_in + self.alpha * (x_out - x_in)


# --------------------------------------------------------------------------
# the SCC solve


@dataclasses.dataclass
class SCCResult:
    energy: float            # E' = E_el + E_rep (no embedding interaction)
    e_el: float
    e_rep: float
    e_band: float            # sum P H0
    e_coul2: float           # 1/2 dq gamma dq
    e_coul3: float           # -1/3 sum Gamma dq_A^3
    minus_ts: float
    dq: np.ndarray           # shell charges (electrons, population - q0)
    P: np.ndarray
    S: np.ndarray
    H0: np.ndarray
    C: np.ndarray
    eps: np.ndarray
    occ: np.ndarray
    iterations: int
    converged: bool
    basis: Basis


def n_electrons(Z, params, charge=0.0) -> float:
    return float(sum(params.elements[int(z)].n_valence for z in Z) - charge)


class SCCProblem:
    """The fixed matrices of one SCC solve (S, H0, gamma, X = S^-1/2, ...) and
    the map from input shell charges to the output density and energy: one
    iteration of the SCC loop (Eqs. 2, 3, 6, 7 and the ESP of Eq. 21)."""

    def __init__(self, Z, xyz, params, cn, esp=None, charge=0.0, extra_fock=None, n_el=None, q0=None,
                 rep_mask=None):
        self.Z, self.xyz, self.params = Z, xyz, params
        self.kT = 3.166811563e-6 * params.t_el
        self.basis = b = make_basis(Z, params)
        self.S = overlap_matrix(Z, xyz, params, b)
        self.H0 = h0_matrix(Z, xyz, params, self.S, cn, b)
        self.gam = gamma_matrix(Z, xyz, params, b)
        # q0: per-shell reference occupations (default: the element's); rep_mask:
        # atoms that take part in the repulsion (default: all) -- both differ
        # from the defaults only at HOP boundaries (oracle/fmo.py)
        self.q0 = shell_param(Z, b, params, "q0_l") if q0 is None else np.asarray(q0, dtype=np.float64)
        self.g3 = atom_param(Z, params, "gamma3")
        if rep_mask is None:
            self.e_rep = repulsion_energy(Z, xyz, params)
        else:
            m = np.asarray(rep_mask, dtype=bool)
            self.e_rep = repulsion_energy(np.asarray(Z)[m], np.asarray(xyz)[m], params)
        self.n_el = n_electrons(Z, params, charge) if n_el is None else n_el
        self.esp = np.zeros(b.n_sh) if esp is None else np.asarray(esp, dtype=np.float64)
        self.extra_fock = extra_fock
        s_val, s_vec = np.linalg.eigh(self.S)
        self.X = (s_vec / np.sqrt(s_val)) @ s_vec.T           # Loewdin orthogonaliser

    def step(self, dq, esp=None):
        """Fock matrix from the input charges dq (and the embedding potential,
        self.esp unless given), eigensolve, occupations, density, Mulliken
        charges and the energy of the output density."""
        import scipy.linalg as sla
        b = self.basis
        sh = b.ao_shell
        nat = len(self.Z)
        esp = self.esp if esp is None else esp
        dq_atom = np.bincount(b.sh_atom, weights=dq, minlength=nat)
        shift = self.gam @ dq - self.g3[b.sh_atom] * dq_atom[b.sh_atom] ** 2 + esp
        F = self.H0 + 0.5 * self.S * (shift[sh][:, None] + shift[sh][None, :])
        if self.extra_fock is not None:
            F = F + self.extra_fock
        eps, Cp = sla.eigh(self.X @ F @ self.X)
        C = self.X @ Cp
        occ, ef, mts = fermi_occupations(eps, self.n_el, self.kT)
        P = (C * occ) @ C.T
        pops = np.bincount(sh, weights=(P * self.S).sum(axis=1), minlength=b.n_sh)  # Eq. 3
        dq_out = pops - self.q0
        dq_out_atom = np.bincount(b.sh_atom, weights=dq_out, minlength=nat)
        e_band = float(np.sum(P * self.H0))
        e2 = 0.5 * float(dq_out @ self.gam @ dq_out)
        e3 = -float(np.sum(self.g3 * dq_out_atom ** 3)) / 3.0
        e_el = e_band + e2 + e3 + mts                                     # Eq. 2
        return dict(dq_out=dq_out, e_el=e_el, e_band=e_band, e2=e2, e3=e3, mts=mts, P=P, C=C,
                    eps=eps, occ=occ)


def scc(Z, xyz, params, cn, esp=None, guess=None, charge=0.0, tol=1e-10, e_tol=1e-10,
        max_iter=300, mixer=None, extra_fock=None, n_el=None) -> SCCResult:
    """One GFN1-xTB SCC solve of a set of atoms.

    cn          coordination numbers of these atoms (taken from the whole
                system in FMO: the CN sum runs over the supersystem)
    esp         per-shell external potential (ESP^I_mu) of Eq. 21; enters the
                Fock matrix as 1/2 S (esp_mu + esp_nu)
    extra_fock  an AO matrix added to F and kept out of the energy (the HOP
                projector)
    Returns the internal energy: the ESP and extra_fock only act through the
    density (READING C-2).
    """
    prob = SCCProblem(Z, xyz, params, cn, esp=esp, charge=charge, extra_fock=extra_fock, n_el=n_el)
    return solve_problem(prob, guess=guess, tol=tol, e_tol=e_tol, max_iter=max_iter, mixer=mixer)


def solve_problem(prob: "SCCProblem", guess=None, tol=1e-10, e_tol=1e-10, max_iter=300,
                  mixer=None) -> SCCResult:
    """The SCC loop of scc() on an already assembled SCCProblem."""
    dq = np.zeros(prob.basis.n_sh) if guess is None else np.asarray(guess, dtype=np.float64).copy()
    mixer = Broyden() if mixer is None else mixer
    e_prev = None
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        r = prob.step(dq)
        diff = np.max(np.abs(r["dq_out"] - dq)) if len(dq) else 0.0
        if e_prev is not None and diff < tol and abs(r["e_el"] - e_prev) < e_tol:
            converged = True
            break
        e_prev = r["e_el"]
        dq = mixer.step(dq, r["dq_out"])
    return SCCResult(energy=r["e_el"] + prob.e_rep, e_el=r["e_el"], e_rep=prob.e_rep, e_band=r["e_band"],
                     e_coul2=r["e2"], e_coul3=r["e3"], minus_ts=r["mts"], dq=r["dq_out"], P=r["P"],
                     S=prob.S, H0=prob.H0, C=r["C"], eps=r["eps"], occ=r["occ"], iterations=it,
                     converged=converged, basis=prob.basis)


def single_point(system, params, tol=1e-10, **kw) -> SCCResult:
    """Unfragmented GFN1-xTB SCC of a whole system (the FMO reference)."""
    cn = coordination_numbers(system.Z, system.xyz, params)
    return scc(system.Z, system.xyz, params, cn, charge=float(np.sum(system.frag_charge)),
               tol=tol, **kw)
