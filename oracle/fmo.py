"""FP64 CPU oracle of FMO1/FMO2/FMO3 with GFN1-xTB fragments.

TEST INFRASTRUCTURE ONLY (see oracle/xtb.py).  It follows Sec. 2.2-2.3 of the
paper step by step:
  Eq. 12      FMO2 energy: sum E_I + sum_{I>J} (E_IJ - E_I - E_J + dE^V_IJ)
  Eqs. 13-14  dimer embedding correction dE^V_IJ from the charge transfer ddq
  Eq. 15      electrostatic dimer (ES-DIM) approximation for far pairs
  Eqs. 16-19  FMO3 energy, trimer interaction energy and its embedding term
  Eqs. 20-21  embedding Fock matrix V^I built from the other fragments'
              Mulliken shell charges (the ESP)
  Sec. 2.3    monomer charges iterated to self-consistency in each other's
              ESP, then dimers and trimers solved in the frozen ESP
READINGS (listed in the design notes):
  C-2  E_I, E_IJ, E_IJK are internal energies; the ESP acts only through the
       density, and dE^V supplies the embedding interaction.
  C-9  the paper asks for monomer charges self-consistent in each other's
       ESP without fixing the iteration.  monomer_loop="global" (default):
       every outer step runs one SCC iteration of every monomer in the ESP of
       the current charges and mixes the concatenated charge vector of all
       monomers with modified Broyden; "nested": every monomer SCC is solved to
       convergence in the ESP of the previous iterate (Jacobi-style, or
       Gauss-Seidel with gauss_seidel=True).  Both have the same fixed point;
       the nested form converges slowly and can diverge for large clusters.
  C-10 SCC dimer iff the closest inter-fragment atom distance < dimer_cut;
       SCC trimer iff all three pair distances < trimer_cut.
  C-11 E^V_{X,Y} sums over fragments K not in the n-mer Y.
  C-12 only SCC trimers contribute; their sub-pair terms are the FMO2 ones.
  C-13 hybrid orbital projection (HOP) at cut covalent bonds: V_HOP =
       params.v_hop (1e6 Eh); the detached BDA keeps its basis and nucleus but
       its reference occupations are scaled to one electron less; its ghost in
       the BAA's fragment has the BDA's element, basis, position and
       supersystem CN, q0 = (1/4, 3/4) on its s and p shell, real gamma and
       third-order terms but no repulsion; both hybrids point from BDA to
       BAA; p functions in x, y, z order.  A bond is healed in every n-mer
       holding both of its fragments.
"""
from __future__ import annotations

import dataclasses
import itertools
import multiprocessing as mp

import numpy as np

from . import xtb

ANGSTROM = 1.0 / 0.529177210903


@dataclasses.dataclass
class FMOOptions:
    level: int = 2
    dimer_cut: float = 4.0 * ANGSTROM          # bohr
    trimer_cut: float = 4.0 * ANGSTROM         # bohr
    all_dimers_scc: bool = False
    scc_tol: float = 1e-10
    e_tol: float = 1e-10
    outer_tol: float = 1e-10
    max_iter: int = 300
    max_outer: int = 200
    gauss_seidel: bool = False
    monomer_loop: str = "global"
    workers: int = 1
    mixer: str = "broyden"


@dataclasses.dataclass
class FMOResult:
    e_fmo1: float
    e_fmo2: float
    e_fmo3: float | None
    e_mono: np.ndarray                  # internal monomer energies E'_I
    dq_mono: list                       # per fragment shell charges
    outer_iterations: int
    dimers: np.ndarray                  # (n_pair, 2) all pairs I<J
    dimer_scc: np.ndarray               # bool: SCC (True) or ES-DIM
    dE_dimer: np.ndarray                # dE_IJ of Eq. 12
    e_dimer: np.ndarray                 # E'_IJ (nan for ES-DIM)
    dEV_dimer: np.ndarray               # dE^V_IJ (0 for ES-DIM)
    trimers: np.ndarray                 # (n_tri, 2) SCC trimers I<J<K
    dE_trimer: np.ndarray               # dE_IJK of Eq. 17
    corr_trimer: np.ndarray             # dE_IJK - dE_IJ - dE_IK - dE_JK
    mono_iters: np.ndarray
    dimer_iters: np.ndarray


C_S, C_P = 0.5, np.sqrt(3.0) / 2.0   # sp3 hybrid coefficients of the HOP hybrid


class _Frags:
    """Per-fragment atom records, shell positions and shell hardnesses.

    A record is (atom, bond): a real atom of the fragment (bond = -1) or the
    ghost of a cut bond's detachment atom (BDA) hosted by the fragment of its
    attachment atom (BAA): a copy of the BDA at its position (Sec. "Covalent
    bond fragmentation", hybrid orbital projection).  A monomer holds every
    record of its fragment; in an n-mer a bond whose BDA and BAA fragments
    are both present is healed (its ghost is left out, the BDA is a normal
    atom), any other cut bond stays detached."""

    def __init__(self, system, params):
        self.system = system
        self.params = params
        nf = system.n_frag
        self.atoms = [np.nonzero(system.frag == f)[0] for f in range(nf)]
        self.cn = xtb.coordination_numbers(system.Z, system.xyz, params)
        self.cut = np.asarray(system.cut_bonds, dtype=np.int64).reshape(-1, 2)
        self.bond_frag = [(int(system.frag[a]), int(system.frag[b])) for a, b in self.cut]
        self.recs = []
        for f in range(nf):
            r = [(int(a), -1) for a in self.atoms[f]]
            r += [(int(self.cut[k, 0]), k) for k in range(len(self.cut)) if self.bond_frag[k][1] == f]
            self.recs.append(r)
        self.sh_pos, self.sh_eta, self.n_sh, self.sh_rec = [], [], [], []
        for f in range(nf):
            at = np.array([a for a, _ in self.recs[f]], dtype=np.int64)
            Z = system.Z[at]
            bas = xtb.make_basis(Z, params)
            self.sh_pos.append(system.xyz[at][bas.sh_atom])
            self.sh_eta.append(xtb.shell_hardness(Z, bas, params))
            self.n_sh.append(bas.n_sh)
            self.sh_rec.append(bas.sh_atom.copy())     # record of each monomer shell

    def gamma(self, I, J):
        return xtb.gamma_between(self.sh_pos[I], self.sh_eta[I], self.sh_pos[J], self.sh_eta[J],
                                 self.params.k_g)

    def present(self, nmer):
        """Per fragment of the n-mer: mask of its records present in the n-mer
        (healed ghosts absent)."""
        return [np.array([bond < 0 or self.bond_frag[bond][0] not in nmer for _, bond in self.recs[f]])
                for f in nmer]

    def shell_mask(self, nmer):
        """Mask over the concatenated monomer shells of the n-mer's fragments:
        True where the shell is also an n-mer shell."""
        pres = self.present(nmer)
        return np.concatenate([pres[k][self.sh_rec[f]] for k, f in enumerate(nmer)])

    def esp_full(self, nmer, dq_mono):
        """ESP^{not X} on every monomer shell of the n-mer's fragments, from the
        monomer charges of every fragment K outside X (Eq. 21 / READING C-11)."""
        out = []
        for I in nmer:
            v = np.zeros(self.n_sh[I])
            for K in range(self.system.n_frag):
                if K in nmer:
                    continue
                v += self.gamma(I, K) @ dq_mono[K]
            out.append(v)
        return np.concatenate(out)

    def esp(self, nmer, dq_mono):
        """ESP^{not X} on the shells of n-mer X."""
        return self.esp_full(nmer, dq_mono)[self.shell_mask(nmer)]

    def closest(self, I, J):
        a = self.system.xyz[self.atoms[I]]
        b = self.system.xyz[self.atoms[J]]
        return float(np.sqrt(((a[:, None, :] - b[None, :, :]) ** 2).sum(-1)).min())

    def problem(self, nmer, esp=None):
        """The SCC problem of n-mer X: real atoms of its fragments plus the
        ghosts of its detached bonds, with (READING C-13)
          - a detached BDA: its reference occupations q0 scaled so that they
            sum to one electron less, and the projector D^BDA = V h h^T;
          - a ghost: the BDA's element, basis, position and supersystem CN,
            q0 = (c_s^2, c_p^2) = (1/4, 3/4) on its s and p shell, no
            repulsion, projector D^ghost = V (1_sp - h h^T);
          - h = c_s s + c_p (b . p) with b the unit vector from BDA to BAA;
        and V^HOP = sum over projected atoms of S[:, atom] D S[atom, :] added to
        the Fock matrix but kept out of the energy (Eqs. of the HOP section)."""
        s, p = self.system, self.params
        recs = [r for k, f in enumerate(nmer) for r, keep in zip(self.recs[f], self.present(nmer)[k]) if keep]
        at = np.array([a for a, _ in recs], dtype=np.int64)
        Z, xyz, cn = s.Z[at], s.xyz[at], self.cn[at]
        bas = xtb.make_basis(Z, p)
        q0 = xtb.shell_param(Z, bas, p, "q0_l")
        rep_mask = np.array([bond < 0 for _, bond in recs])
        proj = []                                   # (record index, bond, kind)
        for i, (a, bond) in enumerate(recs):
            if bond >= 0:
                proj.append((i, bond, "ghost"))
            else:
                for k in range(len(self.cut)):
                    if self.cut[k, 0] == a and self.bond_frag[k][1] not in nmer:
                        proj.append((i, k, "bda"))
        extra = None
        for i, bond, kind in proj:
            sh = np.nonzero(bas.sh_atom == i)[0]
            ls = bas.sh_l[sh]
            if sorted(ls.tolist()) != [0, 1]:
                raise ValueError("a HOP boundary atom needs exactly one s and one p shell")
            s_sh, p_sh = sh[ls == 0][0], sh[ls == 1][0]
            if kind == "ghost":
                q0[s_sh], q0[p_sh] = C_S ** 2, C_P ** 2
            else:
                q0[sh] *= (np.sum(q0[sh]) - 1.0) / np.sum(q0[sh])
            bvec = s.xyz[self.cut[bond, 1]] - s.xyz[self.cut[bond, 0]]
            bvec = bvec / np.linalg.norm(bvec)
            idx = np.concatenate([[bas.sh_ao0[s_sh]], bas.sh_ao0[p_sh] + np.arange(3)])
            h = np.concatenate([[C_S], C_P * bvec])
            D = p.v_hop * (np.outer(h, h) if kind == "bda" else np.eye(4) - np.outer(h, h))
            if extra is None:
                S = xtb.overlap_matrix(Z, xyz, p, bas)
                extra = np.zeros_like(S)
            extra += S[:, idx] @ D @ S[idx, :]
        charge = float(sum(s.frag_charge[f] for f in nmer))
        return xtb.SCCProblem(Z, xyz, p, cn, esp=esp, charge=charge, extra_fock=extra,
                              n_el=float(np.sum(q0)) - charge, q0=q0, rep_mask=rep_mask)

    def solve(self, nmer, esp, guess, opts):
        mixer = xtb.Broyden() if opts.mixer == "broyden" else xtb.LinearMixer(0.4)
        return xtb.solve_problem(self.problem(nmer, esp), guess=guess, tol=opts.scc_tol, e_tol=opts.e_tol,
                                 max_iter=opts.max_iter, mixer=mixer)


def _embedding_correction(fr, nmer, dq, dq_mono):
    """dE^V_X = sum_mu ddq^X_mu ESP^{not X}_mu (Eqs. 13-14, 18) over the
    monomer shells of X: ddq = dq^X - dq^mono on shells of the n-mer, and
    ddq = -dq^mono on the ghost shells of bonds healed in X (the charge the
    ghost carried in its monomer, HOP section)."""
    mask = fr.shell_mask(nmer)
    mono = np.concatenate([dq_mono[f] for f in nmer])
    full = np.zeros_like(mono)
    full[mask] = dq
    return float((full - mono) @ fr.esp_full(nmer, dq_mono))


def _global_monomer_loop(fr, opts):
    """One SCC iteration of every monomer per outer step, in the ESP of the
    current charges, then one modified-Broyden update of all monomer charges
    together; ends when the charges reproduce themselves (READING C-9)."""
    s = fr.system
    nf = s.n_frag
    probs = []
    for I in range(nf):
        probs.append(fr.problem((I,)))
    bounds = np.concatenate([[0], np.cumsum(fr.n_sh)])
    split = lambda x: [x[bounds[I]:bounds[I + 1]] for I in range(nf)]
    x = np.zeros(bounds[-1])
    mixer = xtb.Broyden() if opts.mixer == "broyden" else xtb.LinearMixer(0.4)
    e_prev = None
    for outer in range(1, opts.max_outer + 1):
        parts = split(x)
        outs = [probs[I].step(parts[I], esp=fr.esp((I,), parts)) for I in range(nf)]
        x_out = np.concatenate([o["dq_out"] for o in outs])
        e_mono = np.array([o["e_el"] + probs[I].e_rep for I, o in enumerate(outs)])
        diff = float(np.max(np.abs(x_out - x)))
        e1 = float(np.sum(e_mono))
        if e_prev is not None and diff < opts.outer_tol and abs(e1 - e_prev) < opts.e_tol:
            return [p.copy() for p in split(x_out)], e_mono, outer
        e_prev = e1
        x = mixer.step(x, x_out)
    return [p.copy() for p in split(x_out)], e_mono, opts.max_outer


_POOL_STATE = {}


def _pool_init(system, params):
    _POOL_STATE["fr"] = _Frags(system, params)


def _pool_solve(args):
    nmer, esp, guess, opts = args
    r = _POOL_STATE["fr"].solve(nmer, esp, guess, opts)
    return r.energy, r.dq, r.iterations, r.converged


def fmo(system, params, opts: FMOOptions | None = None) -> FMOResult:
    opts = FMOOptions() if opts is None else opts
    fr = _Frags(system, params)
    nf = system.n_frag
    pool = None
    if opts.workers > 1:
        pool = mp.get_context("spawn").Pool(opts.workers, initializer=_pool_init,
                                            initargs=(system, params))

    def run_many(jobs):
        if pool is None:
            out = []
            for nmer, esp, guess in jobs:
                r = fr.solve(nmer, esp, guess, opts)
                out.append((r.energy, r.dq, r.iterations, r.converged))
            return out
        return pool.map(_pool_solve, [(n, e, g, opts) for (n, e, g) in jobs], chunksize=4)

    try:
        # ---- monomer self-consistency in the ESP (Sec. 2.3)
        dq_mono = [np.zeros(fr.n_sh[I]) for I in range(nf)]
        e_mono = np.zeros(nf)
        mono_iters = np.zeros(nf, dtype=np.int64)
        outer = 0
        if opts.monomer_loop == "global":
            dq_mono, e_mono, outer = _global_monomer_loop(fr, opts)
            mono_iters[:] = outer
        for outer in (range(1, opts.max_outer + 1) if opts.monomer_loop == "nested" else []):
            change = 0.0
            if opts.gauss_seidel:
                for I in range(nf):
                    (e, dq, it, ok), = run_many([((I,), fr.esp((I,), dq_mono), dq_mono[I])])
                    change = max(change, float(np.max(np.abs(dq - dq_mono[I]))))
                    dq_mono[I], e_mono[I], mono_iters[I] = dq, e, mono_iters[I] + it
            else:
                jobs = [((I,), fr.esp((I,), dq_mono), dq_mono[I]) for I in range(nf)]
                res = run_many(jobs)
                for I, (e, dq, it, ok) in enumerate(res):
                    change = max(change, float(np.max(np.abs(dq - dq_mono[I]))))
                    dq_mono[I], e_mono[I], mono_iters[I] = dq, e, mono_iters[I] + it
            if change < opts.outer_tol:
                break
        e_fmo1 = float(np.sum(e_mono))

        # ---- dimers (Eqs. 12-15)
        pairs = np.array([(I, J) for I in range(nf) for J in range(I + 1, nf)], dtype=np.int64).reshape(-1, 2)
        rmin = np.array([fr.closest(I, J) for I, J in pairs])
        scc_pair = np.ones(len(pairs), dtype=bool) if opts.all_dimers_scc else rmin < opts.dimer_cut
        dE = np.zeros(len(pairs))
        e_dim = np.full(len(pairs), np.nan)
        dEV = np.zeros(len(pairs))
        d_iters = np.zeros(len(pairs), dtype=np.int64)
        jobs, where = [], []
        for k, (I, J) in enumerate(pairs):
            if scc_pair[k]:
                mask = fr.shell_mask((I, J))
                esp = fr.esp_full((I, J), dq_mono)
                jobs.append(((I, J), esp[mask], np.concatenate([dq_mono[I], dq_mono[J]])[mask]))
                where.append(k)
            else:
                dE[k] = float(dq_mono[I] @ fr.gamma(I, J) @ dq_mono[J])       # Eq. 15
        for k, (job, (e, dq, it, ok)) in zip(where, zip(jobs, run_many(jobs))):
            I, J = pairs[k]
            dEV[k] = _embedding_correction(fr, (int(I), int(J)), dq, dq_mono)   # Eqs. 13-14
            e_dim[k] = e
            dE[k] = e - e_mono[I] - e_mono[J] + dEV[k]                       # Eq. 12
            d_iters[k] = it
        e_fmo2 = e_fmo1 + float(np.sum(dE))

        # ---- trimers (Eqs. 16-19)
        trimers = np.zeros((0, 3), dtype=np.int64)
        dE3 = np.zeros(0)
        corr = np.zeros(0)
        e_fmo3 = None
        if opts.level >= 3:
            pair_index = {(int(I), int(J)): k for k, (I, J) in enumerate(pairs)}
            near = {(int(I), int(J)) for (I, J), r in zip(pairs, rmin) if r < opts.trimer_cut}
            tri = [t for t in itertools.combinations(range(nf), 3)
                   if (t[0], t[1]) in near and (t[0], t[2]) in near and (t[1], t[2]) in near]
            trimers = np.array(tri, dtype=np.int64).reshape(-1, 3)
            jobs = [(tuple(t), fr.esp(tuple(t), dq_mono),
                     np.concatenate([dq_mono[f] for f in t])[fr.shell_mask(tuple(t))]) for t in tri]
            res = run_many(jobs)
            dE3 = np.zeros(len(tri))
            corr = np.zeros(len(tri))
            for k, (t, job, (e, dq, it, ok)) in enumerate(zip(tri, jobs, res)):
                I, J, K = t
                dEV3 = _embedding_correction(fr, tuple(int(f) for f in t), dq, dq_mono)   # Eq. 18 / C-11
                dE3[k] = e - e_mono[I] - e_mono[J] - e_mono[K] + dEV3        # Eq. 17
                corr[k] = (dE3[k] - dE[pair_index[(I, J)]] - dE[pair_index[(I, K)]]
                           - dE[pair_index[(J, K)]])                         # Eq. 16
            e_fmo3 = e_fmo2 + float(np.sum(corr))
    finally:
        if pool is not None:
            pool.close()
            pool.join()

    return FMOResult(e_fmo1=e_fmo1, e_fmo2=e_fmo2, e_fmo3=e_fmo3, e_mono=e_mono, dq_mono=dq_mono,
                     outer_iterations=outer, dimers=pairs, dimer_scc=scc_pair, dE_dimer=dE,
                     e_dimer=e_dim, dEV_dimer=dEV, trimers=trimers, dE_trimer=dE3,
                     corr_trimer=corr, mono_iters=mono_iters, dimer_iters=d_iters)
