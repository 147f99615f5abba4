"""Pins of the FP64 oracle against things other than itself: closed forms,
limits, brute-force quadrature, invariants of the SCC solution and the FMO
identities that the paper's energy expressions fix."""
import numpy as np
import pytest
from scipy import optimize

from oracle import fmo, xtb
from paper_2606_28022_b300.inputs import geometry as G
from paper_2606_28022_b300.inputs.params import ANGSTROM, KB_HARTREE

from _toytables import hueckel_like, single_s_element, sp_element, toy_params


# ---------------------------------------------------------------- overlap
def test_overlap_ss_single_primitive_closed_form():
    # two normalised s Gaussians: <a|b> = (2 sqrt(ab)/(a+b))^(3/2) exp(-ab/(a+b) R^2)
    p = toy_params({1: single_s_element(1, 0.7, -0.5, 0.5), 2: single_s_element(2, 1.9, -0.5, 0.5)})
    R = 1.37
    S = xtb.overlap_matrix(np.array([1, 2]), np.array([[0, 0, 0], [0.3, -0.5, R]], float), p)
    r2 = 0.3 ** 2 + 0.5 ** 2 + R ** 2
    a, b = 0.7, 1.9
    ref = (2 * np.sqrt(a * b) / (a + b)) ** 1.5 * np.exp(-a * b / (a + b) * r2)
    assert S[0, 1] == pytest.approx(ref, rel=1e-13)
    assert S[0, 0] == pytest.approx(1.0, abs=1e-14) and S[1, 1] == pytest.approx(1.0, abs=1e-14)


def _grid_basis_values(Z, xyz, params, pts):
    """Brute-force values of every AO on a set of points."""
    vals = []
    for a, z in enumerate(Z):
        el = params.elements[int(z)]
        d = pts - xyz[a]
        r2 = (d * d).sum(-1)
        for k, l in enumerate(el.shells_l):
            al = np.asarray(el.alpha[k])
            c = np.asarray(el.coef[k])
            radial = sum(ci * (2 * ai / np.pi) ** 0.75 * np.exp(-ai * r2) *
                         (1.0 if l == 0 else 2 * np.sqrt(ai)) for ai, ci in zip(al, c))
            if l == 0:
                vals.append(radial)
            else:
                for m in range(3):
                    vals.append(radial * d[:, m])
    return np.array(vals)


def test_overlap_sp_brute_force_quadrature():
    p = toy_params({6: sp_element(6, 0.8, 0.6), 1: single_s_element(1, 0.9, -0.4, 0.5)})
    Z = np.array([6, 6, 1])
    xyz = np.array([[0.0, 0.0, 0.0], [1.1, 0.7, -0.4], [-0.5, 1.2, 0.9]])
    S = xtb.overlap_matrix(Z, xyz, p)
    h = 0.12
    ax = np.arange(-9.0, 9.0 + 1e-9, h)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3) + xyz.mean(0)
    v = _grid_basis_values(Z, xyz, p, g)
    Sq = (v @ v.T) * h ** 3
    assert np.max(np.abs(S - Sq)) < 1e-9


def test_overlap_p_block_rotates_as_a_tensor():
    p = toy_params({6: sp_element(6, 0.8, 0.6)})
    Z = np.array([6, 6])
    xyz = np.array([[0.0, 0.0, 0.0], [1.3, -0.4, 0.8]])
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    S1 = xtb.overlap_matrix(Z, xyz, p)
    S2 = xtb.overlap_matrix(Z, xyz @ Q.T, p)
    # AO order per atom: s, px, py, pz -> p block of atom 1 vs atom 2 is S[1:4, 5:8]
    assert np.allclose(Q @ S1[1:4, 5:8] @ Q.T, S2[1:4, 5:8], atol=1e-14)
    assert np.allclose(Q @ S1[1:4, 4], S2[1:4, 4], atol=1e-14)


def test_overlap_water_cluster_properties(params, water64):
    s = water64.subsystem(range(4))
    S = xtb.overlap_matrix(s.Z, s.xyz, params)
    assert np.allclose(S, S.T, atol=1e-14)
    assert np.allclose(np.diag(S), 1.0, atol=1e-12)
    # on-site blocks are the identity (H 1s/2s made orthogonal in the basis)
    b = xtb.make_basis(s.Z, params)
    for a in range(len(s.Z)):
        idx = np.nonzero(b.ao_atom == a)[0]
        assert np.allclose(S[np.ix_(idx, idx)], np.eye(len(idx)), atol=1e-12)
    assert np.linalg.eigvalsh(S).min() > 0


# ---------------------------------------------------------------- CN, gamma, repulsion
def test_cn_counting_function_midpoint_and_limits(params):
    rc = params.elements[1].r_cov + params.elements[8].r_cov
    Z = np.array([8, 1])
    # at R = k2 (Rcov_A + Rcov_B) the count is exactly one half
    xyz = np.array([[0, 0, 0], [0, 0, params.cn_k2 * rc]], float)
    assert xtb.coordination_numbers(Z, xyz, params) == pytest.approx([0.5, 0.5], abs=1e-15)
    near = xtb.coordination_numbers(Z, np.array([[0, 0, 0], [0, 0, 0.3 * rc]], float), params)
    assert near[0] > 1 - 1e-9
    # decreasing with distance towards the R -> infinity value 1/(1+e^k1)
    rs = np.array([1.0, 2.0, 4.0, 8.0, 13.0]) * rc
    vals = [xtb.coordination_numbers(Z, np.array([[0, 0, 0], [0, 0, r]], float), params)[0] for r in rs]
    assert np.all(np.diff(vals) < 0)
    assert vals[-1] > 1.0 / (1.0 + np.exp(params.cn_k1)) and vals[-1] < 1e-5


def test_cn_additive_and_cutoff(params, water64):
    s = water64.subsystem(range(3))
    cn3 = xtb.coordination_numbers(s.Z, s.xyz, params)
    # adding an atom beyond the cutoff leaves every CN unchanged (READING C-3)
    Z = np.append(s.Z, 1)
    xyz = np.vstack([s.xyz, s.xyz.mean(0) + [params.cn_cutoff + 40.0, 0, 0]])
    assert np.allclose(xtb.coordination_numbers(Z, xyz, params)[:-1], cn3, atol=0)
    # pairwise additivity: CN of a water O = sum of its two O-H two-atom counts
    w = water64.subsystem([0])
    cn = xtb.coordination_numbers(w.Z, w.xyz, params)
    pair = [xtb.coordination_numbers(w.Z[[0, k]], w.xyz[[0, k]], params)[0] for k in (1, 2)]
    hh = xtb.coordination_numbers(w.Z[[1, 2]], w.xyz[[1, 2]], params)[0]
    assert cn[0] == pytest.approx(sum(pair), rel=1e-14)
    assert cn[1] == pytest.approx(pair[0] + hh, rel=1e-14)


def test_gamma_limits(params):
    eta = np.array([0.4, 0.7])
    pos = np.zeros((2, 3))
    g0 = xtb.gamma_between(pos[:1], eta[:1], pos[:1], eta[:1], 2.0)
    assert g0[0, 0] == pytest.approx(0.4, rel=1e-15)          # gamma(R=0) = eta
    g = xtb.gamma_between(pos[:1], eta[:1], pos[1:] + [0, 0, 1e4], eta[1:], 2.0)
    assert g[0, 0] * 1e4 == pytest.approx(1.0, rel=1e-7)       # Coulomb tail
    # k_g = 2: Klopman-Ohno 1/sqrt(R^2 + (1/eta_AB)^2) with eta_AB the harmonic mean
    R = 2.3
    g = xtb.gamma_between(pos[:1], eta[:1], np.array([[0, 0, R]]), eta[1:], 2.0)
    eta_ab = 1.0 / (0.5 * (1 / 0.4 + 1 / 0.7))
    assert g[0, 0] == pytest.approx(1.0 / np.sqrt(R * R + eta_ab ** -2), rel=1e-14)


def test_repulsion_short_range_coulomb_limit_and_pair_sum(params):
    Z = np.array([6, 1])
    r = 1e-4
    e = xtb.repulsion_energy(Z, np.array([[0, 0, 0], [0, 0, r]], float), params)
    zz = params.elements[6].z_eff * params.elements[1].z_eff
    assert e * r == pytest.approx(zz, rel=1e-3)
    # three atoms: every unordered pair counted once
    xyz = np.array([[0, 0, 0], [0, 0, 2.0], [0, 1.7, 0]], float)
    Z3 = np.array([6, 1, 8])
    e3 = xtb.repulsion_energy(Z3, xyz, params)
    pairs = sum(xtb.repulsion_energy(Z3[[i, j]], xyz[[i, j]], params) for i, j in [(0, 1), (0, 2), (1, 2)])
    assert e3 == pytest.approx(pairs, rel=1e-14)


# ---------------------------------------------------------------- H0
def test_h0_reduces_to_extended_hueckel(params, water64):
    # with every GFN1 modifier off, Eq. 8 is the Wolfsberg-Helmholz rule of
    # extended Hueckel theory: H_ij = 1.75 S_ij (H_ii + H_jj)/2
    q = hueckel_like(params)
    s = water64.subsystem([0, 1])
    b = xtb.make_basis(s.Z, q)
    S = xtb.overlap_matrix(s.Z, s.xyz, q, b)
    H = xtb.h0_matrix(s.Z, s.xyz, q, S, np.zeros(len(s.Z)), b)
    d = np.diag(H)
    ref = 1.75 * S * 0.5 * (d[:, None] + d[None, :])
    off = b.ao_atom[:, None] != b.ao_atom[None, :]
    assert np.allclose(H[off], ref[off], rtol=1e-14, atol=1e-16)
    levels = [q.elements[int(s.Z[a])].h_l[k] for a, k in zip(b.sh_atom, b.sh_index)]
    assert np.allclose(d, np.array(levels)[b.ao_shell], rtol=0, atol=0)


def test_h0_is_proportional_to_s_within_shell_blocks(params, water64):
    s = water64.subsystem([0, 1])
    b = xtb.make_basis(s.Z, params)
    S = xtb.overlap_matrix(s.Z, s.xyz, params, b)
    cn = xtb.coordination_numbers(s.Z, s.xyz, params)
    H = xtb.h0_matrix(s.Z, s.xyz, params, S, cn, b)
    assert np.allclose(H, H.T, atol=1e-16)
    for i in range(b.n_sh):
        for j in range(b.n_sh):
            if b.sh_atom[i] == b.sh_atom[j]:
                continue
            ii = np.nonzero(b.ao_shell == i)[0]
            jj = np.nonzero(b.ao_shell == j)[0]
            blkS = S[np.ix_(ii, jj)]
            blkH = H[np.ix_(ii, jj)]
            big = np.abs(blkS) > 1e-6
            if big.sum() > 1:
                ratio = blkH[big] / blkS[big]
                assert np.allclose(ratio, ratio[0], rtol=1e-12)


# ---------------------------------------------------------------- Fermi
def test_fermi_aufbau_degenerate_and_entropy():
    kT = KB_HARTREE * 300.0
    n, ef, mts = xtb.fermi_occupations(np.array([-1.0, -0.6, 0.4, 0.9]), 4.0, kT)
    assert np.allclose(n, [2, 2, 0, 0], atol=1e-12) and abs(mts) < 1e-12
    # a doubly degenerate level holding 2 of its 4 places: f = 1/2 each,
    # -T S_el = 2 kT * 2 * [2 * 1/2 ln 1/2] = -4 kT ln 2
    n, ef, mts = xtb.fermi_occupations(np.array([-1.0, -0.5, -0.5, 0.9]), 4.0, kT)
    assert np.allclose(n, [2, 1, 1, 0], atol=1e-9)
    assert ef == pytest.approx(-0.5, abs=1e-9)
    assert mts == pytest.approx(-4 * kT * np.log(2), rel=1e-8)
    assert n.sum() == pytest.approx(4.0, abs=1e-12)


# ---------------------------------------------------------------- Broyden
def test_broyden_solves_a_linear_fixed_point():
    rng = np.random.default_rng(3)
    n = 6
    A = rng.normal(scale=0.3, size=(n, n))
    b = rng.normal(size=n)
    x_star = np.linalg.solve(np.eye(n) - A, b)
    # quasi-Newton on a linear map: converges in about n steps, where plain
    # linear mixing with the same weight needs hundreds
    mix = xtb.Broyden(alpha=0.4, history=20, w0=0.01)
    x = np.zeros(n)
    steps = 0
    while np.max(np.abs(A @ x + b - x)) > 1e-12 and steps < 100:
        x = mix.step(x, A @ x + b)
        steps += 1
    assert steps <= 2 * n + 4
    assert np.max(np.abs(x - x_star)) < 1e-10


# ---------------------------------------------------------------- SCC
def test_scc_two_level_closed_form():
    """Heteronuclear 2-orbital SCC solved independently: closed-form lowest
    root of the 2x2 generalised eigenproblem and a scalar root search for the
    self-consistent charge, with second- and third-order shifts."""
    A = single_s_element(1, 0.9, -0.55, 0.50, gamma3=0.10, z_eff=1.0)
    B = single_s_element(2, 0.6, -0.30, 0.35, gamma3=0.05, z_eff=1.0)
    p = toy_params({1: A, 2: B}, k_poly=None) if False else toy_params({1: A, 2: B})
    p.t_el = 1.0
    Z = np.array([1, 2])
    xyz = np.array([[0, 0, 0], [0, 0, 1.6]], float)
    cn = np.zeros(2)
    r = xtb.scc(Z, xyz, p, cn, tol=1e-12, e_tol=1e-13)
    assert r.converged
    b = r.basis
    S, H0 = r.S, r.H0
    gam = xtb.gamma_matrix(Z, xyz, p, b)
    s = S[0, 1]

    def solve(x):
        dq = np.array([x, -x])
        sig = gam @ dq - np.array([0.10, 0.05]) * dq ** 2
        F = H0 + 0.5 * S * (sig[:, None] + sig[None, :])
        a2, b2, c2 = 1 - s * s, F[0, 0] + F[1, 1] - 2 * s * F[0, 1], F[0, 0] * F[1, 1] - F[0, 1] ** 2
        e = (b2 - np.sqrt(b2 * b2 - 4 * a2 * c2)) / (2 * a2)
        c = np.array([-(F[0, 1] - e * s), F[0, 0] - e])
        c /= np.sqrt(c @ S @ c)
        popA = 2 * (c[0] ** 2 + c[0] * c[1] * s)
        return popA - 1.0 - x, c, dq

    x = optimize.brentq(lambda x: solve(x)[0], -0.9, 0.9, xtol=1e-15)
    _, c, dq = solve(x)
    assert r.dq == pytest.approx(dq, abs=1e-10)
    Pm = 2 * np.outer(c, c)
    e_el = np.sum(Pm * H0) + 0.5 * dq @ gam @ dq - (0.10 * x ** 3 + 0.05 * (-x) ** 3) / 3
    assert r.e_el == pytest.approx(e_el, abs=1e-10)


def test_scc_invariants(params, water64):
    s = water64.subsystem([0, 1, 2])
    r = xtb.single_point(s, params)
    assert r.converged
    nel = xtb.n_electrons(s.Z, params)
    assert np.sum(r.P * r.S) == pytest.approx(nel, abs=1e-10)          # Mulliken (Eq. 3)
    assert r.dq.sum() == pytest.approx(0.0, abs=1e-10)
    assert np.allclose(r.P, r.P.T, atol=1e-14)
    assert np.allclose(r.C.T @ r.S @ r.C, np.eye(len(r.eps)), atol=1e-10)
    # large gap: occupations 2/0, so the density is idempotent, PSP = 2P
    assert np.allclose(r.P @ r.S @ r.P, 2 * r.P, atol=1e-9)


def _energy_functional(r, Z, params, esp):
    """E_el + sum dq * esp as a function of a trial density (Eq. 2 plus the
    embedding interaction), used to test that the Fock matrix of Eq. 7 is its
    derivative: the SCC solution must make it stationary."""
    b = r.basis
    gam = xtb.gamma_matrix(Z, r._xyz, params, b)
    q0 = xtb.shell_param(Z, b, params, "q0_l")
    g3 = xtb.atom_param(Z, params, "gamma3")

    def E(P):
        pops = np.bincount(b.ao_shell, weights=(P * r.S).sum(1), minlength=b.n_sh)
        dq = pops - q0
        dqa = np.bincount(b.sh_atom, weights=dq, minlength=len(Z))
        return np.sum(P * r.H0) + 0.5 * dq @ gam @ dq - np.sum(g3 * dqa ** 3) / 3 + dq @ esp
    return E


@pytest.mark.parametrize("with_esp", [False, True])
def test_scc_energy_is_stationary(params, water64, with_esp):
    s = water64.subsystem([0, 1])
    cn = xtb.coordination_numbers(s.Z, s.xyz, params)
    b = xtb.make_basis(s.Z, params)
    esp = np.random.default_rng(5).normal(scale=0.05, size=b.n_sh) if with_esp else np.zeros(b.n_sh)
    r = xtb.scc(s.Z, s.xyz, params, cn, esp=esp, tol=1e-12, e_tol=1e-13)
    r._xyz = s.xyz
    E = _energy_functional(r, s.Z, params, esp)
    nocc = int(round(r.occ.sum())) // 2
    for i, a in [(nocc - 1, nocc), (nocc - 3, nocc + 2), (0, len(r.eps) - 1)]:
        def rotated(t):
            C = r.C.copy()
            C[:, i] = np.cos(t) * r.C[:, i] + np.sin(t) * r.C[:, a]
            C[:, a] = -np.sin(t) * r.C[:, i] + np.cos(t) * r.C[:, a]
            return (C * r.occ) @ C.T
        t = 1e-4
        slope = (E(rotated(t)) - E(rotated(-t))) / (2 * t)
        curv = (E(rotated(t)) + E(rotated(-t)) - 2 * E(rotated(0))) / t ** 2
        assert abs(slope) < 1e-7
        assert curv > 0.05                       # a minimum along the rotation


def test_scc_fixed_point_is_mixing_independent(params, water64):
    s = water64.subsystem([3, 4])
    a = xtb.single_point(s, params, mixer=xtb.Broyden())
    b = xtb.single_point(s, params, mixer=xtb.LinearMixer(0.3), max_iter=2000)
    assert a.converged and b.converged
    assert a.energy == pytest.approx(b.energy, abs=1e-10)
    assert np.allclose(a.dq, b.dq, atol=1e-9)


# ---------------------------------------------------------------- FMO identities
def test_fmo2_of_two_fragments_equals_full_scc(params, water64):
    s = water64.subsystem([5, 9])
    full = xtb.single_point(s, params)
    r = fmo.fmo(s, params, fmo.FMOOptions(all_dimers_scc=True))
    assert r.e_fmo2 == pytest.approx(full.energy, abs=1e-10)


def test_fmo3_of_three_fragments_equals_full_scc(params, water64):
    s = water64.subsystem([0, 1, 2])
    full = xtb.single_point(s, params)
    r = fmo.fmo(s, params, fmo.FMOOptions(level=3, all_dimers_scc=True, trimer_cut=1e9))
    assert len(r.trimers) == 1
    assert r.e_fmo3 == pytest.approx(full.energy, abs=1e-10)


def test_fmo1_of_far_fragments_is_the_sum_of_isolated_ones(params, water64):
    s = G.separated(water64.subsystem([0, 1, 2, 3]), 1000.0)
    r = fmo.fmo(s, params)
    iso = sum(xtb.single_point(s.subsystem([f]), params).energy for f in range(4))
    assert r.e_fmo1 == pytest.approx(iso, abs=1e-9)
    assert not r.dimer_scc.any()                       # all pairs beyond 4 A


def test_fmo_error_small_and_fmo3_better(params, water64):
    # READING C-2 (internal energies): the fragmentation error of FMO2 is of
    # the size the paper reports for water (<~1e-4 Eh per fragment), and FMO3
    # improves on it.  Counting the embedding energy inside E_I would instead
    # leave errors of the size of the inter-fragment Coulomb energy.
    s = water64.subsystem(list(range(6)))
    full = xtb.single_point(s, params)
    r = fmo.fmo(s, params, fmo.FMOOptions(level=3, all_dimers_scc=True, trimer_cut=1e9))
    e2 = abs(r.e_fmo2 - full.energy) / 6
    e3 = abs(r.e_fmo3 - full.energy) / 6
    assert e2 < 1e-4 and e3 < e2
    assert abs(r.e_fmo1 - full.energy) / 6 > 10 * e2


@pytest.mark.parametrize("loop", ["nested-jacobi", "nested-gauss-seidel"])
def test_monomer_loop_fixed_point_independent_of_order(params, water64, loop):
    # READING C-9: how the monomer charges are iterated does not change the
    # fixed point the paper defines (every monomer self-consistent in the ESP
    # of all others)
    s = water64.subsystem([0, 1, 2, 3, 4])
    a = fmo.fmo(s, params, fmo.FMOOptions(all_dimers_scc=True))          # global Broyden loop
    b = fmo.fmo(s, params, fmo.FMOOptions(all_dimers_scc=True, monomer_loop="nested",
                                          gauss_seidel=(loop == "nested-gauss-seidel")))
    assert a.e_fmo2 == pytest.approx(b.e_fmo2, abs=1e-9)
    assert np.allclose(np.concatenate(a.dq_mono), np.concatenate(b.dq_mono), atol=1e-9)


def test_monomer_charges_are_self_consistent(params, water64):
    # at the fixed point each monomer's SCC, solved alone in the ESP of the
    # other monomers' final charges, reproduces its own charges
    s = water64.subsystem(range(6))
    r = fmo.fmo(s, params, fmo.FMOOptions(level=1, dimer_cut=0.0))
    fr = fmo._Frags(s, params)
    for I in (0, 3, 5):
        alone = fr.solve((I,), fr.esp((I,), r.dq_mono), None, fmo.FMOOptions())
        assert np.allclose(alone.dq, r.dq_mono[I], atol=1e-9)
        assert alone.energy == pytest.approx(r.e_mono[I], abs=1e-9)


def test_esdim_matches_scc_dimer_for_a_far_pair(params, water64):
    # Eq. 15 is the long-range limit of the SCC pair energy
    s = water64.subsystem([0, 1, 2])
    xyz = s.xyz.copy()
    xyz[s.frag == 2] += np.array([0.0, 0.0, 25.0 * ANGSTROM])
    s = G.System(Z=s.Z, xyz=xyz, frag=s.frag, frag_charge=s.frag_charge)
    a = fmo.fmo(s, params, fmo.FMOOptions(all_dimers_scc=True))
    b = fmo.fmo(s, params, fmo.FMOOptions(all_dimers_scc=False))
    far = [k for k, (I, J) in enumerate(a.dimers) if 2 in (I, J)]
    assert not b.dimer_scc[far].any()
    for k in far:
        assert b.dE_dimer[k] == pytest.approx(a.dE_dimer[k], abs=5e-8)


def test_ddq_of_neutral_dimers_sums_to_zero(params, water64):
    # Eq. 14: the charge moved between I and J on dimer formation is
    # conserved: the dimer and its two monomers carry the same total charge,
    # so sum_mu ddq_mu = 0 for every neutral dimer
    s = water64.subsystem([0, 1, 2, 3])
    opts = fmo.FMOOptions(all_dimers_scc=True)
    r = fmo.fmo(s, params, opts)
    assert r.dimer_scc.all()
    fr = fmo._Frags(s, params)
    moved = 0.0
    for I, J in r.dimers:
        X = (int(I), int(J))
        res = fr.solve(X, fr.esp(X, r.dq_mono), np.concatenate([r.dq_mono[I], r.dq_mono[J]]), opts)
        ddq = res.dq - np.concatenate([r.dq_mono[I], r.dq_mono[J]])
        assert abs(np.sum(ddq)) < 1e-10
        moved = max(moved, float(np.max(np.abs(ddq))))
    assert moved > 1e-4          # charge does move between the close pairs


def test_embedding_correction_is_needed_with_its_sign_and_environment(params, water64):
    # Eq. 13: dE^V_IJ = sum_mu ddq_mu ESP^{not IJ}_mu.  Planted mistakes in
    # it (dropped, sign flipped, the partner's charges left in the ESP) must
    # move FMO2 far from the whole-system SCC energy, which the correct form
    # matches closely (an independent number: full xTB, not the oracle's
    # FMO code)
    s = water64.subsystem([0, 1, 2, 3, 4])
    opts = fmo.FMOOptions(all_dimers_scc=True)
    full = xtb.single_point(s, params).energy
    r = fmo.fmo(s, params, opts)
    err = abs(r.e_fmo2 - full)
    dev = float(np.sum(r.dEV_dimer))
    assert err < 0.05 * abs(r.e_fmo2 - dev - full)          # dE^V dropped
    assert err < 0.05 * abs(r.e_fmo2 - 2.0 * dev - full)    # sign flipped
    fr = fmo._Frags(s, params)
    wrong = 0.0
    for k, (I, J) in enumerate(r.dimers):
        X = (int(I), int(J))
        qm = np.concatenate([r.dq_mono[I], r.dq_mono[J]])
        res = fr.solve(X, fr.esp(X, r.dq_mono), qm, opts)
        # ESP^{not I} on I's shells and ESP^{not J} on J's: the partner included
        esp_bad = np.concatenate([fr.esp((X[0],), r.dq_mono), fr.esp((X[1],), r.dq_mono)])
        wrong += float((res.dq - qm) @ esp_bad) - r.dEV_dimer[k]
    assert err < 0.05 * abs(r.e_fmo2 + wrong - full)
    # a six-water cluster: the correct form still beats every mistake
    s6 = water64.subsystem([0, 1, 2, 3, 4, 5])
    full6 = xtb.single_point(s6, params).energy
    r6 = fmo.fmo(s6, params, opts)
    dev6 = float(np.sum(r6.dEV_dimer))
    err6 = abs(r6.e_fmo2 - full6)
    assert err6 < 0.3 * abs(r6.e_fmo2 - dev6 - full6)
    assert err6 < 0.1 * abs(r6.e_fmo2 - 2.0 * dev6 - full6)


# ---------------------------------------------------------------------------
# hybrid orbital projection (HOP) boundaries


def test_polyalanine_generator_sizes_and_closed_shells(params):
    s = G.polyalanine_helix(300, seed=11)
    assert s.n_atoms == 3003 and 100 <= s.n_frag <= 300
    assert len(s.cut_bonds) == s.n_frag - 1
    for f in range(s.n_frag):
        ne = sum(params.elements[int(z)].n_valence for z in s.Z[s.frag == f])
        ne += np.sum(s.frag[s.cut_bonds[:, 1]] == f) - np.sum(s.frag[s.cut_bonds[:, 0]] == f)
        assert ne % 2 == 0
    d = np.linalg.norm(s.xyz[s.cut_bonds[:, 0]] - s.xyz[s.cut_bonds[:, 1]], axis=1) / ANGSTROM
    assert np.allclose(d, 1.525)


def test_hop_two_fragments_fmo2_equals_full_scc(params):
    # with N = 2 the only dimer heals the cut bond and sees no environment,
    # so FMO2 is the SCC of the whole molecule, whatever the monomers hold
    s = G.polyalanine_helix(2)
    full = xtb.single_point(s, params)
    r = fmo.fmo(s, params, fmo.FMOOptions(level=2))
    assert abs(r.e_fmo2 - full.energy) < 1e-9
    assert abs(r.e_fmo1 - full.energy) > 1e-3       # the monomers alone miss the bond


def test_hop_three_fragments_fmo3_equals_full_scc(params):
    s = G.polyalanine_helix(3)
    full = xtb.single_point(s, params)
    r = fmo.fmo(s, params, fmo.FMOOptions(level=3, all_dimers_scc=True, trimer_cut=1e9))
    assert len(r.trimers) == 1
    assert abs(r.e_fmo3 - full.energy) < 1e-9


def _hop_monomer(params, v_hop=None):
    import dataclasses
    p = params if v_hop is None else dataclasses.replace(params, v_hop=v_hop)
    s = G.polyalanine_helix(3)
    fr = fmo._Frags(s, p)
    prob = fr.problem((1,))           # middle residue: one ghost and one detached BDA
    return s, fr, prob, xtb.solve_problem(prob)


def test_hop_projectors_empty_their_orbitals(params):
    s, fr, prob, res = _hop_monomer(params)
    assert res.converged
    assert abs(np.sum(res.dq)) < 1e-9 and abs(np.sum(prob.q0) - prob.n_el) < 1e-12
    b = prob.basis
    recs = [r for r in fr.recs[1]]
    for i, (a, bond) in enumerate(recs):
        bda, baa = fr.cut[bond] if bond >= 0 else (a, None)
        if bond < 0 and not any(fr.cut[k, 0] == a for k in range(len(fr.cut))):
            continue
        k = bond if bond >= 0 else [k for k in range(len(fr.cut)) if fr.cut[k, 0] == a][0]
        u = s.xyz[fr.cut[k, 1]] - s.xyz[fr.cut[k, 0]]
        u /= np.linalg.norm(u)
        sh = np.nonzero(b.sh_atom == i)[0]
        idx = np.concatenate([[b.sh_ao0[sh[0]]], b.sh_ao0[sh[1]] + np.arange(3)])
        h = np.concatenate([[fmo.C_S], fmo.C_P * u])
        if bond < 0:                   # detached BDA: the bond hybrid is empty
            vecs = h[None, :]
        else:                          # ghost: everything but the bond hybrid is empty
            q, _ = np.linalg.qr(np.column_stack([h, np.eye(4)]))
            vecs = q[:, 1:4].T
        for v in vecs:
            w = prob.S[:, idx] @ v
            assert w @ res.P @ w < 1e-4


def test_hop_energy_converges_as_one_over_v(params):
    e = [_hop_monomer(params, v)[3].energy for v in (1e5, 1e6, 1e7)]
    d1, d2 = e[0] - e[1], e[1] - e[2]
    assert abs(d2) < 1e-5
    assert 7.0 < d1 / d2 < 13.0
