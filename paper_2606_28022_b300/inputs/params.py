"""Element parameter table (an input of the method).

The paper writes GFN1-xTB's energy, Fock and H0 expressions (Eqs. 1-10) but
prints none of the element parameters; it refers to the GFN1-xTB publication.
The library therefore takes the table as an input.  This module writes a
*synthetic* GFN1-shaped table for H, C, N and O with textbook-plausible
magnitudes (valence ionisation-potential-like levels, Slater's-rule
exponents, Pauling electronegativities, covalent radii), chosen so that water,
acenes and peptides come out closed shell with large HOMO-LUMO gaps.  A user
can supply a real table through the same structure.

Units: Hartree and bohr.  Shell order per element is the basis order.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import sto

ANGSTROM = 1.0 / 0.529177210903          # bohr per angstrom
KB_HARTREE = 3.166811563e-6              # Boltzmann constant, Eh / K
MAX_Z = 87
MAX_SHELL = 3
MAX_PRIM = 12

SYMBOL = {1: "H", 6: "C", 7: "N", 8: "O"}
NUMBER = {v: k for k, v in SYMBOL.items()}


@dataclasses.dataclass
class Element:
    z: int
    shells_l: list          # angular momentum per shell
    alpha: list             # per shell: exponents of normalised primitives
    coef: list              # per shell: contraction coefficients
    h_l: list               # H_A^l, Eq. 10 (Eh)
    k_cn_l: list            # k_CN,l, Eq. 10
    k_poly_l: list          # k^poly_{A,l}, Eq. 9
    kappa_l: list           # kappa_A^l, Eq. 5
    q0_l: list              # reference shell occupations (electrons)
    eta: float              # eta_A, Eq. 5 (Eh)
    gamma3: float           # Gamma_A, third order (Eh)
    en: float               # electronegativity (Pauling)
    r_cov: float            # covalent radius (bohr)
    z_eff: float            # Z^eff_A, Eq. 11
    alpha_rep: float        # alpha_A, Eq. 11

    @property
    def n_shell(self) -> int:
        return len(self.shells_l)

    @property
    def n_ao(self) -> int:
        return sum(2 * l + 1 for l in self.shells_l)

    @property
    def n_valence(self) -> float:
        return float(sum(self.q0_l))


@dataclasses.dataclass
class Params:
    elements: dict                 # z -> Element
    k_l: tuple = (1.85, 2.25, 2.0)  # k_l of Eq. 8 for s, p, d
    k_en: float = -0.007           # k_EN of Eq. 8
    k_g: float = 2.0               # k_g of Eq. 4
    k_f: float = 1.5               # k_f of Eq. 11
    cn_k1: float = 16.0            # k_1 of the CN counting function
    cn_k2: float = 4.0 / 3.0       # k_2 of the CN counting function
    cn_cutoff: float = 25.0        # bohr; pairs beyond are not counted
    t_el: float = 300.0            # electronic temperature (K)
    v_hop: float = 1.0e6           # HOP projector strength (Eh)
    k_ab_special: dict = dataclasses.field(default_factory=dict)

    def k_ab(self, za: int, zb: int) -> float:
        key = (min(za, zb), max(za, zb))
        return self.k_ab_special.get(key, 1.0)

    def k_ab_matrix(self) -> np.ndarray:
        m = np.ones((MAX_Z, MAX_Z))
        for (a, b), v in self.k_ab_special.items():
            m[a, b] = m[b, a] = v
        return m


def _element(z, shells, **kw) -> Element:
    """shells: list of (n_quantum, l, zeta)."""
    ls, alphas, coefs = [], [], []
    for (n, l, zeta) in shells:
        a, c = sto.contracted_shell(n, l, zeta, 6)
        # a second shell of the same l on the same atom (H 2s) is made
        # orthogonal to the first one, so that on-site overlap blocks are the
        # identity (a reading of the paper; see the design notes)
        for j, lj in enumerate(ls):
            if lj == l:
                a, c = sto.orthogonalise(l, alphas[j], coefs[j], a, c)
        ls.append(l)
        alphas.append(np.asarray(a))
        coefs.append(np.asarray(c))
    return Element(z=z, shells_l=ls, alpha=alphas, coef=coefs, **kw)


def synthetic_gfn1_table() -> Params:
    """The builder-written GFN1-shaped H/C/N/O table used by tests and bench."""
    A = ANGSTROM
    els = {
        1: _element(1, [(1, 0, 1.20), (2, 0, 0.90)],
                    h_l=[-0.405, -0.080], k_cn_l=[-0.004, 0.0],
                    k_poly_l=[-0.10, 0.05], kappa_l=[0.0, -0.20], q0_l=[1.0, 0.0],
                    eta=0.470, gamma3=0.080, en=2.20, r_cov=0.32 * A,
                    z_eff=1.10, alpha_rep=2.20),
        6: _element(6, [(2, 0, 1.63), (2, 1, 1.55)],
                    h_l=[-0.520, -0.375], k_cn_l=[0.006, -0.003],
                    k_poly_l=[-0.05, 0.06], kappa_l=[0.0, -0.10], q0_l=[1.0, 3.0],
                    eta=0.420, gamma3=0.150, en=2.55, r_cov=0.75 * A,
                    z_eff=4.20, alpha_rep=2.30),
        7: _element(7, [(2, 0, 1.95), (2, 1, 1.85)],
                    h_l=[-0.640, -0.470], k_cn_l=[0.006, -0.003],
                    k_poly_l=[-0.06, 0.02], kappa_l=[0.0, -0.05], q0_l=[1.5, 3.5],
                    eta=0.500, gamma3=0.170, en=3.04, r_cov=0.71 * A,
                    z_eff=5.20, alpha_rep=2.45),
        8: _element(8, [(2, 0, 2.27), (2, 1, 2.15)],
                    h_l=[-0.780, -0.560], k_cn_l=[0.006, -0.003],
                    k_poly_l=[-0.06, 0.02], kappa_l=[0.0, 0.05], q0_l=[2.0, 4.0],
                    eta=0.580, gamma3=0.200, en=3.44, r_cov=0.63 * A,
                    z_eff=6.00, alpha_rep=2.60),
    }
    return Params(elements=els, k_ab_special={(1, 1): 0.96, (1, 7): 1.02})


def kT(params: Params) -> float:
    return KB_HARTREE * params.t_el
