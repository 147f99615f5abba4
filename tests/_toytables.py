"""Small hand-made parameter tables for closed-form pins of the oracle."""
import copy

import numpy as np

from paper_2606_28022_b300.inputs.params import Element, Params


def single_s_element(z, alpha, h, eta, q0=1.0, gamma3=0.0, en=2.2, r_cov=1.0, z_eff=1.0,
                     alpha_rep=1.0, k_cn=0.0, k_poly=0.0, kappa=0.0):
    """An element with one s shell made of a single normalised primitive."""
    return Element(z=z, shells_l=[0], alpha=[np.array([alpha])], coef=[np.array([1.0])],
                   h_l=[h], k_cn_l=[k_cn], k_poly_l=[k_poly], kappa_l=[kappa], q0_l=[q0],
                   eta=eta, gamma3=gamma3, en=en, r_cov=r_cov, z_eff=z_eff, alpha_rep=alpha_rep)


def sp_element(z, alpha_s, alpha_p, **kw):
    """One s and one p shell, each a single normalised primitive."""
    base = dict(h_l=[-0.5, -0.4], k_cn_l=[0.0, 0.0], k_poly_l=[0.0, 0.0], kappa_l=[0.0, 0.0],
                q0_l=[1.0, 1.0], eta=0.5, gamma3=0.0, en=2.5, r_cov=1.4, z_eff=2.0, alpha_rep=1.0)
    base.update(kw)
    return Element(z=z, shells_l=[0, 1], alpha=[np.array([alpha_s]), np.array([alpha_p])],
                   coef=[np.array([1.0]), np.array([1.0])], **base)


def toy_params(elements, **kw):
    p = Params(elements=elements, **kw)
    return p


def hueckel_like(params):
    """Copy of a table with every H0 modifier switched off: K_AB = 1,
    k_EN = 0, k_poly = 0, k_CN = 0, and k_l = 1.75 for all l."""
    q = copy.deepcopy(params)
    q.k_l = (1.75, 1.75, 1.75)
    q.k_en = 0.0
    q.k_ab_special = {}
    for el in q.elements.values():
        el.k_poly_l = [0.0] * len(el.shells_l)
        el.k_cn_l = [0.0] * len(el.shells_l)
    return q
