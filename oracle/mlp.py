"""FP64 CPU oracle of the learned initial-charge model (row a14 / config C5).

TEST INFRASTRUCTURE ONLY (see oracle/xtb.py).  The paper has no learned
guess; this is the plain definition of the model the GPU path implements:

  descriptors  per atom, neighbours within RC (6 A) with the cosine cutoff
               fc(r) = (cos(pi r / RC) + 1) / 2:
                 radial   G_{e,k} = sum_{j of element e} exp(-ETA_R (r_ij - RS_k)^2) fc(r_ij)
                          (4 elements x 8 centres RS_k)
                 angular  G_{p,t} = 2^(1-zeta) sum_{j<k, {e_j,e_k} = p} (1 + lambda cos theta_jik)^zeta
                                    exp(-ETA_A (r_ij^2 + r_ik^2)) fc(r_ij) fc(r_ik)
                          (10 unordered element pairs x (lambda, zeta) in
                          (+1,1), (-1,1), (+1,4), (-1,4))
                 ESP      the embedding potential at the atom from the other
                          fragments' shell charges (Eq. 21 with gamma of the
                          atom's first shell)
                 one-hot  element (H, C, N, O)
               77 features; standardised with a stored mean and scale
  model        77 -> 128 -> 128 -> 2, SiLU after the hidden layers; the two
               outputs are the atom's two shell charges
  neutrality   each fragment's shell charges shifted by a common amount so
               that they sum to minus the fragment charge
  two passes   (READING C-16) pass 0 with ESP = 0, pass 1 with the ESP of the
               pass-0 charges
  loss         mean squared error against converged monomer shell charges
  Adam         Kingma & Ba 2015, beta1 0.9, beta2 0.999, eps 1e-8
Distances in angstrom inside the descriptors.
"""
from __future__ import annotations

import numpy as np

from . import xtb

ELEMENTS = (1, 6, 7, 8)
RC = 6.0
ETA_R = 1.0 / (2.0 * 0.5 ** 2)
RS = 0.8 + np.arange(8) * (RC - 0.8) / 7.0
ETA_A = 0.02
ANG_TERMS = ((1.0, 1.0), (-1.0, 1.0), (1.0, 4.0), (-1.0, 4.0))
PAIRS = tuple((a, b) for a in range(4) for b in range(a, 4))
N_FEAT = 4 * len(RS) + len(PAIRS) * len(ANG_TERMS) + 1 + 4
HIDDEN = 128
BOHR_PER_A = 1.0 / 0.529177210903


def cutoff(r):
    return np.where(r < RC, 0.5 * (np.cos(np.pi * r / RC) + 1.0), 0.0)


def geometric_features(Z, xyz_bohr):
    """Radial and angular descriptors and the element one-hot (N x 76)."""
    x = np.asarray(xyz_bohr, dtype=np.float64) / BOHR_PER_A
    el = np.array([ELEMENTS.index(int(z)) for z in Z])
    n = len(Z)
    out = np.zeros((n, N_FEAT - 1))
    nrad = 4 * len(RS)
    for i in range(n):
        d = x - x[i]
        r = np.sqrt((d ** 2).sum(1))
        nb = np.nonzero((r < RC) & (np.arange(n) != i))[0]
        for j in nb:
            out[i, el[j] * len(RS):(el[j] + 1) * len(RS)] += np.exp(-ETA_R * (r[j] - RS) ** 2) * cutoff(r[j])
        for a in range(len(nb)):
            j = nb[a]
            for b in range(a + 1, len(nb)):
                k = nb[b]
                cos = d[j] @ d[k] / (r[j] * r[k])
                w = np.exp(-ETA_A * (r[j] ** 2 + r[k] ** 2)) * cutoff(r[j]) * cutoff(r[k])
                p = PAIRS.index((min(el[j], el[k]), max(el[j], el[k])))
                for t, (lam, zeta) in enumerate(ANG_TERMS):
                    out[i, nrad + p * len(ANG_TERMS) + t] += 2.0 ** (1.0 - zeta) * (1.0 + lam * cos) ** zeta * w
        out[i, N_FEAT - 5 + el[i]] = 1.0
    return out


def esp_feature(system, params, shell_dq):
    """Embedding potential at every atom (its first shell's hardness) from the
    shell charges of all other fragments (Eq. 21)."""
    b = xtb.make_basis(system.Z, params)
    eta = xtb.shell_hardness(system.Z, b, params)
    first = np.array([np.nonzero(b.sh_atom == a)[0][0] for a in range(len(system.Z))])
    sh_frag = system.frag[b.sh_atom]
    pos = system.xyz[b.sh_atom]
    g = xtb.gamma_between(system.xyz, eta[first], pos, eta, params.k_g)      # atoms x shells
    other = system.frag[:, None] != sh_frag[None, :]
    return (g * other) @ shell_dq


def features(system, params, shell_dq_for_esp=None):
    geo = geometric_features(system.Z, system.xyz)
    esp = np.zeros(len(system.Z)) if shell_dq_for_esp is None else esp_feature(system, params, shell_dq_for_esp)
    return np.concatenate([geo[:, :N_FEAT - 5], esp[:, None], geo[:, N_FEAT - 5:]], axis=1)


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    w = lambda fi, fo: rng.normal(0.0, np.sqrt(1.0 / fi), size=(fo, fi))
    return {"W1": w(N_FEAT, HIDDEN), "b1": np.zeros(HIDDEN), "W2": w(HIDDEN, HIDDEN), "b2": np.zeros(HIDDEN),
            "W3": w(HIDDEN, 2) * 0.1, "b3": np.zeros(2), "mean": np.zeros(N_FEAT), "scale": np.ones(N_FEAT)}


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def forward(p, X):
    """Per-atom outputs (N x 2) and the cache for backward."""
    x0 = (X - p["mean"]) * p["scale"]
    z1 = x0 @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x0, z1, h1, z2, h2)


def project(y, frag, frag_charge):
    """Shell charges (atom-major, 2 per atom) with each fragment summing to
    minus its charge (a common shift over the fragment's shells)."""
    q = y.reshape(-1).copy()
    sf = np.repeat(frag, 2)
    for f in range(len(frag_charge)):
        m = sf == f
        q[m] -= (q[m].sum() + frag_charge[f]) / m.sum()
    return q


def loss_and_grad(p, X, frag, frag_charge, target):
    """Mean squared error of the projected shell charges and its gradient with
    respect to every weight (the projection is linear and self-adjoint)."""
    y, (x0, z1, h1, z2, h2) = forward(p, X)
    q = project(y, frag, frag_charge)
    r = q - target
    L = float(r @ r) / len(r)
    gq = 2.0 * r / len(r)
    gy = project(gq.reshape(-1, 2), frag, np.zeros(len(frag_charge))).reshape(-1, 2)
    g = {"W3": gy.T @ h2, "b3": gy.sum(0)}
    gz2 = (gy @ p["W3"]) * dsilu(z2)
    g["W2"], g["b2"] = gz2.T @ h1, gz2.sum(0)
    gz1 = (gz2 @ p["W2"]) * dsilu(z1)
    g["W1"], g["b1"] = gz1.T @ x0, gz1.sum(0)
    return L, g


def adam_step(p, g, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of the weights named in g."""
    for k in g:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] ** 2
        p[k] = p[k] - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)


def predict(p, system, params, geo=None):
    """Two-pass prediction (READING C-16): shell charges of every monomer."""
    X = features(system, params) if geo is None else geo
    q0 = project(forward(p, X)[0], system.frag, system.frag_charge)
    X1 = X.copy()
    X1[:, N_FEAT - 5] = esp_feature(system, params, q0)
    return project(forward(p, X1)[0], system.frag, system.frag_charge)
