"""Least-squares STO-nG expansion of Slater shells (basis construction, an input).

GFN1-xTB works in a minimal Slater-type basis (Sec. 2.1 of the paper).  Both the
CUDA path and the oracle take contracted Gaussians, so every Slater shell is
expanded here into n normalised primitive Gaussians of the same angular
momentum by maximising the overlap with the Slater function (the criterion of
Hehre, Stewart and Pople's STO-nG fits).  The fit is done once for zeta = 1; a
Slater exponent zeta then scales the Gaussian exponents by zeta**2 and leaves
the coefficients unchanged.

Conventions (shared with the C header ``fmo_element``):
  * a primitive is normalised on its own:
      s:  (2a/pi)^(3/4)              exp(-a r^2)
      p:  (2a/pi)^(3/4) * 2 sqrt(a)  x exp(-a r^2)
  * ``coef[k]`` multiplies normalised primitive k and the contraction is
    normalised to one.

Nothing here evaluates the method; these routines only build the basis.
"""
from __future__ import annotations

import functools

import numpy as np
from scipy import optimize

# radial quadrature grid for the fit (r in bohr for zeta = 1): logarithmic,
# trapezoid weights in log r
_LOGR = np.linspace(np.log(1e-6), np.log(60.0), 4001)
_R = np.exp(_LOGR)
_W = _R * (_LOGR[1] - _LOGR[0])


def _slater_radial(n: int, r: np.ndarray) -> np.ndarray:
    """Normalised radial Slater function r^(n-1) exp(-r) (zeta = 1)."""
    f = r ** (n - 1) * np.exp(-r)
    return f / np.sqrt(np.sum(_W * r * r * f * f))


def _gauss_radial(l: int, a: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Radial parts r^l exp(-a r^2), each normalised, shape (len(a), len(r))."""
    g = r[None, :] ** l * np.exp(-a[:, None] * r[None, :] ** 2)
    return g / np.sqrt(np.sum(_W * r * r * g * g, axis=1))[:, None]


def _fit_quality(log_a: np.ndarray, n: int, l: int):
    a = np.exp(log_a)
    target = _slater_radial(n, _R)
    g = _gauss_radial(l, a, _R)
    # Gram matrix and projection of the target onto the primitive span
    G = (g * _W * _R * _R) @ g.T
    b = (g * _W * _R * _R) @ target
    c = np.linalg.solve(G + 1e-14 * np.eye(len(a)), b)
    overlap2 = float(b @ c)          # |<target|best approximant>|^2
    return 1.0 - overlap2, c


@functools.lru_cache(maxsize=None)
def sto_ng(n_quantum: int, l: int, n_prim: int = 6) -> tuple[np.ndarray, np.ndarray, float]:
    """Fit a zeta = 1 Slater shell (principal number n_quantum, angular l).

    Returns (alpha, coef_radial, overlap) where alpha are Gaussian exponents,
    coef_radial the coefficients of the normalised radial primitives and
    overlap = <STO|fit>.
    """
    best = None
    for start in range(3):
        rng = np.random.default_rng(100 + start)
        # even-tempered start spread around the Slater function's width
        base = np.log(0.04) + np.arange(n_prim) * (np.log(600.0) / (n_prim - 1))
        x0 = np.sort(base + rng.normal(0.0, 0.2, n_prim))
        res = optimize.minimize(lambda x: np.log(_fit_quality(x, n_quantum, l)[0]), x0,
                                method="BFGS", options={"gtol": 1e-9, "maxiter": 3000})
        if best is None or res.fun < best.fun:
            best = res
    err, c = _fit_quality(best.x, n_quantum, l)
    order = np.argsort(-best.x)
    return np.exp(best.x)[order], c[order], float(np.sqrt(1.0 - err))


def same_centre_overlap(l: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """<g_a|g_b> for normalised primitives of equal l on one centre.

    For s: (2 sqrt(ab)/(a+b))^(3/2); each unit of l adds one power of the
    same ratio.  Used only to normalise and orthogonalise contractions.
    """
    a = np.asarray(a, dtype=np.float64)[:, None]
    b = np.asarray(b, dtype=np.float64)[None, :]
    return (2.0 * np.sqrt(a * b) / (a + b)) ** (1.5 + l)


def normalise(l: int, alpha: np.ndarray, coef: np.ndarray) -> np.ndarray:
    norm2 = coef @ same_centre_overlap(l, alpha, alpha) @ coef
    return coef / np.sqrt(norm2)


def contracted_shell(n_quantum: int, l: int, zeta: float, n_prim: int = 6):
    """STO-nG contraction of a Slater shell with exponent zeta (normalised)."""
    a1, c1, _ = sto_ng(n_quantum, l, n_prim)
    alpha = a1 * zeta * zeta
    # radial-normalised and 3-D-normalised primitives differ only by a constant
    # factor common to all primitives of one l, so the coefficients carry over.
    return alpha, normalise(l, alpha, c1.copy())


def orthogonalise(l: int, alpha_ref, coef_ref, alpha, coef):
    """Gram-Schmidt: remove the same-centre component of (alpha_ref, coef_ref)
    from (alpha, coef) and renormalise.  The result is one contraction over the
    union of both primitive sets."""
    proj = coef_ref @ same_centre_overlap(l, alpha_ref, alpha) @ coef
    a_new = np.concatenate([alpha, alpha_ref])
    c_new = np.concatenate([coef, -proj * coef_ref])
    return a_new, normalise(l, a_new, c_new)
