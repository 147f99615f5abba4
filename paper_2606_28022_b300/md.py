"""FMO-xTB Born–Oppenheimer molecular dynamics on the GPU FMO energy and gradient.

The paper's stated aim for FMO-xTB is molecular dynamics of large systems, which
needs the energy and the fully analytic gradient (explicit plus response terms)
at every step (Conclusion and outlook; Results, gradient timings).  This module
is the host-side driver of that use:

* velocity Verlet in atomic units (positions in bohr, time in atomic units,
  masses in electron masses), one `fmo_run` + `fmo_get_gradient` per step;
* the initial monomer charges of step n+1 extrapolated from the converged
  charges of the last k+1 steps by the order-k polynomial through them
  (order 0: the previous step's charges).  Every coefficient set sums to one,
  so each fragment's total charge is kept exactly;
* Maxwell–Boltzmann initial velocities with the centre-of-mass motion removed
  and rescaled to the requested temperature.

All arithmetic of the step (integrals, SCC, FMO sums, gradient) runs in the
library's CUDA kernels; this file only moves coordinates, charges and forces.
"""
from __future__ import annotations

import dataclasses
from math import comb

import numpy as np

from . import fmo

AMU_IN_ME = 1822.888486209          # unified atomic mass unit / electron mass (CODATA 2018)
FS_IN_AU = 41.341373335             # 1 fs in atomic units of time (1 a.u. = 0.0241888 fs)
KB_HARTREE = 3.166811563e-6         # Boltzmann constant, Eh/K

# standard atomic weights (IUPAC, conventional values), amu
_MASS_AMU = {1: 1.008, 2: 4.0026, 3: 6.94, 5: 10.81, 6: 12.011, 7: 14.007, 8: 15.999,
             9: 18.998, 11: 22.990, 14: 28.085, 15: 30.974, 16: 32.06, 17: 35.45}


def masses(Z) -> np.ndarray:
    """Atomic masses in electron masses for atomic numbers Z."""
    try:
        return np.array([_MASS_AMU[int(z)] for z in Z]) * AMU_IN_ME
    except KeyError as e:
        raise ValueError(f"no mass for element Z={e.args[0]}") from None


def extrapolation_coefficients(order: int) -> np.ndarray:
    """c[j] multiplying the charges of j steps back (j = 0 newest) so that
    sum_j c[j] q(t-j) is the value at t+1 of the order-`order` polynomial
    through the last order+1 points: c[j] = (-1)^j binom(order+1, j+1)."""
    if order < 0:
        raise ValueError("order must be >= 0")
    return np.array([(-1) ** j * comb(order + 1, j + 1) for j in range(order + 1)], dtype=np.float64)


def extrapolate(history, order: int) -> np.ndarray:
    """Charge guess for the next step from history (oldest first).  With fewer
    than order+1 entries the highest order they support is used."""
    if not history:
        raise ValueError("empty history")
    k = min(order, len(history) - 1)
    c = extrapolation_coefficients(k)
    return sum(c[j] * history[-1 - j] for j in range(k + 1))


def maxwell_boltzmann(m: np.ndarray, temperature_K: float, seed: int) -> np.ndarray:
    """Velocities (n x 3, bohr / a.u. time) drawn at temperature_K, zero total
    momentum, rescaled so that the kinetic temperature with 3N-3 degrees of
    freedom equals temperature_K exactly."""
    m = np.asarray(m, dtype=np.float64)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((len(m), 3)) * np.sqrt(KB_HARTREE * temperature_K / m)[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    dof = 3 * len(m) - 3
    if dof <= 0 or temperature_K == 0.0:
        return np.zeros_like(v)
    t_now = 2.0 * kinetic_energy(m, v) / (dof * KB_HARTREE)
    return v * np.sqrt(temperature_K / t_now)


def kinetic_energy(m: np.ndarray, v: np.ndarray) -> float:
    return 0.5 * float(np.sum(np.asarray(m)[:, None] * v * v))


def velocity_verlet(energy_force, x0, v0, m, dt, n_steps, on_step=None):
    """Integrate x'' = F(x)/m with velocity Verlet.

    energy_force(x) -> (E, F) with F = -dE/dx (n x 3).  Returns arrays of
    positions and velocities (n_steps+1, n, 3) and potential energies
    (n_steps+1,).  on_step(step, x, v, E) is called after each step."""
    m3 = np.asarray(m, dtype=np.float64)[:, None]
    x = np.array(x0, dtype=np.float64)
    v = np.array(v0, dtype=np.float64)
    E, F = energy_force(x)
    xs, vs, es = [x.copy()], [v.copy()], [E]
    for step in range(1, n_steps + 1):
        v = v + (0.5 * dt) * F / m3
        x = x + dt * v
        E, F = energy_force(x)
        v = v + (0.5 * dt) * F / m3
        xs.append(x.copy())
        vs.append(v.copy())
        es.append(E)
        if on_step is not None:
            on_step(step, x, v, E)
    return np.array(xs), np.array(vs), np.array(es)


@dataclasses.dataclass
class Trajectory:
    xyz: np.ndarray               # (n_steps+1, n_atoms, 3) bohr
    vel: np.ndarray               # (n_steps+1, n_atoms, 3) bohr / a.u. time
    e_pot: np.ndarray             # (n_steps+1,) E_FMOn, Eh
    e_kin: np.ndarray             # (n_steps+1,) Eh
    outer_iterations: np.ndarray  # (n_steps+1,) monomer-loop steps of each force call

    @property
    def e_total(self) -> np.ndarray:
        return self.e_pot + self.e_kin


class FmoMD:
    """Velocity Verlet on E_FMOn (options.level) of one library context.

    extrapolation: order of the charge extrapolation across steps (None: every
    step starts from the guess given in opts, e.g. neutral charges)."""

    def __init__(self, g: fmo.FMO, system, opts: fmo.FmoOptions, extrapolation: int | None = 1):
        self.g = g
        self.system = system
        self.opts = type(opts).from_buffer_copy(opts)
        self.opts.want_gradient = 1
        self.extrapolation = extrapolation
        self.m = masses(system.Z)
        self.history: list[np.ndarray] = []
        self.outer: list[int] = []
        g.set_system(system)

    def energy_force(self, x):
        o = type(self.opts).from_buffer_copy(self.opts)
        self.g.set_coordinates(x)
        if self.extrapolation is not None and self.history:
            self.g.set_guess(extrapolate(self.history, self.extrapolation))
            o.guess = 2
        self.g.run(o)
        E = self.g.energies()[self.opts.level - 1]
        F = -self.g.gradient()
        if self.extrapolation is not None:
            self.history.append(self.g.monomers().shell_dq)
            del self.history[:-(self.extrapolation + 1)]
        self.outer.append(int(self.g.stats()["outer_iterations"]))
        return E, F

    def run(self, v0, dt_fs: float, n_steps: int) -> Trajectory:
        self.history.clear()
        self.outer.clear()
        xs, vs, es = velocity_verlet(self.energy_force, self.system.xyz, v0, self.m,
                                     dt_fs * FS_IN_AU, n_steps)
        ek = np.array([kinetic_energy(self.m, v) for v in vs])
        return Trajectory(xs, vs, es, ek, np.array(self.outer))
