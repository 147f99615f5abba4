"""Host logic of the FMO-xTB MD driver: the velocity-Verlet integrator against
the closed-form discrete solution of the harmonic oscillator, time
reversibility, the charge extrapolation's exactness on polynomials and its
conservation of fragment charges, and the Maxwell–Boltzmann start."""
import numpy as np
import pytest

from paper_2606_28022_b300 import md


def test_verlet_harmonic_equals_discrete_closed_form():
    # x'' = -w^2 x from rest: velocity Verlet's positions obey
    # x[n+1] - 2x[n] + x[n-1] = -(w h)^2 x[n], whose solution with v0 = 0 is
    # x[n] = x0 cos(n theta), cos(theta) = 1 - (w h)^2 / 2
    k, mass, h, n = 2.5, 3.0, 0.3, 200
    w = np.sqrt(k / mass)
    x0 = np.array([[0.7, -1.1, 0.2]])

    def ef(x):
        return 0.5 * k * float(np.sum(x * x)), -k * x
    xs, vs, es = md.velocity_verlet(ef, x0, np.zeros_like(x0), np.array([mass]), h, n)
    theta = np.arccos(1.0 - 0.5 * (w * h) ** 2)
    exact = x0[None] * np.cos(theta * np.arange(n + 1))[:, None, None]
    assert np.max(np.abs(xs - exact)) < 1e-12
    # v[n] = (x[n+1] - x[n]) / h - (h / 2) a[n]; the cos(n theta) terms cancel,
    # leaving v[n] = -x0 sin(theta) sin(n theta) / h
    #              = -x0 w sqrt(1 - (w h / 2)^2) sin(n theta)
    vexact = -x0[None] * (w * np.sqrt(1 - 0.25 * (w * h) ** 2)) * np.sin(theta * np.arange(n + 1))[:, None, None]
    assert np.max(np.abs(vs - vexact)) < 1e-12


def test_verlet_time_reversible_on_anharmonic_potential():
    rng = np.random.default_rng(3)
    x0 = rng.standard_normal((5, 3))
    v0 = rng.standard_normal((5, 3)) * 0.1
    m = rng.uniform(1.0, 4.0, 5)

    def ef(x):   # quartic pair potential
        d = x[:, None] - x[None]
        r2 = np.sum(d * d, -1)
        E = 0.25 * np.sum(np.triu(r2 * r2 * 0.01, 1)) + 0.5 * np.sum(x * x)
        F = -(0.01 * np.sum(r2[..., None] * d, 1) + x)
        return E, F
    # the force is the exact negative gradient (checked by central differences)
    e = 1e-6
    g = np.zeros_like(x0)
    for i in range(5):
        for c in range(3):
            xp, xm = x0.copy(), x0.copy()
            xp[i, c] += e
            xm[i, c] -= e
            g[i, c] = (ef(xp)[0] - ef(xm)[0]) / (2 * e)
    assert np.max(np.abs(g + ef(x0)[1])) < 1e-7
    xs, vs, es = md.velocity_verlet(ef, x0, v0, m, 0.05, 100)
    xb, vb, _ = md.velocity_verlet(ef, xs[-1], -vs[-1], m, 0.05, 100)
    assert np.max(np.abs(xb[-1] - x0)) < 1e-11
    assert np.max(np.abs(vb[-1] + v0)) < 1e-11
    ek = np.array([md.kinetic_energy(m, v) for v in vs])
    etot = es + ek
    assert np.max(np.abs(etot - etot[0])) < 1e-3 * (ek.max() - ek.min())


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_extrapolation_exact_on_polynomials_and_keeps_charge(order):
    c = md.extrapolation_coefficients(order)
    assert abs(c.sum() - 1.0) < 1e-15          # fragment charges kept
    rng = np.random.default_rng(order)
    coef = rng.standard_normal((order + 1, 6))
    t = np.arange(order + 1, dtype=np.float64)
    q = [sum(coef[p] * ti ** p for p in range(order + 1)) for ti in t]
    nxt = sum(coef[p] * (order + 1.0) ** p for p in range(order + 1))
    assert np.allclose(md.extrapolate(q, order), nxt, atol=1e-12, rtol=0)
    # one degree higher is not reproduced (unless order is large enough)
    qq = [x + ti ** (order + 1) for x, ti in zip(q, t)]
    assert not np.allclose(md.extrapolate(qq, order), nxt + (order + 1.0) ** (order + 1))


def test_extrapolation_falls_back_to_available_history():
    h = [np.array([1.0, -1.0])]
    assert np.array_equal(md.extrapolate(h, 2), h[0])
    h.append(np.array([2.0, -2.0]))
    assert np.allclose(md.extrapolate(h, 2), [3.0, -3.0])
    with pytest.raises(ValueError):
        md.extrapolate([], 1)


def test_maxwell_boltzmann_start():
    m = md.masses([8, 1, 1] * 10)
    v = md.maxwell_boltzmann(m, 300.0, seed=5)
    assert np.max(np.abs((m[:, None] * v).sum(0))) < 1e-12
    T = 2 * md.kinetic_energy(m, v) / ((3 * len(m) - 3) * md.KB_HARTREE)
    assert abs(T - 300.0) < 1e-9
    with pytest.raises(ValueError):
        md.masses([118])


def test_units():
    # 1 a.u. of time is 24.188843 as; an O-H stretch period (~9 fs) is ~370 a.u.
    assert abs(1.0 / md.FS_IN_AU - 0.0241888433) < 1e-9
    assert abs(md.masses([1])[0] - 1.008 * 1822.888486) < 1e-6


class _FakeFMO:
    """Stand-in context: E = |x|^2 / 2 with converged charges linear in x; the
    monomer loop takes 1 step from a guess within 1e-6 of them, else 11."""

    def __init__(self):
        from paper_2606_28022_b300 import fmo
        self.Monomers = fmo.Monomers
        self.guess = None
        self.guesses = []

    def set_system(self, s):
        self.n = s.n_atoms

    def set_coordinates(self, x):
        self.x = np.asarray(x).reshape(-1, 3).copy()

    def set_guess(self, dq):
        self.guess = np.asarray(dq).copy()

    def run(self, o):
        q = self._q()
        start = self.guess if o.guess == 2 else np.zeros_like(q)
        self.guesses.append((int(o.guess), start))
        self.outer = 1 if np.max(np.abs(start - q)) < 1e-6 else 11
        self.guess = None

    def _q(self):
        return np.array([self.x[:, 0].sum(), -self.x[:, 0].sum()])

    def energies(self):
        return 0.0, 0.5 * float(np.sum(self.x ** 2)), float("nan")

    def gradient(self):
        return self.x.copy()

    def monomers(self):
        q = self._q()
        return self.Monomers(np.zeros(2), q, np.zeros(2, np.int32), np.zeros(2, np.int32))

    def stats(self):
        return {"outer_iterations": self.outer}


def test_fmo_md_driver_against_stand_in_context():
    from paper_2606_28022_b300 import fmo
    from paper_2606_28022_b300.inputs.geometry import System
    s = System(Z=np.array([8, 1, 1]), xyz=np.array([[0.0, 0, 0], [1.8, 0, 0], [-0.5, 1.7, 0]]),
               frag=np.zeros(3, np.int32), frag_charge=np.zeros(1, np.int32))
    g = _FakeFMO()
    opts = fmo.options(level=2, precision="fp64")
    run = md.FmoMD(g, s, opts, extrapolation=1)
    v0 = md.maxwell_boltzmann(run.m, 300.0, seed=0)
    t = run.run(v0, 0.5, 6)
    # E = |x|^2 / 2, F = -x: the driver passes the library's gradient with its sign
    xs, vs, es = md.velocity_verlet(lambda x: (0.5 * float(np.sum(x * x)), -x), s.xyz, v0, run.m,
                                    0.5 * md.FS_IN_AU, 6)
    assert np.array_equal(t.xyz, xs) and np.array_equal(t.e_pot, es)
    # step 0 from the options' guess, every later step from the extrapolated
    # charges: order 0 at step 1, order 1 (2 q_n - q_{n-1}) after that
    assert [k for k, _ in g.guesses] == [0] + [2] * 6
    qs = [np.array([x[:, 0].sum(), -x[:, 0].sum()]) for x in xs]
    assert np.array_equal(g.guesses[1][1], qs[0])
    for n in range(2, 7):
        assert np.allclose(g.guesses[n][1], 2 * qs[n - 1] - qs[n - 2], atol=1e-14, rtol=0)
    assert len(t.outer_iterations) == 7
    # no extrapolation: every step from the options' guess
    g2 = _FakeFMO()
    md.FmoMD(g2, s, opts, extrapolation=None).run(v0, 0.5, 3)
    assert [k for k, _ in g2.guesses] == [0] * 4
