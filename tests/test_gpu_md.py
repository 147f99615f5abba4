"""FMO-xTB molecular dynamics on the device: velocity Verlet on the FMO2
energy and analytic gradient of six waters conserves the total energy, and
starting each step's monomer loop from the extrapolated charges of the earlier
steps gives the same trajectory in fewer monomer-loop steps than starting it
from neutral charges."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu(params):
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo.FMO(params, 0)


# mixed precision: FP32 monomer-loop steps hand over to FP64 ones, and the
# dimers converge in FP64 (want_gradient), so both forms reach the same fixed
# point; the mixed one to its FP64 tolerance through a different path
@pytest.mark.parametrize("precision,tol_x,tol_e", [("fp64", 1e-7, 1e-8), ("mixed", 1e-6, 1e-7)])
def test_fmo2_md_conserves_energy_and_extrapolation_saves_steps(gpu, water64, precision, tol_x, tol_e):
    from paper_2606_28022_b300 import fmo, md
    s = water64.subsystem(range(6))
    opts = fmo.options(level=2, precision=precision, all_dimers_scc=1)
    v0 = md.maxwell_boltzmann(md.masses(s.Z), 300.0, seed=1)
    n_steps, dt_fs = 12, 0.25

    run_x = md.FmoMD(gpu, s, opts, extrapolation=1)
    tx = run_x.run(v0, dt_fs, n_steps)
    run_0 = md.FmoMD(gpu, s, opts, extrapolation=None)
    t0 = run_0.run(v0, dt_fs, n_steps)

    # same trajectory: both start every monomer loop from a different guess
    # but converge it to the same fixed point
    assert np.max(np.abs(tx.xyz - t0.xyz)) < tol_x
    assert np.max(np.abs(tx.e_pot - t0.e_pot)) < tol_e
    # the guess carried across steps shortens the monomer loop
    assert tx.outer_iterations[1:].sum() < t0.outer_iterations[1:].sum()
    # velocity Verlet with the analytic gradient conserves E_pot + E_kin up to
    # its O(h^2) oscillation, small against the exchange of kinetic energy
    ek_range = tx.e_kin.max() - tx.e_kin.min()
    assert ek_range > 0
    assert np.max(np.abs(tx.e_total - tx.e_total[0])) < 0.05 * ek_range
    print(f"{precision}: E_kin range {ek_range:.3e} Eh, |dE_tot| max {np.max(np.abs(tx.e_total - tx.e_total[0])):.3e} Eh, "
          f"monomer-loop steps {tx.outer_iterations.tolist()} vs {t0.outer_iterations.tolist()}")
