"""Failure paths of fmo_run on the GPU, each made to fire without faulting or
hanging anything: every wait in the kernels is bounded by an iteration count
or the run's deadline, and the bad input is a value (a deadline of 1 ns, one
SCC iteration, NaN charges, a learned model that predicts NaN).  Also the
pair-by-pair ESP kernel that replaces the stored gamma matrix when it does not
fit in device memory (options.esp_mode)."""
import numpy as np
import pytest

from oracle import fmo as ofmo

pytestmark = pytest.mark.gpu

STATUS_TIMEOUT, STATUS_NOT_CONVERGED, STATUS_NAN = 5, 4, 6
SCC_TIMEOUT, SCC_MAX_ITER = 3, 1


@pytest.fixture(scope="module")
def gpu(params):
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo.FMO(params, 0)


def _run_status(gpu, **kw):
    from paper_2606_28022_b300 import fmo
    try:
        gpu.run(fmo.options(**kw))
        return 0
    except fmo.FMOError as e:
        return e.status


def test_deadline_stops_the_kernels_with_a_timeout(gpu, water64):
    # nested monomer loop: every monomer SCC checks the deadline after each
    # iteration (the device timer against the run's start stamp)
    gpu.set_system(water64.subsystem(range(8)))
    st = _run_status(gpu, monomer_loop="nested", all_dimers_scc=1, deadline_s=1e-9, max_outer=3)
    assert st == STATUS_TIMEOUT
    mono = gpu.monomers()                       # results stay readable
    assert (mono.status == SCC_TIMEOUT).all()
    assert (mono.iters == 1).all()


def test_one_scc_iteration_is_not_converged_but_readable(gpu, water64):
    gpu.set_system(water64.subsystem(range(8)))
    st = _run_status(gpu, all_dimers_scc=1, max_iter=1)
    assert st == STATUS_NOT_CONVERGED
    e1, e2, _ = gpu.energies()
    assert np.isfinite(e1) and np.isfinite(e2)
    d = gpu.dimers()
    assert (d.iters[d.scc] == 1).all()
    assert np.isfinite(d.dE).all()


def test_nan_start_charges_give_a_nan_status(gpu, water64):
    s = water64.subsystem(range(6))
    gpu.set_system(s)
    n_sh, _ = gpu.sizes()
    gpu.set_guess(np.full(n_sh, np.nan))
    assert _run_status(gpu, guess=2) == STATUS_NAN
    gpu.run()                                   # the context stays usable
    assert np.isfinite(gpu.energies()[1])


def test_failed_learned_guess_restarts_from_neutral(gpu, water64):
    from paper_2606_28022_b300 import fmo
    s = water64.subsystem(range(8))
    gpu.set_system(s)
    gpu.run(fmo.options())
    ref = gpu.energies()
    assert gpu.stats()["guess_restarts"] == 0
    gpu.mlp_init(3)
    w = gpu.mlp_get_weights()
    w[:] = np.nan                               # a model whose every prediction is NaN
    gpu.mlp_set_weights(w)
    gpu.run(fmo.options(guess=1))
    assert gpu.stats()["guess_restarts"] == 1
    assert gpu.energies()[:2] == ref[:2]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pairwise_esp_matches_the_stored_gamma_and_the_oracle(gpu, params, water64, prec):
    s = water64.subsystem(range(12))
    gpu.set_system(s)
    from paper_2606_28022_b300 import fmo
    gpu.run(fmo.options(precision=prec))
    e_auto = gpu.energies()
    dq_auto = gpu.monomers().shell_dq.copy()
    gpu.run(fmo.options(precision=prec, esp_mode="pairwise"))
    e_pair = gpu.energies()
    assert abs(e_pair[1] - e_auto[1]) < 1e-9
    assert np.max(np.abs(gpu.monomers().shell_dq - dq_auto)) < 1e-9
    if prec == "fp64":
        ref = ofmo.fmo(s, params, ofmo.FMOOptions())
        assert abs(e_pair[1] - ref.e_fmo2) < 1e-7
        assert np.max(np.abs(gpu.dimers().dE - ref.dE_dimer)) < 1e-8
