"""Checkpoint / resume on the device: an FMO2 run resumed from the FMO1
checkpoint of the same system equals a direct FMO2 run, its monomer loop ends
after a confirming step, and a covered request returns the stored results
without a launch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu(params):
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo.FMO(params, 0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fmo2_resumed_from_fmo1_equals_direct_run(gpu, params, water64, tmp_path, precision):
    from paper_2606_28022_b300 import checkpoint as ckp
    from paper_2606_28022_b300 import fmo
    s = water64.subsystem(range(16))
    gpu.set_system(s)
    o2 = fmo.options(level=2, precision=precision, all_dimers_scc=1)
    gpu.run(o2)
    e_direct = gpu.energies()
    d_direct = gpu.dimers()
    outer_direct = gpu.stats()["outer_iterations"]

    path = str(tmp_path / f"w16_{precision}.ckpt")
    e1, how = ckp.run_or_resume(gpu, s, params, fmo.options(level=1, precision=precision, all_dimers_scc=1), path)
    assert how is None and ckp.load(path).level == 1
    assert abs(e1[0] - e_direct[0]) < 1e-8
    e2, how = ckp.run_or_resume(gpu, s, params, o2, path)
    assert how == "monomers"
    outer = gpu.stats()["outer_iterations"]
    # from converged charges: FP64 confirms them in one step plus the energy
    # check.  Mixed precision starts with an FP32 step, whose rounding (~1e-6)
    # the FP64 phase then removes from a fresh Broyden history: about half the
    # direct run's steps.
    if precision == "fp64":
        assert outer <= 2 < outer_direct
    else:
        assert outer <= outer_direct // 2 + 1
    d = gpu.dimers()
    assert np.array_equal(d.ij, d_direct.ij)
    assert np.max(np.abs(d.dE - d_direct.dE)) < 1e-8
    assert abs(e2[1] - e_direct[1]) < 1e-8
    # covered by the stored level-2 checkpoint: nothing runs
    runs = gpu.stats()["scc_launches"]
    e3, how = ckp.run_or_resume(gpu, s, params, o2, path)
    assert how == "complete"
    assert np.array_equal(e3, ckp.load(path).energies, equal_nan=True)   # E_FMO3 is NaN at level 2
    assert gpu.stats()["scc_launches"] == runs
    assert e3[1] == e2[1]
