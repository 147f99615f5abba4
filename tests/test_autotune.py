"""The schedule autotuner's cache (no GPU needed): keys, lookup, fallback to
the built-in rule."""
import json

import pytest


@pytest.fixture(scope="module")
def mods():
    from paper_2606_28022_b300 import autotune, build, fmo
    build.build()
    return autotune, fmo


def test_cached_choice_and_rule_fallback(mods, tmp_path, water64):
    autotune, fmo = mods
    s = water64.subsystem(range(8))
    key = autotune.size_class(s, 2, "mixed", "DEV")
    assert key == autotune.size_class(s, 2, "mixed", "DEV")            # deterministic
    assert key != autotune.size_class(s, 3, "mixed", "DEV")
    assert key != autotune.size_class(water64, 2, "mixed", "DEV")
    path = tmp_path / "schedules.json"
    o = autotune.options(s, 2, "mixed", path=str(path), device_name="DEV")
    assert (o.nmer_ctas_per_sm, o.nmer_matrix_smem) == (0, 0)           # nothing cached: the rule
    path.write_text(json.dumps({key: {"nmer_ctas_per_sm": 2, "nmer_matrix_smem": 1, "ms": 1.0}}))
    o = autotune.options(s, 2, "mixed", path=str(path), device_name="DEV", all_dimers_scc=1)
    assert (o.nmer_ctas_per_sm, o.nmer_matrix_smem, o.all_dimers_scc, o.level) == (2, 1, 1, 2)
    o = autotune.options(s, 2, "fp64", path=str(path), device_name="DEV")
    assert (o.nmer_ctas_per_sm, o.nmer_matrix_smem) == (0, 0)           # other size class


def test_knob_values_checked(mods, params, water64):
    _, fmo = mods
    lib = fmo.load_library()
    o = fmo.options(nmer_ctas_per_sm=3)
    assert o.nmer_ctas_per_sm == 3           # the library refuses it in fmo_run (FMO_ERR_ARG), GPU test
