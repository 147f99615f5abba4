"""The C ABI library loads and exports every entry point include/fmo_xtb.h
declares, and the Python structures have the C layout (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmo_xtb.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo.load_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(fmo_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fmo_\w+)", out))
    assert set(names) <= exported


def test_struct_layout_matches_c(tmp_path):
    from paper_2606_28022_b300 import fmo
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "fmo_xtb.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(fmo_element), sizeof(fmo_params),'
                   ' sizeof(fmo_options), sizeof(fmo_stats), offsetof(fmo_params, k_ab),'
                   ' offsetof(fmo_options, dimer_cut) + 1000 * offsetof(fmo_options, mixed_finish)'
                   ' + 1000000 * offsetof(fmo_options, nmer_finish));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [C.sizeof(fmo.FmoElement), C.sizeof(fmo.FmoParams), C.sizeof(fmo.FmoOptions),
                    C.sizeof(fmo.FmoStats), fmo.FmoParams.k_ab.offset,
                    fmo.FmoOptions.dimer_cut.offset + 1000 * fmo.FmoOptions.mixed_finish.offset
                    + 1000000 * fmo.FmoOptions.nmer_finish.offset]


def test_defaults_and_argument_errors(lib):
    from paper_2606_28022_b300 import fmo
    o = fmo.options()
    assert o.level == 2 and o.precision == fmo.PREC_FP64
    assert abs(o.dimer_cut - 4.0 / 0.529177210903) < 1e-12
    assert lib.fmo_create(None, None, 0) == 1                     # FMO_ERR_ARG
    assert lib.fmo_run(None, None, None) == 1
    assert lib.fmo_get_energy(None, None, None, None) == 1
    assert lib.fmo_get_gradient(None, None) == 1
    lib.fmo_destroy(None)                                       # allowed


def test_no_cpu_fallback_without_a_gpu(lib, params):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2606_28022_b300 import fmo
    with pytest.raises(fmo.FMOError) as e:
        fmo.FMO(params)
    assert e.value.status == 2                                  # FMO_ERR_CUDA


def test_sp2_projector_argument_errors_need_no_gpu(lib):
    # sizes are checked before any CUDA call; batch 0 launches nothing
    f = lib.fmo_sp2_projector
    assert f(None, None, 0, 1, 10, None, None, None, None) == 1          # n < 1
    assert f(None, None, 2049, 1, 10, None, None, None, None) == 1       # n > FMO_SP2_MAX_N
    assert f(None, None, 8, -1, 10, None, None, None, None) == 1         # batch < 0
    assert f(None, None, 8, 1, 0, None, None, None, None) == 1           # max_iter < 1
    assert f(None, None, 8, 1, 10, None, None, None, None) == 1          # NULL pointers
    assert f(None, None, 8, 0, 10, None, None, None, None) == 0          # empty batch
    g = lib.fmo_sp2_projector_f32
    assert g(None, None, 0, 1, 10, None, None, None, None) == 1
    assert g(None, None, 8, 1, 10, None, None, None, None) == 1
    assert g(None, None, 8, 0, 10, None, None, None, None) == 0
