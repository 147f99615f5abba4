"""fmo_scc_solve_noalloc, the entry point for callers that cannot allocate
device memory while they run (loops that forbid allocation after start-up,
frameworks whose allocator owns all device memory): its results must equal
those of fmo_run on the same one-fragment system, call after call, although
every call reuses the same fixed scratch array left behind by the previous
one.  With an external shell potential there is no fmo_run counterpart; the
FP64 oracle's SCC in the same potential is the reference there.

Collected last on purpose: if it fails, every other test has already run."""
import ctypes as C

import numpy as np
import pytest

from paper_2606_28022_b300.inputs import geometry as G

pytestmark = pytest.mark.gpu

E_TOL = 1e-8      # Eh, the per-fragment tolerance of the parity tests
DQ_TOL = 1e-7


def _bind(lib):
    f = lib.fmo_scc_solve_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.c_int32, C.c_void_p,
                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_char_p, C.c_int32]
    return f


def _molecules():
    water = G.water_cluster(64, 1).subsystem([7])
    anth, _ = G.anthracene_cluster(128, 2)
    return [("water", water), ("anthracene", anth.subsystem([5])), ("water-again", water)]


def test_noalloc_matches_fmo_run_call_after_call(params):
    torch = pytest.importorskip("torch")
    from paper_2606_28022_b300 import build, fmo
    build.build()
    lib = fmo.load_library()
    solve = _bind(lib)
    cparams = fmo.params_to_c(params)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ref_ctx = fmo.FMO(params, 0)
    for name, mol in _molecules():
        for prec in ("fp64", "mixed"):
            opts = fmo.options(precision=prec)
            # the existing entry point: fmo_run on a one-fragment system
            ref_ctx.set_system(mol)
            ref_ctx.run(opts)
            ref = ref_ctx.monomers()
            # the allocation-free one, on device buffers the caller owns
            Z = np.ascontiguousarray(mol.Z, dtype=np.int32)
            xyz = torch.tensor(mol.xyz, dtype=torch.float64, device=dev).contiguous()
            n_sh = len(ref.shell_dq)
            energy = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            dq = torch.full((n_sh,), float("nan"), dtype=torch.float64, device=dev)
            status = torch.full((1,), -1, dtype=torch.int32, device=dev)
            err = C.create_string_buffer(256)
            stream = torch.cuda.current_stream(dev)
            st = solve(C.byref(cparams), len(Z), Z.ctypes.data_as(C.POINTER(C.c_int32)), xyz.data_ptr(), 0,
                       None, C.byref(opts), energy.data_ptr(), dq.data_ptr(), status.data_ptr(),
                       stream.cuda_stream, err, 256)
            assert st == 0, err.value
            torch.cuda.synchronize(dev)
            assert int(status.item()) == 0, (name, prec)
            tol = E_TOL if prec == "fp64" else 1e-7
            assert abs(float(energy.item()) - float(ref.energy[0])) < tol, (name, prec)
            assert np.max(np.abs(dq.cpu().numpy() - ref.shell_dq)) < DQ_TOL * (1 if prec == "fp64" else 10)
    ref_ctx.close()


def test_noalloc_in_an_external_potential_matches_the_oracle(params):
    # a nonzero potential on every shell (the form of the embedding ESP): the
    # returned energy is the internal one, E_el + E_rep without sum v dq
    torch = pytest.importorskip("torch")
    from oracle import xtb
    from paper_2606_28022_b300 import build, fmo
    build.build()
    lib = fmo.load_library()
    solve = _bind(lib)
    cparams = fmo.params_to_c(params)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    anth, _ = G.anthracene_cluster(128, 2)
    mol = anth.subsystem([9])
    cn = xtb.coordination_numbers(mol.Z, mol.xyz, params)
    n_sh = xtb.make_basis(mol.Z, params).n_sh
    rng = np.random.default_rng(5)
    v = 0.02 * rng.standard_normal(n_sh)
    ref = xtb.scc(mol.Z, mol.xyz, params, cn, esp=v)
    Z = np.ascontiguousarray(mol.Z, dtype=np.int32)
    xyz = torch.tensor(mol.xyz, dtype=torch.float64, device=dev).contiguous()
    esp = torch.tensor(v, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):                       # two calls in a row on the shared scratch
        energy = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        dq = torch.full((n_sh,), float("nan"), dtype=torch.float64, device=dev)
        status = torch.full((1,), -1, dtype=torch.int32, device=dev)
        err = C.create_string_buffer(256)
        st = solve(C.byref(cparams), len(Z), Z.ctypes.data_as(C.POINTER(C.c_int32)), xyz.data_ptr(), 0,
                   esp.data_ptr(), C.byref(fmo.options()), energy.data_ptr(), dq.data_ptr(), status.data_ptr(),
                   stream.cuda_stream, err, 256)
        assert st == 0, err.value
        torch.cuda.synchronize(dev)
        assert int(status.item()) == 0
        assert abs(float(energy.item()) - ref.energy) < E_TOL
        assert np.max(np.abs(dq.cpu().numpy() - ref.dq)) < DQ_TOL


def test_noalloc_rejects_a_molecule_beyond_its_limit(params):
    from paper_2606_28022_b300 import fmo
    lib = fmo.load_library()
    solve = _bind(lib)
    cparams = fmo.params_to_c(params)
    big = G.water_cluster(64, 1).subsystem(range(50))          # 150 atoms > 128
    Z = np.ascontiguousarray(big.Z, dtype=np.int32)
    err = C.create_string_buffer(256)
    opts = fmo.options()
    dummy = C.c_double(0.0)
    st = solve(C.byref(cparams), len(Z), Z.ctypes.data_as(C.POINTER(C.c_int32)), C.addressof(dummy), 0, None,
               C.byref(opts), C.addressof(dummy), C.addressof(dummy), None, None, err, 256)
    assert st == 1 and b"atoms" in err.value
