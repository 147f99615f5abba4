"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs.  Tolerances: 1e-8 Eh per fragment energy and 1e-7 Eh for
FMO totals in the FP64 path; 1e-6 Eh for the totals and 1e-7 Eh per dimer and
trimer interaction energy in the mixed path."""
import numpy as np
import pytest

from oracle import fmo as ofmo
from oracle import xtb
from paper_2606_28022_b300.inputs import geometry as G
from paper_2606_28022_b300.inputs.params import ANGSTROM

pytestmark = pytest.mark.gpu

E_FRAG = 1e-8
E_TOT = 1e-7
E_TOT_MIXED = 1e-6
E_NMER_MIXED = 1e-7   # per dimer / trimer energy, mixed path
DQ = 1e-7


@pytest.fixture(scope="module")
def gpu(params):
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo.FMO(params, 0)


def run_gpu(gpu, system, **kw):
    from paper_2606_28022_b300 import fmo
    gpu.set_system(system)
    gpu.run(fmo.options(**kw))
    return gpu


def compare(g, ref, e_tot=E_TOT, e_frag=E_FRAG, dq_tol=DQ, level=2):
    e1, e2, e3 = g.energies()
    mono = g.monomers()
    assert np.max(np.abs(mono.energy - ref.e_mono)) < e_frag
    assert np.max(np.abs(mono.shell_dq - np.concatenate(ref.dq_mono))) < dq_tol
    assert (mono.status == 0).all()
    assert abs(e1 - ref.e_fmo1) < e_tot
    if level >= 2:
        d = g.dimers()
        assert np.array_equal(d.ij, ref.dimers)
        assert np.array_equal(d.scc, ref.dimer_scc)
        assert np.max(np.abs(d.dE - ref.dE_dimer)) < e_frag
        assert abs(e2 - ref.e_fmo2) < e_tot
    if level >= 3:
        t = g.trimers()
        assert np.array_equal(t.ijk, ref.trimers)
        assert np.max(np.abs(t.corr - ref.corr_trimer), initial=0.0) < e_frag
        assert abs(e3 - ref.e_fmo3) < e_tot


def test_water8_fmo2_all_dimers_fp64(gpu, params, water64):
    s = water64.subsystem(range(8))
    ref = ofmo.fmo(s, params, ofmo.FMOOptions(all_dimers_scc=True))
    compare(run_gpu(gpu, s, all_dimers_scc=1), ref)


def test_water8_nested_monomer_loop_fp64(gpu, params, water64):
    s = water64.subsystem(range(8))
    ref = ofmo.fmo(s, params, ofmo.FMOOptions(all_dimers_scc=True, monomer_loop="nested"))
    compare(run_gpu(gpu, s, all_dimers_scc=1, monomer_loop="nested"), ref)


def test_water12_fmo2_esdim_fp64(gpu, params, water64):
    # the 4.0 A rule splits the pairs into SCC dimers and ES-DIM pairs
    s = water64.subsystem(range(12))
    ref = ofmo.fmo(s, params, ofmo.FMOOptions())
    assert ref.dimer_scc.any() and not ref.dimer_scc.all()
    compare(run_gpu(gpu, s), ref)


def test_water5_fmo3_fp64(gpu, params, water64):
    s = water64.subsystem(range(5))
    ref = ofmo.fmo(s, params, ofmo.FMOOptions(level=3, all_dimers_scc=True, trimer_cut=1e9))
    compare(run_gpu(gpu, s, level=3, all_dimers_scc=1, trimer_cut=1e9), ref, level=3)


def test_two_fragments_equal_full_scc_on_gpu(gpu, params, water64):
    s = water64.subsystem([3, 7])
    full = xtb.single_point(s, params)
    g = run_gpu(gpu, s, all_dimers_scc=1)
    assert abs(g.energies()[1] - full.energy) < E_TOT


def test_single_fragment(gpu, params, water64):
    s = water64.subsystem([2])
    iso = xtb.single_point(s, params)
    g = run_gpu(gpu, s)
    e1, e2, _ = g.energies()
    assert abs(e1 - iso.energy) < E_FRAG and abs(e2 - iso.energy) < E_FRAG
    assert g.dimers().ij.shape == (0, 2)


@pytest.fixture(scope="module")
def anthracene4():
    s, _ = G.anthracene_cluster(128, 2)
    # four mutually close molecules of the seeded crystal
    return s.subsystem([0, 1, 2, 3])


def test_anthracene4_fmo2_fp64(gpu, params, anthracene4):
    ref = ofmo.fmo(anthracene4, params, ofmo.FMOOptions(all_dimers_scc=True))
    compare(run_gpu(gpu, anthracene4, all_dimers_scc=1), ref)


def test_anthracene4_fmo2_mixed(gpu, params, anthracene4):
    ref = ofmo.fmo(anthracene4, params, ofmo.FMOOptions(all_dimers_scc=True))
    g = run_gpu(gpu, anthracene4, all_dimers_scc=1, precision="mixed")
    e1, e2, _ = g.energies()
    assert abs(e2 - ref.e_fmo2) < E_TOT_MIXED
    assert abs(e1 - ref.e_fmo1) < E_TOT_MIXED
    d = g.dimers()
    assert np.max(np.abs(d.dE - ref.dE_dimer)) < E_NMER_MIXED             # every dimer on its own


def test_water8_mixed(gpu, params, water64):
    s = water64.subsystem(range(8))
    ref = ofmo.fmo(s, params, ofmo.FMOOptions(all_dimers_scc=True))
    g = run_gpu(gpu, s, all_dimers_scc=1, precision="mixed")
    assert abs(g.energies()[1] - ref.e_fmo2) < E_TOT_MIXED


def test_new_coordinates_same_topology(gpu, params, water64):
    from paper_2606_28022_b300 import fmo
    s = water64.subsystem(range(4))
    s2 = G.jittered(s, 0.05, 77)
    ref = ofmo.fmo(s2, params, ofmo.FMOOptions(all_dimers_scc=True))
    gpu.set_system(s)
    gpu.run(fmo.options(all_dimers_scc=1))
    gpu.set_coordinates(s2.xyz)
    gpu.run(fmo.options(all_dimers_scc=1))
    compare(gpu, ref)


def test_anthracene32_monomer_loop_fp64_and_mixed(gpu, params):
    # a cluster large enough that plain nested monomer iterations converge
    # slowly: the global loop must reach the oracle's fixed point
    from paper_2606_28022_b300 import fmo
    s, _ = G.anthracene_cluster(128, 2)
    s = s.subsystem(range(32))
    ref = ofmo.fmo(s, params, ofmo.FMOOptions(level=1, dimer_cut=0.0))
    gpu.set_system(s)
    gpu.run(fmo.options(level=1))
    mono = gpu.monomers()
    assert np.max(np.abs(mono.energy - ref.e_mono)) < E_FRAG
    assert np.max(np.abs(mono.shell_dq - np.concatenate(ref.dq_mono))) < DQ
    gpu.run(fmo.options(level=1, precision="mixed"))
    assert abs(gpu.energies()[0] - ref.e_fmo1) < E_TOT_MIXED
    # mixed-precision monomers finish in FP64-grade iterations (double-float
    # products on the FP32 pipe): their energies meet the FP64 bar
    assert np.max(np.abs(gpu.monomers().energy - ref.e_mono)) < E_FRAG


def test_anthracene4_mixed_nmer_finish_iterate(gpu, params, anthracene4):
    # the FP64-iteration finish of mixed-precision dimers reaches the same
    # totals as the default FP64 energy of the FP32 density
    ref = ofmo.fmo(anthracene4, params, ofmo.FMOOptions(all_dimers_scc=True))
    g = run_gpu(gpu, anthracene4, all_dimers_scc=1, precision="mixed", nmer_finish="iterate")
    e_it = g.energies()
    assert abs(e_it[1] - ref.e_fmo2) < E_TOT_MIXED
    g = run_gpu(gpu, anthracene4, all_dimers_scc=1, precision="mixed")
    assert abs(g.energies()[1] - e_it[1]) < E_TOT_MIXED


@pytest.fixture(scope="module")
def pentacene4():
    s, _ = G.pentacene_cluster(660, 4)
    # molecule 0 and its three nearest neighbours of the seeded crystal: every
    # pair is an SCC dimer and the trimers have n = 348 basis functions
    return s.subsystem([0, 2, 93, 1])


def test_pentacene4_fmo3_fp64_and_mixed(gpu, params, pentacene4):
    ref = ofmo.fmo(pentacene4, params, ofmo.FMOOptions(level=3))
    assert len(ref.trimers) > 0
    compare(run_gpu(gpu, pentacene4, level=3), ref, level=3)
    g = run_gpu(gpu, pentacene4, level=3, precision="mixed")
    e1, e2, e3 = g.energies()
    assert abs(e3 - ref.e_fmo3) < E_TOT_MIXED
    assert abs(e2 - ref.e_fmo2) < E_TOT_MIXED
    assert np.max(np.abs(g.dimers().dE - ref.dE_dimer)) < E_NMER_MIXED
    t = g.trimers()
    assert np.array_equal(t.ijk, ref.trimers)
    assert np.max(np.abs(t.dE3 - ref.dE_trimer)) < E_NMER_MIXED
    assert np.max(np.abs(t.corr - ref.corr_trimer)) < E_NMER_MIXED


@pytest.fixture(scope="module")
def ala5():
    # five residues of an alpha-helical polyalanine in fragments of 1-3
    # residues, cut at CA-C(O) with hybrid orbital projection
    return G.polyalanine_helix(5, seed=3)


def test_polyalanine_hop_fmo2_fp64(gpu, params, ala5):
    assert len(ala5.cut_bonds) >= 2
    ref = ofmo.fmo(ala5, params, ofmo.FMOOptions(all_dimers_scc=True))
    compare(run_gpu(gpu, ala5, all_dimers_scc=1), ref)


def test_polyalanine_hop_fmo3_of_three_fragments_equals_full_scc(gpu, params):
    s = G.polyalanine_helix(3)
    full = xtb.single_point(s, params)
    g = run_gpu(gpu, s, level=3, all_dimers_scc=1, trimer_cut=1e9)
    assert abs(g.energies()[2] - full.energy) < E_TOT


def test_polyalanine_hop_fmo2_mixed(gpu, params, ala5):
    # mixed precision with cut bonds: the 1e6 Eh projector stays out of the
    # FP32 products (added in the MO basis from its factors)
    ref = ofmo.fmo(ala5, params, ofmo.FMOOptions(all_dimers_scc=True))
    g = run_gpu(gpu, ala5, all_dimers_scc=1, precision="mixed")
    e1, e2, _ = g.energies()
    assert abs(e2 - ref.e_fmo2) < E_TOT_MIXED
    assert abs(e1 - ref.e_fmo1) < E_TOT_MIXED
    assert np.max(np.abs(g.dimers().dE - ref.dE_dimer)) < E_NMER_MIXED
    assert (g.monomers().status == 0).all()


def test_polyalanine_hop_fmo3_three_fragments_mixed_equals_full_scc(gpu, params):
    s = G.polyalanine_helix(3)
    full = xtb.single_point(s, params)
    g = run_gpu(gpu, s, level=3, all_dimers_scc=1, trimer_cut=1e9, precision="mixed")
    assert abs(g.energies()[2] - full.energy) < E_TOT_MIXED


def test_graph_driven_and_host_driven_monomer_loops_agree(gpu, params, water64):
    from paper_2606_28022_b300 import fmo
    s = water64.subsystem(range(12))
    gpu.set_system(s)
    out = []
    for schedule in (0, 1):
        for prec in ("fp64", "mixed"):
            gpu.run(fmo.options(schedule=schedule, precision=prec))
            out.append((gpu.energies(), gpu.monomers().shell_dq.copy(), gpu.stats()["outer_iterations"]))
    for a, b in ((0, 2), (1, 3)):
        assert out[a][0][:2] == out[b][0][:2]          # FMO1, FMO2 (FMO3 is NaN at level 2)
        assert np.array_equal(out[a][1], out[b][1])
        assert out[a][2] == out[b][2]


def test_nmer_schedules_change_speed_not_results(gpu, params, anthracene4):
    # the autotuner's knobs: CTAs per SM (same arithmetic) and the place of the
    # eigen-solve matrix (Jacobi in shared memory or the tridiagonal solver in
    # global memory: the same solution to FP32 rounding)
    from paper_2606_28022_b300 import fmo
    gpu.set_system(anthracene4)
    out = {}
    for c in (0, 1, 2):
        for m in (0, 1, 2):
            gpu.run(fmo.options(all_dimers_scc=1, precision="mixed", nmer_ctas_per_sm=c, nmer_matrix_smem=m))
            out[(c, m)] = (gpu.energies()[1], gpu.dimers().dE.copy())
    ref = ofmo.fmo(anthracene4, params, ofmo.FMOOptions(all_dimers_scc=True))
    for (c, m), (e2, dE) in out.items():
        assert abs(e2 - ref.e_fmo2) < E_TOT_MIXED
        assert np.max(np.abs(dE - ref.dE_dimer)) < E_NMER_MIXED
    for m in (1, 2):
        assert out[(1, m)][0] == out[(2, m)][0]          # one or two CTAs per SM: bit for bit
    with pytest.raises(fmo.FMOError) as e:
        gpu.run(fmo.options(nmer_ctas_per_sm=3))
    assert e.value.status == 1


def test_beyond_512_basis_functions_two_fragments_equal_full_scc(gpu, params):
    # 96 waters in two fragments of 48 (288 basis functions each): the monomers
    # take the tridiagonal solver from global memory, the dimer (576 > 512
    # functions) falls back to Jacobi on a global-memory matrix; FMO2 of two
    # fragments is the full SCC
    w = G.water_cluster(96, 3)
    nat = len(w.Z)
    frag = (np.arange(nat) // (3 * 48)).astype(w.frag.dtype)
    s = G.System(Z=w.Z, xyz=w.xyz, frag=frag, frag_charge=np.zeros(2))
    full = xtb.single_point(s, params)
    for prec, tol in (("fp64", E_TOT), ("mixed", E_TOT_MIXED)):
        g = run_gpu(gpu, s, all_dimers_scc=1, precision=prec)
        assert abs(g.energies()[1] - full.energy) < tol, prec
