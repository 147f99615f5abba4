"""Checkpoint / resume (host logic): the blob format, the header hash, and
the resume decisions against a stand-in context that records what it is
asked to do.  No device is used."""
import dataclasses

import numpy as np
import pytest

from paper_2606_28022_b300 import checkpoint as ckp
from paper_2606_28022_b300 import fmo
from paper_2606_28022_b300.inputs.geometry import water_cluster


def _opts(**kw):
    o = fmo.FmoOptions()            # plain struct: no library needed
    o.level, o.precision, o.scc_tol, o.dimer_cut = 2, 1, 1e-8, 4.0
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _arrays():
    rng = np.random.default_rng(0)
    return {"energies": rng.standard_normal(3), "mono_shell_dq": rng.standard_normal(17),
            "mono_status": np.arange(5, dtype=np.int32), "dimer_ij": rng.integers(0, 5, (4, 2)).astype(np.int32),
            "dimer_scc": np.array([1, 0, 1, 1], dtype=np.uint8), "trimer_ijk": np.zeros((0, 3), dtype=np.int32)}


def test_blob_round_trip_keeps_every_array_bit_for_bit():
    a = _arrays()
    ck = ckp.loads(ckp.dumps(3, b"\x07" * 32, a))
    assert ck.level == 3 and ck.header == b"\x07" * 32
    assert sorted(ck.arrays) == sorted(a)
    for k, v in a.items():
        assert ck.arrays[k].dtype == v.dtype and ck.arrays[k].shape == v.shape
        assert np.array_equal(ck.arrays[k], v)


@pytest.mark.parametrize("where", [0, 9, 20, 60, -40, -1])
def test_an_altered_byte_is_detected(where):
    blob = bytearray(ckp.dumps(2, b"\x01" * 32, _arrays()))
    blob[where] ^= 0x40
    with pytest.raises(ckp.CheckpointError):
        ckp.loads(bytes(blob))


@pytest.mark.parametrize("cut", [1, 20, 100, 33])
def test_a_truncated_blob_is_detected(cut):
    blob = ckp.dumps(2, b"\x01" * 32, _arrays())
    with pytest.raises(ckp.CheckpointError):
        ckp.loads(blob[:-cut])


def test_header_hash_sees_the_inputs_of_the_results_only(params):
    s = water_cluster(4, 1)
    h0 = ckp.header_hash(s, params, _opts())
    assert h0 == ckp.header_hash(s, params, _opts())
    # what changes results changes the hash
    xyz = s.xyz.copy()
    xyz[3, 1] += 1e-9
    assert ckp.header_hash(dataclasses.replace(s, xyz=xyz), params, _opts()) != h0
    frag = s.frag.copy()
    frag[0], frag[-1] = frag[-1], frag[0]
    assert ckp.header_hash(dataclasses.replace(s, frag=frag), params, _opts()) != h0
    assert ckp.header_hash(s, dataclasses.replace(params, t_el=301.0), _opts()) != h0
    assert ckp.header_hash(s, params, _opts(scc_tol=1e-9)) != h0
    assert ckp.header_hash(s, params, _opts(precision=0)) != h0
    assert ckp.header_hash(s, params, _opts(dimer_cut=4.5)) != h0
    # speed, start and level do not
    assert ckp.header_hash(s, params, _opts(level=3, guess=2, nmer_ctas_per_sm=2, monomer_matrix_smem=2,
                                            deadline_s=5.0, schedule=1)) == h0


class _Stub:
    """Stand-in for an FMO context: results of a fixed level, and a record
    of the guesses and options it was given."""

    def __init__(self, n_frag=3, n_sh=6):
        self.runs, self.guesses = [], []
        self.n_frag, self.n_sh = n_frag, n_sh
        self.level = 0

    def set_guess(self, dq):
        self.guesses.append(np.array(dq))

    def run(self, o, allow_unconverged=False):
        self.runs.append((o.level, o.guess))
        self.level = o.level

    def energies(self):
        return (-1.0 * self.level, -2.0 * self.level, -3.0 * self.level)

    def monomers(self):
        return fmo.Monomers(np.arange(self.n_frag, dtype=float), np.linspace(-0.1, 0.1, self.n_sh),
                            np.ones(self.n_frag, np.int32), np.zeros(self.n_frag, np.int32))

    def dimers(self):
        return fmo.Dimers(np.array([[0, 1]], np.int32), np.array([0.5]), np.array([-7.0]), np.array([0.0]),
                          np.array([True]), np.array([9], np.int32))

    def trimers(self):
        return fmo.Trimers(np.zeros((0, 3), np.int32), np.zeros(0), np.zeros(0))


def test_resume_decisions(tmp_path, params):
    s = water_cluster(3, 1)
    path = str(tmp_path / "run.ckpt")
    g = _Stub()
    # nothing stored: the run goes ahead as asked and leaves a level-1 checkpoint
    e, how = ckp.run_or_resume(g, s, params, _opts(level=1), path)
    assert how is None and g.runs == [(1, 0)] and ckp.load(path).level == 1
    # a higher level: the monomer charges of the checkpoint start the loop
    e, how = ckp.run_or_resume(g, s, params, _opts(level=2), path)
    assert how == "monomers" and g.runs[-1] == (2, 2)
    assert np.array_equal(g.guesses[-1], g.monomers().shell_dq)
    ck = ckp.load(path)
    assert ck.level == 2 and np.array_equal(ck.arrays["dimer_ij"], [[0, 1]])
    # covered: the stored results come back and nothing runs
    n = len(g.runs)
    e2, how = ckp.run_or_resume(g, s, params, _opts(level=1, nmer_ctas_per_sm=2), path)
    assert how == "complete" and len(g.runs) == n and e2 == ck.energies
    # another geometry: refused
    xyz = s.xyz + 0.01
    with pytest.raises(ckp.CheckpointMismatch):
        ckp.run_or_resume(g, dataclasses.replace(s, xyz=xyz), params, _opts(level=2), path)
    assert len(g.runs) == n
