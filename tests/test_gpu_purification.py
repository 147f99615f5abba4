"""SP2 purification on the device (fmo_sp2_projector, fmo_sp2_projector_f32)
against the oracle's occupied-subspace projector, element by element, in FP64
and FP32: one tile, ragged tails over several tiles, the trimer size of the
pentacene workload, empty and full occupation, and the reported failures
(n_occ out of range, no gap)."""
import numpy as np
import pytest

from oracle import purification as pu

pytestmark = pytest.mark.gpu

TOL = 1e-10   # FP64 products: SP2 reaches an idempotent matrix to ~1e-13


def _gapped(n, n_occ, rng, gap=0.2):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    e = np.sort(rng.uniform(-1.0, 1.0, n))
    e[n_occ:] += gap
    F = (Q * e) @ Q.T
    return 0.5 * (F + F.T)


def _run(Fs, occ, max_iter=100, fp32=False):
    import torch
    from paper_2606_28022_b300 import build, fmo
    build.build()
    batch, n = len(Fs), Fs[0].shape[0]
    F = torch.tensor(np.stack(Fs), dtype=torch.float32 if fp32 else torch.float64, device="cuda")
    o = torch.tensor(np.asarray(occ, dtype=np.int32), device="cuda")
    D = torch.empty_like(F)
    W = torch.empty_like(F)
    it = torch.full((batch,), 12345, dtype=torch.int32, device="cuda")
    fmo.sp2_projector(F.data_ptr(), o.data_ptr(), n, batch, max_iter, D.data_ptr(), W.data_ptr(),
                      it.data_ptr(), torch.cuda.current_stream().cuda_stream, fp32=fp32)
    torch.cuda.synchronize()
    return D.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("n", [16, 76, 152, 348])
def test_sp2_equals_occupied_projector(n):
    rng = np.random.default_rng(n)
    occ = [0, n // 3, n // 2, n]
    Fs = [_gapped(n, k, rng) for k in occ]
    D, it = _run(Fs, occ)
    assert np.all(it > 0), it
    for b, k in enumerate(occ):
        ref = pu.occupied_projector(Fs[b], k)
        assert np.max(np.abs(D[b] - ref)) < TOL, (n, k, np.max(np.abs(D[b] - ref)))
        assert abs(np.trace(D[b]) - k) < 1e-10


def test_sp2_reports_bad_occupation_and_missing_gap():
    n = 40
    rng = np.random.default_rng(1)
    Fs = [_gapped(n, 10, rng), _gapped(n, 10, rng), 0.3 * np.eye(n), _gapped(n, 10, rng)]
    D, it = _run(Fs, [-1, n + 1, 20, 10], max_iter=60)
    assert it[0] == -2 and it[1] == -2
    assert it[2] == -1                      # F = c I: no gap at n_occ = 20
    assert it[3] > 0
    assert np.max(np.abs(D[3] - pu.occupied_projector(Fs[3], 10))) < TOL


TOL32 = 2e-4   # FP32 products: rounding of ~n * 6e-8 per step, amplified by 1/gap


@pytest.mark.parametrize("n", [16, 76, 152, 348])
def test_sp2_fp32_equals_occupied_projector_of_the_rounded_matrix(n):
    rng = np.random.default_rng(1000 + n)
    occ = [0, n // 3, n // 2, n]
    Fs = [_gapped(n, k, rng).astype(np.float32) for k in occ]
    D, it = _run(Fs, occ, fp32=True)
    assert D.dtype == np.float32
    assert np.all(it > 0), it
    for b, k in enumerate(occ):
        ref = pu.occupied_projector(Fs[b].astype(np.float64), k)
        err = np.max(np.abs(D[b].astype(np.float64) - ref))
        assert err < TOL32, (n, k, err)
        assert abs(np.trace(D[b].astype(np.float64)) - k) < 1e-3
