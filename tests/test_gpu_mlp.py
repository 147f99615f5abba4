"""Learned initial charges on the GPU against the oracle (oracle/mlp.py):
two-pass prediction with the same (FP16-rounded) weights, the loss and the
weight gradient of the GPU backward kernels, one Adam step, the loss of the
first training epoch, and what the trained guess gains inside fmo_run."""
import numpy as np
import pytest

from oracle import mlp
from paper_2606_28022_b300.inputs import geometry as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu(params):
    from paper_2606_28022_b300 import build, fmo
    build.build()
    return fmo.FMO(params, 0)


def _flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"],
                           p["mean"], p["scale"]]).astype(np.float32)


def _fp16_params(seed, X):
    p = mlp.init_params(seed)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        p[k] = p[k].astype(np.float16).astype(np.float64)
    p["b1"] = (np.random.default_rng(seed + 1).normal(size=128) * 0.1).astype(np.float16).astype(np.float64)
    p["mean"] = X.mean(0).astype(np.float32).astype(np.float64)
    p["scale"] = (1.0 / (X.std(0) + 1.0)).astype(np.float32).astype(np.float64)
    return p


def test_prediction_matches_oracle(gpu, params, water64):
    s = water64.subsystem(range(4))
    X = mlp.features(s, params)
    p = _fp16_params(7, X)
    gpu.set_system(s)
    gpu.mlp_set_weights(_flat(p))
    q = gpu.mlp_predict()
    ref = mlp.predict(p, s, params)
    assert np.max(np.abs(q - ref)) < 1e-4
    for f in range(s.n_frag):
        assert abs(q[np.repeat(s.frag, 2) == f].sum()) < 1e-5


def test_first_epoch_loss_matches_oracle(gpu, params, water64):
    s = water64.subsystem(range(4))
    frames = [G.jittered(s, 0.05, 100 + k) for k in range(2)]
    rng = np.random.default_rng(3)
    targets = rng.normal(size=(2, 2 * s.n_atoms)) * 0.1
    geo = [mlp.features(f, params) for f in frames]
    Xall = np.concatenate(geo)
    p = _fp16_params(11, Xall)
    # the trainer sets the feature statistics from the frames: columns 0-71
    # mean and 1/(std + 1), the potential (0, 10), the one-hot (0, 1)
    p["mean"][:72] = Xall[:, :72].mean(0).astype(np.float32)
    p["scale"][:72] = (1.0 / (Xall[:, :72].std(0) + 1.0)).astype(np.float32)
    p["mean"][72:], p["scale"][72:] = 0.0, np.array([10.0, 1, 1, 1, 1])
    want = np.mean([np.mean((mlp.predict(p, f, params, geo=g) - t) ** 2) for f, g, t in zip(frames, geo, targets)])
    gpu.set_system(s)
    gpu.mlp_set_weights(_flat(p))
    loss = gpu.mlp_train(np.stack([f.xyz for f in frames]), targets, epochs=1, batch_frames=2, lr=1e-3)
    assert abs(loss[0] - want) < 1e-4 * want


def _oracle_loss_grad(p, frames, targets, params):
    """Two-pass training loss (pass-0 potential held fixed) and its gradient,
    averaged over the frames, flat in the GPU weight layout."""
    Ls, gs = [], []
    for f, t in zip(frames, targets):
        X0 = mlp.features(f, params)
        q0 = mlp.project(mlp.forward(p, X0)[0], f.frag, f.frag_charge)
        X1 = X0.copy()
        X1[:, mlp.N_FEAT - 5] = mlp.esp_feature(f, params, q0)
        L, g = mlp.loss_and_grad(p, X1, f.frag, f.frag_charge, t)
        Ls.append(L)
        gs.append(g)
    g = {k: np.mean([x[k] for x in gs], axis=0) for k in gs[0]}
    flat = np.concatenate([g["W1"].ravel(), g["b1"], g["W2"].ravel(), g["b2"], g["W3"].ravel(), g["b3"]])
    return float(np.mean(Ls)), g, flat


def _frames_and_targets(s, n=2, seed=100):
    frames = [G.jittered(s, 0.05, seed + k) for k in range(n)]
    targets = np.random.default_rng(3).normal(size=(n, 2 * s.n_atoms)) * 0.1
    return frames, targets


def test_backward_gradient_matches_oracle(gpu, params, water64):
    s = water64.subsystem(range(4))
    frames, targets = _frames_and_targets(s)
    p = _fp16_params(13, np.concatenate([mlp.features(f, params) for f in frames]))
    gpu.set_system(s)
    gpu.mlp_set_weights(_flat(p))
    loss, g = gpu.mlp_loss_grad(np.stack([f.xyz for f in frames]), targets)
    L, _, gref = _oracle_loss_grad(p, frames, targets, params)
    assert abs(loss - L) < 1e-4 * L
    scale = np.abs(gref).max()
    assert scale > 1e-3
    assert np.max(np.abs(g - gref)) < 2e-3 * scale
    # every layer (W1, W2, W3) on its own
    o = np.cumsum([0, 128 * 77, 128, 128 * 128, 128, 2 * 128, 2])
    for a, b in ((o[0], o[1]), (o[2], o[3]), (o[4], o[5])):
        sc = np.abs(gref[a:b]).max()
        assert np.max(np.abs(g[a:b] - gref[a:b])) < 2e-3 * sc


def test_one_adam_step_matches_oracle(gpu, params, water64):
    s = water64.subsystem(range(4))
    frames, targets = _frames_and_targets(s, seed=300)
    geo = [mlp.features(f, params) for f in frames]
    Xall = np.concatenate(geo)
    p = _fp16_params(17, Xall)
    # the trainer's feature statistics (set from the frames)
    p["mean"][:72] = Xall[:, :72].mean(0).astype(np.float32)
    p["scale"][:72] = (1.0 / (Xall[:, :72].std(0) + 1.0)).astype(np.float32)
    p["mean"][72:], p["scale"][72:] = 0.0, np.array([10.0, 1, 1, 1, 1])
    gpu.set_system(s)
    gpu.mlp_set_weights(_flat(p))
    lr = 1e-3
    gpu.mlp_train(np.stack([f.xyz for f in frames]), targets, epochs=1, batch_frames=len(frames), lr=lr)
    w = gpu.mlp_get_weights()[:26754].astype(np.float64)
    _, g, gflat = _oracle_loss_grad(p, frames, targets, params)
    ref = dict(p)
    mlp.adam_step(ref, {k: g[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3")}, {}, lr, 1)
    wref = np.concatenate([ref["W1"].ravel(), ref["b1"], ref["W2"].ravel(), ref["b2"], ref["W3"].ravel(), ref["b3"]])
    w0 = _flat(p)[:26754].astype(np.float64)
    clear = np.abs(gflat) > 1e-4 * np.abs(gflat).max()       # gradient signs beyond rounding
    assert clear.sum() > 100
    assert np.max(np.abs(w - wref)[clear]) < 1e-6
    assert np.max(np.abs(w - w0)) <= lr * (1 + 1e-5)            # an Adam step moves no weight by more than lr


def test_learned_guess_in_fmo_run(gpu, params, water64):
    from paper_2606_28022_b300 import fmo
    s = water64.subsystem(range(8))
    gpu.set_system(s)
    frames, targets = [], []
    for k in range(6):
        f = G.jittered(s, 0.05, 200 + k)
        gpu.set_coordinates(f.xyz)
        gpu.run(fmo.options(level=1))
        frames.append(f.xyz)
        targets.append(gpu.monomers().shell_dq)
    gpu.mlp_init(5)
    loss = gpu.mlp_train(np.stack(frames), np.stack(targets), epochs=40, batch_frames=2, lr=3e-3)
    assert loss[-1] < 0.5 * loss[0]
    # held-out frames: the same energies, in fewer monomer-loop iterations
    it0_sum = it1_sum = 0
    for k in range(4):
        test = G.jittered(s, 0.05, 999 + k)
        gpu.set_coordinates(test.xyz)
        gpu.run(fmo.options(level=2))
        e0, it0 = gpu.energies(), gpu.stats()["outer_iterations"]
        gpu.run(fmo.options(level=2, guess=1))
        e1, it1 = gpu.energies(), gpu.stats()["outer_iterations"]
        assert abs(e1[1] - e0[1]) < 1e-8 and abs(e1[0] - e0[0]) < 1e-8
        assert (gpu.monomers().status == 0).all()
        assert gpu.stats()["guess_restarts"] == 0
        it0_sum += it0
        it1_sum += it1
    assert it1_sum < it0_sum
