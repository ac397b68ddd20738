"""GPU parity of the learned-guess network (own forward / backward kernels)
against the FP64 oracle (oracle/cnn.py), and the gain of the trained guess.

Tolerances: the FP64 path computes the oracle's sums in another order, within
1e-10 relative (its parameters are the oracle's, rounded to FP32 as the
network stores them); the FP32 path within 1e-4 of the largest gradient
entry of each layer (FP32 accumulation over 2 x 16 x 16 points); the BF16
tensor-core inference within 5e-3 of the largest output, against the oracle
run with the same BF16 rounding of the weights and of every layer input (FP32
against FP64 accumulation can move an activation across a BF16 rounding
boundary).
"""
import numpy as np
import pytest

from oracle import cnn
from oracle import bidomain as ob
from workloads import torso_square_2d, params_2d, stimulus_seeded_disc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def bid():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid as b
    return b


def flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflat(v):
    out, o = [], 0
    for cin, cout in cnn.LAYERS:
        nw = cout * cin * 9
        out.append((v[o:o + nw].reshape(cout, cin, 3, 3), v[o + nw:o + nw + cout]))
        o += nw + cout
    return out


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _params(seed):
    rng = np.random.default_rng(seed)
    p = [(W, rng.normal(scale=0.1, size=b.shape)) for W, b in cnn.init_params(seed)]
    return unflat(f32(flat(p)))


@pytest.mark.parametrize("shape", [(2, 16, 16), (1, 13, 21)])
def test_fp64_gradients_match_oracle(bid, shape):
    B, H, W = shape
    params = _params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(B, H, W, 6))
    t = rng.normal(size=(B, H, W, 2))
    net = bid.Cnn(B * H * W, seed=1)
    net.set_params(flat(params))
    assert np.array_equal(net.get_params(), flat(params))
    lg, grad = net.loss_grad(torch.tensor(x, device=DEV), torch.tensor(t, device=DEV), "fp64")
    lo, go = cnn.loss_and_grads(params, x, t)
    assert abs(lg - lo) <= 1e-12 * abs(lo)
    gof = flat(go)
    assert np.abs(grad - gof).max() <= 1e-10 * np.abs(gof).max()


def test_fp32_gradients_match_oracle(bid):
    B, H, W = 2, 16, 16
    params = _params(5)
    rng = np.random.default_rng(6)
    x = f32(rng.normal(size=(B, H, W, 6)))
    t = f32(rng.normal(size=(B, H, W, 2)))
    net = bid.Cnn(B * H * W, seed=1)
    net.set_params(flat(params))
    xs = torch.tensor(x, dtype=torch.float32, device=DEV)
    ts = torch.tensor(t, dtype=torch.float32, device=DEV)
    lg, grad = net.loss_grad(xs, ts, "fp32")
    lo, go = cnn.loss_and_grads(params, x, t)
    assert abs(lg - lo) <= 1e-5 * abs(lo)
    o = 0
    for dW, db in go:
        for arr in (dW.ravel(), db.ravel()):
            seg = grad[o:o + arr.size]
            assert np.abs(seg - arr).max() <= 1e-4 * max(np.abs(arr).max(), 1e-30)
            o += arr.size


@pytest.mark.parametrize("H,W", [(40, 50), (64, 64), (9, 17)])
def test_bf16_tensor_core_forward_matches_oracle(bid, H, W):
    params = _params(7)
    # W3 and the biases stay FP32 on the device: make W3 BF16-exact so that
    # rounding every weight in the oracle matches the device
    W3, b3 = params[2]
    params[2] = (cnn.round_bf16(W3), b3)
    rng = np.random.default_rng(8)
    x = f32(rng.normal(size=(1, H, W, 6)))
    net = bid.Cnn(H * W, seed=1)
    net.set_params(flat(params))
    y = torch.zeros((1, H, W, 2), dtype=torch.float32, device=DEV)
    net.forward(torch.tensor(x, dtype=torch.float32, device=DEV), y, "bf16")
    yo, _ = cnn.forward(params, x, rnd=cnn.round_bf16)
    yg = y.cpu().numpy().astype(np.float64)
    assert np.abs(yg - yo).max() <= 5e-3 * np.abs(yo).max()
    assert np.abs(yg - yo).mean() <= 5e-4 * np.abs(yo).max()
    # the FP32 direct path agrees with the unrounded oracle
    yf = torch.zeros((1, H, W, 2), dtype=torch.float32, device=DEV)
    net.forward(torch.tensor(x, dtype=torch.float32, device=DEV), yf, "fp32")
    yo32, _ = cnn.forward(params, x)
    assert np.abs(yf.cpu().numpy() - yo32).max() <= 1e-4 * np.abs(yo32).max()


def test_training_reduces_the_loss(bid):
    # fit a fixed local linear map of the inputs (a 3 x 3 stencil on two channels)
    B, H, W = 4, 32, 32
    rng = np.random.default_rng(10)
    x = f32(rng.normal(size=(B, H, W, 6)))
    t = f32(np.stack([0.5 * x[..., 0] - 0.25 * np.roll(x[..., 3], 1, axis=1) + 0.1,
                      0.3 * x[..., 4] - 0.2 * x[..., 1]], axis=-1))
    net = bid.Cnn(B * H * W, seed=2)
    xs = torch.tensor(x, dtype=torch.float32, device=DEV)
    ts = torch.tensor(t, dtype=torch.float32, device=DEV)
    l0 = net.train_step(xs, ts, 1e-3)
    for _ in range(300):
        loss = net.train_step(xs, ts, 1e-3)
    assert loss < 0.05 * l0


def test_learned_guess_gain(bid):
    # 257^2 slice: train the guess online on 80 plain steps (stimulus seed 100),
    # then step a held-out stimulus (seed 200) with and without it.  The
    # learned guess starts PCG closer to the solution: its initial residual
    # is at least 1.5x smaller on the median step (measured 2-5x), it is the
    # one used on nearly every step once three states are known, it never
    # costs iterations, and the solution is unchanged within the tolerance.
    # (Saving a whole iteration at rel-res 1e-10 would take a guess about 100x
    # better than the previous step: one PCG iteration reduces the residual
    # by about that much here.)
    n, dt, steps = 257, 0.1, 60
    mesh, p = torso_square_2d(n), params_2d(dt)
    S = bid.System(mesh, p)
    P = bid.Precond(S, dt, eps=1e-3, precision="fp32")
    net = bid.Cnn(16 * 64 * 64, seed=3)
    G = bid.Guess(S, net, n, n, max_batch_pixels=16 * 64 * 64)

    def state(seed):
        U = torch.zeros(S.N, dtype=torch.float64, device=DEV)
        V = torch.full((S.NH,), p["v_rest"], dtype=torch.float64, device=DEV)
        h = torch.ones(S.NH, dtype=torch.float64, device=DEV)
        I = torch.tensor(stimulus_seeded_disc(mesh, seed=seed)[S.perm[:S.NH]], device=DEV)
        return U, V, h, I

    U, V, h, I = state(100)
    G.push(U, V)
    for k in range(80):
        P.step(U, V, h, I, k * dt, 1)
        G.push(U, V)
        if k >= 3:
            G.train(ncrops=16, crop=64, iters=8, lr=2e-3, seed=k)
    assert all(s > 0 for s in G.scales())
    # held-out run: learned vs plain, same state sequence
    Ua, Va, ha, I2 = state(200)
    Ub, Vb, hb, _ = state(200)
    G.reset()
    G.push(Ua, Va)
    st_l = G.step(P, Ua, Va, ha, I2, 0.0, steps, tol=1e-10)
    its_p = P.step(Ub, Vb, hb, I2, 0.0, steps, tol=1e-10)
    used = st_l[:, 3] > 0
    assert not used[:2].any()                         # fewer than three states: fallback
    assert used[3:].mean() > 0.9                      # the learned guess wins most steps
    ratio = st_l[3:, 2] / st_l[3:, 1]
    assert np.median(ratio) < 1 / 1.5
    assert st_l[:, 0].sum() <= its_p.sum()
    Xa = np.concatenate([Ua.cpu().numpy(), Va.cpu().numpy()])
    Xb = np.concatenate([Ub.cpu().numpy(), Vb.cpu().numpy()])
    assert np.linalg.norm(Xa - Xb) <= 1e-7 * np.linalg.norm(Xb)
