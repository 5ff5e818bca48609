"""GPU parity of the convolutional field generator (include/nmc_cgen.h) against its oracle
(oracle/cgen.py), through the C ABI.

* Exact arithmetic: noise, weights and biases in {-1, 0, 1} with three channels make every
  sum of the four convolutions an integer below 81^3 * 27 < 2^24 (81 terms per output after
  the first layer), so exact in FP32 and in FP64, and the BF16 roundings between layers the
  same on both sides: the logits must be bit-identical (this checks every index, offset and
  periodic wrap).
* General inputs: logits, loss and gradients against the oracle fed the same BF16 operands.
  The kernels accumulate in FP32 and round each layer's output to BF16; where an FP32 sum and
  the FP64 one fall on different sides of a BF16 rounding boundary an activation differs by
  one BF16 unit (2^-8 relative), rarely, so the bars are relative to each array's scale:
  logits 2e-3, loss 1e-4, each layer's weight gradient 3e-2.
* Noise and draws: the Box-Muller noise has mean 0 and variance 1, sampled fields are +-1
  with the frequency sigmoid(logit) says.
* Training: with noise independent of the fields, maximum likelihood drives every logit to
  the fields' log-odds (oracle.cgen.optimal_bias); a short training on fields with a known
  occupation reaches it.
"""
import numpy as np
import pytest

from oracle import cgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_00712_gb300 import nmc as m
    m.load()
    return m, torch


def _flat(params):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


def _gen(nmc, shape, C, n, seed=0):
    T, A, B = shape
    return nmc.ConvGenerator(B, A, T, channels=C, seed=seed, max_batch=n)


def test_forward_is_bit_exact_on_exact_arithmetic(env):
    nmc, torch = env
    shape, C, n = (5, 4, 3), 3, 2
    rng = np.random.default_rng(1)
    params = []
    for co, ci in ((C, 1), (C, C), (C, C), (1, C)):
        W = rng.integers(-1, 2, size=(co, ci, 3, 3, 3)).astype(np.float64)
        b = rng.integers(-1, 2, size=co).astype(np.float64)
        params.append((W, b))
    z = rng.integers(-1, 2, size=(n,) + shape).astype(np.float64)
    want, _ = cgen.forward(params, z, round_bf16=True)
    with _gen(nmc, shape, C, n) as g:
        g.set_params(_flat(params))
        dz = torch.from_numpy(z.astype(np.float32)).cuda()
        dl = torch.empty_like(dz)
        g.forward(dz.data_ptr(), n, dl.data_ptr())
        got = dl.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("shape,C,n", [((40, 8, 8), 32, 3), ((6, 3, 5), 5, 4), ((4, 2, 2), 8, 2)])
def test_forward_loss_and_gradients_match_oracle(env, shape, C, n):
    nmc, torch = env
    rng = np.random.default_rng(sum(shape) + C)
    params = cgen.init_params(C, seed=C, scale=0.25)
    params = [(cgen.bf16(W), b.astype(np.float32).astype(np.float64)) for W, b in params]
    z = rng.normal(size=(n,) + shape)
    s = np.where(rng.random((n,) + shape) < 0.6, 1.0, -1.0)
    want_l, _ = cgen.forward(params, z, round_bf16=True)
    want_loss, want_g = cgen.loss_and_grads(params, z, s, round_bf16=True)
    with _gen(nmc, shape, C, n) as g:
        g.set_params(_flat(params))
        dz = torch.from_numpy(z.astype(np.float32)).cuda()
        dl = torch.empty_like(dz)
        g.forward(dz.data_ptr(), n, dl.data_ptr())
        got_l = dl.cpu().numpy().astype(np.float64)
        df = torch.from_numpy(s.astype(np.int8)).cuda()
        dg = torch.empty(g.n_params(), dtype=torch.float32, device="cuda")
        got_loss = g.loss_grad(dz.data_ptr(), df.data_ptr(), n, dg.data_ptr())
        got_g = dg.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got_l - want_l)) <= 2e-3 * np.max(np.abs(want_l))
    assert abs(got_loss - want_loss) <= 1e-4 * want_loss
    o = 0
    for j, (gW, gb) in enumerate(want_g):
        for ref in (gW.reshape(-1), gb):
            got = got_g[o:o + ref.size]
            o += ref.size
            assert np.max(np.abs(got - ref)) <= 3e-2 * np.max(np.abs(ref)) + 1e-12, j
    assert o == got_g.size


def test_noise_and_draws_have_the_stated_distributions(env):
    nmc, torch = env
    shape, n = (40, 8, 8), 64
    with _gen(nmc, shape, 4, n, seed=9) as g:
        g.set_params(np.zeros(g.n_params(), dtype=np.float32))   # logits 0: p = 1/2
        f = torch.empty((n,) + shape, dtype=torch.int8, device="cuda")
        lg = torch.empty((n,) + shape, dtype=torch.float32, device="cuda")
        g.sample(0, n, f.data_ptr(), lg.data_ptr())
        fields = f.cpu().numpy()
        assert set(np.unique(fields)) <= {-1, 1}
        assert np.all(lg.cpu().numpy() == 0.0)
        m = fields.mean()
        assert abs(m) < 5 * np.sqrt(1.0 / fields.size)       # P(+1) = 1/2
        # a bias moves every logit: P(+1) = sigmoid(b)
        th = np.zeros(g.n_params(), dtype=np.float32)
        th[-1] = 1.0
        g.set_params(th)
        g.sample(0, n, f.data_ptr(), None)
        frac = (f.cpu().numpy() > 0).mean()
        p = 1 / (1 + np.exp(-1.0))
        assert abs(frac - p) < 5 * np.sqrt(p * (1 - p) / fields.size)
        # the noise itself: the first layer's identity picks it up exactly as a logit
        th = np.zeros(g.n_params(), dtype=np.float32)
        C = g.C
        th[13] = 1.0                                 # W0[0][0][1][1][1]: the centre tap
        o1 = C * 27 + C                              # W1 starts here
        th[o1 + 13] = 1.0                            # W1[0][0] centre
        o2 = o1 + C * C * 27 + C
        th[o2 + 13] = 1.0                            # W2[0][0] centre
        o3 = o2 + C * C * 27 + C
        th[o3 + 13] = 1.0                            # W3[0][0] centre
        g.set_params(th)
        g.sample(0, n, f.data_ptr(), lg.data_ptr())
        z = lg.cpu().numpy().reshape(-1)             # relu(z) after three ReLUs
        pos = z[z > 0]
        # half-normal: E = sqrt(2/pi), P(z > 0) = 1/2 (BF16 noise: 2^-9 relative)
        assert abs((z > 0).mean() - 0.5) < 5 * np.sqrt(0.25 / z.size)
        assert abs(pos.mean() - np.sqrt(2 / np.pi)) < 5 * np.sqrt((1 - 2 / np.pi) / pos.size) + 5e-3
        assert abs((pos ** 2).mean() - 1.0) < 0.02


def test_training_reaches_the_maximum_likelihood_log_odds(env):
    """Fields with P(+1) = 0.7 at every entry, noise independent of them: the trained
    generator's mean occupation approaches 0.7 (the closed-form optimum) and its loss the
    entropy of that Bernoulli."""
    nmc, torch = env
    shape, n = (8, 4, 4), 32
    rng = np.random.default_rng(3)
    with _gen(nmc, shape, 8, n, seed=5) as g:
        losses = []
        for step in range(300):
            s = np.where(rng.random((n,) + shape) < 0.7, 1, -1).astype(np.int8)
            df = torch.from_numpy(s).cuda()
            losses.append(g.train_step(df.data_ptr(), n, step * n, 3e-3))
        lg = torch.empty((n,) + shape, dtype=torch.float32, device="cuda")
        f = torch.empty((n,) + shape, dtype=torch.int8, device="cuda")
        g.sample(0, n, f.data_ptr(), lg.data_ptr())
        p = 1 / (1 + np.exp(-lg.cpu().numpy()))
    assert abs(p.mean() - 0.7) < 0.02
    h = -(0.7 * np.log(0.7) + 0.3 * np.log(0.3))
    assert np.mean(losses[-20:]) < h + 0.01
    assert losses[0] > np.mean(losses[-20:])
