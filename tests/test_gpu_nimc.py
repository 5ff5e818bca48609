"""GPU parity of network initialization (include/nmc_gen.h) against oracle/nimc.py.

Generator (FP32 on the device, FP64 in the oracle, same float32 weights): outputs to
5e-5 absolute (sums of up to 13k products of O(0.1) terms in FP32). Bernoulli fields:
bit-exact, both sides comparing the same float32 p in double. Loss path (FP64 both
sides): observables to 1e-10, gradient to 1e-9 relative against automatic
differentiation where the plain inverse is exact (tiny lattice), and to 1e-6 relative
against central differences of the stabilized oracle loss at the paper's honeycomb point.
"""
import numpy as np
import pytest

from oracle import dqmc, nimc
from oracle.dqmc import Model

pytestmark = pytest.mark.gpu

PAPER = Model(6, 6, 1.0, 3.83, 6.0, 0.1, 10, seed=77, lattice="honeycomb")
TINY = Model(2, 1, 1.0, 3.0, 0.6, 0.1, 3, seed=5, lattice="honeycomb")   # N = 4, L_tau = 6
TINY_ARCH = dict(z=(2, 2, 1), c1=3, k1=(3, 2, 1), k2=(3, 2, 1))
TINY_ARCH_OR = [(1, 3, (3, 2, 1)), (3, 1, (3, 2, 1))]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_00712_gb300 import nmc
    nmc.load()
    return torch, nmc


def _gen(nmc, model, arch=None, seed=3, max_batch=8):
    a = nmc.gen_arch(**arch) if arch else nmc.gen_arch()
    return nmc.Generator(model.Lx, model.Ly, model.t, model.U, model.beta, model.dtau,
                         model.n_wrap, arch=a, seed=seed, max_batch=max_batch,
                         lattice=model.lattice)


def test_initial_weights_and_forward_match_oracle(env):
    torch, nmc = env
    arch = [(1, 20, (16, 6, 3)), (20, 1, (36, 6, 3))]
    with _gen(nmc, PAPER, seed=0x51) as g:
        params = g.params()
        ref = nimc.glorot_params(0x51, arch)
        for (W, b), (Wr, br) in zip(params, ref):
            assert np.array_equal(W, Wr.astype(np.float32)) and np.all(b == 0)
        n, n0 = 5, 123
        for stream in (0, 1):
            d_p = torch.empty((n, 60, 12, 6), dtype=torch.float32, device="cuda")
            g.probs(n0, n, stream, d_p.data_ptr())
            z = nimc.generator_input(0x51, n0, n, (10, 2, 2), stream)
            want = nimc.generator([(W.astype(np.float64), b.astype(np.float64))
                                   for (W, b) in params], z)
            assert np.max(np.abs(d_p.cpu().numpy() - want)) < 5e-5


def test_bernoulli_fields_bit_exact(env):
    torch, nmc = env
    with _gen(nmc, PAPER, seed=9) as g:
        n, n0 = 7, 40
        d_p = torch.empty((n, 60, 12, 6), dtype=torch.float32, device="cuda")
        g.probs(n0, n, 1, d_p.data_ptr())
        d_s = torch.empty((n, 60, 72), dtype=torch.int8, device="cuda")
        g.sample_fields(n0, n, 1, d_s.data_ptr())
        p = d_p.cpu().numpy().transpose(0, 1, 3, 2).reshape(n, 60, 72)
        np.testing.assert_array_equal(d_s.cpu().numpy(), nimc.bernoulli_fields(9, p, n0, 1))


def test_generate_mode1_fills_context_fields(env):
    torch, nmc = env
    m = PAPER
    with _gen(nmc, m, seed=4) as g, nmc.Context(m.Lx, m.Ly, m.t, m.U, m.beta, m.dtau,
                                                m.n_wrap, seed=1, n_chains=3, chain_offset=10,
                                                lattice=m.lattice) as c:
        c.generate(mode=1, model=g.g)
        d_s = torch.empty((3, 60, 72), dtype=torch.int8, device="cuda")
        g.sample_fields(10, 3, 1, d_s.data_ptr())
        np.testing.assert_array_equal(c.fields(), d_s.cpu().numpy())
        c.sweep(1, measure=1)
        assert c.measure().max_drift < 1e-6


@pytest.mark.parametrize("model", [TINY, Model(3, 3, 1.0, 3.83, 1.0, 0.1, 5, lattice="honeycomb"),
                                   Model(4, 4, 1.0, 4.0, 2.0, 0.1, 10)])
def test_observables_match_oracle(env, model):
    torch, nmc = env
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-1, 1, size=(3, model.L_tau, model.N)),
                        rng.choice([-1.0, 1.0], size=(2, model.L_tau, model.N))])
    with _gen(nmc, model, arch=_arch_for(model), max_batch=2) as g:
        d_x = torch.from_numpy(x).cuda()
        d_o = torch.empty((5, 2), dtype=torch.float64, device="cuda")
        g.observables(d_x.data_ptr(), 5, d_o.data_ptr())
        got = d_o.cpu().numpy()
    for b in range(5):
        ek, s = nimc.observables(model, x[b])
        assert abs(got[b, 0] - s) < 1e-10 and abs(got[b, 1] - ek) < 1e-10


def _arch_for(model):
    """Any architecture whose output is (L_tau, A, B) for this model."""
    A = 2 * model.Lx if model.lattice == "honeycomb" else model.Lx
    return dict(z=(2, 1, 1), c1=2, k1=(model.L_tau - 1, A, model.Ly), k2=(1, 1, 1))


def test_loss_gradient_matches_autograd_tiny(env):
    torch, nmc = env
    rng = np.random.default_rng(2)
    n = 5
    x = rng.uniform(-0.95, 0.95, size=(n, TINY.L_tau, TINY.N))
    tg = np.stack([rng.uniform(0.3, 0.6, n), rng.uniform(-1.6, -1.2, n)], axis=1)
    xt = torch.tensor(x, requires_grad=True)
    L = nimc.loss_torch_naive(torch, TINY, xt, tg, 3.0, 0.7)
    L.backward()
    with _gen(nmc, TINY, arch=TINY_ARCH, max_batch=2) as g:
        d_x = torch.from_numpy(x).cuda()
        d_t = torch.from_numpy(tg).cuda()
        d_l = torch.empty(n, dtype=torch.float64, device="cuda")
        d_g = torch.empty_like(d_x)
        g.loss_grad(d_x.data_ptr(), n, d_t.data_ptr(), 3.0, 0.7, d_l.data_ptr(), d_g.data_ptr())
        got_l, got_g = d_l.cpu().numpy(), d_g.cpu().numpy()
    assert abs(got_l.sum() - float(L.detach())) < 1e-12 * max(1.0, abs(float(L.detach())))
    ref = xt.grad.numpy()
    assert np.max(np.abs(got_g - ref)) < 1e-9 * np.max(np.abs(ref))


def test_loss_gradient_paper_point_sampled(env):
    torch, nmc = env
    rng = np.random.default_rng(3)
    n = 3
    x = rng.uniform(-1, 1, size=(n, 60, 72))
    x[1] = np.sign(x[1])                     # a Markov-chain-like +-1 configuration
    tg = np.array([[0.72, -1.36], [0.5, -1.2], [0.9, -1.5]])
    with _gen(nmc, PAPER, max_batch=2) as g:
        d_x = torch.from_numpy(x).cuda()
        d_t = torch.from_numpy(tg).cuda()
        d_l = torch.empty(n, dtype=torch.float64, device="cuda")
        d_g = torch.empty_like(d_x)
        g.loss_grad(d_x.data_ptr(), n, d_t.data_ptr(), 2.0, 0.5, d_l.data_ptr(), d_g.data_ptr())
        got_l, got_g = d_l.cpu().numpy(), d_g.cpu().numpy()
    for b in range(n):
        assert abs(got_l[b] - nimc.loss(PAPER, x[b:b + 1], tg[b:b + 1], 2.0, 0.5)) < 1e-10
    entries = [(0, 0, 0), (0, 59, 71), (1, 9, 13), (1, 10, 14), (2, 33, 40), (2, 19, 1)]
    fd = nimc.loss_grad_fd(PAPER, x, tg, 2.0, 0.5, entries, h=1e-5)
    got = np.array([got_g[e] for e in entries])
    scale = np.max(np.abs(got_g))
    assert np.max(np.abs(fd - got)) < 1e-6 * scale, (fd, got)


def test_train_step_matches_oracle(env):
    torch, nmc = env
    rng = np.random.default_rng(4)
    with _gen(nmc, TINY, arch=TINY_ARCH, seed=12, max_batch=2) as g:
        params = [(W.astype(np.float64), rng.normal(scale=0.1, size=b.shape).astype(np.float32)
                   .astype(np.float64)) for (W, b) in g.params()]
        g.set_params(params)
        ids = np.array([3, 0, 7])
        tg = np.stack([rng.uniform(0.3, 0.6, 3), rng.uniform(-1.6, -1.2, 3)], axis=1)
        lr = 1e-3
        loss = g.train_step(ids, tg, 2.0, 0.5, lr)
        after = g.params()
        assert g.steps() == 1
    z = np.stack([nimc.generator_input(12, int(i), 1, (2, 2, 1))[0] for i in ids])
    state = [(np.zeros_like(a), np.zeros_like(a)) for pr in params for a in pr]
    new, _, L, grads = nimc.train_step_naive(TINY, params, state, 1, z, tg, 2.0, 0.5, lr)
    assert abs(loss - L) < 1e-5 * abs(L)
    flat_old = [a for pr in params for a in pr]
    flat_new = [a for pr in new for a in pr]
    flat_gpu = [a for pr in after for a in pr]
    for old, want, got, gr in zip(flat_old, flat_new, flat_gpu, grads):
        big = np.abs(gr) > 1e-3 * np.max(np.abs(gr))
        # step 1 moves each parameter by about lr * sign(g): equal where g is not tiny
        assert np.all(np.abs((got - old) - (want - old))[big] < 1e-3 * lr)
        assert np.all(np.abs(got - old) <= 1.0001 * lr + 1e-7)


def test_training_reduces_the_loss(env):
    torch, nmc = env
    rng = np.random.default_rng(5)
    m = Model(3, 3, 1.0, 3.83, 2.0, 0.1, 5, lattice="honeycomb")
    arch = dict(z=(4, 2, 1), c1=4, k1=(8, 3, 2), k2=(10, 3, 2))   # -> 20 x 6 x 3
    n = 24
    # targets: observables of random +-1 configurations (reachable by the generator)
    x = rng.choice([-1.0, 1.0], size=(n, m.L_tau, m.N))
    tg = np.array([nimc.observables(m, x[b])[::-1] for b in range(n)])
    with _gen(nmc, m, arch=arch, seed=2, max_batch=8) as g:
        hist = g.train(tg, epochs=10, batch=4, lr=2e-2)
        assert g.steps() == 10 * 6
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.9 * hist[0], hist


def test_generated_observables_match_oracle(env):
    torch, nmc = env
    m = Model(3, 3, 1.0, 3.83, 1.0, 0.1, 5, lattice="honeycomb")
    with _gen(nmc, m, arch=_arch_for(m), seed=21, max_batch=2) as g:
        n = 3
        d_p = torch.empty((n, m.L_tau, 6, 3), dtype=torch.float32, device="cuda")
        g.probs(5, n, 1, d_p.data_ptr())
        d_o = torch.empty((n, 2), dtype=torch.float64, device="cuda")
        g.generated_observables(5, n, 1, d_o.data_ptr())
        x = nimc.fields_from_p(d_p.cpu().numpy().astype(np.float64))
        got = d_o.cpu().numpy()
    for b in range(n):
        ek, s = nimc.observables(m, x[b])
        assert abs(got[b, 0] - s) < 1e-10 and abs(got[b, 1] - ek) < 1e-10


def test_series_is_consistent_with_measure(env):
    torch, nmc = env
    m = Model(3, 3, 1.0, 3.83, 2.0, 0.1, 5, seed=3, lattice="honeycomb")
    with nmc.Context(m.Lx, m.Ly, m.t, m.U, m.beta, m.dtau, m.n_wrap, seed=m.seed, n_chains=4,
                     lattice=m.lattice) as c:
        c.generate()
        c.sweep(2, measure=0)
        c.sweep(5, measure=1)
        ser = c.series()
        _, per = c.measure(per_chain=True)
    assert ser.shape == (5, 4, 5)
    for ch in range(4):
        for k, name in enumerate(("energy", "ekin", "double_occ", "s_pipi", "density")):
            assert abs(ser[:, ch, k].mean() - getattr(per[ch], name).mean) < 1e-12


def test_gradient_clip_bounds_the_step(env):
    """With a tiny bound the clipped gradient is far below Adam's epsilon, so the first
    step moves no parameter by more than lr * 1e-3; without a bound it moves by ~lr."""
    torch, nmc = env
    rng = np.random.default_rng(6)
    tg = np.stack([rng.uniform(0.3, 0.6, 2), rng.uniform(-1.6, -1.2, 2)], axis=1)
    moved = []
    for clip in (1e-12, 0.0):
        with _gen(nmc, TINY, arch=TINY_ARCH, seed=8, max_batch=2) as g:
            g.set_clip(clip)
            before = [a.copy() for pr in g.params() for a in pr]
            g.train_step(np.array([0, 1]), tg, 2.0, 0.5, 1e-3)
            after = [a for pr in g.params() for a in pr]
            moved.append(max(float(np.max(np.abs(a - b))) for a, b in zip(after, before)))
    assert moved[0] < 1e-6 and moved[1] > 5e-4, moved
