"""Pins for the network-initialization oracle (oracle/nimc.py): each check compares it
with something other than itself -- a library routine, brute force, finite differences,
closed forms, or the sweep oracle's independent plain-inverse Green's function."""
import numpy as np
import pytest

from oracle import dqmc, nimc
from oracle.dqmc import Model

torch = pytest.importorskip("torch")

TINY = Model(2, 1, 1.0, 3.0, 0.6, 0.1, 3, seed=5, lattice="honeycomb")   # N = 4, L_tau = 6
# tiny network with the paper's structure: 2x2x1 -> (3 ch, 3x2x1) -> 4x3x1 -> (3x2x1) -> 6x4x1
TINY_ARCH = [(1, 3, (3, 2, 1)), (3, 1, (3, 2, 1))]
TINY_Z = (2, 2, 1)


def _targets(B, rng):
    return np.stack([rng.uniform(0.3, 0.6, B), rng.uniform(-1.6, -1.2, B)], axis=1)


def test_conv_transpose_matches_library_and_brute_force():
    """Reading N1 against torch's conv_transpose3d (stride 1, no padding) and a plain
    scatter loop over input positions and kernel offsets."""
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 3, 2))
    W = rng.normal(size=(3, 5, 3, 2, 2))
    b = rng.normal(size=5)
    got = nimc.conv_transpose3d(x, W, b)
    ref = torch.nn.functional.conv_transpose3d(torch.from_numpy(x), torch.from_numpy(W),
                                               torch.from_numpy(b)).numpy()
    assert got.shape == (2, 5, 6, 4, 3)
    assert np.max(np.abs(got - ref)) < 1e-12
    brute = np.zeros_like(got) + b.reshape(1, 5, 1, 1, 1)
    for n in range(2):
        for ci in range(3):
            for i0, i1, i2 in np.ndindex(4, 3, 2):
                for k0, k1, k2 in np.ndindex(3, 2, 2):
                    brute[n, :, i0 + k0, i1 + k1, i2 + k2] += x[n, ci, i0, i1, i2] * W[ci, :, k0, k1, k2]
    assert np.max(np.abs(got - brute)) < 1e-12
    tx = torch.from_numpy(x)
    tg = nimc.conv_transpose3d(tx, torch.from_numpy(W), torch.from_numpy(b), torch)
    assert np.max(np.abs(tg.numpy() - ref)) < 1e-12


def test_paper_network_shapes():
    """SM Sec. II: 10x2x2 input, 20 filters 16x6x3, 1 filter 36x6x3 -> 60x12x6."""
    arch = [(1, 20, (16, 6, 3)), (20, 1, (36, 6, 3))]
    params = nimc.glorot_params(1, arch)
    z = nimc.generator_input(7, 0, 2, (10, 2, 2))
    p = nimc.generator(params, z)
    assert p.shape == (2, 60, 12, 6)
    assert np.all((p > 0) & (p < 1))
    x = nimc.fields_from_p(p)
    assert x.shape == (2, 60, 72)
    # site i = a + 12 b holds p[l, a, b]
    assert x[1, 17, 5 + 12 * 4] == 2 * p[1, 17, 5, 4] - 1


def test_generator_input_and_glorot_statistics():
    z = nimc.generator_input(3, 100, 500, (10, 2, 2))
    assert set(np.unique(z)) == {-1.0, 1.0}
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert not np.array_equal(z[0], z[1])
    arch = [(1, 20, (16, 6, 3)), (20, 1, (36, 6, 3))]
    for (W, b), (cin, cout, ks) in zip(nimc.glorot_params(2, arch), arch):
        rf = np.prod(ks)
        lim = np.sqrt(6 / (cin * rf + cout * rf))
        assert np.all(np.abs(W) <= lim) and np.all(b == 0)
        # uniform on [-lim, lim]: variance lim^2 / 3
        assert abs(W.var() / (lim * lim / 3) - 1) < 0.05


def test_observables_of_pm1_fields_equal_plain_inverse():
    """Reading N3 on +-1 fields equals the sweep oracle's estimators on the plain-inverse
    G_0 (dqmc.green_naive, valid at this small beta), and continuous fields reduce to the
    same formula (x -> B_l uses e^{sigma lam x})."""
    model = Model(3, 3, 1.0, 3.83, 1.0, 0.1, 5, lattice="honeycomb")
    P = dqmc.Propagators(model)
    rng = np.random.default_rng(1)
    for x in (rng.choice([-1.0, 1.0], size=(10, 18)), rng.uniform(-1, 1, size=(10, 18))):
        ek, s = nimc.observables(model, x, P)
        G = [dqmc.green_naive(P, x, sigma, 0) for sigma in dqmc.SIGMAS]
        m = dqmc.measure(P, model, G[0], G[1])
        assert abs(ek - m["ekin"]) < 1e-11 and abs(s - m["s_pipi"]) < 1e-11


def test_loss_gradient_autograd_equals_finite_differences():
    """d(Eq. 4)/dx by autograd through the plain inverse equals central differences of
    the stabilized loss (different G algorithms, different derivative methods)."""
    rng = np.random.default_rng(2)
    x = rng.uniform(-0.9, 0.9, size=(2, TINY.L_tau, TINY.N))
    tg = _targets(2, rng)
    xt = torch.tensor(x, requires_grad=True)
    L = nimc.loss_torch_naive(torch, TINY, xt, tg, 3.0, 0.7)
    L.backward()
    assert abs(float(L.detach()) - nimc.loss(TINY, x, tg, 3.0, 0.7)) < 1e-12
    entries = [(0, 0, 0), (0, 3, 2), (1, 5, 3), (1, 1, 1), (0, 5, 0)]
    fd = nimc.loss_grad_fd(TINY, x, tg, 3.0, 0.7, entries, h=1e-5)
    ag = np.array([xt.grad[e].item() for e in entries])
    assert np.max(np.abs(fd - ag)) < 1e-8 * max(1.0, np.max(np.abs(ag)))
    assert np.max(np.abs(ag)) > 1e-3


def test_loss_gradient_vanishes_at_u0():
    """lam = 0: the weight does not depend on the fields, so neither does the loss."""
    model = Model(2, 1, 1.0, 0.0, 0.6, 0.1, 3, lattice="honeycomb")
    rng = np.random.default_rng(3)
    xt = torch.tensor(rng.uniform(-1, 1, size=(1, 6, 4)), requires_grad=True)
    nimc.loss_torch_naive(torch, model, xt, _targets(1, rng), 1.0, 1.0).backward()
    assert float(xt.grad.abs().max()) == 0.0


def test_parameter_gradients_equal_finite_differences():
    """The generator's backward pass (autograd through reading N1's definition) against
    central differences of the whole loss in parameter space."""
    rng = np.random.default_rng(4)
    params = nimc.glorot_params(9, TINY_ARCH)
    params = [(W, rng.normal(scale=0.1, size=b.shape)) for (W, b) in params]
    z = nimc.generator_input(11, 0, 2, TINY_Z)
    tg = _targets(2, rng)
    state = [(np.zeros_like(a), np.zeros_like(a)) for pr in params for a in pr]
    _, _, L0, grads = nimc.train_step_naive(TINY, params, state, 1, z, tg, 2.0, 0.5, 0.0)

    def total(ps):
        x = nimc.fields_from_p(nimc.generator(ps, z))
        return nimc.loss(TINY, x, tg, 2.0, 0.5)

    assert abs(L0 - total(params)) < 1e-12
    h = 1e-6
    for k, idx in ((0, (0, 1, 2, 1, 0)), (1, (1,)), (2, (2, 0, 1, 0, 0)), (3, (0,))):
        layer, which = divmod(k, 2)
        plus = [list(pr) for pr in params]
        minus = [list(pr) for pr in params]
        plus[layer][which] = plus[layer][which].copy()
        minus[layer][which] = minus[layer][which].copy()
        plus[layer][which][idx] += h
        minus[layer][which][idx] -= h
        fd = (total([tuple(p) for p in plus]) - total([tuple(p) for p in minus])) / (2 * h)
        assert abs(fd - grads[k][idx]) < 1e-7 * max(1.0, abs(fd)), (k, fd, grads[k][idx])


def test_adam_first_steps_closed_form():
    """Step 1: m^ = g, v^ = g^2, so theta moves by -lr g / (|g| + eps); step 2 with a
    constant gradient moves by the same amount (bias corrections cancel)."""
    g = np.array([0.3, -2.0, 1e-9, 0.0])
    th, m, v = nimc.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 1e-3)
    assert np.allclose(th, -1e-3 * g / (np.abs(g) + nimc.ADAM_EPS), rtol=1e-13, atol=0)
    th2, _, _ = nimc.adam_step(th, g, m, v, 2, 1e-3)
    assert np.allclose(th2 - th, th, rtol=1e-12, atol=1e-20)


def test_bernoulli_fields():
    B, L, N = 4, 30, 72
    p = np.full((B, L, N), 0.3, dtype=np.float32)
    s = nimc.bernoulli_fields(5, p, 0)
    assert set(np.unique(s)) <= {-1, 1}
    frac = (s == 1).mean()
    assert abs(frac - 0.3) < 5 * np.sqrt(0.21 / s.size)
    assert np.all(nimc.bernoulli_fields(5, np.zeros((1, L, N), np.float32), 0) == -1)
    assert np.all(nimc.bernoulli_fields(5, np.ones((1, L, N), np.float32), 0) == 1)
    # sample index is the counter word: shifting n0 shifts samples
    assert np.array_equal(nimc.bernoulli_fields(5, p, 2)[0], s[2])
