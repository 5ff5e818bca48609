"""Pins of the convolutional generator's oracle (oracle/cgen.py) against constructions that
do not reuse it: an entry-by-entry periodic convolution, the adjoint identity of the
convolution, central finite differences of the loss, the closed-form maximum-likelihood
bias, translation equivariance, and PyTorch's own float32 -> bfloat16 rounding."""
import numpy as np
import pytest

from oracle import cgen


def _rand(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


@pytest.mark.parametrize("shape", [(4, 3, 2), (3, 3, 3), (2, 1, 5), (5, 4, 4)])
def test_conv_equals_entrywise_periodic_sum(shape):
    h = _rand((2, 3) + shape, 1)
    W = _rand((4, 3, 3, 3, 3), 2)
    b = _rand(4, 3)
    np.testing.assert_allclose(cgen.conv(h, W, b), cgen.conv_bruteforce(h, W, b),
                               rtol=1e-13, atol=1e-13)


def test_grad_input_is_the_adjoint_of_the_convolution():
    """<conv(h) - b, g> = <h, conv_grad_input(g)> for every h, g (no bias)."""
    h = _rand((2, 3, 4, 3, 5), 4)
    g = _rand((2, 5, 4, 3, 5), 5)
    W = _rand((5, 3, 3, 3, 3), 6)
    lhs = np.sum(cgen.conv(h, W, np.zeros(5)) * g)
    rhs = np.sum(h * cgen.conv_grad_input(g, W))
    assert abs(lhs - rhs) < 1e-10 * (abs(lhs) + 1)


def test_grad_weight_is_the_adjoint_in_the_weights():
    """conv is linear in (W, b): <conv_W(h), g> = <W, dL/dW> + <b, dL/db>."""
    h = _rand((2, 2, 3, 4, 2), 7)
    g = _rand((2, 3, 3, 4, 2), 8)
    W = _rand((3, 2, 3, 3, 3), 9)
    b = _rand(3, 10)
    gW, gb = cgen.conv_grad_weight(g, h)
    lhs = np.sum(cgen.conv(h, W, b) * g)
    rhs = np.sum(W * gW) + np.sum(b * gb)
    assert abs(lhs - rhs) < 1e-10 * (abs(lhs) + 1)


def test_loss_gradients_match_finite_differences():
    params = cgen.init_params(2, seed=3, scale=0.4)
    rng = np.random.default_rng(11)
    z = rng.normal(size=(2, 3, 2, 3))
    s = np.where(rng.random((2, 3, 2, 3)) < 0.4, -1.0, 1.0)
    _, grads = cgen.loss_and_grads(params, z, s)
    eps = 1e-6
    for j, (W, b) in enumerate(params):
        for arr, garr in ((W, grads[j][0]), (b, grads[j][1])):
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp = cgen.loss(cgen.forward(params, z)[0], s)
                flat[idx] = old - eps
                lm = cgen.loss(cgen.forward(params, z)[0], s)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - garr.reshape(-1)[idx]) < 1e-7 + 1e-5 * abs(fd), (j, idx)


def test_maximum_likelihood_bias_is_the_log_odds_of_the_fields():
    """All weights zero: the gradient in the last bias vanishes at log(y / (1 - y)) and the
    loss is smallest there -- with noise independent of the fields this is what maximum
    likelihood drives every logit to."""
    rng = np.random.default_rng(5)
    s = np.where(rng.random((4, 3, 2, 2)) < 0.7, 1.0, -1.0)
    z = rng.normal(size=s.shape)
    params = [(np.zeros_like(W), np.zeros_like(b)) for W, b in cgen.init_params(2)]
    b_opt = cgen.optimal_bias(s)
    params[-1] = (params[-1][0], np.array([b_opt]))
    L0, grads = cgen.loss_and_grads(params, z, s)
    assert abs(grads[-1][1][0]) < 1e-15
    for db in (-0.1, 0.1):
        params[-1] = (params[-1][0], np.array([b_opt + db]))
        assert cgen.loss(cgen.forward(params, z)[0], s) > L0
    y = np.mean((1 + s) / 2)
    assert abs(1 / (1 + np.exp(-b_opt)) - y) < 1e-14


def test_periodic_network_is_translation_equivariant():
    params = cgen.init_params(3, seed=2, scale=0.5)
    z = _rand((1, 5, 4, 3), 12)
    shift = (2, 1, 2)
    l0 = cgen.forward(params, z)[0]
    l1 = cgen.forward(params, np.roll(z, shift, axis=(1, 2, 3)))[0]
    np.testing.assert_allclose(l1, np.roll(l0, shift, axis=(1, 2, 3)), rtol=1e-12, atol=1e-12)


def test_bf16_rounding_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    x = np.concatenate([_rand(4000, 13) * 10.0 ** _rand(4000, 14), [0.0, -0.0, 1.0, -2.5]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cgen.bf16(x), ref)
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 (even: 1); 1 + 3 2^-8 halfway
    # between 1 + 2^-7 and 1 + 2^-6 (even: the latter)
    assert cgen.bf16(1 + 2.0 ** -8) == 1.0
    assert cgen.bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6
    assert cgen.bf16(np.pi) == 3.140625
