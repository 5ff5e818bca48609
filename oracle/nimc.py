"""FP64 CPU oracle for network initialization (Algorithm 1, steps 2-3): the generator of
SM Sec. II (3D transposed convolutions with sigmoid activations), the observable loss of
Eq. 4 evaluated through the determinant weight, its gradient, the Adam step, and the
Bernoulli discretization of generated configurations.

TEST INFRASTRUCTURE ONLY (see the package docstring). numpy in float64; PyTorch CPU in
float64 only where a derivative is taken by automatic differentiation.

Paper passages (arXiv 2106.00712):
* SM Sec. II (Hubbard network): input is a random +-1 configuration of shape 10 x 2 x 2;
  two 3D transposed convolutional layers with valid padding and sigmoid activations,
  20 filters of size 16 x 6 x 3, then 1 filter of size 36 x 6 x 3; output 60 x 12 x 6
  (L_tau x 2L x L on the L = 6 honeycomb lattice).
* Eq. 4: Loss = w1 sum_l [S(Q)(G_l) - S(Q)_l]^2 + w2 sum_l [E_k(G_l) - E_k,l]^2, the
  l-th generated configuration against the l-th training sample's observables; S(Gamma)
  and E_k as in the sweep's estimators.
* Footnote to Algorithm 1: for measurement a generated number p in (0,1) maps to 2p - 1;
  for the Markov chain each element is +1 with probability p, else -1.
* SM Sec. II: Adam with learning rate 1e-3, beta1 = 0.9, beta2 = 0.999.

Readings where the paper is silent:
N1 transposed convolution: stride 1, "valid" padding, so each axis grows by k - 1:
   out[b, co, o] = bias[co] + sum_{ci} sum_{k, i: i + k = o} in[b, ci, i] W[ci, co, k]
   (no kernel flip). 10x2x2 -(16,6,3)-> 25x7x4 -(36,6,3)-> 60x12x6 confirms stride 1.
N2 output layout: p[l, a, b] is the field at slice l of site i = a + A*b, A the second
   output axis (A = 2 Lx: a = 2x + sub on the honeycomb, b = y).
N3 generated fields enter B_l = e^{-dtau K} e^{sigma lam diag x(., l)} with continuous
   x = 2p - 1 (footnote); the observables of a configuration are the sweep's estimators
   on its symmetric-Trotter G~ at slice 0.
N4 loss: the printed sums over the batch; w1, w2 balance the two parts (the caller passes
   them; the library's training uses the inverse variances of the training targets).
N5 generator input z: +-1 per element, -1 iff the top bit of Philox word 0 at counter
   (element, sample, stream, tag 2) is set (tag 1's rule for initial fields); stream 0 is
   the training set's fixed inputs, stream 1 fresh inputs for generation.
N6 Bernoulli: s = +1 iff u < p, u = word 0 * 2^-32 at counter (l*N + i, sample, stream,
   tag 3), compared in double with p as given (float32 from the library's generator).
N7 Adam: Kingma & Ba's update with bias corrections and epsilon = 1e-7 (the TensorFlow
   default; the paper trains in TensorFlow and gives no epsilon).
N8 initial weights: Glorot uniform, limit sqrt(6 / (fan_in + fan_out)) with
   fan_in = C_in * prod(k), fan_out = C_out * prod(k); u from Philox word 0 at counter
   (index, layer, 0, tag 4), W = (2u - 1) * limit; biases 0 (TensorFlow's defaults).
"""
import numpy as np

from . import dqmc
from .philox import philox4x32_10, seed_key

TAG_GEN_Z = 2
TAG_BERNOULLI = 3
TAG_PARAM = 4
ADAM_EPS = 1e-7


# ----------------------------------------------------------------------------- network

def conv_transpose3d(x, W, bias, xp=np):
    """Reading N1. x: [B, Cin, D0, D1, D2], W: [Cin, Cout, k0, k1, k2], bias: [Cout]."""
    B, Cin, D0, D1, D2 = x.shape
    _, Cout, k0, k1, k2 = W.shape
    out = xp.zeros((B, Cout, D0 + k0 - 1, D1 + k1 - 1, D2 + k2 - 1), dtype=x.dtype)
    if xp is not np:
        out = out + 0 * bias.sum()   # keep the autograd graph connected when bias is unused
    for a in range(k0):
        for b in range(k1):
            for c in range(k2):
                contrib = xp.einsum("nixyz,io->noxyz", x, W[:, :, a, b, c])
                if xp is np:
                    out[:, :, a:a + D0, b:b + D1, c:c + D2] += contrib
                else:
                    pad = (c, k2 - 1 - c, b, k1 - 1 - b, a, k0 - 1 - a)
                    out = out + xp.nn.functional.pad(contrib, pad)
    return out + bias.reshape(1, Cout, 1, 1, 1)


def sigmoid(a, xp=np):
    return 1.0 / (1.0 + xp.exp(-a))


def generator(params, z, xp=np):
    """SM Sec. II network: layers of (W, bias), each a transposed convolution followed by a
    sigmoid. z: [B, D0, D1, D2] (one input channel). Returns p: [B, L_tau, A, Bdim]."""
    h = z[:, None]
    for (W, bias) in params:
        h = sigmoid(conv_transpose3d(h, W, bias, xp), xp)
    return h[:, 0]


def fields_from_p(p):
    """Readings N2/N3: p [B, L_tau, A, Bdim] -> x [B, L_tau, N] with x = 2p - 1 and site
    i = a + A*b."""
    B, L, A, Bd = p.shape
    return (2.0 * p - 1.0).transpose(0, 1, 3, 2).reshape(B, L, A * Bd)


def generator_input(seed, n0, count, shape, stream=0):
    """Reading N5: +-1 inputs for samples n0 .. n0+count-1 of an input stream (0 for the
    training set, 1 for generation), float64 [count, *shape]."""
    k0, k1 = seed_key(seed)
    size = int(np.prod(shape))
    e = np.arange(size, dtype=np.uint64)[None, :]
    n = (n0 + np.arange(count, dtype=np.uint64))[:, None]
    w0 = philox4x32_10(e, n, stream, TAG_GEN_Z, k0, k1)[0]
    return np.where((w0 >> np.uint64(31)) != 0, -1.0, 1.0).reshape((count,) + tuple(shape))


def glorot_params(seed, arch):
    """Reading N8. arch: list of (Cin, Cout, (k0, k1, k2)) per layer."""
    k0, k1 = seed_key(seed)
    params = []
    for layer, (cin, cout, ks) in enumerate(arch):
        rf = int(np.prod(ks))
        limit = np.sqrt(6.0 / (cin * rf + cout * rf))
        size = cin * cout * rf
        w0 = philox4x32_10(np.arange(size, dtype=np.uint64), layer, 0, TAG_PARAM, k0, k1)[0]
        u = w0.astype(np.float64) * 2.0 ** -32
        W = ((2.0 * u - 1.0) * limit).reshape((cin, cout) + tuple(ks))
        params.append((W, np.zeros(cout)))
    return params


def bernoulli_fields(seed, p_flat, n0, stream=0):
    """Reading N6. p_flat: [B, L_tau, N] probabilities (as given); returns int8 +-1."""
    k0, k1 = seed_key(seed)
    B, L, N = p_flat.shape
    ctr = np.arange(L * N, dtype=np.uint64)[None, :]
    n = (n0 + np.arange(B, dtype=np.uint64))[:, None]
    u = philox4x32_10(ctr, n, stream, TAG_BERNOULLI, k0, k1)[0].astype(np.float64) * 2.0 ** -32
    p = np.asarray(p_flat, dtype=np.float64).reshape(B, L * N)
    return np.where(u < p, 1, -1).astype(np.int8).reshape(B, L, N)


# ----------------------------------------------------------------------------- loss

def observables(model, x, P=None):
    """Reading N3: (E_k, S) of one configuration with continuous fields x [L_tau, N]:
    the sweep's estimators (dqmc.measure) on G~ at slice 0, G_0 from the stabilized
    product over all slices (dqmc.green_scratch)."""
    P = P if P is not None else dqmc.Propagators(model)
    G = [dqmc.green_scratch(P, x, sigma, 0, model.n_wrap) for sigma in dqmc.SIGMAS]
    m = dqmc.measure(P, model, G[0], G[1])
    return m["ekin"], m["s_pipi"]


def loss(model, x, targets, w1, w2, P=None):
    """Eq. 4 over a batch. x: [B, L_tau, N]; targets: [B, 2] = (S_l, E_k,l)."""
    P = P if P is not None else dqmc.Propagators(model)
    total = 0.0
    for b in range(x.shape[0]):
        ek, s = observables(model, x[b], P)
        total += w1 * (s - targets[b][0]) ** 2 + w2 * (ek - targets[b][1]) ** 2
    return total


def loss_grad_fd(model, x, targets, w1, w2, entries, h=1e-5):
    """d Loss / d x at the given (b, l, i) entries by central differences (O(h^2))."""
    P = dqmc.Propagators(model)
    out = []
    for (b, l, i) in entries:
        xp_, xm_ = x[b].copy(), x[b].copy()
        xp_[l, i] += h
        xm_[l, i] -= h
        tb = targets[b:b + 1]
        out.append((loss(model, xp_[None], tb, w1, w2, P) - loss(model, xm_[None], tb, w1, w2, P))
                   / (2 * h))
    return np.array(out)


def _torch_measure(torch, model, P, Gs):
    """dqmc.measure's E_k and S estimators written in torch ops (same formulas)."""
    N = model.N
    Eph = torch.from_numpy(P.expK_ph)
    Emh = torch.from_numpy(P.expK_mh)
    K = torch.from_numpy(P.K)
    Gt = [Eph @ G @ Emh for G in Gs]
    ekin = -sum(torch.trace(K @ g) for g in Gt) / N
    p = torch.from_numpy(dqmc.staggered_signs(model.Lx, model.Ly, model.lattice))
    eye = torch.eye(N, dtype=torch.float64)
    m = torch.diagonal(Gt[1]) - torch.diagonal(Gt[0])
    conn = sum(p @ ((eye - g.T) * g) @ p for g in Gt)
    s = 0.25 * ((p @ m) ** 2 + conn) / N
    return ekin, s


def loss_torch_naive(torch, model, x, targets, w1, w2):
    """Eq. 4 in torch float64 with G_0 = (I + B_{L-1} ... B_0)^{-1} by a plain inverse:
    differentiable, valid only where the plain product is well conditioned (small beta)."""
    P = dqmc.Propagators(model)
    Em = torch.from_numpy(P.expK_m)
    N = model.N
    total = 0.0
    for b in range(x.shape[0]):
        Gs = []
        for sigma in dqmc.SIGMAS:
            A = torch.eye(N, dtype=torch.float64)
            for l in range(model.L_tau):
                A = (Em * torch.exp(sigma * P.lam * x[b, l])[None, :]) @ A
            Gs.append(torch.linalg.inv(torch.eye(N, dtype=torch.float64) + A))
        ek, s = _torch_measure(torch, model, P, Gs)
        total = total + w1 * (s - targets[b][0]) ** 2 + w2 * (ek - targets[b][1]) ** 2
    return total


# ----------------------------------------------------------------------------- training

def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=ADAM_EPS):
    """Reading N7 (Kingma & Ba, Algorithm 1). Returns (theta, m, v) after step t (1-based)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def train_step_naive(model, params, state, t, z, targets, w1, w2, lr):
    """One Adam step on a batch (small beta: plain inverse), by automatic differentiation
    in torch float64 through generator and loss. state: list of (m, v) pairs per tensor.
    Returns (new params, new state, loss value, gradients)."""
    import torch
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True))
          for (W, b) in params]
    zt = torch.from_numpy(np.asarray(z, dtype=np.float64))
    p = generator(tp, zt, torch)
    Bn, L, A, Bd = p.shape
    x = (2.0 * p - 1.0).permute(0, 1, 3, 2).reshape(Bn, L, A * Bd)
    total = loss_torch_naive(torch, model, x, targets, w1, w2)
    total.backward()
    new, new_state, grads = [], [], []
    k = 0
    for (W, b) in tp:
        pair = []
        for tens in (W, b):
            g = tens.grad.numpy()
            th, m, v = adam_step(tens.detach().numpy(), g, state[k][0], state[k][1], t, lr)
            pair.append(th)
            new_state.append((m, v))
            grads.append(g)
            k += 1
        new.append(tuple(pair))
    return new, new_state, float(total.detach()), grads
