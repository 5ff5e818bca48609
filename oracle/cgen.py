"""Oracle for the convolutional field generator. This is test infrastructure: only tests/,
__graft_entry__.smoke() and bench.py's CPU legs may import it. Plain numpy, FP64.

The generator is a second network for the initialization step of network-initialized Monte
Carlo, beside the paper's own network (nimc.py): it maps noise z ~ N(0,1) of the field's shape
(L_tau x Lx x Ly, one channel) to independent Bernoulli logits, one per field entry s(i, l),
through four periodic 3D convolutions with 3 x 3 x 3 kernels:

    h_0 = z,   h_{j+1} = relu(conv_j(h_j))  (j = 0, 1, 2; C channels),   logits = conv_3(h_3),
    conv(h)[co][p] = b[co] + sum_ci sum_{d in {-1,0,1}^3} W[co][ci][d + 1] h[ci][(p + d) mod shape]

(channels 1 -> C -> C -> C -> 1), and it is trained by maximum likelihood on fields the DQMC
produces: the loss of fields s (values +-1, y = (1 + s) / 2) given noise z is the mean over
samples and entries of the Bernoulli negative log-likelihood softplus(l) - y l.

The GPU kernels keep the operands of every convolution (z, the hidden activations, the
weights, and in the backward pass the gradients flowing in) in BF16 and accumulate in FP32;
`bf16` below rounds an array to the nearest BF16 value (ties to even), so a test can give
both sides the same BF16 operands.

The conventions (each written out from the definition above):
    d conv(h)[co][p] / d h[ci][q]      = W[co][ci][q - p + 1]   for q - p in {-1,0,1}^3,
    dL/dh[ci][q]   = sum_co sum_d W[co][ci][d + 1] g[co][(q - d) mod shape],
    dL/dW[co][ci][d + 1] = sum_p g[co][p] h[ci][(p + d) mod shape],
    dL/db[co]      = sum_p g[co][p],
with g = dL/dconv(h) and p ranging over every sample and entry.
"""
import numpy as np

OFFSETS = [(dt, dx, dy) for dt in (-1, 0, 1) for dx in (-1, 0, 1) for dy in (-1, 0, 1)]


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64. Inputs are
    finite; the rounding is done on the float32 bit pattern (bfloat16 is its upper half)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(h, d):
    """h[..., (p + d) mod shape] over the last three axes: out[p] = h[p + d]."""
    return np.roll(h, shift=(-d[0], -d[1], -d[2]), axis=(-3, -2, -1))


def conv(h, W, b):
    """h [n][Cin][T][X][Y], W [Cout][Cin][3][3][3], b [Cout] -> [n][Cout][T][X][Y]."""
    n, cin = h.shape[:2]
    cout = W.shape[0]
    out = np.broadcast_to(b[None, :, None, None, None], (n, cout) + h.shape[2:]).copy()
    for d in OFFSETS:
        hs = shift(h, d)                                   # [n][Cin][...]
        w = W[:, :, d[0] + 1, d[1] + 1, d[2] + 1]          # [Cout][Cin]
        out += np.einsum("oc,nctxy->notxy", w, hs)
    return out


def conv_bruteforce(h, W, b):
    """The same sum, entry by entry (for the pins only)."""
    n, cin, T, X, Y = h.shape
    cout = W.shape[0]
    out = np.zeros((n, cout, T, X, Y))
    for s in range(n):
        for co in range(cout):
            for t in range(T):
                for x in range(X):
                    for y in range(Y):
                        acc = b[co]
                        for ci in range(cin):
                            for (dt, dx, dy) in OFFSETS:
                                acc += (W[co, ci, dt + 1, dx + 1, dy + 1] *
                                        h[s, ci, (t + dt) % T, (x + dx) % X, (y + dy) % Y])
                        out[s, co, t, x, y] = acc
    return out


def conv_grad_input(g, W):
    """dL/dh from g = dL/dconv(h): sum_co sum_d W[co][ci][d] g[co][q - d]."""
    out = np.zeros((g.shape[0], W.shape[1]) + g.shape[2:])
    for d in OFFSETS:
        w = W[:, :, d[0] + 1, d[1] + 1, d[2] + 1]          # [Cout][Cin]
        gs = shift(g, (-d[0], -d[1], -d[2]))               # g[q - d]
        out += np.einsum("oc,notxy->nctxy", w, gs)
    return out


def conv_grad_weight(g, h):
    """dL/dW[co][ci][d] = sum_p g[co][p] h[ci][p + d]; dL/db[co] = sum_p g[co][p]."""
    gW = np.zeros((g.shape[1], h.shape[1], 3, 3, 3))
    for d in OFFSETS:
        gW[:, :, d[0] + 1, d[1] + 1, d[2] + 1] = np.einsum("notxy,nctxy->oc", g, shift(h, d))
    return gW, g.sum(axis=(0, 2, 3, 4))


def init_params(C, seed=0, scale=0.1):
    """Random parameters (layers 1 -> C -> C -> C -> 1) for tests."""
    rng = np.random.default_rng(seed)
    shapes = [(C, 1), (C, C), (C, C), (1, C)]
    return [(rng.normal(size=(co, ci, 3, 3, 3)) * scale, rng.normal(size=co) * scale)
            for co, ci in shapes]


def forward(params, z, round_bf16=False):
    """Logits [n][T][X][Y] and the hidden activations (inputs of each layer) for noise z
    [n][T][X][Y]. round_bf16: every convolution's inputs and weights are BF16 values, as in
    the kernels (the accumulation here stays FP64)."""
    r = bf16 if round_bf16 else (lambda a: a)
    h = r(z[:, None])
    acts = []
    for j, (W, b) in enumerate(params):
        acts.append(h)
        a = conv(h, r(W), b)
        h = r(np.maximum(a, 0.0)) if j < len(params) - 1 else a
    return h[:, 0], acts


def loss(logits, s):
    """Mean Bernoulli negative log-likelihood of fields s (+-1) under the logits."""
    y = (1.0 + s) / 2.0
    return float(np.mean(np.logaddexp(0.0, logits) - y * logits))


def loss_and_grads(params, z, s, round_bf16=False):
    """The loss and its gradients with respect to every W and b (backpropagation through the
    convolutions and the ReLUs). With round_bf16 the gradients flowing into each backward
    convolution are BF16 values too, as in the kernels."""
    r = bf16 if round_bf16 else (lambda a: a)
    logits, acts = forward(params, z, round_bf16)
    y = (1.0 + s) / 2.0
    g = (1.0 / (1.0 + np.exp(-logits)) - y) / logits.size     # dL/dlogits
    g = g[:, None]
    grads = [None] * len(params)
    for j in range(len(params) - 1, -1, -1):
        W, b = params[j]
        gq = r(g)
        gW, gb = conv_grad_weight(gq, acts[j])
        grads[j] = (gW, gb)
        if j > 0:
            g = conv_grad_input(gq, r(W)) * (acts[j] > 0)     # through relu of layer j - 1
    return loss(logits, s), grads


def optimal_bias(s):
    """With every weight zero the logits equal the last bias b for every entry, and the
    loss mean(softplus(b) - y b) is smallest where sigmoid(b) = mean(y): the log-odds of the
    fields' mean occupation."""
    y = np.mean((1.0 + s) / 2.0)
    return float(np.log(y / (1.0 - y)))
