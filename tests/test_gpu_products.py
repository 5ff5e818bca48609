"""The propagation products of the compensated modes, one launch at a time, against an FP64
reference on the CPU.

Each product of the sweep multiplies a chain matrix X (held as FP32 pairs) by a constant
(e^{-+dtau K} or e^{-+dtau K/2}) on the left or the right, with optional diagonal field
factors e^{sigma lam (.)} on the chain operand and on the output and an optional column
scale (the stack product B_l U D of the stabilization, SM Sec. I.2). The reference is the
plain FP64 product of the same FP32-pair-rounded operands. The bar: the error of every
entry, divided by K times the largest |entry| of its chain-operand row and of its constant
column (the scale the exact slicing works to), stays below 2^-42. Sizes span several
128-row tiles with a ragged last tile, every column-tile width and K chunking, and N up
to 320; the tcgen05 path and the SIMT FP32-pair path are both checked.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SPLIT_BF16, FP32X2 = 2, 4
BAR = 2.0 ** -42


@pytest.fixture(scope="module")
def nmc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_00712_gb300 import nmc as m
    m.load()
    return m


def _pair(x):
    hi = x.astype(np.float32).astype(np.float64)
    return hi + (x - hi).astype(np.float32).astype(np.float64)


def _inputs(nmc, N, batch, seed, lattice_const):
    rng = np.random.default_rng(seed)
    if lattice_const is not None:
        Lx, Ly, lat = lattice_const
        cst = nmc.nmc_expk(Lx, Ly, 1.0, -0.1, lat)
    else:
        cst = rng.normal(size=(N, N)) * 10.0 ** rng.uniform(-2, 2, size=(N, 1))
    # rows and columns over six decades, like G after the UDV scalings
    X = (rng.normal(size=(batch, N, N)) * 10.0 ** rng.uniform(-3, 3, size=(batch, N, 1))
         * 10.0 ** rng.uniform(-3, 3, size=(batch, 1, N)))
    fields = np.where(rng.random((batch // 2, N)) < 0.5, -1, 1).astype(np.int8)
    colscale = 10.0 ** rng.uniform(-5, 5, size=(batch, N))
    return cst, X, fields, colscale


def _reference(cst, X, const_is_a, fields, br, bc, cr, cc, lam, colscale):
    cstp, Xp = _pair(cst), _pair(X)
    out = np.empty_like(X)
    for b in range(X.shape[0]):
        sg = 1.0 if b % 2 == 0 else -1.0
        x = Xp[b]
        s = None if fields is None else fields[b // 2].astype(np.float64)
        if s is not None:
            x = x * np.exp(sg * lam * (br * s[:, None] + bc * s[None, :]))
        c = cstp @ x if const_is_a else x @ cstp
        if s is not None:
            c = c * np.exp(sg * lam * (cr * s[:, None] + cc * s[None, :]))
        if colscale is not None:
            c = c * colscale[b][None, :]
        out[b] = c
    return out


def _normalized_error(got, want, cst, X, const_is_a, fields, br, bc, lam, colscale,
                      cr, cc):
    """max |got - want| / (K * rowmax(chain operand) * colmax(constant)) in the product's
    own orientation, with the output factors divided out."""
    N = cst.shape[0]
    worst = 0.0
    for b in range(X.shape[0]):
        sg = 1.0 if b % 2 == 0 else -1.0
        x = np.abs(X[b])
        post = np.ones((N, N))
        if fields is not None:
            s = fields[b // 2].astype(np.float64)
            x = x * np.exp(sg * lam * (br * s[:, None] + bc * s[None, :]))
            post = np.exp(sg * lam * (cr * s[:, None] + cc * s[None, :]))
        if colscale is not None:
            post = post * colscale[b][None, :]
        if const_is_a:   # C = cst x: scale of C[r][c] = max_k |cst[r,k]| * max_k |x[k,c]|
            scale = np.abs(cst).max(axis=1)[:, None] * x.max(axis=0)[None, :]
        else:            # C = x cst: max_k |x[r,k]| * max_k |cst[k,c]|
            scale = x.max(axis=1)[:, None] * np.abs(cst).max(axis=0)[None, :]
        err = np.abs(got[b] - want[b]) / post / (N * np.maximum(scale, 1e-300))
        worst = max(worst, float(err.max()))
    return worst


CASES = [  # N, batch, lattice for the constant (None: a random dense matrix)
    (2, 70, (2, 1, 0)),
    (16, 18, (4, 4, 0)),
    (36, 10, (6, 6, 0)),
    (64, 10, (8, 8, 0)),
    (72, 8, (6, 6, 1)),
    (100, 6, (10, 10, 0)),
    (144, 4, (12, 12, 0)),
    (256, 2, (16, 16, 0)),
    (320, 2, None),
]


@pytest.mark.parametrize("prec", [SPLIT_BF16, FP32X2])
@pytest.mark.parametrize("N,batch,lat", CASES)
@pytest.mark.parametrize("const_is_a", [1, 0])
def test_product_matches_fp64_reference(nmc, prec, N, batch, lat, const_is_a):
    if prec == FP32X2 and N > 144:
        pytest.skip("the SIMT pair path is checked on the smaller sizes")
    cst, X, fields, colscale = _inputs(nmc, N, batch, seed=N + 7 * const_is_a, lattice_const=lat)
    lam = 0.6537   # acosh(e^{dtau U / 2}) at U = 4, dtau = 0.1
    # as the sweep uses them: staging factors on the chain operand when the constant is on the
    # left (e^{V} G e^{-V}), output factors when it is on the right (e^{-V} (T Em) e^{V})
    variants = [(None, 0, 0, 0, 0, None)]
    if const_is_a:
        variants.append((fields, 1, -1, 0, 0, None))
        variants.append((fields, 0, 0, 1, 0, colscale))
    else:
        variants.append((fields, 0, 0, -1, 1, None))
        variants.append((None, 0, 0, 0, 0, colscale))
    for f, br, bc, cr, cc, cs in variants:
        got = nmc.nmc_debug_product(prec, cst, X, const_is_a, fields=f, br=br, bc=bc, cr=cr,
                                    cc=cc, lam=lam, colscale=cs)
        want = _reference(cst, X, const_is_a, f, br, bc, cr, cc, lam, cs)
        assert np.all(np.isfinite(got))
        e = _normalized_error(got, want, cst, X, const_is_a, f, br, bc, lam, cs, cr, cc)
        assert e < BAR, (N, const_is_a, br, bc, cr, cc, e)


def test_tensor_core_product_refuses_sizes_beyond_exactness(nmc):
    """N = 324 (18 x 18) would let the group-2 slice sums pass 2^24 units: refused."""
    X = np.zeros((2, 324, 324))
    with pytest.raises(nmc.NmcError) as e:
        nmc.nmc_debug_product(SPLIT_BF16, np.eye(324), X, 1)
    assert e.value.status == nmc.NMC_EINVAL
    with pytest.raises(nmc.NmcError) as e:
        nmc.Context(18, 18, 1.0, 4.0, 0.2, 0.1, 2, precision=SPLIT_BF16)
    assert e.value.status == nmc.NMC_EINVAL
