"""ctypes binding of libnmc (include/nmc.h): argument marshalling only.

Every function named ``nmc_*`` here calls the C entry point of the same name; failures
raise ``NmcError`` carrying the status and ``nmc_last_error``. All compute runs in the
library's CUDA kernels; there is no fallback: if ``libnmc.so`` is missing or cannot be
loaded, ``load()`` raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# the library this binding loads: the in-tree build, or another build of the same ABI named
# by NMC_LIB_PATH (e.g. the bounds-checked libnmc_debug.so)
LIB_PATH = os.environ.get("NMC_LIB_PATH") or os.path.join(HERE, "libnmc.so")

NMC_OK, NMC_EINVAL, NMC_ENOMEM, NMC_ECUDA, NMC_ENUMERIC, NMC_ETIMEOUT, NMC_ESTATE = range(7)
STATUS_NAMES = {0: "NMC_OK", 1: "NMC_EINVAL", 2: "NMC_ENOMEM", 3: "NMC_ECUDA",
                4: "NMC_ENUMERIC", 5: "NMC_ETIMEOUT", 6: "NMC_ESTATE"}
NMC_FP64, NMC_FP32, NMC_SPLIT_BF16, NMC_TF32X3, NMC_FP32X2 = 0, 1, 2, 3, 4
NMC_SQUARE, NMC_HONEYCOMB = 0, 1
LATTICES = {"square": NMC_SQUARE, "honeycomb": NMC_HONEYCOMB}

# every symbol include/nmc.h declares
EXPORTED = ("nmc_create", "nmc_configure", "nmc_default_options", "nmc_set_fields",
            "nmc_set_fields_device", "nmc_generate", "nmc_sweep", "nmc_sweep_async",
            "nmc_query", "nmc_sync", "nmc_footprint", "nmc_sweep_replay",
            "nmc_measure", "nmc_get_fields", "nmc_get_green", "nmc_get_dims",
            "nmc_checkpoint", "nmc_restore", "nmc_expk", "nmc_series", "nmc_philox", "nmc_philox_device",
            "nmc_drift_history", "nmc_profile", "nmc_kernel_stats", "nmc_graph_stats",
            "nmc_green_noalloc", "nmc_debug_fail_alloc", "nmc_fma_probe", "nmc_debug_product",
            "nmc_restart_chains", "nmc_series_range",
            "nmc_last_error",
            "nmc_version", "nmc_destroy", "nmc_debug_build", "nmc_debug_checks")


class NmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("n_chains", ctypes.c_int), ("delay_k", ctypes.c_int),
                ("precision", ctypes.c_int), ("drift_tol", ctypes.c_double),
                ("chain_offset", ctypes.c_longlong), ("cuda_stream", ctypes.c_void_p),
                ("ph_symmetric", ctypes.c_int), ("sweep_graphs", ctypes.c_int),
                ("stab_pairs", ctypes.c_int)]


class Est(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("err", ctypes.c_double)]


class Obs(ctypes.Structure):
    _fields_ = [("energy", Est), ("ekin", Est), ("double_occ", Est), ("s_pipi", Est),
                ("density", Est), ("sign", Est), ("accept", ctypes.c_double),
                ("max_drift", ctypes.c_double), ("n_meas", ctypes.c_longlong),
                ("n_disagree", ctypes.c_longlong)]

    def as_dict(self):
        out = {}
        for k in ("energy", "ekin", "double_occ", "s_pipi", "density", "sign"):
            e = getattr(self, k)
            out[k] = (e.mean, e.err)
        for k in ("accept", "max_drift", "n_meas", "n_disagree"):
            out[k] = getattr(self, k)
        return out


class GenArch(ctypes.Structure):
    _fields_ = [("z", ctypes.c_int * 3), ("c1", ctypes.c_int), ("k1", ctypes.c_int * 3),
                ("k2", ctypes.c_int * 3)]


EXPORTED_GEN = ("nmc_gen_paper_arch", "nmc_gen_create", "nmc_gen_get_params",
                "nmc_gen_set_params", "nmc_gen_probs", "nmc_gen_sample_fields",
                "nmc_gen_observables", "nmc_gen_generated_observables",
                "nmc_gen_loss_grad", "nmc_gen_train_step",
                "nmc_gen_train", "nmc_gen_steps", "nmc_gen_set_clip", "nmc_gen_last_error", "nmc_gen_destroy")


EXPORTED_CGEN = ("nmc_cgen_create", "nmc_cgen_n_params", "nmc_cgen_get_params",
                 "nmc_cgen_set_params", "nmc_cgen_forward", "nmc_cgen_loss_grad",
                 "nmc_cgen_train_step", "nmc_cgen_sample", "nmc_cgen_destroy")


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("launches", ctypes.c_longlong),
                ("timed", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


_lib = None


def load():
    """Load libnmc.so (raises OSError/FileNotFoundError if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FileNotFoundError(f"{LIB_PATH} not built: run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    u32 = ctypes.c_uint32
    sig = {
        "nmc_create": (i, [i, i, i, d, d, d, d, i, ctypes.c_uint64, P(vp)]),
        "nmc_configure": (i, [vp, P(Options)]),
        "nmc_default_options": (None, [P(Options)]),
        "nmc_set_fields": (i, [vp, vp, sz]),
        "nmc_set_fields_device": (i, [vp, vp, sz]),
        "nmc_generate": (i, [vp, i, vp]),
        "nmc_sweep": (i, [vp, i, i]),
        "nmc_sweep_async": (i, [vp, i, i]),
        "nmc_query": (i, [vp, P(i)]),
        "nmc_sync": (i, [vp]),
        "nmc_footprint": (i, [i, i, i, d, d, d, d, i, P(Options), P(sz)]),
        "nmc_sweep_replay": (i, [vp, vp, sz, i]),
        "nmc_measure": (i, [vp, vp, P(Obs)]),
        "nmc_series": (i, [vp, vp, ctypes.c_longlong, P(ctypes.c_longlong)]),
        "nmc_get_fields": (i, [vp, vp, sz]),
        "nmc_get_green": (i, [vp, i, i, vp]),
        "nmc_get_dims": (i, [vp, P(i), P(i), P(i), P(i)]),
        "nmc_checkpoint": (i, [vp, vp, P(sz)]),
        "nmc_restore": (i, [vp, vp, sz]),
        "nmc_expk": (i, [i, i, i, d, d, vp]),
        "nmc_philox": (None, [u32, u32, u32, u32, u32, u32, P(u32)]),
        "nmc_philox_device": (i, [vp, i, u32, u32, u32, u32, u32, vp, vp]),
        "nmc_drift_history": (i, [vp, vp, ctypes.c_longlong, P(ctypes.c_longlong)]),
        "nmc_profile": (i, [vp, i]),
        "nmc_kernel_stats": (i, [vp, vp, i, P(i), i]),
        "nmc_graph_stats": (i, [vp, P(ctypes.c_longlong), P(ctypes.c_longlong)]),
        "nmc_green_noalloc": (i, [i, i, i, d, vp, vp, i, vp, vp]),
        "nmc_debug_fail_alloc": (None, [ctypes.c_longlong]),
        "nmc_fma_probe": (i, [i, i, i, i, vp, vp]),
        "nmc_restart_chains": (i, [vp, vp, vp, i]),
        "nmc_series_range": (i, [vp, ctypes.c_longlong, ctypes.c_longlong, vp]),
        "nmc_debug_product": (i, [i, i, i, i, vp, vp, vp, i, i, i, i, d, vp, vp]),
        "nmc_last_error": (ctypes.c_char_p, [vp]),
        "nmc_version": (ctypes.c_char_p, []),
        "nmc_debug_build": (i, []),
        "nmc_debug_checks": (ctypes.c_uint, []),
        "nmc_destroy": (None, [vp]),
        # include/nmc_gen.h
        "nmc_gen_paper_arch": (None, [P(GenArch)]),
        "nmc_gen_create": (i, [i, i, i, d, d, d, d, i, P(GenArch), ctypes.c_uint64, i, vp,
                               P(vp)]),
        "nmc_gen_get_params": (i, [vp, vp, vp, vp, vp]),
        "nmc_gen_set_params": (i, [vp, vp, vp, vp, vp]),
        "nmc_gen_probs": (i, [vp, ctypes.c_longlong, i, i, vp]),
        "nmc_gen_sample_fields": (i, [vp, ctypes.c_longlong, i, i, vp]),
        "nmc_gen_observables": (i, [vp, vp, i, vp]),
        "nmc_gen_loss_grad": (i, [vp, vp, i, vp, d, d, vp, vp]),
        "nmc_gen_generated_observables": (i, [vp, ctypes.c_longlong, i, i, vp]),
        "nmc_gen_train_step": (i, [vp, vp, i, vp, d, d, d, P(d)]),
        "nmc_gen_train": (i, [vp, vp, i, i, i, d, d, d, vp]),
        "nmc_gen_steps": (ctypes.c_longlong, [vp]),
        "nmc_gen_set_clip": (i, [vp, d]),
        "nmc_gen_last_error": (ctypes.c_char_p, [vp]),
        "nmc_gen_destroy": (None, [vp]),
        # include/nmc_cgen.h
        "nmc_cgen_create": (i, [i, i, i, i, ctypes.c_uint64, i, vp, P(vp)]),
        "nmc_cgen_n_params": (i, [vp, P(ctypes.c_longlong)]),
        "nmc_cgen_get_params": (i, [vp, vp]),
        "nmc_cgen_set_params": (i, [vp, vp]),
        "nmc_cgen_forward": (i, [vp, vp, i, vp]),
        "nmc_cgen_loss_grad": (i, [vp, vp, vp, i, P(d), vp]),
        "nmc_cgen_train_step": (i, [vp, vp, i, ctypes.c_longlong, ctypes.c_float, P(d)]),
        "nmc_cgen_sample": (i, [vp, ctypes.c_longlong, i, vp, vp]),
        "nmc_cgen_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(ctx, status):
    if status != NMC_OK:
        msg = load().nmc_last_error(ctx) if ctx else b""
        raise NmcError(status, (msg or b"").decode())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


# ------------------------------------------------------------------ raw entry points

def _lattice(lattice):
    return LATTICES[lattice] if isinstance(lattice, str) else int(lattice)


def n_sites(Lx, Ly, lattice=NMC_SQUARE):
    return Lx * Ly * (2 if _lattice(lattice) == NMC_HONEYCOMB else 1)


def nmc_create(Lx, Ly, t, U, beta, dtau, n_wrap, seed, lattice=NMC_SQUARE):
    ctx = ctypes.c_void_p()
    st = load().nmc_create(_lattice(lattice), Lx, Ly, t, U, beta, dtau, n_wrap, seed,
                           ctypes.byref(ctx))
    if st != NMC_OK:
        raise NmcError(st, "nmc_create rejected its arguments")
    return ctx


def nmc_default_options():
    o = Options()
    load().nmc_default_options(ctypes.byref(o))
    return o


def nmc_configure(ctx, opts=None):
    _check(ctx, load().nmc_configure(ctx, ctypes.byref(opts) if opts is not None else None))


def nmc_set_fields(ctx, s):
    s = np.ascontiguousarray(s, dtype=np.int8)
    _check(ctx, load().nmc_set_fields(ctx, _ptr(s), s.size))


def nmc_set_fields_device(ctx, dev_ptr, n):
    _check(ctx, load().nmc_set_fields_device(ctx, ctypes.c_void_p(dev_ptr), n))


def nmc_generate(ctx, mode=0, model=None):
    _check(ctx, load().nmc_generate(ctx, mode, model))


def nmc_sweep(ctx, n_sweeps, measure=1):
    _check(ctx, load().nmc_sweep(ctx, n_sweeps, measure))


def nmc_sweep_async(ctx, n_sweeps, measure=1):
    _check(ctx, load().nmc_sweep_async(ctx, n_sweeps, measure))


def nmc_query(ctx):
    idle = ctypes.c_int(0)
    _check(ctx, load().nmc_query(ctx, ctypes.byref(idle)))
    return bool(idle.value)


def nmc_sync(ctx):
    _check(ctx, load().nmc_sync(ctx))


def nmc_footprint(Lx, Ly, t, U, beta, dtau, n_wrap, opts=None, lattice=NMC_SQUARE):
    n = ctypes.c_size_t(0)
    st = load().nmc_footprint(_lattice(lattice), Lx, Ly, t, U, beta, dtau, n_wrap,
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(n))
    if st != NMC_OK:
        raise NmcError(st, "nmc_footprint")
    return n.value


def nmc_sweep_replay(ctx, accept, measure=1):
    a = np.ascontiguousarray(accept, dtype=np.uint8)
    _check(ctx, load().nmc_sweep_replay(ctx, _ptr(a), a.size, measure))


def nmc_get_dims(ctx):
    v = [ctypes.c_int() for _ in range(4)]
    _check(ctx, load().nmc_get_dims(ctx, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def nmc_measure(ctx, per_chain=False):
    _, _, n_chains, _ = nmc_get_dims(ctx)
    pooled = Obs()
    pc = (Obs * n_chains)() if per_chain else None
    _check(ctx, load().nmc_measure(ctx, ctypes.cast(pc, ctypes.c_void_p) if pc else None,
                                   ctypes.byref(pooled)))
    return (pooled, list(pc)) if per_chain else pooled


def nmc_get_fields(ctx):
    N, L, C, _ = nmc_get_dims(ctx)
    s = np.empty((C, L, N), dtype=np.int8)
    _check(ctx, load().nmc_get_fields(ctx, _ptr(s), s.size))
    return s


def nmc_get_green(ctx, chain, spin):
    N, _, _, _ = nmc_get_dims(ctx)
    G = np.empty((N, N), dtype=np.float64)
    _check(ctx, load().nmc_get_green(ctx, chain, spin, _ptr(G)))
    return G


def nmc_checkpoint(ctx):
    n = ctypes.c_size_t(0)
    _check(ctx, load().nmc_checkpoint(ctx, None, ctypes.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(ctx, load().nmc_checkpoint(ctx, _ptr(buf), ctypes.byref(n)))
    return buf.tobytes()


def nmc_restore(ctx, blob):
    buf = np.frombuffer(blob, dtype=np.uint8).copy()
    _check(ctx, load().nmc_restore(ctx, _ptr(buf), buf.size))


def nmc_expk(Lx, Ly, t, c, lattice=NMC_SQUARE):
    N = n_sites(Lx, Ly, lattice)
    out = np.empty((N, N), dtype=np.float64)
    st = load().nmc_expk(_lattice(lattice), Lx, Ly, t, c, _ptr(out))
    if st != NMC_OK:
        raise NmcError(st, "nmc_expk")
    return out


def nmc_series(ctx):
    """Per measured sweep and chain: (energy, ekin, double_occ, s_pipi, density) estimates,
    float64 [n_sweeps][n_chains][5] (sign-weighted sums over the sweep / sum of signs)."""
    n = ctypes.c_longlong(0)
    _check(ctx, load().nmc_series(ctx, None, 0, ctypes.byref(n)))
    C = nmc_get_dims(ctx)[2]
    buf = np.zeros((max(n.value, 1), C, 8), dtype=np.float64)
    _check(ctx, load().nmc_series(ctx, _ptr(buf), n.value, ctypes.byref(n)))
    buf = buf[:n.value]
    return buf[:, :, :5] / buf[:, :, 5:6]


def nmc_philox(c0, c1, c2, c3, k0, k1):
    out = (ctypes.c_uint32 * 4)()
    load().nmc_philox(c0, c1, c2, c3, k0, k1, out)
    return list(out)


def nmc_philox_device(d_c0_ptr, n, c1, c2, c3, k0, k1, d_out_ptr, stream=None):
    st = load().nmc_philox_device(ctypes.c_void_p(d_c0_ptr), n, c1, c2, c3, k0, k1,
                                  ctypes.c_void_p(d_out_ptr), stream)
    if st != NMC_OK:
        raise NmcError(st, "nmc_philox_device")


def nmc_drift_history(ctx, max_entries=4096):
    """Per-stabilization drift (max over chains), oldest first."""
    out = np.zeros(max_entries, dtype=np.float64)
    n = ctypes.c_longlong(0)
    _check(ctx, load().nmc_drift_history(ctx, _ptr(out), max_entries, ctypes.byref(n)))
    return out[:min(n.value, max_entries)].copy()


def nmc_profile(ctx, enable):
    _check(ctx, load().nmc_profile(ctx, int(bool(enable))))


def nmc_kernel_stats(ctx, reset=False):
    """{class: (launches, timed launches, total event ms)}"""
    arr = (KernelStat * 16)()
    n = ctypes.c_int(0)
    _check(ctx, load().nmc_kernel_stats(ctx, ctypes.cast(arr, ctypes.c_void_p), 16,
                                        ctypes.byref(n), int(bool(reset))))
    return {arr[k].name.decode(): (arr[k].launches, arr[k].timed, arr[k].total_ms)
            for k in range(n.value)}


def nmc_green_noalloc(N, L_tau, n_wrap, lam, d_expK_ptr, d_fields_ptr, n_chains, d_G_ptr,
                      stream=None):
    """G_0 of every chain and spin from device fields into device d_G, using only the
    library's fixed scratch array (no device allocation). Pointers are device addresses."""
    st = load().nmc_green_noalloc(N, L_tau, n_wrap, lam, ctypes.c_void_p(d_expK_ptr),
                                  ctypes.c_void_p(d_fields_ptr), n_chains,
                                  ctypes.c_void_p(d_G_ptr), stream)
    if st != NMC_OK:
        raise NmcError(st, "nmc_green_noalloc")


def nmc_graph_stats(ctx):
    """(sweep graphs recorded, sweeps replayed from a recorded graph) since creation."""
    rec, rep = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(ctx, load().nmc_graph_stats(ctx, ctypes.byref(rec), ctypes.byref(rep)))
    return rec.value, rep.value


def nmc_debug_fail_alloc(n):
    """Make the n-th device allocation from now fail with NMC_ENOMEM (0 = off)."""
    load().nmc_debug_fail_alloc(int(n))


def nmc_fma_probe(kind, blocks, threads, iters, d_out_ptr, stream=None):
    """Launch the FP64 (kind 0) / FP32 (kind 1) multiply-add probe on `stream`."""
    st = load().nmc_fma_probe(kind, blocks, threads, iters, ctypes.c_void_p(d_out_ptr), stream)
    if st != NMC_OK:
        raise NmcError(st, "nmc_fma_probe")


def nmc_debug_product(precision, cst, X, const_is_a, fields=None, br=0, bc=0, cr=0, cc=0,
                      lam=0.0, colscale=None):
    """One batched product of the compensated modes on host arrays (testing hook):
    C[b] = cst @ X[b] (const_is_a) or X[b] @ cst, with the optional field and column
    scalings of include/nmc.h. Returns C as float64 [batch][N][N]."""
    cst = np.ascontiguousarray(cst, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    batch, N, _ = X.shape
    C = np.empty_like(X)
    f = None if fields is None else np.ascontiguousarray(fields, dtype=np.int8)
    cs = None if colscale is None else np.ascontiguousarray(colscale, dtype=np.float64)
    st = load().nmc_debug_product(int(precision), N, batch, int(bool(const_is_a)), _ptr(cst),
                                  _ptr(X), None if f is None else _ptr(f), br, bc, cr, cc,
                                  float(lam), None if cs is None else _ptr(cs), _ptr(C))
    if st != NMC_OK:
        raise NmcError(st, "nmc_debug_product")
    return C


def nmc_restart_chains(ctx, chains, global_ids):
    """Start the given local chains afresh with the given global chain indices."""
    c = np.ascontiguousarray(chains, dtype=np.int32)
    g = np.ascontiguousarray(global_ids, dtype=np.int64)
    if c.shape != g.shape:
        raise ValueError("chains and global_ids differ in length")
    _check(ctx, load().nmc_restart_chains(ctx, _ptr(c), _ptr(g), int(c.size)))


def nmc_series_range(ctx, first, count):
    """Per-sweep accumulators of measured sweeps first .. first + count - 1:
    float64 [count][n_chains][8]."""
    _, _, C, _ = nmc_get_dims(ctx)
    out = np.zeros((int(count), C, 8))
    _check(ctx, load().nmc_series_range(ctx, int(first), int(count), _ptr(out)))
    return out


def nmc_destroy(ctx):
    load().nmc_destroy(ctx)


def nmc_version():
    return load().nmc_version().decode()


# ------------------------------------------------------------------ convenience

class Context:
    """Owning wrapper: ``with Context(...) as c: c.generate(); c.sweep(10)``."""

    def __init__(self, Lx, Ly, t, U, beta, dtau, n_wrap, seed=0, n_chains=1, delay_k=16,
                 precision=NMC_FP64, drift_tol=0.0, chain_offset=0, stream=None,
                 ph_symmetric=0, lattice=NMC_SQUARE, sweep_graphs=1, stab_pairs=0):
        self.ctx = nmc_create(Lx, Ly, t, U, beta, dtau, n_wrap, seed, lattice)
        o = nmc_default_options()
        o.n_chains, o.delay_k, o.precision = n_chains, delay_k, precision
        o.drift_tol, o.chain_offset = drift_tol, chain_offset
        o.cuda_stream = stream
        o.ph_symmetric = int(ph_symmetric)
        o.sweep_graphs = int(sweep_graphs)
        o.stab_pairs = int(stab_pairs)
        try:
            nmc_configure(self.ctx, o)
        except Exception:
            ctx, self.ctx = self.ctx, None
            nmc_destroy(ctx)
            raise

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def close(self):
        if self.ctx is not None:
            nmc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    dims = property(lambda self: nmc_get_dims(self.ctx))

    def set_fields(self, s):
        nmc_set_fields(self.ctx, s)

    def generate(self, mode=0, model=None):
        """mode 0: random fields; mode 1: Bernoulli fields from a Generator (or its handle)."""
        if isinstance(model, Generator):
            model = model.g
        nmc_generate(self.ctx, mode, model)

    def sweep(self, n, measure=1):
        nmc_sweep(self.ctx, n, measure)

    def sweep_async(self, n, measure=1):
        nmc_sweep_async(self.ctx, n, measure)

    def idle(self):
        return nmc_query(self.ctx)

    def sync(self):
        nmc_sync(self.ctx)

    def sweep_replay(self, accept, measure=1):
        nmc_sweep_replay(self.ctx, accept, measure)

    def measure(self, per_chain=False):
        return nmc_measure(self.ctx, per_chain)

    def series(self):
        return nmc_series(self.ctx)

    def fields(self):
        return nmc_get_fields(self.ctx)

    def green(self, chain, spin):
        return nmc_get_green(self.ctx, chain, spin)

    def checkpoint(self):
        return nmc_checkpoint(self.ctx)

    def restore(self, blob):
        nmc_restore(self.ctx, blob)

    def drift_history(self, max_entries=4096):
        return nmc_drift_history(self.ctx, max_entries)

    def profile(self, enable):
        nmc_profile(self.ctx, enable)

    def kernel_stats(self, reset=False):
        return nmc_kernel_stats(self.ctx, reset)

    def graph_stats(self):
        return nmc_graph_stats(self.ctx)

    def restart_chains(self, chains, global_ids):
        nmc_restart_chains(self.ctx, chains, global_ids)

    def series_range(self, first, count):
        return nmc_series_range(self.ctx, first, count)


# ------------------------------------------------------------------ generator (nmc_gen.h)

def gen_arch(z=None, c1=None, k1=None, k2=None):
    """The paper's honeycomb network (SM Sec. II), with any field overridden."""
    a = GenArch()
    load().nmc_gen_paper_arch(ctypes.byref(a))
    if z is not None:
        a.z[:] = list(z)
    if c1 is not None:
        a.c1 = int(c1)
    if k1 is not None:
        a.k1[:] = list(k1)
    if k2 is not None:
        a.k2[:] = list(k2)
    return a


def _gcheck(g, status):
    if status != NMC_OK:
        msg = load().nmc_gen_last_error(g) if g else b""
        raise NmcError(status, (msg or b"").decode())


class ConvGenerator:
    """Owning wrapper of an nmc_cgen: four periodic 3D convolutions (1 -> C -> C -> C -> 1
    channels) from N(0,1) noise to Bernoulli logits per field entry, trained by maximum
    likelihood (include/nmc_cgen.h). Device-pointer arguments are integers (e.g. torch
    ``data_ptr()``); arrays of noise, logits and fields are [n][L_tau][Ly][Lx]."""

    def __init__(self, Lx, Ly, L_tau, channels=32, seed=0, max_batch=64, stream=None):
        h = ctypes.c_void_p()
        st = load().nmc_cgen_create(Lx, Ly, L_tau, channels, seed, max_batch, stream,
                                    ctypes.byref(h))
        if st != NMC_OK:
            raise NmcError(st, "nmc_cgen_create rejected its arguments")
        self.g = h
        self.shape = (L_tau, Ly, Lx)
        self.C = channels
        self.max_batch = max_batch

    def _check(self, st, what):
        if st != NMC_OK:
            raise NmcError(st, what)

    def n_params(self):
        n = ctypes.c_longlong(0)
        self._check(load().nmc_cgen_n_params(self.g, ctypes.byref(n)), "nmc_cgen_n_params")
        return n.value

    def get_params(self):
        th = np.empty(self.n_params(), dtype=np.float32)
        self._check(load().nmc_cgen_get_params(self.g, _ptr(th)), "nmc_cgen_get_params")
        return th

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        if th.size != self.n_params():
            raise ValueError("parameter count")
        self._check(load().nmc_cgen_set_params(self.g, _ptr(th)), "nmc_cgen_set_params")

    def params(self):
        """[(W, b)] per layer from the flat FP32 array (layouts of include/nmc_cgen.h)."""
        th = self.get_params().astype(np.float64)
        C, out, o = self.C, [], 0
        for ci, co in ((1, C), (C, C), (C, C), (C, 1)):
            W = th[o:o + co * ci * 27].reshape(co, ci, 3, 3, 3)
            o += co * ci * 27
            b = th[o:o + co]
            o += co
            out.append((W, b))
        return out

    def forward(self, d_z, n, d_logits):
        self._check(load().nmc_cgen_forward(self.g, d_z, n, d_logits), "nmc_cgen_forward")

    def loss_grad(self, d_z, d_fields, n, d_grad):
        loss = ctypes.c_double(0.0)
        self._check(load().nmc_cgen_loss_grad(self.g, d_z, d_fields, n, ctypes.byref(loss),
                                              d_grad), "nmc_cgen_loss_grad")
        return loss.value

    def train_step(self, d_fields, n, sample0, lr):
        loss = ctypes.c_double(0.0)
        self._check(load().nmc_cgen_train_step(self.g, d_fields, n, sample0, lr,
                                               ctypes.byref(loss)), "nmc_cgen_train_step")
        return loss.value

    def sample(self, n0, n, d_fields, d_logits=None):
        self._check(load().nmc_cgen_sample(self.g, n0, n, d_fields, d_logits),
                    "nmc_cgen_sample")

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def close(self):
        if self.g is not None:
            load().nmc_cgen_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Generator:
    """Owning wrapper of an nmc_gen (generator network, Eq. 4 loss and training).
    Device-pointer arguments are integers (e.g. torch ``data_ptr()``)."""

    def __init__(self, Lx, Ly, t, U, beta, dtau, n_wrap, arch=None, seed=0, max_batch=64,
                 stream=None, lattice=NMC_SQUARE):
        self.arch = arch if arch is not None else gen_arch()
        h = ctypes.c_void_p()
        st = load().nmc_gen_create(_lattice(lattice), Lx, Ly, t, U, beta, dtau, n_wrap,
                                   ctypes.byref(self.arch), seed, max_batch, stream,
                                   ctypes.byref(h))
        if st != NMC_OK:
            raise NmcError(st, "nmc_gen_create rejected its arguments")
        self.g = h
        a = self.arch
        self.k1 = tuple(a.k1)
        self.k2 = tuple(a.k2)
        self.z_shape = tuple(a.z)
        self.c1 = a.c1
        self.L_tau = a.z[0] + a.k1[0] + a.k2[0] - 2
        self.A = a.z[1] + a.k1[1] + a.k2[1] - 2
        self.B = a.z[2] + a.k1[2] + a.k2[2] - 2
        self.N = self.A * self.B

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def close(self):
        if self.g is not None:
            load().nmc_gen_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        W1 = np.zeros((1, self.c1) + self.k1, dtype=np.float32)
        b1 = np.zeros(self.c1, dtype=np.float32)
        W2 = np.zeros((self.c1, 1) + self.k2, dtype=np.float32)
        b2 = np.zeros(1, dtype=np.float32)
        _gcheck(self.g, load().nmc_gen_get_params(self.g, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2)))
        return [(W1, b1), (W2, b2)]

    def set_params(self, params):
        (W1, b1), (W2, b2) = [(np.ascontiguousarray(W, dtype=np.float32),
                               np.ascontiguousarray(b, dtype=np.float32)) for (W, b) in params]
        _gcheck(self.g, load().nmc_gen_set_params(self.g, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2)))

    def probs(self, n0, n, stream_id, d_p):
        _gcheck(self.g, load().nmc_gen_probs(self.g, n0, n, stream_id, ctypes.c_void_p(d_p)))

    def sample_fields(self, n0, n, stream_id, d_fields):
        _gcheck(self.g, load().nmc_gen_sample_fields(self.g, n0, n, stream_id,
                                                     ctypes.c_void_p(d_fields)))

    def observables(self, d_x, n, d_obs):
        _gcheck(self.g, load().nmc_gen_observables(self.g, ctypes.c_void_p(d_x), n,
                                                   ctypes.c_void_p(d_obs)))

    def generated_observables(self, n0, n, stream_id, d_obs):
        _gcheck(self.g, load().nmc_gen_generated_observables(self.g, n0, n, stream_id,
                                                             ctypes.c_void_p(d_obs)))

    def loss_grad(self, d_x, n, d_targets, w1, w2, d_loss=0, d_grad=0):
        _gcheck(self.g, load().nmc_gen_loss_grad(self.g, ctypes.c_void_p(d_x), n,
                                                 ctypes.c_void_p(d_targets), w1, w2,
                                                 ctypes.c_void_p(d_loss or None),
                                                 ctypes.c_void_p(d_grad or None)))

    def train_step(self, ids, targets, w1, w2, lr):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        tg = np.ascontiguousarray(targets, dtype=np.float64)
        out = ctypes.c_double(0)
        _gcheck(self.g, load().nmc_gen_train_step(self.g, _ptr(ids), len(ids), _ptr(tg), w1, w2,
                                                  lr, ctypes.byref(out)))
        return out.value

    def train(self, targets, epochs, batch, lr=1e-3, w1=0.0, w2=0.0):
        tg = np.ascontiguousarray(targets, dtype=np.float64)
        out = np.zeros(max(epochs, 1), dtype=np.float64)
        _gcheck(self.g, load().nmc_gen_train(self.g, _ptr(tg), tg.shape[0], epochs, batch, lr,
                                             w1, w2, _ptr(out)))
        return out[:epochs]

    def steps(self):
        return load().nmc_gen_steps(self.g)

    def set_clip(self, max_norm):
        _gcheck(self.g, load().nmc_gen_set_clip(self.g, max_norm))
