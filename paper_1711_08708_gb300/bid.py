"""Python binding of libbid.so (ctypes): argument marshalling only.

Every computation runs in the C/CUDA library; this module converts numpy
arrays and torch tensors to the plain pointers and sizes of the C ABI
(include/bid.h) and raises ``BidError`` on a non-zero status.  There is no
fallback path: importing it without the built library raises ImportError.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbid.so")

OK, EINVAL, ENOCONV, ESTAGNATE, ECUDA, ETIMEOUT, ENOMEM = range(7)
FP64, FP32, BF16 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16}
SCHEMES = {"euler": 0, "cn": 1, "strang": 2}
ELLIPTIC = {"hchol": 0, "mg": 1}


class BidError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bid error {code}: {msg}")
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_nodes", C.c_int64), ("n_elems", C.c_int64),
                ("coords", C.c_void_p), ("elems", C.c_void_p), ("region", C.c_void_p),
                ("fibre", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("sigma_i", C.c_double * 3), ("sigma_e", C.c_double * 3), ("sigma_T", C.c_double),
                ("chi", C.c_double), ("Cm", C.c_double), ("tau_in", C.c_double),
                ("tau_out", C.c_double), ("tau_open", C.c_double), ("tau_close", C.c_double),
                ("v_gate", C.c_double), ("v_rest", C.c_double), ("v_peak", C.c_double),
                ("stim_t_on", C.c_double), ("stim_t_off", C.c_double), ("mass_lumped", C.c_int32)]


class PrecondOpts(C.Structure):
    _fields_ = [("dt", C.c_double), ("eps", C.c_double), ("precision", C.c_int32),
                ("leaf_size", C.c_int32), ("block", C.c_int32), ("n_threads", C.c_int32),
                ("scheme", C.c_int32), ("elliptic", C.c_int32), ("gpu_build", C.c_int32)]


class PrecondStats(C.Structure):
    _fields_ = [("n1", C.c_int64), ("nk", C.c_int64), ("supernodes1", C.c_int64),
                ("supernodesk", C.c_int64), ("levels1", C.c_int32), ("levelsk", C.c_int32),
                ("dense_entries", C.c_int64), ("lowrank_entries", C.c_int64),
                ("factor_bytes", C.c_int64), ("bytes_p1", C.c_int64), ("bytes_pk", C.c_int64),
                ("alg_bytes_p1", C.c_int64), ("alg_bytes_pk", C.c_int64),
                ("lowrank_blocks", C.c_int64), ("dense_blocks", C.c_int64),
                ("build_seconds", C.c_double), ("dataflow_levels1", C.c_int32),
                ("dataflow_levelsk", C.c_int32), ("dataflow_first1", C.c_int32),
                ("dataflow_firstk", C.c_int32), ("large_levels1", C.c_int32),
                ("large_levelsk", C.c_int32), ("masked_dead1", C.c_int64),
                ("masked_clusters1", C.c_int64), ("alg_bytes_p1_masked", C.c_int64),
                ("flatp_levels1", C.c_int32), ("flatp_levelsk", C.c_int32),
                ("mid_clusters1", C.c_int64), ("mid_clustersk", C.c_int64),
                ("wide_clusters1", C.c_int64), ("wide_clustersk", C.c_int64),
                ("gram_pivots1", C.c_int64), ("gram_pivotsk", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("restarts", C.c_int32),
                ("relres", C.c_double), ("relres_true", C.c_double)]


_VP, _I, _D, _I64P = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_int64)

# name -> (restype, argtypes); every symbol include/bid.h declares
SIGNATURES = {
    "bid_assemble": (_I, [C.POINTER(Mesh), C.POINTER(Params), C.POINTER(_VP)]),
    "bid_system_sizes": (_I, [_VP, _I64P, _I64P, _I64P, _I64P]),
    "bid_get_perm": (_I, [_VP, _VP]),
    "bid_get_mass": (_I, [_VP, _VP, _VP]),
    "bid_precond_opts_default": (None, [C.POINTER(PrecondOpts)]),
    "bid_precond_build": (_I, [_VP, _D, _D, _I, C.POINTER(_VP)]),
    "bid_precond_build_ex": (_I, [_VP, C.POINTER(PrecondOpts), C.POINTER(_VP)]),
    "bid_precond_get_stats": (_I, [_VP, C.POINTER(PrecondStats)]),
    "bid_apply_lambda": (_I, [_VP, _D, _VP, _VP, _VP]),
    "bid_apply_precond": (_I, [_VP, _VP, _VP, _VP]),
    "bid_apply_factor": (_I, [_VP, _I, _VP, _VP, _VP]),
    "bid_apply_factor_noalloc": (_I, [_VP, _I, _VP, _VP, _VP]),
    "bid_profile_classes": (_I, [_VP, _I, _VP, _VP]),
    "bid_solve": (_I, [_VP, _VP, _VP, _VP, _D, _I, C.POINTER(SolveInfo), _VP]),
    "bid_step": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _D, _I, _D, _I, _VP, _VP]),
    "bid_rhs_gate": (_I, [_VP, _VP, _VP, _VP, _I, _VP, _VP]),
    "bid_normalise": (_I, [_VP, _VP, _VP]),
    "bid_destroy_system": (None, [_VP]),
    "bid_destroy_precond": (None, [_VP]),
    "bid_last_error": (C.c_char_p, []),
    "bid_kernel_launches": (C.c_int64, []),
    "bid_host_assemble": (_I, [C.POINTER(Mesh), C.POINTER(Params), C.POINTER(_VP)]),
    "bid_host_csr_size": (_I, [_VP, _I, _I64P, _I64P]),
    "bid_host_csr": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP]),
    "bid_host_factor_solve": (_I, [_VP, _I, _D, _D, _I, _I, _I, _VP, _VP, C.POINTER(PrecondStats)]),
    "bid_host_factor_solve_dataflow": (_I, [_VP, _I, _D, _D, _I, _I, _I, _I, _I, _VP, _VP,
                                            C.POINTER(PrecondStats), _I64P]),
    "bid_host_factor_solve_masked": (_I, [_VP, _D, _I, _I, _I, _VP, _VP, _I64P]),
    "bid_host_mg_solve": (_I, [_VP, _I, _D, _VP, _VP, _VP]),
    "bid_host_destroy": (None, [_VP]),
    "bid_batch_create": (_I, [_VP, _I, C.POINTER(PrecondOpts), _VP, C.POINTER(_VP)]),
    "bid_batch_layout": (_I, [_VP, _VP, _VP]),
    "bid_batch_get_stats": (_I, [_VP, C.POINTER(PrecondStats)]),
    "bid_batch_apply_factor": (_I, [_VP, _I, _VP, _VP, _VP]),
    "bid_batch_apply_precond": (_I, [_VP, _VP, _VP, _VP]),
    "bid_batch_solve": (_I, [_VP, _VP, _VP, _D, _I, _VP, _VP]),
    "bid_batch_step": (_I, [_VP, _VP, _VP, _VP, _D, _I, _D, _I, _VP, _VP]),
    "bid_batch_destroy": (None, [_VP]),
    "bid_tune_leaf": (_I, [_VP, C.POINTER(PrecondOpts), _VP, _I, _I, _VP, _VP]),
    "bid_tune_batch_leaf": (_I, [_VP, _I, C.POINTER(PrecondOpts), _VP, _I, _I, _VP]),
    "bid_host_batch_factor_solve": (_I, [_VP, _I, _I, _D, _D, _VP, _I, _I, _I, _I, _I, _I, _VP, _VP,
                                         C.POINTER(PrecondStats), _I64P]),
    "bid_cnn_nparams": (_I, []),
    "bid_cnn_create": (_I, [_I, C.c_uint64, C.POINTER(_VP)]),
    "bid_cnn_set_params": (_I, [_VP, _VP]),
    "bid_cnn_get_params": (_I, [_VP, _VP]),
    "bid_cnn_loss_grad": (_I, [_VP, _I, _VP, _VP, _I, _I, _I, _VP, _VP, _VP]),
    "bid_cnn_train_step": (_I, [_VP, _VP, _VP, _I, _I, _I, _D, _VP, _VP]),
    "bid_cnn_forward": (_I, [_VP, _I, _VP, _I, _I, _I, _VP, _VP]),
    "bid_cnn_destroy": (None, [_VP]),
    "bid_guess_create": (_I, [_VP, _VP, _I, _I, _VP, _I, C.POINTER(_VP)]),
    "bid_guess_push": (_I, [_VP, _VP, _VP, _VP]),
    "bid_guess_reset": (_I, [_VP]),
    "bid_guess_train": (_I, [_VP, _I, _I, _I, _D, C.c_uint64, _VP, _VP]),
    "bid_guess_scales": (_I, [_VP, _VP]),
    "bid_guess_configure": (_I, [_VP, _I, _I]),
    "bid_guess_predict": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "bid_step_learned": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _D, _I, _D, _I, _VP, _VP]),
    "bid_guess_destroy": (None, [_VP]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(rc):
    if rc != OK:
        raise BidError(rc, lib.bid_last_error().decode(errors="replace"))
    return rc


def _ptr(a):
    """Plain pointer of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _stream(stream=None):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def kernel_launches() -> int:
    return int(lib.bid_kernel_launches())


def make_params(p: dict) -> Params:
    q = Params()
    si = list(p["sigma_i"]) + [p["sigma_i"][-1]] * (3 - len(p["sigma_i"]))
    se = list(p["sigma_e"]) + [p["sigma_e"][-1]] * (3 - len(p["sigma_e"]))
    q.sigma_i = (C.c_double * 3)(*si)
    q.sigma_e = (C.c_double * 3)(*se)
    for k in ("sigma_T", "chi", "Cm", "tau_in", "tau_out", "tau_open", "tau_close", "v_gate",
              "v_rest", "v_peak"):
        setattr(q, k, float(p[k]))
    q.stim_t_on, q.stim_t_off = (float(t) for t in p.get("stim_t", (0.0, 1.0)))
    q.mass_lumped = 1
    return q


class _MeshArrays:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, mesh):
        self.coords = np.ascontiguousarray(mesh.coords, dtype=np.float64)
        self.elems = np.ascontiguousarray(mesh.elems, dtype=np.int32)
        self.region = np.ascontiguousarray(mesh.region, dtype=np.int32)
        self.fibre = np.ascontiguousarray(mesh.fibre, dtype=np.float64)
        self.s = Mesh(mesh.dim, self.coords.shape[0], self.elems.shape[0], self.coords.ctypes.data,
                      self.elems.ctypes.data, self.region.ctypes.data, self.fibre.ctypes.data)


class System:
    """bid_system: S_1, S_i, M, M_H assembled and resident on the current GPU."""

    def __init__(self, mesh, params: dict):
        self.params = dict(params)
        m = _MeshArrays(mesh)
        h = _VP()
        _check(lib.bid_assemble(C.byref(m.s), C.byref(make_params(params)), C.byref(h)))
        self.h = h
        N, NH, n1, ni = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.bid_system_sizes(h, C.byref(N), C.byref(NH), C.byref(n1), C.byref(ni)))
        self.N, self.NH, self.nnz_s1, self.nnz_si = N.value, NH.value, n1.value, ni.value
        self.perm = np.empty(self.N, dtype=np.int64)
        _check(lib.bid_get_perm(h, _ptr(self.perm)))
        self.m = np.empty(self.N)
        self.mH = np.empty(self.NH)
        _check(lib.bid_get_mass(h, _ptr(self.m), _ptr(self.mH)))

    def apply_lambda(self, gamma, x, y, stream=None):
        _check(lib.bid_apply_lambda(self.h, float(gamma), _ptr(x), _ptr(y), _stream(stream)))

    def __del__(self):
        if getattr(self, "h", None):
            lib.bid_destroy_system(self.h)
            self.h = None


def _opts(dt, eps, precision, leaf, block, threads, scheme="euler", elliptic="hchol", gpu_build=None):
    o = PrecondOpts()
    lib.bid_precond_opts_default(C.byref(o))
    o.dt, o.eps = float(dt), float(eps)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.leaf_size, o.block, o.n_threads = int(leaf), int(block), int(threads)
    o.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    o.elliptic = ELLIPTIC[elliptic] if isinstance(elliptic, str) else int(elliptic)
    if gpu_build is not None:
        o.gpu_build = int(bool(gpu_build))
    return o


class Precond:
    """bid_precond: P_Lambda for one time step dt, plus the PCG work vectors."""

    def __init__(self, system: System, dt, eps=0.0, precision="fp64", leaf=16, block=128,
                 threads=0, scheme="euler", elliptic="hchol", gpu_build=None):
        o = _opts(dt, eps, precision, leaf, block, threads, scheme, elliptic, gpu_build)
        h = _VP()
        _check(lib.bid_precond_build_ex(system.h, C.byref(o), C.byref(h)))
        self.h, self.system, self.dt = h, system, float(dt)
        st = PrecondStats()
        _check(lib.bid_precond_get_stats(h, C.byref(st)))
        self.stats = st.as_dict()

    def apply(self, r, z, stream=None):
        _check(lib.bid_apply_precond(self.h, _ptr(r), _ptr(z), _stream(stream)))

    def apply_factor(self, which, b, x, stream=None):
        _check(lib.bid_apply_factor(self.h, int(which), _ptr(b), _ptr(x), _stream(stream)))

    def apply_factor_noalloc(self, which, b, x, stream=None, check=True):
        """bid_apply_factor without any allocation: scratch comes from the
        library's static 16 MiB device array (for callers that cannot call
        cudaMalloc when they solve, e.g. a real-time loop or a fixed memory
        budget).  Returns the status code."""
        rc = lib.bid_apply_factor_noalloc(self.h, int(which), _ptr(b), _ptr(x), _stream(stream))
        if check:
            _check(rc)
        return rc

    def solve(self, Y, X, tol=1e-8, max_iter=200, stream=None, check=True):
        info = SolveInfo()
        rc = lib.bid_solve(self.system.h, self.h, _ptr(Y), _ptr(X), float(tol), int(max_iter),
                           C.byref(info), _stream(stream))
        if check:
            _check(rc)
        return dict(iters=info.iters, status=info.status, restarts=info.restarts,
                    relres=info.relres, relres_true=info.relres_true, rc=rc)

    def step(self, U, V, h, Ist, t0, n_steps, tol=1e-8, max_iter=200, stream=None):
        iters = np.zeros(max(n_steps, 1), dtype=np.int32)
        _check(lib.bid_step(self.system.h, self.h, _ptr(U), _ptr(V), _ptr(h), _ptr(Ist),
                            float(t0), int(n_steps), float(tol), int(max_iter), _ptr(iters),
                            _stream(stream)))
        return iters[:n_steps]

    PROFILE_CLASSES = ("lambda", "p1_solve", "p1_masked", "pk_solve", "si_chain", "pcg_vectors",
                       "residual", "rhs_gate", "normalise")

    def profile_classes(self, reps=10, stream=None):
        """bid_profile_classes: mean ms of one launch of each kernel class
        (overwrites the work vectors; blocking)."""
        ms = np.zeros(len(self.PROFILE_CLASSES))
        _check(lib.bid_profile_classes(self.h, int(reps), _ptr(ms), _stream(stream)))
        return dict(zip(self.PROFILE_CLASSES, ms.tolist()))

    def rhs_gate(self, V, h, Ist, stim_on, Y, stream=None):
        _check(lib.bid_rhs_gate(self.h, _ptr(V), _ptr(h), _ptr(Ist), int(bool(stim_on)), _ptr(Y),
                                _stream(stream)))

    def normalise(self, X, stream=None):
        _check(lib.bid_normalise(self.h, _ptr(X), _stream(stream)))

    def __del__(self):
        if getattr(self, "h", None):
            lib.bid_destroy_precond(self.h)
            self.h = None


def tune_leaf(system: System, dt, eps=0.0, precision="fp64", block=128,
              candidates=(8, 16, 32, 64), reps=5):
    """bid_tune_leaf: the fastest leaf size of `system` among `candidates`
    (timed P_Lambda^-1 applications; cached per system size and options).
    Returns (best, {leaf: ms})."""
    o = _opts(dt, eps, precision, 16, block, 0)
    c = np.ascontiguousarray(candidates, dtype=np.int32)
    ms = np.zeros(c.size)
    best = np.zeros(1, dtype=np.int32)
    _check(lib.bid_tune_leaf(system.h, C.byref(o), _ptr(c), int(c.size), int(reps), _ptr(best),
                             _ptr(ms)))
    return int(best[0]), {int(k): float(v) for k, v in zip(c, ms)}


def tune_batch_leaf(systems, dt, eps=0.0, precision="fp64", block=128,
                    candidates=(8, 16, 32, 64), reps=5):
    """bid_tune_batch_leaf: one tuned leaf size per slice (size classes of
    half an octave, median slice of each class timed)."""
    S = len(systems)
    arr = (_VP * S)(*[s.h.value for s in systems])
    o = _opts(dt, eps, precision, 16, block, 0)
    c = np.ascontiguousarray(candidates, dtype=np.int32)
    out = np.zeros(S, dtype=np.int32)
    _check(lib.bid_tune_batch_leaf(arr, S, C.byref(o), _ptr(c), int(c.size), int(reps), _ptr(out)))
    return [int(v) for v in out]


class Batch:
    """bid_batch: independent slices advanced together (combined layout:
    slice s owns X[off[s]:off[s+1]] = [U_s | V_s] and h[hoff[s]:hoff[s+1]])."""

    def __init__(self, systems, dt, eps=0.0, precision="fp64", leaf=16, block=128, threads=0,
                 scheme="euler", elliptic="hchol"):
        self.systems = list(systems)
        S = len(self.systems)
        o = _opts(dt, eps, precision, leaf if np.isscalar(leaf) else 16, block, threads, scheme, elliptic)
        arr = (_VP * S)(*[s.h.value for s in self.systems])
        lf = None if np.isscalar(leaf) else np.ascontiguousarray(leaf, dtype=np.int32)
        h = _VP()
        _check(lib.bid_batch_create(arr, S, C.byref(o), _ptr(lf), C.byref(h)))
        self.h, self.S, self.dt = h, S, float(dt)
        self.leaf = [int(leaf)] * S if lf is None else [int(v) for v in lf]
        self.off = np.zeros(S + 1, dtype=np.int64)
        self.hoff = np.zeros(S + 1, dtype=np.int64)
        _check(lib.bid_batch_layout(h, _ptr(self.off), _ptr(self.hoff)))
        st = PrecondStats()
        _check(lib.bid_batch_get_stats(h, C.byref(st)))
        self.stats = st.as_dict()

    @property
    def n(self):
        return int(self.off[-1])

    def apply_factor(self, which, b, x, stream=None):
        _check(lib.bid_batch_apply_factor(self.h, int(which), _ptr(b), _ptr(x), _stream(stream)))

    def apply_precond(self, r, z, stream=None):
        _check(lib.bid_batch_apply_precond(self.h, _ptr(r), _ptr(z), _stream(stream)))

    def solve(self, Y, X, tol=1e-8, max_iter=200, stream=None, check=True):
        info = (SolveInfo * self.S)()
        rc = lib.bid_batch_solve(self.h, _ptr(Y), _ptr(X), float(tol), int(max_iter),
                                 C.cast(info, _VP), _stream(stream))
        if check:
            _check(rc)
        return [dict(iters=i.iters, status=i.status, restarts=i.restarts, relres=i.relres,
                     relres_true=i.relres_true) for i in info], rc

    def step(self, X, h, Ist, t0, n_steps, tol=1e-8, max_iter=200, stream=None):
        iters = np.zeros((max(n_steps, 1), self.S), dtype=np.int32)
        _check(lib.bid_batch_step(self.h, _ptr(X), _ptr(h), _ptr(Ist), float(t0), int(n_steps),
                                  float(tol), int(max_iter), _ptr(iters), _stream(stream)))
        return iters[:n_steps]

    def __del__(self):
        if getattr(self, "h", None):
            lib.bid_batch_destroy(self.h)
            self.h = None


class Cnn:
    """bid_cnn: the guess network (3 x 3 convolutions 6 -> 32 -> 32 -> 2)."""

    def __init__(self, max_pixels, seed=0):
        h = _VP()
        _check(lib.bid_cnn_create(int(max_pixels), int(seed), C.byref(h)))
        self.h = h
        self.nparams = int(lib.bid_cnn_nparams())

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float64)
        assert flat.size == self.nparams
        _check(lib.bid_cnn_set_params(self.h, _ptr(flat)))

    def get_params(self):
        out = np.empty(self.nparams)
        _check(lib.bid_cnn_get_params(self.h, _ptr(out)))
        return out

    def loss_grad(self, x, t, precision="fp64", stream=None):
        """x: device (B, H, W, 6), t: device (B, H, W, 2); returns (loss, grad)."""
        B, H, W = (int(v) for v in t.shape[:3])
        loss = np.zeros(1)
        grad = np.empty(self.nparams)
        _check(lib.bid_cnn_loss_grad(self.h, PRECISIONS[precision], _ptr(x), _ptr(t), B, H, W,
                                     _ptr(loss), _ptr(grad), _stream(stream)))
        return float(loss[0]), grad

    def train_step(self, x, t, lr, stream=None):
        B, H, W = (int(v) for v in t.shape[:3])
        loss = np.zeros(1)
        _check(lib.bid_cnn_train_step(self.h, _ptr(x), _ptr(t), B, H, W, float(lr), _ptr(loss),
                                      _stream(stream)))
        return float(loss[0])

    def forward(self, x, y, precision="bf16", stream=None):
        B, H, W = (int(v) for v in y.shape[:3])
        _check(lib.bid_cnn_forward(self.h, PRECISIONS[precision], _ptr(x), B, H, W, _ptr(y),
                                   _stream(stream)))

    def __del__(self):
        if getattr(self, "h", None):
            lib.bid_cnn_destroy(self.h)
            self.h = None


class Guess:
    """bid_guess: history of solved states on the grid + the network."""

    def __init__(self, system: System, net: Cnn, H, W, node_pixel=None, max_batch_pixels=1 << 18):
        if node_pixel is None:
            node_pixel = np.arange(H * W, dtype=np.int32)
        node_pixel = np.ascontiguousarray(node_pixel, dtype=np.int32)
        h = _VP()
        _check(lib.bid_guess_create(system.h, net.h, int(H), int(W), _ptr(node_pixel),
                                    int(max_batch_pixels), C.byref(h)))
        self.h, self.system, self.net = h, system, net

    def push(self, U, V, stream=None):
        _check(lib.bid_guess_push(self.h, _ptr(U), _ptr(V), _stream(stream)))

    def reset(self):
        _check(lib.bid_guess_reset(self.h))

    def configure(self, use_dv=True, policy=0):
        _check(lib.bid_guess_configure(self.h, int(bool(use_dv)), int(policy)))

    def train(self, ncrops=8, crop=128, iters=1, lr=1e-3, seed=0, stream=None):
        loss = np.zeros(1)
        _check(lib.bid_guess_train(self.h, int(ncrops), int(crop), int(iters), float(lr), int(seed),
                                   _ptr(loss), _stream(stream)))
        return float(loss[0])

    def scales(self):
        v = np.zeros(4)
        _check(lib.bid_guess_scales(self.h, _ptr(v)))
        return tuple(float(a) for a in v)

    def predict(self, U, V, X0, stream=None):
        _check(lib.bid_guess_predict(self.h, _ptr(U), _ptr(V), _ptr(X0), _stream(stream)))

    def step(self, P: "Precond", U, V, h, Ist, t0, n_steps, tol=1e-8, max_iter=200, stream=None):
        """bid_step_learned; returns an (n_steps, 4) array: iterations, initial
        residual of the previous-step guess, of the learned guess, used flag."""
        stats = np.zeros((max(n_steps, 1), 4))
        _check(lib.bid_step_learned(self.system.h, P.h, self.h, _ptr(U), _ptr(V), _ptr(h), _ptr(Ist),
                                    float(t0), int(n_steps), float(tol), int(max_iter), _ptr(stats),
                                    _stream(stream)))
        return stats[:n_steps]

    def __del__(self):
        if getattr(self, "h", None):
            lib.bid_guess_destroy(self.h)
            self.h = None


class HostSystem:
    """Host-only assembly and factor replay (no GPU needed)."""

    def __init__(self, mesh, params: dict):
        m = _MeshArrays(mesh)
        h = _VP()
        _check(lib.bid_host_assemble(C.byref(m.s), C.byref(make_params(params)), C.byref(h)))
        self.h = h

    def csr(self, which):
        n, nnz = C.c_int64(), C.c_int64()
        _check(lib.bid_host_csr_size(self.h, which, C.byref(n), C.byref(nnz)))
        ptr = np.empty(n.value + 1, dtype=np.int64)
        col = np.empty(nnz.value, dtype=np.int32)
        val = np.empty(nnz.value)
        _check(lib.bid_host_csr(self.h, which, _ptr(ptr), _ptr(col), _ptr(val), None, None, None))
        return ptr, col, val

    def perm_and_mass(self):
        n0, _ = C.c_int64(), C.c_int64()
        n1 = C.c_int64()
        _check(lib.bid_host_csr_size(self.h, 0, C.byref(n0), None))
        _check(lib.bid_host_csr_size(self.h, 1, C.byref(n1), None))
        perm = np.empty(n0.value, dtype=np.int64)
        m = np.empty(n0.value)
        mH = np.empty(n1.value)
        _check(lib.bid_host_csr(self.h, 0, None, None, None, _ptr(perm), _ptr(m), _ptr(mH)))
        return perm, m, mH

    def factor_solve(self, which, b, gamma=0.0, eps=0.0, leaf=16, block=128, precision="fp64"):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        st = PrecondStats()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lib.bid_host_factor_solve(self.h, int(which), float(gamma), float(eps), int(leaf),
                                         int(block), prec, _ptr(b), _ptr(x), C.byref(st)))
        return x, st.as_dict()

    def mg_solve(self, which, b, gamma=0.0):
        """bid_host_mg_solve: one multigrid V-cycle of S_1 (which = 1, on b minus
        its mean) or of K_m (which = 2) on the host; returns x and the levels."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        lv = C.c_int32()
        _check(lib.bid_host_mg_solve(self.h, int(which), float(gamma), _ptr(b), _ptr(x), C.byref(lv)))
        return x, int(lv.value)

    def factor_solve_masked(self, b, eps=0.0, leaf=16, block=128, precision="fp64"):
        """P_1 replay as the masked solve (b zero outside the heart nodes);
        returns x and (dead clusters, clusters)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        nd = np.zeros(2, dtype=np.int64)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lib.bid_host_factor_solve_masked(self.h, float(eps), int(leaf), int(block), prec, _ptr(b),
                                                _ptr(x), nd.ctypes.data_as(_I64P)))
        return x, (int(nd[0]), int(nd[1]))

    def factor_solve_dataflow(self, which, b, smem_cap=32768, first=1, gamma=0.0, eps=0.0, leaf=16,
                              block=128, precision="fp64"):
        """factor_solve with the flat levels from `first` on replayed in the
        dataflow kernels' signal order; returns x, stats and the schedule."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        st = PrecondStats()
        sched = np.zeros(5, dtype=np.int64)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lib.bid_host_factor_solve_dataflow(self.h, int(which), float(gamma), float(eps), int(leaf),
                                                  int(block), prec, int(smem_cap), int(first), _ptr(b),
                                                  _ptr(x), C.byref(st), sched.ctypes.data_as(_I64P)))
        return x, st.as_dict(), _schedule(sched)

    def __del__(self):
        if getattr(self, "h", None):
            lib.bid_host_destroy(self.h)
            self.h = None


def _schedule(sched):
    lev0, lev1, groups, df, db = (int(v) for v in sched)
    return {"first": lev0, "levels": lev1 - lev0, "groups": groups, "deps_fwd": df, "deps_bwd": db}


def host_batch_factor_solve(systems, which, b, gamma=0.0, eps=0.0, leaf=16, block=128,
                            precision="fp64", smem_cap=0, first=1, masked=False, schedule=False):
    """bid_host_batch_factor_solve over HostSystems (combined layout); the
    entries of the result outside the factor's block are zero.  smem_cap > 0
    replays the flat levels from `first` on in the dataflow kernels' order;
    masked=True (which = 1, b zero on the torso nodes) replays the masked
    forest solve; with schedule=True the schedule (levels, groups, forward and
    backward dependencies) is returned as a third value."""
    S = len(systems)
    arr = (_VP * S)(*[s.h.value for s in systems])
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    lf = None if np.isscalar(leaf) else np.ascontiguousarray(leaf, dtype=np.int32)
    st = PrecondStats()
    sched = np.zeros(5, dtype=np.int64)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib.bid_host_batch_factor_solve(arr, S, int(which), float(gamma), float(eps), _ptr(lf),
                                           int(leaf) if lf is None else 16, int(block), prec,
                                           int(smem_cap), int(first), int(bool(masked)), _ptr(b), _ptr(x),
                                           C.byref(st),
                                           sched.ctypes.data_as(_I64P)))
    if schedule:
        return x, st.as_dict(), _schedule(sched)
    return x, st.as_dict()
