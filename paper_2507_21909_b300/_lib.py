"""ctypes binding of libtrg (argument marshalling only; every step runs in CUDA)."""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_PATH = os.path.join(HERE, "libtrg.so")

TRG_PREC_FP64, TRG_PREC_BF16X3, TRG_PREC_BF16X6, TRG_PREC_BF16X10 = 0, 1, 2, 3
TRG_PREC_OZ4, TRG_PREC_OZ5, TRG_PREC_OZ6 = 4, 5, 6
TRG_PREC_TF32X3, TRG_PREC_OZ7 = 7, 8
EXPORTED = ["trg_init_ising", "trg_init_clock", "trg_step", "trg_free_energy",
            "trg_magnetisation_impurity", "trg_set_params", "trg_set_stream", "trg_diag",
            "trg_get_state", "trg_set_state", "trg_finalize", "trg_last_error",
            "trg_step_timings", "trg_gemm", "trg_kernel_stats", "trg_mem_stats",
            "trg_gemm_noalloc", "trg_sketch_set_net", "trg_sketch_get_net",
            "trg_sketch_forward", "trg_sketch_grad", "trg_sketch_train", "trg_set_sketch_mode",
            "trg_sketch_collect", "trg_sketch_fetch", "trg_sketch_stats", "trg_batch_create",
            "trg_batch_step", "trg_batch_results", "trg_batch_lanes", "trg_batch_free",
            "trg_gu_wen_ratio", "trg_batch_gu_wen", "trg_set_bond_overspan",
            "trg_set_impurity_pair", "trg_internal_energy", "trg_atrg_init_ising",
            "trg_atrg_step", "trg_atrg_free_energy", "trg_atrg_diag", "trg_get_scalars"]

TRG_SKETCH_IN, TRG_SKETCH_PARAMS = 5, 67585


class TrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtrg error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _PATH


def _load():
    if not os.path.exists(_PATH):
        raise ImportError(f"{_PATH} is missing: build it with `python -m paper_2507_21909_b300.build`")
    L = ctypes.CDLL(_PATH)
    d, i, ull, vp = ctypes.c_double, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_void_p
    pd, pi = ctypes.POINTER(d), ctypes.POINTER(i)
    ll, pf = ctypes.c_longlong, ctypes.POINTER(ctypes.c_float)
    pll = ctypes.POINTER(ll)
    sig = {
        "trg_init_ising": [i, d, d], "trg_init_clock": [i, i, d, d], "trg_step": [i, i, i],
        "trg_free_energy": [pd, pd], "trg_magnetisation_impurity": [pd],
        "trg_set_params": [i, i, ull, i], "trg_set_bond_overspan": [i], "trg_set_impurity_pair": [],
        "trg_internal_energy": [pd], "trg_atrg_init_ising": [i, d, d],
        "trg_atrg_step": [i, i, i], "trg_atrg_free_energy": [pd, pd], "trg_atrg_diag": [pd, pd, pi],
        "trg_set_stream": [vp], "trg_diag": [pd, pd, pi],
        "trg_get_state": [i, pi, pi, pd, ctypes.c_longlong],
        "trg_set_state": [d, pi, pd, pd, pd, pi, i, d], "trg_get_scalars": [pd, pd, pi], "trg_finalize": [],
        "trg_step_timings": [pd, i],
        "trg_mem_stats": [ctypes.POINTER(ctypes.c_longlong)] * 3,
        "trg_gemm_noalloc": [i, i, i, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, d,
                             vp, ctypes.c_longlong, vp, ctypes.c_longlong, d, vp,
                             ctypes.c_longlong, vp],
        "trg_kernel_stats": [pd, i, i],
        "trg_gemm": [i, i, i, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, d, pd,
                     ctypes.c_longlong, pd, ctypes.c_longlong, d, pd, ctypes.c_longlong],
        "trg_sketch_set_net": [pf, ll], "trg_sketch_get_net": [pf, ll],
        "trg_sketch_forward": [pf, ll, pf, i], "trg_sketch_grad": [pf, pf, ll, pd, pf],
        "trg_sketch_train": [pf, pf, ll, i, i, ctypes.c_float, ull, pd],
        "trg_set_sketch_mode": [i], "trg_sketch_collect": [ll],
        "trg_sketch_fetch": [pf, pf, ll, pll, pll], "trg_sketch_stats": [pll, pll, i],
        "trg_batch_create": [i, pi, pd, pd, pi, pi, ctypes.POINTER(ull), i, i, i, i],
        "trg_batch_step": [i, pd], "trg_batch_results": [pd, pd, pd, pi],
        "trg_batch_lanes": [pi, pll], "trg_batch_free": [],
        "trg_gu_wen_ratio": [pd], "trg_batch_gu_wen": [pd],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i
    L.trg_last_error.argtypes = []
    L.trg_last_error.restype = ctypes.c_char_p
    return L


lib = _load()


def _check(code):
    if code != 0:
        raise TrgError(code, lib.trg_last_error().decode())


def trg_init_ising(d, beta, h=0.0):
    _check(lib.trg_init_ising(int(d), float(beta), float(h)))


def trg_init_clock(d, q, beta, h=0.0):
    _check(lib.trg_init_clock(int(d), int(q), float(beta), float(h)))


def trg_step(axis, D, sketch_oversample):
    _check(lib.trg_step(int(axis), int(D), int(sketch_oversample)))


def trg_free_energy():
    f, lz = ctypes.c_double(), ctypes.c_double()
    _check(lib.trg_free_energy(ctypes.byref(f), ctypes.byref(lz)))
    return f.value, lz.value


def trg_magnetisation_impurity():
    m = ctypes.c_double()
    _check(lib.trg_magnetisation_impurity(ctypes.byref(m)))
    return m.value


def trg_set_params(q_swap=4, q_rho=4, seed=0x5EED, precision=TRG_PREC_FP64):
    _check(lib.trg_set_params(int(q_swap), int(q_rho), int(seed), int(precision)))


def trg_set_bond_overspan(r_bond=1):
    """ILO form: bond lines keep r_bond D values from the next step on (1 = plain)."""
    _check(lib.trg_set_bond_overspan(int(r_bond)))


def trg_set_impurity_pair():
    """Two-impurity network: the impurity on both sites of the first step's unit cell."""
    _check(lib.trg_set_impurity_pair())


def trg_internal_energy():
    """Ising coupling energy per site -d <s s'> from the merged impurity pair."""
    u = ctypes.c_double()
    _check(lib.trg_internal_energy(ctypes.byref(u)))
    return u.value


def trg_atrg_init_ising(d, beta, h=0.0):
    _check(lib.trg_atrg_init_ising(int(d), float(beta), float(h)))


def trg_atrg_step(axis, D, sketch_oversample):
    _check(lib.trg_atrg_step(int(axis), int(D), int(sketch_oversample)))


def trg_atrg_free_energy():
    f, lz = ctypes.c_double(), ctypes.c_double()
    _check(lib.trg_atrg_free_energy(ctypes.byref(f), ctypes.byref(lz)))
    return f.value, lz.value


def trg_atrg_diag():
    lc, gp, ns = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib.trg_atrg_diag(ctypes.byref(lc), ctypes.byref(gp), ctypes.byref(ns)))
    return lc.value, gp.value, ns.value


def trg_set_stream(stream_ptr=None):
    _check(lib.trg_set_stream(ctypes.c_void_p(stream_ptr or 0)))


def trg_diag():
    lc, g, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib.trg_diag(ctypes.byref(lc), ctypes.byref(g), ctypes.byref(n)))
    return lc.value, g.value, n.value


def trg_get_state(which):
    """Returns (array of shape (d1,d2,d3,d4,r), axes tuple); a three-dimensional state
    (reported by the library as (d1,d2,d3,1,r) with axes[3] = -1) comes back as
    (d1,d2,d3,r) with three axes."""
    dims = (ctypes.c_int * 5)()
    axes = (ctypes.c_int * 4)()
    _check(lib.trg_get_state(int(which), dims, axes, None, 0))
    shape = tuple(dims)
    out = np.empty(shape, dtype=np.float64)
    _check(lib.trg_get_state(int(which), dims, axes,
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size))
    if axes[3] == -1:
        return out.reshape(shape[:3] + shape[4:]), tuple(axes)[:3]
    return out, tuple(axes)


def trg_state_dims(which=0):
    """(d1, d2, d3, d4, r) of a state factor without copying it ((d1, d2, d3, r) in 3D)."""
    dims = (ctypes.c_int * 5)()
    axes = (ctypes.c_int * 4)()
    _check(lib.trg_get_state(int(which), dims, axes, None, 0))
    return tuple(dims)[:3] + tuple(dims)[4:] if axes[3] == -1 else tuple(dims)


def trg_get_scalars():
    """(beta, logsum, nsteps) of the current state."""
    b, ls, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib.trg_get_scalars(ctypes.byref(b), ctypes.byref(ls), ctypes.byref(n)))
    return b.value, ls.value, n.value


def save_state(path):
    """Write the current coarse-graining state (factors, axis order, beta, ln-norm sum,
    step count) to an .npz file; load_state resumes from it."""
    phi, axes = trg_get_state(0)
    psi, _ = trg_get_state(1)
    try:
        psi_imp, _ = trg_get_state(2)
    except TrgError:
        psi_imp = None
    beta, logsum, nsteps = trg_get_scalars()
    arrays = {"phi": phi, "psi": psi, "axes": np.asarray(axes, dtype=np.int64),
              "scalars": np.array([beta, logsum, nsteps], dtype=np.float64)}
    if psi_imp is not None:
        arrays["psi_imp"] = psi_imp
    np.savez(path, **arrays)


def load_state(path):
    with np.load(path) as z:
        beta, logsum, nsteps = z["scalars"]
        psi_imp = z["psi_imp"] if "psi_imp" in z.files else None
        trg_set_state(beta, z["phi"], z["psi"], psi_imp, tuple(int(a) for a in z["axes"]),
                      int(nsteps), logsum)


def trg_set_state(beta, phi, psi, psi_imp, axes, nsteps, logsum):
    """Load a state: 4D factors (d1,d2,d3,d4,r) with four axes, or 3D factors (d1,d2,d3,r)
    with three axes (passed to the library as (d1,d2,d3,1,r) with axes[3] = -1)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    if phi.shape != psi.shape or phi.ndim not in (4, 5):
        raise ValueError("phi and psi must have the same 4- or 5-leg shape")
    if phi.ndim == 4:
        if len(axes) != 3:
            raise ValueError("a three-dimensional state takes three axes")
        shape = phi.shape[:3] + (1,) + phi.shape[3:]
        axes = tuple(axes) + (-1,)
    else:
        shape = phi.shape
    dims = (ctypes.c_int * 5)(*shape)
    ax = (ctypes.c_int * 4)(*axes)
    P = ctypes.POINTER(ctypes.c_double)
    imp = None
    if psi_imp is not None:
        psi_imp = np.ascontiguousarray(psi_imp, dtype=np.float64)
        imp = psi_imp.ctypes.data_as(P)
    _check(lib.trg_set_state(float(beta), dims, phi.ctypes.data_as(P), psi.ctypes.data_as(P),
                             imp, ax, int(nsteps), float(logsum)))


PHASES = ("resplit", "bond_swap", "triad_isometries", "triads_envs", "squeezers",
          "contraction", "impurity", "norm")


def trg_step_timings():
    out = (ctypes.c_double * 8)()
    _check(lib.trg_step_timings(out, 8))
    return dict(zip(PHASES, list(out)))


def trg_gemm(A, B, precision=TRG_PREC_FP64, ta=False, tb=False, alpha=1.0, beta=0.0, C=None):
    """C = alpha op(A) op(B) + beta C on the device (numpy FP64 in and out)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M = A.shape[1] if ta else A.shape[0]
    K = A.shape[0] if ta else A.shape[1]
    N = B.shape[0] if tb else B.shape[1]
    if (B.shape[1] if tb else B.shape[0]) != K:
        raise ValueError("inner dimensions differ")
    C = np.zeros((M, N)) if C is None else np.ascontiguousarray(C, dtype=np.float64).copy()
    P = ctypes.POINTER(ctypes.c_double)
    _check(lib.trg_gemm(int(precision), int(ta), int(tb), M, N, K, float(alpha),
                        A.ctypes.data_as(P), A.shape[1], B.ctypes.data_as(P), B.shape[1],
                        float(beta), C.ctypes.data_as(P), N))
    return C


def trg_kernel_stats(reset=False):
    """Tensor-core GEMM counters: per kind (oz = exact-digit 3..6 digits, tc = split-BF16 or
    3xTF32, x7 = seven-digit FP64-equivalent) the device ms, algorithmic flop (2 M N K),
    tensor-pipe flop and launches; all library launches."""
    out = (ctypes.c_double * 13)()
    _check(lib.trg_kernel_stats(out, 13, int(reset)))
    v = list(out)
    return {"oz_ms": v[0], "oz_flop": v[1], "oz_pipe_flop": v[2], "oz_launches": int(v[3]),
            "tc_ms": v[4], "tc_flop": v[5], "tc_pipe_flop": v[6], "tc_launches": int(v[7]),
            "x7_ms": v[8], "x7_flop": v[9], "x7_pipe_flop": v[10], "x7_launches": int(v[11]),
            "launches": int(v[12])}


def trg_mem_stats():
    v = [ctypes.c_longlong() for _ in range(3)]
    _check(lib.trg_mem_stats(*[ctypes.byref(x) for x in v]))
    return {"in_use": v[0].value, "high_water": v[1].value, "reserved": v[2].value}


def trg_finalize():
    _check(lib.trg_finalize())


# ------------------------------------------------------------------ learned sketch
def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _pf(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def trg_sketch_set_net(params):
    """Load the sketch network (flat FP32 array of TRG_SKETCH_PARAMS values)."""
    p = _f32(params).reshape(-1)
    _check(lib.trg_sketch_set_net(_pf(p), p.size))


def trg_sketch_get_net():
    out = np.empty(TRG_SKETCH_PARAMS, dtype=np.float32)
    _check(lib.trg_sketch_get_net(_pf(out), out.size))
    return out


def trg_sketch_forward(X, bf16=True):
    X = _f32(X)
    u = np.empty(X.shape[0], dtype=np.float32)
    _check(lib.trg_sketch_forward(_pf(X), X.shape[0], _pf(u), int(bool(bf16))))
    return u


def trg_sketch_grad(X, t):
    X, t = _f32(X), _f32(t)
    g = np.empty(TRG_SKETCH_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _check(lib.trg_sketch_grad(_pf(X), _pf(t), X.shape[0], ctypes.byref(loss), _pf(g)))
    return loss.value, g


def trg_sketch_train(X, t, epochs, batch, lr, seed=0):
    X, t = _f32(X), _f32(t)
    loss = ctypes.c_double()
    _check(lib.trg_sketch_train(_pf(X), _pf(t), X.shape[0], int(epochs), int(batch),
                                float(lr), int(seed), ctypes.byref(loss)))
    return loss.value


def trg_set_sketch_mode(mode):
    _check(lib.trg_set_sketch_mode(int(mode)))


def trg_sketch_collect(capacity):
    _check(lib.trg_sketch_collect(int(capacity)))


def trg_sketch_fetch():
    rows, dropped = ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib.trg_sketch_fetch(None, None, 0, ctypes.byref(rows), ctypes.byref(dropped)))
    n = rows.value
    X = np.empty((max(n, 1), TRG_SKETCH_IN), dtype=np.float32)
    t = np.empty(max(n, 1), dtype=np.float32)
    _check(lib.trg_sketch_fetch(_pf(X), _pf(t), max(n, 1), ctypes.byref(rows),
                                ctypes.byref(dropped)))
    return X[:n], t[:n], dropped.value


def trg_sketch_stats(reset=False):
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib.trg_sketch_stats(ctypes.byref(a), ctypes.byref(b), int(reset)))
    return {"learned": a.value, "fallback": b.value}


# ------------------------------------------------------------------ batched instances
def trg_batch_create(model, beta, h, D, p=None, seed=None, lanes=4, q_swap=4, q_rho=4,
                     precision=TRG_PREC_FP64):
    """model[i]: 0 Ising or q (Z_q clock); arrays of equal length n."""
    n = len(model)
    md = np.ascontiguousarray(model, dtype=np.int32)
    bt = np.ascontiguousarray(beta, dtype=np.float64)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    dd = np.ascontiguousarray(D, dtype=np.int32)
    if not (len(bt) == len(hh) == len(dd) == n):
        raise ValueError("arrays must have equal length")
    pi_, pd_ = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    pp = None if p is None else np.ascontiguousarray(p, dtype=np.int32)
    sd = None if seed is None else np.ascontiguousarray(seed, dtype=np.uint64)
    _check(lib.trg_batch_create(
        n, md.ctypes.data_as(pi_), bt.ctypes.data_as(pd_), hh.ctypes.data_as(pd_),
        dd.ctypes.data_as(pi_), None if pp is None else pp.ctypes.data_as(pi_),
        None if sd is None else sd.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)),
        int(lanes), int(q_swap), int(q_rho), int(precision)))
    return n


def trg_batch_step(nsteps=1):
    ms = ctypes.c_double()
    _check(lib.trg_batch_step(int(nsteps), ctypes.byref(ms)))
    return ms.value


def trg_batch_results(n):
    f, lz, m = (np.empty(n) for _ in range(3))
    ns = np.empty(n, dtype=np.int32)
    pd_ = ctypes.POINTER(ctypes.c_double)
    _check(lib.trg_batch_results(f.ctypes.data_as(pd_), lz.ctypes.data_as(pd_),
                                 m.ctypes.data_as(pd_), ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return {"f": f, "lnz": lz, "m": m, "nsteps": ns}


def trg_batch_lanes(n, lanes):
    lane_of = np.empty(n, dtype=np.int32)
    scratch = np.empty(lanes, dtype=np.int64)
    _check(lib.trg_batch_lanes(lane_of.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               scratch.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))))
    return lane_of, scratch


def trg_batch_free():
    _check(lib.trg_batch_free())


def trg_gu_wen_ratio():
    x = ctypes.c_double()
    _check(lib.trg_gu_wen_ratio(ctypes.byref(x)))
    return x.value


def trg_batch_gu_wen(n):
    x = np.empty(n)
    _check(lib.trg_batch_gu_wen(x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return x
