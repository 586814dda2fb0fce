"""GB300 (sm_103a) gap filling of 2-D gridded data with the modified planar rotator (MPR) model.

Python binding of ``libmpr.so`` (C ABI in ``include/mpr.h``). The functions carry the C names
and only marshal arguments; every step of the method runs in the library's CUDA kernels. There
is no CPU fallback: if the library has not been built, every call raises.

Precision setups are named by the paper's three axes X_S X_E X_F (Sec. 2): spin storage, energy,
functions; D = FP64, S = FP32 (functions: hardware intrinsics); for storage also H = FP16 and
B = BF16; for functions also H = FP16 arithmetic where safe (FP16 spins only). E.g. "DDD" (all
FP64), "SDS" (FP32 spins, FP64 energy, FP32 intrinsics), "HDS", "HDH".
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libmpr.so")

MPR_OK = 0
MPR_ERR_INVALID_ARG = 1
MPR_ERR_DEGENERATE = 2
MPR_ERR_NO_PAIRS = 3
MPR_ERR_TUNE_NO_CONVERGE = 4
MPR_ERR_CUDA = 5
MPR_ERR_OOM = 6
MPR_ERR_DEVICE_TIMEOUT = 7
MPR_ERR_STATE = 8

STORE = {"D": 0, "S": 1, "H": 2, "B": 3}
PREC = {"D": 0, "S": 1}
FUNC = {"D": 0, "S": 1, "H": 2}   # X_F also has H: FP16 arithmetic where safe (FP16 spins only)
ACC = {"f64": 0, "kahan": 1}


class MPRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class mpr_options(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("q", ctypes.c_double), ("store", ctypes.c_int),
                ("energy", ctypes.c_int), ("func", ctypes.c_int), ("acc", ctypes.c_int)]


class mpr_tuning(ctypes.Structure):
    _fields_ = [("n_eq", ctypes.c_int), ("n_meas", ctypes.c_int), ("T_lo", ctypes.c_double),
                ("T_hi", ctypes.c_double), ("rel_tol", ctypes.c_double),
                ("ratio_tol", ctypes.c_double), ("max_probes", ctypes.c_int)]


class mpr_info(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("n_sites", ctypes.c_int64),
                ("n_pred", ctypes.c_int64), ("n_bonds", ctypes.c_int64),
                ("n_sample_pairs", ctypes.c_int64), ("zmin", ctypes.c_double),
                ("zmax", ctypes.c_double), ("e_sample", ctypes.c_double), ("T", ctypes.c_double),
                ("sweep", ctypes.c_uint32), ("n_samples", ctypes.c_int), ("n_probes", ctypes.c_int),
                ("e_bond_mean", ctypes.c_double), ("site_updates", ctypes.c_uint64),
                ("device_bytes", ctypes.c_size_t), ("kernel_launches", ctypes.c_uint64),
                ("prof_sweep_ms", ctypes.c_double), ("prof_sweep_launches", ctypes.c_uint64),
                ("sweep_kernel", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def load():
    """Loads libmpr.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        H = ctypes.c_void_p
        P = ctypes.POINTER
        vp, i, d, u32, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64
        sig = {
            "mpr_create": ([i, i, vp, vp, P(H)], i),
            "mpr_create_dev": ([i, i, vp, vp, vp, P(H)], i),
            "mpr_destroy": ([H], None),
            "mpr_trim_memory": ([], i),
            "mpr_set_options": ([H, P(mpr_options)], i),
            "mpr_get_options": ([H, P(mpr_options)], i),
            "mpr_set_stream": ([H, vp], i),
            "mpr_set_tuning": ([H, P(mpr_tuning)], i),
            "mpr_tune_temperature": ([H, P(d)], i),
            "mpr_set_temperature": ([H, d], i),
            "mpr_tune_heating": ([H, d, P(d)], i),
            "mpr_energy_curve": ([i, i, P(mpr_options), P(mpr_tuning), vp, i, vp], i),
            "mpr_tune_from_curve": ([H, vp, vp, i, P(d)], i),
            "mpr_run": ([H, i, i], i),
            "mpr_run_auto": ([H, i, i, i, P(i)], i),
            "mpr_predict": ([H, vp], i),
            "mpr_predict_dev": ([H, vp], i),
            "mpr_energy": ([H, P(d), P(d)], i),
            "mpr_get_info": ([H, P(mpr_info)], i),
            "mpr_set_profiling": ([H, i], i),
            "mpr_set_sweep_kernel": ([H, i], i),
            "mpr_inject_tma_stall": ([H, d], i),
            "mpr_set_proposal": ([H, d, d], i),
            "mpr_get_proposal": ([H, P(d)], i),
            "mpr_get_state": ([H, vp, P(u32)], i),
            "mpr_set_state": ([H, vp, u32], i),
            "mpr_philox4x32_10_dev": ([vp, vp, i, u64, vp], i),
            "mpr_bond_energy_noalloc": ([i, i, vp, d, vp, vp], i),
            "mpr_batch_create": ([i, vp, vp, vp, vp, P(mpr_options), P(H)], i),
            "mpr_batch_destroy": ([H], None),
            "mpr_batch_set_stream": ([H, vp], i),
            "mpr_batch_set_tuning": ([H, P(mpr_tuning)], i),
            "mpr_batch_set_launch": ([H, i, i, i, i], i),
            "mpr_batch_autotune": ([H, i, P(i), P(i), P(i)], i),
            "mpr_batch_fill": ([H, vp, i, i, vp, vp], i),
            "mpr_batch_predict": ([H, i, vp], i),
            "mpr_batch_get_state": ([H, i, vp, P(u32)], i),
            "mpr_batch_get_info": ([H, i, P(mpr_info)], i),
            "mpr_batch_get_stats": ([H, P(i), P(d), P(i), P(i), P(i), P(i)], i),
            "mpr_batch_inject_barrier_fault": ([H, i, d], i),
            "mpr_status_string": ([i], ctypes.c_char_p),
            "mpr_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def exported_symbols():
    """Names the binding expects the library to export (every function of include/mpr.h)."""
    return ["mpr_create", "mpr_create_dev", "mpr_destroy", "mpr_trim_memory", "mpr_set_options",
            "mpr_get_options",
            "mpr_set_stream", "mpr_set_tuning", "mpr_tune_temperature", "mpr_set_temperature",
            "mpr_tune_heating", "mpr_energy_curve", "mpr_tune_from_curve",
            "mpr_run", "mpr_run_auto", "mpr_predict", "mpr_predict_dev", "mpr_energy", "mpr_get_info",
            "mpr_get_state", "mpr_set_state", "mpr_philox4x32_10_dev", "mpr_set_profiling",
            "mpr_set_sweep_kernel", "mpr_inject_tma_stall", "mpr_set_proposal", "mpr_get_proposal",
            "mpr_bond_energy_noalloc", "mpr_status_string", "mpr_last_error",
            "mpr_batch_create", "mpr_batch_destroy", "mpr_batch_set_stream",
            "mpr_batch_set_tuning", "mpr_batch_set_launch", "mpr_batch_autotune",
            "mpr_batch_fill", "mpr_batch_predict", "mpr_batch_get_state", "mpr_batch_get_info",
            "mpr_batch_get_stats",
            "mpr_batch_inject_barrier_fault"]


def _check(st: int, allow=()):
    if st != MPR_OK and st not in allow:
        L = load()
        raise MPRError(st, f"{L.mpr_status_string(st).decode()}: {L.mpr_last_error().decode()}")
    return st


def _f64_host(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None   # torch.cuda.Stream


def _tensor_ptr(t, dtype_name):
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != f"torch.{dtype_name}":
        raise ValueError(f"expected a contiguous CUDA tensor of {dtype_name}")
    return ctypes.c_void_p(t.data_ptr())


# --- the C ABI, one function each --------------------------------------------------------------

def mpr_create(values, mask):
    """values (Ly, Lx) float64 host array, mask (Ly, Lx) nonzero = measured. Returns a handle."""
    v = _f64_host(values)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if v.ndim != 2 or m.shape != v.shape:
        raise ValueError("values and mask must be 2-D arrays of one shape (Ly, Lx)")
    h = ctypes.c_void_p()
    _check(load().mpr_create(v.shape[1], v.shape[0], _ptr(v), _ptr(m), ctypes.byref(h)))
    return h


def mpr_create_dev(values, mask, stream=None):
    """values (Ly, Lx) float64 CUDA tensor, mask (Ly, Lx) uint8 CUDA tensor."""
    if values.dim() != 2 or tuple(mask.shape) != tuple(values.shape):
        raise ValueError("values and mask must be 2-D tensors of one shape (Ly, Lx)")
    h = ctypes.c_void_p()
    _check(load().mpr_create_dev(values.shape[1], values.shape[0], _tensor_ptr(values, "float64"),
                                 _tensor_ptr(mask, "uint8"), _stream_ptr(stream), ctypes.byref(h)))
    return h


def mpr_destroy(h):
    if h is not None and h.value:
        load().mpr_destroy(h)
        h.value = None


def mpr_trim_memory():
    """Returns the device memory cached by the library's pool to the driver."""
    _check(load().mpr_trim_memory())


def make_options(setup: str = "SDS", seed: int = 0, q: float = 0.5, acc: str = "f64") -> mpr_options:
    """setup = X_S X_E X_F, e.g. 'DDD', 'SDS', 'SSS', 'HDS', 'BDS', 'HDH'."""
    if len(setup) != 3 or setup[0] not in STORE or setup[1] not in PREC or setup[2] not in FUNC:
        raise ValueError(f"bad precision setup {setup!r}")
    return mpr_options(seed, q, STORE[setup[0]], PREC[setup[1]], FUNC[setup[2]], ACC[acc])


def mpr_set_options(h, setup: str = "SDS", seed: int = 0, q: float = 0.5, acc: str = "f64"):
    o = make_options(setup, seed, q, acc)
    _check(load().mpr_set_options(h, ctypes.byref(o)))


def mpr_get_options(h) -> dict:
    o = mpr_options()
    _check(load().mpr_get_options(h, ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in mpr_options._fields_}


def mpr_set_stream(h, stream):
    _check(load().mpr_set_stream(h, _stream_ptr(stream)))


def mpr_set_tuning(h, n_eq=200, n_meas=50, T_lo=1e-3, T_hi=10.0, rel_tol=1e-3, ratio_tol=1.001,
                   max_probes=30):
    t = mpr_tuning(n_eq, n_meas, T_lo, T_hi, rel_tol, ratio_tol, max_probes)
    _check(load().mpr_set_tuning(h, ctypes.byref(t)))


def mpr_tune_temperature(h):
    """Returns (T, status); status is MPR_OK or MPR_ERR_TUNE_NO_CONVERGE (T still set)."""
    T = ctypes.c_double()
    st = _check(load().mpr_tune_temperature(h, ctypes.byref(T)), allow=(MPR_ERR_TUNE_NO_CONVERGE,))
    return T.value, st


def mpr_tune_heating(h, factor: float = 1.5):
    """Heating tuning: returns (T, status) like mpr_tune_temperature."""
    T = ctypes.c_double()
    st = load().mpr_tune_heating(h, float(factor), ctypes.byref(T))
    _check(st, allow=(MPR_ERR_TUNE_NO_CONVERGE,))
    return T.value, st


def mpr_energy_curve(Lx: int, Ly: int, T, setup: str = "SDS", seed: int = 0, q: float = 0.5,
                     n_eq: int = 200, n_meas: int = 50) -> np.ndarray:
    """Mean bond energy of the unconditional Lx x Ly lattice at each temperature of T in turn."""
    T = _f64_host(T).ravel()
    e = np.empty_like(T)
    opt = make_options(setup, seed, q)
    tun = mpr_tuning(n_eq, n_meas, 1e-3, 10.0, 1e-3, 1.001, 30)
    _check(load().mpr_energy_curve(int(Lx), int(Ly), ctypes.byref(opt), ctypes.byref(tun),
                                   _ptr(T), T.size, _ptr(e)))
    return e


def mpr_tune_from_curve(h, T, e):
    """Sets T by inverting the tabulated curve e(T): returns (T, status)."""
    T = _f64_host(T).ravel()
    e = _f64_host(e).ravel()
    if T.size != e.size:
        raise ValueError("T and e differ in length")
    out = ctypes.c_double()
    st = load().mpr_tune_from_curve(h, _ptr(T), _ptr(e), T.size, ctypes.byref(out))
    _check(st, allow=(MPR_ERR_TUNE_NO_CONVERGE,))
    return out.value, st


def mpr_set_temperature(h, T: float):
    _check(load().mpr_set_temperature(h, float(T)))


def mpr_run(h, equil: int, samples: int):
    _check(load().mpr_run(h, int(equil), int(samples)))


def mpr_run_auto(h, chunk: int, max_equil: int, samples: int) -> int:
    """Energy-slope equilibration then sampling; returns the equilibration sweeps run."""
    n = ctypes.c_int()
    _check(load().mpr_run_auto(h, int(chunk), int(max_equil), int(samples), ctypes.byref(n)))
    return n.value


def mpr_predict(h) -> np.ndarray:
    info = mpr_get_info(h)
    out = np.empty((info["Ly"], info["Lx"]), dtype=np.float64)
    _check(load().mpr_predict(h, _ptr(out)))
    return out


def mpr_predict_dev(h, out):
    _check(load().mpr_predict_dev(h, _tensor_ptr(out, "float64")))
    return out


def mpr_energy(h):
    """Returns (e_bond of the current state in FP64, e_sample)."""
    eb, es = ctypes.c_double(), ctypes.c_double()
    _check(load().mpr_energy(h, ctypes.byref(eb), ctypes.byref(es)))
    return eb.value, es.value


def mpr_get_info(h) -> dict:
    info = mpr_info()
    _check(load().mpr_get_info(h, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in mpr_info._fields_}


def mpr_set_profiling(h, on: bool = True):
    _check(load().mpr_set_profiling(h, int(bool(on))))


def mpr_set_sweep_kernel(h, kind: int):
    """FP32-function sweep kernel: -1 automatic (default), 0 one tile per block, 1 TMA-fed."""
    _check(load().mpr_set_sweep_kernel(h, int(kind)))


def mpr_set_proposal(h, width: float = 0.0, target: float = 0.0):
    """Metropolis proposal: width 0 uniform (default); else phi + width (2u - 1), rejected outside
    [0, 2 pi), adapted toward acceptance fraction ``target`` while not sampling (0: fixed)."""
    _check(load().mpr_set_proposal(h, float(width), float(target)))


def mpr_get_proposal(h) -> float:
    """Current half-width of the bounded proposal (0.0 when proposals are uniform)."""
    w = ctypes.c_double()
    _check(load().mpr_get_proposal(h, ctypes.byref(w)))
    return w.value


def mpr_inject_tma_stall(h, timeout_s: float = 0.05):
    """Test hook: the next TMA-kernel pass has a wait that runs out (see include/mpr.h)."""
    _check(load().mpr_inject_tma_stall(h, float(timeout_s)))


def mpr_get_state(h):
    info = mpr_get_info(h)
    out = np.empty((info["Ly"], info["Lx"]), dtype=np.float64)
    sw = ctypes.c_uint32()
    _check(load().mpr_get_state(h, _ptr(out), ctypes.byref(sw)))
    return out, sw.value


def mpr_set_state(h, angles, sweep: int):
    a = _f64_host(angles)
    _check(load().mpr_set_state(h, _ptr(a), int(sweep)))


def mpr_philox4x32_10_dev(ctr, seed: int, stream=None):
    """ctr: (n, 4) int32 CUDA tensor holding uint32 counter words; returns (n, 4) int32 words."""
    import torch

    if ctr.dim() != 2 or ctr.shape[1] != 4:
        raise ValueError("ctr must have shape (n, 4)")
    out = torch.empty_like(ctr)
    _check(load().mpr_philox4x32_10_dev(_tensor_ptr(ctr, "int32"), _tensor_ptr(out, "int32"),
                                        ctr.shape[0], int(seed), _stream_ptr(stream)))
    return out


def mpr_bond_energy_noalloc(angles, q: float, out, stream=None):
    """Bond energy of a state held on the device, with no device allocation (for callers that
    cannot allocate: device memory owned by another allocator or a fixed budget, loops that must
    not take the allocator's locks). angles: (Ly, Lx) float64 CUDA tensor;
    out: float64 CUDA tensor of at least one element, written asynchronously on ``stream``."""
    if angles.dim() != 2:
        raise ValueError("angles must be a 2-D tensor (Ly, Lx)")
    _check(load().mpr_bond_energy_noalloc(angles.shape[1], angles.shape[0],
                                          _tensor_ptr(angles, "float64"), float(q),
                                          _tensor_ptr(out, "float64"), _stream_ptr(stream)))
    return out


# --- batches ------------------------------------------------------------------------------------

def mpr_batch_create(values_list, mask_list, setup: str = "SDS", seed: int = 0, q: float = 0.5,
                     acc: str = "f64"):
    """values_list / mask_list: sequences of (Ly_i, Lx_i) host arrays. Returns a batch handle."""
    n = len(values_list)
    if n != len(mask_list) or n == 0:
        raise ValueError("need equally many value and mask arrays, at least one")
    vs = [_f64_host(v) for v in values_list]
    ms = [np.ascontiguousarray(m, dtype=np.uint8) for m in mask_list]
    for v, m in zip(vs, ms):
        if v.ndim != 2 or m.shape != v.shape:
            raise ValueError("each problem needs 2-D values and mask of one shape")
    Lx = (ctypes.c_int * n)(*[v.shape[1] for v in vs])
    Ly = (ctypes.c_int * n)(*[v.shape[0] for v in vs])
    vp = (ctypes.c_void_p * n)(*[v.ctypes.data for v in vs])
    mp = (ctypes.c_void_p * n)(*[m.ctypes.data for m in ms])
    o = make_options(setup, seed, q, acc)
    b = ctypes.c_void_p()
    _check(load().mpr_batch_create(n, Lx, Ly, vp, mp, ctypes.byref(o), ctypes.byref(b)))
    b._n = n
    return b


def mpr_batch_destroy(b):
    if b is not None and b.value:
        load().mpr_batch_destroy(b)
        b.value = None


def mpr_batch_set_stream(b, stream):
    _check(load().mpr_batch_set_stream(b, _stream_ptr(stream)))


def mpr_batch_set_tuning(b, n_eq=200, n_meas=50, T_lo=1e-3, T_hi=10.0, rel_tol=1e-3,
                         ratio_tol=1.001, max_probes=30):
    t = mpr_tuning(n_eq, n_meas, T_lo, T_hi, rel_tol, ratio_tol, max_probes)
    _check(load().mpr_batch_set_tuning(b, ctypes.byref(t)))


def mpr_batch_set_launch(b, tile_rows: int = 32, tile_cols: int = 128, blocks_per_sm: int = 0,
                         mode: int = 2):
    """Tile of tile_rows x tile_cols half-lattice entries (8/16/32 x 128 or 16/32 x 64); mode 0:
    persistent cooperative kernel, 1: the same as a one-node graph, 2: graph with a device-side
    while loop over per-pass kernels."""
    _check(load().mpr_batch_set_launch(b, tile_rows, tile_cols, blocks_per_sm, int(mode)))


def mpr_batch_autotune(b, sweeps: int = 10):
    """Returns (tile_rows, tile_cols, blocks_per_sm, mode) of the fastest launch shape."""
    r, c, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().mpr_batch_autotune(b, sweeps, ctypes.byref(r), ctypes.byref(c), ctypes.byref(k)))
    return r.value, c.value, k.value, mpr_batch_get_stats(b)["mode"]


def mpr_batch_fill(b, equil: int, samples: int, T=None):
    """One launch; T None = tune every problem. Returns (T array, status array)."""
    n = b._n
    Tin = None if T is None else np.ascontiguousarray(T, dtype=np.float64)
    Tout = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    _check(load().mpr_batch_fill(b, None if Tin is None else _ptr(Tin), equil, samples, _ptr(Tout),
                                 _ptr(st)), allow=(MPR_ERR_TUNE_NO_CONVERGE,))
    return Tout, st


def mpr_batch_predict(b, i: int):
    info = mpr_batch_get_info(b, i)
    out = np.empty((info["Ly"], info["Lx"]))
    _check(load().mpr_batch_predict(b, i, _ptr(out)))
    return out


def mpr_batch_get_state(b, i: int):
    info = mpr_batch_get_info(b, i)
    out = np.empty((info["Ly"], info["Lx"]))
    sw = ctypes.c_uint32()
    _check(load().mpr_batch_get_state(b, i, _ptr(out), ctypes.byref(sw)))
    return out, sw.value


def mpr_batch_get_info(b, i: int) -> dict:
    info = mpr_info()
    _check(load().mpr_batch_get_info(b, i, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in mpr_info._fields_}


def mpr_batch_get_stats(b) -> dict:
    it, ms = ctypes.c_int(), ctypes.c_double()
    r, c, k, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().mpr_batch_get_stats(b, ctypes.byref(it), ctypes.byref(ms), ctypes.byref(r),
                                      ctypes.byref(c), ctypes.byref(k), ctypes.byref(m)))
    return {"iterations": it.value, "fill_ms": ms.value, "tile_rows": r.value, "tile_cols": c.value,
            "blocks_per_sm": k.value, "mode": m.value}


def mpr_batch_inject_barrier_fault(b, extra_arrivals: int = 1, timeout_s: float = 0.05):
    _check(load().mpr_batch_inject_barrier_fault(b, extra_arrivals, float(timeout_s)))


def mpr_status_string(st: int) -> str:
    return load().mpr_status_string(st).decode()


def mpr_last_error() -> str:
    return load().mpr_last_error().decode()


class GapFiller:
    """Owns one handle: ``GapFiller(z, mask, setup='SDS').fill(equil, samples)``, or step by step
    ``p.tune(); p.run(equil, samples); p.predict()``. Values and mask are numpy arrays (host) or
    CUDA tensors (device, read on ``stream``)."""

    def __init__(self, values, mask, setup: str = "SDS", seed: int = 0, q: float = 0.5,
                 acc: str = "f64", stream=None):
        if hasattr(values, "is_cuda"):
            self.h = mpr_create_dev(values, mask, stream)
        else:
            self.h = mpr_create(values, mask)
            if stream is not None:
                mpr_set_stream(self.h, stream)
        if (setup, seed, q, acc) != ("SDS", 0, 0.5, "f64"):
            mpr_set_options(self.h, setup, seed, q, acc)

    def fill(self, equil: int, samples: int, T=None):
        if T is None:
            self.tune()
        else:
            self.set_temperature(T)
        self.run(equil, samples)
        return self.predict()

    def tune(self):
        """Temperature tuning (returns T; the status is kept in ``tune_status``)."""
        self.T, self.tune_status = mpr_tune_temperature(self.h)
        return self.T

    def set_temperature(self, T: float):
        mpr_set_temperature(self.h, T)
        self.T, self.tune_status = T, MPR_OK

    def run(self, equil: int, samples: int):
        mpr_run(self.h, equil, samples)

    def predict(self, out=None):
        """Prediction as a numpy array, or written into the CUDA tensor ``out``."""
        if out is not None:
            mpr_predict_dev(self.h, out)
            return out
        return mpr_predict(self.h)

    def info(self):
        return mpr_get_info(self.h)

    def close(self):
        mpr_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


Problem = GapFiller
