"""FP64 CPU oracle of the MPR gap-filling method (Sec. 2, Eq. 2 of Lach, Borovsky, Zukovic).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers. The CUDA library never imports, links or runs anything here,
and nothing here imports the CUDA library.

The arithmetic lives in ``mpr_oracle.c`` (plain C, FP64, one site at a time); this module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmpr_oracle.so")
_SOURCES = [os.path.join(_HERE, "mpr_oracle.c")]
_HEADERS = [os.path.join(_HERE, "mpr_oracle.h")]
_lock = threading.Lock()
_lib = None

TWO_PI = 2.0 * np.pi


class Cfg(ctypes.Structure):
    _fields_ = [
        ("Lx", ctypes.c_int),
        ("Ly", ctypes.c_int),
        ("q", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("problem", ctypes.c_uint32),
        ("ubits", ctypes.c_int),
        ("width", ctypes.c_double),
    ]


class TuneCfg(ctypes.Structure):
    _fields_ = [
        ("n_eq", ctypes.c_int),
        ("n_meas", ctypes.c_int),
        ("T_lo", ctypes.c_double),
        ("T_hi", ctypes.c_double),
        ("rel_tol", ctypes.c_double),
        ("ratio_tol", ctypes.c_double),
        ("max_probes", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so x86 and Arm round alike)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SOURCES + _HEADERS)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp] + _SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            d, i, u32, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
            vp = ctypes.c_void_p
            L.mpro_philox.argtypes = [i, i, vp, vp, vp]
            L.mpro_philox.restype = None
            L.mpro_philox_n.argtypes = [i, i, i, vp, vp, vp]
            L.mpro_philox_n.restype = None
            L.mpro_site_words.argtypes = [P(Cfg), i, i, u32, i, P(u32), P(u32)]
            L.mpro_site_words.restype = None
            L.mpro_uniform.argtypes = [P(Cfg), u32]
            L.mpro_uniform.restype = d
            L.mpro_site_uniforms.argtypes = [P(Cfg), i, i, u32, P(d), P(d)]
            L.mpro_site_uniforms.restype = None
            L.mpro_map.argtypes = [i, vp, vp, vp, P(d), P(d)]
            L.mpro_map.restype = i
            L.mpro_init.argtypes = [P(Cfg), vp, vp]
            L.mpro_init.restype = None
            L.mpro_overrelax.argtypes = [d, d, d, d, P(d)]
            L.mpro_overrelax.restype = d
            L.mpro_update_site.argtypes = [P(Cfg), vp, vp, i, i, d, u32, P(d), P(d), P(i)]
            L.mpro_update_site.restype = d
            L.mpro_half_sweep.argtypes = [P(Cfg), vp, vp, d, u32, i, vp, vp]
            L.mpro_half_sweep.restype = ctypes.c_int64
            L.mpro_sweep.argtypes = [P(Cfg), vp, vp, d, u32, vp, vp]
            L.mpro_sweep.restype = ctypes.c_int64
            L.mpro_run_adapt.argtypes = [P(Cfg), vp, vp, d, u32, i, d, vp]
            L.mpro_run_adapt.restype = None
            L.mpro_energy_bond.argtypes = [P(Cfg), vp]
            L.mpro_energy_bond.restype = d
            L.mpro_energy_sample.argtypes = [P(Cfg), vp, vp, P(d), P(ctypes.c_int64)]
            L.mpro_energy_sample.restype = i
            L.mpro_run.argtypes = [P(Cfg), vp, vp, d, u32, i, vp, vp]
            L.mpro_run.restype = None
            L.mpro_tune.argtypes = [P(Cfg), vp, vp, d, P(u32), P(TuneCfg), P(d), vp, vp, P(i)]
            L.mpro_tune.restype = i
            L.mpro_tune_heating.argtypes = [P(Cfg), vp, vp, d, P(u32), P(TuneCfg), d, P(d), vp,
                                            vp, P(i)]
            L.mpro_tune_heating.restype = i
            L.mpro_energy_curve.argtypes = [P(Cfg), vp, i, P(TuneCfg), P(u32), vp]
            L.mpro_energy_curve.restype = None
            L.mpro_invert_curve.argtypes = [vp, vp, i, d, P(d)]
            L.mpro_invert_curve.restype = i
            L.mpro_equilibrate.argtypes = [P(Cfg), vp, vp, d, P(u32), i, i, d]
            L.mpro_equilibrate.restype = i
            L.mpro_predict.argtypes = [i, vp, i, vp, vp, d, d, vp]
            L.mpro_predict.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def overrelax(q: float, hx: float, hy: float, phi: float):
    """Over-relaxation of one angle in the local field (hx, hy); returns (new angle, margin)."""
    m = ctypes.c_double()
    f = lib().mpro_overrelax(q, hx, hy, phi, ctypes.byref(m))
    return f, m.value


def invert_curve(T, e, e_s):
    """(status, T) where the log-T interpolant of the tabulated curve e(T) reaches e_s."""
    T, e = _f64(T), _f64(e)
    out = ctypes.c_double()
    st = lib().mpro_invert_curve(_ptr(T), _ptr(e), T.size, e_s, ctypes.byref(out))
    return st, out.value


def philox(width: int, rounds: int, ctr, key) -> np.ndarray:
    """Philox-4xW-R block function on one counter; returns 4 words as uint64."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().mpro_philox(width, rounds, _ptr(c), _ptr(k), _ptr(out))
    return out


def philox_many(width: int, rounds: int, ctr, key) -> np.ndarray:
    """The block function on an (n, 4) array of counters; returns (n, 4) uint64 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros_like(c)
    lib().mpro_philox_n(width, rounds, c.shape[0], _ptr(c), _ptr(k), _ptr(out))
    return out


class Oracle:
    """One conditional MPR problem: an Lx x Ly grid with values z and a measured mask."""

    def __init__(self, Lx: int, Ly: int, seed: int = 0, q: float = 0.5, problem: int = 0,
                 ubits: int = 32, width: float = 0.0):
        self.cfg = Cfg(Lx, Ly, q, seed, problem, ubits, width)
        self.Lx, self.Ly, self.q = Lx, Ly, q

    # --- random numbers ---------------------------------------------------------------------
    def site_words(self, x: int, y: int, sweep: int, tag: int = 0):
        a, b = ctypes.c_uint32(), ctypes.c_uint32()
        lib().mpro_site_words(ctypes.byref(self.cfg), x, y, sweep, tag, ctypes.byref(a),
                              ctypes.byref(b))
        return a.value, b.value

    def uniform(self, w: int) -> float:
        return lib().mpro_uniform(ctypes.byref(self.cfg), w)

    def site_uniforms(self, x: int, y: int, sweep: int):
        """(proposal, acceptance) uniforms of the Metropolis move of site (x, y) at a sweep."""
        a, b = ctypes.c_double(), ctypes.c_double()
        lib().mpro_site_uniforms(ctypes.byref(self.cfg), x, y, sweep, ctypes.byref(a),
                                 ctypes.byref(b))
        return a.value, b.value

    # --- mapping and state ------------------------------------------------------------------
    def map(self, z, mask):
        """Returns (phi, zmin, zmax) or raises ValueError on degenerate data."""
        z = _f64(z).reshape(-1)
        m = _u8(mask).reshape(-1)
        phi = np.zeros_like(z)
        lo, hi = ctypes.c_double(), ctypes.c_double()
        st = lib().mpro_map(z.size, _ptr(z), _ptr(m), _ptr(phi), ctypes.byref(lo), ctypes.byref(hi))
        if st != 0:
            raise ValueError("degenerate data: fewer than two measured sites or zmax == zmin")
        return phi.reshape(self.Ly, self.Lx), lo.value, hi.value

    def init(self, phi, mask) -> np.ndarray:
        phi = _f64(phi).copy()
        m = _u8(mask)
        lib().mpro_init(ctypes.byref(self.cfg), _ptr(m), _ptr(phi))
        return phi

    # --- moves ------------------------------------------------------------------------------
    def update_site(self, phi, mask, x, y, T, sweep):
        phi = _f64(phi)
        m = _u8(mask)
        mm, om = ctypes.c_double(), ctypes.c_double()
        f = lib().mpro_update_site(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), x, y, T, sweep,
                                   ctypes.byref(mm), ctypes.byref(om), None)
        return f, mm.value, om.value

    def accepted(self, phi, mask, T, sweep) -> int:
        """Accepted Metropolis proposals of one sweep from phi (the sweep itself is discarded)."""
        phi = _f64(phi).copy()
        m = _u8(mask)
        return lib().mpro_sweep(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), T, sweep, None, None)

    def run_adapt(self, phi, mask, T, sweep0, nsweeps, target):
        """Adapted-width sweeps: returns (phi, widths used per sweep); the final width stays in
        the oracle (self.cfg.width)."""
        phi = _f64(phi).copy()
        m = _u8(mask)
        w = np.zeros(max(nsweeps, 1))
        lib().mpro_run_adapt(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), T, sweep0, nsweeps,
                             target, _ptr(w))
        return phi, w[:nsweeps]

    def sweep(self, phi, mask, T, sweep, margins: bool = False):
        """Returns the new state (and the per-site Metropolis / over-relaxation margins)."""
        phi = _f64(phi).copy()
        m = _u8(mask)
        if margins:
            mm = np.empty_like(phi)
            om = np.empty_like(phi)
            lib().mpro_sweep(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), T, sweep, _ptr(mm), _ptr(om))
            return phi, mm, om
        lib().mpro_sweep(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), T, sweep, None, None)
        return phi

    def half_sweep(self, phi, mask, T, sweep, colour):
        """One colour of a sweep; returns (state, met_margin, or_margin), margins +inf elsewhere."""
        phi = _f64(phi).copy()
        m = _u8(mask)
        mm = np.full_like(phi, np.inf)
        om = np.full_like(phi, np.inf)
        lib().mpro_half_sweep(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), T, sweep, colour,
                              _ptr(mm), _ptr(om))
        return phi, mm, om

    def run(self, phi, mask, T, sweep0, nsweeps, acc=None, energies: bool = False):
        """In-place on copies: returns (phi, acc, energies)."""
        phi = _f64(phi).copy()
        m = _u8(mask)
        accp = None
        if acc is not None:
            acc = _f64(acc).copy()
            accp = _ptr(acc)
        e = np.zeros(max(nsweeps, 1)) if energies else None
        lib().mpro_run(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), T, sweep0, nsweeps, accp,
                       _ptr(e) if energies else None)
        return phi, acc, (e[:nsweeps] if energies else None)

    # --- energies ---------------------------------------------------------------------------
    def energy_bond(self, phi) -> float:
        phi = _f64(phi)
        return lib().mpro_energy_bond(ctypes.byref(self.cfg), _ptr(phi))

    def energy_sample(self, phi, mask):
        phi = _f64(phi)
        m = _u8(mask)
        e, n = ctypes.c_double(), ctypes.c_int64()
        st = lib().mpro_energy_sample(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), ctypes.byref(e),
                                      ctypes.byref(n))
        if st != 0:
            raise ValueError("no measured nearest-neighbour pair")
        return e.value, n.value

    # --- tuning and prediction --------------------------------------------------------------
    def tune(self, phi, mask, e_s, sweep, n_eq=200, n_meas=50, T_lo=1e-3, T_hi=10.0,
             rel_tol=1e-3, ratio_tol=1.001, max_probes=30):
        """Returns (status, T, phi, next_sweep, trace) with trace = [(T, e_b), ...]."""
        phi = _f64(phi).copy()
        m = _u8(mask)
        t = TuneCfg(n_eq, n_meas, T_lo, T_hi, rel_tol, ratio_tol, max_probes)
        sw = ctypes.c_uint32(sweep)
        T = ctypes.c_double()
        tT = np.zeros(max_probes)
        te = np.zeros(max_probes)
        n = ctypes.c_int()
        st = lib().mpro_tune(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), e_s, ctypes.byref(sw),
                             ctypes.byref(t), ctypes.byref(T), _ptr(tT), _ptr(te), ctypes.byref(n))
        trace = list(zip(tT[: n.value].tolist(), te[: n.value].tolist()))
        return st, T.value, phi, sw.value, trace

    def tune_heating(self, phi, mask, e_s, sweep, factor=1.5, n_eq=200, n_meas=50, T_lo=1e-3,
                     T_hi=10.0, rel_tol=1e-3, ratio_tol=1.001, max_probes=30):
        """Heating tuning: returns (status, T, phi, next_sweep, trace) like tune()."""
        phi = _f64(phi).copy()
        m = _u8(mask)
        t = TuneCfg(n_eq, n_meas, T_lo, T_hi, rel_tol, ratio_tol, max_probes)
        sw = ctypes.c_uint32(sweep)
        T = ctypes.c_double()
        tT = np.zeros(max_probes)
        te = np.zeros(max_probes)
        n = ctypes.c_int()
        st = lib().mpro_tune_heating(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), e_s,
                                     ctypes.byref(sw), ctypes.byref(t), factor, ctypes.byref(T),
                                     _ptr(tT), _ptr(te), ctypes.byref(n))
        trace = list(zip(tT[: n.value].tolist(), te[: n.value].tolist()))
        return st, T.value, phi, sw.value, trace

    def energy_curve(self, T, n_eq=200, n_meas=50, sweep=0):
        """Mean e_b of the unconditional lattice (no frozen site) at each T in turn."""
        T = _f64(T)
        e = np.zeros(max(T.size, 1))
        t = TuneCfg(n_eq, n_meas, 1e-3, 10.0, 1e-3, 1.001, 30)
        sw = ctypes.c_uint32(sweep)
        lib().mpro_energy_curve(ctypes.byref(self.cfg), _ptr(T), T.size, ctypes.byref(t),
                                ctypes.byref(sw), _ptr(e))
        return e[: T.size]

    def equilibrate(self, phi, mask, T, sweep, chunk, max_sweeps, z=2.0):
        """Energy-slope equilibration: returns (phi, sweeps run, next sweep)."""
        phi = _f64(phi).copy()
        m = _u8(mask)
        sw = ctypes.c_uint32(sweep)
        n = lib().mpro_equilibrate(ctypes.byref(self.cfg), _ptr(phi), _ptr(m), T,
                                   ctypes.byref(sw), chunk, max_sweeps, z)
        return phi, n, sw.value

    def predict(self, acc, nsamples, z, mask, zmin, zmax) -> np.ndarray:
        acc = _f64(acc)
        z = _f64(z)
        m = _u8(mask)
        out = np.empty_like(z)
        lib().mpro_predict(z.size, _ptr(acc), nsamples, _ptr(z), _ptr(m), zmin, zmax, _ptr(out))
        return out

    # --- the whole method -------------------------------------------------------------------
    def gap_fill(self, z, mask, equil, samples, tune=True, T=None, **tune_kw):
        """create -> (tune) -> equil + samples sweeps -> prediction. Returns a dict."""
        phi, zmin, zmax = self.map(z, mask)
        phi = self.init(phi, mask)
        e_s, n_pairs = self.energy_sample(phi, mask)
        sweep = 0
        status, trace = 0, []
        if tune:
            status, T, phi, sweep, trace = self.tune(phi, mask, e_s, sweep, **tune_kw)
        phi, _, _ = self.run(phi, mask, T, sweep, equil)
        sweep += equil
        acc = np.zeros_like(phi)
        phi, acc, e = self.run(phi, mask, T, sweep, samples, acc=acc, energies=True)
        sweep += samples
        zhat = self.predict(acc, samples, z, mask, zmin, zmax)
        return dict(zhat=zhat, T=T, status=status, e_s=e_s, n_pairs=n_pairs, trace=trace,
                    e_samples=e, phi=phi, sweep=sweep, zmin=zmin, zmax=zmax, acc=acc)
