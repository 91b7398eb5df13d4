"""CPU oracle for the DPSNN-style grid simulation.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product path never
does.  The simulator itself is plain C (``snn_oracle.c``), compiled with
``-O2 -ffp-contract=off`` so that each float operation is one correctly rounded
binary32 operation in source order; it steps on one thread (the tests may let
extra threads generate synapse rows, pure functions of seed and source).  It
shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-fPIC", "-shared"]

K = 1250
ZTAB = 4096
KMAX = 16

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc) if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("gx", ctypes.c_int32), ("gy", ctypes.c_int32),
        ("lambda_", ctypes.c_float), ("p_local", ctypes.c_float),
        ("out_degree", ctypes.c_int32), ("n_delay", ctypes.c_int32), ("min_delay", ctypes.c_int32),
        ("dt_ms", ctypes.c_float), ("record_format", ctypes.c_int32),
        ("bin_steps", ctypes.c_int32),
        ("tau_m", ctypes.c_float * 3), ("C_m", ctypes.c_float * 3), ("E_L", ctypes.c_float * 3),
        ("V_th", ctypes.c_float * 3), ("V_r", ctypes.c_float * 3), ("tau_arp", ctypes.c_float * 3),
        ("alpha_c", ctypes.c_float * 3), ("tau_c", ctypes.c_float * 3), ("g_c", ctypes.c_float * 3),
        ("J", (ctypes.c_float * 3) * 3), ("dJ_frac", ctypes.c_float),
        ("J_ext", ctypes.c_float * 3), ("dJ_ext_frac", ctypes.c_float),
        ("nu_ext", ctypes.c_float * 3), ("N_ext", ctypes.c_float * 3),
    ]


def make_params(d: dict) -> Params:
    p = Params()
    p.gx, p.gy = int(d["gx"]), int(d["gy"])
    p.lambda_ = float(d["lambda"])
    p.p_local = float(d["p_local"])
    p.out_degree = int(d["out_degree"])
    p.n_delay = int(d["n_delay"])
    p.min_delay = int(d.get("min_delay", 1))
    p.dt_ms = float(d["dt_ms"])
    p.record_format = int(d["record_format"])
    p.bin_steps = int(d["bin_steps"])
    for name in ("tau_m", "C_m", "E_L", "V_th", "V_r", "tau_arp", "alpha_c", "tau_c", "g_c",
                 "J_ext", "nu_ext", "N_ext"):
        arr = getattr(p, name)
        for i in range(3):
            arr[i] = float(d[name][i])
    for a in range(3):
        for b in range(3):
            p.J[a][b] = float(d["J"][a][b])
    p.dJ_frac = float(d["dJ_frac"])
    p.dJ_ext_frac = float(d["dJ_ext_frac"])
    return p


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    vp, u32, i32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
    P = ctypes.POINTER
    lib.orc_create.restype = vp
    lib.orc_create.argtypes = [P(Params), u64]
    lib.orc_destroy.argtypes = [vp]
    lib.orc_run.argtypes = [vp, u32]
    lib.orc_time.restype = u32
    lib.orc_time.argtypes = [vp]
    lib.orc_n.restype = i32
    lib.orc_n.argtypes = [vp]
    lib.orc_raster_len.restype = sz
    lib.orc_raster_len.argtypes = [vp]
    lib.orc_raster.argtypes = [vp, vp, vp]
    lib.orc_rates_bins.restype = sz
    lib.orc_rates_bins.argtypes = [vp]
    lib.orc_rates.argtypes = [vp, vp]
    lib.orc_state.argtypes = [vp, vp, vp, vp]
    lib.orc_ring.argtypes = [vp, vp]
    lib.orc_counters.argtypes = [vp, vp]
    lib.orc_ztab.argtypes = [vp, vp]
    lib.orc_pop_tables.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp]
    lib.orc_cdf_row.argtypes = [vp, i32, vp]
    lib.orc_build_row.argtypes = [vp, u32, vp, vp]
    lib.orc_synapse.argtypes = [vp, u32, u32, vp, vp]
    lib.orc_enable_trace.argtypes = [vp, u32, u32]
    lib.orc_trace.argtypes = [vp, vp, vp]
    lib.orc_neuron_trace.argtypes = [P(Params), i32, ctypes.c_float, ctypes.c_float, u32, vp, vp, vp, vp]
    lib.orc_philox4x32_10.argtypes = [vp, u32, u32, vp]
    lib.orc_row_build_seconds.restype = ctypes.c_double
    lib.orc_row_build_seconds.argtypes = [vp]
    lib.orc_configure_rows.argtypes = [vp, i32, i32]
    lib.orc_inv_phi.restype = ctypes.c_double
    lib.orc_inv_phi.argtypes = [ctypes.c_double]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def philox(ctr, key0: int, key1: int) -> np.ndarray:
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF, _ptr(out))
    return out


def inv_phi(p: float) -> float:
    return _load().orc_inv_phi(float(p))


def neuron_trace(params: dict, pop: int, V0: float, c0: float, inputs) -> tuple:
    """Run one isolated neuron with per-step input (2^-16 mV units)."""
    lib = _load()
    I = np.ascontiguousarray(inputs, dtype=np.int32)
    n = I.size
    V = np.zeros(n, np.float32)
    c = np.zeros(n, np.float32)
    s = np.zeros(n, np.uint8)
    pp = make_params(params)
    lib.orc_neuron_trace(ctypes.byref(pp), pop, V0, c0, n, _ptr(I), _ptr(V), _ptr(c), _ptr(s))
    return V, c, s.astype(bool)


class OracleNet:
    """One simulated network held by the C oracle."""

    def __init__(self, params: dict, seed: int):
        self._lib = _load()
        self.params = dict(params)
        self._p = make_params(params)
        h = self._lib.orc_create(ctypes.byref(self._p), ctypes.c_uint64(seed))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ctypes.c_void_p(h)
        self.G = params["gx"] * params["gy"]
        self.N = self.G * K
        self.M = params["out_degree"]
        self.D = params["n_delay"] + 1

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def t(self) -> int:
        return self._lib.orc_time(self._h)

    def run(self, steps: int):
        self._lib.orc_run(self._h, int(steps))

    def raster(self):
        n = self._lib.orc_raster_len(self._h)
        t = np.zeros(n, np.uint32)
        ids = np.zeros(n, np.uint32)
        if n:
            self._lib.orc_raster(self._h, _ptr(t), _ptr(ids))
        return t, ids

    def rates(self) -> np.ndarray:
        nb = self._lib.orc_rates_bins(self._h)
        out = np.zeros((nb, self.G, 3), np.uint32)
        if nb:
            self._lib.orc_rates(self._h, _ptr(out))
        return out

    def state(self):
        V = np.zeros(self.N, np.float32)
        c = np.zeros(self.N, np.float32)
        ref = np.zeros(self.N, np.int32)
        self._lib.orc_state(self._h, _ptr(V), _ptr(c), _ptr(ref))
        return V, c, ref

    def ring(self) -> np.ndarray:
        out = np.zeros((self.D, self.N), np.int32)
        self._lib.orc_ring(self._h, _ptr(out))
        return out

    def configure_rows(self, threads: int = 1, keep: bool = True) -> None:
        """Test-harness setting with no effect on results: threads that generate
        the rows a step needs, and whether generated rows stay cached."""
        self._lib.orc_configure_rows(self._h, int(threads), 1 if keep else 0)

    def row_build_seconds(self) -> float:
        """Wall time the oracle spent generating rows on first use."""
        return self._lib.orc_row_build_seconds(self._h)

    def counters(self) -> dict:
        out = np.zeros(3, np.uint64)
        self._lib.orc_counters(self._h, _ptr(out))
        return {"spikes": int(out[0]), "rec_events": int(out[1]), "ext_events": int(out[2])}

    def row(self, s: int):
        keys = np.zeros(self.M, np.uint32)
        w = np.zeros(self.M, np.float32)
        self._lib.orc_build_row(self._h, int(s), _ptr(keys), _ptr(w))
        return keys, w

    def synapse(self, s: int, j: int):
        key = ctypes.c_uint32(0)
        w = ctypes.c_float(0.0)
        self._lib.orc_synapse(self._h, int(s), int(j), ctypes.byref(key), ctypes.byref(w))
        return key.value, w.value

    def rows(self, sources) -> tuple:
        """Rows of several sources stacked: keys [n, M] u32 and weights [n, M] f32."""
        src = list(sources)
        keys = np.zeros((len(src), self.M), np.uint32)
        w = np.zeros((len(src), self.M), np.float32)
        for i, s in enumerate(src):
            self._lib.orc_build_row(self._h, int(s), _ptr(keys[i]), _ptr(w[i]))
        return keys, w

    def ztab(self) -> np.ndarray:
        out = np.zeros(ZTAB, np.float32)
        self._lib.orc_ztab(self._h, _ptr(out))
        return out

    def pop_tables(self, p: int) -> dict:
        prop = np.zeros(3, np.float32)
        narp = ctypes.c_int32(0)
        thr = np.zeros(KMAX, np.uint64)
        amp = np.zeros(ZTAB, np.int32)
        self._lib.orc_pop_tables(self._h, p, _ptr(prop), ctypes.byref(narp), _ptr(thr), _ptr(amp))
        return {"pvv": prop[0], "pvc": prop[1], "pcc": prop[2], "narp": narp.value,
                "thr": thr, "amp": amp}

    def cdf_row(self, ms: int) -> np.ndarray:
        out = np.zeros(max(self.G - 1, 0), np.uint32)
        if self.G > 1:
            self._lib.orc_cdf_row(self._h, int(ms), _ptr(out))
        return out

    def enable_trace(self, t0: int, steps: int):
        if self._lib.orc_enable_trace(self._h, int(t0), int(steps)) != 0:
            raise MemoryError("trace allocation failed")
        self._trace_steps = steps

    def trace(self):
        rec = np.zeros((self._trace_steps, self.N), np.int32)
        ext = np.zeros((self._trace_steps, self.N), np.int32)
        self._lib.orc_trace(self._h, _ptr(rec), _ptr(ext))
        return rec, ext


def simulate(params: dict, seed: int, steps: int, row_threads: int = 1, keep_rows: bool = True) -> dict:
    """Run one network for `steps` steps from its initial state and return every
    result the parity tests compare: raster (steps, ids), rate counts, final
    V, c and refractory counters, and the event counters.  A plain function so
    that a spawned process pool can run it."""
    o = OracleNet(params, seed)
    try:
        o.configure_rows(row_threads, keep_rows)
        o.run(steps)
        ts, ids = o.raster()
        V, c, ref = o.state()
        return {"t": o.t, "steps": ts, "ids": ids, "rates": o.rates(), "V": V, "c": c, "ref": ref,
                "counters": o.counters(), "row_build_seconds": o.row_build_seconds()}
    finally:
        o.close()
