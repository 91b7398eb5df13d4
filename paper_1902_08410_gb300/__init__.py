"""GB300 (sm_103a) simulator of a DPSNN-style cortical grid (Pastorelli et al. 2019).

Thin Python binding over the C ABI in ``include/snn.h`` (``libsnn.so``): every
step of the simulation runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch, when present, supplies the CUDA stream and the
caching allocator.  There is no CPU fallback: without the compiled library or a
CUDA device every call raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import SnnLaunch, SnnParams, SnnStats

SNN_OK = 0
ERRORS = {-1: "SNN_ERR_ARG", -2: "SNN_ERR_OOM", -3: "SNN_ERR_CUDA",
          -5: "SNN_ERR_BUFFER", -6: "SNN_ERR_LIMIT", -7: "SNN_ERR_STATE"}
REC_F32 = 0
REC_I16 = 1
K = 1250


class SnnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile libsnn.so for sm_103a (in-tree)."""
    return _native.build(force=force)


def lib():
    return _native.load()


def _check(rc: int):
    if rc != SNN_OK:
        raise SnnError(rc, lib().snn_last_error().decode())


def make_params(d: dict) -> SnnParams:
    p = SnnParams()
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


def footprint(params: dict) -> int:
    """Device bytes a network with these parameters holds once built."""
    out = ctypes.c_size_t(0)
    pp = make_params(params)
    _check(lib().snn_footprint(ctypes.byref(pp), ctypes.byref(out)))
    return out.value


# ---------------------------------------------------------------------------
# PyTorch plumbing: caching allocator and current stream
# ---------------------------------------------------------------------------
_torch_alloc_fns = None


def use_torch_allocator() -> None:
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_alloc_fns
    import torch

    def _alloc(nbytes, _ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:
            return None

    def _free(ptr, _ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    fns = (_native.ALLOC_FN(_alloc), _native.FREE_FN(_free))
    _check(lib().snn_set_allocator(fns[0], fns[1], None))
    _torch_alloc_fns = fns


def use_cuda_malloc() -> None:
    global _torch_alloc_fns
    _check(lib().snn_set_allocator(_native.ALLOC_FN(0), _native.FREE_FN(0), None))
    _torch_alloc_fns = None


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Network:
    """One simulated grid network resident on the GPU."""

    def __init__(self, params: dict, seed: int, stream=None):
        self._lib = lib()
        self.params = dict(params)
        self.seed = int(seed)
        self._p = make_params(params)
        h = ctypes.c_void_p()
        st = _current_stream() if stream is None else ctypes.c_void_p(int(stream))
        _check(self._lib.snn_build_network(ctypes.byref(self._p), ctypes.c_uint64(self.seed), st, ctypes.byref(h)))
        self._h = h
        self.G = params["gx"] * params["gy"]
        self.N = self.G * K
        self.M = params["out_degree"]

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.snn_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, steps: int) -> None:
        _check(self._lib.snn_run(self._h, ctypes.c_uint64(int(steps))))

    def spikes(self, t0: int = 0, t1: int | None = None):
        """Spikes with t0 <= step < t1 as (steps, ids), ordered by (step, id)."""
        if t1 is None:
            t1 = 1 << 32
        n = ctypes.c_size_t(0)
        rc = self._lib.snn_read_spikes(self._h, t0, t1, None, None, 0, ctypes.byref(n))
        if rc not in (SNN_OK, -5):
            _check(rc)
        st = np.empty(n.value, np.uint32)
        ids = np.empty(n.value, np.uint32)
        _check(self._lib.snn_read_spikes(self._h, t0, t1, _ptr(st), _ptr(ids), n.value, ctypes.byref(n)))
        return st, ids

    def rates(self) -> np.ndarray:
        """Spike counts [bin][module][F, B, I]."""
        n = ctypes.c_size_t(0)
        rc = self._lib.snn_rates(self._h, None, 0, ctypes.byref(n))
        if rc not in (SNN_OK, -5):
            _check(rc)
        out = np.zeros(n.value, np.uint32)
        _check(self._lib.snn_rates(self._h, _ptr(out), n.value, ctypes.byref(n)))
        return out.reshape(-1, self.G, 3)

    def state(self):
        V = np.zeros(self.N, np.float32)
        c = np.zeros(self.N, np.float32)
        ref = np.zeros(self.N, np.int32)
        _check(self._lib.snn_read_state(self._h, _ptr(V), _ptr(c), _ptr(ref), self.N))
        return V, c, ref

    def row(self, s: int):
        keys = np.zeros(self.M, np.uint32)
        w = np.zeros(self.M, np.float32)
        _check(self._lib.snn_read_row(self._h, int(s), _ptr(keys), _ptr(w), self.M))
        return keys, w

    def stats(self) -> dict:
        st = SnnStats()
        _check(self._lib.snn_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in SnnStats._fields_}

    @property
    def launch(self) -> dict:
        c = SnnLaunch()
        _check(self._lib.snn_get_launch(self._h, ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in SnnLaunch._fields_}

    @launch.setter
    def launch(self, cfg: dict) -> None:
        cur = self.launch
        cur.update(cfg)
        c = SnnLaunch(**cur)
        _check(self._lib.snn_set_launch(self._h, ctypes.byref(c)))

    def autotune(self, trial_steps: int = 200, path: int | None = None) -> dict:
        """Choose the launch shape (see snn_autotune); `path` 0 or 1 keeps the
        tuner on that launch path (snn_autotune_path)."""
        if path is None:
            _check(self._lib.snn_autotune(self._h, int(trial_steps)))
        else:
            _check(self._lib.snn_autotune_path(self._h, int(trial_steps), int(path)))
        return self.launch

    def time_kernels(self, steps: int) -> dict:
        """Time the next `steps` steps (see snn_time_kernels): event-bracketed
        spans of the update and delivery launches, and the step time of the same
        steps as a plain graph (ms); the network advances by `steps`."""
        out = (ctypes.c_double * 3)()
        _check(self._lib.snn_time_kernels(self._h, int(steps), out))
        return {"update_ms": out[0], "deliver_ms": out[1], "step_ms": out[2]}



def run_concurrent(nets, steps) -> None:
    """Advance several networks on the two-kernel path, each on its own stream,
    with their kernels overlapping on the GPU (see snn_run_concurrent)."""
    nets = list(nets)
    if isinstance(steps, int):
        steps = [steps] * len(nets)
    hs = (ctypes.c_void_p * len(nets))(*[n.handle.value for n in nets])
    st = (ctypes.c_uint64 * len(nets))(*[int(s) for s in steps])
    _check(lib().snn_run_concurrent(hs, st, len(nets)))


def autotune_batch(nets, trial_steps: int = 200) -> dict:
    """Choose the fused-kernel shape for a batch (see snn_autotune_batch); returns it."""
    nets = list(nets)
    hs = (ctypes.c_void_p * len(nets))(*[n.handle.value for n in nets])
    _check(lib().snn_autotune_batch(hs, len(nets), int(trial_steps)))
    return nets[0].launch


def autotune_concurrent(nets, trial_steps: int = 200) -> list:
    """Choose two-kernel shapes for networks run together by run_concurrent
    (see snn_autotune_concurrent); returns every network's shape."""
    nets = list(nets)
    hs = (ctypes.c_void_p * len(nets))(*[n.handle.value for n in nets])
    _check(lib().snn_autotune_concurrent(hs, len(nets), int(trial_steps)))
    return [n.launch for n in nets]


def run_batch(nets, steps) -> None:
    """Advance several networks together with one fused kernel per time step."""
    nets = list(nets)
    if isinstance(steps, int):
        steps = [steps] * len(nets)
    hs = (ctypes.c_void_p * len(nets))(*[n.handle.value for n in nets])
    st = (ctypes.c_uint64 * len(nets))(*[int(s) for s in steps])
    _check(lib().snn_run_batch(hs, st, len(nets)))
