"""Build and load ``libsnn.so`` (the C ABI of include/snn.h) in-tree.

The library is compiled with nvcc for sm_103a only.  Device code is built with
``-fmad=false`` and host code with ``-ffp-contract=off`` so that no multiply
and add is fused anywhere on the simulation path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
CSRC = os.path.join(_HERE, "csrc")
BUILD = os.path.join(_HERE, "_build")
LIB = os.path.join(BUILD, "libsnn.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off,-O2,-fno-fast-math", f"-I{INCLUDE}"]
SOURCES = ["snn_kernels.cu", "snn_host.cpp", "snn_noalloc.cu"]
HEADERS = ["snn_internal.h", "snn_raster.h"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "snn.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libsnn.so if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, *NVCC_FLAGS, "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj, *ARCH]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lpthread", "-lrt"])
    os.replace(tmp, LIB)
    return LIB


# ---------------------------------------------------------------------------
# ctypes mirror of include/snn.h
# ---------------------------------------------------------------------------
class SnnParams(ctypes.Structure):
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


class SnnStats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_uint64), ("spikes", ctypes.c_uint64), ("rec_events", ctypes.c_uint64),
                ("ext_events", ctypes.c_uint64), ("n_neurons", ctypes.c_uint64), ("n_synapses", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("record_bytes", ctypes.c_uint64), ("build_ms", ctypes.c_double),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64)]


class SnnLaunch(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("update_block", ctypes.c_int32), ("deliver_warps", ctypes.c_int32),
                ("fused_block", ctypes.c_int32), ("fused_items_per_sm", ctypes.c_int32),
                ("window_steps", ctypes.c_int32), ("deliver_lanes", ctypes.c_int32),
                ("update_groups", ctypes.c_int32), ("l2_persist", ctypes.c_int32),
                ("deliver_blocks", ctypes.c_int32), ("overlap", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# every symbol declared in include/snn.h
EXPORTS = ["snn_set_allocator", "snn_footprint", "snn_build_network", "snn_run", "snn_run_batch",
           "snn_read_spikes", "snn_rates", "snn_read_state", "snn_read_row", "snn_get_stats",
           "snn_get_launch", "snn_set_launch", "snn_autotune", "snn_autotune_path", "snn_free", "snn_last_error",
           "snn_time_kernels", "snn_build_rows_static", "snn_run_concurrent",
           "snn_autotune_batch", "snn_autotune_concurrent"]

_lib = None


def load(build_if_needed: bool = True):
    """Load libsnn.so (building it first if needed) and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        build()
    if not os.path.exists(LIB):
        raise RuntimeError(f"native library missing: {LIB}; run paper_1902_08410_gb300.build()")
    lib = ctypes.CDLL(LIB)
    vp, u32, i32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "snn_set_allocator": ([ALLOC_FN, FREE_FN, vp], ctypes.c_int),
        "snn_footprint": ([P(SnnParams), P(sz)], ctypes.c_int),
        "snn_build_network": ([P(SnnParams), u64, vp, P(vp)], ctypes.c_int),
        "snn_run": ([vp, u64], ctypes.c_int),
        "snn_run_batch": ([P(vp), P(u64), i32], ctypes.c_int),
        "snn_run_concurrent": ([P(vp), P(u64), i32], ctypes.c_int),
        "snn_read_spikes": ([vp, u64, u64, vp, vp, sz, P(sz)], ctypes.c_int),
        "snn_rates": ([vp, vp, sz, P(sz)], ctypes.c_int),
        "snn_read_state": ([vp, vp, vp, vp, sz], ctypes.c_int),
        "snn_read_row": ([vp, u32, vp, vp, sz], ctypes.c_int),
        "snn_get_stats": ([vp, P(SnnStats)], ctypes.c_int),
        "snn_get_launch": ([vp, P(SnnLaunch)], ctypes.c_int),
        "snn_set_launch": ([vp, P(SnnLaunch)], ctypes.c_int),
        "snn_autotune": ([vp, u32], ctypes.c_int),
        "snn_autotune_path": ([vp, u32, i32], ctypes.c_int),
        "snn_autotune_batch": ([P(vp), i32, u32], ctypes.c_int),
        "snn_autotune_concurrent": ([P(vp), i32, u32], ctypes.c_int),
        "snn_free": ([vp], None),
        "snn_last_error": ([], ctypes.c_char_p),
        "snn_time_kernels": ([vp, u32, P(ctypes.c_double)], ctypes.c_int),
        "snn_build_rows_static": ([P(SnnParams), u64, vp, P(sz), vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib
