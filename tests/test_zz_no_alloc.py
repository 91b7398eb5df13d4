"""snn_build_rows_static: construction into caller-owned device memory with no
device allocation by the library.

The entry point serves callers that cannot let a library call cudaMalloc (all
device memory handed out by their own pool, or a loop that cannot take
cudaMalloc's latency).  Its rows must be the same bytes as those of
snn_build_network; the check is bit-exact, like every other row comparison in
these tests, on two calls in a row (the second reusing the static scratch the
first one filled).
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1902_08410_gb300 as snn
    snn.build()
    return snn, torch


def _row_bytes(p):
    m_pad = (p["out_degree"] + 7) // 8 * 8
    return m_pad, m_pad * 4 + m_pad * (2 if p["record_format"] == W.REC_I16 else 4)


def _build_static(snn, torch, p, seed):
    lib = snn.lib()
    pp = snn.make_params(p)
    need = ctypes.c_size_t(0)
    assert lib.snn_build_rows_static(ctypes.byref(pp), seed, None, ctypes.byref(need), None) == 0
    buf = torch.empty(need.value, dtype=torch.uint8, device="cuda")   # caller-owned memory
    have = ctypes.c_size_t(need.value)
    stream = torch.cuda.current_stream()
    rc = lib.snn_build_rows_static(ctypes.byref(pp), seed, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(have),
                                   ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.snn_last_error()
    torch.cuda.synchronize()
    return buf.cpu().numpy()


def _compare(snn, p, seed, host_rows, sources=None):
    net = snn.Network(p, seed)
    m_pad, rb = _row_bytes(p)
    M = p["out_degree"]
    rows = host_rows.reshape(net.N, rb)
    for s in (range(net.N) if sources is None else sources):
        keys, w = net.row(s)
        got_keys = rows[s, :M * 4].view(np.uint32)
        assert np.array_equal(got_keys, keys), s
        if p["record_format"] == W.REC_I16:
            got_w = rows[s, m_pad * 4:m_pad * 4 + M * 2].view(np.int16).astype(np.float32) / np.float32(1024.0)
        else:
            got_w = rows[s, m_pad * 4:m_pad * 4 + M * 4].view(np.float32)
        assert np.array_equal(got_w, w), s
    net.close()


def test_static_scratch_rows_match_build_network_twice(env):
    snn, torch = env
    cases = [(W.base_params(3, 2, 0.4, record_format=W.REC_F32), 5),
             (W.base_params(2, 2, 1.0, "AW", record_format=W.REC_I16, p_local=-1.0), 9)]
    for p, seed in cases:           # two calls in a row, different grids and formats
        _compare(snn, p, seed, _build_static(snn, torch, p, seed))


def test_static_scratch_limits(env):
    snn, torch = env
    lib = snn.lib()
    big = snn.make_params(W.base_params(40, 40, 1.0))        # 1600 modules > 1024
    n = ctypes.c_size_t(1 << 40)
    assert lib.snn_build_rows_static(ctypes.byref(big), 1, ctypes.c_void_p(16), ctypes.byref(n), None) == -6
    small = snn.make_params(W.base_params(2, 2, 1.0))
    need = ctypes.c_size_t(0)
    assert lib.snn_build_rows_static(ctypes.byref(small), 1, None, ctypes.byref(need), None) == 0
    buf = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    short = ctypes.c_size_t(need.value - 16)
    assert lib.snn_build_rows_static(ctypes.byref(small), 1, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(short),
                                     None) == -5
    assert short.value == need.value


def test_static_scratch_at_its_module_limit(env):
    """Exactly 1024 modules (32x32, the most the static scratch serves): the
    threshold table fills its whole region and the Gaussian table sits right
    behind it.  Sampled rows, the first and the last source included."""
    snn, torch = env
    p = W.base_params(32, 32, 1.0, record_format=W.REC_I16)
    p["out_degree"] = 8
    rows = _build_static(snn, torch, p, 3)
    n = 32 * 32 * W.K
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([[0, 1, 1249, 1250, n // 2, n - 1251, n - 1],
                                       rng.integers(0, n, 200)]))
    _compare(snn, p, 3, rows, sample)


def test_static_scratch_refuses_a_capturing_stream(env):
    """The tables are uploaded from host memory that the call frees on return,
    so a call on a stream being captured into a graph is refused."""
    import os
    snn, torch = env
    lib = snn.lib()
    cudart = None
    for cand in (os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcudart.so"),
                 "libcudart.so"):
        try:
            cudart = ctypes.CDLL(cand)
            break
        except OSError:
            continue
    if cudart is None:
        pytest.skip("libcudart.so not found")
    p = W.base_params(2, 2, 1.0)
    pp = snn.make_params(p)
    need = ctypes.c_size_t(0)
    assert lib.snn_build_rows_static(ctypes.byref(pp), 1, None, ctypes.byref(need), None) == 0   # warm-up
    buf = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    capture_thread_local = 1                               # cudaStreamCaptureModeThreadLocal
    assert cudart.cudaStreamBeginCapture(sp, capture_thread_local) == 0
    have = ctypes.c_size_t(need.value)
    rc = lib.snn_build_rows_static(ctypes.byref(pp), 1, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(have), sp)
    graph = ctypes.c_void_p()
    assert cudart.cudaStreamEndCapture(sp, ctypes.byref(graph)) == 0
    if graph.value:
        cudart.cudaGraphDestroy(graph)
    assert rc == -1, lib.snn_last_error()
    # the stream is usable afterwards
    rc = lib.snn_build_rows_static(ctypes.byref(pp), 1, ctypes.c_void_p(buf.data_ptr()), ctypes.byref(have), sp)
    assert rc == 0, lib.snn_last_error()
    stream.synchronize()
