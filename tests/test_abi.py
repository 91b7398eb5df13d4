"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/snn.h declares, and its host-side logic (argument checks,
footprint, failure without a device) behaves as documented."""
import ctypes
import os
import re

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def snn():
    import paper_1902_08410_gb300 as snn
    snn.build()
    return snn


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "snn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(snn_[a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_expected_entry_points():
    names = _declared_functions()
    for required in ("snn_build_network", "snn_run", "snn_read_spikes", "snn_rates", "snn_run_batch"):
        assert required in names


def test_library_exports_every_declared_symbol(snn):
    from paper_1902_08410_gb300 import _native
    lib = ctypes.CDLL(_native.LIB)
    names = _declared_functions()
    assert set(names) == set(_native.EXPORTS), set(names) ^ set(_native.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_footprint_host_only(snn):
    p = W.base_params(24, 24, 1.0)
    b = snn.footprint(p)
    N = 24 * 24 * 1250
    records = N * 1128 * 8
    assert records < b < records * 1.2
    p16 = W.base_params(24, 24, 1.0, record_format=W.REC_I16)
    assert snn.footprint(p16) < b


def test_footprint_follows_min_delay(snn):
    """2 max(1, min_delay) input buffers and a history of n_delay + max(1, min_delay)
    step slots, int32 per padded neuron each (include/snn.h, snn_footprint)."""
    p1 = W.base_params(2, 2, 1.0)
    p10 = dict(p1, min_delay=10)
    n_pad = 5120                                   # 5000 neurons rounded up to 128
    extra_buffers = (2 * 10 - 2 * 1) * n_pad * 4
    extra_history = ((20 + 10) - (20 + 1)) * n_pad * 4
    assert snn.footprint(p10) - snn.footprint(p1) == extra_buffers + extra_history
    assert snn.footprint(dict(p1, min_delay=0)) == snn.footprint(p1)   # 0 is read as 1


@pytest.mark.parametrize("field,value,code", [
    ("gx", 0, -1), ("lambda", 0.0, -1), ("n_delay", 0, -1), ("n_delay", 300, -1),
    ("record_format", 7, -1), ("out_degree", 5000, -6), ("gx", 120, -6), ("bin_steps", 0, -1),
    ("min_delay", 21, -1), ("min_delay", -1, -1),
])
def test_invalid_parameters_rejected(snn, field, value, code):
    p = W.base_params(2, 2, 1.0)
    p[field] = value
    if field == "gx" and value == 120:
        p["gy"] = 120          # 18M neurons: beyond the 24-bit target index
    with pytest.raises(snn.SnnError) as ei:
        snn.footprint(p)
    assert ei.value.code == code


def test_no_cpu_fallback_without_gpu(snn):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(snn.SnnError) as ei:
        snn.Network(W.base_params(1, 1, 1.0), 1, stream=0)
    assert ei.value.code == -3
