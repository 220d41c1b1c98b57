"""The C ABI boundary without a GPU: libgcp.so builds for sm_103a, loads,
and exports every entry point include/*.h declares; the binding declares a
signature for each; the oracle library shares nothing with it."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[ \t]*(?!#)[\w \t\*]*?\b(gcp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2605_20353_gb300 import build

    return build.build()


def test_header_declares_the_core_calls():
    names = _declared()
    for n in ["gcp_create", "gcp_sample", "gcp_loss", "gcp_grad", "gcp_adam_step", "gcp_fit"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_path]).decode()
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_loads_and_has_every_signature(lib_path):
    import paper_2605_20353_gb300 as gcp

    lib = gcp.load()
    for n in _declared():
        assert n in gcp.SIGNATURES, f"binding lacks {n}"
        assert hasattr(lib, n)


def test_library_is_built_for_sm_103a_only(lib_path):
    out = subprocess.check_output(["cuobjdump", "--list-elf", lib_path]).decode()
    arches = set(re.findall(r"sm_\d+a?", out))
    assert arches == {"sm_103a"}, arches


def test_oracle_and_gpu_library_share_no_code():
    gpu_src = glob.glob(os.path.join(ROOT, "paper_2605_20353_gb300", "**", "*.*"), recursive=True)
    for f in gpu_src:
        if f.endswith((".cu", ".cuh", ".h", ".py")):
            text = open(f).read()
            assert "oracle" not in re.findall(r"(?:import|include)\s+[\"<]?(\w+)", text), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".c", ".py")):
            text = open(f).read()
            assert "paper_2605_20353_gb300" not in text and "gcp.h" not in text, f


def test_host_argument_checks_need_no_gpu(lib_path):
    """Creation rejects bad arguments on the host before touching the GPU."""
    import ctypes

    import numpy as np

    import paper_2605_20353_gb300 as gcp

    lib = gcp.load()
    dims = np.array([4, 3, 2], dtype=np.int64)
    coords = np.array([[0, 0, 0], [3, 2, 1]], dtype=np.int32)
    vals = np.array([1.0, 2.0], dtype=np.float32)
    h = ctypes.c_void_p()
    bad = np.array([[0, 0, 0], [4, 0, 0]], dtype=np.int32)  # out of range
    assert lib.gcp_create(3, dims.ctypes.data, 2, bad.ctypes.data, vals.ctypes.data, 4, 1, None,
                          ctypes.byref(h)) == 1
    assert b"out of range" in lib.gcp_last_error(None)
    neg = np.array([1.0, -2.0], dtype=np.float32)  # Poisson data must be >= 0
    assert lib.gcp_create(3, dims.ctypes.data, 2, coords.ctypes.data, neg.ctypes.data, 4, 1, None,
                          ctypes.byref(h)) == 8
    nan = np.array([1.0, np.nan], dtype=np.float32)
    assert lib.gcp_create(3, dims.ctypes.data, 2, coords.ctypes.data, nan.ctypes.data, 4, 0, None,
                          ctypes.byref(h)) == 1
    assert h.value is None


def test_factor_list_and_scale_reject_null_arguments_on_the_host(lib_path):
    import paper_2605_20353_gb300 as gcp

    lib = gcp.load()
    assert lib.gcp_set_factor_list(None, None) == 1
    assert lib.gcp_grad_factors_async(None, None, 0, 1, 1, None, None) == 1
    assert lib.gcp_scale_async(None, None, None, None, 4) == 1
    assert lib.gcp_grad_norm(None, None) == 1


def test_l2_probe_rejects_bad_sizes_on_the_host(lib_path):
    """The measurement probe checks its sizes before any CUDA call."""
    import paper_2605_20353_gb300 as gcp

    lib = gcp.load()
    assert lib.gcp_probe_l2(3, 32, 4, 16, 1024, 1, None) == 1  # unknown kind
    assert lib.gcp_probe_l2(0, 24, 4, 16, 1024, 1, None) == 1  # row not a power of two
    assert b"power of two" in lib.gcp_last_error(None)
    assert lib.gcp_probe_l2(0, 32, 9, 16, 1024, 1, None) == 1  # more rows per op than modes
    assert lib.gcp_probe_l2(2, 32, 4, 8, 1024, 1, None) == 1  # unaligned buffer


def test_fit_presets_are_valid_adam_settings():
    import paper_2605_20353_gb300 as gcp

    for name, p in gcp.FIT_PRESETS.items():
        a = p["adam"]
        assert a.lr > 0 and 0 <= a.beta1 < 1 and 0 <= a.beta2 < 1 and a.eps >= 0, name
        assert 0 < p["decay"] < 1, name
    assert gcp.FIT_PRESETS["gcp_sgd_tuned"]["adam"].lr == 0.035817
    assert gcp.FIT_PRESETS["gcp_fedadam_tuned"]["meta_rate"] == 0.029976


def test_binding_refuses_undersized_or_mistyped_buffers():
    """The C ABI takes bare device pointers, so the binding checks element
    type, length and contiguity before it passes an address."""
    import torch

    import paper_2605_20353_gb300 as gcp

    gcp._check_buf(np.zeros(10, np.float32), 10, "float32", "G_out")
    gcp._check_buf(torch.zeros(3, dtype=torch.float64), 1, "float64", "dloss")
    gcp._check_buf(None, 10, "float32", "G_out")
    bad = [
        (np.zeros(9, np.float32), "float32"),                   # too short
        (np.zeros(10, np.float64), "float32"),                  # wrong type
        (np.zeros((10, 2), np.float32)[:, 0], "float32"),       # strided
        (torch.zeros(10, dtype=torch.float32), "float64"),      # a float32 loss buffer
        (torch.zeros(20, dtype=torch.float32)[::2], "float32"),  # strided tensor
    ]
    for buf, dtype in bad:
        with pytest.raises(ValueError):
            gcp._check_buf(buf, 10 if dtype == "float32" else 1, dtype, "buf")
