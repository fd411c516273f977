"""The C-ABI library builds for sm_103a and exports every entry point that
include/kmx.h declares (CPU only: symbols are resolved, nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\*\s]+?\b(kmx_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import shutil

    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2409_15615_gb300 import build

    return ctypes.CDLL(build.build())


def test_header_declares_the_stage_calls():
    names = _declared()
    for n in ("kmx_voxelize", "kmx_build_grid", "kmx_normals", "kmx_fasterpfh", "kmx_match", "kmx_create",
              "kmx_sync", "kmx_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_default_is_host_only(lib):
    # kmx_params_default touches no device: callable without a GPU
    from paper_2409_15615_gb300 import kmx

    p = kmx.params_default(0.1, viewpoint=(1.0, 2.0, 3.0))
    assert abs(p.r_normal - 0.35) < 1e-6 and abs(p.r_fpfh - 0.5) < 1e-6
    assert p.tau_num == 3 and abs(p.tau_lin - 0.99) < 1e-7 and p.hist_bins == 11
    assert list(p.viewpoint) == [1.0, 2.0, 3.0]
    bad = kmx.Params()
    assert kmx.library().kmx_params_default(-1.0, ctypes.byref(bad)) == kmx.KMX_EINVAL


def test_context_setters_refuse_a_null_context_without_a_device(lib):
    # argument checks come before any CUDA call, so they run without a GPU
    from paper_2409_15615_gb300 import kmx

    L = kmx.library()
    assert L.kmx_set_match_residency(None, 1) == kmx.KMX_EINVAL
    assert L.kmx_set_stream(None, None) == kmx.KMX_EINVAL
    assert L.kmx_reserve(None, 0) == kmx.KMX_EINVAL
    assert L.kmx_sync(None) == kmx.KMX_EINVAL


def test_pair_stream_needs_a_slot():
    from paper_2409_15615_gb300 import pipeline

    with pytest.raises(ValueError):
        pipeline.PairStream(None, 1, 1, slots=0)
