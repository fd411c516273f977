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


def _header_params():
    """name -> (return type, [parameter types]) of every declaration in
    include/kmx.h, comments removed."""
    out = {}
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*((?:const\s+)?[\w\s\*]+?)\b(kmx_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.M):
            ret, name, args = m.group(1).strip(), m.group(2), m.group(3).strip()
            params = [] if args in ("", "void") else [" ".join(a.split()) for a in args.split(",")]
            out[name] = (ret, params)
    return out


def _kind_of_c(decl):
    """The ctypes kind a C parameter or return type needs."""
    d = decl.replace("const ", "")
    if "*" in d:
        return "char_p" if re.match(r"^char\s*\*$", d.strip()) else "pointer"
    base = d.split()[0]
    return {"int64_t": "i64", "int32_t": "i32", "int": "i32", "kmx_status": "i32", "float": "f32",
            "double": "f64", "void": "void", "size_t": "u64"}[base]


def _kind_of_ctypes(t):
    import ctypes as C

    if t is None:
        return "void"
    if t is C.c_char_p:
        return "char_p"
    if t is C.c_void_p or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "pointer"
    return {C.c_int64: "i64", C.c_int32: "i32", C.c_float: "f32", C.c_double: "f64", C.c_uint64: "u64"}[t]


def test_binding_signatures_match_the_header():
    """Every entry point the ctypes binding declares has the header's
    parameter count and, position by position, the same kind (pointer, int32,
    int64, float, double): a call through the binding passes what the C ABI
    expects."""
    from paper_2409_15615_gb300 import kmx

    hdr = _header_params()
    for name, (res, args) in kmx.signatures().items():
        assert name in hdr, name
        ret, params = hdr[name]
        assert len(params) == len(args), (name, params, args)
        # a parameter's type is everything but its name
        want = []
        for p in params:
            m = re.match(r"^(.*?)(\w+)$", p)
            want.append(_kind_of_c(m.group(1).strip()))
        got = [_kind_of_ctypes(a) for a in args]
        assert want == got, (name, want, got)
        assert _kind_of_c(ret) == _kind_of_ctypes(res), (name, ret, res)
