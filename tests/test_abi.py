"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/ofv.h declares, and rejects bad arguments before
touching the device.  Also checks that the oracle and the CUDA path share
no code."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2509_25924_gb300 as ofv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ofv_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_function():
    declared = _declared_functions()
    assert declared, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", ofv.lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (ofv_[a-z0-9_]+)", out))
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    lib = ctypes.CDLL(ofv.lib_path)
    for name in declared:
        assert hasattr(lib, name)


def test_binding_names_match_the_header():
    declared = _declared_functions()
    for name in declared:
        assert hasattr(ofv, name), f"binding lacks {name}"


def test_defaults_follow_the_documented_values():
    p = ofv.ofv_default_params()
    assert (p.levels_psl, p.kernel_radius, p.iterations, p.norm_radius) == (2, 4, 3, 0)
    assert (p.input, p.bit_depth, p.storage, p.path, p.prefilter) == (ofv.OFV_IN_U16, 12, ofv.OFV_STORE_F32,
                                                                      ofv.OFV_PATH_FUSED, 0)
    assert abs(p.det_rel_eps - 1e-6) < 1e-12 and abs(p.norm_eps - 1e-2) < 1e-9
    assert (p.window, p.window_sigma, p.increment_form, p.warm_start) == (ofv.OFV_WINDOW_BOX, 0.0, 0, 0)
    assert p.tile_edge == 0


@pytest.mark.parametrize("cname,mirror", [("ofv_params", "Params"), ("ofv_pair", "Pair")])
def test_struct_layout_matches_the_header(tmp_path, cname, mirror):
    """The ctypes mirrors of ofv_params and ofv_pair have the C structs' size
    and field offsets (compiled against include/ofv.h with the host compiler)."""
    cls = getattr(ofv, mirror)
    names = [f[0] for f in cls._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'    printf("%zu\\n", offsetof({cname}, {n}));\n' for n in names)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "ofv.h"\nint main(void) {\n'
                   f'    printf("%zu\\n", sizeof({cname}));\n' + body + '    return 0;\n}\n')
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call(["gcc", "-I", inc, str(src), "-o", str(exe)])
    out = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert out[0] == ctypes.sizeof(cls)
    assert out[1:] == [getattr(cls, n).offset for n in names]


@pytest.mark.parametrize("field,value", [
    ("levels_psl", -1), ("levels_psl", 16), ("kernel_radius", 0), ("kernel_radius", 17),
    ("iterations", 0), ("iterations", 65), ("norm_radius", -1), ("input", 7), ("storage", 3),
    ("path", 3), ("prefilter", 2), ("bit_depth", 0), ("bit_depth", 17), ("det_rel_eps", float("nan")),
    ("norm_eps", 0.0), ("max_batch", -1), ("max_batch", 9), ("window", 2), ("window", -1),
    ("increment_form", 2), ("warm_start", -1), ("warm_start", 57), ("tile_edge", -1), ("tile_edge", 40),
    ("tile_edge", 16), ("tile_edge", 64),
])
def test_invalid_parameters_are_rejected_on_the_host(field, value):
    p = ofv.ofv_default_params(**{field: value})
    with pytest.raises(ofv.OfvError) as ei:
        ofv.ofv_create(1024, 1024, p)
    assert ei.value.status == ofv.OFV_ERR_INVALID_ARG


@pytest.mark.parametrize("kw", [dict(kernel_radius=12, tile_edge=48), dict(path=ofv.OFV_PATH_PLAIN, tile_edge=32),
                                dict(kernel_radius=6, tile_edge=48), dict(kernel_radius=8, tile_edge=48)])
def test_tile_edge_must_be_one_of_the_radius_edges_on_the_block_path(kw):
    """The block kernel (fused path, KR 1..10) has two tile edges per radius:
    48 or 32 for KR <= 5, 64 or 32 for KR 6..10."""
    p = ofv.ofv_default_params(levels_psl=1, **kw)
    with pytest.raises(ofv.OfvError) as ei:
        ofv.ofv_create(1024, 1024, p)
    assert ei.value.status == ofv.OFV_ERR_INVALID_ARG


@pytest.mark.parametrize("sigma", [0.0, -1.0, float("nan"), float("inf")])
def test_gaussian_window_needs_a_finite_positive_sigma(sigma):
    p = ofv.ofv_default_params(window=ofv.OFV_WINDOW_GAUSS, window_sigma=sigma)
    with pytest.raises(ofv.OfvError) as ei:
        ofv.ofv_create(256, 256, p)
    assert ei.value.status == ofv.OFV_ERR_INVALID_ARG


def test_u8_bit_depth_limit():
    p = ofv.ofv_default_params(input=ofv.OFV_IN_U8, bit_depth=12)
    with pytest.raises(ofv.OfvError) as ei:
        ofv.ofv_create(256, 256, p)
    assert ei.value.status == ofv.OFV_ERR_INVALID_ARG


@pytest.mark.parametrize("H,W,psl,kr", [(32, 32, 2, 4), (64, 17, 1, 5), (0, 64, 0, 1), (64, 64, 3, 4),
                                        (100000, 100000, 0, 1)])
def test_shape_limits(H, W, psl, kr):
    p = ofv.ofv_default_params(levels_psl=psl, kernel_radius=kr)
    with pytest.raises(ofv.OfvError) as ei:
        ofv.ofv_create(H, W, p)
    assert ei.value.status == ofv.OFV_ERR_SHAPE
    assert "coarsest" in ofv.ofv_last_error() or "H" in ofv.ofv_last_error()


def test_null_arguments_are_rejected():
    lib = ctypes.CDLL(ofv.lib_path)
    lib.ofv_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.ofv_create.restype = ctypes.c_int
    assert lib.ofv_create(64, 64, None, None) == ofv.OFV_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    assert lib.ofv_create(64, 64, None, ctypes.byref(out)) == ofv.OFV_ERR_INVALID_ARG
    assert out.value is None
    lib.ofv_compute.argtypes = [ctypes.c_void_p] * 6
    lib.ofv_compute.restype = ctypes.c_int
    assert lib.ofv_compute(None, None, None, None, None, None) == ofv.OFV_ERR_INVALID_ARG
    lib.ofv_destroy.argtypes = [ctypes.c_void_p]
    lib.ofv_destroy.restype = ctypes.c_int
    assert lib.ofv_destroy(None) == ofv.OFV_OK


def test_null_arguments_of_the_later_entry_points_are_rejected():
    lib = ctypes.CDLL(ofv.lib_path)
    P, I, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    lib.ofv_compute_sequence_host.argtypes = [P, I, P, Z, P, P, Z, P]
    lib.ofv_compute_sequence_host.restype = I
    assert lib.ofv_compute_sequence_host(None, 3, None, 0, None, None, 0, None) == ofv.OFV_ERR_INVALID_ARG
    lib.ofv_backward.argtypes = [P] * 9
    lib.ofv_backward.restype = I
    assert lib.ofv_backward(None, None, None, None, None, None, None, None, None) == ofv.OFV_ERR_INVALID_ARG
    lib.ofv_vorticity.argtypes = [I, I, I, P, P, Z, P, P]
    lib.ofv_vorticity.restype = I
    assert lib.ofv_vorticity(8, 8, 1, None, None, 64, None, None) == ofv.OFV_ERR_INVALID_ARG
    lib.ofv_recirculation_area.argtypes = [I, I, I, P, Z, P, P, P]
    lib.ofv_recirculation_area.restype = I
    assert lib.ofv_recirculation_area(8, 8, 1, None, 64, None, None, None) == ofv.OFV_ERR_INVALID_ARG
    # shape and stride checks come before any device work
    dummy = ctypes.c_void_p(16)
    assert lib.ofv_vorticity(0, 8, 1, dummy, dummy, 64, dummy, None) == ofv.OFV_ERR_SHAPE
    assert lib.ofv_vorticity(8, 8, 1, dummy, dummy, 63, dummy, None) == ofv.OFV_ERR_INVALID_ARG
    assert lib.ofv_recirculation_area(8, 8, 0, dummy, 64, None, dummy, None) == ofv.OFV_ERR_SHAPE
    lib.ofv_probe.argtypes = [I, I, I, P, P, Z, I, P, P, P]
    lib.ofv_probe.restype = I
    assert lib.ofv_probe(8, 8, 1, None, dummy, 64, 4, dummy, dummy, None) == ofv.OFV_ERR_INVALID_ARG
    assert lib.ofv_probe(8, 8, 1, dummy, dummy, 64, 0, dummy, dummy, None) == ofv.OFV_ERR_SHAPE
    assert lib.ofv_probe(8, 8, 1, dummy, dummy, 63, 4, dummy, dummy, None) == ofv.OFV_ERR_INVALID_ARG
    assert lib.ofv_probe(8, 8, 1, dummy, dummy, 64, 4, ctypes.c_void_p(20), dummy, None) == ofv.OFV_ERR_INVALID_ARG
    lib.ofv_set_mask.argtypes = [P, P, P]
    lib.ofv_set_mask.restype = I
    assert lib.ofv_set_mask(None, dummy, None) == ofv.OFV_ERR_INVALID_ARG


def test_status_strings():
    assert ofv.ofv_status_string(ofv.OFV_ERR_SHAPE) == "OFV_ERR_SHAPE"
    assert ofv.ofv_status_string(99) == "OFV_ERR_UNKNOWN"


def _py_and_c_sources(d):
    for base, _, files in os.walk(os.path.join(ROOT, d)):
        for f in files:
            if f.endswith((".py", ".c", ".h", ".cu", ".cuh", ".cpp")):
                yield os.path.join(base, f)


def test_oracle_and_cuda_path_share_no_code():
    for f in _py_and_c_sources("oracle"):
        text = open(f).read()
        assert "paper_2509_25924_gb300" not in text and "ofv.h" not in text, f
    for f in _py_and_c_sources("paper_2509_25924_gb300"):
        text = open(f).read()
        assert not re.search(r"\boracle\b", text.replace("oracle-free", "")), f
        assert "ofv_oracle" not in text, f


def test_batched_rejects_bad_arguments_on_the_host():
    p = ofv.ofv_default_params()
    lib = ctypes.CDLL(ofv.lib_path)
    lib.ofv_compute_batched.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.ofv_compute_batched.restype = ctypes.c_int
    assert lib.ofv_compute_batched(None, 1, None, None) == ofv.OFV_ERR_INVALID_ARG
    lib.ofv_graph_create_batched.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.ofv_graph_create_batched.restype = ctypes.c_int
    out = ctypes.c_void_p(1)
    assert lib.ofv_graph_create_batched(None, 1, None, None) == ofv.OFV_ERR_INVALID_ARG
    assert lib.ofv_graph_create_batched(None, 1, None, ctypes.byref(out)) == ofv.OFV_ERR_INVALID_ARG
    assert out.value is None  # *out is cleared on failure


def _prototypes():
    """name -> list of parameter declarations of every ofv_* function in include/*.h."""
    out = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ofv_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", text):
            params = [p.strip() for p in m.group(2).split(",")]
            out[m.group(1)] = [] if params in ([""], ["void"]) else params
    return out


def _c_kind(decl):
    if "*" in decl or "ofv_stream_t" in decl:
        return "pointer"
    if "size_t" in decl:
        return "size_t"
    if "double" in decl or "float" in decl:
        return "float"
    return "int"  # int and the enum types


def _ctypes_kind(t):
    if t is ctypes.c_void_p or t is ctypes.c_char_p or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "pointer"
    if t is ctypes.c_size_t:
        return "size_t"
    if t in (ctypes.c_float, ctypes.c_double):
        return "float"
    return "int"


def test_binding_argtypes_match_the_header_prototypes():
    """Each bound entry point takes as many arguments as its prototype, of
    the same kinds (pointer, size_t, int, floating point)."""
    protos = _prototypes()
    assert protos, "no prototypes found"
    lib = ofv._lib
    for name, params in protos.items():
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None, f"{name}: no argtypes set"
        assert len(argtypes) == len(params), f"{name}: {len(argtypes)} argtypes, prototype has {len(params)}"
        for k, (decl, t) in enumerate(zip(params, argtypes)):
            assert _c_kind(decl) == _ctypes_kind(t), f"{name} argument {k} ({decl!r}) bound as {t}"
