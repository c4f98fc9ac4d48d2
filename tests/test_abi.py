"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function include/knnd.h declares, and rejects
bad arguments on the host before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2202_00517_gb300 import _lib, build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "knnd.h")


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return _lib.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(knnd_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_exported(lib):
    names = _declared()
    assert "knnd_build" in names and "knnd_round" in names and "knnd_init_graph" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(_lib.EXPORTS) == names


def test_version_and_status_strings(lib):
    assert lib.knnd_version() >= 100
    for code in range(0, -8, -1):
        s = _lib.status_string(code)
        assert s and s != "unknown status"
    assert _lib.status_string(-99) == "unknown status"


def test_struct_layouts():
    # host structs of the header: twelve int32 params and a float; build info 8 + 64*8 + 65*8 + 7*8 + 8
    # bytes; stats 3 int64 + 6 int64 + 6 double
    assert ctypes.sizeof(_lib.knnd_params) == 52
    assert ctypes.sizeof(_lib.knnd_build_info) == 8 + 64 * 8 + 65 * 8 + 7 * 8 + 8
    assert ctypes.sizeof(_lib.knnd_stats) == 3 * 8 + 6 * 8 + 6 * 8


@pytest.mark.parametrize("n,m,K,dtype,prec", [
    (1000, 6, 1, 0, 1),          # K < 2
    (1000, 6, 65, 0, 1),         # K > KNND_MAX_K
    (10, 6, 10, 0, 1),           # K >= n
    (1000, 0, 10, 0, 1),         # m < 1
    (1000, 129, 10, 0, 1),       # m > KNND_MAX_M
    (2**31, 6, 10, 0, 1),        # n >= 2^31
    (2, 6, 1, 0, 1),             # n < 3
    (1000, 6, 10, 7, 1),         # bad dtype
    (1000, 6, 10, 0, 9),         # bad precision
])
def test_create_rejects_bad_shapes(lib, n, m, K, dtype, prec):
    h = ctypes.c_void_p(1234)
    st = lib.knnd_create(ctypes.byref(h), n, m, K, dtype, prec, None, None)
    assert st == _lib.KNND_EINVAL
    assert h.value is None


def test_create_rejects_bad_params(lib):
    h = ctypes.c_void_p()
    for prm in (_lib.knnd_params(0, 10, 1, 0, 0, 1), _lib.knnd_params(100, 0, 1, 0, 0, 1),
                _lib.knnd_params(100, 65, 1, 0, 0, 1), _lib.knnd_params(100, 10, 1, 0, 0, 2),
                _lib.knnd_params(100, 10, 1, 0, 0, 0, -0.5), _lib.knnd_params(100, 10, 1, 0, 0, 0, 2.0),
                _lib.knnd_params(100, 10, 1, 0, 0, 0, 0.0, 4),             # no such comparator
                _lib.knnd_params(100, 10, 1, 0, 0, 0, 0.0, 0, 3),         # no such loop
                _lib.knnd_params(100, 10, 1, 0, 1, 0, 0.0, 0, _lib.KNND_LOOP_GRAPH),  # graph loop with timing
                _lib.knnd_params(100, 10, 1, 0, 0, 0, 0.0, 0, 0, 65),     # split share out of range
                _lib.knnd_params(100, 10, 1, 0, 0, 0, 0.0, 0, 0, -1),
                _lib.knnd_params(100, 10, 1, 0, 0, 0, 0.0, 0, 0, 0, 5),   # merge keeps 4 or 8
                _lib.knnd_params(100, 10, 1, 0, 0, 0, 0.0, 0, 0, 0, 0, 9),   # join blocks out of range
                _lib.knnd_params(100, 10, 1, 0, 0, 0, 0.0, 0, 0, 0, 0, 0, 3)):  # no such join form
        assert lib.knnd_create(ctypes.byref(h), 1000, 6, 10, 0, 1, ctypes.byref(prm), None) == _lib.KNND_EINVAL
    assert lib.knnd_create(None, 1000, 6, 10, 0, 1, None, None) == _lib.KNND_EINVAL


def test_null_handle_calls(lib):
    info = _lib.knnd_build_info()
    st = _lib.knnd_stats()
    assert lib.knnd_build(None, None, 6, 0, None, None, None, ctypes.byref(info)) == _lib.KNND_EINVAL
    assert lib.knnd_build_host(None, None, 6, 0, None, None, ctypes.byref(info)) == _lib.KNND_EINVAL
    assert lib.knnd_round(None, None, 6, 0, 1, None, None, None, None, None) == _lib.KNND_EINVAL
    assert lib.knnd_init_graph(None, None, 6, 0, None, None, None) == _lib.KNND_EINVAL
    assert lib.knnd_prepare(None, None, 6) == _lib.KNND_EINVAL
    assert lib.knnd_fcc(None, None, 0, 0, None) == _lib.KNND_EINVAL
    assert lib.knnd_sync(None) == _lib.KNND_EINVAL
    assert lib.knnd_set_stream(None, None) == _lib.KNND_EINVAL
    assert lib.knnd_get_stats(None, ctypes.byref(st)) == _lib.KNND_EINVAL
    assert lib.knnd_reset_stats(None) == _lib.KNND_EINVAL
    lib.knnd_destroy(None)


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2202_00517_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_binding_argument_checks(lib):
    # the Python binding rejects bad tensors itself (ValueError, also under
    # python -O) before the library or a device is reached
    import torch

    from paper_2202_00517_gb300 import api
    p = torch.rand(50, 4, dtype=torch.float64)
    with pytest.raises(ValueError):
        api.build_batched([], [], [])
    with pytest.raises(ValueError):
        api.build_batched([p, p], [5], [1, 2])      # one K for two instances
    with pytest.raises(ValueError):
        api.build_batched([p], [5], [1])            # host tensor
    h = api.Handle.__new__(api.Handle)              # no device: checks only
    h.n, h.m, h.K, h.torch_dtype = 50, 4, 5, torch.float64
    with pytest.raises(ValueError):
        h._check_points(p)                          # host tensor
    with pytest.raises(ValueError):
        h.build_host(p.t().contiguous().t(), 1)     # coordinates not contiguous
    with pytest.raises(ValueError):
        h.build_host(p[:40], 1)                     # wrong n
    with pytest.raises(ValueError):
        h.build_host(p.float(), 1)                  # wrong dtype


def test_header_constants_match_the_binding():
    # every integer #define of include/knnd.h has the same value in the binding
    text = open(HEADER).read()
    found = 0
    for name, expr in re.findall(r"^#define\s+(KNND_[A-Z0-9_]+)\s+([-()0-9<\s]+?)\s*(?:/\*.*)?$", text, flags=re.M):
        value = eval(expr, {"__builtins__": {}})  # digits, parentheses, minus and shifts only
        if name.startswith("KNND_PHASE_"):
            assert _lib.PHASES[value] == name[len("KNND_PHASE_"):].lower(), name
        else:
            assert getattr(_lib, name) == value, name
        found += 1
    assert found >= 35


def test_header_structs_match_the_binding():
    # field names, order and widths of every struct of include/knnd.h equal the
    # binding's ctypes layout (a size check alone misses two swapped fields)
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    width = {"int32_t": 4, "int64_t": 8, "uint64_t": 8, "float": 4, "double": 8}
    consts = {k: getattr(_lib, k) for k in dir(_lib) if k.startswith("KNND_")}
    structs = re.findall(r"typedef struct\s*\{(.*?)\}\s*(knnd_\w+)\s*;", text, flags=re.S)
    assert {s for _, s in structs} >= {"knnd_params", "knnd_build_info", "knnd_stats", "knnd_instance"}
    for body, name in structs:
        fields = re.findall(r"([\w\s]+?\*?)\s*\b(\w+)\s*(?:\[([^\]]+)\])?\s*;", body)
        py = getattr(_lib, name)._fields_
        assert [f[1] for f in fields] == [f[0] for f in py], name
        for (ctype, fname, dim), (_, pytype) in zip(fields, py):
            ctype = ctype.replace("const", "").strip()
            n = eval(dim, {"__builtins__": {}}, consts) if dim else 1
            w = 8 if ctype.endswith("*") else width[ctype]
            assert ctypes.sizeof(pytype) == w * n, f"{name}.{fname}"


def test_missing_library_fails_loudly(monkeypatch):
    # no silent fallback: without the built CUDA library the binding raises
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(os.path.join(ROOT, "no_such_dir", "libknnd.so"))


def test_binding_signatures_match_the_prototypes(lib):
    # each function the binding types takes as many arguments as its prototype
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = dict(re.findall(r"\b(knnd_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S))
    for name in _lib.EXPORTS:
        args = protos[name].strip()
        n = 0 if args in ("", "void") else args.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, name
