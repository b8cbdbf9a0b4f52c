"""The C-ABI library loads and exports every entry point of include/lsh.h, and its
host-only validation (workspace sizing) behaves; no GPU calls."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1411_0330_gb300 import lsh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1411_0330_gb300 import build
    build.build()
    return lsh.load_library(build_if_missing=False)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lsh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsh_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lsh.EXPORTS)


def test_status_strings(lib):
    for s in range(10):
        assert lib.lsh_status_string(s)
    assert lib.lsh_status_string(0) == b"ok"


K1, MU1 = 0.8333333333333334, 0.38461538461538464
K2, MU2 = 5.555555555555555, 4.166666666666667
EL = np.array([[K1, MU1], [K2, MU2]])


def test_workspace_size_scales(lib):
    s64 = lsh.workspace_size((64, 64, 64), EL, physics=lsh.ELASTIC, green=lsh.FILTERED)
    s128 = lsh.workspace_size((128, 128, 128), EL, physics=lsh.ELASTIC, green=lsh.FILTERED)
    assert 7.5 < s128 / s64 < 8.5
    # all 6 load systems at once: 6 x (4 FP64 fields + spectrum) + shared table
    assert 2.5e9 < s128 < 4.0e9
    one = lsh.workspace_size((128, 128, 128), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, max_systems=1)
    assert 0.5e9 < one < 1.0e9
    mixed = lsh.workspace_size((128, 128, 128), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    assert mixed > s128
    batch = lsh.workspace_size((32, 32, 32), EL, physics=lsh.ELASTIC, nbatch=10, max_systems=12)
    assert batch < lsh.workspace_size((32, 32, 32), EL, physics=lsh.ELASTIC, nbatch=10)


@pytest.mark.parametrize("shape", [(32, 32), (7, 5), (12, 10, 6), (1, 3, 4), (48, 96, 32), (256, 256, 256)])
def test_supported_sizes(lib, shape):
    d = len(shape)
    assert lsh.workspace_size(shape, np.array([np.eye(d), 3 * np.eye(d)])) > 0


@pytest.mark.parametrize("shape", [(11, 8), (8, 8, 13)])
def test_unsupported_prime_factor(lib, shape):
    d = len(shape)
    with pytest.raises(lsh.LSHError) as e:
        lsh.workspace_size(shape, np.array([np.eye(d)]))
    assert e.value.status == lsh.ERR_UNSUPPORTED_SIZE


def test_invalid_arguments(lib):
    with pytest.raises(lsh.LSHError) as e:  # elasticity needs dim 3
        lsh.workspace_size((8, 8), EL, physics=lsh.ELASTIC)
    assert e.value.status == lsh.ERR_INVALID_ARG
    # anisotropic conductivities that share eigenvectors with A0 are accepted ...
    lsh.workspace_size((8, 8), np.array([[[2.0, 0.5], [0.5, 1.0]]]))
    with pytest.raises(lsh.LSHError) as e:  # ... tensors without common eigenvectors are not
        lsh.workspace_size((8, 8), np.array([[[2.0, 0.5], [0.5, 1.0]], [[2.0, 0.0], [0.0, 1.0]]]))
    assert e.value.status == lsh.ERR_UNSUPPORTED
    with pytest.raises(lsh.LSHError) as e:  # reference not positive definite
        lsh.workspace_size((8, 8), np.array([np.eye(2)]), ref=-np.eye(2))
    assert e.value.status == lsh.ERR_REFERENCE_INDEFINITE
    with pytest.raises(lsh.LSHError) as e:  # A - A0 singular but nonzero
        lsh.workspace_size((8, 8), np.array([np.diag([1.0, 2.0])]), ref=np.eye(2))
    assert e.value.status == lsh.ERR_SINGULAR_CONTRAST
    with pytest.raises(lsh.LSHError) as e:  # scale field requires an explicit reference
        lsh.workspace_size((8, 8, 8), EL, physics=lsh.ELASTIC, has_scale=True)
    assert e.value.status == lsh.ERR_INVALID_ARG


def test_product_sources_do_not_use_the_oracle():
    """Nothing in the product package includes, imports or links oracle/."""
    pkg = os.path.join(ROOT, "paper_1411_0330_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "lsh_oracle" not in txt, f


def header_constants():
    """name -> value of every enumerator in include/lsh.h."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lsh.h")).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(LSH_[A-Z0-9_]+)\s*=\s*(\d+)", src)}


def test_binding_constants_match_the_header():
    """Every constant of the binding has the value of the header's enumerator of the same name
    (LSH_ prefix; the physics and Green-operator families drop their middle word)."""
    h = header_constants()
    alias = {"ELASTIC": "LSH_ELASTIC_ISO", "TRUNCATED": "LSH_GREEN_TRUNCATED", "FILTERED": "LSH_GREEN_FILTERED",
             "FD": "LSH_GREEN_FD"}
    names = ["OK", "ERR_INVALID_ARG", "ERR_UNSUPPORTED_SIZE", "ERR_REFERENCE_INDEFINITE", "ERR_SINGULAR_CONTRAST",
             "ERR_BREAKDOWN", "ERR_NOT_CONVERGED", "ERR_WORKSPACE", "ERR_CUDA", "ERR_UNSUPPORTED", "SCALAR",
             "ELASTIC", "TRUNCATED", "FILTERED", "FD", "FP64", "MIXED", "F64", "F32", "F64_DF", "SOLVER_AUTO",
             "SOLVER_CG", "SOLVER_MINRES", "SOLVER_BASIC", "SOLVER_SYMMLQ"]
    for n in names:
        assert getattr(lsh, n) == h[alias.get(n, "LSH_" + n)], n


def header_struct_fields(name):
    """(field name, array length, kind) of `typedef struct <name> { ... }` in include/lsh.h,
    in order; kind is int, float, double, longlong or ptr."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lsh.h")).read(), flags=re.S)
    body = re.search(r"typedef struct " + name + r"\s*\{(.*?)\}", src, flags=re.S).group(1)
    types = {"const", "unsigned", "signed", "char", "short", "int", "long", "float", "double", "size_t"}
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        words = decl.replace("*", " * ").replace(",", " , ").split()
        base = [w for w in words if w in types]
        kind = "longlong" if base.count("long") == 2 else next((k for k in ("double", "float") if k in base), "int")
        for item in " ".join(w for w in words if w not in types).split(","):
            m = re.match(r"\s*(\*?)\s*(\w+)\s*(?:\[(\d+)\])?", item)
            out.append((m.group(2), int(m.group(3)) if m.group(3) else 1, "ptr" if m.group(1) else kind))
    return out


def _ctypes_kind(t):
    t = getattr(t, "_type_", t) if hasattr(t, "_length_") else t
    if t is ctypes.c_void_p or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_float: "float", ctypes.c_double: "double",
            ctypes.c_longlong: "longlong"}[t]


@pytest.mark.parametrize("cname,pyname", [("lsh_problem", "_Problem"), ("lsh_solve_opts", "_Opts"),
                                          ("lsh_solve_info", "_Info"), ("lsh_tune_report", "_TuneReport"),
                                          ("lsh_profile", "_Profile")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes mirrors of the ABI structs have the header's fields, in order, with the
    same array lengths and element kinds (a drift would shift every later field)."""
    py = [(n, getattr(t, "_length_", 1), _ctypes_kind(t)) for n, t in getattr(lsh, pyname)._fields_]
    assert py == header_struct_fields(cname)
