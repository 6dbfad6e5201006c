"""CPU checks of the C-ABI library: it builds, loads, and exports every function that
include/helm.h declares (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1012_5379_gb300 import build
    path = build.build()
    try:
        return ctypes.CDLL(path)
    except OSError as e:  # pragma: no cover - needs libcudart on the loader path
        pytest.skip(f"libhelm.so does not load here: {e}")


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("helm_setup", "helm_precond_apply", "helm_solve", "helm_destroy", "helm_batch_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1012_5379_gb300 import helm
    assert sorted(helm.EXPORTS) == declared_functions()


def test_last_error_is_callable_without_gpu(lib):
    lib.helm_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.helm_last_error(), bytes)   # "" unless an earlier call failed


def test_setup_rejects_bad_grid_without_touching_the_device(lib):
    class Grid(ctypes.Structure):
        _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("ecs_frac", ctypes.c_double),
                    ("theta_gamma", ctypes.c_double), ("ecs_sides", ctypes.c_int)]
    lib.helm_setup.restype = ctypes.c_int
    lib.helm_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    g = Grid(5, 15, 0.125, 0.5)
    rc = lib.helm_setup(ctypes.byref(g), None, ctypes.c_double(1.0), ctypes.c_double(0.3), None, None,
                        ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert b"dim" in lib.helm_last_error()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1012_5379_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_setup_rejects_a_basis_longer_than_the_limit(lib):
    """min(restart, maxit) above HELM_MAX_BASIS is refused before any device work."""
    class Grid(ctypes.Structure):
        _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("ecs_frac", ctypes.c_double),
                    ("theta_gamma", ctypes.c_double), ("ecs_sides", ctypes.c_int)]

    class Opts(ctypes.Structure):
        _fields_ = [(f, ctypes.c_int) for f in ("nu1", "nu2", "s", "coarsest_n", "precond_prec", "restart", "maxit")] + \
                   [("csl_eps", ctypes.c_double), ("smoother", ctypes.c_int)]
    hdr = open(os.path.join(ROOT, "include", "helm.h")).read()
    limit = int(re.search(r"#define HELM_MAX_BASIS (\d+)", hdr).group(1))
    lib.helm_setup.restype = ctypes.c_int
    lib.helm_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    g = Grid(2, 15, 0.125, 0.5)
    o = Opts(0, 0, 0, 0, 0, 0, limit + 1, 0.0, 0)
    rc = lib.helm_setup(ctypes.byref(g), None, ctypes.c_double(1.0), ctypes.c_double(0.3), ctypes.byref(o), None,
                        ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert b"HELM_MAX_BASIS" in lib.helm_last_error()


def test_setup_rejects_a_negative_complex_shift(lib):
    """csl_eps (the complex shifted Laplacian variant's shift) must be finite and >= 0."""
    class Grid(ctypes.Structure):
        _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("ecs_frac", ctypes.c_double),
                    ("theta_gamma", ctypes.c_double), ("ecs_sides", ctypes.c_int)]

    class Opts(ctypes.Structure):
        _fields_ = [(f, ctypes.c_int) for f in ("nu1", "nu2", "s", "coarsest_n", "precond_prec", "restart", "maxit")] + \
                   [("csl_eps", ctypes.c_double), ("smoother", ctypes.c_int)]
    lib.helm_setup.restype = ctypes.c_int
    lib.helm_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    g = Grid(2, 15, 0.125, 0.5)
    o = Opts(0, 0, 0, 0, 0, 0, 0, -0.5, 0)
    rc = lib.helm_setup(ctypes.byref(g), None, ctypes.c_double(1.0), ctypes.c_double(0.0), ctypes.byref(o), None,
                        ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert b"csl_eps" in lib.helm_last_error()


def test_setup_rejects_the_polynomial_smoother_with_a_shift(lib):
    """The polynomial smoother (Sec. 4) is built for the CSG preconditioner alone."""
    class Grid(ctypes.Structure):
        _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("ecs_frac", ctypes.c_double),
                    ("theta_gamma", ctypes.c_double), ("ecs_sides", ctypes.c_int)]

    class Opts(ctypes.Structure):
        _fields_ = [(f, ctypes.c_int) for f in ("nu1", "nu2", "s", "coarsest_n", "precond_prec", "restart", "maxit")] + \
                   [("csl_eps", ctypes.c_double), ("smoother", ctypes.c_int)]
    lib.helm_setup.restype = ctypes.c_int
    lib.helm_last_error.restype = ctypes.c_char_p
    hdr = open(os.path.join(ROOT, "include", "helm.h")).read()
    poly = int(re.search(r"#define HELM_SMOOTHER_POLY (\d+)", hdr).group(1))
    out = ctypes.c_void_p()
    g = Grid(2, 15, 0.125, 0.5)
    o = Opts(0, 0, 0, 0, 0, 0, 0, 0.5, poly)
    rc = lib.helm_setup(ctypes.byref(g), None, ctypes.c_double(5.0), ctypes.c_double(0.2), ctypes.byref(o), None,
                        ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert b"polynomial smoother" in lib.helm_last_error()


def test_setup_rejects_an_unknown_layer_placement(lib):
    class Grid(ctypes.Structure):
        _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("ecs_frac", ctypes.c_double),
                    ("theta_gamma", ctypes.c_double), ("ecs_sides", ctypes.c_int)]
    lib.helm_setup.restype = ctypes.c_int
    lib.helm_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    for sides, frac, word in ((2, 0.125, b"ecs_sides"), (0, 0.6, b"ecs_frac"), (1, 1.0, b"ecs_frac")):
        g = Grid(2, 15, frac, 0.5, sides)
        rc = lib.helm_setup(ctypes.byref(g), None, ctypes.c_double(1.0), ctypes.c_double(0.3), None, None,
                            ctypes.byref(out))
        assert rc == -1 and out.value is None
        assert word in lib.helm_last_error()


def test_binding_declares_every_double_parameter_as_double():
    """The ctypes binding passes a C `double` parameter as c_double (a pointer or an int
    there makes every call fail), for every prototype of the header."""
    from paper_1012_5379_gb300 import helm as H
    lib = H.load()
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    checked = 0
    for m in re.finditer(r"\b(?:int|void|unsigned long long|const char\*)\s+(helm_\w+)\s*\(([^;{]*?)\)\s*;", src):
        name, params = m.group(1), m.group(2).strip()
        fn = getattr(lib, name)
        if not params or params == "void" or fn.argtypes is None:
            continue
        for i, p in enumerate(x.strip() for x in params.split(",")):
            if re.match(r"^double\s+\w+$", p):
                assert fn.argtypes[i] is ctypes.c_double, (name, i, p)
                checked += 1
    assert checked >= 8
