"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without a GPU,
and exports every entry point include/vecchia.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vecchia.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vecchia_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2403_07412_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vecchia_plan_create", "vecchia_loglik", "vecchia_loglik_grad", "vecchia_plan_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2403_07412_gb300 import vecchia

    assert set(declared_functions()) <= set(vecchia.SIGNATURES)


def test_strerror_and_argument_checks_without_gpu(libpath):
    from paper_2403_07412_gb300 import vecchia

    L = vecchia.lib()
    assert L.vecchia_strerror(0) == b"success"
    assert L.vecchia_strerror(2).startswith(b"conditional")
    # argument validation happens before any CUDA call
    out = ctypes.c_void_p()
    assert L.vecchia_plan_create(None, 10, 5, 1, 0, None, None, ctypes.byref(out)) == vecchia.EINVAL
    xy = (ctypes.c_double * 4)(0.1, 0.2, 0.3, 0.4)
    assert L.vecchia_plan_create(xy, 2, 0, 1, 0, None, None, ctypes.byref(out)) == vecchia.EINVAL
    assert L.vecchia_plan_create(xy, 2, 151, 1, 0, None, None, ctypes.byref(out)) == vecchia.EINVAL
    assert L.vecchia_plan_create(xy, 2, 5, 7, 0, None, None, ctypes.byref(out)) == vecchia.EINVAL
    bad = (ctypes.c_double * 4)(0.1, float("nan"), 0.3, 0.4)
    assert L.vecchia_plan_create(bad, 2, 1, 1, 0, None, None, ctypes.byref(out)) == vecchia.EINVAL
    th = (ctypes.c_double * 4)(1.0, -0.1, 0.5, 0.0)
    assert L.vecchia_matern(None, 1, th, None, None, None) == vecchia.EINVAL
    assert L.vecchia_loglik(None, None, th, None, None) == vecchia.EINVAL
    L.vecchia_pivot_reciprocal.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    assert L.vecchia_pivot_reciprocal(None, -1, None, None) == vecchia.EINVAL
    assert L.vecchia_pivot_reciprocal(None, 3, None, None) == vecchia.EINVAL
    assert L.vecchia_pivot_reciprocal(None, 0, None, None) == vecchia.OK


def test_sphere_plan_argument_checks_without_gpu(libpath):
    from paper_2403_07412_gb300 import vecchia

    L = vecchia.lib()
    out = ctypes.c_void_p()
    ll = (ctypes.c_double * 4)(-90.0, 35.0, -89.0, 36.0)
    bad_lat = (ctypes.c_double * 4)(-90.0, 95.0, -89.0, 36.0)
    # planar orderings, latitude beyond the pole, non-positive radius: rejected before any CUDA call
    assert L.vecchia_plan_create_sphere(ll, 2, 1, vecchia.ORDER_MAXMIN, 0, None, 6371.0, None,
                                        ctypes.byref(out)) == vecchia.EINVAL
    assert L.vecchia_plan_create_sphere(ll, 2, 1, vecchia.ORDER_MORTON, 0, None, 6371.0, None,
                                        ctypes.byref(out)) == vecchia.EINVAL
    assert L.vecchia_plan_create_sphere(bad_lat, 2, 1, vecchia.ORDER_RANDOM, 0, None, 6371.0, None,
                                        ctypes.byref(out)) == vecchia.EINVAL
    assert L.vecchia_plan_create_sphere(ll, 2, 1, vecchia.ORDER_RANDOM, 0, None, 0.0, None,
                                        ctypes.byref(out)) == vecchia.EINVAL
    assert L.vecchia_plan_create_sphere(ll, 2, 1, vecchia.ORDER_RANDOM, 0, None, float("inf"), None,
                                        ctypes.byref(out)) == vecchia.EINVAL


def test_predict_argument_checks_without_gpu(libpath):
    from paper_2403_07412_gb300 import vecchia

    L = vecchia.lib()
    xy = (ctypes.c_double * 2)(0.5, 0.5)
    th = (ctypes.c_double * 4)(1.0, 0.1, 0.5, 0.0)
    assert L.vecchia_predict(None, xy, 1, None, th, None, None, None, None) == vecchia.EINVAL

