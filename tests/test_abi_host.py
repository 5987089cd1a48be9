"""Host-side checks of the C-ABI library (no GPU needed).

* libcmb3d.so loads and exports every function include/cmb3d.h declares, and
  the Python binding declares a prototype for each;
* argument validation answers before any CUDA call;
* the host-only C_l -> P(k) inversion agrees with the oracle's forward
  projection (same design matrix) and fits the small spectrum;
* the product package and the oracle do not import each other.
"""
import ast
import os
import re

import numpy as np
import pytest

from paper_2507_15703_gb300 import cmb3d
from oracle import cmb3d_oracle as orc
from synth import cl_family

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cmb3d.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(cmb3d.LIB_PATH):
        from paper_2507_15703_gb300.build import build
        build()
    return cmb3d.load()


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cmb3d_\w+)\s*\(", text)))


def test_header_symbols_exported(lib):
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
        assert name in cmb3d.PROTOTYPES, name
    assert set(cmb3d.PROTOTYPES) == set(names)


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert cmb3d.cmb3d_strerror(code).startswith("CMB3D_")
    assert "unknown" in cmb3d.cmb3d_strerror(12345)


@pytest.mark.parametrize("N", [4, 12, 4096, 0, -8])
def test_plan_rejects_unsupported_sizes(lib, N):
    with pytest.raises(cmb3d.Cmb3dError) as e:
        cmb3d.cmb3d_plan(N, 2.2, 1.0, np.zeros((1, 3)))
    assert e.value.status == cmb3d.CMB3D_EUNSUPPORTED


@pytest.mark.parametrize("kw", [dict(L=1.5), dict(L=-1.0), dict(r=0.0), dict(interp=2), dict(flags=1 << 10),
                                dict(L=float("nan"))])
def test_plan_rejects_bad_arguments(lib, kw):
    args = dict(N=64, L=2.2, r=1.0, interp=1, flags=0)
    args.update(kw)
    with pytest.raises(cmb3d.Cmb3dError) as e:
        cmb3d.cmb3d_plan(args["N"], args["L"], args["r"], np.zeros((1, 3)), args["interp"], args["flags"])
    assert e.value.status == cmb3d.CMB3D_EINVAL


def test_plan_rejects_nonfinite_pixels(lib):
    with pytest.raises(cmb3d.Cmb3dError) as e:
        cmb3d.cmb3d_plan(64, 2.2, 1.0, np.array([[0.0, np.inf, 1.0]]))
    assert e.value.status == cmb3d.CMB3D_EINVAL


def test_fit_pk_rejects_bad_spectra(lib):
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.cmb3d_fit_pk([2, 3, 3], [1.0, 1.0, 1.0], 64, 2.2, 1.0, 64)
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.cmb3d_fit_pk([2, 3], [1.0, -1.0], 64, 2.2, 1.0, 64)
    with pytest.raises(cmb3d.Cmb3dError):
        cmb3d.cmb3d_fit_pk([2, 3], [1.0, 1.0], 64, 2.2, 1.0, 4)


def test_fit_pk_small_family_matches_oracle_projection(lib):
    ell, cl = cl_family(128, 1e3, 22.0, 100.0)
    kn, pk, err = cmb3d.cmb3d_fit_pk(ell, cl, 64, 2.2, 1.0, 256)
    np.testing.assert_allclose(kn, orc.knodes_for_box(64, 2.2, 256), rtol=1e-14)
    assert np.all(pk >= 0)
    fwd = orc.cl_matrix(ell, kn, 1.0) @ pk          # the oracle's own design matrix
    oracle_err = np.max(np.abs(fwd - cl) / cl)
    assert err < 1e-3
    assert abs(oracle_err - err) <= 1e-6 + 1e-6 * err


def test_fit_pk_closed_form_gaussian(lib):
    """C_l of P(k) = A exp(-s^2 k^2) (closed form via I_{l+1/2}) are refitted to
    a forward-projected error below 1e-3."""
    from scipy.special import ive
    A, S, R = 3.0, 0.05, 1.0
    ell = np.arange(2, 41, dtype=np.float64)
    cl = 16 * np.pi ** 2 * A * np.pi / (4 * R * S * S) * ive(ell + 0.5, R * R / (2 * S * S))
    kn, pk, err = cmb3d.cmb3d_fit_pk(ell, cl, 64, 2.2, R, 128)
    assert err < 1e-3
    fwd = orc.cl_matrix(ell, kn, R) @ pk
    np.testing.assert_allclose(fwd, cl, rtol=2e-3)


def _imports(path):
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            mods.add(node.module.split(".")[0])
    return mods


def test_product_and_oracle_are_independent():
    pkg = os.path.join(ROOT, "paper_2507_15703_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                assert "oracle" not in _imports(os.path.join(dirpath, f)), f
            if f.endswith((".cu", ".cuh", ".cpp", ".h")):
                assert "oracle" not in open(os.path.join(dirpath, f)).read().lower().replace(
                    "oracle-independent", ""), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            assert "paper_2507_15703_gb300" not in _imports(os.path.join(ROOT, "oracle", f)), f


@pytest.mark.parametrize("N,M,h", [(16, 16, 6), (32, 8, 12), (16, 64, 1), (32, 32, 32)])
def test_gamma_sqrt_table_matches_oracle(lib, N, M, h):
    """The 2-D method's per-q square roots (FP64 Jacobi in the library, numpy
    eigh in the oracle) agree to FP32 rounding; unreached q stay zero."""
    from oracle import fourier2d as f2
    L = 2.2
    k = np.linspace(0.0, np.sqrt(3) * np.pi * N / L, 64)
    pk = 1e-3 / (1.0 + (k / 6.0) ** 3)
    tab = cmb3d.cmb3d_gamma_sqrt_table(N, M, h, L, k, pk)
    ref = f2.sqrt_gamma_table(N, M, h, L, k, pk)
    for q in range(tab.shape[0]):
        if q in ref:
            assert np.max(np.abs(tab[q] - ref[q])) <= 1e-6 * np.max(np.abs(ref[q])), q
        else:
            assert not tab[q].any()


@pytest.mark.parametrize("kw,status", [
    (dict(N=8), "CMB3D_EUNSUPPORTED"), (dict(h=33), "CMB3D_EUNSUPPORTED"), (dict(N=16, h=20), "CMB3D_EUNSUPPORTED"),
    (dict(M=0), "CMB3D_EINVAL"), (dict(z0=float("nan")), "CMB3D_EINVAL"), (dict(L=0.0), "CMB3D_EINVAL"),
    (dict(flags=1 << 4), "CMB3D_EUNSUPPORTED"), (dict(flags=1 << 6), "CMB3D_EUNSUPPORTED"),
    (dict(flags=1 << 10), "CMB3D_EINVAL")])
def test_plan_2d_rejects_bad_arguments(lib, kw, status):
    args = dict(N=64, M=32, h=8, L=2.2, r=1.0, z0=0.5, flags=0)
    args.update(kw)
    with pytest.raises(cmb3d.Cmb3dError) as e:
        cmb3d.cmb3d_plan_2d(args["N"], args["M"], args["h"], args["L"], args["r"], args["z0"], np.zeros((1, 3)), 3,
                            args["flags"])
    assert e.value.status == getattr(cmb3d, status)
