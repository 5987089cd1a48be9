"""The library's linear-programming inversion (paper Sec. II.B) against its
FP64 oracle (oracle/lp_inversion.py), on the host (no GPU needed).

The matrix and targets are compared element by element.  The linear program
can have several optimal x (a degenerate optimum), so the solutions are
compared by what is unique, the optimal objective c^T x (against HiGHS), and
by validity: x >= 0 and A x >= b on the oracle's own A and b.
"""
import ctypes as C
import math

import numpy as np
import pytest
from scipy.special import ive

from oracle import lp_inversion as lp
from paper_2507_15703_gb300 import cmb3d
from synth import cl_family

CASES = {
    # name: (ell, cl) family, R, theta_max, beam, dr, dk, kmax
    "family64_cap20": ("fam128", 1.0, math.radians(20.0), 0.0, 1 / 500, 0.0, math.sqrt(3) * math.pi * 64 / 2.2),
    "family64_beam_cap40": ("fam128", 1.0, math.radians(40.0), 0.01, 0.0, 0.0, math.sqrt(3) * math.pi * 64 / 2.2),
    "family768_cap20_R2": ("fam768", 2.0, math.radians(20.0), 0.0, 2 / 3000, 0.0, 800.0),
    "gauss_cap30": ("gauss", 1.0, math.radians(30.0), 0.0, 0.01, 0.0, 150.0),
    "family64_cap120_dk": ("fam128", 1.0, math.radians(120.0), 0.0, 0.01, 1.5, 90.0),
}


def spectrum(kind):
    if kind == "fam128":
        return cl_family(128, 1e3, 22.0, 100.0)
    if kind == "fam768":
        return cl_family(768, 1e3, 22.0, 600.0)
    A0, S = 3.0, 0.05
    ell = np.arange(0, 401)
    return ell, 16 * np.pi ** 2 * A0 * np.pi / (4 * S * S) * ive(ell + 0.5, 1 / (2 * S * S))


@pytest.fixture(scope="module")
def lib():
    import os
    if not os.path.exists(cmb3d.LIB_PATH):
        from paper_2507_15703_gb300.build import build
        build()
    return cmb3d.load()


def args_of(name):
    kind, R, th, beam, dr, dk, kmax = CASES[name]
    ell, cl = spectrum(kind)
    return ell, cl, R, th, beam, dr, dk, kmax


@pytest.mark.parametrize("name", sorted(CASES))
def test_system_matches_oracle(lib, name):
    ell, cl, R, th, beam, dr, dk, kmax = args_of(name)
    r, kn, A, b = cmb3d.cmb3d_lp_system(ell, cl, R, th, beam, dr, dk, kmax)
    r_o, th_o, kn_o = lp.lp_grid(R, th, beam, dr, dk, kmax)
    assert r.shape == r_o.shape and kn.shape == kn_o.shape
    np.testing.assert_array_equal(r, r_o)
    np.testing.assert_array_equal(kn, kn_o)
    A_o = lp.lp_matrix(r_o, kn_o)
    b_o = lp.lp_targets(th_o, ell, cl, beam)
    assert np.max(np.abs(A - A_o)) <= 1e-13 * np.max(np.abs(A_o))
    assert np.max(np.abs(b - b_o)) <= 1e-12 * abs(b_o[0])


@pytest.mark.parametrize("name", sorted(CASES))
def test_solution_is_optimal_and_feasible(lib, name):
    ell, cl, R, th, beam, dr, dk, kmax = args_of(name)
    kn, pk, obj, xi_err = cmb3d.cmb3d_fit_pk_lp(ell, cl, R, th, beam, dr, dk, kmax)
    kn_o, pk_o, info = lp.invert_xi_lp(ell, cl, R, th, beam, dr, dk, kmax)
    A, b = info["A"], info["b"]
    np.testing.assert_array_equal(kn, kn_o)
    assert pk[-1] == 0.0 and np.all(pk >= 0.0)
    x = pk[:-1]
    c = A.sum(axis=0)
    assert obj == pytest.approx(c @ x, rel=1e-12)
    assert obj == pytest.approx(info["objective"], rel=1e-9)                 # the unique optimal value
    assert np.min(A @ x - b) >= -1e-9 * abs(b[0])                           # feasible on the oracle's A, b
    assert xi_err == pytest.approx(np.max(np.abs(A @ x - b)) / abs(b[0]), rel=1e-6, abs=1e-12)


def test_exact_solution_is_found_when_one_exists(lib):
    ell, cl, R, th, beam, dr, dk, kmax = args_of("gauss_cap30")
    kn, pk, obj, xi_err = cmb3d.cmb3d_fit_pk_lp(ell, cl, R, th, beam, dr, dk, kmax)
    r, _, A, b = cmb3d.cmb3d_lp_system(ell, cl, R, th, beam, dr, dk, kmax)
    assert obj == pytest.approx(b.sum(), rel=1e-9)
    assert xi_err <= 1e-8


def test_workload_sized_program_matches_highs(lib):
    """The 20-degree cap with the 512^2 x 22-layer box's largest |k| and
    dr = 1/3000 (2053 separations x 522 nodes)."""
    ell, cl = cl_family(768, 1e3, 22.0, 600.0)
    a = (ell, cl, 1.0, math.radians(20.0), 0.0, 1 / 3000, 0.0, math.sqrt(3) * math.pi / 0.0034)
    kn, pk, obj, _ = cmb3d.cmb3d_fit_pk_lp(*a)
    _, _, info = lp.invert_xi_lp(*a)
    assert info["A"].shape == (2053, 522)
    assert obj == pytest.approx(info["objective"], rel=1e-9)
    assert np.min(info["A"] @ pk[:-1] - info["b"]) >= -1e-9 * abs(info["b"][0])


@pytest.mark.parametrize("kw,status", [
    (dict(theta_max=0.0), "CMB3D_EINVAL"), (dict(theta_max=4.0), "CMB3D_EINVAL"),
    (dict(dr=0.0, beam=0.0), "CMB3D_EINVAL"), (dict(kmax=1.0), "CMB3D_EINVAL"),
    (dict(R=-1.0), "CMB3D_EINVAL"), (dict(beam=float("nan")), "CMB3D_EINVAL"),
    (dict(dr=1e-7), "CMB3D_EUNSUPPORTED"), (dict(dk=1e-4, kmax=100.0), "CMB3D_EUNSUPPORTED"),
    (dict(dr=1e-4, kmax=20000.0), "CMB3D_EUNSUPPORTED"),                 # tableau above 6.4e7
])
def test_bad_arguments(lib, kw, status):
    ell, cl = cl_family(128, 1e3, 22.0, 100.0)
    a = dict(R=1.0, theta_max=0.3, beam=0.0, dr=0.01, dk=0.0, kmax=100.0)
    a.update(kw)
    with pytest.raises(cmb3d.Cmb3dError) as e:
        cmb3d.cmb3d_lp_system(ell, cl, a["R"], a["theta_max"], a["beam"], a["dr"], a["dk"], a["kmax"])
    assert e.value.status == getattr(cmb3d, status)


def test_bad_spectra_and_capacity(lib):
    ell, cl = cl_family(128, 1e3, 22.0, 100.0)
    for e2, c2 in [(ell[::-1].copy(), cl), (ell, -cl), (ell + 0.5, cl)]:
        with pytest.raises(cmb3d.Cmb3dError) as e:
            cmb3d.cmb3d_fit_pk_lp(e2, c2, 1.0, 0.3, 0.0, 0.01, 0.0, 100.0)
        assert e.value.status == cmb3d.CMB3D_EINVAL
    ea, ca = np.ascontiguousarray(ell, np.float64), np.ascontiguousarray(cl, np.float64)
    kn, pk = np.empty(4), np.empty(4)
    nk, obj, err = C.c_int(0), C.c_double(0), C.c_double(0)
    dp = C.POINTER(C.c_double)
    st = lib.cmb3d_fit_pk_lp(ea.ctypes.data_as(dp), ca.ctypes.data_as(dp), ea.size, 1.0, 0.3, 0.0, 0.01, 0.0,
                             100.0, 4, kn.ctypes.data_as(dp), pk.ctypes.data_as(dp), C.byref(nk), C.byref(obj),
                             C.byref(err))
    assert st == cmb3d.CMB3D_EINVAL                                          # 4 < nk + 1


def test_degenerate_programs_have_their_closed_forms(lib):
    """One unknown (kmax = dk): the least x with A_i0 x >= b_i, i.e.
    max_i b_i / A_i0.  One separation (r_max < dr, only r = 0): the objective
    sum_i (A x)_i is (A x)_0 >= b_0, so its minimum is b_0 exactly."""
    ell, cl = cl_family(128, 1e3, 22.0, 100.0)
    _, _, A, b = cmb3d.cmb3d_lp_system(ell, cl, 1.0, 0.3, 0.0, 0.01, 2.0, 2.0)
    assert A.shape == (60, 1) and np.all(A[:, 0] > 0)
    kn, pk, obj, _ = cmb3d.cmb3d_fit_pk_lp(ell, cl, 1.0, 0.3, 0.0, 0.01, 2.0, 2.0)
    assert len(pk) == 2 and pk[1] == 0.0
    assert pk[0] == pytest.approx(np.max(b / A[:, 0]), rel=1e-12)
    _, _, A1, b1 = cmb3d.cmb3d_lp_system(ell, cl, 1.0, 0.3, 0.0, 1.0, 0.0, 50.0)
    assert A1.shape[0] == 1
    _, pk1, obj1, err1 = cmb3d.cmb3d_fit_pk_lp(ell, cl, 1.0, 0.3, 0.0, 1.0, 0.0, 50.0)
    assert obj1 == pytest.approx(b1[0], rel=1e-12) and err1 <= 1e-12
    assert A1[0] @ pk1[:-1] == pytest.approx(b1[0], rel=1e-12)
