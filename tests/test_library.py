"""Host-side checks of the C ABI library (no GPU needed): it builds for sm_103a, loads, and
exports every function that include/arrabit.h declares."""
import ctypes

import numpy as np
import pytest

from paper_1507_06078_gb300 import arrabit as arb
from paper_1507_06078_gb300 import build as B
from paper_1507_06078_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    B.build()
    return arb.load()


def test_every_declared_symbol_is_exported(lib):
    names = arb.header_functions()
    assert "arb_solve" in names and "arb_filter" in names and len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a prototype for each of them
    assert set(names) <= set(arb._PROTOS)


def test_status_strings_and_defaults(lib):
    assert lib.arb_status_string(0) == b"ok"
    assert lib.arb_status_string(-4) == b"iterate lost numerical rank"
    o = arb.arb_options_default(20)
    assert (o.p, o.q, o.degree, o.maxit, o.maxit1, o.maxit2) == (22, 1, 3, 30, 10, 5)
    assert np.isnan(o.shift_sigma)
    assert ctypes.sizeof(arb.arb_options) == 4 * 10 + 8 * 4
    assert ctypes.sizeof(arb.arb_info) == 8 * 8 + 8 + 4 * 6


@pytest.mark.parametrize("d", [1, 3, 10, 15, 20])
def test_host_filter_coefficients_match_oracle(lib, d):
    # the library's host-side coefficients (cosine-sum formula) against the oracle's
    # collocation solve: two independent derivations of the Section 5 interpolant
    from oracle import arrabit_oracle as O
    c = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, d)
    np.testing.assert_allclose(c, O.interpolant_cheb_coeffs(d), atol=2e-15)
    e = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBYSHEV, d)
    np.testing.assert_array_equal(e, O.chebyshev_T_coeffs(d))


def test_bad_coefficient_requests_rejected(lib):
    buf = np.zeros(70)
    assert lib.arb_filter_coefficients(0, 0, buf.ctypes.data) == arb.ARB_INVALID_ARG
    assert lib.arb_filter_coefficients(0, 61, buf.ctypes.data) == arb.ARB_INVALID_ARG
    assert lib.arb_filter_coefficients(7, 3, buf.ctypes.data) == arb.ARB_INVALID_ARG


def test_server_footprint_formula(lib):
    # 7 FP64 n x p blocks + 2 FP64 n x (q+1)p blocks + small state; mixed adds FP32 copies
    f = arb.arb_server_footprint(1000, 5000, 30, 1, arb.ARB_FP64)
    base = 1000 * (7 * 30 + 2 * 60) * 8
    assert base < f < base + (80 << 20)
    fm = arb.arb_server_footprint(1000, 5000, 30, 1, arb.ARB_MIXED)
    assert fm > f
    fdf = arb.arb_server_footprint(1000, 5000, 30, 1, arb.ARB_MIXED_DF)
    assert fdf == fm + 5000 * 8  # plus the double-float copy of A's values
    assert arb.arb_server_footprint(1000, 5000, 30, 1, 7) == -1
    assert arb.arb_server_footprint(0, 0, 30, 1, 0) == -1


def test_symmetry_check_host_only(lib):
    # host-side check of CSR arrays (no device involved): stencil Laplacians and a
    # symmetric random matrix pass, a one-sided perturbation or entry fails, malformed
    # arrays are rejected
    import scipy.sparse as sp
    A = I.laplacian_3d(6)
    assert arb.arb_csr_check_symmetric(A.n, A.rowptr, A.col, A.val) == arb.ARB_OK
    rng = np.random.default_rng(1)
    M = sp.random(300, 300, density=0.05, random_state=rng, format="csr")
    M = (M + M.T).tocsr()
    assert arb.arb_csr_check_symmetric(300, M.indptr, M.indices, M.data) == arb.ARB_OK
    v = M.data.copy()
    v[5] += 1e-6
    assert arb.arb_csr_check_symmetric(300, M.indptr, M.indices, v) == arb.ARB_NOT_SYMMETRIC
    assert arb.arb_csr_check_symmetric(300, M.indptr, M.indices, v, 1e-5) == arb.ARB_OK
    U = sp.triu(M, k=1).tocsr()  # strictly upper part only
    if U.nnz:
        assert arb.arb_csr_check_symmetric(300, U.indptr, U.indices, U.data) == arb.ARB_NOT_SYMMETRIC
    bad = A.rowptr.copy()
    bad[-1] += 1
    assert arb.arb_csr_check_symmetric(A.n, bad, A.col, A.val) == arb.ARB_INVALID_ARG
