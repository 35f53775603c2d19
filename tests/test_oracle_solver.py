"""The full oracle solver (Algorithm 8, MPM) pinned to closed-form spectra, dense
brute force and the invariants the method guarantees."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import arrabit_oracle as O
from paper_1507_06078_gb300 import inputs as I

from conftest import laplacian_2d_eigs, laplacian_3d_eigs


def _scipy(A):
    return O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)


def _check_invariants(A, r, tol, normA):
    n, k = r.evecs.shape
    Q = r.evecs
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-12)
    R = A @ Q - Q * r.evals[None, :]
    assert np.linalg.norm(R, axis=0).max() <= tol * normA
    # sign convention: largest-magnitude entry positive
    idx = np.argmax(np.abs(Q), axis=0)
    assert np.all(Q[idx, np.arange(k)] > 0)


def test_oracle_2d64_closed_form():
    W = I.workload_2d64()
    A = _scipy(W.A)
    X0 = I.gaussian_block(W.A.n, W.p, W.seed)
    r = O.arrabit_mpm(A, W.k, X0, which="smallest", tol=W.tol, q=W.q, degree=W.degree)
    assert r.converged
    lam = laplacian_2d_eigs(64)[:W.k]
    assert np.max(np.abs(r.evals - lam) / np.maximum(1.0, np.abs(lam))) <= 1e-10
    assert r.maxres <= W.tol
    _check_invariants(A, r, W.tol, 8.0)
    # partial trace check of Section 5 ("monitor the computed partial trace")
    assert abs(r.evals.sum() - lam.sum()) <= 1e-9


@pytest.mark.parametrize("m,k,p", [(8, 4, 6), (16, 10, 12), (32, 12, 16)])
def test_oracle_2d_small_grids(m, k, p):
    A = I.laplacian_2d(m)
    X0 = I.gaussian_block(A.n, p, 100 + m)
    r = O.arrabit_mpm(_scipy(A), k, X0, which="smallest", tol=1e-10, q=1, degree=8)
    lam = laplacian_2d_eigs(m)[:k]
    assert r.converged
    np.testing.assert_allclose(r.evals, lam, atol=1e-10)


@pytest.mark.parametrize("m,k,p,q", [(8, 6, 8, 1), (12, 10, 14, 2)])
def test_oracle_3d_small_grids(m, k, p, q):
    A = I.laplacian_3d(m)
    X0 = I.gaussian_block(A.n, p, 200 + m)
    r = O.arrabit_mpm(_scipy(A), k, X0, which="smallest", tol=1e-9, q=q, degree=12)
    lam = laplacian_3d_eigs(m)[:k]
    assert r.converged
    np.testing.assert_allclose(r.evals, lam, atol=1e-9)
    _check_invariants(_scipy(A), r, 1e-9, 12.0)


def _random_sparse_spd(n, density, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr")
    M = M + M.T
    return (M + sp.diags(rng.uniform(0, 3, n))).tocsr()


@pytest.mark.parametrize("which", ["largest", "smallest"])
def test_oracle_bruteforce_random_sparse(which):
    n, k, p = 400, 8, 12
    A = _random_sparse_spd(n, 0.02, 77)
    wref = np.linalg.eigvalsh(A.toarray())
    X0 = I.gaussian_block(n, p, 31)
    r = O.arrabit_mpm(A, k, X0, which=which, tol=1e-10, q=1, degree=10)
    assert r.converged
    want = wref[:k] if which == "smallest" else wref[::-1][:k]
    np.testing.assert_allclose(r.evals, want, atol=1e-9 * max(1, np.abs(wref).max()))


def test_oracle_plain_chebyshev_filter_variant():
    A = I.laplacian_2d(16)
    X0 = I.gaussian_block(A.n, 12, 5)
    r = O.arrabit_mpm(_scipy(A), 10, X0, which="smallest", tol=1e-9, q=1, degree=6,
                      filter_kind="chebyshev")
    assert r.converged
    np.testing.assert_allclose(r.evals, laplacian_2d_eigs(16)[:10], atol=1e-9)


def test_oracle_horner_path_matches():
    A = I.laplacian_2d(16)
    X0 = I.gaussian_block(A.n, 12, 6)
    r = O.arrabit_mpm(_scipy(A), 10, X0, which="smallest", tol=1e-10, q=1, degree=6,
                      poly_eval="horner")
    assert r.converged
    np.testing.assert_allclose(r.evals, laplacian_2d_eigs(16)[:10], atol=1e-10)


def test_oracle_locking_path():
    # a tolerance tight enough that continuation runs and pairs get locked
    A = I.laplacian_2d(20)
    X0 = I.gaussian_block(A.n, 14, 8)
    r = O.arrabit_mpm(_scipy(A), 12, X0, which="smallest", tol=1e-12, q=1, degree=8)
    assert r.converged
    np.testing.assert_allclose(r.evals, laplacian_2d_eigs(20)[:12], atol=1e-11)
    assert any(h.n_locked > 0 for h in r.history) or r.outer_iters <= 3


def test_augmentation_helps():
    # Section 6.2: ARR (q >= 1) needs no more outer iterations than plain RR (q = 0)
    A = I.laplacian_2d(24)
    X0 = I.gaussian_block(A.n, 16, 9)
    r0 = O.arrabit_mpm(_scipy(A), 12, X0, which="smallest", tol=1e-8, q=0, degree=6)
    r1 = O.arrabit_mpm(_scipy(A), 12, X0, which="smallest", tol=1e-8, q=1, degree=6)
    assert r1.converged
    assert r1.outer_iters <= r0.outer_iters


def test_inner_fixed_schedule():
    A = I.laplacian_2d(12)
    X0 = I.gaussian_block(A.n, 8, 10)
    r = O.arrabit_mpm(_scipy(A), 6, X0, which="smallest", tol=1e-9, q=1, degree=6,
                      inner_fixed=4, maxit=20)
    assert all(h.n_filters == 4 for h in r.history)
    assert r.converged


def test_golden_fixture_matches_closed_form_and_oracle():
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    g = json.load(open(os.path.join(here, "laplace2d_64_oracle.json")))
    lam = laplacian_2d_eigs(64)[:g["k"]]
    np.testing.assert_allclose(g["evals"], lam, atol=1e-10)
    c = json.load(open(os.path.join(here, "interpolant_coeffs.json")))["coeffs"]
    for d, a in c.items():
        np.testing.assert_allclose(a, O.interpolant_cheb_coeffs(int(d)), atol=1e-15)


def test_oracle_b_every_arr_reading():
    # Section 5's reading (b refreshed after every ARR) reaches the same pairs as
    # Algorithm 8's literal continuation-only update
    A = I.laplacian_3d(12)
    X0 = I.gaussian_block(A.n, 24, 12)
    r_lit = O.arrabit_mpm(_scipy(A), 20, X0, which="smallest", tol=1e-8, q=2, degree=10)
    r_arr = O.arrabit_mpm(_scipy(A), 20, X0, which="smallest", tol=1e-8, q=2, degree=10, b_update="every_arr")
    assert r_lit.converged and r_arr.converged
    lam = laplacian_3d_eigs(12)[:20]
    np.testing.assert_allclose(r_arr.evals, lam, atol=1e-9)
    np.testing.assert_allclose(r_lit.evals, lam, atol=1e-9)
    assert r_arr.history[-1].b > r_arr.history[0].b  # b moved towards lambda_{k+q} of B
