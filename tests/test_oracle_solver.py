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
    # Deflation (eq. defl, Algorithm 8): with the first continuation tolerance tol_1 = 1e-3
    # the lock threshold is tol_1^2 = 1e-6, so the leading pairs, which converge first, are
    # locked while the rest iterate; the later outer iterations then run with a non-empty
    # Q_c (projection of X and Z, merge of locked and new Ritz pairs)
    A = I.laplacian_2d(20)
    X0 = I.gaussian_block(A.n, 14, 8)
    B = _scipy(A)
    r = O.arrabit_mpm(B, 12, X0, which="smallest", tol=1e-10, q=1, degree=8, tol1=1e-3)
    assert r.converged
    assert any(h.n_locked > 0 for h in r.history)
    lam = laplacian_2d_eigs(20)[:12]
    np.testing.assert_allclose(r.evals, lam, atol=1e-12)
    # the merged set stays orthonormal to rounding level (a partial projection against the
    # locked block leaves ~1e-13 of it in the free block)
    assert np.abs(r.evecs.T @ r.evecs - np.eye(12)).max() <= 1e-13
    _check_invariants(B, r, 1e-10, 8.0)


def test_oracle_locking_grows_to_all_locked():
    # k = p and a tolerance below what FP64 residuals reach: the pairs lock as they pass the
    # floor of the threshold (1e-14), until the whole block is locked (the all-locked exit)
    A = I.laplacian_2d(20)
    X0 = I.gaussian_block(A.n, 10, 8)
    r = O.arrabit_mpm(_scipy(A), 10, X0, which="smallest", tol=1e-15, q=1, degree=8, tol1=1e-2)
    assert r.stop_reason == "all_locked"
    assert max(h.n_locked for h in r.history) > 0
    np.testing.assert_allclose(r.evals, laplacian_2d_eigs(20)[:10], atol=1e-13)
    np.testing.assert_allclose(r.evecs.T @ r.evecs, np.eye(10), atol=1e-13)


@pytest.mark.parametrize("slip", ["dropped", "sign", "half", "transposed"])
def test_planted_project_out_slip_is_caught(monkeypatch, slip):
    # each plausible mistake in X - Q_c (Q_c^T X) fails one of the locking-path pins above:
    # the solve raises, misses an eigenvalue, or loses orthogonality of the merged set
    def bad(Qc, X):
        if Qc is None or Qc.shape[1] == 0:
            return X
        if slip == "dropped":
            return X
        if slip == "sign":
            return X + Qc @ (Qc.T @ X)
        if slip == "half":
            return X - 0.5 * Qc @ (Qc.T @ X)
        return X - Qc[:, ::-1] @ (Qc.T @ X)

    monkeypatch.setattr(O, "project_out", bad)
    A = I.laplacian_2d(20)
    X0 = I.gaussian_block(A.n, 14, 8)
    lam = laplacian_2d_eigs(20)[:12]
    try:
        r = O.arrabit_mpm(_scipy(A), 12, X0, which="smallest", tol=1e-10, q=1, degree=8, tol1=1e-3)
    except RuntimeError:
        return
    err = np.max(np.abs(r.evals - lam))
    orth = np.abs(r.evecs.T @ r.evecs - np.eye(12)).max()
    assert err > 1e-10 or orth > 1e-13


def test_pad_ritz_invariants():
    # completing a short Ritz set: the first columns and values are kept, the new columns
    # are orthonormal and orthogonal to the kept ones, and their values are Rayleigh
    # quotients (so they lie inside the spectrum of B)
    A = _scipy(I.laplacian_2d(12))
    wref, Vref = np.linalg.eigh(A.toarray())
    Y, w = Vref[:, -3:][:, ::-1], wref[-3:][::-1]
    pool = I.gaussian_block(A.shape[0], 6, 41)
    Yp, wp = O.pad_ritz(A, Y, w, 7, pool)
    assert Yp.shape == (A.shape[0], 7) and wp.shape == (7,)
    np.testing.assert_array_equal(Yp[:, :3], Y)
    np.testing.assert_array_equal(wp[:3], w)
    np.testing.assert_allclose(Yp.T @ Yp, np.eye(7), atol=1e-13)
    assert np.all(wp[3:] >= wref[0] - 1e-12) and np.all(wp[3:] <= wref[-1] + 1e-12)
    # a full set is returned unchanged; a short one without a pool is an error
    Yf, wf = O.pad_ritz(A, Yp, wp, 7, None)
    assert Yf is Yp and wf is wp
    with pytest.raises(RuntimeError):
        O.pad_ritz(A, Y, w, 7, None)


def test_oracle_rank_deficient_start_block_is_padded():
    # duplicated start columns: X keeps rank 5 through the filter, the q = 1 subspace has
    # dimension 10 < p = 14, so the Ritz set is completed from the pool; the solve still
    # reaches the dense eigenvalues
    n, k, p = 400, 8, 14
    A = _random_sparse_spd(n, 0.02, 77)
    wref = np.linalg.eigvalsh(A.toarray())
    G = I.gaussian_block(n, 5, 32)
    X0 = np.hstack([G, G, G[:, :4]])
    pool = I.gaussian_block(n, p, 33)
    r = O.arrabit_mpm(A, k, X0, which="largest", tol=1e-10, q=1, degree=10, pad_pool=pool)
    assert r.history[0].rank == 10
    assert r.converged
    np.testing.assert_allclose(r.evals, wref[::-1][:k], atol=1e-9 * np.abs(wref).max())


def test_residual_denominators_use_the_original_eigenvalue():
    # eq. resi divides by max(1, |lambda_i|) with lambda_i an eigenvalue of A.  For the
    # smallest pairs of A = L + 200 I the method runs on sigma I - A, whose Ritz values
    # mu_i = sigma - lambda_i are near 8, far from lambda_i near 200: the reported
    # residuals must equal ||A x_i - lambda_i x_i|| / |lambda_i| recomputed from the pairs
    L = _scipy(I.laplacian_2d(16))
    A = (L + 200.0 * sp.identity(L.shape[0])).tocsr()
    X0 = I.gaussian_block(L.shape[0], 12, 13)
    r = O.arrabit_mpm(A, 10, X0, which="smallest", tol=1e-6, q=1, degree=4)
    assert r.converged
    direct = np.linalg.norm(A @ r.evecs - r.evecs * r.evals[None, :], axis=0) / np.abs(r.evals)
    big = r.res > 1e-11  # far above the ~1e-16 rounding of the recomputation
    assert big.sum() >= 5
    np.testing.assert_allclose(r.res[big], direct[big], rtol=0.01)
    np.testing.assert_allclose(r.evals, 200.0 + laplacian_2d_eigs(16)[:10], rtol=1e-9)


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


def test_planted_residual_denominator_slip_is_caught(monkeypatch):
    # dividing by max(1, |mu_i|) of the shifted operator instead of max(1, |lambda_i|)
    # makes the reported residuals ~25x too large on the shifted Laplacian above
    real = O.residual_norms
    monkeypatch.setattr(O, "residual_norms", lambda B, X, mu, lam: real(B, X, mu, mu))
    L = _scipy(I.laplacian_2d(16))
    A = (L + 200.0 * sp.identity(L.shape[0])).tocsr()
    X0 = I.gaussian_block(L.shape[0], 12, 13)
    r = O.arrabit_mpm(A, 10, X0, which="smallest", tol=1e-6, q=1, degree=4)
    direct = np.linalg.norm(A @ r.evecs - r.evecs * r.evals[None, :], axis=0) / np.abs(r.evals)
    big = r.res > 1e-11
    assert not np.allclose(r.res[big], direct[big], rtol=0.01)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_arr_exact_on_a_krylov_invariant_subspace(q):
    # Algorithm 5 on a diagonal B: a column supported on q + 1 coordinates spans, with its
    # first q powers, exactly those coordinate vectors, so ARR returns exactly the q + 1
    # diagonal entries there (descending) with the unit vectors as Ritz vectors
    n = 50
    dvals = np.linspace(-1.0, 3.0, n) ** 3
    B = sp.diags(dvals).tocsr()
    support = [3, 17, 41][: q + 1]
    X = np.zeros((n, 1))
    X[support, 0] = [1.0, -2.0, 0.5][: q + 1]
    Y, w = O.arr(B, X, q, npairs=q + 1)
    want = np.sort(dvals[support])[::-1]
    np.testing.assert_allclose(w, want, atol=1e-13)
    for j in range(q + 1):
        i = support[int(np.argmin(np.abs(dvals[support] - w[j])))]
        assert abs(abs(Y[i, j]) - 1.0) <= 1e-12


# ---------------------------------------------------------------- GN inner solver (Algorithm 4)
def _filter_of(B, coef, a, b):
    return lambda Y: O.poly_clenshaw(B - a * sp.identity(B.shape[0], format="csr"), Y, 0.0, b - a, coef)


def test_gn_step_fixed_points():
    # GN minimises ||X X^T - F||_F for F = rho(B): X* = V_S diag(sqrt(f_S)) Q (eigenvectors
    # of any subset S of positive eigenvalues f_S of F, any orthogonal Q) is a fixed point
    n = 40
    dvals = np.linspace(0.0, 3.0, n)
    B = sp.diags(dvals).tocsr()
    coef = O.interpolant_cheb_coeffs(6)
    F = _filter_of(B, coef, 0.0, 2.5)
    f = O.filter_value(coef, dvals, 0.0, 2.5)
    S = [39, 37, 35, 34]
    assert np.all(f[S] > 0)
    Xs = np.zeros((n, 4))
    Xs[S, range(4)] = np.sqrt(f[S])
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((4, 4)))
    for X in (Xs, Xs @ Q):
        np.testing.assert_allclose(O.gn_step(F, X), X, rtol=0, atol=1e-12 * np.abs(X).max())


def test_gn_step_equals_section_2_closed_form():
    # Section 2.5 writes the GN step as X + (I - X (X^T X)^{-1} X^T / 2)(F X (X^T X)^{-1} - X);
    # Algorithm 4 writes it as Z - X (Y^T Z - I)/2 with Y = X (X^T X)^{-1}, Z = F Y
    A = _scipy(I.laplacian_2d(9))
    coef = O.interpolant_cheb_coeffs(5)
    F = _filter_of(A, coef, 0.0, 6.0)
    X = np.random.default_rng(2).standard_normal((A.shape[0], 5))
    Gi = np.linalg.inv(X.T @ X)
    closed = X + (np.eye(A.shape[0]) - 0.5 * X @ Gi @ X.T) @ (F(X @ Gi) - X)
    np.testing.assert_allclose(O.gn_step(F, X), closed, rtol=0, atol=1e-10 * np.abs(closed).max())


@pytest.mark.parametrize("slip", ["half_dropped", "sign", "no_identity"])
def test_planted_gn_slips_are_caught(slip):
    n = 30
    dvals = np.linspace(0.0, 2.0, n)
    B = sp.diags(dvals).tocsr()
    coef = O.interpolant_cheb_coeffs(4)
    F = _filter_of(B, coef, 0.0, 1.5)
    f = O.filter_value(coef, dvals, 0.0, 1.5)
    X = np.zeros((n, 3))
    X[[29, 25, 7], range(3)] = np.sqrt(np.abs(f[[29, 25, 7]]))

    def bad(Fn, X):
        Y = X @ np.linalg.inv(X.T @ X)
        Z = Fn(Y)
        if slip == "half_dropped":
            return Z - X @ (Y.T @ Z - np.eye(3))
        if slip == "sign":
            return Z + X @ (Y.T @ Z - np.eye(3)) / 2
        return Z - X @ (Y.T @ Z) / 2

    Xr = np.random.default_rng(3).standard_normal((n, 3))
    # the slip either moves the fixed point or changes the step on a generic X
    assert (not np.allclose(bad(F, X), X, atol=1e-10)) or (not np.allclose(bad(F, Xr), O.gn_step(F, Xr), atol=1e-10))


@pytest.mark.parametrize("m,k,p", [(20, 12, 14), (32, 12, 16)])
def test_oracle_gn_inner_solver_closed_form(m, k, p):
    A = _scipy(I.laplacian_2d(m))
    X0 = I.gaussian_block(A.shape[0], p, 8)
    r = O.arrabit_mpm(A, k, X0, which="smallest", tol=1e-10, q=1, degree=8, inner="gn")
    assert r.converged
    np.testing.assert_allclose(r.evals, laplacian_2d_eigs(m)[:k], rtol=0, atol=1e-10)
    _check_invariants(A, r, 1e-10, 8.0)


def test_oracle_gn_bruteforce_random_sparse():
    n, k, p = 400, 8, 12
    A = _random_sparse_spd(n, 0.02, 77)
    wref = np.linalg.eigvalsh(A.toarray())
    r = O.arrabit_mpm(A, k, I.gaussian_block(n, p, 31), which="largest", tol=1e-10, q=1, degree=10, inner="gn")
    assert r.converged
    np.testing.assert_allclose(r.evals, wref[::-1][:k], atol=1e-9 * np.abs(wref).max())


# ---------------------------------------------------------------- adaptive q and d (Section 5)
def test_degree_rule_special_cases():
    # rho_d(a) = psi_d(-1) = f_d(-1) = 0 (t = -1 is an interpolation node), so mu*_{k+q} = a
    # gives the ratio 0 and the smallest degree, 3; equal Ritz values give the ratio 1 and
    # the cap
    assert O.next_degree("chebinterp", 5.0, 0.0, 0.0, 4.0, 15) == 3
    assert O.next_degree("chebinterp", 3.0, 3.0, 0.0, 4.0, 15) == 15
    assert O.next_degree("chebinterp", 3.0, 3.0, 0.0, 4.0, 7) == 7
    # a gap just above b needs a higher degree than a wide one
    d_close = O.next_degree("chebinterp", 4.02, 4.0, 0.0, 4.0, 40)
    d_wide = O.next_degree("chebinterp", 4.5, 4.0, 0.0, 4.0, 40)
    assert 3 <= d_wide < d_close <= 40


def test_degree_rule_against_brute_force_ratios():
    # the chosen degree is the first d >= 3 whose ratio of interpolant values (computed
    # here by numpy's Chebyshev series, not the oracle's recurrence) is below 0.9
    import numpy.polynomial.chebyshev as npc
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b = 0.0, rng.uniform(1.0, 5.0)
        mkq = b * rng.uniform(0.8, 1.05)
        mk = mkq + b * rng.uniform(0.0, 0.2)
        d = O.next_degree("chebinterp", mk, mkq, a, b, 25)
        ratio = lambda dd: (npc.chebval(2 * (mkq - a) / (b - a) - 1, O.interpolant_cheb_coeffs(dd))  # noqa: E731
                            / npc.chebval(2 * (mk - a) / (b - a) - 1, O.interpolant_cheb_coeffs(dd)))
        if d < 25:
            assert ratio(d) < 0.9
        for dd in range(3, d):
            assert not ratio(dd) < 0.9


def test_oracle_adaptive_degree_and_blocks():
    A = _scipy(I.laplacian_3d(16))
    X0 = I.gaussian_block(A.shape[0], 36, 3)
    lam = laplacian_3d_eigs(16)[:30]
    r = O.arrabit_mpm(A, 30, X0, which="smallest", tol=1e-10, q=1, degree=3, adapt_q=True, adapt_d=True)
    assert r.converged
    np.testing.assert_allclose(r.evals, lam, rtol=0, atol=1e-10)
    ds = [h.degree for h in r.history]
    assert ds[0] == 3 and max(ds) > 3 and max(ds) <= 15
    r2 = O.arrabit_mpm(A, 30, X0, which="smallest", tol=1e-10, q=1, degree=3, adapt_q=True)
    qs = [h.q for h in r2.history]
    assert qs[0] == 1 and max(qs) > 1 and max(qs) <= 3 and qs == sorted(qs)
    np.testing.assert_allclose(r2.evals, lam, rtol=0, atol=1e-10)
