"""Pins of the CPU oracle to facts outside itself: closed forms, library routines,
invariants and brute force.  Each oracle function has at least one check here that a
plausible slip (dropped term, wrong sign, transposed operand) would fail; the planted
mistakes at the end demonstrate that for the core pieces."""
import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest
import scipy.sparse as sp

from oracle import arrabit_oracle as O
from paper_1507_06078_gb300 import inputs as I

RNG = np.random.default_rng(1234)


def sym(m, rng=RNG):
    a = rng.standard_normal((m, m))
    return 0.5 * (a + a.T)


def known_spectrum(w, rng=RNG):
    """Q diag(w) Q^T with Q a product of Householder reflectors (spectrum known)."""
    m = len(w)
    Q = np.eye(m)
    for _ in range(3):
        v = rng.standard_normal(m)
        v /= np.linalg.norm(v)
        Q = Q - 2.0 * np.outer(Q @ v, v)
    return Q @ np.diag(w) @ Q.T


# ---------------------------------------------------------------- Gershgorin
def test_gershgorin_laplacians():
    A2 = I.laplacian_2d(10)
    lo, hi = O.gershgorin_bounds(O.csr_to_scipy(A2.n, A2.rowptr, A2.col, A2.val))
    assert (lo, hi) == (0.0, 8.0)
    A3 = I.laplacian_3d(5)
    lo, hi = O.gershgorin_bounds(O.csr_to_scipy(A3.n, A3.rowptr, A3.col, A3.val))
    assert (lo, hi) == (0.0, 12.0)


def test_gershgorin_contains_spectrum():
    M = sym(40)
    lo, hi = O.gershgorin_bounds(sp.csr_matrix(M))
    w = np.linalg.eigvalsh(M)
    assert lo <= w.min() and w.max() <= hi


# ---------------------------------------------------------------- Section 5 interpolant
@pytest.mark.parametrize("d", [1, 2, 3, 5, 10, 15, 20])
def test_interpolant_hits_f_at_nodes(d):
    a = O.interpolant_cheb_coeffs(d)
    t = -np.cos(np.arange(d + 1) * np.pi / d)  # second-kind points, written out here
    f = np.maximum(t, 0.0) ** (10 * d)
    np.testing.assert_allclose(npc.chebval(t, a), f, atol=1e-14)


@pytest.mark.parametrize("d", [3, 10, 15, 20])
def test_interpolant_value_at_one_and_dct_formula(d):
    a = O.interpolant_cheb_coeffs(d)
    assert abs(npc.chebval(1.0, a) - 1.0) < 1e-14
    # independent closed form for interpolation at x_j = cos(j pi/d):
    # a_k = (2/d) sum'' f(x_j) cos(j k pi/d), first and last terms halved, a_0 and a_d halved
    j = np.arange(d + 1)
    x = np.cos(j * np.pi / d)
    f = np.maximum(x, 0.0) ** (10 * d)
    w = np.ones(d + 1)
    w[0] = w[-1] = 0.5
    ak = np.array([(2.0 / d) * np.sum(w * f * np.cos(j * kk * np.pi / d)) for kk in range(d + 1)])
    ak[0] *= 0.5
    ak[-1] *= 0.5
    np.testing.assert_allclose(a, ak, atol=1e-15)


def test_interpolant_low_profile_inside_interval():
    # Section 5: inside [-1, 1] the interpolants stay low except near t = 1
    for d in (3, 5, 7):
        a = O.interpolant_cheb_coeffs(d)
        t = np.linspace(-1, 0.5, 2001)
        assert np.max(np.abs(npc.chebval(t, a))) < 0.25


@pytest.mark.parametrize("d", [1, 4, 10, 20])
def test_cheb_to_monomial(d):
    a = O.interpolant_cheb_coeffs(d)
    g = O.cheb_to_monomial(a)
    assert len(g) == d + 1
    t = np.linspace(-1.2, 1.2, 31)
    np.testing.assert_allclose(np.polyval(g, t), npc.chebval(t, a), atol=1e-9 * max(1, np.abs(g).max()))


def test_eval_cheb_series_and_T_d():
    rng = np.random.default_rng(5)
    a = rng.standard_normal(9)
    t = np.linspace(-1.5, 1.5, 41)
    np.testing.assert_allclose(O.eval_cheb_series(a, t), npc.chebval(t, a), rtol=1e-13, atol=1e-13)
    th = np.linspace(0, np.pi, 17)
    for d in (1, 2, 7, 20):
        np.testing.assert_allclose(O.eval_cheb_series(O.chebyshev_T_coeffs(d), np.cos(th)),
                                   np.cos(d * th), atol=1e-12)


# ---------------------------------------------------------------- Alg. 7 / Clenshaw filter
@pytest.mark.parametrize("evaluator", ["alg7", "clenshaw"])
@pytest.mark.parametrize("d", [1, 2, 3, 10])
def test_filter_exact_on_diagonal_matrix(evaluator, d):
    # eq. poly-A: rho(A) = Q rho(Lambda) Q^T; for diagonal A, rho(A) X = diag(rho(lambda)) X
    rng = np.random.default_rng(d)
    lam = np.sort(rng.uniform(0.0, 5.0, 60))
    B = sp.diags(lam).tocsr()
    X = rng.standard_normal((60, 7))
    a, b = 0.0, 3.0
    coef = O.interpolant_cheb_coeffs(d)
    if evaluator == "alg7":
        Y = O.poly_alg7(B, X, a, b, O.cheb_to_monomial(coef))
    else:
        Y = O.poly_clenshaw(B, X, a, b, coef)
    rho = npc.chebval((2 * lam - a - b) / (b - a), coef)
    np.testing.assert_allclose(Y, rho[:, None] * X, rtol=1e-11, atol=1e-12)


def test_filter_on_laplacian_eigenvectors():
    # closed-form eigenvectors of the 2D Dirichlet Laplacian: sin products
    m = 12
    A = I.laplacian_2d(m)
    B = O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)
    x = np.arange(1, m + 1)
    pairs = [(1, 1), (2, 5), (7, 3), (12, 12)]
    V = np.stack([np.outer(np.sin(np.pi * i * x / (m + 1)), np.sin(np.pi * j * x / (m + 1))).T.ravel()
                  for i, j in pairs], axis=1)
    lam = np.array([4 - 2 * np.cos(np.pi * i / (m + 1)) - 2 * np.cos(np.pi * j / (m + 1)) for i, j in pairs])
    coef = O.interpolant_cheb_coeffs(6)
    Y = O.poly_clenshaw(B, V, 0.0, 6.0, coef)
    rho = npc.chebval((2 * lam - 6.0) / 6.0, coef)
    np.testing.assert_allclose(Y, V * rho[None, :], atol=1e-12)


@pytest.mark.parametrize("d", [2, 5, 10])
def test_horner_equals_clenshaw(d):
    A = I.laplacian_2d(9)
    B = O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)
    X = np.random.default_rng(3).standard_normal((A.n, 5))
    coef = O.interpolant_cheb_coeffs(d)
    Y1 = O.poly_alg7(B, X, 0.0, 4.5, O.cheb_to_monomial(coef))
    Y2 = O.poly_clenshaw(B, X, 0.0, 4.5, coef)
    np.testing.assert_allclose(Y1, Y2, rtol=1e-9, atol=1e-9 * np.abs(Y2).max())


def test_plain_chebyshev_filter():
    lam = np.linspace(-1.0, 1.3, 23)
    X = np.ones((23, 1))
    Y = O.poly_clenshaw(sp.diags(lam).tocsr(), X, -1.0, 1.0, O.chebyshev_T_coeffs(5))
    np.testing.assert_allclose(Y[:, 0], npc.chebval(lam, [0, 0, 0, 0, 0, 1]), atol=1e-13)


# ---------------------------------------------------------------- dense helpers
def test_rcond_against_library_and_closed_form():
    w = np.array([4.0, 2.0, 1.0, 0.5, 1e-3])
    assert abs(O.rcond_spd(np.diag(w)) - 1e-3 / 4.0) < 1e-18
    rng = np.random.default_rng(9)
    Xb = rng.standard_normal((200, 12)) @ np.diag(np.logspace(0, -3, 12))
    G = Xb.T @ Xb
    ref = 1.0 / np.linalg.cond(G, 1)
    assert abs(O.rcond_spd(G) - ref) <= 1e-8 * ref
    # singular Gram (duplicated column) -> 0 or numerically tiny
    Xs = np.hstack([Xb, Xb[:, :1]])
    assert O.rcond_spd(Xs.T @ Xs) < 1e-14


def test_orth_basis_and_rank():
    rng = np.random.default_rng(11)
    Z = rng.standard_normal((100, 8))
    U = O.orth(Z)
    assert U.shape == (100, 8)
    np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-14)
    np.testing.assert_allclose(U @ (U.T @ Z), Z, atol=1e-12)
    Zd = np.hstack([Z[:, :5], Z[:, :3] @ rng.standard_normal((3, 4))])
    assert O.orth(Zd).shape[1] == 5


@pytest.mark.parametrize("m", [1, 2, 3, 10, 37])
def test_jacobi_against_lapack(m):
    H = sym(m)
    w, V = O.jacobi_eigh(H)
    wref = np.sort(np.linalg.eigvalsh(H))[::-1]
    np.testing.assert_allclose(w, wref, atol=1e-13 * max(1, np.abs(wref).max()))
    np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-13)
    np.testing.assert_allclose(H @ V, V * w[None, :], atol=1e-12)
    assert np.all(np.diff(w) <= 0)


def test_jacobi_known_spectrum_with_clusters():
    w0 = np.array([5.0, 5.0, 5.0, 2.0, 2.0, 1e-9, 0.0, -3.0, -3.0, 7.5])
    H = known_spectrum(w0)
    w, V = O.jacobi_eigh(H)
    np.testing.assert_allclose(w, np.sort(w0)[::-1], atol=1e-13)
    np.testing.assert_allclose(H @ V, V * w[None, :], atol=1e-12)
    w, V = O.jacobi_eigh(np.zeros((4, 4)))
    np.testing.assert_array_equal(w, np.zeros(4))


def test_rayleigh_ritz_invariant_subspace():
    A = I.laplacian_2d(10)
    B = O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)
    wref, Vref = np.linalg.eigh(B.toarray())
    rng = np.random.default_rng(2)
    Z = Vref[:, -6:] @ rng.standard_normal((6, 6))
    Y, w = O.rayleigh_ritz(B, Z)
    np.testing.assert_allclose(w, wref[-6:][::-1], atol=1e-13)
    np.testing.assert_allclose(Y.T @ Y, np.eye(6), atol=1e-13)
    np.testing.assert_allclose(O.residual_norms(B, Y, w, w), 0.0, atol=1e-13)


def test_augment_spans_krylov_and_unit_columns():
    A = I.laplacian_2d(8)
    B = O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)
    X = np.random.default_rng(4).standard_normal((A.n, 3))
    Z = O.augment(B, X, 2)
    assert Z.shape == (A.n, 9)
    np.testing.assert_allclose(np.linalg.norm(Z, axis=0), 1.0, atol=1e-15)
    K = np.hstack([X, B @ X, B @ (B @ X)])
    P = Z @ np.linalg.pinv(Z)
    np.testing.assert_allclose(P @ K, K, atol=1e-9 * np.abs(K).max())


# ---------------------------------------------------------------- planted mistakes
def _clenshaw_dropped_b2(B, X, a, b, coef):
    d = len(coef) - 1
    c0 = (a + b) / (a - b)
    c1 = 2.0 / (b - a)
    S = lambda Y: c1 * (B @ Y) + c0 * Y  # noqa: E731
    b1 = coef[d] * X
    for j in range(d - 1, 0, -1):
        b1 = coef[j] * X + 2.0 * S(b1)  # the "- b_{j+2}" term dropped
    return coef[0] * X + S(b1)


def test_planted_clenshaw_slip_is_caught():
    lam = np.linspace(0, 5, 30)
    B = sp.diags(lam).tocsr()
    X = np.ones((30, 1))
    coef = O.interpolant_cheb_coeffs(6)
    rho = npc.chebval((2 * lam - 3.0) / 3.0, coef)
    Y = _clenshaw_dropped_b2(B, X, 0.0, 3.0, coef)
    assert not np.allclose(Y[:, 0], rho, atol=1e-8)


def test_planted_jacobi_sign_slip_is_caught(monkeypatch):
    real_sqrt = math.sqrt

    # flip the sign convention of t: the rotation then fails to annihilate h_ij
    def bad_jacobi(H, tol=1e-15, max_sweeps=8):
        A = np.array(H, dtype=float)
        m = A.shape[0]
        V = np.eye(m)
        for _ in range(max_sweeps):
            for i in range(m - 1):
                for j in range(i + 1, m):
                    if A[i, j] == 0.0:
                        continue
                    th = (A[j, j] - A[i, i]) / (2 * A[i, j])
                    t = -np.sign(th or 1.0) / (abs(th) + real_sqrt(th * th + 1))
                    c = 1 / real_sqrt(t * t + 1)
                    s = t * c
                    ci, cj = A[:, i].copy(), A[:, j].copy()
                    A[:, i], A[:, j] = c * ci - s * cj, s * ci + c * cj
                    ri, rj = A[i, :].copy(), A[j, :].copy()
                    A[i, :], A[j, :] = c * ri - s * rj, s * ri + c * rj
                    vi, vj = V[:, i].copy(), V[:, j].copy()
                    V[:, i], V[:, j] = c * vi - s * vj, s * vi + c * vj
        w = np.diag(A)
        o = np.argsort(-w)
        return w[o], V[:, o]

    H = sym(8)
    w, V = bad_jacobi(H)
    assert not np.allclose(H @ V, V * w[None, :], atol=1e-8)


def test_planted_interpolation_nodes_slip_is_caught():
    d = 8
    # first-kind points instead of second-kind: still interpolates something, but not
    # f_d at the second-kind nodes
    t1 = np.cos((2 * np.arange(d + 1) + 1) * np.pi / (2 * d + 2))
    T = np.cos(np.outer(np.arccos(t1), np.arange(d + 1)))
    a_bad = np.linalg.solve(T, np.maximum(t1, 0) ** (10 * d))
    t = -np.cos(np.arange(d + 1) * np.pi / d)
    assert not np.allclose(npc.chebval(t, a_bad), np.maximum(t, 0) ** (10 * d), atol=1e-6)


@pytest.mark.parametrize("which", ["laplace2d", "diag", "chung_lu"])
def test_lanczos_bounds_enclose_the_spectrum(which):
    # the estimates of the far ends of the spectrum contain the true extreme eigenvalues
    # (residual margins) and are close to them (Kaniel-Paige: extreme Ritz values converge
    # first)
    import scipy.sparse as sp

    from paper_1507_06078_gb300 import inputs as I
    if which == "laplace2d":
        A = sp.csr_matrix(I.laplacian_2d(20).to_dense())
    elif which == "diag":
        A = sp.diags(np.linspace(-3.0, 5.0, 500)).tocsr()
    else:
        C, _ = I.chung_lu_laplacian(1500, seed=3)
        A = sp.csr_matrix((C.val, C.col, C.rowptr), shape=(C.n, C.n))
    lam = np.linalg.eigvalsh(A.toarray())
    lo, hi = O.lanczos_bounds(A, 32, 99)
    assert lo <= lam[0] and hi >= lam[-1]
    span = lam[-1] - lam[0]
    assert hi - lam[-1] <= 0.05 * span and lam[0] - lo <= 0.05 * span
    # far tighter than Gershgorin on the graph Laplacian
    if which == "chung_lu":
        assert hi < 0.5 * O.gershgorin_bounds(A)[1]


def test_sell_oracle_pins():
    # SELL-C-sigma oracle against properties fixed by the format's definition: a diagonal
    # pattern (every row length 1) keeps the identity order and has no padding; C = 1 with
    # sigma = n is a global sort by decreasing length; sigma = 1 keeps the original order
    from oracle import sell_oracle as S
    perm, ln, cptr, src = S.sell_c_sigma(list(range(11)), 4, 8)
    assert perm.tolist() == list(range(10)) and cptr[-1] == 12 and (src >= 0).sum() == 10
    rowptr = [0, 2, 2, 7, 8, 11]
    perm, ln, cptr, src = S.sell_c_sigma(rowptr, 1, 5)
    assert perm.tolist() == [2, 4, 0, 3, 1] and ln.tolist() == [5, 3, 2, 1, 0]
    assert cptr.tolist() == [0, 5, 8, 10, 11, 11]
    perm, ln, cptr, src = S.sell_c_sigma(rowptr, 2, 1)
    assert perm.tolist() == [0, 1, 2, 3, 4] and cptr.tolist() == [0, 4, 14, 20]
