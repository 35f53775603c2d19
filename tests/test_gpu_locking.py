"""Deflation (eq. defl), the merge of locked and new Ritz pairs (Algorithm 8) and the
completion of a short Ritz set, on the GPU through the C ABI, against the oracle and the
closed-form / dense spectra.

The first continuation tolerance tol_1 is a parameter of Algorithm 8; a loose tol_1 lets
the lock threshold max(1e-14, tol_t^2) catch the leading pairs while the others still
iterate, and the later outer iterations project X and the augmented block against a
non-empty Q_c.  The same settings lock pairs in the oracle (pinned in
test_oracle_solver.py)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import arrabit_oracle as O
from paper_1507_06078_gb300 import inputs as I

from conftest import laplacian_2d_eigs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def arb():
    from paper_1507_06078_gb300 import arrabit, build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return arrabit


@pytest.fixture(scope="module")
def ctx(arb):
    c = arb.Context(0)
    yield c
    c.close()


def scipy_of(A):
    return O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)


def _opts(arb, k, p, q, d, **kw):
    o = arb.arb_options_default(k)
    o.p, o.q, o.degree = p, q, d
    for key, v in kw.items():
        setattr(o, key, v)
    return o


def test_solve_locks_pairs_against_oracle(arb, ctx):
    # tol_1 = 0.03: after the second outer iteration maxres (~1e-6) is below tol_1, the
    # continuation sets tol_t = 3e-4 and the lock threshold tol_t^2 = 9e-8, which the
    # leading pairs have passed by then - several pairs are locked and the last outer
    # iterations run against a non-empty Q_c, in the oracle and on the GPU alike
    A = I.laplacian_2d(20)
    k, p = 12, 14
    X0 = I.gaussian_block(A.n, p, 9)
    mat = arb.Matrix.from_csr(ctx, A)
    o = _opts(arb, k, p, 1, 8, tol1=0.03)
    r = arb.arb_solve(ctx, mat, k, arb.ARB_SMALLEST, 1e-10, o, x0=X0, evecs="host")
    assert r.status == arb.ARB_OK, r.info
    assert r.info["max_locked"] > 0, r.info
    ref = O.arrabit_mpm(scipy_of(A), k, X0, which="smallest", tol=1e-10, q=1, degree=8, tol1=0.03)
    assert max(h.n_locked for h in ref.history) > 0
    lam = laplacian_2d_eigs(20)[:k]
    np.testing.assert_allclose(r.evals, ref.evals, rtol=0, atol=1e-10)
    np.testing.assert_allclose(r.evals, lam, rtol=0, atol=1e-10)
    Q = r.evecs
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-12)
    R = scipy_of(A) @ Q - Q * r.evals[None, :]
    assert np.linalg.norm(R, axis=0).max() <= 1e-10 * 8.0


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_locking_grows_to_all_locked(arb, ctx, precision):
    # k = p and a tolerance below the FP64 residual floor: pairs lock as they reach the
    # threshold floor 1e-14 until the whole block is locked (ARB_STOP_ALL_LOCKED), as in
    # the oracle with the same inputs.  With ARB_MIXED the FP32 phase never locks (its
    # residuals stop far above the thresholds); its FP64 refinement locks the same way.
    # (ARB_MIXED_DF's double-float filter leaves residuals near 1e-13, above the 1e-14
    # floor of the threshold, so it stops on the stall rule instead.)
    A = I.laplacian_2d(20)
    k = p = 10
    X0 = I.gaussian_block(A.n, p, 8)
    mat = arb.Matrix.from_csr(ctx, A)
    o = _opts(arb, k, p, 1, 8, tol1=1e-2, precision=precision)
    r = arb.arb_solve(ctx, mat, k, arb.ARB_SMALLEST, 1e-15, o, x0=X0, evecs="host")
    ref = O.arrabit_mpm(scipy_of(A), k, X0, which="smallest", tol=1e-15, q=1, degree=8, tol1=1e-2)
    assert ref.stop_reason == "all_locked"
    assert r.info["stop_reason"] == "all_locked", r.info
    assert r.status == arb.ARB_NOT_CONVERGED
    assert r.info["n_locked"] == p
    np.testing.assert_allclose(r.evals, laplacian_2d_eigs(20)[:k], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.evals, ref.evals, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.evecs.T @ r.evecs, np.eye(k), atol=1e-12)


def test_solve_rank_deficient_start_block_is_padded(arb, ctx):
    # duplicated start columns: the q = 1 subspace has dimension 10 < p = 14 in the first
    # outer iteration, so the Ritz block is completed with Gaussian columns; the solve
    # reaches the dense eigenvalues (the oracle completes it from its own pool and reaches
    # them too: test_oracle_rank_deficient_start_block_is_padded)
    from paper_1507_06078_gb300.inputs import CSR
    n, k, p = 400, 8, 14
    rng = np.random.default_rng(77)
    M = sp.random(n, n, density=0.02, random_state=rng, format="csr")
    M = (M + M.T + sp.diags(rng.uniform(0, 3, n))).tocsr()
    M.sort_indices()
    A = CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    G = I.gaussian_block(n, 5, 32)
    X0 = np.ascontiguousarray(np.hstack([G, G, G[:, :4]]))
    mat = arb.Matrix.from_csr(ctx, A)
    for precision in (0, 2):
        o = _opts(arb, k, p, 1, 10, precision=precision)
        r = arb.arb_solve(ctx, mat, k, arb.ARB_LARGEST, 1e-10, o, x0=X0, evecs="host")
        assert r.status == arb.ARB_OK, r.info
        wref = np.linalg.eigvalsh(M.toarray())
        np.testing.assert_allclose(r.evals, wref[::-1][:k], rtol=0, atol=1e-9 * np.abs(wref).max())
        np.testing.assert_allclose(r.evecs.T @ r.evecs, np.eye(k), atol=1e-12)
