"""The Gauss-Newton inner solver (Algorithm 8's GN branch, Algorithm 4) and the adaptive
augmentation count and polynomial degree of Section 5 (eqs. block, hat-d, degree) on the
GPU through the C ABI, against the oracle (the same options), closed-form spectra and
dense eigenvalues."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import arrabit_oracle as O
from paper_1507_06078_gb300 import inputs as I

from conftest import laplacian_2d_eigs, laplacian_3d_eigs

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


@pytest.mark.parametrize("m,k,p", [(20, 12, 14), (32, 12, 16)])
def test_gn_solve_against_oracle_and_closed_form(arb, ctx, m, k, p):
    A = I.laplacian_2d(m)
    X0 = I.gaussian_block(A.n, p, 8)
    mat = arb.Matrix.from_csr(ctx, A)
    r = arb.arb_solve(ctx, mat, k, arb.ARB_SMALLEST, 1e-10, _opts(arb, k, p, 1, 8, inner=arb.ARB_INNER_GN), x0=X0)
    assert r.status == arb.ARB_OK, r.info
    ref = O.arrabit_mpm(scipy_of(A), k, X0, which="smallest", tol=1e-10, q=1, degree=8, inner="gn")
    lam = laplacian_2d_eigs(m)[:k]
    np.testing.assert_allclose(r.evals, ref.evals, rtol=0, atol=1e-10)
    np.testing.assert_allclose(r.evals, lam, rtol=0, atol=1e-10)
    Q = r.evecs
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-12)
    assert np.linalg.norm(scipy_of(A) @ Q - Q * r.evals[None, :], axis=0).max() <= 1e-10 * 8.0


def test_gn_lockstep_fixed_schedule(arb, ctx):
    # a fixed inner schedule (four GN steps per outer iteration, b refreshed after every
    # ARR) makes the outer iterations of the GPU and the oracle the same sequence of operations
    A = I.laplacian_2d(16)
    X0 = I.gaussian_block(A.n, 12, 10)
    mat = arb.Matrix.from_csr(ctx, A)
    o = _opts(arb, 10, 12, 1, 8, inner=arb.ARB_INNER_GN, inner_fixed=4, maxit=20, b_update=1)
    r = arb.arb_solve(ctx, mat, 10, arb.ARB_SMALLEST, 1e-9, o, x0=X0)
    ref = O.arrabit_mpm(scipy_of(A), 10, X0, which="smallest", tol=1e-9, q=1, degree=8, inner="gn",
                        inner_fixed=4, maxit=20, b_update="every_arr")
    assert ref.converged
    assert r.info["n_filters"] == 4 * r.info["outer_iters"]
    assert r.info["outer_iters"] == ref.outer_iters
    np.testing.assert_allclose(r.evals, ref.evals, rtol=0, atol=1e-9)
    np.testing.assert_allclose(r.evals, laplacian_2d_eigs(16)[:10], rtol=0, atol=1e-9)


@pytest.mark.parametrize("precision", [0, 2])
def test_gn_bruteforce_random_sparse_largest(arb, ctx, precision):
    from paper_1507_06078_gb300.inputs import CSR
    n, k, p = 400, 8, 12
    rng = np.random.default_rng(77)
    M = sp.random(n, n, density=0.02, random_state=rng, format="csr")
    M = (M + M.T + sp.diags(rng.uniform(0, 3, n))).tocsr()
    M.sort_indices()
    A = CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    mat = arb.Matrix.from_csr(ctx, A)
    o = _opts(arb, k, p, 1, 10, inner=arb.ARB_INNER_GN, precision=precision)
    r = arb.arb_solve(ctx, mat, k, arb.ARB_LARGEST, 1e-10, o, x0=I.gaussian_block(n, p, 31))
    assert r.status == arb.ARB_OK, r.info
    wref = np.linalg.eigvalsh(M.toarray())
    np.testing.assert_allclose(r.evals, wref[::-1][:k], rtol=0, atol=1e-9 * np.abs(wref).max())


def test_adaptive_degree_against_oracle(arb, ctx):
    A = I.laplacian_3d(16)
    X0 = I.gaussian_block(A.n, 36, 3)
    mat = arb.Matrix.from_csr(ctx, A)
    o = _opts(arb, 30, 36, 1, 3, adapt=arb.ARB_ADAPT_DEGREE)
    r = arb.arb_solve(ctx, mat, 30, arb.ARB_SMALLEST, 1e-10, o, x0=X0)
    assert r.status == arb.ARB_OK, r.info
    ref = O.arrabit_mpm(scipy_of(A), 30, X0, which="smallest", tol=1e-10, q=1, degree=3, adapt_d=True)
    lam = laplacian_3d_eigs(16)[:30]
    np.testing.assert_allclose(r.evals, ref.evals, rtol=0, atol=1e-10)
    np.testing.assert_allclose(r.evals, lam, rtol=0, atol=1e-10)
    # the degree rule ran: the last degree is the oracle's (the rule reads the same Ritz values)
    assert r.info["final_d"] > 3
    assert r.info["final_d"] == ref.history[-1].degree


@pytest.mark.parametrize("precision", [0, 2])
def test_adaptive_blocks_and_degree(arb, ctx, precision):
    A = I.laplacian_3d(16)
    X0 = I.gaussian_block(A.n, 36, 3)
    mat = arb.Matrix.from_csr(ctx, A)
    o = _opts(arb, 30, 36, 1, 3, adapt=arb.ARB_ADAPT_Q | arb.ARB_ADAPT_DEGREE, precision=precision)
    r = arb.arb_solve(ctx, mat, 30, arb.ARB_SMALLEST, 1e-10, o, x0=X0)
    assert r.status == arb.ARB_OK, r.info
    np.testing.assert_allclose(r.evals, laplacian_3d_eigs(16)[:30], rtol=0, atol=1e-10)
    assert 1 <= r.info["final_q"] <= 3 and 3 <= r.info["final_d"] <= 15
    # q alone: the rule of eq. block raises it on this spectrum (as in the oracle)
    o2 = _opts(arb, 30, 36, 1, 3, adapt=arb.ARB_ADAPT_Q)
    r2 = arb.arb_solve(ctx, mat, 30, arb.ARB_SMALLEST, 1e-10, o2, x0=X0)
    ref2 = O.arrabit_mpm(scipy_of(A), 30, X0, which="smallest", tol=1e-10, q=1, degree=3, adapt_q=True)
    assert max(h.q for h in ref2.history) > 1
    if precision == 0:
        assert r2.info["final_q"] > 1
    np.testing.assert_allclose(r2.evals, laplacian_3d_eigs(16)[:30], rtol=0, atol=1e-10)


def test_bad_inner_and_adapt_options_rejected(arb, ctx):
    A = I.laplacian_2d(8)
    mat = arb.Matrix.from_csr(ctx, A)
    for kw in ({"inner": 7}, {"adapt": 8}, {"d_max": 99}):
        o = _opts(arb, 4, 6, 1, 4, **kw)
        with pytest.raises(arb.ArbError) as e:
            arb.arb_solve(ctx, mat, 4, arb.ARB_SMALLEST, 1e-8, o, x0=I.gaussian_block(A.n, 6, 1))
        assert e.value.status == arb.ARB_INVALID_ARG
