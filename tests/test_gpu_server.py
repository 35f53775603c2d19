"""Serving: continuous batching of solves (arb_server_*).  Each request's result must be
the same alone and in a concurrent mix; admission follows the HBM footprint."""
import numpy as np
import pytest
import scipy.sparse as sp

from conftest import laplacian_3d_eigs
from paper_1507_06078_gb300 import inputs as I

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


def _opts(arb, k, p, q, d, precision=0):
    o = arb.arb_options_default(k)
    o.p, o.q, o.degree, o.precision = p, q, d, precision
    return o


def _random_spd(n, seed):
    from paper_1507_06078_gb300.inputs import CSR
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=0.02, random_state=rng, format="csr")
    M = (M + M.T + sp.diags(rng.uniform(0, 3, n))).tocsr()
    M.sort_indices()
    return CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def _mix(arb, ctx):
    # (matrix, k, which, tol, options): 2D/3D Laplacians, a random SPD matrix from both
    # ends, the 64x64 workload and a mixed-precision request
    specs = [
        (I.laplacian_2d(24), 10, 1, 1e-10, _opts(arb, 10, 14, 1, 8)),
        (I.laplacian_2d(32), 12, 1, 1e-10, _opts(arb, 12, 16, 1, 8)),
        (I.laplacian_3d(12), 20, 1, 1e-8, _opts(arb, 20, 24, 2, 10)),
        (_random_spd(400, 5), 8, 0, 1e-10, _opts(arb, 8, 12, 1, 10)),
        (_random_spd(400, 6), 8, 1, 1e-10, _opts(arb, 8, 12, 1, 10)),
        (I.laplacian_2d(64), 20, 1, 1e-10, _opts(arb, 20, 30, 1, 10)),
        (I.laplacian_3d(16), 20, 1, 1e-8, _opts(arb, 20, 24, 2, 10, precision=1)),
    ]
    out = []
    for i, (A, k, which, tol, o) in enumerate(specs):
        out.append((arb.Matrix.from_csr(ctx, A), k, which, tol, o, I.gaussian_block(A.n, o.p, 700 + i)))
    return out


def test_server_mix_matches_standalone(arb, ctx):
    mix = _mix(arb, ctx)
    alone = [arb.arb_solve(ctx, m, k, w, tol, o, x0=x0) for (m, k, w, tol, o, x0) in mix]
    srv = arb.Server(0, hbm_budget_bytes=8 << 30, max_slots=3)
    try:
        tickets = [srv.submit(m, k, w, tol, o, x0=x0) for (m, k, w, tol, o, x0) in mix]
        got = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    for a, g in zip(alone, got):
        assert g.status == a.status
        # identical kernel sequence per request: the same numbers, in the mix or alone
        np.testing.assert_allclose(g.evals, a.evals, rtol=0, atol=1e-12)
        np.testing.assert_allclose(g.evecs, a.evecs, rtol=0, atol=1e-12)
        assert g.info["latency_s"] > 0.0
        assert g.info["outer_iters"] == a.info["outer_iters"]


def test_server_rejects_oversize_request(arb, ctx):
    A = I.laplacian_3d(40)
    m = arb.Matrix.from_csr(ctx, A)
    need = arb.arb_server_footprint(A.n, A.nnz, 48, 2, 0)
    srv = arb.Server(0, hbm_budget_bytes=need // 2, max_slots=2)
    try:
        with pytest.raises(arb.ArbError) as e:
            srv.submit(m, 40, 1, 1e-8, _opts(arb, 40, 48, 2, 10))
        assert e.value.status == arb.ARB_REJECTED
    finally:
        srv.close()


def test_server_queue_timeout_and_memory_bound_admission(arb, ctx):
    # budget for one request at a time: the second waits for the first's memory
    big = I.laplacian_3d(32)
    small = I.laplacian_2d(24)
    mb, ms = arb.Matrix.from_csr(ctx, big), arb.Matrix.from_csr(ctx, small)
    ob, os_ = _opts(arb, 40, 48, 2, 10), _opts(arb, 10, 14, 1, 8)
    fb = arb.arb_server_footprint(big.n, big.nnz, 48, 2, 0)
    fs = arb.arb_server_footprint(small.n, small.nnz, 14, 1, 0)
    srv = arb.Server(0, hbm_budget_bytes=max(fb, fs) + min(fb, fs) // 2, max_slots=2)
    try:
        t1 = srv.submit(mb, 40, 1, 1e-8, ob, x0=I.gaussian_block(big.n, 48, 1))
        t2 = srv.submit(ms, 10, 1, 1e-10, os_, x0=I.gaussian_block(small.n, 14, 2))
        assert srv.wait(t2, timeout_ms=0) is None  # still queued behind the big one
        r1 = srv.wait(t1)
        r2 = srv.wait(t2)
    finally:
        srv.close()
    from conftest import laplacian_2d_eigs, laplacian_3d_eigs
    np.testing.assert_allclose(r1.evals, laplacian_3d_eigs(32)[:40], atol=1e-9)
    np.testing.assert_allclose(r2.evals, laplacian_2d_eigs(24)[:10], atol=1e-10)
    assert r2.info["latency_s"] >= r1.info["latency_s"] * 0.5


def test_solve_batched_matches_standalone(arb, ctx):
    # uneven diffusion instances (the batched workload's family) plus Laplacians
    probs = []
    for i, A in enumerate([I.diffusion_2d(20, 1), I.diffusion_2d(36, 2), I.laplacian_2d(28), I.diffusion_2d(48, 3),
                           I.laplacian_3d(10)]):
        k = 6 + 2 * i
        p = int(round(1.5 * k))
        o = _opts(arb, k, p, 1, 10, precision=i % 2)
        probs.append(dict(mat=arb.Matrix.from_csr(ctx, A), k=k, which=1, tol=1e-8, opts=o,
                          x0=I.gaussian_block(A.n, p, 900 + i), A=A))
    st, res = arb.arb_solve_batched(ctx, probs, max_concurrent=3)
    assert st == arb.ARB_OK
    for pr, r in zip(probs, res):
        alone = arb.arb_solve(ctx, pr["mat"], pr["k"], 1, 1e-8, pr["opts"], x0=pr["x0"])
        np.testing.assert_allclose(r.evals, alone.evals, rtol=0, atol=1e-12)
        wref = np.linalg.eigvalsh(pr["A"].to_dense())[:pr["k"]]
        np.testing.assert_allclose(r.evals, wref, atol=1e-8 * max(1.0, np.abs(wref).max()))


def test_server_concurrent_block_jacobi(arb, ctx):
    # Rayleigh-Ritz orders above 96 run the cooperative block-Jacobi kernel; three slots run
    # it concurrently, each on its share of the device, and every result matches the
    # standalone solve
    mix = []
    for i, m in enumerate([14, 15, 16]):
        A = I.laplacian_3d(m)
        k, p = 50, 64
        mix.append((arb.Matrix.from_csr(ctx, A), k, _opts(arb, k, p, 1, 10), I.gaussian_block(A.n, p, 800 + i), m))
    alone = [arb.arb_solve(ctx, mat, k, 1, 1e-8, o, x0=x0) for (mat, k, o, x0, m) in mix]
    srv = arb.Server(0, hbm_budget_bytes=8 << 30, max_slots=3)
    try:
        tickets = [srv.submit(mat, k, 1, 1e-8, o, x0=x0) for (mat, k, o, x0, m) in mix]
        got = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    for a, g, (mat, k, o, x0, m) in zip(alone, got, mix):
        assert g.status == arb.ARB_OK
        np.testing.assert_allclose(g.evals, a.evals, rtol=0, atol=1e-12)
        np.testing.assert_allclose(g.evals, laplacian_3d_eigs(m)[:k], atol=1e-8)
