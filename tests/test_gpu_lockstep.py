"""Lock-step batched solves (arb_solve_lockstep: every instance's multi-power steps of a
round filtered in one persistent batched launch, rounds captured into CUDA graphs) and the
SpMM autotuner, against standalone arb_solve calls, dense eigenvalues and the oracle."""
import numpy as np
import pytest

from oracle import arrabit_oracle as O
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


def _opts(arb, k, p, q, d, **kw):
    o = arb.arb_options_default(k)
    o.p, o.q, o.degree = p, q, d
    for key, v in kw.items():
        setattr(o, key, v)
    return o


def _problems(arb, ctx, precisions, inner=None):
    probs = []
    mats = [I.diffusion_2d(20, 1), I.diffusion_2d(36, 2), I.laplacian_2d(28), I.diffusion_2d(48, 3),
            I.laplacian_3d(10), I.diffusion_2d(40, 4)]
    for i, A in enumerate(mats):
        k = 6 + 2 * i
        p = int(round(1.5 * k))
        kw = {"precision": precisions[i % len(precisions)], "b_update": 1}
        if inner is not None and i % 2 == 1:
            kw["inner"] = inner
        o = _opts(arb, k, p, 1, 12, **kw)
        probs.append(dict(mat=arb.Matrix.from_csr(ctx, A), k=k, which=arb.ARB_SMALLEST, tol=1e-9, opts=o,
                          x0=I.gaussian_block(A.n, p, 900 + i), A=A))
    return probs


@pytest.mark.parametrize("flags", [0, 1])
def test_lockstep_matches_standalone_and_dense(arb, ctx, flags):
    # FP64 and mixed (FP32 phase + FP64 refinement) instances of uneven sizes, widths and
    # precisions: the same eigenpairs as one arb_solve each (the batched filter does the
    # single-instance arithmetic; the column sums of squares are added in another order)
    probs = _problems(arb, ctx, [0, 1])
    st, res, stats = arb.arb_solve_lockstep(ctx, probs, flags=flags)
    assert st == arb.ARB_OK, [r.info for r in res]
    assert stats["rounds"] > 0 and stats["batched_launches"] > 0
    if flags & arb.ARB_BATCH_GRAPHS:
        assert stats["graphs_captured"] > 0 and stats["graph_launches"] > 0, stats
    for pr, r in zip(probs, res):
        alone = arb.arb_solve(ctx, pr["mat"], pr["k"], pr["which"], pr["tol"], pr["opts"], x0=pr["x0"])
        np.testing.assert_allclose(r.evals, alone.evals, rtol=0, atol=1e-10)
        wref = np.linalg.eigvalsh(pr["A"].to_dense())[:pr["k"]]
        np.testing.assert_allclose(r.evals, wref, rtol=0, atol=1e-9 * max(1.0, np.abs(wref).max()))
        Q = r.evecs
        np.testing.assert_allclose(Q.T @ Q, np.eye(pr["k"]), atol=1e-10)
        assert r.info["maxres"] <= 10 * pr["tol"]


def test_lockstep_with_single_step_instances(arb, ctx):
    # GN instances and double-float refinements take their inner steps alone, in the same
    # rounds as the batched ones
    probs = _problems(arb, ctx, [0, 2], inner=arb.ARB_INNER_GN)
    st, res, stats = arb.arb_solve_lockstep(ctx, probs, flags=arb.ARB_BATCH_GRAPHS)
    assert st == arb.ARB_OK, [r.info for r in res]
    assert stats["single_steps"] > 0 and stats["batched_launches"] > 0
    for pr, r in zip(probs, res):
        wref = np.linalg.eigvalsh(pr["A"].to_dense())[:pr["k"]]
        np.testing.assert_allclose(r.evals, wref, rtol=0, atol=1e-9 * max(1.0, np.abs(wref).max()))


def test_lockstep_against_oracle_on_diffusion_instances(arb, ctx):
    # the batched workload's family (lognormal-coefficient diffusion, p = 1.5 k) against the
    # oracle run with the same options, on two of the instances
    ws = I.batched_diffusion_instances(count=3, base_seed=30000, side_range=(32, 56))
    probs = []
    for w in ws:
        o = _opts(arb, w.k, w.p, 1, 20, b_update=1)
        probs.append(dict(mat=arb.Matrix.from_csr(ctx, w.A), k=w.k, which=arb.ARB_SMALLEST, tol=1e-9, opts=o,
                          x0=I.gaussian_block(w.A.n, w.p, w.seed), w=w))
    st, res, stats = arb.arb_solve_lockstep(ctx, probs, flags=arb.ARB_BATCH_GRAPHS | arb.ARB_BATCH_AUTOTUNE)
    assert st == arb.ARB_OK, [r.info for r in res]
    for pr, r in list(zip(probs, res))[:2]:
        w = pr["w"]
        ref = O.arrabit_mpm(O.csr_to_scipy(w.A.n, w.A.rowptr, w.A.col, w.A.val), w.k, pr["x0"], which="smallest",
                            tol=1e-9, q=1, degree=20, b_update="every_arr")
        scale = max(1.0, np.abs(ref.evals).max())
        np.testing.assert_allclose(r.evals, ref.evals, rtol=0, atol=1e-10 * scale)


def test_autotune_keeps_results(arb, ctx):
    # the tuner only changes how the SpMM is laid out on the GPU: every candidate sums each
    # row in CSR order, so a filter gives the same block after tuning
    A = I.chung_lu_laplacian(6000, seed=5)[0]
    mat = arb.Matrix.from_csr(ctx, A)
    X = torch.from_numpy(I.gaussian_block(A.n, 48, 2).astype(np.float32)).cuda()
    coef = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, 6)
    before = arb.arb_filter_f32(ctx, mat, -1.0, 2.0, 0.0, 1.9, coef, X).cpu().numpy()
    choice = arb.arb_matrix_autotune(ctx, mat, 48)
    assert choice["sell_C"] in (0, 8, 32) and choice["vec"] in (1, 2, 4) and choice["ms"] > 0
    assert mat.sell_info()[0] == choice["sell_C"]
    after = arb.arb_filter_f32(ctx, mat, -1.0, 2.0, 0.0, 1.9, coef, X).cpu().numpy()
    np.testing.assert_array_equal(after, before)
