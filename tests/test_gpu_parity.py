"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances (FP64 throughout): a fused step reorders the sums of the oracle only within a
row (at most 7 nonzeros here) and across Clenshaw steps, so filter outputs agree to a few
ulps of the largest intermediate; 1e-12 relative to max|Y| is the bar.  Gram products
reduce over n rows in a different order: 1e-13 relative to ||X|| ||Y||.  Eigenvalues of
the dense Jacobi solver: 1e-13 relative to ||H||.  End-to-end eigenvalues: 1e-10 relative
to max(1, |lambda|), the target the method is run to; residuals <= tol.
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def scipy_of(A):
    return O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)


# ------------------------------------------------------------------ SpMM and filter
@pytest.mark.parametrize("ncols", [1, 2, 7, 30, 33, 64, 65, 130])
def test_spmm_matches_oracle(arb, ctx, ncols):
    A = I.laplacian_2d(37)  # n = 1369: not a multiple of any tile
    mat = arb.Matrix.from_csr(ctx, A)
    X = I.gaussian_block(A.n, ncols, 11)
    B = -1.0 * scipy_of(A) + 8.0 * sp.identity(A.n)
    Y = host(arb.arb_spmm(ctx, mat, -1.0, 8.0, dev(X)))
    ref = B @ X
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_spmm_strided_views(arb, ctx):
    A = I.laplacian_3d(9)
    mat = arb.Matrix.from_csr(ctx, A)
    big = dev(I.gaussian_block(A.n, 50, 3))
    X = big[:, 3:40]  # odd offset, leading dimension 50
    Yb = torch.zeros((A.n, 41), dtype=torch.float64, device="cuda")
    arb.arb_spmm(ctx, mat, 1.0, 0.0, X, Yb[:, 1:38])
    ref = scipy_of(A) @ host(big)[:, 3:40]
    np.testing.assert_allclose(host(Yb)[:, 1:38], ref, atol=1e-13 * np.abs(ref).max())
    assert np.all(host(Yb)[:, 0] == 0) and np.all(host(Yb)[:, 38:] == 0)


@pytest.mark.parametrize("d", [1, 2, 3, 10, 20])
@pytest.mark.parametrize("kind", [0, 1])
def test_filter_matches_oracle(arb, ctx, d, kind):
    A = I.laplacian_2d(40)
    mat = arb.Matrix.from_csr(ctx, A)
    B = 8.0 * sp.identity(A.n, format="csr") - scipy_of(A)
    ncols = 30
    X = I.gaussian_block(A.n, ncols, 5)
    xs = np.linspace(0.5, 2.0, ncols)
    a, b = 0.0, 3.7
    coef = O.interpolant_cheb_coeffs(d) if kind == 0 else O.chebyshev_T_coeffs(d)
    colss = torch.zeros(ncols, dtype=torch.float64, device="cuda")
    Y = host(arb.arb_filter(ctx, mat, -1.0, 8.0, a, b, arb.arb_filter_coefficients(kind, d), dev(X),
                            xscale=dev(xs), colss=colss))
    Bs = B - a * sp.identity(A.n, format="csr")
    ref = O.poly_clenshaw(Bs, X * xs[None, :], 0.0, b - a, coef)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(host(colss), np.sum(ref * ref, axis=0), rtol=1e-11)
    if d <= 10:  # Algorithm 7 as printed (monomial Horner) agrees at moderate degree
        ref7 = O.poly_alg7(Bs, X * xs[None, :], 0.0, b - a, O.cheb_to_monomial(coef))
        np.testing.assert_allclose(Y, ref7, rtol=0, atol=1e-9 * scale)


@pytest.mark.parametrize("d,ncols", [(1, 7), (3, 30), (10, 64), (20, 130), (5, 128), (20, 240)])
def test_filter_f32_against_oracle(arb, ctx, d, ncols):
    # FP32 filter of the mixed path vs the FP64 oracle.  Each Clenshaw pass adds a few
    # u32 of relative rounding, growing roughly linearly in d: an FP32 emulation of the same
    # recurrence in numpy measures 1.2e-7 (d=1) .. 1.3e-6 (d=20) of max|Y| on these
    # inputs, so 1e-5 of max|Y| is the bar.
    A = I.laplacian_2d(40)
    mat = arb.Matrix.from_csr(ctx, A)
    B = 8.0 * sp.identity(A.n, format="csr") - scipy_of(A)
    X = I.gaussian_block(A.n, ncols, 5)
    xs = np.linspace(0.5, 2.0, ncols)
    a, b = 0.0, 3.7
    coef = O.interpolant_cheb_coeffs(d)
    colss = torch.zeros(ncols, dtype=torch.float64, device="cuda")
    X32 = dev(X).float()
    Y = host(arb.arb_filter_f32(ctx, mat, -1.0, 8.0, a, b, coef, X32, xscale=dev(xs), colss=colss))
    ref = O.poly_clenshaw(B, X.astype(np.float32).astype(np.float64) * xs[None, :], 0.0, b, coef)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-5 * scale)
    np.testing.assert_allclose(host(colss), np.sum(ref * ref, axis=0), rtol=1e-4)


@pytest.mark.parametrize("d,ncols,diffusion", [(1, 7, False), (3, 30, False), (10, 64, True), (20, 131, False),
                                                (20, 240, False), (15, 33, True)])
def test_filter_df_against_oracle(arb, ctx, d, ncols, diffusion):
    # double-float filter vs the FP64 oracle.  Each double-float product or sum is good to
    # about 2^-46 of its operands; the FP32 filter's error grows to ~22 u32 of max|Y| at
    # d = 20 on these inputs, the same growth at 2^-46 is ~3e-13, so 1e-11 of max|Y| is the
    # bar (odd widths exercise the pad column; the diffusion matrix has non-integer values
    # that do not fit one FP32 number).
    A = I.diffusion_2d(40, 3) if diffusion else I.laplacian_2d(40)
    mat = arb.Matrix.from_csr(ctx, A)
    B = scipy_of(A)
    sigma = O.gershgorin_bounds(B)[1]
    Bs = sigma * sp.identity(A.n, format="csr") - B
    X = I.gaussian_block(A.n, ncols, 5)
    xs = np.linspace(0.5, 2.0, ncols)
    a, b = 0.0, 0.45 * sigma
    coef = O.interpolant_cheb_coeffs(d)
    colss = torch.zeros(ncols, dtype=torch.float64, device="cuda")
    Y = host(arb.arb_filter_df(ctx, mat, -1.0, sigma, a, b, coef, dev(X), xscale=dev(xs), colss=colss))
    ref = O.poly_clenshaw(Bs, X * xs[None, :], 0.0, b, coef)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(host(colss), np.sum(ref * ref, axis=0), rtol=1e-10)
    # and far below the FP32 filter's error on the same inputs
    Y32 = host(arb.arb_filter_f32(ctx, mat, -1.0, sigma, a, b, coef, dev(X).float(), xscale=dev(xs)))
    ref32 = O.poly_clenshaw(Bs, X.astype(np.float32).astype(np.float64) * xs[None, :], 0.0, b, coef)
    assert np.abs(Y - ref).max() * 1e3 < max(np.abs(Y32 - ref32).max(), 1e-300)


def test_filter_on_closed_form_eigenvectors(arb, ctx):
    # spectral mapping (eq. poly-A): rho(A) v = rho(lambda) v for the sin-product eigenvectors
    m = 20
    A = I.laplacian_3d(m)
    mat = arb.Matrix.from_csr(ctx, A)
    x = np.arange(1, m + 1)
    modes = [(1, 1, 1), (2, 1, 1), (3, 2, 1), (5, 5, 5), (20, 1, 7)]
    cols, lams = [], []
    for (i, j, l) in modes:
        v = np.einsum("a,b,c->cba", np.sin(np.pi * i * x / (m + 1)), np.sin(np.pi * j * x / (m + 1)),
                      np.sin(np.pi * l * x / (m + 1))).ravel()
        cols.append(v / np.linalg.norm(v))
        lams.append(6 - 2 * np.cos(np.pi * i / (m + 1)) - 2 * np.cos(np.pi * j / (m + 1))
                    - 2 * np.cos(np.pi * l / (m + 1)))
    V = np.stack(cols, axis=1)
    np.testing.assert_allclose(scipy_of(A) @ V, V * np.array(lams)[None, :], atol=1e-12)
    coef = O.interpolant_cheb_coeffs(20)
    a, b = 0.0, 11.5
    Y = host(arb.arb_filter(ctx, mat, -1.0, 12.0, a, b, coef, dev(V)))
    rho = O.rho_d(coef, 12.0 - np.array(lams), a, b)
    np.testing.assert_allclose(Y, V * rho[None, :], atol=1e-12 * np.abs(rho).max())


# ------------------------------------------------------------------ dense kernels
@pytest.mark.parametrize("n,na,nb", [(1, 1, 1), (17, 3, 5), (1000, 30, 30), (4099, 65, 130), (20000, 64, 64)])
def test_gram_matches_numpy(arb, ctx, n, na, nb):
    X = I.gaussian_block(n, na, 1)
    Y = I.gaussian_block(n, nb, 2)
    C = host(arb.arb_gram(ctx, dev(X), dev(Y)))
    ref = X.T @ Y
    # reordered sums: within 1e-13 ||x_i|| ||y_j|| per entry
    bound = 1e-13 * np.outer(np.linalg.norm(X, axis=0), np.linalg.norm(Y, axis=0))
    assert np.all(np.abs(C - ref) <= bound)
    G = host(arb.arb_gram(ctx, dev(X), dev(X)))  # symmetric path
    bx = 1e-13 * np.outer(np.linalg.norm(X, axis=0), np.linalg.norm(X, axis=0))
    assert np.all(np.abs(G - X.T @ X) <= bx)
    assert np.array_equal(G, G.T)


# leading dimensions that are multiples of 4 take the tensor cores (ragged against the
# 128 x 64 CTA tile and the 32-row steps); the others the CUDA-core kernel
@pytest.mark.parametrize("n,na,nb", [(1, 1, 1), (33, 3, 5), (1000, 32, 36), (4099, 68, 132), (20000, 64, 64),
                                     (100003, 240, 240), (50000, 720, 240), (7, 200, 132), (300, 4, 8)])
def test_gram_f32_tensor_cores(arb, ctx, n, na, nb):
    # split-TF32 tcgen05 products carry ~21 significand bits and are summed in FP32 over
    # 256-row runs, the CUDA-core kernel sums FP32 products over 64-row runs: both within
    # the FP32 bound of a few u32 * sqrt(run) relative to ||x_i|| ||y_j||
    X = I.gaussian_block(n, na, 11).astype(np.float32)
    Y = I.gaussian_block(n, nb, 12).astype(np.float32)
    Xd, Yd = dev(X).float(), dev(Y).float()
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    C = host(arb.arb_gram_f32(ctx, Xd, Yd))
    nx, ny = np.linalg.norm(X64, axis=0), np.linalg.norm(Y64, axis=0)
    err = np.abs(C - X64.T @ Y64) / np.outer(nx, ny)
    assert err.max() <= 1e-6, err.max()
    G = host(arb.arb_gram_f32(ctx, Xd, Xd))  # symmetric path
    assert np.array_equal(G, G.T)
    assert (np.abs(G - X64.T @ X64) / np.outer(nx, nx)).max() <= 1e-6


@pytest.mark.parametrize("n,na,nb,pad", [(1, 8, 4, 0), (300, 7, 5, 0), (1000, 17, 33, 0), (4099, 240, 240, 0),
                                         (20000, 720, 240, 0), (5000, 100, 300, 0), (777, 64, 48, 1),
                                         (2_097_152, 720, 240, 0)])
def test_gemm_tall_f32_matches_numpy(arb, ctx, n, na, nb, pad):
    # leading dimensions rounded up to multiples of 4 take the tensor cores (na >= 8); pad = 1
    # makes them odd (CUDA cores).  Per entry within 1e-6 of sum_k |In_ik| |W_kj| (split TF32,
    # FP32 sums); at full size on 4096 sampled rows
    g = torch.Generator(device="cuda").manual_seed(n + na + nb)
    la, lb = (na + 3) // 4 * 4 + pad, (nb + 3) // 4 * 4 + pad
    In = torch.randn((n, la), dtype=torch.float32, device="cuda", generator=g)[:, :na]
    W = torch.randn((na, nb), dtype=torch.float64, device="cuda", generator=g)
    Out0 = torch.randn((n, lb), dtype=torch.float32, device="cuda", generator=g)[:, :nb]
    rows = torch.arange(n, device="cuda") if n <= 20000 else torch.randint(0, n, (4096,), device="cuda", generator=g)
    Wf = W.float().double()  # W enters as FP32
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
        Out = Out0.clone()
        arb.arb_gemm_tall_f32(ctx, In, W, alpha, beta, Out)
        Is, Os, O0 = In[rows].double(), Out[rows].double(), Out0[rows].double()
        ref = alpha * (Is @ Wf) + beta * O0
        bound = 1e-6 * (Is.abs() @ Wf.abs()) + 1e-7 * O0.abs() + 1e-30
        assert bool(((Os - ref).abs() <= bound).all()), float(((Os - ref).abs() / bound).max())
    if n <= 20000:  # beta = 0 never reads Out
        Out = torch.full((n, lb), float("nan"), dtype=torch.float32, device="cuda")[:, :nb]
        arb.arb_gemm_tall_f32(ctx, In, W, 1.0, 0.0, Out)
        assert bool(torch.isfinite(Out).all())


@pytest.mark.parametrize("m", [1, 2, 3, 10, 31, 64, 65, 96, 97, 200, 256, 720])
def test_syevj_matches_oracle_jacobi(arb, ctx, m):
    rng = np.random.default_rng(m)
    H = rng.standard_normal((m, m))
    H = 0.5 * (H + H.T)
    w, V, sweeps = arb.arb_syevj(ctx, dev(H))
    w, V = host(w), host(V)
    if m <= 65:
        wo, _ = O.jacobi_eigh(H)
        np.testing.assert_allclose(w, wo, atol=1e-13 * np.linalg.norm(H))
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(H))[::-1], atol=1e-13 * np.linalg.norm(H))
    np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-13 * m)
    np.testing.assert_allclose(H @ V, V * w[None, :], atol=1e-12 * np.linalg.norm(H))
    assert sweeps < 60


def test_syevj_clusters_and_zero(arb, ctx):
    w0 = np.array([5.0, 5.0, 5.0, 2.0, 2.0, 1e-9, 0.0, -3.0, -3.0, 7.5, 7.5])
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((11, 11)))
    H = Q @ np.diag(w0) @ Q.T
    w, V, _ = arb.arb_syevj(ctx, dev(H))
    np.testing.assert_allclose(host(w), np.sort(w0)[::-1], atol=1e-13 * 15)
    w, V, s = arb.arb_syevj(ctx, dev(np.zeros((4, 4))))
    assert np.all(host(w) == 0) and s == 0


def test_rcond_matches_oracle(arb, ctx):
    rng = np.random.default_rng(9)
    X = rng.standard_normal((3000, 12)) @ np.diag(np.logspace(0, -3, 12))
    xs = np.linspace(1.0, 3.0, 12)
    rc = arb.arb_rcond_gram(ctx, dev(X), xscale=dev(xs))
    Xs = X * xs[None, :]
    ref = O.rcond_spd(Xs.T @ Xs)
    assert abs(rc - ref) <= 1e-8 * ref
    Xd = np.hstack([X, X[:, :1]])
    assert arb.arb_rcond_gram(ctx, dev(Xd)) < 1e-14


def test_orth_spans_and_rank(arb, ctx):
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((5000, 20))
    Z[:, 15:] = Z[:, :5] @ rng.standard_normal((5, 5))  # rank 15
    U = host(arb.arb_orth(ctx, dev(Z)))
    assert U.shape[1] == 15
    np.testing.assert_allclose(U.T @ U, np.eye(15), atol=1e-13)
    Uo = O.orth(Z)
    assert Uo.shape[1] == 15
    np.testing.assert_allclose(U @ (U.T @ Uo), Uo, atol=1e-11)


def test_rayleigh_ritz_matches_oracle(arb, ctx):
    A = I.laplacian_2d(30)
    mat = arb.Matrix.from_csr(ctx, A)
    B = 8.0 * sp.identity(A.n, format="csr") - scipy_of(A)
    Z = I.gaussian_block(A.n, 24, 3)
    Y, w = arb.arb_rayleigh_ritz(ctx, mat, -1.0, 8.0, dev(Z))
    Yo, wo = O.rayleigh_ritz(B, Z)
    np.testing.assert_allclose(host(w), wo, atol=1e-12 * 8)
    Y = host(Y)
    np.testing.assert_allclose(Y.T @ Y, np.eye(24), atol=1e-12)
    P, Po = Y @ Y.T, Yo @ Yo.T
    assert np.abs(P - Po).max() < 1e-10


@pytest.mark.parametrize("q", [0, 1, 2])
def test_arr_matches_oracle(arb, ctx, q):
    A = I.laplacian_2d(32)
    mat = arb.Matrix.from_csr(ctx, A)
    B = 8.0 * sp.identity(A.n, format="csr") - scipy_of(A)
    X = I.gaussian_block(A.n, 16, 8)
    # a few oracle filter steps so X is the kind of block ARR sees
    coef = O.interpolant_cheb_coeffs(6)
    for _ in range(3):
        X = O.normalize_columns(O.poly_clenshaw(B, X, 0.0, 4.0, coef))
    Y, w, rank = arb.arb_arr(ctx, mat, -1.0, 8.0, dev(X), q)
    Yo, wo = O.arr(B, X, q)
    assert rank == (q + 1) * 16
    np.testing.assert_allclose(host(w), wo, atol=1e-11 * 8)
    Y = host(Y)
    res = O.residual_norms(B, Y, host(w), host(w))
    reso = O.residual_norms(B, Yo, wo, wo)
    np.testing.assert_allclose(res, reso, atol=1e-9)


# ------------------------------------------------------------------ double-float dense products
@pytest.fixture(scope="module")
def ctx_df(arb):
    c = arb.Context(0)
    c.set_dense_df(True)
    yield c
    c.close()


@pytest.mark.parametrize("n,na,nb", [(1, 1, 1), (17, 3, 5), (1000, 30, 30), (4099, 65, 130), (20000, 64, 64),
                                     (100003, 240, 240)])
def test_gram_df_matches_numpy(arb, ctx_df, n, na, nb):
    # operands split into hi + lo FP32 (2^-48 relative), Dot2 sums folded every 64 terms
    # into a double-float running sum: the FP64 kernel's per-entry bound holds
    X = I.gaussian_block(n, na, 1)
    Y = I.gaussian_block(n, nb, 2)
    C = host(arb.arb_gram(ctx_df, dev(X), dev(Y)))
    bound = 1e-13 * np.outer(np.linalg.norm(X, axis=0), np.linalg.norm(Y, axis=0))
    assert np.all(np.abs(C - X.T @ Y) <= bound)
    Xd = dev(X)
    G = host(arb.arb_gram(ctx_df, Xd, Xd))  # one operand: the symmetric path, exactly symmetric
    bx = 1e-13 * np.outer(np.linalg.norm(X, axis=0), np.linalg.norm(X, axis=0))
    assert np.all(np.abs(G - X.T @ X) <= bx)
    assert np.array_equal(G, G.T)


def test_gram_df_extreme_magnitudes(arb, ctx_df):
    # columns scaled over 1e-15 .. 1e15 (within the double-float split's range): relative
    # accuracy per entry is unchanged
    X = I.gaussian_block(5000, 8, 7) * np.logspace(-15, 15, 8)[None, :]
    G = host(arb.arb_gram(ctx_df, dev(X), dev(X)))
    nrm = np.linalg.norm(X, axis=0)
    assert np.all(np.abs(G - X.T @ X) <= 1e-13 * np.outer(nrm, nrm))


@pytest.mark.parametrize("m", [33, 60, 96, 97, 200, 256, 720])
def test_syevj_double_float_matches_numpy(arb, ctx_df, m):
    # orders above 32 on a double-float context: the rotations and block products carry
    # ~2^-48 relative error per step and the sweeps stop at off(H) <= 1e-13 ||H||_F
    rng = np.random.default_rng(1000 + m)
    H = rng.standard_normal((m, m))
    H = 0.5 * (H + H.T)
    nH = np.linalg.norm(H)
    w, V, sweeps = arb.arb_syevj(ctx_df, dev(H))
    w, V = host(w), host(V)
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(H))[::-1], atol=2e-13 * nH)
    np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(H @ V, V * w[None, :], atol=1e-12 * nH)
    assert sweeps < 60


@pytest.mark.parametrize("scale", [2.0 ** 90, 2.0 ** -90, 3.0e-7])
def test_syevj_double_float_graded_and_scaled(arb, ctx_df, scale):
    # a graded spectrum with a cluster, scaled far outside FP32's range: the kernel's exact
    # power-of-two scaling keeps every split entry representable
    m = 150
    rng = np.random.default_rng(77)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    w0 = np.concatenate([np.logspace(0, -12, m - 10), np.full(10, 0.5)]) * scale
    H = (Q * w0[None, :]) @ Q.T
    H = 0.5 * (H + H.T)
    w, V, sweeps = arb.arb_syevj(ctx_df, dev(H))
    w, V = host(w), host(V)
    nH = np.linalg.norm(H)
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(H))[::-1], atol=2e-13 * nH)
    np.testing.assert_allclose(V.T @ V, np.eye(m), atol=1e-12)
    np.testing.assert_allclose(H @ V, V * w[None, :], atol=1e-12 * nH)
    assert sweeps < 60


def test_orth_rr_arr_in_double_float_mode(arb, ctx_df):
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((5000, 20))
    Z[:, 15:] = Z[:, :5] @ rng.standard_normal((5, 5))  # rank 15
    U = host(arb.arb_orth(ctx_df, dev(Z)))
    assert U.shape[1] == 15
    np.testing.assert_allclose(U.T @ U, np.eye(15), atol=1e-12)
    Uo = O.orth(Z)
    np.testing.assert_allclose(U @ (U.T @ Uo), Uo, atol=1e-11)
    A = I.laplacian_2d(32)
    mat = arb.Matrix.from_csr(ctx_df, A)
    B = 8.0 * sp.identity(A.n, format="csr") - scipy_of(A)
    Z = I.gaussian_block(A.n, 24, 3)
    Y, w = arb.arb_rayleigh_ritz(ctx_df, mat, -1.0, 8.0, dev(Z))
    Yo, wo = O.rayleigh_ritz(B, Z)
    np.testing.assert_allclose(host(w), wo, atol=1e-12 * 8)
    np.testing.assert_allclose(host(Y).T @ host(Y), np.eye(24), atol=1e-12)
    X = I.gaussian_block(A.n, 16, 8)
    coef = O.interpolant_cheb_coeffs(6)
    for _ in range(3):
        X = O.normalize_columns(O.poly_clenshaw(B, X, 0.0, 4.0, coef))
    Y, w, rank = arb.arb_arr(ctx_df, mat, -1.0, 8.0, dev(X), 2)
    Yo, wo = O.arr(B, X, 2)
    assert rank == 48
    np.testing.assert_allclose(host(w), wo, atol=1e-11 * 8)
    np.testing.assert_allclose(O.residual_norms(B, host(Y), host(w), host(w)), O.residual_norms(B, Yo, wo, wo),
                               atol=1e-9)


def test_solve_fp64_with_double_float_dense_products(arb, ctx_df):
    # the whole FP64 method with every Gram / tall-skinny product in double-float
    W = I.workload_2d64()
    X0 = I.gaussian_block(W.A.n, W.p, W.seed)
    r = _solve(arb, ctx_df, W.A, W.k, W.p, W.q, W.degree, W.tol, X0)
    assert r.status == arb.ARB_OK, r.info
    lam = np.array(json_golden()["evals"])
    assert np.max(np.abs(r.evals - lam) / np.maximum(1.0, np.abs(lam))) <= 1e-10
    Q = r.evecs
    np.testing.assert_allclose(Q.T @ Q, np.eye(W.k), atol=1e-12)
    assert np.linalg.norm(scipy_of(W.A) @ Q - Q * r.evals[None, :], axis=0).max() <= W.tol * 8.0


# ------------------------------------------------------------------ whole method
def _solve(arb, ctx, A, k, p, q, d, tol, X0, which=1, **kw):
    mat = arb.Matrix.from_csr(ctx, A)
    o = arb.arb_options_default(k)
    o.p, o.q, o.degree = p, q, d
    for key, v in kw.items():
        setattr(o, key, v)
    return arb.arb_solve(ctx, mat, k, which, tol, o, x0=X0, evecs="host")


def _projector_distance(Q1, Q2):
    return np.abs(Q1 @ Q1.T - Q2 @ Q2.T).max()


def test_solve_2d64_against_oracle_and_closed_form(arb, ctx):
    W = I.workload_2d64()
    X0 = I.gaussian_block(W.A.n, W.p, W.seed)
    r = _solve(arb, ctx, W.A, W.k, W.p, W.q, W.degree, W.tol, X0)
    assert r.status == arb.ARB_OK, r.info
    ref = O.arrabit_mpm(scipy_of(W.A), W.k, X0, which="smallest", tol=W.tol, q=W.q, degree=W.degree)
    lam = laplacian_2d_eigs(64)[:W.k]
    denom = np.maximum(1.0, np.abs(lam))
    assert np.max(np.abs(r.evals - ref.evals) / denom) <= 1e-10
    assert np.max(np.abs(r.evals - lam) / denom) <= 1e-10
    Q = r.evecs
    A = scipy_of(W.A)
    np.testing.assert_allclose(Q.T @ Q, np.eye(W.k), atol=1e-12)
    R = A @ Q - Q * r.evals[None, :]
    assert np.linalg.norm(R, axis=0).max() <= W.tol * 8.0
    # the first 20 eigenvalues end on a complete cluster: compare spectral projectors
    assert _projector_distance(Q, ref.evecs) < 1e-8
    assert r.info["maxres"] <= W.tol


@pytest.mark.parametrize("which", [0, 1])
def test_solve_bruteforce_random_sparse(arb, ctx, which):
    from paper_1507_06078_gb300.inputs import CSR
    n, k, p = 400, 8, 12
    rng = np.random.default_rng(77)
    M = sp.random(n, n, density=0.02, random_state=rng, format="csr")
    M = (M + M.T + sp.diags(rng.uniform(0, 3, n))).tocsr()
    M.sort_indices()
    A = CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    X0 = I.gaussian_block(n, p, 31)
    r = _solve(arb, ctx, A, k, p, 1, 10, 1e-10, X0, which=which)
    wref = np.linalg.eigvalsh(M.toarray())
    want = wref[:k] if which == 1 else wref[::-1][:k]
    np.testing.assert_allclose(r.evals, want, atol=1e-9 * np.abs(wref).max())


@pytest.mark.parametrize("precision", [0, 2])
def test_solve_chung_lu_scaled(arb, ctx, precision):
    # the power-law graph Laplacian family of the Chung-Lu workload, scaled down: rows from
    # 2 to hundreds of nonzeros (the general, non-short-row SpMM), FP32-rounded values;
    # k smallest against LAPACK
    A, _ = I.chung_lu_laplacian(3000, seed=11)
    k, p = 20, 30
    X0 = I.gaussian_block(A.n, p, 5)
    r = _solve(arb, ctx, A, k, p, 1, 15, 1e-8, X0, precision=precision)
    assert r.status == arb.ARB_OK, r.info
    lam = np.linalg.eigvalsh(A.to_dense())[:k]
    np.testing.assert_allclose(r.evals, lam, atol=1e-9)
    Q = r.evecs
    R = scipy_of(A) @ Q - Q * r.evals[None, :]
    assert np.linalg.norm(R, axis=0).max() <= 1e-8 * 8.0


@pytest.mark.parametrize("which", ["chung_lu", "laplace3d"])
def test_sell_spmm_and_filters_match_csr(arb, ctx, which):
    # SELL-C-sigma (C = 32, sigma = 1024) walks the rows in sorted order but sums each row's
    # nonzeros in CSR order: SpMM and all three filter arithmetics are bitwise equal to the
    # CSR kernels (power-law rows of 2 to hundreds of nonzeros; 7-point stencil rows)
    if which == "chung_lu":
        A, _ = I.chung_lu_laplacian(20000, seed=3)
        shift, b = 2.0, 1.9
    else:
        A = I.laplacian_3d(24)
        shift, b = 12.0, 11.9
    m_csr = arb.Matrix.from_csr(ctx, A)
    m_sell = arb.Matrix.from_csr(ctx, A)
    m_sell.set_sell(32, 1024)
    c, sg, slots = m_sell.sell_info()
    assert (c, sg) == (32, 1024) and A.nnz <= slots < 2 * A.nnz + 32 * 1024
    X = dev(I.gaussian_block(A.n, 40, 7))
    y_csr = host(arb.arb_spmm(ctx, m_csr, 1.0, 0.0, X))
    y_sell = host(arb.arb_spmm(ctx, m_sell, 1.0, 0.0, X))
    np.testing.assert_array_equal(y_sell, y_csr)
    Xh = host(X)
    ref = scipy_of(A) @ Xh
    np.testing.assert_allclose(y_sell, ref, atol=1e-13 * (abs(scipy_of(A)) @ abs(Xh)).max())
    coef = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, 8)
    for f, Xin in ((arb.arb_filter, X), (arb.arb_filter_f32, X.float()), (arb.arb_filter_df, X)):
        a = host(f(ctx, m_csr, -1.0, shift, 0.0, b, coef, Xin))
        s_ = host(f(ctx, m_sell, -1.0, shift, 0.0, b, coef, Xin))
        np.testing.assert_array_equal(s_, a)
    m_sell.set_sell(0, 0)
    assert m_sell.sell_info() == (0, 0, 0)
    np.testing.assert_array_equal(host(arb.arb_spmm(ctx, m_sell, 1.0, 0.0, X)), y_csr)


@pytest.mark.parametrize("precision", [0, 2])
def test_solve_chung_lu_sell(arb, ctx, precision):
    # the scaled Chung-Lu solve on the SELL-C-sigma copy: k smallest against LAPACK
    A, _ = I.chung_lu_laplacian(3000, seed=11)
    k, p = 20, 30
    X0 = I.gaussian_block(A.n, p, 5)
    mat = arb.Matrix.from_csr(ctx, A)
    mat.set_sell(32, 256)
    o = arb.arb_options_default(k)
    o.p, o.q, o.degree, o.precision = p, 1, 15, precision
    r = arb.arb_solve(ctx, mat, k, 1, 1e-8, o, x0=X0, evecs="host")
    assert r.status == arb.ARB_OK, r.info
    lam = np.linalg.eigvalsh(A.to_dense())[:k]
    np.testing.assert_allclose(r.evals, lam, atol=1e-9)
    R = scipy_of(A) @ r.evecs - r.evecs * r.evals[None, :]
    assert np.linalg.norm(R, axis=0).max() <= 1e-8 * 8.0


@pytest.fixture(scope="module")
def chung_lu_125k():
    return I.chung_lu_laplacian(125000, seed=4242)[0]


def test_solve_chung_lu_125k_keeps_small_directions(arb, ctx, chung_lu_125k):
    # 1/8 of the C2 scale, k = 50: the first filter leaves the block's singular values
    # spread far beyond what a Gram pass resolves (the near-zero eigenvalue dominates);
    # orth must recover the truncated directions or the basis collapses to rank ~2 and the
    # solve stalls at maxres 0.25 (the oracle, with pivoted QR, converges in 4 outer
    # iterations).  Checked by properties: residuals within the near-tolerance stop rule's
    # bound, orthogonality, and the smallest eigenvalue near 0 (the connected graph's
    # Laplacian has an exact 0, which the FP32 rounding of the values perturbs by ~u32)
    A = chung_lu_125k
    k, p = 50, 60
    mat = arb.Matrix.from_csr(ctx, A)
    o = arb.arb_options_default(k)
    o.p, o.q, o.degree = p, 1, 15
    r = arb.arb_solve(ctx, mat, k, 1, 1e-8, o, x0=I.gaussian_block(A.n, p, 5), evecs="host")
    assert r.status == arb.ARB_OK, r.info
    Q, lam = r.evecs, r.evals
    assert abs(lam[0]) <= 1e-7 and np.all(np.diff(lam) >= -1e-12)
    R = scipy_of(A) @ Q - Q * lam[None, :]
    assert np.linalg.norm(R, axis=0).max() <= 1e-8 * 10.0
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-10)


def test_matrix_from_fp32_values(arb, ctx):
    # FP32 values widened on the device give the same matrix (and solve) as the FP64 upload
    # of the same numbers; device-pointer uploads record the longest row too
    A, _ = I.chung_lu_laplacian(1200, seed=2)  # values are FP32 numbers already
    m64 = arb.Matrix.from_csr(ctx, A)
    m32 = arb.Matrix(ctx, A.n, A.rowptr, A.col, A.val.astype(np.float32))
    X = dev(I.gaussian_block(A.n, 8, 3))
    np.testing.assert_array_equal(host(arb.arb_spmm(ctx, m32, 1.0, 0.0, X)), host(arb.arb_spmm(ctx, m64, 1.0, 0.0, X)))
    o = arb.arb_options_default(6)
    o.p, o.q, o.degree = 10, 1, 10
    r32 = arb.arb_solve(ctx, m32, 6, 1, 1e-9, o, x0=I.gaussian_block(A.n, 10, 4))
    r64 = arb.arb_solve(ctx, m64, 6, 1, 1e-9, o, x0=I.gaussian_block(A.n, 10, 4))
    np.testing.assert_array_equal(r32.evals, r64.evals)


def test_solve_lockstep_fixed_schedule(arb, ctx):
    A = I.laplacian_2d(16)
    X0 = I.gaussian_block(A.n, 12, 10)
    r = _solve(arb, ctx, A, 10, 12, 1, 6, 1e-9, X0, inner_fixed=4, maxit=20)
    ref = O.arrabit_mpm(scipy_of(A), 10, X0, which="smallest", tol=1e-9, q=1, degree=6, inner_fixed=4,
                        maxit=20)
    assert r.info["n_filters"] == 4 * r.info["outer_iters"]
    np.testing.assert_allclose(r.evals, ref.evals, atol=1e-9)
    np.testing.assert_allclose(r.evals, laplacian_2d_eigs(16)[:10], atol=1e-9)


def test_solve_3d_scaled(arb, ctx):
    m, k, p = 24, 30, 36
    A = I.laplacian_3d(m)
    X0 = I.gaussian_block(A.n, p, 99)
    r = _solve(arb, ctx, A, k, p, 2, 12, 1e-8, X0)
    assert r.status == arb.ARB_OK, r.info
    lam = laplacian_3d_eigs(m)[:k]
    np.testing.assert_allclose(r.evals, lam, atol=1e-9)


def test_solve_rejects_bad_arguments(arb, ctx):
    A = I.laplacian_2d(8)
    X0 = I.gaussian_block(A.n, 12, 1)
    with pytest.raises(arb.ArbError) as e:
        _solve(arb, ctx, A, 20, 12, 1, 5, 1e-8, X0)  # k > p
    assert e.value.status == arb.ARB_INVALID_ARG
    with pytest.raises(arb.ArbError):
        _solve(arb, ctx, A, 10, 12, 5, 5, 1e-8, X0)  # (q+1) p >= n
    with pytest.raises(arb.ArbError):
        _solve(arb, ctx, A, 10, 12, 1, 0, 1e-8, X0)  # degree 0
    with pytest.raises(arb.ArbError):
        arb.Matrix(ctx, 4, np.array([0, 1, 2, 3, 5]), np.array([0, 1, 2, 3, 9]), np.ones(5))


def test_device_start_block_matches_host_generator(arb, ctx):
    # x0 = NULL draws X0 on the device from the same Philox stream as the input generator
    A = I.laplacian_2d(20)
    k, p = 8, 10
    o = arb.arb_options_default(k)
    o.p, o.q, o.degree, o.seed = p, 1, 8, 4242
    mat = arb.Matrix.from_csr(ctx, A)
    r_dev = arb.arb_solve(ctx, mat, k, 1, 1e-10, o, x0=None)
    r_host = arb.arb_solve(ctx, mat, k, 1, 1e-10, o, x0=I.gaussian_block(A.n, p, 4242))
    # the two start blocks differ in the last bits of log/cos, which can move an inner
    # stop decision; the converged pairs agree all the same
    np.testing.assert_allclose(r_dev.evals, r_host.evals, atol=1e-10)


@pytest.mark.parametrize("n,ncols", [(1, 1), (7, 3), (1000, 30), (333, 17)])
def test_gaussian_block_matches_input_generator(arb, ctx, n, ncols):
    Xd = host(arb.arb_gaussian_block(ctx, n, ncols, 987654321987))
    Xh = I.gaussian_block(n, ncols, 987654321987)
    # same counters and uniforms; the host rounds 2*pi*u before cos/sin while the device
    # uses sincospi(2u), so values near a zero of cos/sin differ by ~eps * |r| absolutely
    np.testing.assert_allclose(Xd, Xh, rtol=1e-14, atol=1e-14)


def test_solve_mixed_2d64_against_oracle(arb, ctx):
    # FP32 phase + FP64 refinement must land on the FP64 oracle's pairs (spec bar:
    # eigenvalue relative error <= 1e-10, relative residual <= tol)
    W = I.workload_2d64()
    X0 = I.gaussian_block(W.A.n, W.p, W.seed)
    r = _solve(arb, ctx, W.A, W.k, W.p, W.q, W.degree, W.tol, X0, precision=arb.ARB_MIXED)
    assert r.status == arb.ARB_OK, r.info
    ref = json_golden()
    lam = np.array(ref["evals"])
    assert np.max(np.abs(r.evals - lam) / np.maximum(1.0, np.abs(lam))) <= 1e-10
    Q = r.evecs
    R = scipy_of(W.A) @ Q - Q * r.evals[None, :]
    assert np.linalg.norm(R, axis=0).max() <= W.tol * 8.0
    np.testing.assert_allclose(Q.T @ Q, np.eye(W.k), atol=1e-12)
    assert r.info["outer_iters_fp32"] >= 1


def test_solve_mixed_df_2d64_against_oracle(arb, ctx):
    # FP32 phase + refinement with the double-float filter: the same bar as the FP64 path
    W = I.workload_2d64()
    X0 = I.gaussian_block(W.A.n, W.p, W.seed)
    r = _solve(arb, ctx, W.A, W.k, W.p, W.q, W.degree, W.tol, X0, precision=arb.ARB_MIXED_DF)
    assert r.status == arb.ARB_OK, r.info
    lam = np.array(json_golden()["evals"])
    assert np.max(np.abs(r.evals - lam) / np.maximum(1.0, np.abs(lam))) <= 1e-10
    Q = r.evecs
    R = scipy_of(W.A) @ Q - Q * r.evals[None, :]
    assert np.linalg.norm(R, axis=0).max() <= W.tol * 8.0
    np.testing.assert_allclose(Q.T @ Q, np.eye(W.k), atol=1e-12)
    assert r.info["maxres"] <= W.tol


@pytest.mark.parametrize("precision", [1, 2])
def test_solve_mixed_3d_scaled(arb, ctx, precision):
    m, k, p = 24, 30, 36
    A = I.laplacian_3d(m)
    X0 = I.gaussian_block(A.n, p, 99)
    r = _solve(arb, ctx, A, k, p, 2, 12, 1e-8, X0, precision=precision)
    assert r.status == arb.ARB_OK, r.info
    np.testing.assert_allclose(r.evals, laplacian_3d_eigs(m)[:k], atol=1e-9)


def json_golden():
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "laplace2d_64_oracle.json")
    return json.load(open(here))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_solve_b_every_arr_against_oracle(arb, ctx, precision):
    A = I.laplacian_3d(12)
    X0 = I.gaussian_block(A.n, 24, 12)
    r = _solve(arb, ctx, A, 20, 24, 2, 10, 1e-8, X0, b_update=1, precision=precision)
    ref = O.arrabit_mpm(scipy_of(A), 20, X0, which="smallest", tol=1e-8, q=2, degree=10, b_update="every_arr")
    assert r.status == arb.ARB_OK, r.info
    np.testing.assert_allclose(r.evals, ref.evals, atol=1e-9)
    np.testing.assert_allclose(r.evals, laplacian_3d_eigs(12)[:20], atol=1e-9)


def test_filter_batched_padded_rows(arb, ctx):
    # blocks whose leading dimension is a multiple of the 16-byte vector but whose width is
    # not: the batched kernel reads whole vectors inside the leading dimension (never past
    # the block's last row) and writes only the block's columns
    specs = [(I.diffusion_2d(30, 5), 13, 6, True), (I.laplacian_3d(9), 30, 12, True), (I.laplacian_2d(17), 7, 5, True),
             (I.diffusion_2d(21, 6), 7, 4, False), (I.laplacian_2d(19), 65, 7, False)]
    jobs, singles, pads = [], [], []
    for i, (A, ncols, d, f32) in enumerate(specs):
        mat = arb.Matrix.from_csr(ctx, A)
        sigma = O.gershgorin_bounds(O.csr_to_scipy(A.n, A.rowptr, A.col, A.val))[1]
        ld = (ncols + 3) // 4 * 4 + 4
        dt = torch.float32 if f32 else torch.float64
        Xf = torch.full((A.n, ld), 3.0, dtype=dt, device="cuda")
        Xf[:, :ncols] = dev(I.gaussian_block(A.n, ncols, 70 + i)).to(dt)
        Yf = torch.full((A.n, ld), 7.0, dtype=dt, device="cuda")
        coef = O.interpolant_cheb_coeffs(d)
        colss = torch.zeros(ncols, dtype=torch.float64, device="cuda")
        jobs.append(dict(mat=mat, op_scale=-1.0, op_shift=sigma, a=0.0, b=0.6 * sigma, coef=coef, X=Xf[:, :ncols],
                         Y=Yf[:, :ncols], colss=colss))
        Xc = Xf[:, :ncols].contiguous()
        singles.append(host((arb.arb_filter_f32 if f32 else arb.arb_filter)(ctx, mat, -1.0, sigma, 0.0, 0.6 * sigma,
                                                                          coef, Xc)))
        pads.append((Yf, ncols))
    arb.arb_filter_batched(ctx, jobs)
    for single, (Yf, ncols), job in zip(singles, pads, jobs):
        Yh = host(Yf)
        np.testing.assert_array_equal(Yh[:, :ncols], single)
        assert np.all(Yh[:, ncols:] == 7.0)  # the padding is never written
        np.testing.assert_allclose(host(job["colss"]), np.sum(single.astype(np.float64) ** 2, axis=0), rtol=1e-10)


def test_filter_batched_matches_single_instance_filters(arb, ctx):
    # uneven instances (sizes, widths, degrees, both precisions) in one persistent launch,
    # each compared with its own single-instance filter and with the oracle
    specs = [(I.diffusion_2d(40, 1), 12, 10, True), (I.laplacian_3d(14), 30, 20, True),
             (I.laplacian_2d(33), 7, 3, False), (I.diffusion_2d(25, 2), 65, 8, False),
             (I.laplacian_2d(20), 130, 1, True), (I.diffusion_2d(60, 3), 96, 15, True)]
    jobs, refs = [], []
    for i, (A, ncols, d, f32) in enumerate(specs):
        mat = arb.Matrix.from_csr(ctx, A)
        B = O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)
        sigma = O.gershgorin_bounds(B)[1]
        X = I.gaussian_block(A.n, ncols, 40 + i)
        xs = np.linspace(0.5, 1.5, ncols)
        coef = O.interpolant_cheb_coeffs(d)
        Xd = dev(X).float() if f32 else dev(X)
        colss = torch.zeros(ncols, dtype=torch.float64, device="cuda")
        jobs.append(dict(mat=mat, op_scale=-1.0, op_shift=sigma, a=0.0, b=0.6 * sigma, coef=coef, X=Xd,
                         xscale=dev(xs), colss=colss))
        single = (arb.arb_filter_f32 if f32 else arb.arb_filter)(ctx, mat, -1.0, sigma, 0.0, 0.6 * sigma, coef, Xd,
                                                                 xscale=dev(xs))
        Bs = sigma * sp.identity(A.n, format="csr") - B
        Xin = (X.astype(np.float32).astype(np.float64) if f32 else X) * xs[None, :]
        ref = O.poly_clenshaw(Bs, Xin, 0.0, 0.6 * sigma, coef)
        refs.append((host(single), ref, f32))
    outs = arb.arb_filter_batched(ctx, jobs)
    for (single, ref, f32), Y, job in zip(refs, outs, jobs):
        Yh = host(Y)
        np.testing.assert_array_equal(Yh, single)  # same arithmetic as the single-instance kernel
        scale = np.abs(ref).max()
        np.testing.assert_allclose(Yh, ref, rtol=0, atol=(1e-5 if f32 else 1e-12) * scale)
        np.testing.assert_allclose(host(job["colss"]), np.sum(Yh.astype(np.float64) ** 2, axis=0), rtol=1e-10)
