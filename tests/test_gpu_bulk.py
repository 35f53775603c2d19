"""The bulk-copy pipelined FP32 SpMM (rows of at most 32 nonzeros, 16-byte aligned rows,
ncols a multiple of 4) against the register-staged kernel, which takes the same blocks
when they are not 16-byte aligned: both form every output with the same FP32 operations
in the same order, so the filter results must be bitwise equal; and both against the
FP64 oracle filter at the FP32 tolerance."""
import numpy as np
import pytest

from oracle import arrabit_oracle as O
from paper_1507_06078_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    from paper_1507_06078_gb300 import arrabit, build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = arrabit.Context(0)
    yield arrabit, ctx
    ctx.close()


@pytest.mark.parametrize("grid,ncols,d", [(24, 240, 20), (17, 64, 3), (9, 8, 1), (30, 1024, 4), (5, 4, 2)])
def test_bulk_filter_bitwise_equals_register_kernel(env, grid, ncols, d):
    arb, ctx = env
    A = I.laplacian_3d(grid)  # n not a multiple of the 4-row groups for 17, 9, 5
    mat = arb.Matrix.from_csr(ctx, A)
    Xh = I.gaussian_block(A.n, ncols, 3).astype(np.float32)
    X = torch.from_numpy(Xh).cuda()
    coef = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, d)
    xs = torch.from_numpy(np.linspace(0.5, 1.5, ncols)).cuda()
    ss_a = torch.zeros(ncols, dtype=torch.float64, device="cuda")
    Ya = arb.arb_filter_f32(ctx, mat, -1.0, 12.0, 0.0, 11.5, coef, X, xscale=xs, colss=ss_a)
    # the same numbers in blocks shifted by one float: no 16-byte alignment, register kernel
    big = torch.zeros((A.n, ncols + 4), dtype=torch.float32, device="cuda")
    Xm = big[:, 1:ncols + 1]
    Xm.copy_(X)
    outb = torch.zeros((A.n, ncols + 4), dtype=torch.float32, device="cuda")
    Ym = outb[:, 1:ncols + 1]
    ss_b = torch.zeros(ncols, dtype=torch.float64, device="cuda")
    arb.arb_filter_f32(ctx, mat, -1.0, 12.0, 0.0, 11.5, coef, Xm, xscale=xs, Y=Ym, colss=ss_b)
    torch.cuda.synchronize()
    assert torch.equal(Ya, Ym)
    # column sums of squares: same terms summed in another order
    torch.testing.assert_close(ss_a, ss_b, rtol=1e-12, atol=0)
    # and the FP64 oracle at the FP32 tolerance of the filter tests
    B = 12.0 * O.sp.identity(A.n) - O.csr_to_scipy(A.n, A.rowptr, A.col, A.val)
    ref = O.poly_clenshaw(B.tocsr(), Xh.astype(np.float64) * np.linspace(0.5, 1.5, ncols)[None, :], 0.0, 11.5,
                          coef)
    np.testing.assert_allclose(Ya.cpu().numpy(), ref, rtol=0, atol=1e-5 * np.abs(ref).max())
