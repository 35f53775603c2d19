"""arb_gram_noalloc: the Gram product for callers that cannot let a library allocate
device memory (applications whose device memory belongs to their own pool allocator, and
latency-bound loops that must not meet cudaMalloc's implicit synchronisation).  Its
partial sums live in the library's static device scratch.  It must give the host product
X^T Y and arb_gram's result, also on a second call that reuses the scratch, allocate no
device memory, and refuse shapes that do not fit.  Collected last so a stop-at-first-
failure run has already run every other test."""
import numpy as np
import pytest

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


def _blk(n, m, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.randn((n, m), dtype=torch.float64, device="cuda", generator=g)


@pytest.mark.parametrize("n,na,nb,same", [(100000, 240, 240, True), (5000, 30, 70, False), (333, 1, 17, False),
                                          (2_000_000, 240, 240, True)])
def test_noalloc_gram_matches_gram_on_two_calls(env, n, na, nb, same):
    arb, ctx = env
    for call in range(2):  # the second call reuses the scratch left by the first
        X = _blk(n, na, 10 * call + 1)
        Y = X if same else _blk(n, nb, 10 * call + 2)
        ref = arb.arb_gram(ctx, X, Y)
        C = torch.full((na, nb), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        arb.arb_gram_noalloc(ctx, X, Y, C)
        torch.cuda.synchronize()
        if call == 1:  # once the library's module is loaded, a call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free0
        # the host product in FP64, and arb_gram's: same products, sums split differently
        # over rows - the Gram tolerance of the parity tests, 1e-13 ||x_i|| ||y_j||
        Xh, Yh = X.cpu().numpy(), Y.cpu().numpy()
        host = Xh.T @ Yh
        bound = 1e-13 * np.outer(np.linalg.norm(Xh, axis=0), np.linalg.norm(Yh, axis=0))
        Ch = C.cpu().numpy()
        assert np.isfinite(Ch).all()
        assert np.all(np.abs(Ch - host) <= bound)
        assert np.all(np.abs(Ch - ref.cpu().numpy()) <= bound)


def test_noalloc_gram_refuses_shapes_beyond_scratch(env):
    arb, ctx = env
    X = _blk(64, 1025, 3)
    C = torch.zeros((1025, 1025), dtype=torch.float64, device="cuda")
    with pytest.raises(arb.ArbError) as e:
        arb.arb_gram_noalloc(ctx, X, X, C)
    assert e.value.status == arb.ARB_INVALID_ARG
    assert torch.all(C == 0)
