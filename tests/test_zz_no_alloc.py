"""arb_gram_noalloc: the Gram product for callers that cannot allocate device memory
(graph-capturing code, applications with their own memory pool).  Its partial sums live
in the library's static device scratch; it must give arb_gram's result, also on a second
call that reuses the scratch, and refuse shapes that do not fit.  Collected last so a
stop-at-first-failure run has already run every other test."""
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
        arb.arb_gram_noalloc(ctx, X, Y, C)
        torch.cuda.synchronize()
        # same products, sums split differently over rows: the Gram tolerance of the parity
        # tests, 1e-13 ||x_i|| ||y_j|| per entry
        bound = 1e-13 * torch.outer(X.norm(dim=0), Y.norm(dim=0))
        assert torch.isfinite(C).all()
        assert bool(((C - ref).abs() <= bound).all())


def test_noalloc_gram_refuses_shapes_beyond_scratch(env):
    arb, ctx = env
    X = _blk(64, 1025, 3)
    C = torch.zeros((1025, 1025), dtype=torch.float64, device="cuda")
    with pytest.raises(arb.ArbError) as e:
        arb.arb_gram_noalloc(ctx, X, X, C)
    assert e.value.status == arb.ARB_INVALID_ARG
    assert torch.all(C == 0)
