"""Host-side checks of the C ABI library (no GPU needed): it builds for sm_103a, loads, and
exports every function that include/arrabit.h declares."""
import ctypes

import numpy as np
import pytest

from paper_1507_06078_gb300 import arrabit as arb
from paper_1507_06078_gb300 import build as B
from paper_1507_06078_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    B.build()
    return arb.load()


def test_every_declared_symbol_is_exported(lib):
    names = arb.header_functions()
    assert "arb_solve" in names and "arb_filter" in names and len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a prototype for each of them
    assert set(names) <= set(arb._PROTOS)


def test_status_strings_and_defaults(lib):
    assert lib.arb_status_string(0) == b"ok"
    assert lib.arb_status_string(-4) == b"iterate lost numerical rank"
    o = arb.arb_options_default(20)
    assert (o.p, o.q, o.degree, o.maxit, o.maxit1, o.maxit2) == (22, 1, 3, 30, 10, 5)
    assert np.isnan(o.shift_sigma)
    assert ctypes.sizeof(arb.arb_options) == 4 * 10 + 8 * 4 + 4 * 4
    assert ctypes.sizeof(arb.arb_info) == 8 * 8 + 8 + 4 * 10


@pytest.mark.parametrize("d", [1, 3, 10, 15, 20])
def test_host_filter_coefficients_match_oracle(lib, d):
    # the library's host-side coefficients (cosine-sum formula) against the oracle's
    # collocation solve: two independent derivations of the Section 5 interpolant
    from oracle import arrabit_oracle as O
    c = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBINTERP, d)
    np.testing.assert_allclose(c, O.interpolant_cheb_coeffs(d), atol=2e-15)
    e = arb.arb_filter_coefficients(arb.ARB_FILTER_CHEBYSHEV, d)
    np.testing.assert_array_equal(e, O.chebyshev_T_coeffs(d))


def test_bad_coefficient_requests_rejected(lib):
    buf = np.zeros(70)
    assert lib.arb_filter_coefficients(0, 0, buf.ctypes.data) == arb.ARB_INVALID_ARG
    assert lib.arb_filter_coefficients(0, 61, buf.ctypes.data) == arb.ARB_INVALID_ARG
    assert lib.arb_filter_coefficients(7, 3, buf.ctypes.data) == arb.ARB_INVALID_ARG


def test_server_footprint_formula(lib):
    # 7 FP64 n x p blocks + 2 FP64 n x (q+1)p blocks + small state; mixed adds FP32 copies
    f = arb.arb_server_footprint(1000, 5000, 30, 1, arb.ARB_FP64)
    base = 1000 * (7 * 30 + 2 * 60) * 8
    assert base < f < base + (80 << 20)
    fm = arb.arb_server_footprint(1000, 5000, 30, 1, arb.ARB_MIXED)
    assert fm > f
    fdf = arb.arb_server_footprint(1000, 5000, 30, 1, arb.ARB_MIXED_DF)
    assert fdf == fm + 5000 * 8  # plus the double-float copy of A's values
    assert arb.arb_server_footprint(1000, 5000, 30, 1, 7) == -1
    assert arb.arb_server_footprint(0, 0, 30, 1, 0) == -1


def test_symmetry_check_host_only(lib):
    # host-side check of CSR arrays (no device involved): stencil Laplacians and a
    # symmetric random matrix pass, a one-sided perturbation or entry fails, malformed
    # arrays are rejected
    import scipy.sparse as sp
    A = I.laplacian_3d(6)
    assert arb.arb_csr_check_symmetric(A.n, A.rowptr, A.col, A.val) == arb.ARB_OK
    rng = np.random.default_rng(1)
    M = sp.random(300, 300, density=0.05, random_state=rng, format="csr")
    M = (M + M.T).tocsr()
    assert arb.arb_csr_check_symmetric(300, M.indptr, M.indices, M.data) == arb.ARB_OK
    v = M.data.copy()
    v[5] += 1e-6
    assert arb.arb_csr_check_symmetric(300, M.indptr, M.indices, v) == arb.ARB_NOT_SYMMETRIC
    assert arb.arb_csr_check_symmetric(300, M.indptr, M.indices, v, 1e-5) == arb.ARB_OK
    U = sp.triu(M, k=1).tocsr()  # strictly upper part only
    if U.nnz:
        assert arb.arb_csr_check_symmetric(300, U.indptr, U.indices, U.data) == arb.ARB_NOT_SYMMETRIC
    bad = A.rowptr.copy()
    bad[-1] += 1
    assert arb.arb_csr_check_symmetric(A.n, bad, A.col, A.val) == arb.ARB_INVALID_ARG


# A worked SELL-C-sigma example from the format's definition (Kreutzer et al. 2014, Sec. 2),
# derived by hand: 6 rows of lengths 1, 3, 2, 0, 2, 1 (CSR entries 0..8), C = 2, sigma = 4.
# Window rows 0-3 sorted longest first: 1 (3), 2 (2), 0 (1), 3 (0); window rows 4-5: 4 (2),
# 5 (1).  Chunks: positions {0, 1} width 3 -> 6 slots, {2, 3} width 1 -> 2 slots, {4, 5}
# width 2 -> 4 slots.  Column-major slots: chunk 0 holds row 1's entries 1, 2, 3 at slots
# 0, 2, 4 and row 2's entries 4, 5 at slots 1, 3; chunk 1 row 0's entry 0 at slot 6; chunk 2
# row 4's entries 6, 7 at slots 8, 10 and row 5's entry 8 at slot 9.
SELL_EXAMPLE = dict(rowptr=[0, 1, 4, 6, 6, 8, 9], C=2, sigma=4, perm=[1, 2, 0, 3, 4, 5], length=[3, 2, 1, 0, 2, 1],
                    chunk_start=[0, 6, 8, 12], src=[1, 4, 2, 5, 3, -1, 0, -1, 6, 8, 7, -1])


def test_sell_layout_worked_example(lib):
    from oracle import sell_oracle as S
    ex = SELL_EXAMPLE
    for got in (S.sell_c_sigma(ex["rowptr"], ex["C"], ex["sigma"]),
                arb.arb_sell_layout(np.array(ex["rowptr"]), ex["C"], ex["sigma"])):
        perm, ln, cptr, src = got
        assert perm.tolist() == ex["perm"] and ln.tolist() == ex["length"]
        assert cptr.tolist() == ex["chunk_start"] and src.tolist() == ex["src"]


@pytest.mark.parametrize("C,sigma", [(32, 1024), (4, 8), (1, 1), (32, 1), (7, 100), (64, 5000)])
def test_sell_layout_matches_oracle_on_power_law_rows(lib, C, sigma):
    # the library's host layout equals the oracle's, integer for integer; the layout
    # reproduces A x from its slots alone and stores every nonzero exactly once
    from oracle import sell_oracle as S
    A, _ = I.chung_lu_laplacian(3000, seed=5)
    lo = S.sell_c_sigma(A.rowptr, C, sigma)
    li = arb.arb_sell_layout(A.rowptr, C, sigma)
    for a, b in zip(lo, li):
        np.testing.assert_array_equal(a, b)
    perm, ln, cptr, src = lo
    assert sorted(src[src >= 0].tolist()) == list(range(A.nnz))
    x = np.random.default_rng(C + sigma).standard_normal(A.n)
    dense = A.to_dense()
    np.testing.assert_allclose(S.sell_matvec(perm, ln, cptr, src, A.col, A.val, C, x), dense @ x, atol=1e-12)
    # lengths never increase inside a window
    for w0 in range(0, A.n, sigma):
        seg = ln[w0:w0 + sigma]
        assert np.all(np.diff(seg) <= 0)


def test_sell_layout_rejects_bad_arguments(lib):
    rp = np.array([0, 1, 2], dtype=np.int32)
    with pytest.raises(arb.ArbError):
        arb.arb_sell_layout(rp, 0, 4)
    with pytest.raises(arb.ArbError):
        arb.arb_sell_layout(rp, 2, 0)
    with pytest.raises(arb.ArbError):
        arb.arb_sell_layout(np.array([0, 2, 1], dtype=np.int32), 2, 4)


@pytest.mark.parametrize("rowptr,C,sigma", [([0], 32, 1024), ([0, 3], 32, 1024), ([0, 0, 0], 4, 2),
                                            ([0, 2, 3, 7], 8, 2), ([0, 1, 1, 4, 4, 6], 2, 100)])
def test_sell_layout_edge_cases_match_oracle(lib, rowptr, C, sigma):
    # empty matrix, one row, empty rows, a chunk wider than the matrix, a window wider than it
    from oracle import sell_oracle as S
    lo = S.sell_c_sigma(rowptr, C, sigma)
    li = arb.arb_sell_layout(np.array(rowptr), C, sigma)
    for a, b in zip(lo, li):
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("fn", ["arb_gram", "arb_gram_f32", "arb_gram_noalloc"])
def test_gram_bindings_refuse_mismatched_shapes_before_any_launch(fn):
    # the C entry points take no row count for Y and none for C: a short Y or a small C
    # would be read or written out of bounds, so the binding refuses them before it
    # touches a pointer (host tensors here: nothing reaches the library)
    torch = pytest.importorskip("torch")
    f = getattr(arb, fn)
    dt = torch.float32 if fn == "arb_gram_f32" else torch.float64
    X = torch.zeros((100, 4), dtype=dt)
    with pytest.raises(ValueError, match="rows"):
        f(None, X, torch.zeros((99, 3), dtype=dt), torch.zeros((4, 3), dtype=torch.float64))
    with pytest.raises(ValueError, match="C_out"):
        f(None, X, torch.zeros((100, 3), dtype=dt), torch.zeros((4, 2), dtype=torch.float64))
    with pytest.raises(ValueError, match="C_out"):
        f(None, X, torch.zeros((100, 3), dtype=dt), torch.zeros((3, 4), dtype=torch.float64))


def test_struct_layouts_match_the_header(tmp_path):
    # the binding's ctypes structures against the C compiler's layout of include/arrabit.h:
    # size and the offset of every field, for every structure the calls pass by pointer
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [arb.arb_options, arb.arb_info, arb.arb_filter_job, arb.arb_batch_stats]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "arrabit.h"', "int main(void) {"]
    for s in structs:
        name = s.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in s._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, field, value = line.split()
            got[(name, field)] = int(value)
    for s in structs:
        name = s.__name__
        assert got[(name, "size")] == ctypes.sizeof(s), name
        for f, _ in s._fields_:
            assert got[(name, f)] == getattr(s, f).offset, (name, f)
