"""Plain-Python statement of the SELL-C-sigma sparse layout (Kreutzer, Hager, Wellein,
Fehske & Bishop, "A unified sparse matrix data format for efficient general sparse
matrix-vector multiplication on modern processors with wide SIMD units", SIAM J. Sci.
Comput. 36(5), 2014, Section 2: the SELL-C-sigma format).

TEST INFRASTRUCTURE ONLY.  Only the test-suite may import it; the library never does and
shares no code with it.  It is the layout the library's block SpMM reads when a matrix is
given a SELL copy; the eigensolver's arithmetic does not depend on it.

The definition followed, step by step:
1. Sorting scope: the rows are taken in windows of sigma consecutive rows; within a window
   they are ordered by decreasing number of nonzeros (rows of equal length keep their
   original order).
2. Chunks: the sorted rows are cut into chunks of C consecutive rows (the last may be
   short).
3. Each chunk is padded to the length of its longest row and stored column by column:
   entry j of the chunk's row r sits at chunk_start + j * C + r.
"""
import numpy as np


def sell_c_sigma(rowptr, C, sigma):
    """Return (perm, length, chunk_start, src) of the SELL-C-sigma layout of a CSR pattern.

    perm[i]: original row at sorted position i; length[i]: its nonzero count;
    chunk_start[c]: first slot of chunk c (one extra entry: the slot count);
    src[s]: CSR index of the nonzero in slot s, or -1 for padding.
    """
    rowptr = [int(v) for v in rowptr]
    n = len(rowptr) - 1
    row_len = [rowptr[i + 1] - rowptr[i] for i in range(n)]
    # step 1: sort inside each window of sigma rows, longest first, stable
    perm = []
    for w0 in range(0, n, sigma):
        window = list(range(w0, min(n, w0 + sigma)))
        window.sort(key=lambda r: -row_len[r])  # Python's sort is stable
        perm.extend(window)
    length = [row_len[r] for r in perm]
    # steps 2-3: chunks of C sorted rows, each padded to its longest row, column-major
    nchunks = (n + C - 1) // C
    chunk_start = [0]
    for c in range(nchunks):
        rows = range(c * C, min(n, (c + 1) * C))
        width = max((length[i] for i in rows), default=0)
        chunk_start.append(chunk_start[-1] + width * C)
    src = [-1] * chunk_start[-1]
    for i in range(n):
        c, r = divmod(i, C)
        for j in range(length[i]):
            src[chunk_start[c] + j * C + r] = rowptr[perm[i]] + j
    return (np.array(perm, dtype=np.int64), np.array(length, dtype=np.int64),
            np.array(chunk_start, dtype=np.int64), np.array(src, dtype=np.int64))


def sell_matvec(perm, length, chunk_start, src, col, val, C, x):
    """y = A x computed from the SELL slots alone (row by row in sorted order)."""
    y = np.zeros(len(perm), dtype=np.float64)
    for i in range(len(perm)):
        c, r = divmod(i, C)
        s = 0.0
        for j in range(int(length[i])):
            e = src[chunk_start[c] + j * C + r]
            s += val[e] * x[col[e]]
        y[perm[i]] = s
    return y
