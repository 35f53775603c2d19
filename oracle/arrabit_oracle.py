"""Plain FP64 CPU oracle for ARRABIT-MPM (Wen & Zhang, "Block algorithms with augmented
Rayleigh-Ritz projections for large-scale eigenpair computation", arXiv 1507.06078).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct statement of what
the CUDA library computes.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import it; the library never does,
and it shares no code with the library (inputs arrive as plain arrays).

Everything is float64.  Library primitives used as single steps: scipy.sparse matrix
products, scipy's pivoted Householder QR, Cholesky factor/solve, and numpy's Chebyshev
basis conversion.  The dense symmetric eigensolver is a hand-written cyclic Jacobi.

Readings of the paper taken where it is silent or inconsistent:

* Alg. 1 writes H = V^T Sigma V but Y = U V; we take H = V Sigma V^T with the columns of
  V the eigenvectors, sorted by descending Ritz value (ties keep index order).
* orth(Z) in Alg. 1 is unspecified; here: Householder QR with column pivoting, rank
  truncated where |R_ii| <= max(n, m) * eps * |R_00|.
* Columns of the augmented block [X, AX, ..., A^q X] are scaled to unit 2-norm before
  orthonormalisation (does not change the span).
* The interpolant has degree d and interpolates f_d(t) = max(0, t)^(10 d) at the d+1
  Chebyshev points of the second kind (Section 5, eqs. def:fN and chebfun-f).
* rcond in the inner stop rule is the exact reciprocal 1-norm condition number of
  X^T X (inverse via Cholesky); a failed Cholesky means rc = 0.
* The projection X - Q_c (Q_c^T X) is applied after every inner step, as Alg. 8 places it.
* b is updated only at a continuation step (b = mu_{k+q}), as Alg. 8 does.
* tol_1 = max(1e-6, tol) when tol <= 1e-8, else tol (no continuation).
* Lock threshold is max(1e-14, tol_t^2) with the current tol_t; only the k wanted
  pairs are candidates for locking.
* Stall rule (ii): stop when the best maxres so far was reached 3 or more outer
  iterations ago.  Rule (iii): h counts wanted pairs with res_i < 0.1 tol.
* For the smallest eigenpairs the method runs on B = sigma I - A with sigma an upper
  bound of A's spectrum, the tighter of Gershgorin's and a 32-step Lanczos estimate with
  residual margins (Section 5 estimates the spectrum's far end; the paper calls eigs);
  a = sigma - that bound.  For the largest, a = the corresponding lower bound.  Residuals use the
  original eigenvalue estimate lambda_i = sigma - mu_i in the denominator, and the
  reported eigenvalues are the Rayleigh quotients x_i^T A x_i on the original A.
* If orth(Z) leaves fewer than p directions, the Ritz set is padded with columns
  of a caller-supplied Gaussian block, orthogonalised against the basis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

EPS = np.finfo(np.float64).eps


# -------------------------------------------------------------------------------------
# Matrix helpers
# -------------------------------------------------------------------------------------
def csr_to_scipy(n, rowptr, col, val) -> sp.csr_matrix:
    """Wrap CSR arrays as a float64 scipy matrix."""
    return sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(col), np.asarray(rowptr)),
                         shape=(n, n))


def gershgorin_bounds(B: sp.csr_matrix) -> tuple[float, float]:
    """Gershgorin interval [min_i (B_ii - R_i), max_i (B_ii + R_i)], R_i = sum_{j!=i} |B_ij|.

    Stands in for the eigs call that the paper uses to estimate lambda_n (Section 5,
    "Estimation of lambda_n and lambda_{k+q}"): any lower bound of the spectrum works.
    """
    diag = B.diagonal()
    absrow = np.asarray(abs(B).sum(axis=1)).ravel()
    radius = absrow - np.abs(diag)
    return float(np.min(diag - radius)), float(np.max(diag + radius))


# -------------------------------------------------------------------------------------
# Section 5: polynomial accelerators
# -------------------------------------------------------------------------------------
def chebyshev_points(N: int) -> np.ndarray:
    """Chebyshev points of the second kind t_j = -cos(j pi / N), j = 0..N (Section 5)."""
    j = np.arange(N + 1)
    return -np.cos(j * np.pi / N)


def f_d(t, d: int):
    """f_d(t) = (f_1(t))^d with f_1(t) = max(0, t)^10 (Section 5, eq. def:fN)."""
    return np.maximum(0.0, np.asarray(t, dtype=np.float64)) ** (10 * d)


def interpolant_cheb_coeffs(d: int) -> np.ndarray:
    """Coefficients a_0..a_d of psi_d = sum_k a_k T_k, the degree-d interpolant of f_d at
    the d+1 Chebyshev points of the second kind (Section 5, eq. chebfun-f).

    Written as the definition: solve the (d+1)x(d+1) collocation system
    sum_k a_k T_k(t_j) = f_d(t_j), with T_k(t) = cos(k arccos t).
    """
    t = chebyshev_points(d)
    T = np.cos(np.outer(np.arccos(np.clip(t, -1.0, 1.0)), np.arange(d + 1)))
    return np.linalg.solve(T, f_d(t, d))


def chebyshev_T_coeffs(d: int) -> np.ndarray:
    """Coefficient vector e_d of the plain Chebyshev polynomial T_d (eq. cheby-poly)."""
    e = np.zeros(d + 1)
    e[d] = 1.0
    return e


def cheb_to_monomial(a: np.ndarray) -> np.ndarray:
    """Gamma_d = (gamma_1, ..., gamma_{d+1}) of eq. chebfun-f, highest power first."""
    mono = np.polynomial.chebyshev.cheb2poly(a)  # lowest power first
    return mono[::-1].copy()


def eval_cheb_series(a: np.ndarray, t) -> np.ndarray:
    """sum_k a_k T_k(t) by the three-term recurrence of eq. cheby-poly (any real t)."""
    t = np.asarray(t, dtype=np.float64)
    T_prev = np.ones_like(t)
    out = a[0] * T_prev
    if len(a) == 1:
        return out
    T_cur = t.copy()
    out = out + a[1] * T_cur
    for k in range(2, len(a)):
        T_prev, T_cur = T_cur, 2.0 * t * T_cur - T_prev
        out = out + a[k] * T_cur
    return out


def rho_d(a_coef: np.ndarray, lam, a: float, b: float):
    """rho_d(t) = psi_d((2t - a - b)/(b - a)) (Section 5, eq. rhod)."""
    return eval_cheb_series(a_coef, (2.0 * np.asarray(lam) - a - b) / (b - a))


def poly_alg7(B, X: np.ndarray, a: float, b: float, gamma: np.ndarray) -> np.ndarray:
    """Y = poly(B, X, a, b, Gamma_d) exactly as Algorithm 7 states it (monomial Horner).

    c0 = (a+b)/(a-b), c1 = 2/(b-a); Y = gamma_1 X; for j = 1..d: Y = c0 Y + c1 B Y + gamma_{j+1} X.
    """
    d = len(gamma) - 1
    c0 = (a + b) / (a - b)
    c1 = 2.0 / (b - a)
    Y = gamma[0] * X
    for j in range(1, d + 1):
        Y = c0 * Y + c1 * (B @ Y) + gamma[j] * X
    return Y


def poly_clenshaw(B, X: np.ndarray, a: float, b: float, coef: np.ndarray) -> np.ndarray:
    """The same Y = psi_d(S) X, S = c1 B + c0 I (the affine map of eq. rhod), evaluated in
    the Chebyshev basis by Clenshaw's recurrence:
    b_{d+1} = b_{d+2} = 0, b_j = coef_j X + 2 S b_{j+1} - b_{j+2} (j = d..1),
    Y = coef_0 X + S b_1 - b_2.
    """
    d = len(coef) - 1
    c0 = (a + b) / (a - b)
    c1 = 2.0 / (b - a)

    def S(Y):
        return c1 * (B @ Y) + c0 * Y

    if d == 0:
        return coef[0] * X
    b2 = np.zeros_like(X)
    b1 = coef[d] * X
    for j in range(d - 1, 0, -1):
        b1, b2 = coef[j] * X + 2.0 * S(b1) - b2, b1
    return coef[0] * X + S(b1) - b2


# -------------------------------------------------------------------------------------
# Dense building blocks
# -------------------------------------------------------------------------------------
def normalize_columns(X: np.ndarray) -> np.ndarray:
    """x_i <- x_i / ||x_i||_2 (the MPM normalisation of Section 3 and Alg. 8)."""
    nrm = np.linalg.norm(X, axis=0)
    nrm[nrm == 0.0] = 1.0
    return X / nrm


def project_out(Qc: np.ndarray, X: np.ndarray) -> np.ndarray:
    """X - Q_c (Q_c^T X) (Alg. 8 projection; Section 5, "Deflation")."""
    if Qc is None or Qc.shape[1] == 0:
        return X
    return X - Qc @ (Qc.T @ X)


def rcond_spd(G: np.ndarray) -> float:
    """Reciprocal 1-norm condition number 1/(||G||_1 ||G^{-1}||_1) of a symmetric matrix
    (eq. inn-stop).  The inverse comes from a Cholesky factorisation; a failed
    factorisation (G not numerically positive definite) gives 0."""
    G = 0.5 * (G + G.T)
    try:
        c = sla.cho_factor(G, lower=False, check_finite=True)
    except (np.linalg.LinAlgError, ValueError):
        return 0.0
    Ginv = sla.cho_solve(c, np.eye(G.shape[0]))
    n1 = np.abs(G).sum(axis=0).max()
    n1i = np.abs(Ginv).sum(axis=0).max()
    if not np.isfinite(n1i) or n1i == 0.0:
        return 0.0
    return float(1.0 / (n1 * n1i))


def orth(Z: np.ndarray) -> np.ndarray:
    """An orthonormal basis U of the numerical range of Z (Alg. 1, first step).

    Householder QR with column pivoting; columns with |R_ii| <= max(n, m) eps |R_00| are
    dropped as numerically dependent."""
    if Z.shape[1] == 0:
        return Z.copy()
    Q, R, _ = sla.qr(Z, mode="economic", pivoting=True)
    dR = np.abs(np.diag(R))
    if dR.size == 0 or dR[0] == 0.0:
        return Q[:, :0]
    tol = max(Z.shape) * EPS * dR[0]
    r = int(np.sum(dR > tol))
    return Q[:, :r]


def jacobi_eigh(H: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigen-decomposition H = V diag(w) V^T of a symmetric matrix by the cyclic (row by
    row) Jacobi method: each rotation J in the (i, j) plane, J_ii = J_jj = c, J_ij = s,
    J_ji = -s, with t = sign(theta)/(|theta| + sqrt(theta^2 + 1)), theta = (h_jj - h_ii)/(2 h_ij),
    c = 1/sqrt(1+t^2), s = t c, zeroes h_ij of J^T H J.  Sweeps stop once the off-diagonal
    Frobenius norm is <= tol * ||H||_F.  Returns w sorted descending (stable) and V.
    """
    A = np.array(H, dtype=np.float64, copy=True)
    A = 0.5 * (A + A.T)
    m = A.shape[0]
    V = np.eye(m)
    normF = np.linalg.norm(A)
    if m <= 1 or normF == 0.0:
        w = np.diag(A).copy()
        order = np.argsort(-w, kind="stable")
        return w[order], V[:, order]
    for _ in range(max_sweeps):
        offd = A - np.diag(np.diag(A))
        off = math.sqrt(float(np.sum(offd * offd)))
        if off <= tol * normF:
            break
        for i in range(m - 1):
            for j in range(i + 1, m):
                hij = A[i, j]
                if hij == 0.0:
                    continue
                theta = (A[j, j] - A[i, i]) / (2.0 * hij)
                sgn = 1.0 if theta >= 0.0 else -1.0
                t = sgn / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                ci = A[:, i].copy()
                cj = A[:, j].copy()
                A[:, i] = c * ci - s * cj
                A[:, j] = s * ci + c * cj
                ri = A[i, :].copy()
                rj = A[j, :].copy()
                A[i, :] = c * ri - s * rj
                A[j, :] = s * ri + c * rj
                A[i, j] = 0.0
                A[j, i] = 0.0
                vi = V[:, i].copy()
                vj = V[:, j].copy()
                V[:, i] = c * vi - s * vj
                V[:, j] = s * vi + c * vj
    w = np.diag(A).copy()
    order = np.argsort(-w, kind="stable")
    return w[order], V[:, order]


def rayleigh_ritz(B, Z: np.ndarray):
    """(Y, Sigma) = RR(B, Z), Algorithm 1: U = orth(Z); H = U^T B U; H = V Sigma V^T;
    Y = U V.  Ritz values descending; Y has as many columns as the rank of Z."""
    U = orth(Z)
    if U.shape[1] == 0:
        return U, np.zeros(0)
    H = U.T @ (B @ U)
    H = 0.5 * (H + H.T)
    w, V = jacobi_eigh(H)
    return U @ V, w


def augment(B, X: np.ndarray, q: int) -> np.ndarray:
    """Z = [X, BX, ..., B^q X] (Alg. 5, eq. S:ARR), each column scaled to unit norm."""
    blocks = [X]
    for _ in range(q):
        blocks.append(B @ blocks[-1])
    return normalize_columns(np.hstack(blocks))


def arr(B, X: np.ndarray, q: int, npairs: int | None = None):
    """(Y, Sigma) = ARR(B, X, q), Algorithm 5: RR on the augmentation, keep the leading
    ``npairs`` (default: the width of X) Ritz pairs."""
    Y, w = rayleigh_ritz(B, augment(B, X, q))
    if npairs is None:
        npairs = X.shape[1]
    return Y[:, :npairs], w[:npairs]


def residual_norms(B, X: np.ndarray, mu: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """res_i = ||B x_i - mu_i x_i|| / max(1, |lam_i|) (eq. resi; lam_i the eigenvalue
    estimate in the original problem's terms, equal to mu_i when B = A)."""
    R = B @ X - X * mu[None, :]
    return np.linalg.norm(R, axis=0) / np.maximum(1.0, np.abs(lam))


def pad_ritz(B, Y: np.ndarray, w: np.ndarray, want: int, pool: np.ndarray | None):
    """Complete a Ritz set with fewer than ``want`` vectors by orthonormalising the next
    columns of a Gaussian ``pool`` against it (Rayleigh quotients as their values)."""
    if Y.shape[1] >= want:
        return Y, w
    if pool is None:
        raise RuntimeError("Ritz set smaller than the block and no padding pool given")
    need = want - Y.shape[1]
    P = pool[:, :need].copy()
    for _ in range(2):
        P = P - Y @ (Y.T @ P)
    P = orth(P)
    for _ in range(2):
        P = P - Y @ (Y.T @ P)
    P = normalize_columns(P)
    rq = np.einsum("ij,ij->j", P, B @ P)
    return np.hstack([Y, P]), np.concatenate([w, rq])


def gn_step(apply_filter, X: np.ndarray) -> np.ndarray:
    """One Gauss-Newton inner step of Algorithm 8 (the GN branch; Algorithm 4 with the
    polynomial accelerator in place of A): Y = X (X^T X)^{-1}, Z = poly(A - aI, Y, ...),
    X+ = Z - X (Y^T Z - I) / 2.  (X^T X)^{-1} comes from a Cholesky factorisation; a
    rank-deficient X (failed factorisation) raises numpy.linalg.LinAlgError."""
    G = X.T @ X
    c = sla.cho_factor(0.5 * (G + G.T), lower=False, check_finite=True)
    Y = sla.cho_solve(c, X.T).T
    Z = apply_filter(Y)
    return Z - X @ (Y.T @ Z - np.eye(X.shape[1])) / 2.0


def filter_value(coef: np.ndarray, mu, a: float, b: float):
    """rho_d(mu) for the filter Algorithm 8 applies, poly(B - aI, ., 0, b - a, Gamma_d):
    psi_d at the image of mu - a under the map of [0, b - a] onto [-1, 1]."""
    return eval_cheb_series(coef, 2.0 * (np.asarray(mu, dtype=np.float64) - a) / (b - a) - 1.0)


def next_degree(filter_kind: str, mu_k: float, mu_kq: float, a: float, b: float, d_max: int) -> int:
    """The polynomial degree rule of Section 5 (eqs. hat-d and degree): the smallest d >= 3
    with rho_d(mu*_{k+q}) / rho_d(mu*_k) < 0.9, capped at d_max (d_max when no d up to
    d_max qualifies)."""
    for d in range(3, d_max + 1):
        coef = interpolant_cheb_coeffs(d) if filter_kind == "chebinterp" else chebyshev_T_coeffs(d)
        rk = float(filter_value(coef, mu_k, a, b))
        rkq = float(filter_value(coef, mu_kq, a, b))
        if rk > 0.0 and np.isfinite(rk) and np.isfinite(rkq) and rkq / rk < 0.9:
            return d
    return d_max


# -------------------------------------------------------------------------------------
# Algorithm 8 (MPM or GN inner solver)
# -------------------------------------------------------------------------------------
@dataclass
class OuterRecord:
    """What one outer iteration of Algorithm 8 did."""

    n_filters: int
    rc: list
    maxres: float
    tol_t: float
    b: float
    n_locked: int
    rank: int
    q: int = 1       # augmentation blocks of this iteration's ARR
    degree: int = 0  # polynomial degree of this iteration's filters


@dataclass
class OracleResult:
    evals: np.ndarray  # k eigenvalues of A (ascending for smallest, descending for largest)
    evecs: np.ndarray  # n x k
    res: np.ndarray  # relative residuals of the k pairs
    maxres: float
    converged: bool
    stop_reason: str
    outer_iters: int
    n_spmm_cols: int  # sum over block products of the block width ("SpMV count")
    a: float
    b0: float
    sigma: float
    history: list = field(default_factory=list)


def lanczos_bounds(A: sp.csr_matrix, steps: int, seed: int) -> tuple[float, float]:
    """Estimates (lo, hi) of the extreme eigenvalues of A (Section 5 estimates the far end
    of the spectrum; the paper calls eigs): ``steps`` steps of plain Lanczos from the
    Gaussian column of stream ``seed``, the extreme eigenvalues theta of the tridiagonal
    matrix widened by their residual bounds |beta_m y_m| and by 1e-3 max(1, |theta|)."""
    from paper_1507_06078_gb300.inputs import gaussian_block
    n = A.shape[0]
    steps = min(steps, n)
    v = gaussian_block(n, 1, seed)[:, 0]
    v = v / np.sqrt(v @ v)
    vp = np.zeros(n)
    al, be, bprev = [], [], 0.0
    for _ in range(steps):
        w = A @ v
        a = float(v @ w)
        w = w - a * v - bprev * vp
        b = math.sqrt(max(float(w @ w), 0.0))
        al.append(a)
        be.append(b)
        if not b > 1e-12 * max(1.0, abs(a)):
            break
        vp, v, bprev = v, w / b, b
    m = len(al)
    T = np.diag(al) + np.diag(be[:m - 1], 1) + np.diag(be[:m - 1], -1)
    th, Y = np.linalg.eigh(T)
    hi = th[-1] + abs(be[-1] * Y[-1, -1]) + 1e-3 * max(1.0, abs(th[-1]))
    lo = th[0] - abs(be[-1] * Y[-1, 0]) - 1e-3 * max(1.0, abs(th[0]))
    return float(lo), float(hi)


# Input convention shared with the library, not arithmetic of the method: the Lanczos start
# column is the Gaussian stream number seed + 0x9E3779B97F4A7C15 (mod 2^64), so that both
# sides start the spectrum estimate from the same column of the seeded input generator
BOUND_SEED_OFFSET = 0x9E3779B97F4A7C15


def arrabit_mpm(A: sp.csr_matrix, k: int, X0: np.ndarray, which: str = "smallest",
                tol: float = 1e-10, q: int = 1, degree: int = 10, maxit: int = 30,
                maxit1: int = 10, maxit2: int = 5, tol1: float | None = None,
                filter_kind: str = "chebinterp", sigma: float | None = None,
                inner_fixed: int = 0, pad_pool: np.ndarray | None = None,
                poly_eval: str = "clenshaw", b_update: str = "continuation",
                seed: int = 20150722, inner: str = "mpm", adapt_q: bool = False, q_max: int = 3,
                adapt_d: bool = False, d_max: int = 15) -> OracleResult:
    """ARRABIT with the multi-power inner solver, Algorithm 8, for the k largest (or, via
    B = sigma I - A, smallest) eigenpairs of symmetric A.  The block width is
    p = X0.shape[1] = k + guard vectors.  ``inner_fixed`` > 0 replaces the inner stop rule
    by exactly that many inner steps per outer iteration (for lock-step tests).
    ``b_update`` = "continuation" refreshes b = mu_{k+q} only at a continuation step, as
    Algorithm 8 does; "every_arr" refreshes it after every ARR projection, as the
    estimation paragraph of Section 5 describes.  ``inner`` = "gn" takes Algorithm 8's GN
    branch instead of MPM.  ``adapt_q`` raises q by one (up to q_max) after an ARR when
    eq. block holds; ``adapt_d`` sets the degree after every ARR by eqs. hat-d and degree
    (cap d_max); ``degree`` and ``q`` are then the initial values.
    """
    A = sp.csr_matrix(A, dtype=np.float64)
    n, p = X0.shape
    if not (0 < k <= p and (q + 1) * p < n):
        raise ValueError("need 0 < k <= p and (q+1) p < n")
    # the far end of the spectrum: the tighter of Gershgorin's bound and a Lanczos estimate
    glo, ghi = gershgorin_bounds(A)
    llo, lhi = lanczos_bounds(A, 32, (seed + BOUND_SEED_OFFSET) % (1 << 64))
    lo_A, hi_A = max(glo, llo), min(ghi, lhi)
    if which == "smallest":
        if sigma is None:
            sigma = hi_A
        B = (sp.identity(n, format="csr") * sigma - A).tocsr()
        a = sigma - hi_A

        def to_orig(mu):
            return sigma - mu
    elif which == "largest":
        sigma = 0.0
        B = A
        a = lo_A

        def to_orig(mu):
            return mu
    else:
        raise ValueError(which)

    # interval [a, b] (Section 5): a = lower bound of B's spectrum (above), b = smallest
    # Ritz value of orth(X0)
    U0 = orth(X0)
    H0 = U0.T @ (B @ U0)
    b = float(jacobi_eigh(H0)[0][-1])
    b0 = b
    n_spmm_cols = U0.shape[1]
    if filter_kind not in ("chebinterp", "chebyshev"):
        raise ValueError(filter_kind)
    if inner not in ("mpm", "gn"):
        raise ValueError(inner)

    def coefficients(d):
        return interpolant_cheb_coeffs(d) if filter_kind == "chebinterp" else chebyshev_T_coeffs(d)

    def apply_filter(X):
        # Alg. 8 calls poly(B - aI, X, 0, b - a, Gamma_d) with the current degree
        Bs = B - a * sp.identity(n, format="csr")
        coef = coefficients(degree)
        if poly_eval == "horner":
            return poly_alg7(Bs, X, 0.0, b - a, cheb_to_monomial(coef))
        return poly_clenshaw(Bs, X, 0.0, b - a, coef)

    # the augmentation count may grow only while (q + 1) p < n (Algorithm 5's requirement)
    q_cap = max(q, min(q_max, (n - 1) // p - 1)) if adapt_q else q
    mu_best = None
    maxres_prev = None

    if tol1 is None:
        tol1 = max(1e-6, tol) if tol <= 1e-8 else tol
    tol_t = max(tol1, tol)
    Qc = np.zeros((n, 0))
    Sc = np.zeros(0)
    X = np.array(X0, dtype=np.float64, copy=True)
    best = math.inf
    best_iter = 0
    history = []
    stop_reason = "maxit"
    res = None
    Xall = None
    mu = None
    j = 0
    for j in range(1, maxit + 1):
        rc = math.inf
        rcs = []
        nf = 0
        i1_max = maxit1 if inner_fixed <= 0 else 1
        for _ in range(i1_max):
            n_inner = maxit2 if inner_fixed <= 0 else inner_fixed
            lost_rank = False
            for _ in range(n_inner):
                if inner == "mpm":
                    X = normalize_columns(apply_filter(X))
                else:
                    try:
                        X = gn_step(apply_filter, X)
                    except np.linalg.LinAlgError:
                        # X^T X is not numerically positive definite: the GN step is
                        # undefined; end the inner loop and let the ARR step take over
                        lost_rank = True
                        break
                X = project_out(Qc, X)
                nf += 1
                n_spmm_cols += degree * X.shape[1]
            if inner_fixed > 0 or lost_rank:
                break
            rcp = rc
            rc = rcond_spd(X.T @ X)
            rcs.append(rc)
            if rc <= tol_t or rc / rcp > 0.99:
                break
        # augmentation, projection, RR (ARR step)
        Z = augment(B, X, q)
        n_spmm_cols += q * X.shape[1]
        Z = project_out(Qc, Z)
        Y, w = rayleigh_ritz(B, Z)
        n_spmm_cols += Y.shape[1]
        rank = Y.shape[1]
        # extract the p leading pairs of (Q_c, Sigma_c) and (Y, w)
        allv = np.hstack([Qc, Y])
        allw = np.concatenate([Sc, w])
        order = np.argsort(-allw, kind="stable")[:p]
        Xall, mu = allv[:, order], allw[order]
        padded = Xall.shape[1] < p  # mu_{k+q} of a padding column is no estimate of b
        Xall, mu = pad_ritz(B, Xall, mu, p, pad_pool)
        lam = to_orig(mu)
        res = residual_norms(B, Xall, mu, lam)
        n_spmm_cols += p
        maxres = float(np.max(res[:k]))
        if maxres < best:
            best, best_iter = maxres, j
            mu_best = (float(mu[k - 1]), float(mu[p - 1]))  # the most accurate Ritz values so far
        rec = OuterRecord(nf, rcs, maxres, tol_t, b, Qc.shape[1], rank, q, degree)
        history.append(rec)
        # outer stop rules (eq. out-stop and cases (i)-(iii))
        h = int(np.sum(res[:k] < 0.1 * tol))
        if maxres <= tol:
            stop_reason = "converged"
            break
        if maxres < (1.0 + 9.0 * h / k) * tol:
            stop_reason = "near_tol"
            break
        if j - best_iter >= 3:
            stop_reason = "stalled"
            break
        # continuation (eq. contin)
        if maxres <= tol_t:
            tol_t = max(1e-2 * tol_t, tol)
            b = float(mu[p - 1]) if not padded else b
        elif b_update == "every_arr":
            b = float(mu[p - 1]) if not padded else b
        # deflation (eq. defl)
        thr = max(1e-14, tol_t ** 2)
        lock = np.zeros(p, dtype=bool)
        lock[:k] = res[:k] <= thr
        Qc, Sc = Xall[:, lock], mu[lock]
        X = Xall[:, ~lock]
        if X.shape[1] == 0:
            stop_reason = "all_locked"
            break
        # augmentation blocks (eq. block): small decay of the relevant Ritz values of the
        # shifted operator B - aI the inner solver works on, and a disappointing decrease
        # of the residuals
        if adapt_q and maxres_prev is not None and q < q_cap:
            if (mu[p - 1] - a) / (mu[k - 1] - a) > 0.95 and maxres / maxres_prev > 0.1:
                q += 1
        maxres_prev = maxres
        # polynomial degree (eqs. hat-d, degree) from the most accurate Ritz values so far
        if adapt_d and mu_best is not None:
            degree = next_degree(filter_kind, mu_best[0], mu_best[1], a, b, d_max)
    # report the k leading pairs in the original problem's terms
    Xk = Xall[:, :k]
    lam_rq = np.einsum("ij,ij->j", Xk, A @ Xk)
    if which == "smallest":
        order = np.argsort(lam_rq, kind="stable")
    else:
        order = np.argsort(-lam_rq, kind="stable")
    Xk = Xk[:, order]
    lam_rq = lam_rq[order]
    res_k = res[:k][order]
    # sign convention: largest-magnitude entry of each vector positive
    idx = np.argmax(np.abs(Xk), axis=0)
    sgn = np.sign(Xk[idx, np.arange(k)])
    sgn[sgn == 0] = 1.0
    Xk = Xk * sgn[None, :]
    return OracleResult(evals=lam_rq, evecs=Xk, res=res_k, maxres=float(np.max(res_k)),
                        converged=stop_reason in ("converged", "near_tol"),
                        stop_reason=stop_reason, outer_iters=j, n_spmm_cols=int(n_spmm_cols),
                        a=a, b0=b0, sigma=float(sigma), history=history)
