"""Write tests/golden/*.json from the CPU oracle only (run from the repository root:
``python tests/golden/make_golden.py``).  Stored values are the oracle's; the tests that
read them also check them against closed forms."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import arrabit_oracle as O  # noqa: E402
from paper_1507_06078_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    coefs = {str(d): O.interpolant_cheb_coeffs(d).tolist() for d in (3, 6, 10, 15, 20)}
    with open(os.path.join(HERE, "interpolant_coeffs.json"), "w") as f:
        json.dump({"source": "oracle.interpolant_cheb_coeffs (Section 5, eq. chebfun-f)",
                   "coeffs": coefs}, f, indent=1)
    W = I.workload_2d64()
    A = O.csr_to_scipy(W.A.n, W.A.rowptr, W.A.col, W.A.val)
    X0 = I.gaussian_block(W.A.n, W.p, W.seed)
    r = O.arrabit_mpm(A, W.k, X0, which=W.which, tol=W.tol, q=W.q, degree=W.degree)
    out = {"source": "oracle.arrabit_mpm (Algorithm 8, MPM) on " + W.name,
           "k": W.k, "p": W.p, "q": W.q, "degree": W.degree, "tol": W.tol, "seed": W.seed,
           "evals": r.evals.tolist(), "maxres": r.maxres, "outer_iters": r.outer_iters,
           "a": r.a, "b0": r.b0, "sigma": r.sigma, "stop_reason": r.stop_reason}
    with open(os.path.join(HERE, "laplace2d_64_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
