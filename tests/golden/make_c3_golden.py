"""Writes the oracle's eigenvalues of the full-size graded complex workload (test fixture).

Workload: G = B D, n = 4096, B complex Gaussian (re, im i.i.d. N(0, 1/2)) drawn from the seeded
generator of ``paper_1008_0201_gb300.inputs.config3_graded_complex``, D = diag(10^(-8 i / n)),
J = I, so H = G G^* is positive definite and the one-sided method diagonalizes the graded
A = G^* G (Sec. 2.1).  The oracle (sequential row-cyclic one-sided Jacobi in FP64, Sec. 2.1 with
the complex rotation of Eq. (2.1)) runs once on the CPU; this takes about half an hour, so its
result is stored and keyed by a hash of the Gaussian draws B (the grading D is recomputed by
the reader: a last-bit difference in 10^x between platforms changes no eigenvalue beyond the
tolerance).

Only ``oracle/`` computes the eigenvalues.  kappa_2(B_hat) (B with unit columns), which sets the
tolerance 50 n eps kappa_2(B_hat) (and kappa_2(A) = kappa_2(B_hat)^2 for the looser one), is a
LAPACK singular value computation, a library primitive.

Usage:  python tests/golden/make_c3_golden.py [n]     (default n = 4096)
Output: tests/golden/c3_graded_complex_n<n>.txt
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1008_0201_gb300 import inputs  # noqa: E402


def draws_hash(G, n):
    """sha256 of the Gaussian draws B = G D^-1, recomputed from the generator (not from G)."""
    g = inputs.rng(3, 0)
    re = g.standard_normal((n, n))
    im = g.standard_normal((n, n))
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(re).tobytes())
    h.update(np.ascontiguousarray(im).tobytes())
    return h.hexdigest()


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 4096
    G, J = inputs.config3_graded_complex(n)
    digest = draws_hash(G, n)
    Bh = G / np.linalg.norm(G, axis=0)
    s = np.linalg.svd(Bh, compute_uv=False)
    kappa_bhat = float(s[0] / s[-1])
    t0 = time.time()
    ref = oracle.solve(G, J, want_v=False)
    secs = time.time() - t0
    if ref["status"] != 0:
        raise SystemExit("oracle did not converge: status %d" % ref["status"])
    off_rel, max_scaled = oracle.check_offdiag(ref["Gf"])
    path = os.path.join(HERE, "c3_graded_complex_n%d.txt" % n)
    with open(path + ".tmp", "w") as f:
        f.write("# Oracle eigenvalues of the graded complex workload G = B D, n = %d, J = I\n" % n)
        f.write("# (sequential row-cyclic one-sided Jacobi, FP64, Sec. 2.1 / Eq. (2.1)); ascending.\n")
        f.write("# written by tests/golden/make_c3_golden.py\n")
        f.write("n %d\n" % n)
        f.write("draws_sha256 %s\n" % digest)
        f.write("kappa2_bhat %.17g\n" % kappa_bhat)
        f.write("oracle_sweeps %d\n" % ref["sweeps"])
        f.write("oracle_rotations %d\n" % ref["rotations"])
        f.write("oracle_seconds %.1f\n" % secs)
        f.write("oracle_off_rel %.6g\n" % off_rel)
        f.write("oracle_max_scaled %.6g\n" % max_scaled)
        f.write("lambda\n")
        for v in ref["lam"]:
            f.write("%.17g\n" % v)
    os.replace(path + ".tmp", path)
    print("wrote", path, "sweeps", ref["sweeps"], "seconds %.1f" % secs)


if __name__ == "__main__":
    main()
