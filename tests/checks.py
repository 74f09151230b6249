"""Shared comparison helpers for the GPU-vs-oracle tests (tolerances stated once here).

Tolerances (eps = 2^-53, n = order):
  eigenvalues      |lam - lam_oracle| / |lam_oracle| <= 50 n eps kappa2(A)
  off-norm         off_F(G^T G) / ||G||_F^2 <= n eps        (returned G, long double)
  J-unitarity      ||V^T J V - J_out||_F <= 100 n eps
  factor residual  ||G0 V - G||_F / ||G0||_F <= 100 n eps
  eigenvectors     sin angle(u, u_oracle) <= 50 n eps kappa2(A) / relgap (+ 1e-14 floor)
with A = D^-1 G^T G D^-1 (D = column norms), i.e. kappa2(A) = kappa2(G with unit columns)^2,
the scaled matrix the one-sided method diagonalizes.
"""
import numpy as np

import oracle

EPS = 2.0 ** -53


def kappa_A(G):
    B = G / np.linalg.norm(G, axis=0)
    s = np.linalg.svd(B, compute_uv=False)
    return (s[0] / s[-1]) ** 2


def compare(G0, J, out, ref=None, check_vectors=True, kappa=None):
    """Checks a GPU result dict (lam, G, U, V as numpy) against the oracle; returns metrics."""
    m, n = G0.shape
    if ref is None:
        ref = oracle.solve(G0, J)
    assert ref["status"] == 0
    if kappa is None:
        kappa = kappa_A(G0)
    lam = out["lam"]
    rel = np.max(np.abs(lam - ref["lam"]) / np.abs(ref["lam"]))
    bound_lam = 50 * n * EPS * kappa
    assert rel <= bound_lam, ("eigenvalue error", rel, bound_lam)
    off_rel, max_scaled = oracle.check_offdiag(out["G"])
    assert off_rel <= n * EPS, ("off-norm", off_rel, n * EPS)
    res = {"eig_rel": rel, "eig_bound": bound_lam, "off_rel": off_rel, "max_scaled": max_scaled}
    J_out = np.where(lam < 0, -1, 1).astype(np.int8)
    if out.get("V") is not None:
        V = out["V"]
        vjv = oracle.check_vjv(V, J, J_out)
        assert vjv <= 100 * n * EPS, ("V^T J V - J", vjv, 100 * n * EPS)
        resid = oracle.check_factor_residual(G0, V, out["G"])
        assert resid <= 100 * n * EPS, ("G0 V - G", resid)
        res.update(vjv=vjv, resid=resid)
    if check_vectors and out.get("U") is not None:
        U = out["U"]
        Ur = ref["U"]
        lr = ref["lam"]
        worst = 0.0
        for i in range(n):
            gaps = np.abs(lr - lr[i]) / np.abs(lr[i])
            gaps[i] = np.inf
            relgap = gaps.min()
            u = U[:, i] / np.linalg.norm(U[:, i])
            v = Ur[:, i] / np.linalg.norm(Ur[:, i])
            s = np.linalg.norm(u - np.dot(u, v) * v)  # sin of the angle, no 1 - cos^2 cancellation
            bound = 50 * n * EPS * kappa / relgap + 1e-14
            assert s <= bound, ("eigenvector", i, s, bound)
            worst = max(worst, s * relgap / (50 * n * EPS * kappa))
        res["vec_frac_of_bound"] = worst
    return res


def to_np(out):
    o = dict(out)
    for k in ("lam", "G", "U", "V"):
        if o.get(k) is not None:
            o[k] = o[k].detach().cpu().numpy()
    return o
