"""Shared comparison helpers for the GPU-vs-oracle tests (tolerances stated once here).

Tolerances (eps = 2^-53, n = order):
  eigenvalues      |lam - lam_oracle| / |lam_oracle| <= 50 n eps kappa2(A)
  off-norm         off_F(G^T G) / ||G||_F^2 <= n eps        (returned G, long double)
  J-unitarity      ||V^T J V - J_out||_F <= 100 n eps max(1, ||V||_2^2)
  factor residual  ||G0 V - G||_F / ||G0||_F <= 100 n eps max(1, ||V||_2)
  eigenvectors     sin angle(u, u_oracle) <= 50 n eps kappa2(A) / relgap (+ 1e-14 floor)
with A = D^-1 G^T G D^-1 (D = column norms), i.e. kappa2(A) = kappa2(G with unit columns)^2,
the scaled matrix the one-sided method diagonalizes.  V is orthogonal for J = I (||V||_2 = 1);
a J-unitary V can be large when the factor has nearly parallel columns of opposite sign, and
the rounding errors of its products (and of the oracle's own V) grow with ||V||_2^2.

Results of the FP32-only sweeps are held to the same bounds with eps = 2^-24, except the
off-norm: its threshold is the FP32 rotation tolerance max(n, 8 sqrt(m)) eps_32 (an FP32 Gram of
m rows resolves scaled off-diagonals down to ~eps_32 sqrt(m)), doubled for the Gram's own error.
"""
import numpy as np

import oracle

EPS = 2.0 ** -53
EPS32 = 2.0 ** -24


def kappa_A(G):
    B = G / np.linalg.norm(G, axis=0)
    s = np.linalg.svd(B, compute_uv=False)
    return (s[0] / s[-1]) ** 2


def compare(G0, J, out, ref=None, check_vectors=True, kappa=None, eps=EPS):
    """Checks a GPU result dict (lam, G, U, V as numpy) against the oracle; returns metrics.
    eps = EPS32 checks a result of the FP32-only sweeps."""
    m, n = G0.shape
    off_bound = n * eps if eps == EPS else 2.0 * max(n, 8.0 * np.sqrt(m)) * eps
    if ref is None:
        ref = oracle.solve(G0, J)
    assert ref["status"] == 0
    if kappa is None:
        kappa = kappa_A(G0)
    lam = out["lam"]
    rel = np.max(np.abs(lam - ref["lam"]) / np.abs(ref["lam"]))
    bound_lam = 50 * n * eps * kappa
    assert rel <= bound_lam, ("eigenvalue error", rel, bound_lam)
    off_rel, max_scaled = oracle.check_offdiag(out["G"])
    assert off_rel <= off_bound, ("off-norm", off_rel, off_bound)
    res = {"eig_rel": rel, "eig_bound": bound_lam, "off_rel": off_rel, "max_scaled": max_scaled}
    J_out = np.where(lam < 0, -1, 1).astype(np.int8)
    if out.get("V") is not None:
        V = out["V"]
        nv = np.linalg.norm(V, 2)
        vjv = oracle.check_vjv(V, J, J_out)
        assert vjv <= 100 * n * eps * max(1.0, nv * nv), ("V^T J V - J", vjv, 100 * n * eps, nv)
        resid = oracle.check_factor_residual(G0, V, out["G"])
        assert resid <= 100 * n * eps * max(1.0, nv), ("G0 V - G", resid, nv)
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
            s = np.linalg.norm(u - np.vdot(v, u) * v)  # sin of the angle (any complex phase)
            bound = 50 * n * eps * kappa / relgap + 1e-14
            assert s <= bound, ("eigenvector", i, s, bound)
            if np.isfinite(relgap):
                worst = max(worst, s * relgap / (50 * n * eps * kappa))
        res["vec_frac_of_bound"] = worst
    return res


def to_np(out):
    o = dict(out)
    for k in ("lam", "G", "U", "V"):
        if o.get(k) is not None:
            o[k] = o[k].detach().cpu().numpy()
    return o
