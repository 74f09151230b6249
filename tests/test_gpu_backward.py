"""Backward kernel (jacobi_eig_backward) and the autograd.Function, against the oracle's
reference gradient and central finite differences of the GPU forward map.

Workload shape: H = G G^T + 0.1 I (SPD), loss = sum_i w_i lambda_i + ||U[:, :k]^T C||^2 with
seeded w and C; the solver runs on the Cholesky factor of H (preprocessing on the host, as the
paper factors H before the Jacobi sweeps).  Tolerances: the GPU H_bar matches the oracle's
(computed from the oracle's own eigenpairs) to 1e-9 relative; finite differences
(h = 1e-6, FP64) to 1e-5 relative.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _spd(n, g):
    G = g.standard_normal((n, n))
    return G @ G.T + 0.1 * np.eye(n)


def _forward(Hs, dev, J=None, k=4):
    """GPU eigenpairs of each H (batch, n, n) through the Cholesky factor."""
    import torch

    from paper_1008_0201_gb300 import binding

    L = np.stack([np.linalg.cholesky(H) for H in Hs])
    out = binding.jacobi_eig_batched_uniform(torch.from_numpy(L).to(dev), J, binding.default_opts(want_v=0))
    torch.cuda.synchronize()
    return out["lam"], out["U"]


def _loss_grads(lam, U, w, C, k):
    import torch

    Uk = U[..., :k]
    loss = (lam * w).sum() + ((Uk.transpose(-1, -2) @ C) ** 2).sum()
    lam_bar = w.expand_as(lam).clone()
    U_bar = torch.zeros_like(U)
    U_bar[..., :k] = 2.0 * C @ (C.transpose(-1, -2) @ Uk)
    return loss, lam_bar, U_bar


def test_backward_matches_oracle_gradient(cuda_dev):
    import torch

    import oracle
    from paper_1008_0201_gb300 import binding

    g = np.random.default_rng(31)
    n, batch, k = 40, 3, 4
    Hs = np.stack([_spd(n, g) for _ in range(batch)])
    w = torch.from_numpy(g.standard_normal(n)).to(cuda_dev)
    C = torch.from_numpy(g.standard_normal((n, 2))).to(cuda_dev)
    lam, U = _forward(Hs, cuda_dev)
    _, lam_bar, U_bar = _loss_grads(lam, U, w, C, k)
    Hb, _ = binding.jacobi_eig_backward(lam, U, lam_bar, U_bar)
    Hb = Hb.cpu().numpy()
    for b in range(batch):
        assert np.array_equal(Hb[b], Hb[b].T)
        # oracle gradient from the oracle's own eigenpairs
        ref = oracle.solve(np.linalg.cholesky(Hs[b]), np.ones(n, dtype=np.int8))
        lr, Ur = ref["lam"], ref["U"]
        Urk = Ur[:, :k]
        Cn = C.cpu().numpy()
        Ubr = np.zeros_like(Ur)
        Ubr[:, :k] = 2.0 * Cn @ (Cn.T @ Urk)
        Hr = oracle.eig_backward(lr, Ur, w.cpu().numpy(), Ubr)
        err = np.linalg.norm(Hb[b] - Hr) / np.linalg.norm(Hr)
        assert err <= 1e-9, err


def test_backward_finite_differences(cuda_dev):
    import torch

    from paper_1008_0201_gb300 import binding

    g = np.random.default_rng(32)
    n, k = 24, 3
    H = _spd(n, g)
    w = torch.from_numpy(g.standard_normal(n)).to(cuda_dev)
    C = torch.from_numpy(g.standard_normal((n, 2))).to(cuda_dev)
    lam, U = _forward(H[None], cuda_dev)
    _, lam_bar, U_bar = _loss_grads(lam, U, w, C, k)
    Hb = binding.jacobi_eig_backward(lam, U, lam_bar, U_bar)[0][0].cpu().numpy()
    h = 1e-6
    Es = []
    for _ in range(6):
        E = g.standard_normal((n, n))
        E = (E + E.T) / 2
        Es.append(E / np.linalg.norm(E))
    Hp = np.stack([H + h * E for E in Es] + [H - h * E for E in Es])
    lp, Up = _forward(Hp, cuda_dev)
    for i, E in enumerate(Es):
        Lp = _loss_grads(lp[i], Up[i], w, C, k)[0].item()
        Lm = _loss_grads(lp[i + len(Es)], Up[i + len(Es)], w, C, k)[0].item()
        fd = (Lp - Lm) / (2 * h)
        got = float(np.sum(Hb * E))
        assert abs(got - fd) <= 1e-5 * max(1.0, abs(fd)), (got, fd)


def test_backward_diagonal_closed_form(cuda_dev):
    """H diagonal: U is a permutation and, with U_bar = 0, H_bar = lambda_bar on the diagonal
    positions of the sorted eigenvalues (dlambda_i/dH = e_i e_i^T)."""
    import torch

    from paper_1008_0201_gb300 import binding

    d = np.array([4.0, 1.0, 9.0, 2.25, 6.25, 0.5])
    lam, U = _forward(np.diag(d)[None], cuda_dev)
    lam_bar = torch.tensor([[0.5, -2.0, 1.0, 3.0, -0.75, 2.0]], dtype=torch.float64, device=cuda_dev)
    Hb = binding.jacobi_eig_backward(lam, U, lam_bar, None)[0][0].cpu().numpy()
    order = np.argsort(d)
    want = np.zeros((6, 6))
    for i, p in enumerate(order):
        want[p, p] = lam_bar[0, i].item()
    assert np.allclose(Hb, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("hyperbolic", [False, True])
def test_autograd_factor_finite_differences(cuda_dev, hyperbolic):
    """G_bar from the autograd.Function (J-adjusted: 2 H_bar G J) against finite differences
    of the loss with respect to the factor itself."""
    import torch

    from paper_1008_0201_gb300 import autograd

    g = np.random.default_rng(33 + int(hyperbolic))
    n, batch, k = 20, 2, 3
    G = torch.from_numpy(g.standard_normal((batch, n, n)) + 3.0 * np.eye(n)).to(cuda_dev)
    J = None
    if hyperbolic:
        Jn = np.ones((batch, n), dtype=np.int8)
        Jn[:, g.choice(n, size=6, replace=False)] = -1
        J = torch.from_numpy(Jn).to(cuda_dev)
    w = torch.from_numpy(g.standard_normal(n)).to(cuda_dev)
    C = torch.from_numpy(g.standard_normal((n, 2))).to(cuda_dev)

    def loss_of(Gx):
        lam, U = autograd.eigh_factor(Gx, J)
        return _loss_grads(lam, U, w, C, k)[0]

    Gv = G.clone().requires_grad_(True)
    loss_of(Gv).backward()
    Gbar = Gv.grad.cpu().numpy()
    h = 1e-6
    for _ in range(4):
        E = g.standard_normal((batch, n, n))
        E /= np.linalg.norm(E)
        Et = torch.from_numpy(E).to(cuda_dev)
        with torch.no_grad():
            fd = (loss_of(G + h * Et).item() - loss_of(G - h * Et).item()) / (2 * h)
        got = float(np.sum(Gbar * E))
        assert abs(got - fd) <= 1e-5 * max(1.0, abs(fd)), (got, fd)


def test_backward_full_size_sampled(cuda_dev):
    """The differentiation workload at full size (256 problems of order 256): every H_bar is
    exactly symmetric and finite; two sampled problems match the oracle gradient."""
    import torch

    import oracle
    from paper_1008_0201_gb300 import binding, inputs

    G, w_np, C_np = inputs.config5_backward()
    batch, n, _ = G.shape
    k = 8
    Hs = np.einsum("bij,bkj->bik", G, G) + 0.1 * np.eye(n)
    w = torch.from_numpy(w_np).to(cuda_dev)
    C = torch.from_numpy(C_np).to(cuda_dev)
    lam, U = _forward(Hs, cuda_dev)
    _, lam_bar, U_bar = _loss_grads(lam, U, w, C, k)
    Hb, _ = binding.jacobi_eig_backward(lam, U, lam_bar, U_bar)
    torch.cuda.synchronize()
    assert torch.isfinite(Hb).all()
    assert torch.equal(Hb, Hb.transpose(-1, -2))
    Hb = Hb.cpu().numpy()
    for b in (0, 201):
        ref = oracle.solve(np.linalg.cholesky(Hs[b]), np.ones(n, dtype=np.int8))
        Ur = ref["U"]
        Ubr = np.zeros_like(Ur)
        Ubr[:, :k] = 2.0 * C_np @ (C_np.T @ Ur[:, :k])
        Hr = oracle.eig_backward(ref["lam"], Ur, w_np, Ubr)
        err = np.linalg.norm(Hb[b] - Hr) / np.linalg.norm(Hr)
        assert err <= 1e-9, (b, err)


def test_backward_kernel_vs_oracle_same_inputs(cuda_dev):
    """The backward kernel alone: the oracle's backward applied to the GPU's own eigenpairs must
    give the GPU's H_bar to FP64 product accuracy (the n x n products run as FP16 digit products;
    n = 150 leaves ragged 64 x 32 tiles)."""
    import torch

    import oracle
    from paper_1008_0201_gb300 import binding

    g = np.random.default_rng(47)
    n, batch, k = 150, 2, 5
    Hs = np.stack([_spd(n, g) for _ in range(batch)])
    w = torch.from_numpy(g.standard_normal(n)).to(cuda_dev)
    C = torch.from_numpy(g.standard_normal((n, 3))).to(cuda_dev)
    lam, U = _forward(Hs, cuda_dev)
    _, lam_bar, U_bar = _loss_grads(lam, U, w, C, k)
    Hb, _ = binding.jacobi_eig_backward(lam, U, lam_bar, U_bar)
    Hb = Hb.cpu().numpy()
    for b in range(batch):
        Hr = oracle.eig_backward(lam[b].cpu().numpy(), U[b].cpu().numpy(), lam_bar[b].cpu().numpy(),
                                 U_bar[b].cpu().numpy())
        err = np.linalg.norm(Hb[b] - Hr) / np.linalg.norm(Hr)
        assert err <= 1e-12, err
