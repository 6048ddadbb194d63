"""Differentiation form: x = A(theta)^{-1} b with loss 1/2 ||x||^2 on the
parameterised 7-point diffusion-advection operator.  The library backward
(transposed solve through the stored factors + gradient gather) is checked
against a dense torch autograd gradient on a 6^3 copy and against central
finite differences (step 1e-6, 64 random directions) on the 32^3 operator."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
S = pytest.importorskip("paper_2512_04389_b300.slu")
from paper_2512_04389_b300.autograd import lu_solve  # noqa: E402


def _dev(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def test_gradient_matches_dense_autograd_6cube():
    s = workloads.grid7_theta(6)
    P = S.Plan(s.n, s.colptr, s.rowidx, b_min=8)
    v = _dev(s.values).requires_grad_(True)
    b = _dev(s.rhs[:, 0]).requires_grad_(True)
    x = lu_solve(v, b, P)
    (0.5 * (x * x).sum()).backward()
    # dense reference with torch autograd
    rows = torch.as_tensor(s.rowidx.astype(np.int64), device="cuda")
    cols = torch.as_tensor(np.repeat(np.arange(s.n), np.diff(s.colptr)),
                           device="cuda")
    v2 = _dev(s.values).requires_grad_(True)
    b2 = _dev(s.rhs[:, 0]).requires_grad_(True)
    A = torch.zeros((s.n, s.n), dtype=torch.float64, device="cuda")
    A = A.index_put((rows, cols), v2)
    x2 = torch.linalg.solve(A, b2)
    (0.5 * (x2 * x2).sum()).backward()
    assert torch.allclose(x, x2, rtol=1e-12, atol=1e-14)
    gv, gv2 = v.grad, v2.grad
    assert (gv - gv2).abs().max() <= 1e-10 * gv2.abs().max()
    assert (b.grad - b2.grad).abs().max() <= 1e-10 * b2.grad.abs().max()


def test_gradient_central_differences_32cube():
    s = workloads.grid7_theta(32)
    P = S.Plan(s.n, s.colptr, s.rowidx)
    v0 = _dev(s.values)
    b0 = _dev(s.rhs[:, 0])
    v = v0.clone().requires_grad_(True)
    b = b0.clone().requires_grad_(True)
    x = lu_solve(v, b, P)
    (0.5 * (x * x).sum()).backward()
    F = S.Factor(P, v0)

    def loss(vals, rhs):
        F.refactor(vals)
        y = F.solve(rhs)
        return 0.5 * float((y * y).sum())

    rng = np.random.default_rng(11)
    h = 1e-6
    worst = 0.0
    for _ in range(64):
        d = _dev(rng.standard_normal(s.values.size))
        d *= v0.abs()                      # relative perturbation per entry
        fd = (loss(v0 + h * d, b0) - loss(v0 - h * d, b0)) / (2 * h)
        an = float((v.grad * d).sum())
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-30))
    assert worst <= 1e-5
    for _ in range(4):
        db = _dev(rng.standard_normal(s.n))
        fd = (loss(v0, b0 + h * db) - loss(v0, b0 - h * db)) / (2 * h)
        an = float((b.grad * db).sum())
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_multiple_rhs_gradient():
    s = workloads.grid7_theta(6, nrhs=3)
    P = S.Plan(s.n, s.colptr, s.rowidx, b_min=8)
    v = _dev(s.values).requires_grad_(True)
    B = _dev(s.rhs).requires_grad_(True)
    X = lu_solve(v, B, P)
    (X.sum() + 0.5 * (X * X).sum()).backward()
    A = np.zeros((s.n, s.n))
    A[s.rowidx, np.repeat(np.arange(s.n), np.diff(s.colptr))] = s.values
    Xd = np.linalg.solve(A, s.rhs)
    G = 1.0 + Xd
    Lam = np.linalg.solve(A.T, G)
    cols = np.repeat(np.arange(s.n), np.diff(s.colptr))
    gref = -(Lam[s.rowidx] * Xd[cols]).sum(1)
    assert np.abs(v.grad.cpu().numpy() - gref).max() <= 1e-10 * np.abs(gref).max()
    assert np.abs(B.grad.cpu().numpy() - Lam).max() <= 1e-10 * np.abs(Lam).max()
