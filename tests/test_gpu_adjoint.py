"""The transpose (adjoint) side on the GPU: eta^A vectors, the left-hand (Y) response route and
alpha "from both sides", and the adjoint product at the o=24, v=160, naux=800 workload.

* eta^A = dE_A/dT + lambda A[mu^A] against the oracle's eta_vec (Jacobians of f + mu^A and f).
* cc_lr_solve_left (Y^B(w) (A + w) = -(eta^B + F X^B(w)), g = Y^B . xi^A + eta^A . X^B) equals
  cc_lr_solve (X-only route) and the oracle's alpha, in FP64 and in the mixed modes.
* o=24, v=160: Y A from the autograd wrapper's backward against central finite differences
  (h = 1e-5) of the forward sigma along a random direction, the Lambda solve, and alpha from
  both sides at Cholesky scale 0.06 (the synthetic integrals need a scale for the solves to
  converge).
"""
import numpy as np
import pytest
import torch

from oracle import response as R
from oracle.integrals import as_t
from paper_2604_12914_gb300.inputs import make_config, make_system, random_amplitudes

from gpu_helpers import gpu_context, oracle_setup, rel_err

pytestmark = pytest.mark.gpu


def _converged_small(o=3, v=8, naux=12, seed=5, scale=0.2):
    s = make_system(o, v, naux, seed=seed, scale=scale)
    f, g, L, _, _ = oracle_setup(s, np.zeros((o, v)), np.zeros((o, o, v, v)))
    t1, t2, _ = R.solve_ccsd(f, g, o, L=L)
    return s, R.Problem(f, g, L, o, t1, t2)


def test_eta_vectors_match_oracle():
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy())
    A = P.jacobian_matrix()
    lam = torch.linalg.solve(A.transpose(0, 1), -P.eta0())
    for comp in range(3):
        e1, e2 = ctx.cc_lr_eta(comp, tol=1e-12)
        r1, r2 = P.unpack(P.eta_vec(as_t(s.mu[comp]), lam))
        err = rel_err(e1, e2, r1.numpy(), r2.numpy())
        print(f"eta^{comp}: relative error {err:.2e}")
        assert err < 1e-9
    ctx.close()


@pytest.mark.parametrize("prec,method", [("fp64", "gmres"), ("fp64", "block"), ("tf32", "gmres"), ("bf16x3", "block")])
def test_alpha_from_both_sides(prec, method):
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy(), prec=prec)
    ctx.cc_lr_set_solver(method)
    if prec != "fp64":
        ctx.cc_lr_set_refinement("3xtf32")
    # 3xTF32 refinement residuals floor near 5e-7 relative (complex64 data, FP32 accumulation)
    tol = 1e-11 if prec == "fp64" else 1e-6
    for omega in (0.0, 0.0428):
        ar, _ = ctx.cc_lr_solve([omega], (0, 1, 2), tol=tol)
        al, st = ctx.cc_lr_solve_left([omega], (0, 1, 2), tol=tol)
        ref = R.alpha(P, [as_t(m) for m in s.mu], omega).numpy()
        d_lr = np.abs(al[0] - ar[0]).max()
        d_ref = np.abs(al[0] - ref).max()
        print(f"{prec}/{method} omega={omega}: |alpha_left - alpha_right| {d_lr:.2e}, |alpha_left - oracle| {d_ref:.2e}")
        lim = 1e-7 * np.abs(ref).max() if prec == "fp64" else 1e-4
        assert d_lr < lim and d_ref < lim
        assert st["converged"] == 1
    ctx.close()


@pytest.fixture(scope="module")
def c4sys():
    return make_config("C4", seed=4)


@pytest.mark.parametrize("prec,h,tol", [("fp64", 1e-5, 1e-8), ("3xtf32", 1.0, 5e-5), ("tf32", 1.0, 3e-3)])
def test_c4_adjoint_vs_finite_differences(c4sys, prec, h, tol):
    """Y A through SigmaFn.backward against the central difference of L(X) = Re <W, sigma(X)>
    along a random direction E, at o=24, v=160, naux=800.  sigma is linear in X, so the central
    difference is exact for any step: h = 1e-5 in FP64; in complex64 the rounding of sigma(X)
    (about 1e-7 relative) would swamp a step that small, so h = 1 there."""
    from paper_2604_12914_gb300 import binding
    from paper_2604_12914_gb300.autograd import sigma as sigma_fn
    s = c4sys
    dev = torch.device("cuda")
    ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec=prec)
    x1, x2 = (torch.tensor(a, device=dev) for a in random_amplitudes(s.o, s.v, seed=31))
    e1, e2 = (torch.tensor(a, device=dev) for a in random_amplitudes(s.o, s.v, seed=32))
    w1, w2 = (torch.tensor(a, device=dev) for a in random_amplitudes(s.o, s.v, seed=33))

    def loss(p1, p2):
        s1, s2 = sigma_fn(ctx, p1, p2)
        return (w1 * s1).sum().real + 0.25 * (w2 * s2).sum().real

    z1 = x1.clone().requires_grad_(True)
    z2 = x2.clone().requires_grad_(True)
    loss(z1, z2).backward()
    # directional derivative from the gradient: d/dh L(X + h E) = Re <grad*, E> (PyTorch's
    # convention for a real function of complex inputs), doubles through the same weights
    g1, g2 = z1.grad, z2.grad
    dd_grad = float((torch.conj(g1) * e1).sum().real + (torch.conj(g2) * e2).sum().real)
    with torch.no_grad():
        fd = (float(loss(x1 + h * e1, x2 + h * e2)) - float(loss(x1 - h * e1, x2 - h * e2))) / (2 * h)
    print(f"C4 {prec}: adjoint {dd_grad:.10e} vs central difference {fd:.10e}")
    assert abs(dd_grad - fd) <= tol * abs(fd)
    ctx.close()


def test_c4_lambda_and_alpha_from_both_sides(c4sys):
    """o=24, v=160: the Lambda equations (transpose products) and alpha by the X-only and the
    left-hand routes, mixed precision (TF32 corrections, 3xTF32 residuals, FP64 vectors)."""
    s = make_config("C4", seed=4, scale=0.06)
    from paper_2604_12914_gb300 import binding
    ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec="tf32")
    ctx.cc_lr_set_refinement("3xtf32")
    ctx.cc_lr_set_solver("block")
    ar, st_r = ctx.cc_lr_solve([0.0428], (2,), tol=1e-6)
    al, st_l = ctx.cc_lr_solve_left([0.0428], (2,), tol=1e-6)
    d = abs(al[0, 0, 0] - ar[0, 0, 0])
    print(f"C4 alpha_zz right {ar[0, 0, 0]:.8f} left {al[0, 0, 0]:.8f} |d| {d:.2e}; right {st_r}; left {st_l}")
    assert st_r["converged"] == 1 and st_l["converged"] == 1
    assert d < 1e-4
    ctx.close()


@pytest.mark.parametrize("prec,tol_alpha", [("fp64", 1e-8), ("tf32", 1e-5)])
def test_alpha_to_absolute_tolerance(prec, tol_alpha):
    """cc_lr_solve_alpha_tol: solves tightened until the left- and right-route alphas agree within
    tol_alpha; the result then agrees with the oracle's alpha (which shares no code) within the
    1e-4 a.u. target, and the estimate is below tol_alpha."""
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy(), prec=prec)
    if prec != "fp64":
        ctx.cc_lr_set_refinement("3xtf32")
    al, est, st = ctx.cc_lr_solve_alpha_tol([0.0428], (0, 1, 2), tol_alpha=tol_alpha)
    ref = R.alpha(P, [as_t(m) for m in s.mu], 0.0428).numpy()
    err = np.abs(al[0] - ref).max()
    print(f"{prec}: tol_alpha {tol_alpha:.0e}: estimate {est:.2e}, |alpha - oracle| {err:.2e}, {st}")
    assert est < tol_alpha
    assert err < (1e-6 * np.abs(ref).max() if prec == "fp64" else 1e-4)
    ctx.close()
