"""GPU ground-state CCSD (Sec. 2.2: amplitude equations and energy) against the CPU oracle.

The library forms Omega(T) from two Jacobian products at the Gauss-Legendre nodes of [0, 1]
(exact: Omega(sT) is quartic in s) and E(T) over packed amplitudes; the oracle evaluates the
residual and energy term by term (pinned against brute-force second quantisation).
Tolerances, relative to max |Omega|: FP64 1e-10; 3xTF32 5e-5; bf16x3 5e-4 (the sigma-product
accuracies of those modes).  The energy never goes through a sigma product: 1e-12 in every mode.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd, response as R
from oracle.integrals import as_t
from paper_2604_12914_gb300.inputs import make_system, random_amplitudes

from gpu_helpers import gpu_context, oracle_setup

pytestmark = pytest.mark.gpu

CASES = [
    # (o, v, naux, seed, scale, t1_scale)
    (2, 4, 6, 1, 0.5, 0.2),
    (5, 13, 21, 2, 0.6, 0.1),
    (3, 67, 40, 3, 0.4, 0.05),     # two 64-wide tiles with a ragged tail
    (10, 40, 200, 1, 0.3, 0.05),   # o=10, v=40, naux=200
]
TOL = {"fp64": 1e-10, "3xtf32": 5e-5, "bf16x3": 5e-4}


def _amps(s, seed, t1_scale):
    a1, a2 = random_amplitudes(s.o, s.v, seed=seed, s1=0.2, s2=0.2)
    return a1 * (t1_scale / 0.2), a2


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "bf16x3"])
@pytest.mark.parametrize("case", CASES)
def test_residual_and_energy_match_oracle(case, prec):
    o, v, naux, seed, scale, t1s = case
    s = make_system(o, v, naux, seed=seed, scale=scale)
    t1, t2 = _amps(s, seed + 50, t1s)
    f, g, L, T1, T2 = oracle_setup(s, t1, t2)
    r1, r2 = (x.numpy() for x in ccsd.residual(f, g, T1, T2))
    e = complex(ccsd.energy(f, g, T1, T2))
    ctx = gpu_context(s, t1=t1, t2=t2, prec=prec)
    g1, g2, ge = ctx.cc_lr_ccsd_residual(t1, t2)
    sc = max(np.abs(r1).max(), np.abs(r2).max())
    err = max(np.abs(g1 - r1).max(), np.abs(g2 - r2).max()) / sc
    assert err < TOL[prec], err
    assert np.abs(g2 + g2.transpose(1, 0, 2, 3)).max() < 1e-12 * sc
    assert abs(ge - e) < 1e-12 * abs(e)
    # the context's own amplitudes and sigma are untouched by the residual call
    x1, x2 = random_amplitudes(o, v, seed=seed + 9)
    before = ctx.cc_lr_sigma(x1, x2)
    ctx.cc_lr_ccsd_residual(0.5 * t1, 0.5 * t2)
    after = ctx.cc_lr_sigma(x1, x2)
    d = max(np.abs(before[0] - after[0]).max(), np.abs(before[1] - after[1]).max())
    assert d <= (1e-13 if prec == "fp64" else 1e-5) * np.abs(before[1]).max()   # split-K order only
    ctx.close()


def test_residual_zero_amplitudes_is_bare_hamiltonian():
    """Omega(0) = <mu|H|Phi_0>: zero singles (canonical Fock), <ab||ij> doubles; E(0) = 0."""
    s = make_system(4, 11, 30, seed=6, scale=0.5)
    z1, z2 = np.zeros((4, 11), complex), np.zeros((4, 4, 11, 11), complex)
    f, g, L, _, _ = oracle_setup(s, z1, z2)
    ctx = gpu_context(s, t1=z1, t2=z2)
    g1, g2, ge = ctx.cc_lr_ccsd_residual(z1, z2)
    vvoo = torch.einsum("abij->ijab", g[4:, 4:, :4, :4]).numpy()
    assert np.abs(g1).max() == 0.0 and ge == 0.0
    assert np.abs(g2 - vvoo).max() < 1e-14 * np.abs(vvoo).max()
    ctx.close()


def test_solve_matches_oracle_newton():
    """o=3, v=8: the converged T and E equal the oracle's Newton solution (explicit Jacobian)."""
    o, v = 3, 8
    s = make_system(o, v, 16, seed=5, scale=0.2)
    f, g, L, _, _ = oracle_setup(s, np.zeros((o, v)), np.zeros((o, o, v, v)))
    t1c, t2c, _ = R.solve_ccsd(f, g, o, L=L, tol=1e-13)
    ec = complex(ccsd.energy(f, g, t1c, t2c))
    ctx = gpu_context(s)                      # T1 = 0, first-order T2
    e, rn, its = ctx.cc_lr_ccsd(tol=1e-12, max_iterations=120, prec="fp64")
    assert rn < 1e-12 and its > 2
    gt1, gt2 = ctx.cc_lr_get_t()
    sc = max(np.abs(t1c.numpy()).max(), np.abs(t2c.numpy()).max())
    assert np.abs(gt1 - t1c.numpy()).max() < 1e-10 * sc
    assert np.abs(gt2 - t2c.numpy()).max() < 1e-10 * sc
    assert abs(e - ec) < 1e-12 * abs(ec)
    ctx.close()


@pytest.fixture(scope="module")
def c1_solved():
    s = make_system(10, 40, 200, seed=1, scale=0.05)
    ctx = gpu_context(s)
    e, rn, its = ctx.cc_lr_ccsd(tol=1e-10, prec="fp64")
    t1, t2 = ctx.cc_lr_get_t()
    yield s, ctx, e, rn, its, t1, t2
    ctx.close()


def test_solve_c1_residual_and_energy(c1_solved):
    """o=10, v=40, naux=200: the oracle's residual vanishes at the library's T; E agrees."""
    s, ctx, e, rn, its, t1, t2 = c1_solved
    assert rn < 1e-10
    f, g, L, T1, T2 = oracle_setup(s, t1, t2)
    r1, r2 = ccsd.residual(f, g, T1, T2)
    assert float(r1.abs().max()) < 1e-9 and float(r2.abs().max()) < 1e-9
    assert abs(e - complex(ccsd.energy(f, g, T1, T2))) < 1e-12 * abs(e)
    # the amplitudes are antisymmetric and no longer the first-order guess
    assert np.abs(t2 + t2.transpose(1, 0, 2, 3)).max() < 1e-14
    assert np.abs(t1).max() > 1e-4


def test_response_after_solve_equals_fresh_context(c1_solved):
    """After the solve every T-dependent quantity is rebuilt: sigma and alpha(omega) equal those
    of a context created with the converged amplitudes."""
    s, ctx, e, rn, its, t1, t2 = c1_solved
    fresh = gpu_context(s, t1=t1, t2=t2)
    x1, x2 = random_amplitudes(10, 40, seed=3)
    a = ctx.cc_lr_sigma(x1, x2)
    b = fresh.cc_lr_sigma(x1, x2)
    assert max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-12 * np.abs(b[1]).max()
    al, _ = ctx.cc_lr_solve([0.0, 0.0428], (2,), tol=1e-10)
    bl, _ = fresh.cc_lr_solve([0.0, 0.0428], (2,), tol=1e-10)
    assert np.abs(al - bl).max() < 1e-8 * np.abs(bl).max()
    fresh.close()


@pytest.mark.parametrize("prec,tol", [("3xtf32", 1e-5), ("bf16x3", 1e-4)])
def test_solve_tensor_core_residual(c1_solved, prec, tol):
    """The same equations with the residual's sigma products on the tensor cores (|Omega(0)| = 2.5
    here, so the residual's floor is the mode's relative accuracy times that): the converged T is
    the FP64 solution within |A^-1| tol (the smallest denominator is about 0.4) and E within
    |<ij||ab>| |dT|."""
    s, _, e64, _, _, t1, t2 = c1_solved
    ctx = gpu_context(s, prec=prec)
    e, rn, its = ctx.cc_lr_ccsd(tol=tol)
    assert rn < tol
    g1, g2 = ctx.cc_lr_get_t()
    assert max(np.abs(g1 - t1).max(), np.abs(g2 - t2).max()) < 10 * tol
    assert abs(e - e64) < 30 * tol
    ctx.close()


def test_solve_reports_no_convergence():
    s = make_system(3, 8, 16, seed=5, scale=0.2)
    ctx = gpu_context(s)
    e, rn, its = ctx.cc_lr_ccsd(tol=1e-14, max_iterations=2, allow_noconv=True)
    assert its == 2 and rn > 1e-14
    from paper_2604_12914_gb300 import binding
    with pytest.raises(binding.CclrError) as ei:
        ctx.cc_lr_ccsd(tol=1e-14, max_iterations=1)
    assert ei.value.status == binding.CCLR_ENOCONV
    ctx.close()


def test_solve_two_electrons_equals_fci():
    """o=2: the library's converged CCSD energy is the exact (FCI) correlation energy of the state
    the CC wave function represents, and its amplitudes reproduce that state."""
    from oracle import secondq
    o, v = 2, 6
    s = make_system(o, v, 10, seed=6, scale=0.4)
    f, g, L, _, _ = oracle_setup(s, np.zeros((o, v)), np.zeros((o, o, v, v)))
    ctx = gpu_context(s)
    e, rn, its = ctx.cc_lr_ccsd(tol=1e-12, max_iterations=200, prec="fp64")
    gt1, gt2 = ctx.cc_lr_get_t()
    bf = secondq.BruteForce(f.numpy(), g.numpy(), o)
    w, U = bf.fci()
    st, ov = secondq.cc_state_overlap(U, gt1, gt2, bf)
    assert ov > 1 - 1e-10
    assert abs(e - (w[st] - bf.e_ref)) < 1e-11 * max(1.0, abs(e))
    ctx.close()
