"""Full-size GPU parity: the workloads' own sizes, checked on sampled entries.

The oracle cannot hold v^4 tensors at these sizes; oracle.sampled evaluates single sigma
entries straight from the Cholesky vectors (pinned entry by entry against the full term
list at small sizes).  The GPU runs the same launch configuration bench.py times.
Tolerance: |sigma_gpu - sigma_oracle| <= tol * rms(sigma_oracle) per sampled entry,
tol = 1e-10 for FP64 and 2e-5 for the complex64 paths.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd, sampled
from oracle.integrals import as_t
from paper_2604_12914_gb300.inputs import make_config, random_amplitudes

from gpu_helpers import gpu_context

pytestmark = pytest.mark.gpu


def _sample_check(name, prec, tol, n2=10, n1=6, seed=2):
    s = make_config(name, seed=seed)
    o, v = s.o, s.v
    ctx = gpu_context(s, prec=prec)                # T1 = 0, first-order T2 formed on the GPU
    x1, x2 = random_amplitudes(o, v, seed=17)
    g1, g2 = ctx.cc_lr_sigma(x1, x2)
    _, gt2 = ctx.cc_lr_get_t()
    ctx.close()
    eps, L = as_t(s.eps), as_t(s.L)
    t2 = ccsd.first_order_t2_from_L(eps, L, o)
    assert np.abs(gt2 - t2.numpy()).max() < 1e-11 * float(t2.abs().max())
    E = sampled.EntrySigma(eps, L, torch.zeros(o, v, dtype=torch.complex128), t2)
    E.set_x(as_t(x1), as_t(x2))
    rms2 = np.sqrt(np.mean(np.abs(g2) ** 2))
    rms1 = np.sqrt(np.mean(np.abs(g1) ** 2))
    rng = np.random.default_rng(5)
    picks = [(0, 1, 0, 1), (o - 2, o - 1, v - 2, v - 1), (o - 1, 0, v - 1, 0)]
    while len(picks) < n2:
        i, j = rng.choice(o, 2, replace=False)
        a, b = rng.choice(v, 2, replace=False)
        picks.append((int(i), int(j), int(a), int(b)))
    for (i, j, a, b) in picks:
        ref = complex(E.sigma2(i, j, a, b))
        assert abs(g2[i, j, a, b] - ref) <= tol * rms2, (i, j, a, b, g2[i, j, a, b], ref)
    for k in range(n1):
        i, a = int(rng.integers(o)), int(rng.integers(v))
        if k == 0:
            i, a = o - 1, v - 1
        ref = complex(E.sigma1(i, a))
        assert abs(g1[i, a] - ref) <= tol * rms1, (i, a, g1[i, a], ref)
    # antisymmetry at full size
    assert np.abs(g2 + g2.transpose(1, 0, 2, 3)).max() <= 1e-6 * np.abs(g2).max()
    assert np.abs(g2 + g2.transpose(0, 1, 3, 2)).max() <= 1e-6 * np.abs(g2).max()


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("3xtf32", 5e-5), ("tf32", 3e-3)])
def test_c2_sigma_c64_sampled_entries(prec, tol):
    _sample_check("C2", prec, tol)


def test_c4_sigma_fp64_sampled_entries():
    _sample_check("C4", "fp64", 1e-10, n2=8, n1=4, seed=4)
