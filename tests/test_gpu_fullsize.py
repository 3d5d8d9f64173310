"""Full-size GPU parity: the workloads' own sizes, in the launch configuration bench.py times.

The oracle cannot hold v^4 tensors at o=32, v=240 (53 GB).  Its reference there is
oracle.sampled: every sigma term but the particle-particle ladder for the whole vector
(``sigma_rest``, vectorised), plus the ladder entry by entry straight from the Cholesky
vectors; both are pinned against the explicit-tensor term list at small sizes.  At o=24,
v=160 the oracle's chunked whole-vector sigma (``sigma_blocked``) gives every entry.

Checks, per precision mode on one context (FP64, FP32 CUDA cores, 3xTF32, bf16x3, TF32):
* sigma: 512 sampled doubles entries (corners included) and every singles entry,
  |sigma_gpu - sigma_oracle| <= tol * rms(sigma_oracle) per entry;
* sigma^T: the bilinear identity <Y, A X> = <sigma^T(Y), X> with Y supported on the 512
  sampled doubles entries and every singles entry (so A X comes from the oracle and
  sigma^T(Y) from the GPU), to tol relative to sum_mu |Y_mu| |sigma_mu|;
* antisymmetry of the doubles block at full size.
tol = 1e-10 (FP64), 2e-5 (FP32), 5e-5 (3xTF32), 5e-4 (bf16x3), 3e-3 (TF32): FP32 accumulation
over K ~ v^2 terms gives about sqrt(K) 6e-8; TF32 keeps 10 mantissa bits per operand; the bf16x3
split neglects terms of about 3 x 2^-16 of each product.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd, sampled
from oracle.integrals import as_t
from paper_2604_12914_gb300.inputs import make_config, random_amplitudes

from gpu_helpers import gpu_context

pytestmark = pytest.mark.gpu

MODES = [("fp64", 1e-10), ("fp32", 2e-5), ("3xtf32", 5e-5), ("bf16x3", 5e-4), ("tf32", 3e-3)]
N2 = 512


def _picks(o, v, n, seed):
    """n distinct canonical doubles entries (i<j, a<b), corners first."""
    rng = np.random.default_rng(seed)
    out = [(0, 1, 0, 1), (o - 2, o - 1, v - 2, v - 1), (0, o - 1, 0, v - 1), (o - 2, o - 1, 0, 1)]
    seen = set(out)
    while len(out) < n:
        i, j = sorted(rng.choice(o, 2, replace=False).tolist())
        a, b = sorted(rng.choice(v, 2, replace=False).tolist())
        if (i, j, a, b) not in seen:
            seen.add((i, j, a, b))
            out.append((i, j, a, b))
    return out


@pytest.fixture(scope="module")
def c2():
    """C2 system (seed 2, T1 = 0, first-order T2 formed by the library), one random X, and the
    oracle's reference: all singles, 512 doubles entries, from the same seeded inputs."""
    s = make_config("C2", seed=2)
    o, v = s.o, s.v
    x1, x2 = random_amplitudes(o, v, seed=17)
    eps, L = as_t(s.eps), as_t(s.L)
    t2 = ccsd.first_order_t2_from_L(eps, L, o)
    E = sampled.EntrySigma(eps, L, torch.zeros(o, v, dtype=torch.complex128), t2)
    E.set_x(as_t(x1), as_t(x2))
    r1, r2rest = E.sigma_rest()
    picks = _picks(o, v, N2, seed=5)
    ref2 = np.empty(len(picks), complex)
    for k, (i, j, a, b) in enumerate(picks):
        # the ladder entry sum_ef <ab|ef>~ X_ij^ef with <ab|ef>~ = sum_P L~_ae L~_bf
        lad = complex(((E.Lvv[:, a, :] @ E.x2[i, j]) * E.Lvv[:, b, :]).sum())
        ref2[k] = complex(r2rest[i, j, a, b]) + lad
    ref = {"sys": s, "x1": x1, "x2": x2, "t2": t2.numpy(), "r1": r1.numpy(), "picks": picks, "r2": ref2}
    del E, r2rest
    return ref


@pytest.fixture(scope="module")
def c2_ctx(c2):
    s = c2["sys"]
    ctx = gpu_context(s, prec="fp64")            # T1 = 0, first-order T2 formed on the GPU
    yield ctx
    ctx.close()


def test_c2_first_order_t2(c2, c2_ctx):
    _, gt2 = c2_ctx.cc_lr_get_t()
    t2 = c2["t2"]
    assert np.abs(gt2 - t2).max() < 1e-11 * np.abs(t2).max()


@pytest.mark.parametrize("prec,tol", MODES)
def test_c2_sigma_and_transpose_sampled(c2, c2_ctx, prec, tol):
    ctx = c2_ctx
    ctx.cc_lr_set_precision(prec)
    o, v = c2["sys"].o, c2["sys"].v
    x1, x2, r1, ref2, picks = c2["x1"], c2["x2"], c2["r1"], c2["r2"], c2["picks"]
    g1, g2 = ctx.cc_lr_sigma(x1, x2)
    rms1 = np.sqrt(np.mean(np.abs(r1) ** 2))
    rms2 = np.sqrt(np.mean(np.abs(ref2) ** 2))
    idx = tuple(np.array(picks).T)
    got2 = g2[idx]
    err2 = np.abs(got2 - ref2).max()
    err1 = np.abs(g1 - r1).max()
    print(f"C2 {prec}: max |d sigma2| / rms = {err2 / rms2:.2e} over {len(picks)} entries, "
          f"max |d sigma1| / rms = {err1 / rms1:.2e} over {o * v} entries")
    assert err2 <= tol * rms2
    assert err1 <= tol * rms1
    amax = np.abs(g2).max()
    assert np.abs(g2 + g2.transpose(1, 0, 2, 3)).max() <= 1e-6 * amax
    assert np.abs(g2 + g2.transpose(0, 1, 3, 2)).max() <= 1e-6 * amax
    del g2
    # sigma^T against the oracle's A X through <Y, A X> = <sigma^T(Y), X>
    rng = np.random.default_rng(41)
    y1 = (rng.standard_normal((o, v)) + 1j * rng.standard_normal((o, v))) / np.sqrt(2)
    w = (rng.standard_normal(len(picks)) + 1j * rng.standard_normal(len(picks))) / np.sqrt(2)
    y2 = np.zeros((o, o, v, v), complex)
    for (i, j, a, b), wk in zip(picks, w):
        y2[i, j, a, b] = wk
        y2[j, i, a, b] = -wk
        y2[i, j, b, a] = -wk
        y2[j, i, b, a] = wk
    z1, z2 = ctx.cc_lr_sigma_T(y1, y2)
    lhs = np.sum(z1 * x1) + 0.25 * np.sum(z2 * x2)
    rhs = np.sum(y1 * r1) + np.sum(w * ref2)
    scale = np.sum(np.abs(y1 * r1)) + np.sum(np.abs(w * ref2))
    print(f"C2 {prec}: sigma^T bilinear |lhs - rhs| / scale = {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= tol * scale


@pytest.fixture(scope="module")
def c4():
    s = make_config("C4", seed=4)
    o, v = s.o, s.v
    x1, x2 = random_amplitudes(o, v, seed=19)
    eps, L = as_t(s.eps), as_t(s.L)
    t2 = ccsd.first_order_t2_from_L(eps, L, o)
    E = sampled.EntrySigma(eps, L, torch.zeros(o, v, dtype=torch.complex128), t2)
    E.set_x(as_t(x1), as_t(x2))
    r1, r2 = E.sigma_blocked(a_chunk=16)
    return {"sys": s, "x1": x1, "x2": x2, "r1": r1.numpy(), "r2": r2.numpy()}


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("3xtf32", 5e-5)])
def test_c4_sigma_full_vector(c4, prec, tol):
    """o=24, v=160, naux=800: every entry of sigma against the oracle's whole-vector sigma, and
    sigma^T through the bilinear identity with dense random Y."""
    s = c4["sys"]
    ctx = gpu_context(s, prec=prec)
    x1, x2, r1, r2 = c4["x1"], c4["x2"], c4["r1"], c4["r2"]
    g1, g2 = ctx.cc_lr_sigma(x1, x2)
    num = np.sum(np.abs(g1 - r1) ** 2) + 0.25 * np.sum(np.abs(g2 - r2) ** 2)
    den = np.sum(np.abs(r1) ** 2) + 0.25 * np.sum(np.abs(r2) ** 2)
    rel = float(np.sqrt(num / den))
    print(f"C4 {prec}: relative error of sigma over unique amplitudes {rel:.2e}")
    assert rel < tol
    y1, y2 = random_amplitudes(s.o, s.v, seed=23)
    z1, z2 = ctx.cc_lr_sigma_T(y1, y2)
    lhs = np.sum(z1 * x1) + 0.25 * np.sum(z2 * x2)
    rhs = np.sum(y1 * r1) + 0.25 * np.sum(y2 * r2)
    scale = np.sum(np.abs(y1 * r1)) + 0.25 * np.sum(np.abs(y2 * r2))
    print(f"C4 {prec}: sigma^T bilinear |lhs - rhs| / scale = {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= tol * scale
    ctx.close()
