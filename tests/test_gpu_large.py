"""Parity at the two largest workloads, o=40, v=320, naux=1600 and o=56, v=480, naux=3000, in
the tensor-core modes, on sampled entries: the oracle's per-entry sigma (oracle.sampled, with the
whole Wovvo block formed once) for 512 canonical doubles entries and 64 singles entries, from
the same seeded inputs.  The library runs in its lean configuration (complex64 intermediates
built in FP32, no FP64 state), as at these sizes in bench.py.

The o=56, v=480 case needs about 100 GB of host memory and several minutes of CPU time for the
oracle; it runs when CCLR_TEST_LARGEST=1.
"""
import os

import numpy as np
import pytest
import torch

from oracle import ccsd, sampled
from oracle.integrals import as_t
from paper_2604_12914_gb300.inputs import make_config, random_amplitudes

pytestmark = pytest.mark.gpu


def _picks(o, v, n, seed):
    rng = np.random.default_rng(seed)
    out = [(0, 1, 0, 1), (o - 2, o - 1, v - 2, v - 1), (0, o - 1, 0, v - 1)]
    seen = set(out)
    while len(out) < n:
        i, j = sorted(rng.choice(o, 2, replace=False).tolist())
        a, b = sorted(rng.choice(v, 2, replace=False).tolist())
        if (i, j, a, b) not in seen:
            seen.add((i, j, a, b))
            out.append((i, j, a, b))
    return out


def _check(cfg, modes, n2=512, n1=64):
    from paper_2604_12914_gb300 import binding
    s = make_config(cfg)
    o, v = s.o, s.v
    x1, x2 = random_amplitudes(o, v, seed=17)
    ctx = binding.Context(o, v, s.naux, s.eps, s.L, s.mu, prec=modes[0][0])
    ctx.cc_lr_set_refinement("3xtf32")          # lean: no FP64 state
    got = {}
    for prec, _ in modes:
        ctx.cc_lr_set_precision(prec)
        g1, g2 = ctx.cc_lr_sigma(x1, x2)
        got[prec] = (g1, g2)
        mem = ctx.cc_lr_memory()
        print(f"{cfg} {prec}: device memory held {mem[0] / 1e9:.1f} GB, peak {mem[1] / 1e9:.1f} GB")
    ctx.close()
    eps, L = as_t(s.eps), as_t(s.L)
    del s
    t2 = ccsd.first_order_t2_from_L(eps, L, o)
    E = sampled.EntrySigma(eps, L, torch.zeros(o, v, dtype=torch.complex128), t2)
    del L
    E.set_x(as_t(x1), as_t(x2))
    E.Wovvo_full()
    picks = _picks(o, v, n2, seed=7)
    ref2 = np.array([complex(E.sigma2(*p)) for p in picks])
    rng = np.random.default_rng(8)
    singles = [(o - 1, v - 1)] + [(int(rng.integers(o)), int(rng.integers(v))) for _ in range(n1 - 1)]
    ref1 = np.array([complex(E.sigma1(i, a)) for i, a in singles])
    idx2, idx1 = tuple(np.array(picks).T), tuple(np.array(singles).T)
    rms2 = np.sqrt(np.mean(np.abs(ref2) ** 2))
    rms1 = np.sqrt(np.mean(np.abs(ref1) ** 2))
    for prec, tol in modes:
        g1, g2 = got[prec]
        e2 = np.abs(g2[idx2] - ref2).max() / rms2
        e1 = np.abs(g1[idx1] - ref1).max() / rms1
        print(f"{cfg} {prec}: max |d sigma2| / rms {e2:.2e} over {n2} entries, max |d sigma1| / rms {e1:.2e} over {n1}")
        assert e2 <= tol and e1 <= tol
        amax = np.abs(g2).max()
        assert np.abs(g2 + g2.transpose(1, 0, 2, 3)).max() <= 1e-6 * amax


def test_c3_sigma_sampled_entries():
    _check("C3", [("tf32", 3e-3), ("3xtf32", 5e-5), ("bf16x3", 5e-4)])


@pytest.mark.skipif(os.environ.get("CCLR_TEST_LARGEST") != "1", reason="o=56 v=480: set CCLR_TEST_LARGEST=1")
def test_c5_sigma_sampled_entries():
    _check("C5", [("tf32", 3e-3), ("bf16x3", 5e-4)])
