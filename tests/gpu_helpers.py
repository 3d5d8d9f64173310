"""Helpers shared by the GPU parity tests: build a libcclr context and the matching oracle."""
import numpy as np
import torch

from oracle import ccsd, jacobian as J, response as R
from oracle.integrals import as_t, eri_anti


def gpu_context(sysm, t1=None, t2=None, prec="fp64", lam=None):
    from paper_2604_12914_gb300 import binding
    return binding.Context(sysm.o, sysm.v, sysm.naux, sysm.eps, sysm.L, sysm.mu,
                           t1=t1, t2=t2, lam1=None if lam is None else lam[0],
                           lam2=None if lam is None else lam[1], prec=prec)


def oracle_setup(sysm, t1, t2):
    L = as_t(sysm.L)
    g = eri_anti(L)
    f = torch.diag(as_t(sysm.eps).to(torch.complex128))
    return f, g, L, as_t(t1), as_t(t2)


def oracle_sigma(sysm, t1, t2, x1, x2):
    f, g, L, T1, T2 = oracle_setup(sysm, t1, t2)
    D = J.Dressed(f, L, T1, T2)
    s1, s2 = J.sigma_terms(D, as_t(x1), as_t(x2))
    return s1.numpy(), s2.numpy()


def oracle_sigma_T(sysm, t1, t2, y1, y2):
    f, g, L, T1, T2 = oracle_setup(sysm, t1, t2)
    z1, z2 = J.sigma_T(f, g, T1, T2, as_t(y1), as_t(y2))
    return z1.numpy(), z2.numpy()


def rel_err(a1, a2, b1, b2):
    """||a - b|| / ||b|| over unique amplitudes (weights 1 and 1/4)."""
    num = np.sum(np.abs(a1 - b1) ** 2) + 0.25 * np.sum(np.abs(a2 - b2) ** 2)
    den = np.sum(np.abs(b1) ** 2) + 0.25 * np.sum(np.abs(b2) ** 2)
    return float(np.sqrt(num / den))


def wdot(a1, a2, b1, b2):
    return np.sum(a1 * b1) + 0.25 * np.sum(a2 * b2)
