"""Small shared helpers for the oracle tests (build an oracle Problem from a System)."""
import numpy as np
import torch

from oracle import ccsd, response as R
from oracle.integrals import as_t, eri_anti


def oracle_problem(sysm, t1=None, t2=None, offdiag_fock=None, converge=False):
    L = as_t(sysm.L)
    g = eri_anti(L)
    f = torch.diag(as_t(sysm.eps).to(torch.complex128))
    if offdiag_fock is not None:
        f = f + as_t(offdiag_fock)
    no = sysm.o
    if converge:
        t1c, t2c, _ = R.solve_ccsd(f, g, no, L=L)
        return R.Problem(f, g, L, no, t1c, t2c)
    if t2 is None:
        t2 = ccsd.first_order_t2(torch.real(torch.diagonal(f)), g, no)
    if t1 is None:
        t1 = as_t(sysm.t1)
    return R.Problem(f, g, L, no, as_t(t1), as_t(t2))


def hermitian(rng, n, s=1.0):
    m = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return s * (m + m.conj().T) / 2
