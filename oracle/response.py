"""Linear-response quantities and alpha(omega) -- oracle, test infrastructure.

Sec. 2.2 definitions, with the Lagrangian L(T) = E(T) + lambda . Omega(T):

* xi^B_nu = <nu|e^{-T} B e^{T}|Phi_0>.  Omega is linear in the Hamiltonian, so
  xi^B = Omega[f + B](T) - Omega[f](T) exactly (B one-body).
* eta0 = dE/dT; ground-state Lambda from lambda A = -eta0 (stationarity of L).
* eta^A_nu = <(1+Lambda)|[A-bar, tau_nu]|Phi_0> = d/dt_nu [E_A(T) + lambda . xi^A(T)],
  E_A = <Phi_0|A-bar|Phi_0> (same derivative identity as A = dOmega/dT).
* F_nu,gamma = <(1+Lambda)|[[H-bar, tau_nu], tau_gamma]|Phi_0> = d^2 L / dt_nu dt_gamma,
  so (F X^A) . X^B is the mixed second directional derivative of L (exact by stencil:
  L is quartic in T).
* X^B(omega) from (A - omega) X = -xi^B (alpha -> 0+); Y^B(omega) from
  Y (A + omega) = -(eta^B + F X^B(omega)).
* g(A,B;w) = eta^A . X^B(w) + eta^B . X^A(-w) + (F X^A(-w)) . X^B(w);
  <<A;B>>_w = 1/2 [g(A,B;w) + conj g(A,B;-w)] (P(A,B) swaps A and B and conjugates);
  alpha_AB(w) = -<<A;B>>_w.
* Damped response (complex frequency z = w + i gamma, the same sigma with a complex shift):
  <<A;B>>_z = 1/2 [g(A,B;z) + conj g(A,B;-z*)], which is the real-frequency formula at
  gamma = 0 and, for exact states, equals the sum over states continued to complex z
  (the conjugate term of the exact function at -z* is the function at z).
Dot products are bilinear over unique amplitudes (singles, i<j a<b doubles).
"""
from __future__ import annotations

import numpy as np
import torch

from . import ccsd, jacobian
from .integrals import C128

STENCIL = ((-1.0, 2.0), (8.0, 1.0), (-8.0, -1.0), (1.0, -2.0))   # (coefficient, step)


class Problem:
    """A CCSD response problem with explicit antisymmetrised integrals (small n)."""

    def __init__(self, f, g, L, no, t1, t2):
        self.f, self.g, self.L, self.no = f, g, L, no
        self.nv = f.shape[0] - no
        self.t1, self.t2 = t1, t2

    # -- packed (unique amplitude) helpers
    def pack(self, x1, x2):
        return ccsd.pack(x1, x2)

    def unpack(self, vec):
        return ccsd.unpack(vec, self.no, self.nv)

    @property
    def nvec(self):
        return ccsd.n_amp(self.no, self.nv)

    def omega(self, t1=None, t2=None, f=None):
        return ccsd.residual(self.f if f is None else f, self.g,
                             self.t1 if t1 is None else t1, self.t2 if t2 is None else t2)

    def energy(self, t1=None, t2=None, f=None):
        return ccsd.energy(self.f if f is None else f, self.g,
                           self.t1 if t1 is None else t1, self.t2 if t2 is None else t2)

    # -- Jacobian
    def sigma(self, x1, x2):
        D = jacobian.Dressed(self.f, self.L, self.t1, self.t2)
        return jacobian.sigma_terms(D, x1, x2)

    def jacobian_matrix(self, t1=None, t2=None, f=None):
        """Explicit A over unique amplitudes, column by column."""
        t1 = self.t1 if t1 is None else t1
        t2 = self.t2 if t2 is None else t2
        f = self.f if f is None else f
        D = jacobian.Dressed(f, self.L, t1, t2)
        N = self.nvec
        A = torch.zeros(N, N, dtype=C128)
        for k in range(N):
            e = torch.zeros(N, dtype=C128)
            e[k] = 1.0
            x1, x2 = self.unpack(e)
            A[:, k] = self.pack(*jacobian.sigma_terms(D, x1, x2))
        return A

    # -- right-hand sides and left vectors
    def xi(self, B, t1=None, t2=None):
        """xi^B = Omega[f + B] - Omega[f] (exact: Omega is linear in H)."""
        r1a, r2a = self.omega(t1, t2, f=self.f + B)
        r1b, r2b = self.omega(t1, t2)
        return r1a - r1b, r2a - r2b

    def eta0(self):
        """dE/dT over unique amplitudes: [f_ia + sum_jb <ij||ab> t_jb ; <ij||ab>]."""
        o, v = slice(0, self.no), slice(self.no, None)
        goovv = self.g[o, o, v, v]
        e1 = self.f[o, v] + torch.einsum("ijab,jb->ia", goovv, self.t1)
        return self.pack(e1, goovv)

    def lam(self):
        """Ground-state Lambda: lambda A = -eta0."""
        A = self.jacobian_matrix()
        return torch.linalg.solve(A.transpose(0, 1), -self.eta0())

    def step(self, x1, x2):
        nt = float(torch.sqrt((self.t1.abs() ** 2).sum() + 0.25 * (self.t2.abs() ** 2).sum()))
        nx = float(torch.sqrt((x1.abs() ** 2).sum() + 0.25 * (x2.abs() ** 2).sum()))
        return max(nt, 1e-2) / max(nx, 1e-300) * 0.25

    def eta_dot(self, A, lam, x1, x2):
        """eta^A . X = d/de [E_A(T + eX) + lambda . xi^A(T + eX)] (4-point stencil)."""
        o, v = slice(0, self.no), slice(self.no, None)
        val = (A[o, v] * x1).sum()                      # dE_A/dT . X, E_A = sum A_ia t_ia
        h = self.step(x1, x2)
        acc = 0.0
        for c, k in STENCIL:
            xi1, xi2 = self.xi(A, self.t1 + k * h * x1, self.t2 + k * h * x2)
            acc = acc + c * (lam @ self.pack(xi1, xi2))
        return val + acc / (12.0 * h)

    def lagrangian(self, lam, t1, t2):
        r1, r2 = self.omega(t1, t2)
        return self.energy(t1, t2) + lam @ self.pack(r1, r2)

    def fxx(self, lam, xa, xb):
        """(F X^A) . X^B = d^2 L(T + e1 X^A + e2 X^B)/de1 de2 (nested exact stencils)."""
        ha = self.step(*xa)
        hb = self.step(*xb)
        acc = 0.0
        for ca, ka in STENCIL:
            for cb, kb in STENCIL:
                t1 = self.t1 + ka * ha * xa[0] + kb * hb * xb[0]
                t2 = self.t2 + ka * ha * xa[1] + kb * hb * xb[1]
                acc = acc + ca * cb * self.lagrangian(lam, t1, t2)
        return acc / (144.0 * ha * hb)

    # -- vectors needed by the left-hand (Y) route
    def eta_vec(self, B, lam):
        """eta^B as a vector: dE_B/dT + lambda (A[f+B] - A[f])."""
        o, v = slice(0, self.no), slice(self.no, None)
        e = self.pack(B[o, v], torch.zeros(self.no, self.no, self.nv, self.nv, dtype=C128))
        dA = self.jacobian_matrix(f=self.f + B) - self.jacobian_matrix()
        return e + dA.transpose(0, 1) @ lam

    def fx_vec(self, lam, x):
        """F X = d/de [lambda A(T + eX) + eta0(T + eX)] (4-point stencil)."""
        x1, x2 = self.unpack(x)
        h = self.step(x1, x2)
        o, v = slice(0, self.no), slice(self.no, None)
        goovv = self.g[o, o, v, v]
        acc = torch.zeros(self.nvec, dtype=C128)
        for c, k in STENCIL:
            A = self.jacobian_matrix(self.t1 + k * h * x1, self.t2 + k * h * x2)
            acc = acc + c * (A.transpose(0, 1) @ lam)
        d_eta0 = self.pack(torch.einsum("ijab,jb->ia", goovv, x1), torch.zeros_like(x2))
        return acc / (12.0 * h) + d_eta0


def solve_ccsd(f, g, no, t1=None, t2=None, tol=1e-12, maxit=60, L=None):
    """Ground-state CCSD by Newton iterations with the explicit Jacobian (small spaces)."""
    nv = f.shape[0] - no
    if t2 is None:
        t2 = ccsd.first_order_t2(torch.real(torch.diagonal(f)), g, no)
    if t1 is None:
        t1 = torch.zeros(no, nv, dtype=C128)
    P = Problem(f, g, L, no, t1, t2)
    for it in range(maxit):
        r1, r2 = ccsd.residual(f, g, P.t1, P.t2)
        r = P.pack(r1, r2)
        if float(r.abs().max()) < tol:
            return P.t1, P.t2, it
        A = P.jacobian_matrix()
        dt = torch.linalg.solve(A, -r)
        d1, d2 = P.unpack(dt)
        P.t1, P.t2 = P.t1 + d1, P.t2 + d2
    raise RuntimeError("CCSD did not converge")


def solve_x(A, xi_vec, omega):
    """(A - omega) X = -xi."""
    N = A.shape[0]
    return torch.linalg.solve(A - omega * torch.eye(N, dtype=C128), -xi_vec)


def alpha(P: Problem, ops, omega: float, lam=None, A=None, gamma: float = 0.0):
    """Complex 3x3 (or k x k) polarisability alpha_AB(z) = -<<A;B>>_z, z = omega + i gamma
    (gamma = 0: the undamped response)."""
    if A is None:
        A = P.jacobian_matrix()
    if lam is None:
        lam = torch.linalg.solve(A.transpose(0, 1), -P.eta0())
    k = len(ops)
    z = complex(omega, gamma)
    xi = [P.pack(*P.xi(op)) for op in ops]
    X = {}
    for shift in {z, -z, z.conjugate(), -z.conjugate()}:
        X[shift] = [P.unpack(solve_x(A, xi[b], shift)) for b in range(k)]

    def g(a, b, w):
        # g(A,B;w) = eta^A . X^B(w) + eta^B . X^A(-w) + (F X^A(-w)) . X^B(w)
        return (P.eta_dot(ops[a], lam, *X[w][b]) + P.eta_dot(ops[b], lam, *X[-w][a])
                + P.fxx(lam, X[-w][a], X[w][b]))

    out = torch.zeros(k, k, dtype=C128)
    for a in range(k):
        for b in range(k):
            out[a, b] = -0.5 * (g(a, b, z) + torch.conj(g(a, b, -z.conjugate())))
    return out


def g_left(P: Problem, opA, opB, omega: float, lam=None, A=None):
    """g(A,B;w) by the left-hand route: Y^B(w) . xi^A + eta^A . X^B(w)."""
    if A is None:
        A = P.jacobian_matrix()
    if lam is None:
        lam = torch.linalg.solve(A.transpose(0, 1), -P.eta0())
    N = A.shape[0]
    xiB = P.pack(*P.xi(opB))
    xiA = P.pack(*P.xi(opA))
    XB = solve_x(A, xiB, omega)
    rhs = -(P.eta_vec(opB, lam) + P.fx_vec(lam, XB))
    YB = torch.linalg.solve((A + omega * torch.eye(N, dtype=C128)).transpose(0, 1), rhs)
    etaA = P.eta_vec(opA, lam)
    return YB @ xiA + etaA @ XB
