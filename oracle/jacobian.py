"""sigma = A X, the CC Jacobian times a vector -- oracle, test infrastructure.

Sec. 2.2 defines A_mu,nu = <mu|[H-bar_0, tau_nu]|Phi_0>.  Because all excitation
operators commute, d/de e^{-(T+eX)} H e^{T+eX} = [H-bar, X], so A = dOmega/dT exactly at
any T (converged or not).  Two independent routes:

* ``sigma_stencil``: the definition.  Omega is a polynomial of degree <= 4 in (T1, T2),
  so the 4-point central stencil [-O(T+2hX) + 8 O(T+hX) - 8 O(T-hX) + O(T-2hX)]/(12h)
  is exact for any h (only rounding error remains).
* ``sigma_terms``: <mu|(H-bar X)_connected|Phi_0> written term by term with the exact
  two-body elements of H-bar in the T1-dressed form.  T1 dressing: the Cholesky
  vectors become L~ = (1 - t) L (1 + t) (t_ai = t_i^a, the only non-zero block), the
  one-body operator h~ = (1 - t) h (1 + t) and the dressed Fock f~ = h~ + sum_k <pk||qk>~;
  then H-bar = e^{-T2} H~ e^{T2}.  Integrals with more than two virtual indices
  (<ab||ef>~, <am||ef>~, <ab||ej>~) are only ever used through L~ (Sec. 3: higher-rank
  integrals are evaluated on the fly from the Cholesky vectors).

``sigma_T`` is the transpose product Y A (bilinear, no conjugation) by reverse-mode
differentiation of Omega.
"""
from __future__ import annotations

import torch

from . import ccsd
from .integrals import C128

ein = torch.einsum


def _P(x, d0, d1):
    return x - x.transpose(d0, d1)


def sigma_stencil(f, g, t1, t2, x1, x2, h: float | None = None):
    """sigma = dOmega(T + eX)/de at e = 0 by the polynomial-exact 4-point stencil."""
    if h is None:
        nt = float(torch.sqrt((t1.abs() ** 2).sum() + 0.25 * (t2.abs() ** 2).sum()))
        nx = float(torch.sqrt((x1.abs() ** 2).sum() + 0.25 * (x2.abs() ** 2).sum()))
        h = max(nt, 1e-2) / max(nx, 1e-300) * 0.5
    out1 = torch.zeros_like(t1)
    out2 = torch.zeros_like(t2)
    for c, k in ((-1.0, 2.0), (8.0, 1.0), (-8.0, -1.0), (1.0, -2.0)):
        r1, r2 = ccsd.residual(f, g, t1 + k * h * x1, t2 + k * h * x2)
        out1 = out1 + c * r1
        out2 = out2 + c * r2
    return out1 / (12.0 * h), out2 / (12.0 * h)


def sigma_T(f, g, t1, t2, y1, y2):
    """(Y A)_nu = sum_mu Y_mu dOmega_mu/dt_nu over unique amplitudes, as full tensors.

    Computed by reverse-mode differentiation of Omega.  For a holomorphic map PyTorch
    returns J^H v, so Y A = conj(vjp(conj(Y))).  The singles weight is 1 and the
    doubles weight 1/4 (unique amplitudes i<j, a<b); the returned doubles block is
    antisymmetric.
    """
    a1 = t1.detach().clone().requires_grad_(True)
    a2 = t2.detach().clone().requires_grad_(True)
    r1, r2 = ccsd.residual(f, g, a1, a2)
    gy1, gy2 = torch.autograd.grad((r1, r2), (a1, a2), grad_outputs=(y1.conj(), 0.25 * y2.conj()))
    z1 = gy1.conj().resolve_conj()
    z2 = gy2.conj().resolve_conj()
    # weight 1/4 on doubles and projection onto antisymmetric tensors
    z2 = _P(_P(z2, 0, 1), 2, 3)
    return z1, z2


# ------------------------------------------------------------------------------------
# T1-dressed Hamiltonian and the connected H-bar X term list
# ------------------------------------------------------------------------------------

class Dressed:
    """T1-dressed Cholesky vectors, Fock matrix and the exact two-body H-bar elements."""

    def __init__(self, f, L, t1, t2):
        no, nv = t1.shape
        n = no + nv
        self.no, self.nv = no, nv
        o, v = slice(0, no), slice(no, n)
        self.o, self.v = o, v
        tm = torch.zeros(n, n, dtype=C128)
        tm[v, o] = t1.transpose(0, 1)                    # t_ai = t_i^a
        one = torch.eye(n, dtype=C128)
        Xl, Xr = one - tm, one + tm
        self.Lt = ein("pq,Pqr,rs->Pps", Xl, L, Xr)      # L~ = (1 - t) L (1 + t)
        h = f - self._G(L)                               # one-body part of H
        self.f = Xl @ h @ Xr + self._G(self.Lt)          # dressed Fock f~
        self.t1, self.t2 = t1, t2
        gt = lambda a, b, c, d: self.ints(a, b, c, d)
        self._cache = {}
        oovv = gt("o", "o", "v", "v")
        self.oovv = oovv
        # exact two-body elements of H-bar = e^{-T2} H~ e^{T2}
        self.Fov = self.f[o, v]
        self.Foo = self.f[o, o] + 0.5 * ein("inef,mnef->mi", t2, oovv)
        self.Fvv = self.f[v, v] - 0.5 * ein("mnaf,mnef->ae", t2, oovv)
        self.Woooo = gt("o", "o", "o", "o") + 0.5 * ein("ijef,mnef->mnij", t2, oovv)
        self.Wovvo = gt("o", "v", "v", "o") - ein("jnfb,mnef->mbej", t2, oovv)
        self.Wooov = gt("o", "o", "o", "v")
        self.Wovoo = (gt("o", "v", "o", "o") - ein("me,ijbe->mbij", self.Fov, t2)
                      + 0.5 * ein("mbef,ijef->mbij", gt("o", "v", "v", "v"), t2)
                      + _P(ein("mnie,jnbe->mbij", self.Wooov, t2), 2, 3))
        self.Wvvvo = (gt("v", "v", "v", "o") - ein("me,miab->abei", self.Fov, t2)
                      + 0.5 * ein("mnei,mnab->abei", gt("o", "o", "v", "o"), t2)
                      - _P(ein("mbef,miaf->abei", gt("o", "v", "v", "v"), t2), 0, 1))

    def _G(self, L):
        no = self.no
        J = ein("Ppq,Pkk->pq", L, L[:, :no, :no])
        K = ein("Ppk,Pkq->pq", L[:, :, :no], L[:, :no, :])
        return J - K

    def ints(self, a, b, c, d):
        """<pq||rs>~ block with p in a, q in b, r in c, s in d ('o' or 'v'), from L~."""
        key = a + b + c + d
        if key not in self._cache:
            S = {"o": self.o, "v": self.v}
            Lt = self.Lt
            g = (ein("Ppr,Pqs->pqrs", Lt[:, S[a], S[c]], Lt[:, S[b], S[d]])
                 - ein("Pps,Pqr->pqrs", Lt[:, S[a], S[d]], Lt[:, S[b], S[c]]))
            self._cache[key] = g
        return self._cache[key]


def sigma_terms(D: Dressed, x1, x2):
    """sigma = <mu|(H-bar X)_c|Phi_0>, singles and doubles (connected terms only)."""
    t2 = D.t2
    oovv = D.oovv
    Lt, o, v = D.Lt, D.o, D.v
    # ---- singles
    s1 = (ein("ae,ie->ia", D.Fvv, x1)
          - ein("mi,ma->ia", D.Foo, x1)
          + ein("maei,me->ia", D.Wovvo, x1)
          + ein("me,imae->ia", D.Fov, x2)
          + 0.5 * ein("amef,imef->ia", D.ints("v", "o", "v", "v"), x2)
          - 0.5 * ein("mnie,mnae->ia", D.Wooov, x2))
    # ---- doubles
    s2 = _P(ein("be,ijae->ijab", D.Fvv, x2), 2, 3)
    s2 = s2 - _P(ein("mj,imab->ijab", D.Foo, x2), 0, 1)
    s2 = s2 + 0.5 * ein("mnij,mnab->ijab", D.Woooo, x2)
    # particle-particle ladder 1/2 sum_ef W_abef X_ij^ef with the exact element
    # W_abef = <ab||ef>~ + 1/2 sum_mn t_mn^ab <mn||ef>; <ab|ef>~ from L~_vv
    s2 = s2 + 0.5 * ein("abef,ijef->ijab", D.ints("v", "v", "v", "v"), x2)
    Z = 0.5 * ein("mnef,ijef->mnij", oovv, x2)
    s2 = s2 + 0.5 * ein("mnab,mnij->ijab", t2, Z)
    s2 = s2 + _P(_P(ein("mbej,imae->ijab", D.Wovvo, x2), 0, 1), 2, 3)
    s2 = s2 + _P(ein("abej,ie->ijab", D.Wvvvo, x1), 0, 1)
    s2 = s2 - _P(ein("mbij,ma->ijab", D.Wovoo, x1), 2, 3)
    # three-body parts of H-bar
    Xvv = ein("bmef,mf->be", D.ints("v", "o", "v", "v"), x1) - 0.5 * ein("mnef,mnbf->be", oovv, x2)
    s2 = s2 + _P(ein("be,ijae->ijab", Xvv, t2), 2, 3)
    Xoo = ein("mnje,ne->mj", D.Wooov, x1) + 0.5 * ein("mnef,jnef->mj", oovv, x2)
    s2 = s2 - _P(ein("mj,imab->ijab", Xoo, t2), 0, 1)
    return s1, s2
