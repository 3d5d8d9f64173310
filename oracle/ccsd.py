"""Spin-orbital CCSD energy and residual -- oracle, test infrastructure.

Sec. 2.2: |Psi> = e^T |Phi_0>, T1 = sum t_i^a {a+_a a_i}, T2 = 1/4 sum t_ij^ab
{a+_a a+_b a_j a_i}; E = <Phi_0|H-bar|Phi_0>, Omega_mu = <mu|H-bar|Phi_0> with
H-bar = e^{-T} H e^{T}.  The paper prints no residual; the terms below are the
standard published spin-orbital CCSD equations (intermediates F_ae, F_mi, F_me,
W_mnij, W_abef, W_mbej), written for a general (non-diagonal) Fock matrix and for
complex spinors: the projections of H on doubly and singly excited determinants are
<ab||ij> and f_ai.  Omega here is the full residual (diagonal Fock kept inside the F
intermediates), so Omega = 0 at convergence and A = dOmega/dT at any T.

Amplitude arrays: t1[i, a], t2[i, j, a, b] (antisymmetric in ij and in ab);
integrals g[p, q, r, s] = <pq||rs> over n = o + v spinors, occupied first.
"""
from __future__ import annotations

import torch

from .integrals import C128


def _P(x: torch.Tensor, d0: int, d1: int) -> torch.Tensor:
    """Antisymmetriser P(pq) X = X - X(p<->q)."""
    return x - x.transpose(d0, d1)


def blocks(g: torch.Tensor, no: int):
    o, v = slice(0, no), slice(no, None)
    return {
        "oooo": g[o, o, o, o], "ooov": g[o, o, o, v], "oovo": g[o, o, v, o],
        "oovv": g[o, o, v, v], "ovoo": g[o, v, o, o], "ovov": g[o, v, o, v],
        "ovvo": g[o, v, v, o], "ovvv": g[o, v, v, v], "vovv": g[v, o, v, v],
        "vvoo": g[v, v, o, o], "vvvo": g[v, v, v, o], "vvvv": g[v, v, v, v],
        "vooo": g[v, o, o, o],
    }


def energy(f: torch.Tensor, g: torch.Tensor, t1: torch.Tensor, t2: torch.Tensor) -> torch.Tensor:
    """Correlation energy <Phi_0|H-bar|Phi_0> - E_ref (Sec. 2.2).

    E = sum f_ia t_i^a + 1/4 sum <ij||ab> t_ij^ab + 1/2 sum <ij||ab> t_i^a t_j^b.
    """
    no = t1.shape[0]
    o, v = slice(0, no), slice(no, None)
    goovv = g[o, o, v, v]
    return (torch.einsum("ia,ia->", f[o, v], t1)
            + 0.25 * torch.einsum("ijab,ijab->", goovv, t2)
            + 0.5 * torch.einsum("ijab,ia,jb->", goovv, t1, t1))


def residual(f: torch.Tensor, g: torch.Tensor, t1: torch.Tensor, t2: torch.Tensor):
    """Omega_1 [o,v] and Omega_2 [o,o,v,v] = <mu|e^{-T} H e^{T}|Phi_0> (Sec. 2.2)."""
    no = t1.shape[0]
    o, v = slice(0, no), slice(no, None)
    B = blocks(g, no)
    fov, foo, fvv = f[o, v], f[o, o], f[v, v]
    ein = torch.einsum

    tt = ein("ia,jb->ijab", t1, t1)
    tau_s = t2 + 0.5 * (tt - tt.transpose(2, 3))          # tau-tilde
    tau = t2 + tt - tt.transpose(2, 3)

    Fae = (fvv - 0.5 * ein("me,ma->ae", fov, t1)
           + ein("mf,mafe->ae", t1, B["ovvv"])
           - 0.5 * ein("mnaf,mnef->ae", tau_s, B["oovv"]))
    Fmi = (foo + 0.5 * ein("ie,me->mi", t1, fov)
           + ein("ne,mnie->mi", t1, B["ooov"])
           + 0.5 * ein("inef,mnef->mi", tau_s, B["oovv"]))
    Fme = fov + ein("nf,mnef->me", t1, B["oovv"])

    Wmnij = (B["oooo"] + _P(ein("je,mnie->mnij", t1, B["ooov"]), 2, 3)
             + 0.25 * ein("ijef,mnef->mnij", tau, B["oovv"]))
    Wabef = (B["vvvv"] - _P(ein("mb,amef->abef", t1, B["vovv"]), 0, 1)
             + 0.25 * ein("mnab,mnef->abef", tau, B["oovv"]))
    Wmbej = (B["ovvo"] + ein("jf,mbef->mbej", t1, B["ovvv"])
             - ein("nb,mnej->mbej", t1, B["oovo"])
             - ein("jnfb,mnef->mbej", 0.5 * t2 + ein("jf,nb->jnfb", t1, t1), B["oovv"]))

    # singles
    r1 = (f[v, o].transpose(0, 1).clone()
          + ein("ie,ae->ia", t1, Fae)
          - ein("ma,mi->ia", t1, Fmi)
          + ein("imae,me->ia", t2, Fme)
          - ein("nf,naif->ia", t1, B["ovov"])
          - 0.5 * ein("imef,maef->ia", t2, B["ovvv"])
          - 0.5 * ein("mnae,nmei->ia", t2, B["oovo"]))

    # doubles
    Fbe = Fae - 0.5 * ein("mb,me->be", t1, Fme)
    Fmj = Fmi + 0.5 * ein("je,me->mj", t1, Fme)
    r2 = ein("abij->ijab", B["vvoo"]).clone()
    r2 = r2 + _P(ein("ijae,be->ijab", t2, Fbe), 2, 3)
    r2 = r2 - _P(ein("imab,mj->ijab", t2, Fmj), 0, 1)
    r2 = r2 + 0.5 * ein("mnab,mnij->ijab", tau, Wmnij)
    r2 = r2 + 0.5 * ein("ijef,abef->ijab", tau, Wabef)
    ring = ein("imae,mbej->ijab", t2, Wmbej) - ein("ie,ma,mbej->ijab", t1, t1, B["ovvo"])
    r2 = r2 + _P(_P(ring, 0, 1), 2, 3)
    r2 = r2 + _P(ein("ie,abej->ijab", t1, B["vvvo"]), 0, 1)
    r2 = r2 - _P(ein("ma,mbij->ijab", t1, B["ovoo"]), 2, 3)
    return r1, r2


def first_order_t2(eps: torch.Tensor, g: torch.Tensor, no: int) -> torch.Tensor:
    """t_ij^ab = <ab||ij> / (e_i + e_j - e_a - e_b): the first-order doubles.

    Sec. 2.3 prints <ij||ab> in the numerator (real-orbital habit); for complex
    spinors the amplitude that cancels the first-order residual is <ab||ij>/D,
    i.e. the complex conjugate of <ij||ab>/D.
    """
    o, v = slice(0, no), slice(no, None)
    eo, ev = eps[o], eps[v]
    D = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    return torch.einsum("abij->ijab", g[v, v, o, o]) / D


def first_order_t2_from_L(eps: torch.Tensor, L: torch.Tensor, no: int) -> torch.Tensor:
    """Same amplitudes as first_order_t2, with <ab|ij> = sum_P L^P_ai L^P_bj formed directly."""
    Lvo = L[:, no:, :no]
    w = torch.einsum("Pai,Pbj->ijab", Lvo, Lvo)
    eo, ev = eps[:no], eps[no:]
    D = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    return (w - w.transpose(0, 1)) / D


# ---- unique-amplitude packing: vec = [t1 (o*v), t2 for i<j, a<b (P_o*P_v)] ----

def pair_index(n: int):
    i, j = torch.triu_indices(n, n, offset=1)
    return i, j


def pack(t1: torch.Tensor, t2: torch.Tensor) -> torch.Tensor:
    no, nv = t1.shape
    oi, oj = pair_index(no)
    vi, vj = pair_index(nv)
    t2p = t2[oi, oj][:, vi, vj]
    return torch.cat([t1.reshape(-1), t2p.reshape(-1)])


def unpack(vec: torch.Tensor, no: int, nv: int):
    n1 = no * nv
    oi, oj = pair_index(no)
    vi, vj = pair_index(nv)
    t1 = vec[:n1].reshape(no, nv)
    t2p = vec[n1:].reshape(len(oi), len(vi))
    t2 = torch.zeros(no, no, nv, nv, dtype=vec.dtype)
    blk = torch.zeros(len(oi), nv, nv, dtype=vec.dtype)
    blk[:, vi, vj] = t2p
    blk[:, vj, vi] = -t2p
    t2[oi, oj] = blk
    t2[oj, oi] = -blk
    return t1, t2


def n_amp(no: int, nv: int) -> int:
    return no * nv + (no * (no - 1) // 2) * (nv * (nv - 1) // 2)


def dot(a1, a2, b1, b2) -> torch.Tensor:
    """Bilinear (no conjugation) product over unique amplitudes: sum_ia + 1/4 sum_ijab."""
    return (a1 * b1).sum() + 0.25 * (a2 * b2).sum()
