"""Two-electron integrals from Cholesky vectors (Sec. 3) -- oracle, test infrastructure.

Convention (the paper only says "Cholesky vectors"): physicist integrals
    <pq|rs> = (pr|qs) = sum_P L^P_pr L^P_qs,
each L^P Hermitian, as for real-AO Cholesky vectors transformed to spinors.
Antisymmetrised: <pq||rs> = <pq|rs> - <pq|sr>.
"""
from __future__ import annotations

import numpy as np
import torch

C128 = torch.complex128


def as_t(x) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        return x.to(C128) if x.is_complex() else x.to(torch.float64)
    x = np.asarray(x)
    return torch.from_numpy(x.astype(np.complex128) if np.iscomplexobj(x) else x.astype(np.float64))


def eri_phys(L: torch.Tensor) -> torch.Tensor:
    """Full <pq|rs> tensor [n,n,n,n] = sum_P L^P_pr L^P_qs (Sec. 3)."""
    return torch.einsum("Ppr,Pqs->pqrs", L, L)


def eri_anti(L: torch.Tensor) -> torch.Tensor:
    """Full <pq||rs> = <pq|rs> - <pq|sr>."""
    g = eri_phys(L)
    return g - g.transpose(2, 3)


def fock_from_h(h: torch.Tensor, g_anti: torch.Tensor, no: int) -> torch.Tensor:
    """f_pq = h_pq + sum_k <pk||qk> over occupied k (normal ordering w.r.t. Phi_0)."""
    return h + torch.einsum("pkqk->pq", g_anti[:, :no, :, :no])


def h_from_fock(f: torch.Tensor, g_anti: torch.Tensor, no: int) -> torch.Tensor:
    """Inverse of fock_from_h: the one-body operator whose Fock matrix is f."""
    return f - torch.einsum("pkqk->pq", g_anti[:, :no, :, :no])


def pivoted_cholesky(G: np.ndarray, tau: float, max_vec: int | None = None):
    """Single-step pivoted Cholesky of a Hermitian PSD matrix (Sec. 3).

    Vectors are added, each at the largest remaining diagonal, until that diagonal
    falls below tau.  Returns K [N, m] with G ~= K K^H and the final max residual
    diagonal.
    """
    G = np.array(G, dtype=np.complex128)
    N = G.shape[0]
    d = np.real(np.diag(G)).copy()
    vecs = []
    max_vec = N if max_vec is None else max_vec
    while len(vecs) < max_vec:
        p = int(np.argmax(d))
        if d[p] < tau:
            break
        col = G[:, p].copy()
        for k in vecs:
            col -= k * np.conj(k[p])
        k = col / np.sqrt(d[p])
        vecs.append(k)
        d -= np.abs(k) ** 2
    K = np.stack(vecs, axis=1) if vecs else np.zeros((N, 0), np.complex128)
    return K, float(d.max()) if N else 0.0
