"""Brute-force second quantisation on determinant bit strings -- oracle, test infrastructure.

Everything here is built from creation/annihilation operators acting on Slater
determinants, with no diagrammatic formula: H = sum h_pq a+_p a_q + 1/4 sum <pq||rs>
a+_p a+_q a_s a_r, T from the operator strings of Sec. 2.2 (a+_a a_i and
1/4 a+_a a+_b a_j a_i), e^{+-T} by the terminating power series, H-bar =
e^{-T} H e^{T} as a matrix, and the projections <mu|H-bar|Phi_0>.  Also the full CI
spectrum of H and the exact sum-over-states response function (Eq. sos).
Only for tiny spaces (n <= 12 spinors, N <= 3 electrons).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def space(n: int, N: int):
    dets = [sum(1 << p for p in c) for c in itertools.combinations(range(n), N)]
    return dets, {d: k for k, d in enumerate(dets)}


def _apply(ops, det):
    """Apply an operator string (rightmost first); ops = [(dagger, p), ...] left to right."""
    sign = 1
    for dag, p in reversed(ops):
        occ = (det >> p) & 1
        if dag == occ:          # a+ on occupied or a on empty
            return 0, None
        if bin(det & ((1 << p) - 1)).count("1") & 1:
            sign = -sign
        det ^= (1 << p)
    return sign, det


def op_matrix(terms, dets, index):
    """Matrix of sum_k c_k * (operator string k) in the determinant basis."""
    dim = len(dets)
    M = np.zeros((dim, dim), dtype=np.complex128)
    for c, ops in terms:
        if c == 0:
            continue
        for col, d in enumerate(dets):
            s, d2 = _apply(ops, d)
            if s:
                row = index.get(d2)
                if row is not None:
                    M[row, col] += s * c
    return M


def one_body(h, dets, index):
    n = h.shape[0]
    terms = [(h[p, q], [(1, p), (0, q)]) for p in range(n) for q in range(n)]
    return op_matrix(terms, dets, index)


def two_body(g, dets, index):
    """1/4 sum_pqrs <pq||rs> a+_p a+_q a_s a_r."""
    n = g.shape[0]
    terms = []
    for p, q, r, s in itertools.product(range(n), repeat=4):
        c = g[p, q, r, s]
        if c != 0 and p != q and r != s:
            terms.append((0.25 * c, [(1, p), (1, q), (0, s), (0, r)]))
    return op_matrix(terms, dets, index)


def t_operator(t1, t2, no, dets, index):
    """T1 + T2 with the operator strings of Sec. 2.2."""
    nv = t1.shape[1]
    terms = []
    for i in range(no):
        for a in range(nv):
            terms.append((t1[i, a], [(1, no + a), (0, i)]))
    for i, j in itertools.product(range(no), repeat=2):
        for a, b in itertools.product(range(nv), repeat=2):
            if i != j and a != b:
                terms.append((0.25 * t2[i, j, a, b], [(1, no + a), (1, no + b), (0, j), (0, i)]))
    return op_matrix(terms, dets, index)


def expm_nilpotent(T):
    E = np.eye(T.shape[0], dtype=np.complex128)
    term = E.copy()
    for k in range(1, T.shape[0] + 1):
        term = term @ T / k
        if not np.any(term):
            break
        E = E + term
    return E


class BruteForce:
    """Determinant-space machinery for N = no electrons in n spinors."""

    def __init__(self, f, g, no):
        self.f = np.asarray(f, dtype=np.complex128)
        self.g = np.asarray(g, dtype=np.complex128)
        self.no = no
        self.n = self.f.shape[0]
        self.nv = self.n - no
        self.dets, self.index = space(self.n, no)
        self.ref = (1 << no) - 1
        # h = f - sum_k <pk||qk>: the one-body operator whose Fock matrix is f
        h = self.f - np.einsum("pkqk->pq", self.g[:, :no, :, :no])
        self.H = one_body(h, self.dets, self.index) + two_body(self.g, self.dets, self.index)
        self.e_ref = self.H[self.index[self.ref], self.index[self.ref]]

    def ket(self, ops):
        """sign and row of the determinant ops|Phi_0>."""
        s, d = _apply(ops, self.ref)
        return s, self.index[d]

    def project(self, vec):
        """Singles/doubles components <mu|vec> with mu the excited determinants of Sec. 2.2."""
        no, nv = self.no, self.nv
        r1 = np.zeros((no, nv), np.complex128)
        r2 = np.zeros((no, no, nv, nv), np.complex128)
        for i in range(no):
            for a in range(nv):
                s, k = self.ket([(1, no + a), (0, i)])
                r1[i, a] = s * vec[k]
        for i, j in itertools.product(range(no), repeat=2):
            for a, b in itertools.product(range(nv), repeat=2):
                if i != j and a != b:
                    s, k = self.ket([(1, no + a), (1, no + b), (0, j), (0, i)])
                    r2[i, j, a, b] = s * vec[k]
        return r1, r2

    def hbar(self, t1, t2, op=None):
        T = t_operator(np.asarray(t1), np.asarray(t2), self.no, self.dets, self.index)
        Ep, Em = expm_nilpotent(T), expm_nilpotent(-T)
        return Em @ (self.H if op is None else op) @ Ep

    def residual(self, t1, t2):
        """Omega_mu = <mu|e^{-T} H e^{T}|Phi_0> and E_corr = <Phi_0|H-bar|Phi_0> - E_ref."""
        Hb = self.hbar(t1, t2)
        col = Hb[:, self.index[self.ref]]
        r1, r2 = self.project(col)
        return r1, r2, col[self.index[self.ref]] - self.e_ref

    def one_body_op(self, m):
        return one_body(np.asarray(m, dtype=np.complex128), self.dets, self.index)

    def xi(self, m, t1, t2):
        """xi_mu = <mu|e^{-T} V e^{T}|Phi_0> for a one-body V (Sec. 2.2)."""
        col = self.hbar(t1, t2, self.one_body_op(m))[:, self.index[self.ref]]
        return self.project(col)

    def fci(self):
        w, U = np.linalg.eigh(self.H)
        return w, U


def sos_response(w, U, ops_A, ops_B, omega, state):
    """Exact <<A;B>>_omega over eigenstates (Eq. sos), relative to eigenstate `state`.

    <<A;B>>_w = sum_k <0|A|k><k|B|0>/(w - w_k) - <0|B|k><k|A|0>/(w + w_k),
    with w_k = E_k - E_0 and the sum over k != 0.
    """
    psi0 = U[:, state]
    val = 0.0 + 0.0j
    for k in range(len(w)):
        if k == state:
            continue
        wk = w[k] - w[state]
        psik = U[:, k]
        a0k = psi0.conj() @ ops_A @ psik
        bk0 = psik.conj() @ ops_B @ psi0
        b0k = psi0.conj() @ ops_B @ psik
        ak0 = psik.conj() @ ops_A @ psi0
        val += a0k * bk0 / (omega - wk) - b0k * ak0 / (omega + wk)
    return val


def cc_state_overlap(U, t1, t2, bf: "BruteForce"):
    """Index of the eigenvector best matching e^T|Phi_0> (the CC state)."""
    T = t_operator(np.asarray(t1), np.asarray(t2), bf.no, bf.dets, bf.index)
    v = expm_nilpotent(T)[:, bf.index[bf.ref]]
    v = v / np.linalg.norm(v)
    ov = np.abs(U.conj().T @ v)
    return int(np.argmax(ov)), float(ov.max())
