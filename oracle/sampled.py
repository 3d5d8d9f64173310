"""sigma = A X one output entry at a time, straight from the Cholesky vectors -- oracle,
test infrastructure.

The same connected H-bar X term list as ``jacobian.sigma_terms`` (Sec. 2.2 Jacobian, exact
two-body H-bar elements in the T1-dressed form), but every H-bar element is formed only for
the indices one output entry needs, from the T1-dressed Cholesky vectors L~ (Sec. 3: the
integrals with more than two virtual indices are built on the fly).  Nothing of size v^3
or v^4 is ever held, so this runs at the full workload sizes where the explicit tensors of
``jacobian`` do not fit; its cost is O(o^2 v^2 + naux v^2) per entry.  It is pinned against
``jacobian.sigma_terms`` entry by entry at small sizes.

The same terms vectorised over whole blocks: ``sigma1_all`` (every singles entry),
``sigma_rest`` (every term but the particle-particle ladder) and ``sigma_blocked`` (the whole
vector, the ladder's <ab|ef>~ formed chunk by chunk of a from L~_vv, never held whole).  They
are the oracle's whole-vector sigma at sizes where the v^4 tensor does not fit, and the CPU
timing of one sigma; pinned against ``jacobian.sigma_terms`` at small sizes.
"""
from __future__ import annotations

import torch

from .integrals import C128

ein = torch.einsum


class EntrySigma:
    def __init__(self, eps, L, t1, t2):
        no, nv = t1.shape
        n = no + nv
        self.no, self.nv = no, nv
        o, v = slice(0, no), slice(no, n)
        self.t1, self.t2 = t1, t2
        # undressed blocks and the one-body part h = f - sum_k <pk||qk>
        Loo, Lov, Lvo, Lvv = L[:, o, o], L[:, o, v], L[:, v, o], L[:, v, v]
        f = torch.diag(eps.to(C128))
        tr = ein("Pkk->P", Loo)
        h = f - (ein("Ppq,P->pq", L, tr) - ein("Ppk,Pkq->pq", L[:, :, o], L[:, o, :]))
        # T1 dressing L~ = (1 - t) L (1 + t), t_ai = t_i^a, block by block
        self.Loo = Loo + ein("Pib,jb->Pij", Lov, t1)
        self.Lov = Lov.clone()
        Mvv = Lvv - ein("ma,Pmb->Pab", t1, Lov)
        Mvo = Lvo - ein("ma,Pmi->Pai", t1, Loo)
        self.Lvv = Mvv
        self.Lvo = Mvo + ein("Pab,ib->Pai", Mvv, t1)
        # dressed Fock f~ = (1 - t) h (1 + t) + sum_k <pk||qk>~ (oo, ov, vv blocks)
        hoo, hov, hvv = h[o, o], h[o, v], h[v, v]
        trt = ein("Pkk->P", self.Loo)
        self.foo = (hoo + hov @ t1.T + ein("Pij,P->ij", self.Loo, trt)
                    - ein("Pik,Pkj->ij", self.Loo, self.Loo))
        self.fov = hov + ein("Pia,P->ia", self.Lov, trt) - ein("Pik,Pka->ia", self.Loo, self.Lov)
        self.fvv = (hvv - t1.T @ hov + ein("Pab,P->ab", self.Lvv, trt)
                    - ein("Pak,Pkb->ab", self.Lvo, self.Lov))
        # stored blocks with at most two virtual indices
        self.oovv = ein("Pme,Pnf->mnef", self.Lov, self.Lov)
        self.oovv = self.oovv - self.oovv.transpose(2, 3)
        self.ooov = ein("Pmi,Pne->mnie", self.Loo, self.Lov) - ein("Pme,Pni->mnie", self.Lov, self.Loo)
        # the same blocks in the layouts the per-entry matrix-vector products read
        self.oovv_m = self.oovv.reshape(no, -1)                                    # [m][nef]
        self.oovv_e = self.oovv.permute(2, 0, 1, 3).reshape(nv, -1).contiguous()    # [e][mnf]
        self.oovv_me = self.oovv.permute(0, 2, 1, 3).reshape(no * nv, -1).contiguous()  # [me][nf]
        self.oovv_mn = self.oovv.reshape(no * no, -1)                              # [mn][ef]
        self.Lov_m = self.Lov.permute(1, 0, 2).reshape(no, -1).contiguous()         # [m][Pe]
        self.naux = L.shape[0]
        # one-body and oooo elements are cheap as whole matrices (at most o^4 v^2 work)
        t2e = t2.permute(2, 0, 1, 3).reshape(nv, -1)
        self.Fvv = self.fvv - 0.5 * (t2e @ self.oovv_e.T)                              # [b][e]
        self.Foo = self.foo + 0.5 * (self.oovv_m @ t2.reshape(no, -1).T)               # [m][j]
        w = ein("Pmi,Pnj->mnij", self.Loo, self.Loo)
        self.Woooo = (w - w.transpose(2, 3)
                      + 0.5 * (self.oovv_mn @ t2.reshape(no * no, -1).T).reshape(no, no, no, no))

    def set_x(self, x1, x2):
        self.x1, self.x2 = x1, x2
        self.w = ein("Pmf,mf->P", self.Lov, x1)
        self._z = {}
        no, nv = self.no, self.nv
        u = ein("Pbf,mf->Pbm", self.Lvv, x1)
        self.Xvv = (ein("Pbe,P->be", self.Lvv, self.w) - ein("Pbm,Pme->be", u, self.Lov)
                    - 0.5 * (x2.permute(2, 0, 1, 3).reshape(nv, -1) @ self.oovv_e.T))
        self.Xoo = ein("mnje,ne->mj", self.ooov, x1) + 0.5 * (self.oovv_m @ x2.reshape(no, -1).T)
        self.Z = 0.5 * (self.oovv_mn @ x2.reshape(no * no, -1).T).reshape(no, no, no, no)

    # ---- H-bar elements on demand (index conventions as in jacobian.Dressed)
    def Fvv_row(self, b):          # Fvv[b, e]
        return self.Fvv[b]

    def Foo_col(self, j):          # Foo[m, j]
        return self.Foo[:, j]

    def Woooo_ij(self, i, j):      # Woooo[m, n, i, j]
        return self.Woooo[:, :, i, j]

    def Wovvo_bj(self, b, j):      # Wovvo[m, b, e, j] over (m, e)
        if getattr(self, "_wovvo", None) is not None:      # the whole block, when formed
            return self._wovvo[:, b, :, j]
        w = ein("Pme,P->me", self.Lov, self.Lvo[:, b, j]) - ein("Pm,Pe->me", self.Loo[:, :, j], self.Lvv[:, b, :])
        return w - (self.oovv_me @ self.t2[j, :, :, b].reshape(-1)).reshape(self.no, self.nv)

    def Wvvvo_abj(self, a, b, j):  # Wvvvo[a, b, e, j] over e
        t2 = self.t2
        w = ein("Pe,P->e", self.Lvv[:, a, :], self.Lvo[:, b, j]) - ein("P,Pe->e", self.Lvo[:, a, j], self.Lvv[:, b, :])
        w = w - ein("me,m->e", self.fov, t2[:, j, a, b])
        w = w - 0.5 * ein("mne,mn->e", self.ooov[:, :, j, :], t2[:, :, a, b])   # <mn||ej> = -<mn||je>

        def ring(bb, aa):  # sum_mf <m bb||e f>~ t_mj^{aa f}
            y = ein("Pf,mf->Pm", self.Lvv[:, bb, :], t2[:, j, aa, :])
            r = ein("Pme,Pm->e", self.Lov, y)
            return r - ein("Pe,P->e", self.Lvv[:, bb, :], ein("Pmf,mf->P", self.Lov, t2[:, j, aa, :]))
        return w - (ring(b, a) - ring(a, b))

    def Wovoo_bij(self, b, i, j):  # Wovoo[m, b, i, j] over m
        t2 = self.t2
        w = ein("Pm,P->m", self.Loo[:, :, i], self.Lvo[:, b, j]) - ein("Pm,P->m", self.Loo[:, :, j], self.Lvo[:, b, i])
        w = w - ein("me,e->m", self.fov, t2[i, j, b, :])
        y = ein("Pf,ef->Pe", self.Lvv[:, b, :], t2[i, j])
        w = w + self.Lov_m @ y.reshape(-1)
        w = w + ein("mne,ne->m", self.ooov[:, :, i, :], t2[j, :, b, :]) - ein("mne,ne->m", self.ooov[:, :, j, :], t2[i, :, b, :])
        return w

    def Xvv_row(self, b):          # Xvv[b, e]
        return self.Xvv[b]

    def Xoo_col(self, j):          # Xoo[m, j]
        return self.Xoo[:, j]

    def Z_ij(self, i, j):
        return self.Z[:, :, i, j]

    def Zp_i(self, i):             # sum_mf L~_mf X_im^ef over (P, e)
        if i not in self._z:
            self._z[i] = ein("Pmf,mef->Pe", self.Lov, self.x2[i])
        return self._z[i]

    # ---- entries
    def sigma1(self, i, a):
        x1, x2 = self.x1, self.x2
        val = (self.Fvv_row(a) @ x1[i] - self.Foo_col(i) @ x1[:, a]
               + (self.Wovvo_bj(a, i) * x1).sum()
               + (self.fov * x2[i, :, a, :]).sum()
               + ein("Pe,Pe->", self.Lvv[:, a, :], self.Zp_i(i))
               - 0.5 * ein("mne,mne->", self.ooov[:, :, i, :], x2[:, :, a, :]))
        return val

    def sigma2(self, i, j, a, b):
        x1, x2, t2 = self.x1, self.x2, self.t2

        def base_ab(i, j, a, b):
            return (self.Fvv_row(b) @ x2[i, j, a] - self.Wovoo_bij(b, i, j) @ x1[:, a]
                    + self.Xvv_row(b) @ t2[i, j, a])

        def base_ij(i, j, a, b):
            return (-self.Foo_col(j) @ x2[i, :, a, b] + self.Wvvvo_abj(a, b, j) @ x1[i]
                    - self.Xoo_col(j) @ t2[i, :, a, b])

        def ring(i, j, a, b):
            return (self.Wovvo_bj(b, j) * x2[i, :, a, :]).sum()

        val = base_ab(i, j, a, b) - base_ab(i, j, b, a)
        val = val + base_ij(i, j, a, b) - base_ij(j, i, a, b)
        val = val + 0.5 * (self.Woooo_ij(i, j) * x2[:, :, a, b]).sum()
        val = val + ((self.Lvv[:, a, :] @ x2[i, j]) * self.Lvv[:, b, :]).sum()
        val = val + 0.5 * (t2[:, :, a, b] * self.Z_ij(i, j)).sum()
        val = val + ring(i, j, a, b) - ring(j, i, a, b) - ring(i, j, b, a) + ring(j, i, b, a)
        return val

    # ---- whole vectors, vectorised over entries (same terms as sigma1 / sigma2 above)
    def sigma1_all(self):
        """Every singles entry sigma_1[i, a] at once: the terms of sigma1() with the sums over
        (i, a) written as one einsum each (Wovvo is formed whole: o^2 v^2 entries)."""
        x1, x2 = self.x1, self.x2
        Wovvo = self.Wovvo_full()
        Zp = ein("Pmf,imef->iPe", self.Lov, x2)
        return (ein("ae,ie->ia", self.Fvv, x1) - ein("mi,ma->ia", self.Foo, x1)
                + ein("maei,me->ia", Wovvo, x1)
                + ein("me,imae->ia", self.fov, x2)
                + ein("Pae,iPe->ia", self.Lvv, Zp)
                - 0.5 * ein("mnie,mnae->ia", self.ooov, x2))

    def Wovvo_full(self):
        """Wovvo[m, b, e, j] = <mb||ej>~ - sum_nf <mn||ef> t_jn^fb (every (b, j) of Wovvo_bj)."""
        if getattr(self, "_wovvo", None) is None:
            self._wovvo = (ein("Pme,Pbj->mbej", self.Lov, self.Lvo) - ein("Pmj,Pbe->mbej", self.Loo, self.Lvv)
                           - ein("mnef,jnfb->mbej", self.oovv, self.t2))
        return self._wovvo

    def Wovoo_full(self, b_chunk=16):
        """Wovoo[m, b, i, j] for every (b, i, j) (the terms of Wovoo_bij); the <mb|ef>~ t_ij^ef
        part is formed in chunks of b from L~ (no tensor with three virtual indices is held
        whole)."""
        if getattr(self, "_wovoo", None) is not None:
            return self._wovoo
        t2 = self.t2
        w = (ein("Pmi,Pbj->mbij", self.Loo, self.Lvo) - ein("Pmj,Pbi->mbij", self.Loo, self.Lvo)
             - ein("me,ijbe->mbij", self.fov, t2)
             + ein("mnie,jnbe->mbij", self.ooov, t2) - ein("mnje,inbe->mbij", self.ooov, t2))
        for b0 in range(0, self.nv, b_chunk):
            b1 = min(self.nv, b0 + b_chunk)
            G = ein("Pme,Pbf->mbef", self.Lov, self.Lvv[:, b0:b1])    # <mb|ef>~ for the chunk
            w[:, b0:b1] += ein("mbef,ijef->mbij", G, t2)
        self._wovoo = w
        return w

    def wx_all(self):
        """WX[i, j, a, b] = sum_e Wvvvo[a, b, e, j] x_i^e for every entry (the terms of Wvvvo_abj
        with the sum over e taken first: U = L~_ae x_ie, s = L~_me x_ie, V_mbif = <mb||ef>~ x_ie)."""
        x1, t2 = self.x1, self.t2
        U = ein("Pae,ie->Pai", self.Lvv, x1)
        s = ein("Pme,ie->Pmi", self.Lov, x1)
        c = ein("me,ie->mi", self.fov, x1)
        d = ein("mnje,ie->mnji", self.ooov, x1)
        V = ein("Pmi,Pbf->mbif", s, self.Lvv) - ein("Pmf,Pbi->mbif", self.Lov, U)
        r = ein("Pai,Pbj->ijab", U, self.Lvo) - ein("Paj,Pbi->ijab", self.Lvo, U)
        r = r - ein("mi,mjab->ijab", c, t2) - 0.5 * ein("mnji,mnab->ijab", d, t2)
        r = r - ein("mbif,mjaf->ijab", V, t2) + ein("maif,mjbf->ijab", V, t2)
        return r

    def sigma_rest(self):
        """sigma_1 and every sigma_2 term except the particle-particle ladder, vectorised."""
        x1, x2, t2 = self.x1, self.x2, self.t2
        s1 = self.sigma1_all()
        Wovoo = self.Wovoo_full()
        Wovvo = self.Wovvo_full()
        Rab = (ein("be,ijae->ijab", self.Fvv, x2) - ein("mbij,ma->ijab", Wovoo, x1)
               + ein("be,ijae->ijab", self.Xvv, t2))
        Rij = (-ein("mj,imab->ijab", self.Foo, x2) + self.wx_all() - ein("mj,imab->ijab", self.Xoo, t2))
        s2 = Rab - Rab.transpose(2, 3) + Rij - Rij.transpose(0, 1)
        s2 = s2 + 0.5 * ein("mnij,mnab->ijab", self.Woooo, x2) + 0.5 * ein("mnab,mnij->ijab", t2, self.Z)
        ring = ein("mbej,imae->ijab", Wovvo, x2)
        s2 = s2 + ring - ring.transpose(0, 1) - ring.transpose(2, 3) + ring.transpose(0, 1).transpose(2, 3)
        return s1, s2

    def ladder_chunk(self, a0, a1, out):
        """out[i, j, a, b] += sum_ef <ab|ef>~ X_ij^ef for a0 <= a < a1 (= 1/2 sum <ab||ef>~ X_ij^ef,
        X antisymmetric in ef), with <ab|ef>~ = sum_P L~_ae L~_bf formed for the chunk only."""
        g = ein("Pae,Pbf->abef", self.Lvv[:, a0:a1], self.Lvv)
        out[:, :, a0:a1, :] += ein("abef,ijef->ijab", g, self.x2)

    def sigma_blocked(self, a_chunk=8):
        """The whole sigma = A X: sigma_rest plus the ladder formed chunk by chunk of a from L~_vv
        (nothing with four virtual indices is held whole; the explicit-tensor term list of
        jacobian.sigma_terms needs v^4 entries)."""
        s1, s2 = self.sigma_rest()
        for a0 in range(0, self.nv, a_chunk):
            self.ladder_chunk(a0, min(self.nv, a0 + a_chunk), s2)
        return s1, s2
