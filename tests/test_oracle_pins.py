"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

* residual and energy vs brute-force second quantisation (e^{-T} H e^{T} on determinants)
* Jacobian: connected term list vs the polynomial-exact stencil of Omega, and
  entry by entry vs finite differences of the brute-force residual at o=2, v=4
* transpose product: bilinear identity and the explicit transpose
* xi vs brute force; eta0 vs finite differences of E
* alpha vs the exact sum over states at o=2 (CCSD = FCI for two electrons)
* static alpha vs the finite-field second derivative of the CCSD energy at o=3
* left (Y) route = right (X-only) route; Hermiticity of alpha
* Cholesky: pivoted decomposition reconstructs (pr|qs) within the threshold
"""
import numpy as np
import pytest
import torch

from oracle import ccsd, jacobian as J, response as R, secondq
from oracle.integrals import as_t, eri_anti, eri_phys, pivoted_cholesky
from paper_2604_12914_gb300.inputs import make_system, random_amplitudes, make_config

from oracle_helpers import oracle_problem, hermitian

C = torch.complex128


def _system(o, v, naux, seed, scale, t1_scale=0.0):
    return make_system(o, v, naux, seed=seed, scale=scale, t1_scale=t1_scale)


@pytest.mark.parametrize("o,v,naux", [(2, 4, 6), (3, 5, 8)])
def test_residual_energy_vs_brute_force(o, v, naux, rng):
    s = _system(o, v, naux, seed=3, scale=0.5, t1_scale=0.3)
    L = as_t(s.L)
    g = eri_anti(L)
    f = torch.diag(as_t(s.eps).to(C)) + as_t(hermitian(rng, o + v, 0.1))   # non-canonical
    a1, a2 = random_amplitudes(o, v, seed=9, s1=0.3, s2=0.3)
    t1, t2 = as_t(a1), as_t(a2)
    bf = secondq.BruteForce(f.numpy(), g.numpy(), o)
    r1b, r2b, eb = bf.residual(t1.numpy(), t2.numpy())
    r1, r2 = ccsd.residual(f, g, t1, t2)
    e = ccsd.energy(f, g, t1, t2)
    assert abs(e.item() - eb) < 1e-12
    assert np.abs(r1.numpy() - r1b).max() < 1e-12
    assert np.abs(r2.numpy() - r2b).max() < 1e-12 * max(1.0, np.abs(r2b).max())


def test_integrals_bruteforce_sum():
    s = make_config("C1")
    L = as_t(s.L)
    g = eri_phys(L)
    rng = np.random.default_rng(0)
    for _ in range(20):
        p, q, r, t = rng.integers(0, s.n, 4)
        ref = sum(s.L[P, p, r] * s.L[P, q, t] for P in range(s.naux))
        assert abs(g[p, q, r, t].item() - ref) < 1e-10
    # Hermiticity <pq|rs>* = <rs|pq> and particle symmetry <pq|rs> = <qp|sr>
    sub = g[:12, :12, :12, :12]
    assert torch.allclose(sub.conj(), sub.permute(2, 3, 0, 1), atol=1e-12)
    assert torch.allclose(sub, sub.permute(1, 0, 3, 2), atol=1e-12)


@pytest.mark.parametrize("case", ["T0", "T2", "T1", "T1T2"])
def test_sigma_terms_vs_stencil(case):
    o, v, naux = 3, 6, 10
    s = _system(o, v, naux, seed=3, scale=0.5)
    L = as_t(s.L)
    g = eri_anti(L)
    f = torch.diag(as_t(s.eps).to(C))
    a1, a2 = random_amplitudes(o, v, seed=9, s1=0.3, s2=0.3)
    t1 = as_t(a1) if "T1" in case else torch.zeros(o, v, dtype=C)
    t2 = as_t(a2) if "T2" in case else torch.zeros(o, o, v, v, dtype=C)
    x1, x2 = map(as_t, random_amplitudes(o, v, seed=11))
    s1, s2 = J.sigma_stencil(f, g, t1, t2, x1, x2)
    q1, q2 = J.sigma_terms(J.Dressed(f, L, t1, t2), x1, x2)
    scale = float(s2.abs().max())
    assert float((s1 - q1).abs().max()) < 1e-12 * scale
    assert float((s2 - q2).abs().max()) < 1e-12 * scale


def test_jacobian_entrywise_vs_bruteforce_fd():
    """A_mu,nu at o=2, v=4 from central differences of the brute-force residual."""
    o, v = 2, 4
    s = _system(o, v, 6, seed=5, scale=0.4, t1_scale=0.2)
    P = oracle_problem(s)
    a1, a2 = random_amplitudes(o, v, seed=4, s1=0.2, s2=0.2)
    P.t1, P.t2 = as_t(a1), as_t(a2)
    A = P.jacobian_matrix()
    bf = secondq.BruteForce(P.f.numpy(), P.g.numpy(), o)
    N = P.nvec
    h = 1e-4
    Afd = np.zeros((N, N), complex)
    for k in range(N):
        e = torch.zeros(N, dtype=C)
        e[k] = 1.0
        d1, d2 = P.unpack(e)
        cols = []
        for sgn in (+1, -1):
            r1, r2, _ = bf.residual((P.t1 + sgn * h * d1).numpy(), (P.t2 + sgn * h * d2).numpy())
            cols.append(P.pack(torch.from_numpy(r1), torch.from_numpy(r2)).numpy())
        Afd[:, k] = (cols[0] - cols[1]) / (2 * h)
    assert np.abs(A.numpy() - Afd).max() < 1e-6 * np.abs(Afd).max()


def test_sigma_linear_and_antisymmetric():
    o, v = 3, 7
    s = _system(o, v, 9, seed=6, scale=0.5, t1_scale=0.1)
    P = oracle_problem(s)
    x1, x2 = map(as_t, random_amplitudes(o, v, seed=1))
    y1, y2 = map(as_t, random_amplitudes(o, v, seed=2))
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    s_x = P.sigma(x1, x2)
    s_y = P.sigma(y1, y2)
    s_c = P.sigma(a * x1 + b * y1, a * x2 + b * y2)
    ref = (a * s_x[0] + b * s_y[0], a * s_x[1] + b * s_y[1])
    sc = float(s_c[1].abs().max())
    assert float((s_c[0] - ref[0]).abs().max()) < 1e-13 * sc
    assert float((s_c[1] - ref[1]).abs().max()) < 1e-13 * sc
    s2 = s_x[1]
    assert float((s2 + s2.transpose(0, 1)).abs().max()) < 1e-13 * sc
    assert float((s2 + s2.transpose(2, 3)).abs().max()) < 1e-13 * sc


def test_sigma_T_bilinear_and_explicit_transpose():
    o, v = 2, 4
    s = _system(o, v, 6, seed=7, scale=0.5, t1_scale=0.2)
    P = oracle_problem(s)
    x1, x2 = map(as_t, random_amplitudes(o, v, seed=1))
    y1, y2 = map(as_t, random_amplitudes(o, v, seed=2))
    sx = P.sigma(x1, x2)
    sty = J.sigma_T(P.f, P.g, P.t1, P.t2, y1, y2)
    lhs = ccsd.dot(y1, y2, *sx)
    rhs = ccsd.dot(*sty, x1, x2)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    A = P.jacobian_matrix()
    z = A.transpose(0, 1) @ P.pack(y1, y2)
    assert float((P.pack(*sty) - z).abs().max()) < 1e-12 * float(z.abs().max())


def test_xi_vs_bruteforce():
    o, v = 3, 5
    s = _system(o, v, 8, seed=8, scale=0.5, t1_scale=0.2)
    P = oracle_problem(s)
    a1, a2 = random_amplitudes(o, v, seed=3, s1=0.3, s2=0.3)
    P.t1, P.t2 = as_t(a1), as_t(a2)
    B = as_t(s.mu[2])
    bf = secondq.BruteForce(P.f.numpy(), P.g.numpy(), o)
    r1b, r2b = bf.xi(B.numpy(), P.t1.numpy(), P.t2.numpy())
    r1, r2 = P.xi(B)
    assert np.abs(r1.numpy() - r1b).max() < 1e-12
    assert np.abs(r2.numpy() - r2b).max() < 1e-12


def test_eta0_vs_energy_fd():
    o, v = 3, 5
    s = _system(o, v, 8, seed=9, scale=0.5, t1_scale=0.2)
    P = oracle_problem(s)
    a1, a2 = random_amplitudes(o, v, seed=5, s1=0.3, s2=0.3)
    P.t1, P.t2 = as_t(a1), as_t(a2)
    e0 = P.eta0()
    d1, d2 = map(as_t, random_amplitudes(o, v, seed=6))
    h = 1e-3
    fd = sum(c * P.energy(P.t1 + k * h * d1, P.t2 + k * h * d2) for c, k in R.STENCIL) / (12 * h)
    assert abs(fd - e0 @ P.pack(d1, d2)) < 1e-10 * abs(fd)


@pytest.mark.parametrize("omega,gamma", [(0.0, 0.05), (0.0428, 0.01), (0.7, 0.02)])
def test_damped_alpha_vs_sum_over_states(omega, gamma):
    """Two electrons, complex frequency z = omega + i gamma: the damped CC response equals
    Eq. sos continued to complex z (no symmetry in z is assumed by the sum; 0.7 lies near
    an excitation, where the damping matters)."""
    o, v = 2, 4
    s = _system(o, v, 6, seed=2, scale=0.3)
    P = oracle_problem(s, converge=True)
    bf = secondq.BruteForce(P.f.numpy(), P.g.numpy(), o)
    w, U = bf.fci()
    st, ov = secondq.cc_state_overlap(U, P.t1.numpy(), P.t2.numpy(), bf)
    assert ov > 1 - 1e-10
    mu = [as_t(m) for m in s.mu]
    ops = [bf.one_body_op(m.numpy()) for m in mu]
    z = complex(omega, gamma)
    al = R.alpha(P, mu, omega, gamma=gamma).numpy()
    sos = np.array([[-secondq.sos_response(w, U, ops[a], ops[b], z, st) for b in range(3)]
                    for a in range(3)])
    assert np.abs(al - sos).max() < 1e-10 * np.abs(sos).max()
    d = np.diag(al)
    if omega == 0.0:
        # imaginary frequency: Hermitian operators give a real diagonal
        assert np.abs(d.imag).max() < 1e-12 * np.abs(d).max()
    else:
        # absorption: damping gives the diagonal a nonzero imaginary part of one sign
        assert np.all(d.imag > 0) or np.all(d.imag < 0)


@pytest.mark.parametrize("omega", [0.0, 0.0428])
def test_alpha_vs_sum_over_states(omega):
    """Two electrons: CCSD is exact, so CC linear response equals Eq. sos."""
    o, v = 2, 4
    s = _system(o, v, 6, seed=2, scale=0.3)
    P = oracle_problem(s, converge=True)
    bf = secondq.BruteForce(P.f.numpy(), P.g.numpy(), o)
    w, U = bf.fci()
    st, ov = secondq.cc_state_overlap(U, P.t1.numpy(), P.t2.numpy(), bf)
    assert ov > 1 - 1e-10
    mu = [as_t(m) for m in s.mu]
    ops = [bf.one_body_op(m.numpy()) for m in mu]
    al = R.alpha(P, mu, omega).numpy()
    sos = np.array([[-secondq.sos_response(w, U, ops[a], ops[b], omega, st) for b in range(3)]
                    for a in range(3)])
    assert np.abs(al - sos).max() < 1e-10 * np.abs(sos).max()
    # Hermitian tensor, real diagonal
    assert np.abs(al - al.conj().T).max() < 1e-12 * np.abs(al).max()
    # excitation energies: eig(A) = FCI excitation energies from the CC state
    eigA = np.sort(np.linalg.eigvals(P.jacobian_matrix().numpy()).real)
    exc = np.sort(np.delete(w - w[st], st))
    assert np.abs(eigA - exc).max() < 1e-10


def test_left_route_equals_right_route():
    o, v = 2, 5
    s = _system(o, v, 6, seed=12, scale=0.3)
    P = oracle_problem(s, converge=True)
    mu = [as_t(m) for m in s.mu]
    omega = 0.05
    A = P.jacobian_matrix()
    lam = torch.linalg.solve(A.transpose(0, 1), -P.eta0())
    gl = R.g_left(P, mu[0], mu[2], omega, lam=lam, A=A)
    xi = [P.pack(*P.xi(m)) for m in mu]
    Xb = P.unpack(R.solve_x(A, xi[2], omega))
    Xa = P.unpack(R.solve_x(A, xi[0], -omega))
    gr = P.eta_dot(mu[0], lam, *Xb) + P.eta_dot(mu[2], lam, *Xa) + P.fxx(lam, Xa, Xb)
    assert abs(gl - gr) < 1e-10 * abs(gr)


@pytest.mark.slow
def test_static_alpha_vs_finite_field():
    """o=3: unconjugated g(A,B;0) = d^2 E / dF_A dF_B (unrelaxed orbitals, V = +F mu)."""
    o, v = 3, 5
    s = _system(o, v, 8, seed=14, scale=0.3)
    P = oracle_problem(s, converge=True)
    mu = [as_t(m) for m in s.mu]
    A = P.jacobian_matrix()
    lam = torch.linalg.solve(A.transpose(0, 1), -P.eta0())

    def e_field(FA, FB, a, b):
        f = P.f + FA * mu[a] + FB * mu[b]
        t1, t2, _ = R.solve_ccsd(f, P.g, o, t1=P.t1, t2=P.t2, tol=1e-13, L=P.L)
        return ccsd.energy(f, P.g, t1, t2).item()

    h = 2e-3
    for a, b in [(2, 2), (0, 2)]:
        d2 = (e_field(h, h, a, b) - e_field(h, -h, a, b) - e_field(-h, h, a, b) + e_field(-h, -h, a, b)) / (4 * h * h)
        xi = [P.pack(*P.xi(m)) for m in mu]
        Xa = P.unpack(R.solve_x(A, xi[a], 0.0))
        Xb = P.unpack(R.solve_x(A, xi[b], 0.0))
        g = P.eta_dot(mu[a], lam, *Xb) + P.eta_dot(mu[b], lam, *Xa) + P.fxx(lam, Xa, Xb)
        assert abs(g - d2) < 2e-5 * abs(d2), (a, b, g, d2)


def test_cholesky_reconstruction():
    """(pr|qs) supermatrix from the C1-sized L: pivoted CD to tau reproduces it within tau."""
    s = make_system(6, 14, 40, seed=1)
    n = s.n
    Lm = s.L.reshape(s.naux, n * n)                       # row P, column (p,r)
    # G_(pr),(sq) = (pr|qs) = sum_P L^P_pr L^P_qs, with L^P_qs = conj(L^P_sq)
    G = Lm.T @ np.conj(Lm)
    assert np.abs(G - G.conj().T).max() < 1e-10
    for tau in (1e-2, 1e-5):
        K, dmax = pivoted_cholesky(G, tau)
        assert K.shape[1] <= s.naux
        assert dmax < tau
        assert np.abs(G - K @ K.conj().T).max() <= tau + 1e-10


def test_first_order_amplitudes_cancel_first_order_residual():
    o, v = 3, 6
    s = _system(o, v, 8, seed=15, scale=1.0)
    L = as_t(s.L)
    f = torch.diag(as_t(s.eps).to(C))
    res = []
    for lam_ in (1e-3, 2e-3):
        g = eri_anti(L * np.sqrt(lam_))
        t2 = ccsd.first_order_t2(as_t(s.eps), g, o)
        r1, r2 = ccsd.residual(f, g, torch.zeros(o, v, dtype=C), t2)
        res.append(float(r2.abs().max()))
    # remaining residual is second order in the interaction
    assert 3.5 < res[1] / res[0] < 4.5


def test_entrywise_sigma_matches_term_list():
    """oracle.sampled (per-entry, Cholesky on the fly) = jacobian.sigma_terms entry by entry."""
    from oracle import sampled
    o, v = 4, 9
    s = _system(o, v, 13, seed=3, scale=0.5, t1_scale=0.2)
    L = as_t(s.L)
    f = torch.diag(as_t(s.eps).to(C))
    _, a2 = random_amplitudes(o, v, seed=9, s1=0.2, s2=0.3)
    t1, t2 = as_t(s.t1), as_t(a2)
    x1, x2 = map(as_t, random_amplitudes(o, v, seed=11))
    q1, q2 = J.sigma_terms(J.Dressed(f, L, t1, t2), x1, x2)
    E = sampled.EntrySigma(as_t(s.eps), L, t1, t2)
    E.set_x(x1, x2)
    rng = np.random.default_rng(1)
    sc = float(q2.abs().max())
    for _ in range(12):
        i, j = rng.integers(0, o, 2)
        a, b = rng.integers(0, v, 2)
        assert abs(E.sigma2(i, j, a, b) - q2[i, j, a, b]) < 1e-12 * sc
        assert abs(E.sigma1(i, a) - q1[i, a]) < 1e-12 * sc


@pytest.mark.parametrize("o,v,naux,seed", [(3, 6, 8, 15), (4, 5, 11, 16)])
def test_first_order_t2_from_L_matches_explicit_integrals(o, v, naux, seed):
    """The Cholesky-direct first-order doubles (<ab|ij> = sum_P L^P_ai L^P_bj formed straight
    from L, the reference for every full-size T2 check) equal first_order_t2 on the explicit
    <pq||rs>, which the first-order-residual pin above fixes."""
    s = _system(o, v, naux, seed=seed, scale=1.0)
    L = as_t(s.L)
    eps = as_t(s.eps)
    ref = ccsd.first_order_t2(eps, eri_anti(L), o)
    got = ccsd.first_order_t2_from_L(eps, L, o)
    assert float((got - ref).abs().max()) < 1e-13 * float(ref.abs().max())
    # antisymmetric in (i,j) and (a,b), and <ab||ij> / D entry by entry from the sum over P
    assert float((got + got.transpose(0, 1)).abs().max()) < 1e-14 * float(ref.abs().max())
    i, j, a, b = 0, o - 1, 1, v - 1
    num = sum(s.L[P, o + a, i] * s.L[P, o + b, j] - s.L[P, o + a, j] * s.L[P, o + b, i] for P in range(naux))
    den = s.eps[i] + s.eps[j] - s.eps[o + a] - s.eps[o + b]
    assert abs(got[i, j, a, b].item() - num / den) < 1e-12 * abs(num / den)


@pytest.mark.parametrize("t1_scale,a_chunk", [(0.0, 3), (0.2, 2)])
def test_blocked_sigma_matches_term_list(t1_scale, a_chunk):
    """oracle.sampled's vectorised whole-vector sigma (ladder formed chunk by chunk of a from L~,
    ragged last chunk) and its all-singles block equal jacobian.sigma_terms, which the stencil
    and the brute-force Jacobian pin."""
    from oracle import sampled
    o, v = 3, 7
    s = _system(o, v, 9, seed=3, scale=0.5, t1_scale=t1_scale)
    L = as_t(s.L)
    f = torch.diag(as_t(s.eps).to(C))
    _, a2 = random_amplitudes(o, v, seed=9, s1=0.2, s2=0.3)
    t1, t2 = as_t(s.t1), as_t(a2)
    x1, x2 = map(as_t, random_amplitudes(o, v, seed=11))
    q1, q2 = J.sigma_terms(J.Dressed(f, L, t1, t2), x1, x2)
    E = sampled.EntrySigma(as_t(s.eps), L, t1, t2)
    E.set_x(x1, x2)
    b1, b2 = E.sigma_blocked(a_chunk=a_chunk)
    sc = float(q2.abs().max())
    assert float((b1 - q1).abs().max()) < 1e-13 * sc
    assert float((b2 - q2).abs().max()) < 1e-13 * sc
    assert float((E.sigma1_all() - q1).abs().max()) < 1e-13 * sc


@pytest.mark.parametrize("o,v,naux,seed", [(2, 4, 6, 3), (3, 7, 12, 4)])
def test_residual_is_gauss_legendre_integral_of_jacobian(o, v, naux, seed):
    """Omega(T) = Omega(0) + int_0^1 A(sT) T ds, and two Gauss-Legendre nodes integrate it exactly.

    Omega(sT) is a quartic polynomial in s (Sec. 2.2: H-bar truncates at four T), so its
    s-derivative A(sT) T is cubic.  This ties the term-list Jacobian to the term-list residual at
    a finite T (the finite-difference pins only test it locally); a one-node (midpoint) rule must
    fail, so the check has teeth.
    """
    s = _system(o, v, naux, seed=seed, scale=0.5)
    L = as_t(s.L)
    g = eri_anti(L)
    f = torch.diag(as_t(s.eps).to(C))
    a1, a2 = random_amplitudes(o, v, seed=seed + 1, s1=0.3, s2=0.3)
    t1, t2 = as_t(a1), as_t(a2)
    r1, r2 = ccsd.residual(f, g, t1, t2)
    z1, z2 = ccsd.residual(f, g, torch.zeros_like(t1), torch.zeros_like(t2))
    h = 0.5 / np.sqrt(3.0)
    q = [J.sigma_terms(J.Dressed(f, L, sn * t1, sn * t2), t1, t2) for sn in (0.5 - h, 0.5 + h)]
    g1 = z1 + 0.5 * (q[0][0] + q[1][0])
    g2 = z2 + 0.5 * (q[0][1] + q[1][1])
    scale = float(r2.abs().max())
    assert float((g1 - r1).abs().max()) < 1e-12 * scale
    assert float((g2 - r2).abs().max()) < 1e-12 * scale
    m1, m2 = J.sigma_terms(J.Dressed(f, L, 0.5 * t1, 0.5 * t2), t1, t2)
    assert float((z2 + m2 - r2).abs().max()) > 1e-4 * scale


def test_ccsd_energy_two_electrons_equals_fci():
    """Two electrons: CCSD is exact, so the converged correlation energy is the FCI eigenvalue of
    the state the CC wave function represents, minus the reference energy (Sec. 2.2 energy)."""
    o, v = 2, 5
    s = _system(o, v, 8, seed=6, scale=0.4)
    P = oracle_problem(s, converge=True)
    bf = secondq.BruteForce(P.f.numpy(), P.g.numpy(), o)
    w, U = bf.fci()
    st, ov = secondq.cc_state_overlap(U, P.t1.numpy(), P.t2.numpy(), bf)
    assert ov > 1 - 1e-10
    e = complex(ccsd.energy(P.f, P.g, P.t1, P.t2))
    assert abs(e - (w[st] - bf.e_ref)) < 1e-11 * max(1.0, abs(e))
