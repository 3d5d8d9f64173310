"""GPU parity: libcclr (through the C ABI) against the CPU oracle, element by element.

Tolerances: FP64 path 1e-10 relative (unique-amplitude 2-norm); complex64 paths 2e-5
(FP32 CUDA cores) -- FP32 accumulation over K ~ v^2 terms of O(1) products gives
relative rounding ~ sqrt(K) * 6e-8.
"""
import numpy as np
import pytest
import torch

from oracle import ccsd, response as R, secondq
from oracle.integrals import as_t, eri_anti
from paper_2604_12914_gb300.inputs import make_system, make_config, random_amplitudes

from gpu_helpers import gpu_context, oracle_sigma, oracle_sigma_T, oracle_setup, rel_err, wdot

pytestmark = pytest.mark.gpu

CASES = [
    # (o, v, naux, seed, scale, t1_scale)
    (2, 4, 6, 1, 0.5, 0.2),
    (5, 13, 21, 2, 0.6, 0.1),
    (3, 67, 40, 3, 0.4, 0.05),     # v spans two 64-wide GEMM tiles with a ragged tail
    (10, 40, 200, 1, 1.0, 0.0),    # C1 sizes, T1 = 0, MP2 T2 (the config's own recipe)
]


def _amps(s, seed, t1_scale):
    a1, a2 = random_amplitudes(s.o, s.v, seed=seed, s1=0.2, s2=0.2)
    t1 = a1 * (t1_scale / 0.2) if t1_scale else np.zeros_like(a1)
    return t1, a2


@pytest.mark.parametrize("case", CASES)
def test_sigma_fp64_matches_oracle(case):
    o, v, naux, seed, scale, t1s = case
    s = make_system(o, v, naux, seed=seed, scale=scale)
    if (o, v) == (10, 40):
        f, g, L, _, _ = oracle_setup(s, np.zeros((o, v)), np.zeros((o, o, v, v)))
        t2 = ccsd.first_order_t2(as_t(s.eps), g, o).numpy()
        t1 = np.zeros((o, v), complex)
        ctx = gpu_context(s, t1=None, t2=None)     # library forms the first-order T2 itself
        gt1, gt2 = ctx.cc_lr_get_t()
        assert np.abs(gt2 - t2).max() < 1e-12 * np.abs(t2).max()
    else:
        t1, t2 = _amps(s, seed + 100, t1s)
        ctx = gpu_context(s, t1=t1, t2=t2)
    x1, x2 = random_amplitudes(o, v, seed=seed + 7, nvec=2)
    g1, g2 = ctx.cc_lr_sigma(x1, x2)
    for r in range(2):
        r1, r2 = oracle_sigma(s, t1, t2, x1[r], x2[r])
        assert rel_err(g1[r], g2[r], r1, r2) < 1e-10
        # antisymmetry of the doubles block
        assert np.abs(g2[r] + g2[r].transpose(1, 0, 2, 3)).max() < 1e-10 * np.abs(g2[r]).max()
    ctx.close()


@pytest.mark.parametrize("case", CASES[:3])
def test_sigma_T_fp64_matches_oracle_and_bilinear(case):
    o, v, naux, seed, scale, t1s = case
    s = make_system(o, v, naux, seed=seed, scale=scale)
    t1, t2 = _amps(s, seed + 100, t1s)
    ctx = gpu_context(s, t1=t1, t2=t2)
    y1, y2 = random_amplitudes(o, v, seed=seed + 9)
    z1, z2 = ctx.cc_lr_sigma_T(y1, y2)
    r1, r2 = oracle_sigma_T(s, t1, t2, y1, y2)
    assert rel_err(z1, z2, r1, r2) < 1e-10
    x1, x2 = random_amplitudes(o, v, seed=seed + 11)
    s1, s2 = ctx.cc_lr_sigma(x1, x2)
    lhs = wdot(y1, y2, s1, s2)
    rhs = wdot(z1, z2, x1, x2)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("3xtf32", 5e-5), ("bf16x3", 3e-4), ("tf32", 3e-3)])
def test_sigma_c64_matches_oracle(prec, tol):
    o, v, naux, seed, scale, t1s = CASES[2]
    s = make_system(o, v, naux, seed=seed, scale=scale)
    t1, t2 = _amps(s, seed + 100, t1s)
    ctx = gpu_context(s, t1=t1, t2=t2, prec=prec)
    x1, x2 = random_amplitudes(o, v, seed=3)
    g1, g2 = ctx.cc_lr_sigma(x1, x2)
    r1, r2 = oracle_sigma(s, t1, t2, x1, x2)
    assert rel_err(g1, g2, r1, r2) < tol
    z1, z2 = ctx.cc_lr_sigma_T(x1, x2)
    q1, q2 = oracle_sigma_T(s, t1, t2, x1, x2)
    assert rel_err(z1, z2, q1, q2) < tol
    ctx.close()


def test_xi_matches_oracle():
    s = make_system(4, 11, 17, seed=4, scale=0.5)
    t1, t2 = _amps(s, 40, 0.1)
    ctx = gpu_context(s, t1=t1, t2=t2)
    f, g, L, T1, T2 = oracle_setup(s, t1, t2)
    P = R.Problem(f, g, L, s.o, T1, T2)
    for comp in range(3):
        x1, x2 = ctx.cc_lr_xi(comp)
        r1, r2 = P.xi(as_t(s.mu[comp]))
        assert rel_err(x1, x2, r1.numpy(), r2.numpy()) < 1e-12
    ctx.close()


def _converged_small(o=3, v=8, naux=12, seed=5, scale=0.2):
    s = make_system(o, v, naux, seed=seed, scale=scale)
    f, g, L, _, _ = oracle_setup(s, np.zeros((o, v)), np.zeros((o, o, v, v)))
    t1, t2, _ = R.solve_ccsd(f, g, o, L=L)
    return s, R.Problem(f, g, L, o, t1, t2)


@pytest.mark.parametrize("method", ["gmres", "diis"])
def test_solve_x_and_lambda_match_oracle(method):
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy())
    ctx.cc_lr_set_solver(method)
    A = P.jacobian_matrix()
    for comp, omega in [(2, 0.0), (0, 0.0428), (1, -0.0428)]:
        x1, x2, st = ctx.cc_lr_solve_x(omega, comp, tol=1e-11)
        xi = P.pack(*P.xi(as_t(s.mu[comp])))
        ref = P.unpack(R.solve_x(A, xi, omega))
        assert rel_err(x1, x2, ref[0].numpy(), ref[1].numpy()) < 1e-9
        assert st["converged"] == 1
    l1, l2 = ctx.cc_lr_lambda(tol=1e-11)
    lam = torch.linalg.solve(A.transpose(0, 1), -P.eta0())
    r1, r2 = P.unpack(lam)
    assert rel_err(l1, l2, r1.numpy(), r2.numpy()) < 1e-9
    ctx.close()


@pytest.mark.parametrize("omega", [0.0, 0.0428])
def test_alpha_matches_oracle(omega):
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy())
    al, st = ctx.cc_lr_solve([omega], (0, 1, 2), tol=1e-11)
    ref = R.alpha(P, [as_t(m) for m in s.mu], omega).numpy()
    assert np.abs(al[0] - ref).max() < 1e-6 * np.abs(ref).max()
    assert np.abs(al[0] - al[0].conj().T).max() < 1e-8 * np.abs(ref).max()
    ctx.close()


def test_alpha_two_electrons_equals_sum_over_states():
    """o=2: GPU alpha against the exact FCI sum over states (Eq. sos)."""
    s = make_system(2, 4, 6, seed=2, scale=0.3)
    f, g, L, _, _ = oracle_setup(s, np.zeros((2, 4)), np.zeros((2, 2, 4, 4)))
    t1, t2, _ = R.solve_ccsd(f, g, 2, L=L)
    ctx = gpu_context(s, t1=t1.numpy(), t2=t2.numpy())
    bf = secondq.BruteForce(f.numpy(), g.numpy(), 2)
    w, U = bf.fci()
    st, _ = secondq.cc_state_overlap(U, t1.numpy(), t2.numpy(), bf)
    ops = [bf.one_body_op(m) for m in s.mu]
    for omega in (0.0, 0.0428):
        al, _ = ctx.cc_lr_solve([omega], (0, 1, 2), tol=1e-12)
        sos = np.array([[-secondq.sos_response(w, U, ops[a], ops[b], omega, st) for b in range(3)]
                        for a in range(3)])
        assert np.abs(al[0] - sos).max() < 1e-7 * np.abs(sos).max()
    ctx.close()


@pytest.mark.parametrize("M,N,K", [(128, 120, 64), (300, 257, 1200), (37, 5, 9000), (1000, 700, 31)])
@pytest.mark.parametrize("mode", [1, 2, 3])
def test_tensor_core_gemm_selftest(M, N, K, mode):
    """tcgen05 complex GEMM (TF32 / 3xTF32 on kind::tf32, bf16x3 on kind::f16) against FP64 on
    random data, ragged shapes."""
    from paper_2604_12914_gb300 import binding
    e_tc, e_fp32 = binding.cc_lr_selftest_gemm(M, N, K, mode)
    print(f"selftest M={M} N={N} K={K} mode={mode}: tensor-core {e_tc:.3e}  fp32 {e_fp32:.3e}")
    assert e_tc >= 0, "tensor-core path not taken"
    # relative to max |C|: TF32 keeps 10 mantissa bits per operand (2^-11 rounding);
    # 3xTF32 recovers about 2^-21 per product, but the tensor-core accumulation error was
    # measured to grow linearly with K (4e-7, 5e-6, 5e-5 at K = 64, 1200, 9000), while the
    # FP32 CUDA-core sum grows ~ sqrt(K)
    # bf16x3: hi + lo BF16 parts keep 16 significant bits, the neglected lo.lo and remainder
    # terms are about 3 x 2^-16 of each product
    tol = {1: 4e-3, 2: 1e-8 * K + 2e-6, 3: 2e-4 + 1e-8 * K}[mode]
    assert e_tc < tol, (e_tc, e_fp32)
    assert e_fp32 < 2e-5


@pytest.mark.parametrize("prec", ["tf32", "3xtf32"])
def test_alpha_mixed_precision_within_1e4(prec):
    """Mixed-precision alpha (tensor-core sigma, FP64 residual/refinement/subspace/alpha)
    against the FP64 oracle: |delta alpha| < 1e-4 a.u. for every entry."""
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy(), prec=prec)
    for omega in (0.0, 0.0428):
        al, st = ctx.cc_lr_solve([omega], (0, 1, 2), tol=1e-8)
        ref = R.alpha(P, [as_t(m) for m in s.mu], omega).numpy()
        assert np.abs(al[0] - ref).max() < 1e-4, (prec, omega, np.abs(al[0] - ref).max())
        assert st["refinements"] > 0
    ctx.close()


def test_alpha_tensor_core_refinement_within_1e4():
    """TF32 corrections refined with 3xTF32 residuals (no FP64 sigma anywhere: residuals,
    polish and the F X stencil on the tensor cores; norms, updates, subspace and alpha in FP64)
    against the FP64 oracle: |delta alpha| < 1e-4 a.u. for every entry."""
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy(), prec="tf32")
    ctx.cc_lr_set_refinement("3xtf32")
    for omega in (0.0, 0.0428):
        al, st = ctx.cc_lr_solve([omega], (0, 1, 2), tol=1e-6)
        ref = R.alpha(P, [as_t(m) for m in s.mu], omega).numpy()
        err = np.abs(al[0] - ref).max()
        print(f"omega={omega}: |delta alpha| = {err:.2e}, max|alpha| = {np.abs(ref).max():.3f}, {st}")
        assert err < 1e-4, (omega, err)
        assert st["refinements"] > 0
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("tf32", 3e-3), ("3xtf32", 5e-5)])
def test_batched_sigma_matches_single(prec, tol):
    """Several right-hand sides share each formed <ab||ef>~ block; results equal the oracle."""
    o, v, naux, seed, scale, t1s = CASES[3]
    s = make_system(o, v, naux, seed=seed, scale=scale)
    f, g, L, _, _ = oracle_setup(s, np.zeros((o, v)), np.zeros((o, o, v, v)))
    t2 = ccsd.first_order_t2(as_t(s.eps), g, o).numpy()
    t1 = np.zeros((o, v), complex)
    ctx = gpu_context(s, prec=prec)
    x1, x2 = random_amplitudes(o, v, seed=21, nvec=3)
    b1, b2 = ctx.cc_lr_sigma(x1, x2)
    z1, z2 = ctx.cc_lr_sigma_T(x1, x2)
    for r in range(3):
        r1, r2 = oracle_sigma(s, t1, t2, x1[r], x2[r])
        assert rel_err(b1[r], b2[r], r1, r2) < tol
        q1, q2 = oracle_sigma_T(s, t1, t2, x1[r], x2[r])
        assert rel_err(z1[r], z2[r], q1, q2) < tol
        u1, u2 = ctx.cc_lr_sigma(x1[r], x2[r])
        assert rel_err(u1, u2, b1[r], b2[r]) < tol
    ctx.close()


def test_autograd_sigma_function():
    """SigmaFn backward = J^H grad (holomorphic convention) on the antisymmetric subspace."""
    from paper_2604_12914_gb300.autograd import sigma as sigma_fn
    s = make_system(3, 6, 9, seed=31, scale=0.5, t1_scale=0.1)
    t1, t2 = _amps(s, 32, 0.1)
    ctx = gpu_context(s, t1=t1, t2=t2)
    dev = torch.device("cuda")

    def antisym(z):
        y = z - z.transpose(0, 1)
        return 0.5 * (y - y.transpose(2, 3))

    a1, a2 = random_amplitudes(3, 6, seed=33)
    z1 = torch.tensor(a1, device=dev, requires_grad=True)
    z2 = torch.tensor(a2, device=dev, requires_grad=True)

    def f(p1, p2):
        return sigma_fn(ctx, p1, antisym(p2))

    assert torch.autograd.gradcheck(f, (z1, z2), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)
    # a real scalar of the output: gradient equals the explicit transpose product
    w1, w2 = random_amplitudes(3, 6, seed=34)
    W1 = torch.tensor(w1, device=dev)
    W2 = torch.tensor(w2, device=dev)
    s1, s2 = f(z1, z2)
    loss = (W1 * s1).sum().real + 0.25 * (W2 * s2).sum().real
    loss.backward()
    ref1, ref2 = oracle_sigma_T(s, t1, t2, w1, w2)
    # PyTorch reports 2 dL/dz* = conj(dL/dz) for a real L: here conj((W A)_singles)
    assert np.abs(z1.grad.cpu().numpy() - np.conj(ref1)).max() < 1e-9 * np.abs(ref1).max()
    ctx.close()


def test_bounded_wait_gives_up_and_context_survives():
    """A device wait that nothing completes ends after its limit with CCLR_ETIMEOUT; the
    CUDA context stays usable (a sigma afterwards still matches the oracle)."""
    from paper_2604_12914_gb300 import binding
    st, flag = binding.cc_lr_selftest_timeout(2000)
    assert flag == 1 and st == binding.CCLR_ETIMEOUT
    assert "gave up" in binding.load().cc_lr_last_error().decode()
    o, v, naux, seed, scale, t1s = CASES[1]
    s = make_system(o, v, naux, seed=seed, scale=scale)
    t1, t2 = _amps(s, seed + 100, t1s)
    ctx = gpu_context(s, t1=t1, t2=t2, prec="tf32")
    x1, x2 = random_amplitudes(o, v, seed=3)
    g1, g2 = ctx.cc_lr_sigma(x1, x2)
    r1, r2 = oracle_sigma(s, t1, t2, x1, x2)
    assert rel_err(g1, g2, r1, r2) < 3e-3
    ctx.close()


def _graph_context(s, prec, **kw):
    from paper_2604_12914_gb300 import binding
    stream = torch.cuda.Stream()
    ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec=prec, stream=stream.cuda_stream, **kw)
    return ctx, stream


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("tf32", 1e-5)])
def test_graph_replay_matches_eager_sigma(prec, tol):
    """CUDA-graph replay of the sigma and sigma^T programs gives the eager results (the second
    identical product is captured, later ones replay it)."""
    o, v, naux, seed, scale, t1s = CASES[2]
    s = make_system(o, v, naux, seed=seed, scale=scale)
    t1, t2 = _amps(s, seed + 100, t1s)
    ctx, stream = _graph_context(s, prec, t1=t1, t2=t2)
    x1, x2 = random_amplitudes(o, v, seed=3)
    e1, e2 = ctx.cc_lr_sigma(x1, x2)
    f1, f2 = ctx.cc_lr_sigma_T(x1, x2)
    ctx.cc_lr_set_graphs(True)
    for _ in range(4):
        g1, g2 = ctx.cc_lr_sigma(x1, x2)
        assert rel_err(g1, g2, e1, e2) < tol
        h1, h2 = ctx.cc_lr_sigma_T(x1, x2)
        assert rel_err(h1, h2, f1, f2) < tol
    caps, launches = ctx.cc_lr_graph_stats()
    assert caps == 2 and launches >= 4, (caps, launches)
    # a different input through the same buffers replays the same graph
    y1, y2 = random_amplitudes(o, v, seed=4)
    g1, g2 = ctx.cc_lr_sigma(y1, y2)
    ctx.cc_lr_set_graphs(False)
    r1, r2 = ctx.cc_lr_sigma(y1, y2)
    assert rel_err(g1, g2, r1, r2) < tol
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_graph_replay_solve_alpha(prec):
    """alpha with every solver product replayed from CUDA graphs matches the oracle."""
    s, P = _converged_small()
    ctx, stream = _graph_context(s, prec, t1=P.t1.numpy(), t2=P.t2.numpy())
    ctx.cc_lr_set_graphs(True)
    al, st = ctx.cc_lr_solve([0.0428], (0, 1, 2), tol=1e-8)
    ref = R.alpha(P, [as_t(m) for m in s.mu], 0.0428).numpy()
    err = np.abs(al[0] - ref).max()
    caps, launches = ctx.cc_lr_graph_stats()
    print(f"{prec}: |delta alpha| {err:.2e}, graph captures {caps}, launches {launches}, {st}")
    assert err < (1e-6 * np.abs(ref).max() if prec == "fp64" else 1e-4)
    assert launches > caps > 0
    ctx.close()


@pytest.mark.parametrize("prec,refine", [("fp64", "fp64"), ("tf32", "fp64"), ("tf32", "3xtf32")])
def test_block_solver_alpha_matches_oracle(prec, refine):
    """Block GMRES (all components and both frequency signs advanced together, one batched
    operator product per iteration) gives the oracle's alpha."""
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy(), prec=prec)
    ctx.cc_lr_set_solver("block")
    if prec != "fp64":
        ctx.cc_lr_set_refinement(refine)
    tol = 1e-10 if prec == "fp64" else (1e-8 if refine == "fp64" else 1e-6)
    al, st = ctx.cc_lr_solve([0.0428], (0, 1, 2), tol=tol)
    ref = R.alpha(P, [as_t(m) for m in s.mu], 0.0428).numpy()
    err = np.abs(al[0] - ref).max()
    print(f"{prec}/{refine}: |delta alpha| {err:.2e}, {st}")
    assert err < (1e-6 * np.abs(ref).max() if prec == "fp64" else 1e-4)
    assert st["converged"] == 1
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("tf32", 1e-5), ("3xtf32", 1e-6)])
def test_stored_ladder_ablation_matches_on_the_fly(prec, tol):
    """The stored packed <ab||ef>~ (ablation) gives the on-the-fly sigma: first product forms and
    keeps it, later ones reuse it; the transpose product is unchanged."""
    o, v, naux, seed, scale, t1s = CASES[2]
    s = make_system(o, v, naux, seed=seed, scale=scale)
    t1, t2 = _amps(s, seed + 100, t1s)
    ctx = gpu_context(s, t1=t1, t2=t2, prec=prec)
    x1, x2 = random_amplitudes(o, v, seed=3, nvec=2)
    e1, e2 = ctx.cc_lr_sigma(x1, x2)
    f1, f2 = ctx.cc_lr_sigma_T(x1[0], x2[0])
    ctx.cc_lr_set_ladder_storage(True)
    for _ in range(2):
        g1, g2 = ctx.cc_lr_sigma(x1, x2)
        for r in range(2):
            assert rel_err(g1[r], g2[r], e1[r], e2[r]) < tol
    h1, h2 = ctx.cc_lr_sigma_T(x1[0], x2[0])
    assert rel_err(h1, h2, f1, f2) < tol
    r1, r2 = oracle_sigma(s, t1, t2, x1[0], x2[0])
    assert rel_err(g1[0], g2[0], r1, r2) < (3e-3 if prec == "tf32" else 5e-5)
    ctx.close()


@pytest.mark.parametrize("method,prec", [("gmres", "fp64"), ("block", "fp64"), ("block", "tf32")])
def test_damped_alpha_matches_oracle(method, prec):
    """Damped response at z = omega + i gamma (complex shift in the solver and preconditioner)
    against the oracle's damped alpha; mixed precision with tensor-core refinement."""
    s, P = _converged_small()
    ctx = gpu_context(s, t1=P.t1.numpy(), t2=P.t2.numpy(), prec=prec)
    ctx.cc_lr_set_solver(method)
    if prec != "fp64":
        ctx.cc_lr_set_refinement("3xtf32")
    mu = [as_t(m) for m in s.mu]
    for omega, gamma in [(0.0428, 0.01), (0.0, 0.05)]:
        al, st = ctx.cc_lr_solve([omega], (0, 1, 2), tol=1e-10 if prec == "fp64" else 1e-6, gamma=gamma)
        ref = R.alpha(P, mu, omega, gamma=gamma).numpy()
        err = np.abs(al[0] - ref).max()
        print(f"{method}/{prec} z={omega}+{gamma}i: |delta alpha| {err:.2e}, {st}")
        assert err < (1e-6 * np.abs(ref).max() if prec == "fp64" else 1e-4)
    ctx.close()


def test_damped_alpha_two_electrons_equals_sum_over_states():
    """o=2: the GPU damped alpha equals the exact sum over states at complex frequency."""
    s = make_system(2, 4, 6, seed=2, scale=0.3)
    f, g, L, _, _ = oracle_setup(s, np.zeros((2, 4)), np.zeros((2, 2, 4, 4)))
    t1, t2, _ = R.solve_ccsd(f, g, 2, L=L)
    ctx = gpu_context(s, t1=t1.numpy(), t2=t2.numpy())
    bf = secondq.BruteForce(f.numpy(), g.numpy(), 2)
    w, U = bf.fci()
    st, _ = secondq.cc_state_overlap(U, t1.numpy(), t2.numpy(), bf)
    ops = [bf.one_body_op(m) for m in s.mu]
    for omega, gamma in [(0.0428, 0.01), (0.7, 0.02)]:
        al, _ = ctx.cc_lr_solve([omega], (0, 1, 2), tol=1e-12, gamma=gamma)
        z = complex(omega, gamma)
        sos = np.array([[-secondq.sos_response(w, U, ops[a], ops[b], z, st) for b in range(3)]
                        for a in range(3)])
        assert np.abs(al[0] - sos).max() < 1e-7 * np.abs(sos).max()
    ctx.close()


def test_gemm_autotuner_caches_shapes_and_keeps_results():
    """The tile autotuner: the first tensor-core sigma tunes every GEMM shape it meets (rows in
    cc_lr_gemm_tuning with the candidates timed, the best no slower than the rules' choice), and
    the tuned launches give the same sigma as the rules' configuration (autotune off).  The table is
    per process, so the sizes here (o=9, v=44) are ones no other test tunes."""
    s = make_system(9, 44, 180, seed=3)
    x1, x2 = random_amplitudes(s.o, s.v, seed=3)
    from paper_2604_12914_gb300 import binding
    ref = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec="3xtf32")
    ref.cc_lr_set_autotune(False)
    n_before = len(ref.cc_lr_gemm_tuning())
    r1, r2 = ref.cc_lr_sigma(x1, x2)
    ref.close()
    ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec="3xtf32")
    g1, g2 = ctx.cc_lr_sigma(x1, x2)
    tab = ctx.cc_lr_gemm_tuning()
    assert len(tab) > n_before
    for row in tab:
        if row["tried"] > 0:
            assert row["ms_best"] <= row["ms_rule"] * 1.0001
    h1, h2 = ctx.cc_lr_sigma(x1, x2)         # tuned shapes: cached configuration
    assert rel_err(g1, g2, r1, r2) < 1e-6
    assert rel_err(h1, h2, r1, r2) < 1e-6
    print(f"{len(tab)} tuned shapes; e.g. {tab[:3]}")
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("tf32", 1e-6)])
def test_packed_sigma_entry_point_matches_full_layout(prec, tol):
    """cc_lr_sigma_packed (unique amplitudes i<j, a<b, device arrays) equals cc_lr_sigma in the full
    layout, for a batch of right-hand sides and for the transpose."""
    o, v, naux, seed, scale, t1s = CASES[2]
    s = make_system(o, v, naux, seed=seed, scale=scale)
    t1, t2 = _amps(s, seed + 100, t1s)
    ctx = gpu_context(s, t1=t1, t2=t2, prec=prec)
    x1, x2 = random_amplitudes(o, v, seed=5, nvec=3)
    oi, oj = np.triu_indices(o, 1)
    vi, vj = np.triu_indices(v, 1)

    def pack(a1, a2):
        return np.concatenate([a1.reshape(-1), a2[oi, oj][:, vi, vj].reshape(-1)])

    xp = torch.tensor(np.stack([pack(x1[r], x2[r]) for r in range(3)]), device="cuda")
    for transpose in (False, True):
        g1, g2 = ctx.cc_lr_sigma(x1, x2, transpose=transpose)
        sp = torch.empty_like(xp)
        ctx.sigma_packed(xp, sp, nrhs=3, transpose=transpose)
        got = sp.cpu().numpy()
        for r in range(3):
            ref = pack(g1[r], g2[r])
            assert np.abs(got[r] - ref).max() < tol * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("omega,omega_im", [(0.0, 0.0), (0.0428, 0.0), (0.7, 0.02)])
def test_preconditioner_reciprocal_within_fp64_rounding(omega, omega_im):
    """The preconditioner's Newton-Raphson FP64 reciprocal against host IEEE division."""
    from paper_2604_12914_gb300 import binding
    err = binding.cc_lr_selftest_precond(1 << 20, omega, omega_im, seed=5)
    assert err < 1e-15, err
