// C ABI of libcclr (declared in include/cclr.h): context life cycle, sigma / sigma^T, the
// preconditioned DIIS linear solver in FP64, the ground-state Lambda, and alpha(omega).
#include <array>
#include <chrono>
#include <cmath>
#include <limits>
#include <complex>
#include <cstring>
#include <memory>

#include "../../include/cclr.h"
#include "../../include/cclr_testing.h"

#include <cstdio>
#include <cstdlib>
#include <random>
#include "model.cuh"
#include "tc_gemm.cuh"

using namespace cclr;
using zd = std::complex<double>;

namespace {
thread_local std::string g_last_error = "";

int fail(int status, const std::string &msg) {
  g_last_error = msg;
  return status;
}

// Amplitude vector, complex128, contiguous: singles [o][v] then the doubles block -- packed
// unique amplitudes [(i<j)][(a<b)] for the solver's vectors, the full [o][o][v][v] tensor for
// boundary staging.
struct AVec {
  DevBuf b;
  void *p1() const { return b.p; }
  void *p2(int64_t n1) const { return (char *)b.p + n1 * 16; }
};
}  // namespace

struct cclr_ctx {
  MemAcct acct;                   // device memory of this context (first member: released last)
  std::unique_ptr<Model> M;
  int o = 0, v = 0, naux = 0;
  int64_t n1 = 0, n2 = 0, n2p = 0;  // singles, full doubles o^2 v^2, packed doubles P_o P_v
  int device_ptrs = 0;
  cudaStream_t st = nullptr;
  bool have_lambda = false;
  AVec lam;                       // ground-state Lambda (packed)
  AVec fullA, fullB;              // full-layout complex128 scratch (xi, shifted amplitudes, unpacking)
  std::vector<AVec> stage_in, stage_out;  // host <-> device staging (full complex128), per RHS
  CstSet shift;                   // intermediates at shifted amplitudes (F X stencils)
  CstSet onebody[3];              // H-bar of each dipole component alone (eta^A = lambda A[mu^A])
  AVec eta_v[3];                  // eta^A vectors (packed), formed once lambda is known
  bool eta_ok[3] = {false, false, false};
  CstSet shift64;                 // their complex64 rounding (tensor-core F X stencils)
  // arithmetic of the mixed modes' accurate sigma products: the refinement residuals, the
  // final polish and the F X stencils (CCLR_FP64, or CCLR_C64_3XTF32 on the tensor cores)
  int hi_prec = CCLR_FP64;
  int sigma_calls = 0;

  // length of a solver vector (packed) and of a full-layout vector
  int64_t ntot() const { return n1 + n2p; }
  int64_t nfull() const { return n1 + n2; }
  // CCLR_VERBOSE=1 prints solver residual histories to stderr (diagnostics)
  static bool verbose() {
    static const bool v = std::getenv("CCLR_VERBOSE") && std::getenv("CCLR_VERBOSE")[0] == '1';
    return v;
  }

  void alloc_vec(AVec &v_) { if (!v_.b.p) v_.b.alloc((size_t)ntot() * 16); }
  void alloc_full(AVec &v_) { if (!v_.b.p) v_.b.alloc((size_t)nfull() * 16); }

  // bilinear (herm = 0) or Hermitian (herm = 1) product over unique amplitudes, FP64 accumulation
  zd dot(const void *a, const void *b, int herm) {
    double2 *part = M->E.dot_scratch();
    double2 *res = M->E.dot_results();
    vec_dot(C128, ntot(), a, b, herm, part, res, 0, st);
    double2 h;
    CCLR_CUDA(cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
    CCLR_CUDA(cudaStreamSynchronize(st));
    return zd(h.x, h.y);
  }
  // (a NaN or infinite vector gives a NaN or infinite norm: the solvers test for it)
  double norm(const void *a) {
    const double d = dot(a, a, 1).real();
    return std::isfinite(d) ? std::sqrt(std::max(0.0, d)) : std::numeric_limits<double>::quiet_NaN();
  }
  void axpy(zd a, const void *x, void *y) { vec_axpy(C128, ntot(), zc(a.real(), a.imag()), x, y, st); }
  void copy(const void *x, void *y) { CCLR_CUDA(cudaMemcpyAsync(y, x, (size_t)ntot() * 16, cudaMemcpyDeviceToDevice, st)); }
  void scal(zd a, void *y) { vec_scal(C128, ntot(), zc(a.real(), a.imag()), y, st); }
  void precond(zd omega, const void *r, void *out) {
    vec_precond(C128, n1, M->D1.as<double>(), omega.real(), omega.imag(), r, out, st);
    vec_precond(C128, n2p, M->D2.as<double>(), omega.real(), omega.imag(), (const char *)r + n1 * 16,
                (char *)out + n1 * 16, st);
  }
  // packed <-> full layouts (complex128 packed; the full side in dtype dt)
  void unpack_to(const void *packed, void *full, int dt) {
    M->E.permute(zc(1), make_tens((void *)packed, C128, {n1}), "a", make_tens(full, dt, {n1}), "a", false);
    unpack_doubles(C128, dt, o, v, (const char *)packed + n1 * 16, (char *)full + n1 * dt_size(dt), zc(1), false, st);
  }
  void pack_from(const void *full, int dt, void *packed) {
    M->E.permute(zc(1), make_tens((void *)full, dt, {n1}), "a", make_tens(packed, C128, {n1}), "a", false);
    pack_doubles(dt, C128, o, v, (const char *)full + n1 * dt_size(dt), (char *)packed + n1 * 16, st);
  }

  // s = A x (dir +1) or x A (dir -1) in the current precision; x, s packed complex128 vectors
  void op(int dir, const void *x, void *s, const CstSet *set = nullptr) { op_batch(dir, 1, &x, &s, set); }

  // the same for nr packed vectors at once (the ladder's integral blocks are formed once for
  // all): each is unpacked into a fixed full-layout buffer in the set's precision, the sigma
  // program runs on those, and the results are packed back.  The buffers stay at fixed
  // addresses, so repeated products can replay one captured CUDA graph.
  std::vector<DevBuf> xfs[2], sfs[2];  // full-layout operands of the sigma program, per dtype and RHS
  void stage_full(int dt, int nr) {
    auto &xf = xfs[dt], &sf = sfs[dt];
    if ((int)xf.size() < nr) { xf.resize(nr); sf.resize(nr); }
    for (int r = 0; r < nr; ++r)
      if (!xf[r].p) { xf[r].alloc((size_t)nfull() * dt_size(dt)); sf[r].alloc((size_t)nfull() * dt_size(dt)); }
  }
  // right-hand sides per batched product: the per-RHS full-layout staging (and, in the
  // transpose, x2-bar) and the ladder's packed operands must fit in a third of what is free
  int batch_cap(int dir, int dt, int nr) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      (void)cudaGetLastError();
      return nr;
    }
    if (acct.budget) free_b = std::min(free_b, acct.budget > acct.used ? acct.budget - acct.used : (size_t)0);
    const double per = (double)nfull() * dt_size(dt) * (dir < 0 ? 3 : 2) + (double)n2p * 8 * 4;
    const int fit = (int)(free_b / 3.0 / per);
    return std::max(1, std::min(nr, fit));
  }
  int last_products = 1;  // batched products the last op_batch was split into
  void op_batch(int dir, int nr, const void *const *xs, void *const *ss, const CstSet *set = nullptr) {
    if (set == nullptr) set = &M->cst_for(M->prec);
    const int cap = batch_cap(dir, set->dt, nr);
    last_products = (nr + cap - 1) / cap;
    if (cap < nr) {  // several batched products, each sharing its formed blocks
      for (int r0 = 0; r0 < nr; r0 += cap) op_batch_chunk(dir, std::min(cap, nr - r0), xs + r0, ss + r0, set);
      return;
    }
    op_batch_chunk(dir, nr, xs, ss, set);
  }
  // the most device memory one product held beyond what stayed allocated after it (workspace,
  // staging, ladder blocks released in a budgeted context): solvers keep this much free
  size_t op_transient = 0;
  void op_batch_chunk(int dir, int nr, const void *const *xs, void *const *ss, const CstSet *set) {
    struct PeakScope {  // the account's peak over this product alone, then restored
      MemAcct &a;
      size_t saved, &out;
      PeakScope(MemAcct &a_, size_t &out_) : a(a_), saved(a_.peak), out(out_) { a.peak = a.used; }
      ~PeakScope() {
        out = std::max(out, a.peak > a.used ? a.peak - a.used : (size_t)0);
        a.peak = std::max(saved, a.peak);
      }
    } peak_scope(acct, op_transient);
    sigma_calls += nr;
    const int dt = set->dt;
    const size_t es = dt_size(dt);
    stage_full(dt, nr);
    auto &xf = xfs[dt], &sf = sfs[dt];
    std::vector<const void *> a1(nr), a2(nr);
    std::vector<void *> b1(nr), b2(nr);
    for (int r = 0; r < nr; ++r) {
      unpack_to(xs[r], xf[r].p, dt);
      a1[r] = xf[r].p;
      a2[r] = (const char *)xf[r].p + n1 * es;
      b1[r] = sf[r].p;
      b2[r] = (char *)sf[r].p + n1 * es;
    }
    M->apply_batch(dir, *set, nr, a1.data(), a2.data(), b1.data(), b2.data());
    for (int r = 0; r < nr; ++r) pack_from(sf[r].p, dt, ss[r]);
  }
  // sigma of full-layout complex128 vectors (the boundary's layout), nr at once
  void op_batch_full(int dir, int nr, const void *const *xs, void *const *ss) {
    sigma_calls += nr;
    const CstSet *set = &M->cst_for(M->prec);
    const int dt = set->dt;
    const size_t es = dt_size(dt);
    // complex64 products and graph replay go through the fixed full-layout buffers
    const bool stage = dt == C64 || M->graphs;
    if (stage) stage_full(dt, nr);
    auto &xf = xfs[dt], &sf = sfs[dt];
    std::vector<const void *> a1(nr), a2(nr);
    std::vector<void *> b1(nr), b2(nr);
    for (int r = 0; r < nr; ++r) {
      const void *x = xs[r];
      void *s = ss[r];
      if (stage) {
        M->E.permute(zc(1), make_tens((void *)x, C128, {nfull()}), "a", make_tens(xf[r].p, dt, {nfull()}), "a", false);
        x = xf[r].p;
        s = sf[r].p;
      }
      a1[r] = x;
      a2[r] = (const char *)x + n1 * es;
      b1[r] = s;
      b2[r] = (char *)s + n1 * es;
    }
    M->apply_batch(dir, *set, nr, a1.data(), a2.data(), b1.data(), b2.data());
    if (stage)
      for (int r = 0; r < nr; ++r)
        M->E.permute(zc(1), make_tens(sf[r].p, dt, {nfull()}), "a", make_tens(ss[r], C128, {nfull()}), "a", false);
  }

  // Solve (Op - omega) x = b.  FP64 mode: preconditioned DIIS.  Mixed modes: iterative
  // refinement -- the residual r = b - (Op - omega) x is formed with the FP64 sigma and
  // normed and applied in FP64; each correction (Op - omega) d = r is solved by DIIS with
  // the tensor-core sigma (TF32: two digits per correction, 3xTF32: five).
  int refinements = 0;
  // warm: x holds a start vector (its residual is formed first) instead of zero
  double solve(int dir, zd omega, const void *b, void *x, double tol, int depth, int maxit,
               int *its, bool warm = false) {
    if (M->prec == CCLR_FP64) return solve_diis(dir, omega, b, x, tol, depth, maxit, its, warm);
    const int lo = M->prec;
    const double inner_tol = lo == CCLR_C64_TF32 ? 1e-2 : 1e-5;
    // each correction gets a bounded number of DIIS steps: near its precision floor the
    // low-precision DIIS stalls, and one more FP64 residual is cheaper than stalling
    const int inner_cap = lo == CCLR_C64_TF32 ? 30 : 40;
    AVec s, r, d, xb;
    alloc_vec(s);
    alloc_vec(r);
    alloc_vec(d);
    alloc_vec(xb);
    const double bn = std::max(norm(b), 1e-300);
    if (!warm) CCLR_CUDA(cudaMemsetAsync(x, 0, (size_t)ntot() * 16, st));
    copy(b, r.b.p);
    double rel = 1.0, rel_prev = 1e300;
    int used = 0;
    bool stalled = false;
    for (int outer = 0; outer < 40 && used < maxit; ++outer) {
      if (outer > 0 || warm) {
        M->prec = hi_prec;
        op(dir, x, s.b.p);
        M->prec = lo;
        ++refinements;
        copy(b, r.b.p);
        axpy(zd(-1), s.b.p, r.b.p);
        axpy(zd(omega), x, r.b.p);
      }
      rel = norm(r.b.p) / bn;
      if (verbose()) std::fprintf(stderr, "cclr refine dir=%d omega=%g outer=%d rel=%.3e\n", dir, omega.real(), outer, rel);
      if (!(rel == rel)) throw Error(3, "solver produced NaN residual");
      if (rel > 0.5 * rel_prev) {
        // the last correction did not help: go back to the best iterate and stop refining
        if (rel > rel_prev) {
          copy(xb.b.p, x);
          rel = rel_prev;
        }
        stalled = true;
        break;
      }
      if (rel < tol) break;
      copy(x, xb.b.p);
      rel_prev = rel;
      int inner = 0;
      solve_diis(dir, omega, r.b.p, d.b.p, std::max(inner_tol, 0.3 * tol / rel), depth,
                 std::min(inner_cap, maxit - used), &inner);
      used += inner;
      if (its) *its += inner;
      axpy(zd(1), d.b.p, x);
    }
    if ((stalled || rel >= tol) && used < maxit) {
      // finish in the accurate arithmetic, warm-started from the refined solution
      M->prec = hi_prec;
      int rest = 0;
      rel = solve_diis(dir, omega, b, x, tol, depth, maxit - used, &rest, true);
      M->prec = lo;
      if (its) *its += rest;
      if (verbose()) std::fprintf(stderr, "cclr finish prec=%d dir=%d iterations=%d rel=%.3e\n", hi_prec, dir, rest, rel);
    }
    return rel;
  }

  // Krylov method of the linear solves: 1 = restarted GMRES (default), 0 = DIIS.
  int method = 1;  // 1 GMRES, 0 DIIS, 2 block GMRES over the right-hand sides of cc_lr_solve
  int krylov = 30;
  int maxit = 300;  // iterations per linear solve, all precisions together

  double solve_diis(int dir, zd omega, const void *b, void *x, double tol, int depth, int maxit,
                    int *its, bool warm = false) {
    if (method >= 1) return solve_gmres(dir, omega, b, x, tol, krylov, maxit, its, warm);
    return solve_pulay(dir, omega, b, x, tol, depth, maxit, its, warm);
  }

  // Right-preconditioned restarted GMRES(m) on (Op - omega) x = b in the current precision:
  // preconditioner P = (D - omega)^-1 (diagonal of A), modified Gram-Schmidt in the
  // weighted Hermitian inner product (singles 1, doubles 1/4), Givens rotations and the
  // small least-squares problem on the host in FP64.
  std::vector<AVec> kv;  // Krylov basis (kept between calls unless the context is budgeted)
  double solve_gmres(int dir, zd omega, const void *b, void *x, double tol, int m, int maxit,
                     int *its, bool warm) {
    // Mixed modes: the Krylov basis of these correction solves is stored in complex64 (half the
    // bytes; the correction is refined by an accurate residual, and rounding the orthonormal basis
    // to FP32 costs far less accuracy than the products in the correction's own arithmetic). The
    // Arnoldi dots, updates and the Hessenberg algebra stay in FP64.
    const bool v64 = M->prec != CCLR_FP64;
    const size_t vbytes = (size_t)ntot() * (v64 ? 8 : 16);
    m = std::max(2, std::min(m, 100));
    if (acct.budget) m = std::min(m, block_restart(1, 0.2, v64 ? 8 : 16));
    struct Release {
      cclr_ctx *c;
      ~Release() {
        if (c->M->lean) c->kv.clear();
      }
    } rel_guard{this};
    if ((int)kv.size() < m + 1) kv.resize(m + 1);
    for (int k = 0; k <= m; ++k)
      if (kv[k].b.bytes != vbytes) kv[k].b.alloc(vbytes);
    AVec z, w, vt;
    alloc_vec(z);
    alloc_vec(w);
    if (v64) alloc_vec(vt);
    const Tens k128 = make_tens(nullptr, C128, {ntot()});
    // basis vector i as complex128 (converted into vt in the mixed modes)
    auto basis = [&](int i) -> const void * {
      if (!v64) return kv[i].b.p;
      Tens src = make_tens(kv[i].b.p, C64, {ntot()}), dst = k128;
      dst.p = vt.b.p;
      M->E.permute(zc(1), src, "a", dst, "a", false);
      return vt.b.p;
    };
    // kv[i] = scale * v (v complex128)
    auto store = [&](const void *v, int i, double scale) {
      if (!v64) {
        copy(v, kv[i].b.p);
        scal(zd(scale), kv[i].b.p);
        return;
      }
      Tens src = k128, dst = make_tens(kv[i].b.p, C64, {ntot()});
      src.p = (void *)v;
      M->E.permute(zc(scale), src, "a", dst, "a", false);
    };
    const double bn = std::max(norm(b), 1e-300);
    if (!warm) CCLR_CUDA(cudaMemsetAsync(x, 0, (size_t)ntot() * 16, st));
    double rel = 1.0;
    int used = 0;
    std::vector<zd> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
    while (used < maxit) {
      // r = b - (Op - omega) x, in w
      copy(b, w.b.p);
      if (warm || used > 0) {
        op(dir, x, z.b.p);
        axpy(zd(-1), z.b.p, w.b.p);
        axpy(zd(omega), x, w.b.p);
      }
      warm = true;
      double beta = norm(w.b.p);
      rel = beta / bn;
      if (verbose()) std::fprintf(stderr, "cclr gmres dir=%d omega=%g it=%d rel=%.3e prec=%d\n", dir, omega.real(), used, rel, M->prec);
      if (!(rel == rel)) throw Error(3, "solver produced NaN residual");
      if (rel < tol || beta == 0.0) break;
      store(w.b.p, 0, 1.0 / beta);
      std::fill(g.begin(), g.end(), zd(0));
      g[0] = beta;
      int j = 0;
      for (; j < m && used < maxit; ++j) {
        precond(omega, basis(j), z.b.p);
        op(dir, z.b.p, w.b.p);
        axpy(zd(-omega), z.b.p, w.b.p);
        ++used;
        if (its) ++*its;
        for (int i = 0; i <= j; ++i) {
          const void *vi = basis(i);
          const zd hij = dot(vi, w.b.p, 1);
          H[(size_t)i * m + j] = hij;
          axpy(-hij, vi, w.b.p);
        }
        const double hn = norm(w.b.p);
        H[(size_t)(j + 1) * m + j] = hn;
        if (hn > 0) store(w.b.p, j + 1, 1.0 / hn);
        // apply previous rotations to column j, then a new one
        for (int i = 0; i < j; ++i) {
          const zd a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * c;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
        }
        const zd a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
        const double den = std::sqrt(std::norm(a) + std::norm(c));
        cs[j] = den > 0 ? a / den : zd(1);
        sn[j] = den > 0 ? c / den : zd(0);
        H[(size_t)j * m + j] = std::conj(cs[j]) * a + std::conj(sn[j]) * c;
        H[(size_t)(j + 1) * m + j] = 0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = std::conj(cs[j]) * g[j];
        rel = std::abs(g[j + 1]) / bn;
        if (verbose()) std::fprintf(stderr, "cclr gmres dir=%d omega=%g it=%d est=%.3e\n", dir, omega.real(), used, rel);
        if (rel < tol || hn == 0.0) { ++j; break; }
      }
      // y = H(0:j,0:j)^-1 g(0:j); x += P (sum_i y_i v_i)
      std::vector<zd> y(j);
      for (int i = j - 1; i >= 0; --i) {
        zd t = g[i];
        for (int k = i + 1; k < j; ++k) t -= H[(size_t)i * m + k] * y[k];
        const zd d = H[(size_t)i * m + i];
        y[i] = std::abs(d) > 0 ? t / d : zd(0);
      }
      CCLR_CUDA(cudaMemsetAsync(w.b.p, 0, (size_t)ntot() * 16, st));
      for (int i = 0; i < j; ++i) axpy(y[i], basis(i), w.b.p);
      precond(omega, w.b.p, z.b.p);
      axpy(zd(1), z.b.p, x);
      if (rel < tol) {
        // true residual for the return value
        copy(b, w.b.p);
        op(dir, x, z.b.p);
        axpy(zd(-1), z.b.p, w.b.p);
        axpy(zd(omega), x, w.b.p);
        rel = norm(w.b.p) / bn;
        if (rel < tol) break;
      }
    }
    CCLR_CUDA(cudaStreamSynchronize(st));
    return rel;
  }

  struct BlockSys {
    std::vector<AVec> V;  // Krylov basis
    AVec z, w;
    std::vector<zd> H, cs, sn, g;
    double bn = 1.0;
    int j = 0;
    bool done = false, cyc = false;
  };
  std::vector<BlockSys> blk;

  // frees the solver's Krylov bases and the full-layout scratch at the end of a solve call
  void release_scratch() {
    kv.clear();
    blk.clear();
    fullA.b.release();
    fullB.b.release();
  }

  // Block solve: nr independent systems (Op - omega_r) x_r = b_r advanced in lockstep, so that
  // each iteration applies the operator to every unconverged system in one batched product
  // (the ladder's <ab||ef>~ blocks are formed once per iteration for all of them).  Each system
  // keeps its own restarted, right-preconditioned GMRES (the method of solve_gmres); rel[r]
  // receives its final relative residual, its[r] its iteration count.
  void gmres_block(int dir, const std::vector<zd> &om, const std::vector<const void *> &b,
                   const std::vector<void *> &x, const std::vector<double> &tol, int m, int maxit,
                   std::vector<int> &its, std::vector<double> &rel, bool warm) {
    const int nr = (int)b.size();
    its.assign(nr, 0);
    rel.assign(nr, 1.0);
    if (nr == 0) return;
    m = std::max(2, std::min(m, 100));
    if ((int)blk.size() < nr) blk.resize(nr);  // kept between calls (no reallocation per solve)
    auto &S = blk;
    for (int r = 0; r < nr; ++r) {
      BlockSys &q = S[r];
      if ((int)q.V.size() < m + 1) q.V.resize(m + 1);
      for (int k = 0; k <= m; ++k) alloc_vec(q.V[k]);
      q.done = false;
      q.cyc = false;
      q.j = 0;
      alloc_vec(q.z);
      alloc_vec(q.w);
      q.H.assign((size_t)(m + 1) * m, zd(0));
      q.cs.assign(m, zd(0));
      q.sn.assign(m, zd(0));
      q.g.assign(m + 1, zd(0));
      q.bn = std::max(norm(b[r]), 1e-300);
      if (!warm) CCLR_CUDA(cudaMemsetAsync(x[r], 0, (size_t)ntot() * 16, st));
    }
    int used = 0;
    std::vector<int> act;
    std::vector<const void *> in;
    std::vector<void *> out;
    auto batch = [&](const std::vector<int> &ids, bool from_x) {
      in.clear();
      out.clear();
      for (int r : ids) {
        in.push_back(from_x ? (const void *)x[r] : (const void *)S[r].z.b.p);
        out.push_back(S[r].w.b.p);
      }
      if (!ids.empty()) op_batch(dir, (int)ids.size(), in.data(), out.data());
    };
    while (used < maxit) {
      // true residuals of the systems still running
      act.clear();
      for (int r = 0; r < nr; ++r)
        if (!S[r].done) act.push_back(r);
      if (act.empty()) break;
      for (int r : act) copy(b[r], S[r].V[0].b.p);
      if (warm || used > 0) {
        batch(act, true);
        for (int r : act) {
          axpy(zd(-1), S[r].w.b.p, S[r].V[0].b.p);
          axpy(zd(om[r]), x[r], S[r].V[0].b.p);
        }
      }
      warm = true;
      std::vector<int> cyc;
      for (int r : act) {
        BlockSys &q = S[r];
        const double beta = norm(q.V[0].b.p);
        rel[r] = beta / q.bn;
        if (!(rel[r] == rel[r])) throw Error(3, "solver produced NaN residual");
        if (verbose()) std::fprintf(stderr, "cclr block gmres r=%d dir=%d omega=%g it=%d rel=%.3e prec=%d\n", r, dir, om[r].real(), its[r], rel[r], M->prec);
        if (rel[r] < tol[r] || beta == 0.0) {
          q.done = true;
          continue;
        }
        scal(zd(1.0 / beta), q.V[0].b.p);
        std::fill(q.g.begin(), q.g.end(), zd(0));
        q.g[0] = beta;
        q.j = 0;
        q.cyc = true;
        cyc.push_back(r);
      }
      if (cyc.empty()) break;
      for (int j = 0; j < m && used < maxit; ++j) {
        std::vector<int> step;
        for (int r : cyc)
          if (S[r].cyc) step.push_back(r);
        if (step.empty()) break;
        for (int r : step) precond(om[r], S[r].V[j].b.p, S[r].z.b.p);
        batch(step, false);
        ++used;
        for (int r : step) {
          BlockSys &q = S[r];
          ++its[r];
          axpy(zd(-om[r]), q.z.b.p, q.w.b.p);
          for (int i = 0; i <= j; ++i) {
            const zd hij = dot(q.V[i].b.p, q.w.b.p, 1);
            q.H[(size_t)i * m + j] = hij;
            axpy(-hij, q.V[i].b.p, q.w.b.p);
          }
          const double hn = norm(q.w.b.p);
          q.H[(size_t)(j + 1) * m + j] = hn;
          if (hn > 0) {
            copy(q.w.b.p, q.V[j + 1].b.p);
            scal(zd(1.0 / hn), q.V[j + 1].b.p);
          }
          for (int i = 0; i < j; ++i) {
            const zd a = q.H[(size_t)i * m + j], c_ = q.H[(size_t)(i + 1) * m + j];
            q.H[(size_t)i * m + j] = std::conj(q.cs[i]) * a + std::conj(q.sn[i]) * c_;
            q.H[(size_t)(i + 1) * m + j] = -q.sn[i] * a + q.cs[i] * c_;
          }
          const zd a = q.H[(size_t)j * m + j], c_ = q.H[(size_t)(j + 1) * m + j];
          const double den = std::sqrt(std::norm(a) + std::norm(c_));
          q.cs[j] = den > 0 ? a / den : zd(1);
          q.sn[j] = den > 0 ? c_ / den : zd(0);
          q.H[(size_t)j * m + j] = std::conj(q.cs[j]) * a + std::conj(q.sn[j]) * c_;
          q.H[(size_t)(j + 1) * m + j] = 0;
          q.g[j + 1] = -q.sn[j] * q.g[j];
          q.g[j] = std::conj(q.cs[j]) * q.g[j];
          q.j = j + 1;
          const double est = std::abs(q.g[j + 1]) / q.bn;
          if (est < tol[r] || hn == 0.0 || its[r] >= maxit) q.cyc = false;
        }
      }
      // x_r += P (sum_i y_i v_i) with y from each system's own triangular system
      for (int r : cyc) {
        BlockSys &q = S[r];
        const int jr = q.j;
        std::vector<zd> y(jr);
        for (int i = jr - 1; i >= 0; --i) {
          zd t = q.g[i];
          for (int k = i + 1; k < jr; ++k) t -= q.H[(size_t)i * m + k] * y[k];
          const zd d = q.H[(size_t)i * m + i];
          y[i] = std::abs(d) > 0 ? t / d : zd(0);
        }
        CCLR_CUDA(cudaMemsetAsync(q.w.b.p, 0, (size_t)ntot() * 16, st));
        for (int i = 0; i < jr; ++i) axpy(y[i], q.V[i].b.p, q.w.b.p);
        precond(om[r], q.w.b.p, q.z.b.p);
        axpy(zd(1), q.z.b.p, x[r]);
        if (its[r] >= maxit) q.done = true;
      }
    }
    // final true residuals of the systems that stopped on an estimate or the iteration limit
    act.clear();
    for (int r = 0; r < nr; ++r) act.push_back(r);
    for (int r : act) copy(b[r], S[r].V[0].b.p);
    batch(act, true);
    for (int r : act) {
      axpy(zd(-1), S[r].w.b.p, S[r].V[0].b.p);
      axpy(zd(om[r]), x[r], S[r].V[0].b.p);
      rel[r] = norm(S[r].V[0].b.p) / S[r].bn;
    }
    CCLR_CUDA(cudaStreamSynchronize(st));
  }

  // The block form of solve(): in FP64 one block GMRES; in the mixed modes a refinement whose
  // residuals (accurate precision) and corrections (working precision) are both batched.
  void solve_block(int dir, const std::vector<zd> &om, const std::vector<const void *> &b,
                   const std::vector<void *> &x, double tol, int maxit, std::vector<int> &its,
                   std::vector<double> &rel, bool warm = false) {
    const int nr = (int)b.size();
    const int m = block_restart(nr, M->lean ? 0.2 : 0.5);
    if (M->prec == CCLR_FP64) {
      gmres_block(dir, om, b, x, std::vector<double>(nr, tol), m, maxit, its, rel, warm);
      return;
    }
    const int lo = M->prec;
    const double inner_tol = lo == CCLR_C64_TF32 ? 1e-2 : 1e-5;
    const int inner_cap = lo == CCLR_C64_TF32 ? 30 : 40;
    std::vector<AVec> sv(nr), rv(nr), dv(nr), xb(nr);
    std::vector<double> bn(nr), prev(nr, 1e300);
    std::vector<int> state(nr, 0);  // 0 refining, 1 converged, 2 stalled or out of iterations
    its.assign(nr, 0);
    rel.assign(nr, 1.0);
    for (int r = 0; r < nr; ++r) {
      alloc_vec(sv[r]); alloc_vec(rv[r]); alloc_vec(dv[r]); alloc_vec(xb[r]);
      bn[r] = std::max(norm(b[r]), 1e-300);
      if (!warm) CCLR_CUDA(cudaMemsetAsync(x[r], 0, (size_t)ntot() * 16, st));
      copy(b[r], rv[r].b.p);
    }
    for (int outer = 0; outer < 40; ++outer) {
      std::vector<int> act;
      for (int r = 0; r < nr; ++r)
        if (state[r] == 0) act.push_back(r);
      if (act.empty()) break;
      if (outer > 0 || warm) {
        std::vector<const void *> in;
        std::vector<void *> out;
        for (int r : act) { in.push_back(x[r]); out.push_back(sv[r].b.p); }
        M->prec = hi_prec;
        op_batch(dir, (int)act.size(), in.data(), out.data());
        M->prec = lo;
        ++refinements;
        for (int r : act) {
          copy(b[r], rv[r].b.p);
          axpy(zd(-1), sv[r].b.p, rv[r].b.p);
          axpy(zd(om[r]), x[r], rv[r].b.p);
        }
      }
      std::vector<int> go;
      std::vector<zd> gom;
      std::vector<double> gtol;
      std::vector<const void *> gb;
      std::vector<void *> gx;
      for (int r : act) {
        rel[r] = norm(rv[r].b.p) / bn[r];
        if (!(rel[r] == rel[r])) throw Error(3, "solver produced NaN residual");
        if (verbose()) std::fprintf(stderr, "cclr block refine r=%d dir=%d omega=%g outer=%d rel=%.3e\n", r, dir, om[r].real(), outer, rel[r]);
        if (rel[r] > 0.5 * prev[r]) {  // the last correction did not help
          if (rel[r] > prev[r]) {
            copy(xb[r].b.p, x[r]);
            rel[r] = prev[r];
          }
          state[r] = 2;
          continue;
        }
        if (rel[r] < tol) { state[r] = 1; continue; }
        if (its[r] >= maxit) { state[r] = 2; continue; }
        copy(x[r], xb[r].b.p);
        prev[r] = rel[r];
        go.push_back(r);
        gom.push_back(om[r]);
        gtol.push_back(std::max(inner_tol, 0.3 * tol / rel[r]));
        gb.push_back(rv[r].b.p);
        gx.push_back(dv[r].b.p);
      }
      if (go.empty()) continue;
      int cap = inner_cap;
      for (int r : go) cap = std::min(cap, maxit - its[r]);
      std::vector<int> inner_its;
      std::vector<double> inner_rel;
      gmres_block(dir, gom, gb, gx, gtol, std::min(m, cap), std::max(1, cap), inner_its, inner_rel, false);
      for (size_t k = 0; k < go.size(); ++k) {
        its[go[k]] += inner_its[k];
        axpy(zd(1), dv[go[k]].b.p, x[go[k]]);
      }
    }
    // systems that stalled or ran out: finish in the accurate arithmetic, warm-started
    std::vector<int> fin;
    std::vector<zd> fom;
    std::vector<const void *> fb;
    std::vector<void *> fx_;
    int rest_cap = maxit;
    for (int r = 0; r < nr; ++r)
      if (rel[r] >= tol && its[r] < maxit) {
        fin.push_back(r); fom.push_back(om[r]); fb.push_back(b[r]); fx_.push_back(x[r]);
        rest_cap = std::min(rest_cap, maxit - its[r]);
      }
    if (!fin.empty()) {
      std::vector<int> fits;
      std::vector<double> frel;
      M->prec = hi_prec;
      gmres_block(dir, fom, fb, fx_, std::vector<double>(fin.size(), tol), m, rest_cap, fits, frel, true);
      M->prec = lo;
      for (size_t k = 0; k < fin.size(); ++k) {
        its[fin[k]] += fits[k];
        rel[fin[k]] = frel[k];
      }
    }
  }

  // restart length of the block solver: the Krylov bases of all systems must fit in half of
  // the free device memory (and of what the context's budget leaves)
  int block_restart(int nr, double frac = 0.5, int bytes_per_entry = 16) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      (void)cudaGetLastError();
      return krylov;
    }
    if (acct.budget) {
      size_t avail = acct.budget > acct.used ? acct.budget - acct.used : (size_t)0;
      // once a product has run, its transient memory is known and is all that must stay free
      if (op_transient) {
        const size_t keep = op_transient + op_transient / 8;
        avail = avail > keep ? avail - keep : 0;
        frac = 0.9;
      }
      free_b = std::min(free_b, avail);
    }
    const double vec = (double)ntot() * bytes_per_entry;
    // four complex128 work vectors besides the basis
    const int fit = (int)((frac * (double)free_b - 4.0 * (double)ntot() * 16) / (vec * std::max(1, nr))) - 1;
    return std::max(2, std::min(krylov, fit));
  }

  // Preconditioned DIIS (Pulay extrapolation over Jacobi steps) on (Op - omega) x = b.
  double solve_pulay(int dir, zd omega, const void *b, void *x, double tol, int depth, int maxit,
                     int *its, bool warm = false) {
    depth = std::max(2, std::min(depth, 16));
    std::vector<AVec> X(depth), Er(depth);
    for (auto &a : X) alloc_vec(a);
    for (auto &a : Er) alloc_vec(a);
    AVec s, r;
    alloc_vec(s);
    alloc_vec(r);
    const double bn = std::max(norm(b), 1e-300);
    if (!warm) precond(omega, b, x);
    std::vector<zd> B((size_t)depth * depth);
    int nh = 0, head = 0;
    double rel = 1e300;
    for (int it = 0; it < maxit; ++it) {
      op(dir, x, s.b.p);
      copy(b, r.b.p);
      axpy(zd(-1), s.b.p, r.b.p);
      axpy(zd(omega), x, r.b.p);
      rel = norm(r.b.p) / bn;
      if (its) ++*its;
      if (verbose()) std::fprintf(stderr, "cclr diis dir=%d omega=%g it=%d rel=%.3e prec=%d\n", dir, omega.real(), it, rel, M->prec);
      if (!(rel == rel)) throw Error(3, "solver produced NaN residual");
      if (rel < tol) break;
      int k = head;
      head = (head + 1) % depth;
      nh = std::min(nh + 1, depth);
      precond(omega, r.b.p, Er[k].b.p);
      copy(x, X[k].b.p);
      axpy(zd(1), Er[k].b.p, X[k].b.p);
      for (int l = 0; l < depth; ++l) {
        if (!(nh == depth || l < nh)) continue;  // slot not filled yet
        zd d = dot(Er[k].b.p, Er[l].b.p, 1);
        B[(size_t)k * depth + l] = d;
        B[(size_t)l * depth + k] = std::conj(d);
      }
      if (nh < 2) {
        copy(X[k].b.p, x);
        continue;
      }
      // slots in use: if nh < depth they are 0..nh-1, else all
      std::vector<int> idx;
      for (int l = 0; l < depth; ++l)
        if (nh == depth || l < nh) idx.push_back(l);
      int m = (int)idx.size();
      double sc = 0.0;
      for (int a : idx) sc = std::max(sc, std::abs(B[(size_t)a * depth + a]));
      if (sc <= 0) sc = 1.0;
      std::vector<zd> Am((size_t)(m + 1) * (m + 1)), rhs(m + 1, 0.0);
      for (int a = 0; a < m; ++a) {
        for (int c = 0; c < m; ++c) Am[(size_t)a * (m + 1) + c] = B[(size_t)idx[a] * depth + idx[c]] / sc;
        Am[(size_t)a * (m + 1) + m] = 1.0;
        Am[(size_t)m * (m + 1) + a] = 1.0;
      }
      Am[(size_t)m * (m + 1) + m] = 0.0;
      rhs[m] = 1.0;
      std::vector<zd> c = solve_small(Am, rhs, m + 1);
      CCLR_CUDA(cudaMemsetAsync(x, 0, (size_t)ntot() * 16, st));
      for (int a = 0; a < m; ++a) axpy(c[a], X[idx[a]].b.p, x);
    }
    CCLR_CUDA(cudaStreamSynchronize(st));
    return rel;
  }

  static std::vector<zd> solve_small(std::vector<zd> A, std::vector<zd> b, int N) {
    for (int c = 0; c < N; ++c) {
      int piv = c;
      for (int r = c + 1; r < N; ++r)
        if (std::abs(A[(size_t)r * N + c]) > std::abs(A[(size_t)piv * N + c])) piv = r;
      if (piv != c) {
        for (int k = 0; k < N; ++k) std::swap(A[(size_t)c * N + k], A[(size_t)piv * N + k]);
        std::swap(b[c], b[piv]);
      }
      zd d = A[(size_t)c * N + c];
      if (std::abs(d) < 1e-300) d = 1e-300;
      for (int r = c + 1; r < N; ++r) {
        zd f = A[(size_t)r * N + c] / d;
        for (int k = c; k < N; ++k) A[(size_t)r * N + k] -= f * A[(size_t)c * N + k];
        b[r] -= f * b[c];
      }
    }
    std::vector<zd> x(N);
    for (int r = N - 1; r >= 0; --r) {
      zd s = b[r];
      for (int k = r + 1; k < N; ++k) s -= A[(size_t)r * N + k] * x[k];
      zd d = A[(size_t)r * N + r];
      if (std::abs(d) < 1e-300) d = 1e-300;
      x[r] = s / d;
    }
    return x;
  }

  // xi^comp at amplitudes (t1d, t2d) (full layouts), written packed into out
  void xi_vec(int comp, const void *t1d, const void *t2d, void *out) {
    alloc_full(fullA);
    const int64_t nn = (int64_t)M->n * M->n;
    M->xi((char *)M->mu.p + (size_t)comp * nn * 16, t1d, t2d, fullA.p1(), fullA.p2(n1));
    pack_from(fullA.b.p, C128, out);
  }

  // ---- ground-state CCSD: the amplitude equations Omega(T) = 0 and the energy (Sec. 2.2) ----
  CstSet gs;  // intermediates at s T, s a quadrature node of the residual (scratch)

  // the arithmetic of a ground-state product: a cclr_prec, or -1 for the context's own
  int gs_prec(int p) const {
    if (p < 0) p = M->prec;
    if (p > 4) throw Error(CCLR_EINVAL, "unknown precision mode");
    if (p == CCLR_FP64 && M->fp64_gone)
      throw Error(CCLR_EUNSUPPORTED, "FP64 products are unavailable: this budgeted context freed its FP64 inputs");
    return p;
  }

  // Omega(T), packed, at the packed amplitudes tp, with the sigma products in precision p.
  // CCSD is at most quartic in T, so Omega(sT) is a polynomial of degree four in s, and its
  // derivative d/ds Omega(sT) = A(sT) T is the Jacobian product of the sigma program with the
  // intermediates built at sT.  Hence Omega(T) = Omega(0) + int_0^1 A(sT) T ds, and the
  // two-point Gauss-Legendre rule on [0, 1] (nodes 1/2 -+ 1/(2 sqrt 3), weights 1/2) integrates
  // the cubic integrand exactly.  Omega(0) = <mu|H|Phi_0> is f_ai (zero for the canonical Fock
  // matrix diag(eps)) and <ab||ij>, the complex conjugate of <ij||ab> for Hermitian L^P.
  void ccsd_residual(int p, const void *tp, void *r) {
    alloc_full(fullA);
    alloc_full(fullB);
    AVec sv;
    alloc_vec(sv);
    unpack_to(tp, fullA.b.p, C128);
    CCLR_CUDA(cudaMemsetAsync(r, 0, (size_t)n1 * 16, st));
    vec_conj(n2p, M->oovv_packed(), (char *)r + n1 * 16, st);
    const Tens TA = make_tens(fullA.b.p, C128, {nfull()}), TB = make_tens(fullB.b.p, C128, {nfull()});
    const double h = 0.5 / std::sqrt(3.0);
    const int saved = M->prec;
    try {
      for (double s : {0.5 - h, 0.5 + h}) {
        M->E.permute(zc(s), TA, "a", TB, "a", false);
        // complex64 intermediates at s T built on the tensor cores in 3xTF32 (FP32-level accuracy,
        // a few times faster than the FP32 CUDA cores) when the products use them too
        M->build_set(fullB.p1(), fullB.p2(n1), gs, p == CCLR_FP64 ? C128 : C64,
                     p == CCLR_FP64 || p == CCLR_C64_FP32 ? 0 : 2);
        M->prec = p;
        op(+1, tp, sv.b.p, &gs);
        M->prec = saved;
        axpy(zd(0.5), sv.b.p, r);
      }
    } catch (...) {
      M->prec = saved;
      throw;
    }
  }

  // E(T) = sum_ia f_ia t_ia + 1/4 sum <ij||ab> t_ijab + 1/2 sum <ij||ab> t_ia t_jb
  //      = sum over i<j, a<b of <ij||ab> tau_ijab (f_ia = 0), packed amplitudes tp
  zd ccsd_energy(const void *tp) {
    DevBuf tau((size_t)std::max<int64_t>(1, n2p) * 16);
    tau_packed(o, v, tp, (const char *)tp + n1 * 16, tau.p, st);
    double2 *part = M->E.dot_scratch();
    double2 *res = M->E.dot_results();
    vec_dot(C128, n2p, M->oovv_packed(), tau.p, 0, part, res, 0, st);
    double2 e;
    CCLR_CUDA(cudaMemcpyAsync(&e, res, sizeof(e), cudaMemcpyDeviceToHost, st));
    CCLR_CUDA(cudaStreamSynchronize(st));
    return zd(e.x, e.y);
  }

  // the context's amplitudes (M->t1, M->t2, full layouts) packed into out
  void pack_t(void *out) {
    CCLR_CUDA(cudaMemcpyAsync(out, M->t1.p, (size_t)n1 * 16, cudaMemcpyDeviceToDevice, st));
    pack_doubles(C128, C128, o, v, M->t2.p, (char *)out + n1 * 16, st);
  }

  // New amplitudes (packed tp): every quantity that depends on T is rebuilt (intermediates in the
  // working precision, the preconditioner) or dropped (Lambda, eta, the stencil and one-body sets).
  void set_amplitudes(const void *tp) {
    CCLR_CUDA(cudaMemcpyAsync(M->t1.p, tp, (size_t)n1 * 16, cudaMemcpyDeviceToDevice, st));
    unpack_doubles(C128, C128, o, v, (const char *)tp + n1 * 16, M->t2.p, zc(1), false, st);
    M->release_set(gs);
    M->release_set(shift);
    M->release_set(shift64);
    for (auto &b : onebody) M->release_set(b);
    for (int k = 0; k < 3; ++k) eta_ok[k] = false;
    have_lambda = false;
    M->release_set(M->c128);
    M->release_set(M->c64);
    M->clear_graphs();
    M->cst_for(M->prec);
    M->build_diagonal();
    CCLR_CUDA(cudaStreamSynchronize(st));
  }

  // Quasi-Newton iterations T <- T - Omega(T) / D, D the orbital-energy differences (the
  // diagonal of the T = 0 Jacobian), with Pulay extrapolation over the last `depth` steps
  // (error vectors Omega / D).  Starts from the context's amplitudes; returns the final norm of
  // the packed residual and leaves the final amplitudes packed in tv.
  double ccsd_solve(int p, double tol, int maxit, int depth, AVec &tv, int *its) {
    depth = std::max(2, std::min(depth, 16));
    alloc_vec(tv);
    pack_t(tv.b.p);
    {  // D from diag(eps): Foo = diag(eps_occ), Fvv = diag(eps_vir)
      DevBuf f((size_t)(o * o + v * v) * 16);
      CCLR_CUDA(cudaMemsetAsync(f.p, 0, f.bytes, st));
      void *foo = f.p, *fvv = (char *)f.p + (size_t)o * o * 16;
      set_diag(o, M->eps.as<double>(), foo, st);
      set_diag(v, M->eps.as<double>() + o, fvv, st);
      build_diag(o, v, foo, fvv, M->D1.as<double>(), M->D2.as<double>(), st);
      CCLR_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<AVec> X(depth), Er(depth);
    AVec r;
    alloc_vec(r);
    std::vector<zd> B((size_t)depth * depth);
    int nh = 0, head = 0;
    double rn = 1e300, rn0 = 1e300;
    for (int it = 0; it < maxit; ++it) {
      ccsd_residual(p, tv.b.p, r.b.p);
      rn = norm(r.b.p);
      if (its) ++*its;
      if (verbose()) std::fprintf(stderr, "cclr ccsd it=%d |Omega|=%.3e prec=%d\n", it, rn, p);
      if (!(rn == rn)) throw Error(3, "ground-state iteration produced a non-finite residual");
      if (it == 0) rn0 = rn;
      if (rn > 1e3 * rn0)
        throw Error(3, "ground-state iteration diverged (residual " + std::to_string(rn) + " from " +
                           std::to_string(rn0) + "): the amplitudes are left unchanged");
      if (rn < tol) break;
      const int k = head;
      head = (head + 1) % depth;
      nh = std::min(nh + 1, depth);
      alloc_vec(X[k]);
      alloc_vec(Er[k]);
      precond(zd(0), r.b.p, Er[k].b.p);  // Omega / D
      scal(zd(-1), Er[k].b.p);           // the Jacobi step -Omega / D
      copy(tv.b.p, X[k].b.p);
      axpy(zd(1), Er[k].b.p, X[k].b.p);
      for (int l = 0; l < depth; ++l) {
        if (!(nh == depth || l < nh)) continue;
        const zd d = dot(Er[k].b.p, Er[l].b.p, 1);
        B[(size_t)k * depth + l] = d;
        B[(size_t)l * depth + k] = std::conj(d);
      }
      if (nh < 2) {
        copy(X[k].b.p, tv.b.p);
        continue;
      }
      std::vector<int> idx;
      for (int l = 0; l < depth; ++l)
        if (nh == depth || l < nh) idx.push_back(l);
      const int m = (int)idx.size();
      double sc = 0.0;
      for (int a : idx) sc = std::max(sc, std::abs(B[(size_t)a * depth + a]));
      if (sc <= 0) sc = 1.0;
      std::vector<zd> Am((size_t)(m + 1) * (m + 1)), rhs(m + 1, 0.0);
      for (int a = 0; a < m; ++a) {
        for (int c2 = 0; c2 < m; ++c2) Am[(size_t)a * (m + 1) + c2] = B[(size_t)idx[a] * depth + idx[c2]] / sc;
        Am[(size_t)a * (m + 1) + m] = 1.0;
        Am[(size_t)m * (m + 1) + a] = 1.0;
      }
      rhs[m] = 1.0;
      const std::vector<zd> cf = solve_small(Am, rhs, m + 1);
      CCLR_CUDA(cudaMemsetAsync(tv.b.p, 0, (size_t)ntot() * 16, st));
      for (int a = 0; a < m; ++a) axpy(cf[a], X[idx[a]].b.p, tv.b.p);
    }
    CCLR_CUDA(cudaStreamSynchronize(st));
    return rn;
  }

  // eta0 = dE/dT = [ sum_jb <ij||ab> t_jb ; <ij||ab> ] (canonical Fock: f_ia = 0), packed
  void eta0(void *out) {
    const void *oovv = M->oovv_packed();
    Tens e1 = make_tens(out, C128, {o, v});
    M->E.zero(e1);
    packed_doubles_dot_singles(o, v, oovv, M->t1.p, out, zc(1), st);
    CCLR_CUDA(cudaMemcpyAsync((char *)out + n1 * 16, oovv, (size_t)n2p * 16, cudaMemcpyDeviceToDevice, st));
    // f_ia of diag(eps) is zero; the one-body h keeps any ov part of the input Fock
  }

  void ensure_lambda(double tol, int depth, cclr_stats *stats) {
    if (have_lambda) return;
    auto t0 = std::chrono::steady_clock::now();
    alloc_vec(lam);
    AVec b;
    alloc_vec(b);
    eta0(b.b.p);
    scal(zd(-1), b.b.p);
    int its = 0;
    double rel = solve(-1, 0.0, b.b.p, lam.b.p, tol, depth, maxit, &its);
    if (stats) {
      stats->iterations += its;
      stats->time_lambda_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      stats->max_rel_residual = std::max(stats->max_rel_residual, rel);
      if (rel >= tol) stats->converged = 0;
    }
    have_lambda = true;
  }

  // step length for the polynomial-exact stencils
  double step(const void *x) {
    double nx = norm(x);
    double nt = tnorm();  // ||T|| over unique amplitudes
    return std::max(nt, 1e-2) / std::max(nx, 1e-300) * 0.25;
  }
  double tnorm() {
    // t1, t2 are separate buffers: assemble weighted norm
    double2 *part = M->E.dot_scratch();
    double2 *res = M->E.dot_results();
    vec_dot(C128, n1, M->t1.p, M->t1.p, 1, part, res, 0, st);
    vec_dot(C128, n2, M->t2.p, M->t2.p, 1, part, res, 1, st);
    double2 h[2];
    CCLR_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st));
    CCLR_CUDA(cudaStreamSynchronize(st));
    return std::sqrt(h[0].x + 0.25 * h[1].x);
  }

  // shifted amplitudes T + k h X (X packed) into the full-layout scratch fullB
  AVec &shifted(const void *x, double kh) {
    alloc_full(fullB);
    CCLR_CUDA(cudaMemcpyAsync(fullB.p1(), M->t1.p, (size_t)n1 * 16, cudaMemcpyDeviceToDevice, st));
    CCLR_CUDA(cudaMemcpyAsync(fullB.p2(n1), M->t2.p, (size_t)n2 * 16, cudaMemcpyDeviceToDevice, st));
    vec_axpy(C128, n1, zc(kh), x, fullB.p1(), st);
    unpack_doubles(C128, C128, o, v, (const char *)x + n1 * 16, fullB.p2(n1), zc(kh), true, st);
    return fullB;
  }

  // eta^A = dE_A/dT + lambda dxi^A/dT = [mu^A_ia ; 0] + lambda A[mu^A], with A[mu^A] the
  // Jacobian of the one-body operator mu^A alone (xi^A(T) = Omega[mu^A](T), Omega linear in the
  // Hamiltonian): the transpose program on mu^A's own H-bar set, in FP64.  Packed, cached.
  const void *eta_vec(int comp) {
    if (!eta_ok[comp]) {
      const int64_t nn = (int64_t)M->n * M->n;
      const void *mub = (char *)M->mu.p + (size_t)comp * nn * 16;
      if (!onebody[comp].valid) M->build_set_onebody(mub, M->t1.p, M->t2.p, onebody[comp]);
      alloc_vec(eta_v[comp]);
      op(-1, lam.b.p, eta_v[comp].b.p, &onebody[comp]);
      Tens muA = make_tens((void *)mub, C128, {M->n, M->n});
      M->E.permute(zc(1), muA.slice(0, 0, o).slice(1, o, M->n), "ia", make_tens(eta_v[comp].b.p, C128, {o, v}), "ia",
                   true);
      eta_ok[comp] = true;
    }
    return eta_v[comp].b.p;
  }

  // eta^A . X (bilinear over unique amplitudes)
  zd eta_dot(int comp, const void *x) { return dot(eta_vec(comp), x, 0); }

  // eta^A . X = sum_ia mu^A_ia X_ia + d/de lambda . xi^A(T + eX)   (4-point stencil; the
  // definition, kept as a check of eta_vec)
  zd eta_dot_stencil(int comp, const void *x) {
    const int64_t nn = (int64_t)M->n * M->n;
    Tens muA = make_tens((char *)M->mu.p + (size_t)comp * nn * 16, C128, {M->n, M->n});
    // sum_ia mu_ia X_ia
    DevBuf mov((size_t)n1 * 16);
    Tens mo = make_tens(mov.p, C128, {o, v});
    M->E.permute(zc(1), muA.slice(0, 0, o).slice(1, o, M->n), "ia", mo, "ia", false);
    double2 *part = M->E.dot_scratch();
    double2 *res = M->E.dot_results();
    vec_dot(C128, n1, mov.p, x, 0, part, res, 0, st);
    double2 hv;
    CCLR_CUDA(cudaMemcpyAsync(&hv, res, sizeof(hv), cudaMemcpyDeviceToHost, st));
    CCLR_CUDA(cudaStreamSynchronize(st));
    zd val(hv.x, hv.y);
    const double h = step(x);
    static const double cs[4] = {-1, 8, -8, 1}, ks[4] = {2, 1, -1, -2};
    AVec xv;
    alloc_vec(xv);
    zd acc = 0.0;
    for (int s = 0; s < 4; ++s) {
      AVec &ts = shifted(x, ks[s] * h);
      xi_vec(comp, ts.p1(), ts.p2(n1), xv.b.p);
      acc += cs[s] * dot(lam.b.p, xv.b.p, 0);
    }
    return val + acc / (12.0 * h);
  }

  // F X = d/de [ lambda A(T + eX) + eta0(T + eX) ]  (4-point stencil over rebuilt H-bar)
  void fx(const void *x, void *out) {
    const double h = step(x);
    static const double cs[4] = {-1, 8, -8, 1}, ks[4] = {2, 1, -1, -2};
    AVec sv;
    alloc_vec(sv);
    CCLR_CUDA(cudaMemsetAsync(out, 0, (size_t)ntot() * 16, st));
    // a budgeted context holds one set of intermediates at a time: the working set is freed while
    // the stencil's sets exist and rebuilt on its next use
    if (M->lean) {
      M->release_set(M->c64);
      M->release_set(M->c128);
    }
    for (int s = 0; s < 4; ++s) {
      // and the products' own buffers are freed before each build, whose temporaries need the room
      if (M->lean) {
        M->release_product_buffers();
        for (auto &v : xfs) v.clear();
        for (auto &v : sfs) v.clear();
      }
      AVec &ts = shifted(x, ks[s] * h);
      const int saved = M->prec;
      const int use = M->prec == CCLR_FP64 ? CCLR_FP64 : hi_prec;
      M->prec = use;
      if (use == CCLR_FP64) {
        M->build_set(ts.p1(), ts.p2(n1), shift, C128);
        op(-1, lam.b.p, sv.b.p, &shift);
      } else {
        // intermediates at the shifted amplitudes built in FP32 on the CUDA cores: at o=32,
        // v=240 the resulting alpha agreed with FP64-built, complex64-rounded sets to 1e-9
        // relative, for a sixth of the time
        M->build_set(ts.p1(), ts.p2(n1), shift64, C64);
        op(-1, lam.b.p, sv.b.p, &shift64);
      }
      M->prec = saved;
      axpy(zd(cs[s] / (12.0 * h)), sv.b.p, out);
    }
    // d eta0 / dT along X: sum_jb <ij||ab> X_jb (singles only)
    packed_doubles_dot_singles(o, v, M->oovv_packed(), x, out, zc(1), st);
    if (M->lean) {  // the stencil's set is rebuilt for every X: not kept in a budgeted context
      M->release_set(shift64);
      M->release_set(shift);
      fullB.b.release();
    }
    CCLR_CUDA(cudaStreamSynchronize(st));
  }
};

namespace {
template <typename F> int guarded(F &&f) {
  try {
    f();
    return CCLR_OK;
  } catch (const Error &e) {
    return fail(e.status, e.what());
  } catch (const std::exception &e) {
    return fail(CCLR_EDEVICE, e.what());
  }
}

// the same with the call's device allocations charged to (and limited by) the context's account
template <typename F> int guarded_ctx(cclr_ctx *c, F &&f) {
  AcctScope scope(&c->acct);
  return guarded(std::forward<F>(f));
}

}  // namespace

namespace cclr {
// Records msg as the thread's last error (cc_lr_last_error) and returns status; for entry
// points defined in other translation units.
int record_error(int status, const std::string &msg) { return fail(status, msg); }
}  // namespace cclr

namespace {

// cudaMemcpyDefault: the direction follows from the pointers (unified addressing), so host
// and device arrays are both accepted whatever device_ptrs said at init.
void to_dev(cclr_ctx *c, const double *src, void *dst, size_t bytes) {
  CCLR_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->st));
}
void from_dev(cclr_ctx *c, const void *src, double *dst, size_t bytes) {
  CCLR_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->st));
}
}  // namespace

extern "C" {

cclr_status cc_lr_init(cclr_ctx **ctx, int o, int v, int naux, const double *eps, const double *L,
                       const double *mu, const double *t1, const double *t2, const double *lam1,
                       const double *lam2, int prec, size_t hbm_budget_bytes, int device_ptrs,
                       void *cuda_stream) {
  if (!ctx) return (cclr_status)fail(CCLR_EINVAL, "ctx is NULL");
  *ctx = nullptr;
  if (o < 1 || v < 1 || naux < 1) return (cclr_status)fail(CCLR_EINVAL, "o, v and naux must be >= 1");
  if (!eps || !L || !mu) return (cclr_status)fail(CCLR_EINVAL, "eps, L and mu are required");
  if (prec < 0 || prec > 4) return (cclr_status)fail(CCLR_EINVAL, "unknown precision mode");
  if ((lam1 == nullptr) != (lam2 == nullptr)) return (cclr_status)fail(CCLR_EINVAL, "lam1 and lam2 must both be given or both be NULL");
  auto c = new cclr_ctx();
  c->acct.budget = hbm_budget_bytes;
  int st = guarded_ctx(c, [&] {
    c->o = o; c->v = v; c->naux = naux;
    c->n1 = (int64_t)o * v;
    c->n2 = (int64_t)o * o * v * v;
    c->n2p = (int64_t)o * (o - 1) / 2 * ((int64_t)v * (v - 1) / 2);
    c->device_ptrs = device_ptrs;
    c->st = (cudaStream_t)cuda_stream;
    int dev = 0;
    CCLR_CUDA(cudaGetDevice(&dev));
    c->M.reset(new Model(o, v, naux, c->st));
    c->M->prec = prec;
    c->M->lean = hbm_budget_bytes > 0;
    // prepared constant operands of the tensor-core contractions are kept (up to 8 GB) unless the
    // context has a budget
    c->M->E.prep_cache_cap = c->M->lean ? 0 : (size_t)8 << 30;
    c->M->upload_inputs(eps, L, mu, t1, t2, device_ptrs);
    c->M->cst_for(prec);      // intermediates in the working precision
    c->M->build_diagonal();
    if (lam1) {
      c->alloc_vec(c->lam);
      c->alloc_full(c->fullA);
      to_dev(c, lam1, c->fullA.p1(), (size_t)c->n1 * 16);
      to_dev(c, lam2, c->fullA.p2(c->n1), (size_t)c->n2 * 16);
      c->pack_from(c->fullA.b.p, C128, c->lam.b.p);
      c->have_lambda = true;
    }
    CCLR_CUDA(cudaStreamSynchronize(c->st));
  });
  if (st != CCLR_OK) {
    delete c;
    return (cclr_status)st;
  }
  *ctx = c;
  return CCLR_OK;
}

static cclr_status sigma_common(cclr_ctx *c, int dir, int nrhs, const double *x1, const double *x2,
                                double *s1, double *s2) {
  if (!c || nrhs < 0 || (nrhs > 0 && (!x1 || !x2 || !s1 || !s2)))
    return (cclr_status)fail(CCLR_EINVAL, "bad sigma arguments");
  return (cclr_status)guarded_ctx(c, [&] {
    // all right-hand sides go through the device together (shared integral formation)
    const int chunk = std::max(1, std::min(nrhs, 32));
    for (int r0 = 0; r0 < nrhs; r0 += chunk) {
      const int nr = std::min(chunk, nrhs - r0);
      if ((int)c->stage_in.size() < nr) {
        c->stage_in.resize(nr);
        c->stage_out.resize(nr);
      }
      std::vector<const void *> xs(nr);
      std::vector<void *> ss(nr);
      for (int q = 0; q < nr; ++q) {
        const int r = r0 + q;
        c->alloc_full(c->stage_in[q]);
        c->alloc_full(c->stage_out[q]);
        to_dev(c, x1 + (size_t)r * c->n1 * 2, c->stage_in[q].p1(), (size_t)c->n1 * 16);
        to_dev(c, x2 + (size_t)r * c->n2 * 2, c->stage_in[q].p2(c->n1), (size_t)c->n2 * 16);
        xs[q] = c->stage_in[q].b.p;
        ss[q] = c->stage_out[q].b.p;
      }
      c->op_batch_full(dir, nr, xs.data(), ss.data());
      for (int q = 0; q < nr; ++q) {
        const int r = r0 + q;
        from_dev(c, c->stage_out[q].p1(), s1 + (size_t)r * c->n1 * 2, (size_t)c->n1 * 16);
        from_dev(c, c->stage_out[q].p2(c->n1), s2 + (size_t)r * c->n2 * 2, (size_t)c->n2 * 16);
      }
    }
    CCLR_CUDA(cudaStreamSynchronize(c->st));
  });
}

cclr_status cc_lr_sigma(cclr_ctx *c, int nrhs, const double *x1, const double *x2, double *s1, double *s2) {
  return sigma_common(c, +1, nrhs, x1, x2, s1, s2);
}

cclr_status cc_lr_sigma_T(cclr_ctx *c, int nrhs, const double *y1, const double *y2, double *s1, double *s2) {
  return sigma_common(c, -1, nrhs, y1, y2, s1, s2);
}

cclr_status cc_lr_sigma_packed(cclr_ctx *c, int nrhs, int transpose, const double *x, double *s) {
  if (!c || nrhs < 0 || (transpose != 0 && transpose != 1) || (nrhs > 0 && (!x || !s)))
    return (cclr_status)fail(CCLR_EINVAL, "bad sigma_packed arguments");
  return (cclr_status)guarded_ctx(c, [&] {
    const int64_t n = c->ntot();
    std::vector<const void *> xs(nrhs);
    std::vector<void *> ss(nrhs);
    for (int r = 0; r < nrhs; ++r) {
      xs[r] = x + (size_t)r * n * 2;
      ss[r] = s + (size_t)r * n * 2;
    }
    // all right-hand sides in one batched product (device pointers of the current device; host
    // arrays are refused: the packed entry point stages nothing)
    for (int r = 0; r < nrhs; ++r) {
      cudaPointerAttributes a{};
      CCLR_CUDA(cudaPointerGetAttributes(&a, xs[r]));
      CCLR_REQUIRE(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged,
                   "cc_lr_sigma_packed needs device arrays");
    }
    if (nrhs > 0) c->op_batch(transpose ? -1 : +1, nrhs, xs.data(), ss.data());
    CCLR_CUDA(cudaStreamSynchronize(c->st));
  });
}

cclr_status cc_lr_xi(cclr_ctx *c, int comp, double *xi1, double *xi2) {
  if (!c || comp < 0 || comp > 2 || !xi1 || !xi2) return (cclr_status)fail(CCLR_EINVAL, "bad xi arguments");
  return (cclr_status)guarded_ctx(c, [&] {
    c->alloc_full(c->fullA);
    const int64_t nn = (int64_t)c->M->n * c->M->n;
    c->M->xi((char *)c->M->mu.p + (size_t)comp * nn * 16, c->M->t1.p, c->M->t2.p, c->fullA.p1(), c->fullA.p2(c->n1));
    from_dev(c, c->fullA.p1(), xi1, (size_t)c->n1 * 16);
    from_dev(c, c->fullA.p2(c->n1), xi2, (size_t)c->n2 * 16);
    CCLR_CUDA(cudaStreamSynchronize(c->st));
  });
}

cclr_status cc_lr_solve_x(cclr_ctx *c, double omega, int comp, double tol, int diis_depth,
                          double *x1, double *x2, cclr_stats *stats) {
  if (!c || comp < 0 || comp > 2 || !x1 || !x2 || !(tol > 0)) return (cclr_status)fail(CCLR_EINVAL, "bad solve_x arguments");
  double rel = 0;
  int st = guarded_ctx(c, [&] {
    auto t0 = std::chrono::steady_clock::now();
    AVec b, x;
    c->alloc_vec(b);
    c->alloc_vec(x);
    c->xi_vec(comp, c->M->t1.p, c->M->t2.p, b.b.p);
    c->scal(zd(-1), b.b.p);
    int its = 0;
    int calls0 = c->sigma_calls;
    rel = c->solve(+1, omega, b.b.p, x.b.p, tol, diis_depth, c->maxit, &its);
    c->alloc_full(c->fullA);
    c->unpack_to(x.b.p, c->fullA.b.p, C128);
    from_dev(c, c->fullA.p1(), x1, (size_t)c->n1 * 16);
    from_dev(c, c->fullA.p2(c->n1), x2, (size_t)c->n2 * 16);
    CCLR_CUDA(cudaStreamSynchronize(c->st));
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      stats->iterations = its;
      stats->refinements = c->refinements;
      stats->sigma_calls = c->sigma_calls - calls0;
      stats->converged = rel < tol;
      stats->max_rel_residual = rel;
      stats->time_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
  });
  if (st != CCLR_OK) return (cclr_status)st;
  return rel < tol ? CCLR_OK : (cclr_status)fail(CCLR_ENOCONV, "solve_x: residual " + std::to_string(rel));
}

cclr_status cc_lr_lambda(cclr_ctx *c, double tol, double *lam1, double *lam2) {
  if (!c || !lam1 || !lam2) return (cclr_status)fail(CCLR_EINVAL, "bad lambda arguments");
  return (cclr_status)guarded_ctx(c, [&] {
    c->ensure_lambda(tol, 8, nullptr);
    c->alloc_full(c->fullA);
    c->unpack_to(c->lam.b.p, c->fullA.b.p, C128);
    from_dev(c, c->fullA.p1(), lam1, (size_t)c->n1 * 16);
    from_dev(c, c->fullA.p2(c->n1), lam2, (size_t)c->n2 * 16);
    CCLR_CUDA(cudaStreamSynchronize(c->st));
  });
}

// Right (X) solves of every component at the shifts in sh, in one block or one by one.
static void solve_right(cclr_ctx *c, int dir, const std::vector<zd> &sh, const std::vector<const void *> &bs,
                        const std::vector<void *> &xs, double tol, int diis_depth, cclr_stats &loc,
                        bool warm = false) {
  if (c->method == 2) {
    // every system of a block keeps its own Krylov basis and six work vectors: the systems go in
    // blocks small enough that each gets a restart length of min(subspace, 20) in the memory left
    const int n = (int)bs.size();
    int g = n;
    while (g > 1 && c->block_restart(g, c->M->lean ? 0.2 : 0.5) < std::min(c->krylov, 20) + 6) g = (g + 1) / 2;
    for (int k0 = 0; k0 < n; k0 += g) {
      const int k1 = std::min(n, k0 + g);
      std::vector<zd> s2(sh.begin() + k0, sh.begin() + k1);
      std::vector<const void *> b2(bs.begin() + k0, bs.begin() + k1);
      std::vector<void *> x2(xs.begin() + k0, xs.begin() + k1);
      std::vector<int> its;
      std::vector<double> rels;
      c->solve_block(dir, s2, b2, x2, tol, c->maxit, its, rels, warm);
      for (size_t k = 0; k < its.size(); ++k) {
        loc.iterations += its[k];
        loc.max_rel_residual = std::max(loc.max_rel_residual, rels[k]);
        if (!(rels[k] < tol)) loc.converged = 0;
      }
    }
    return;
  }
  for (size_t k = 0; k < bs.size(); ++k) {
    int its = 0;
    const double rel = c->solve(dir, sh[k], bs[k], xs[k], tol, diis_depth, c->maxit, &its, warm);
    loc.iterations += its;
    loc.max_rel_residual = std::max(loc.max_rel_residual, rel);
    if (!(rel < tol)) loc.converged = 0;
  }
}

// alpha at z = omega + i gamma for every omega (gamma = 0: the undamped response):
//   g(A,B;w) = eta^A X^B(w) + eta^B X^A(-w) + (F X^A(-w)) X^B(w),
//   <<A;B>>_z = 1/2 [g(A,B;z) + conj g(A,B;-z*)],  alpha = -<<A;B>>,
// so X^C is needed at the shifts z, -z, z*, -z* (two of them when gamma = 0, one at z = 0).
static cclr_status solve_alpha(cclr_ctx *c, int nomega, const double *omegas, double gamma, int ncomp,
                               const int *comps, double tol, int diis_depth, double *alpha, cclr_stats *stats) {
  if (!c || nomega < 1 || !omegas || ncomp < 1 || ncomp > 3 || !comps || !alpha || !(tol > 0) || !(gamma >= 0))
    return (cclr_status)fail(CCLR_EINVAL, "bad solve arguments");
  for (int k = 0; k < ncomp; ++k)
    if (comps[k] < 0 || comps[k] > 2) return (cclr_status)fail(CCLR_EINVAL, "component out of range");
  cclr_stats loc;
  std::memset(&loc, 0, sizeof(loc));
  loc.converged = 1;
  int st = guarded_ctx(c, [&] {
    int calls0 = c->sigma_calls;
    c->ensure_lambda(tol, diis_depth, &loc);
    // the distinct shifts over every frequency (z, -z, z*, -z* of each); slot[w][k] = the index of
    // the shift the k-th of them uses at frequency w
    std::vector<zd> shifts;
    std::vector<std::array<int, 4>> slot(nomega);
    for (int w = 0; w < nomega; ++w) {
      const zd z(omegas[w], gamma);
      const zd want[4] = {z, -z, std::conj(z), -std::conj(z)};
      for (int k = 0; k < 4; ++k) {
        int f = -1;
        for (size_t q = 0; q < shifts.size(); ++q)
          if (shifts[q] == want[k]) f = (int)q;
        if (f < 0) {
          f = (int)shifts.size();
          shifts.push_back(want[k]);
        }
        slot[w][k] = f;
      }
    }
    const int ns = (int)shifts.size();
    std::vector<AVec> X((size_t)ncomp * ns);
    auto t0 = std::chrono::steady_clock::now();
    std::vector<AVec> B(ncomp);
    for (int a = 0; a < ncomp; ++a) {
      c->alloc_vec(B[a]);
      c->xi_vec(comps[a], c->M->t1.p, c->M->t2.p, B[a].b.p);
      c->scal(zd(-1), B[a].b.p);
      for (int q = 0; q < ns; ++q) c->alloc_vec(X[(size_t)a * ns + q]);
    }
    {
      // every component and shift of every frequency: one block (method 2: the operator is applied
      // to all unconverged systems at once) or one solve after another
      std::vector<zd> oms;
      std::vector<const void *> bs;
      std::vector<void *> xs;
      for (int a = 0; a < ncomp; ++a)
        for (int q = 0; q < ns; ++q) {
          oms.push_back(shifts[q]);
          bs.push_back(B[a].b.p);
          xs.push_back(X[(size_t)a * ns + q].b.p);
        }
      solve_right(c, +1, oms, bs, xs, tol, diis_depth, loc);
    }
    auto t1 = std::chrono::steady_clock::now();
    loc.time_solve_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
    // eta^A . X^B at every shift, and F X^A where a frequency needs it (-z for g(z), z* for g(-z*))
    std::vector<zd> ED((size_t)ncomp * ncomp * ns);
    for (int a = 0; a < ncomp; ++a)
      for (int b = 0; b < ncomp; ++b)
        for (int q = 0; q < ns; ++q)
          ED[((size_t)a * ncomp + b) * ns + q] = c->eta_dot(comps[a], X[(size_t)b * ns + q].b.p);
    std::vector<AVec> FX((size_t)ncomp * ns);
    std::vector<char> have((size_t)ncomp * ns, 0);
    auto FXq = [&](int a, int q) -> AVec & {
      const size_t id = (size_t)a * ns + q;
      if (!have[id]) {
        c->alloc_vec(FX[id]);
        c->fx(X[id].b.p, FX[id].b.p);
        have[id] = 1;
      }
      return FX[id];
    };
    for (int w = 0; w < nomega; ++w) {
      auto Xs = [&](int a, int k) -> AVec & { return X[(size_t)a * ns + slot[w][k]]; };
      auto EDs = [&](int a, int b, int k) { return ED[((size_t)a * ncomp + b) * ns + slot[w][k]]; };
      for (int a = 0; a < ncomp; ++a)
        for (int b = 0; b < ncomp; ++b) {
          // k: 0 = z, 1 = -z, 2 = z*, 3 = -z*
          zd gp = EDs(a, b, 0) + EDs(b, a, 1) + c->dot(FXq(a, slot[w][1]).b.p, Xs(b, 0).b.p, 0);
          zd gm = EDs(a, b, 3) + EDs(b, a, 2) + c->dot(FXq(a, slot[w][2]).b.p, Xs(b, 3).b.p, 0);
          zd al = -0.5 * (gp + std::conj(gm));
          size_t k = (((size_t)w * ncomp + a) * ncomp + b) * 2;
          alpha[k] = al.real();
          alpha[k + 1] = al.imag();
        }
    }
    loc.time_alpha_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    loc.sigma_calls = c->sigma_calls - calls0;
    loc.refinements = c->refinements;
    c->release_scratch();
  });
  if (stats) *stats = loc;
  if (st != CCLR_OK) return (cclr_status)st;
  return loc.converged ? CCLR_OK : (cclr_status)fail(CCLR_ENOCONV, "solve: tolerance not met");
}

// alpha by the left-hand route (Sec. 2.2): X^B(w) from (A - w) X = -xi^B, Y^B(w) from
// Y (A + w) = -(eta^B + F X^B(w)), and g(A,B;w) = Y^B(w) . xi^A + eta^A . X^B(w);
// <<A;B>>_w = 1/2 [g(A,B;w) + conj g(A,B;-w)], alpha = -<<A;B>>.  The same X and F X give the
// X-only route g(A,B;w) = eta^A X^B(w) + eta^B X^A(-w) + (F X^A(-w)) X^B(w) with dot products
// only; both routes converge to one alpha, so their largest difference is an a-posteriori
// estimate of the error (*est).  tol_alpha > 0: the solves are tightened (warm-started from the
// previous solutions) until that estimate is below tol_alpha or the residual target reaches
// tol_floor.
static cclr_status solve_alpha_left(cclr_ctx *c, int nomega, const double *omegas, int ncomp, const int *comps,
                                    double tol, int diis_depth, double *alpha, cclr_stats *stats,
                                    double tol_alpha = 0.0, double *est = nullptr) {
  if (!c || nomega < 1 || !omegas || ncomp < 1 || ncomp > 3 || !comps || !alpha || !(tol > 0))
    return (cclr_status)fail(CCLR_EINVAL, "bad solve_left arguments");
  for (int k = 0; k < ncomp; ++k)
    if (comps[k] < 0 || comps[k] > 2) return (cclr_status)fail(CCLR_EINVAL, "component out of range");
  cclr_stats loc;
  std::memset(&loc, 0, sizeof(loc));
  loc.converged = 1;
  double est_all = 0.0;
  bool alpha_met = true;
  int st = guarded_ctx(c, [&] {
    const int calls0 = c->sigma_calls;
    // residual floor of the arithmetic: FP64, or the accurate products of the mixed modes
    const double tol_floor = c->M->prec == CCLR_FP64 || c->hi_prec == CCLR_FP64 ? 1e-12 : 8e-7;
    // Lambda enters both routes alike (the estimate does not see its error): with a tol_alpha
    // target it is solved near the floor
    c->ensure_lambda(tol_alpha > 0.0 ? std::max(1.5 * tol_floor, 1e-10) : tol, diis_depth, &loc);
    std::vector<AVec> XI(ncomp), RB(ncomp);
    for (int a = 0; a < ncomp; ++a) {
      c->alloc_vec(XI[a]);
      c->alloc_vec(RB[a]);
      c->xi_vec(comps[a], c->M->t1.p, c->M->t2.p, XI[a].b.p);
      c->copy(XI[a].b.p, RB[a].b.p);
      c->scal(zd(-1), RB[a].b.p);
    }
    for (int w = 0; w < nomega; ++w) {
      std::vector<zd> shifts{zd(omegas[w])};
      if (omegas[w] != 0.0) shifts.push_back(zd(-omegas[w]));
      const int ns = (int)shifts.size();
      auto slot = [&](int k) { return (k == 1 && ns == 2) ? 1 : 0; };  // k = 0: +w, 1: -w
      std::vector<AVec> X((size_t)ncomp * ns), Y((size_t)ncomp * ns), LB((size_t)ncomp * ns), FXv((size_t)ncomp * ns);
      double tw = tol;
      bool warm = false;
      for (int level = 0;; ++level) {
        auto t0 = std::chrono::steady_clock::now();
        std::vector<zd> sh;
        std::vector<const void *> bs;
        std::vector<void *> xs;
        for (int b = 0; b < ncomp; ++b)
          for (int q = 0; q < ns; ++q) {
            c->alloc_vec(X[(size_t)b * ns + q]);
            sh.push_back(shifts[q]);
            bs.push_back(RB[b].b.p);
            xs.push_back(X[(size_t)b * ns + q].b.p);
          }
        cclr_stats lvl;
        std::memset(&lvl, 0, sizeof(lvl));
        lvl.converged = 1;
        solve_right(c, +1, sh, bs, xs, tw, diis_depth, lvl, warm);
        auto t1 = std::chrono::steady_clock::now();
        // F X^B(s), and the left right-hand sides -(eta^B + F X^B(s)); Y^B(s) with the shift -s
        std::vector<zd> lsh;
        std::vector<const void *> lbs;
        std::vector<void *> ys;
        for (int b = 0; b < ncomp; ++b)
          for (int q = 0; q < ns; ++q) {
            const size_t id = (size_t)b * ns + q;
            c->alloc_vec(FXv[id]);
            c->fx(X[id].b.p, FXv[id].b.p);
            c->alloc_vec(LB[id]);
            c->copy(FXv[id].b.p, LB[id].b.p);
            c->axpy(zd(1), c->eta_vec(comps[b]), LB[id].b.p);
            c->scal(zd(-1), LB[id].b.p);
            c->alloc_vec(Y[id]);
            lsh.push_back(-shifts[q]);
            lbs.push_back(LB[id].b.p);
            ys.push_back(Y[id].b.p);
          }
        auto t2 = std::chrono::steady_clock::now();
        solve_right(c, -1, lsh, lbs, ys, tw, diis_depth, lvl, warm);
        auto t3 = std::chrono::steady_clock::now();
        double e = 0.0;
        for (int a = 0; a < ncomp; ++a)
          for (int b = 0; b < ncomp; ++b) {
            // k = 0: +w, 1: -w
            auto gL = [&](int k) {
              const size_t id = (size_t)b * ns + slot(k);
              return c->dot(Y[id].b.p, XI[a].b.p, 0) + c->eta_dot(comps[a], X[id].b.p);
            };
            auto gR = [&](int k) {
              const size_t xb = (size_t)b * ns + slot(k), xa = (size_t)a * ns + slot(1 - k);
              return c->eta_dot(comps[a], X[xb].b.p) + c->eta_dot(comps[b], X[xa].b.p) +
                     c->dot(FXv[xa].b.p, X[xb].b.p, 0);
            };
            const zd al = -0.5 * (gL(0) + std::conj(gL(1)));
            const zd ar = -0.5 * (gR(0) + std::conj(gR(1)));
            e = std::max(e, std::abs(al - ar));
            const size_t k = (((size_t)w * ncomp + a) * ncomp + b) * 2;
            alpha[k] = al.real();
            alpha[k + 1] = al.imag();
          }
        auto t4 = std::chrono::steady_clock::now();
        loc.iterations += lvl.iterations;
        loc.time_solve_ms += std::chrono::duration<double, std::milli>((t1 - t0) + (t3 - t2)).count();
        loc.time_alpha_ms += std::chrono::duration<double, std::milli>((t2 - t1) + (t4 - t3)).count();
        if (cclr_ctx::verbose()) std::fprintf(stderr, "cclr alpha level %d tol %.2e estimate %.3e\n", level, tw, e);
        const bool last = tol_alpha <= 0.0 || e < tol_alpha || tw <= tol_floor || level >= 8;
        if (last) {
          loc.max_rel_residual = std::max(loc.max_rel_residual, lvl.max_rel_residual);
          if (!lvl.converged) loc.converged = 0;
          est_all = std::max(est_all, e);
          if (tol_alpha > 0.0 && !(e < tol_alpha)) alpha_met = false;
          break;
        }
        // tighten by the estimate's distance from the target (first-order error in the residual)
        tw = std::max(tol_floor, tw * std::min(0.3, std::max(0.01, 0.3 * tol_alpha / e)));
        warm = true;
      }
    }
    loc.sigma_calls = c->sigma_calls - calls0;
    loc.refinements = c->refinements;
    c->release_scratch();
  });
  if (stats) *stats = loc;
  if (est) *est = est_all;
  if (st != CCLR_OK) return (cclr_status)st;
  if (!alpha_met) return (cclr_status)fail(CCLR_ENOCONV, "solve_alpha_tol: estimate " + std::to_string(est_all) + " above tol_alpha");
  return loc.converged || tol_alpha > 0.0 ? CCLR_OK : (cclr_status)fail(CCLR_ENOCONV, "solve_left: tolerance not met");
}

cclr_status cc_lr_solve_left(cclr_ctx *c, int nomega, const double *omegas, int ncomp, const int *comps,
                             double tol, int diis_depth, double *alpha, cclr_stats *stats) {
  return solve_alpha_left(c, nomega, omegas, ncomp, comps, tol, diis_depth, alpha, stats);
}

cclr_status cc_lr_solve_alpha_tol(cclr_ctx *c, int nomega, const double *omegas, int ncomp, const int *comps,
                                  double tol_alpha, int diis_depth, double *alpha, double *alpha_err,
                                  cclr_stats *stats) {
  if (!(tol_alpha > 0) || !alpha_err) return (cclr_status)fail(CCLR_EINVAL, "tol_alpha must be > 0 and alpha_err given");
  // the first residual target: loose (the estimate drives it down from there)
  return solve_alpha_left(c, nomega, omegas, ncomp, comps, 1e-4, diis_depth, alpha, stats, tol_alpha, alpha_err);
}

cclr_status cc_lr_eta(cclr_ctx *c, int comp, double tol, double *eta1, double *eta2) {
  if (!c || comp < 0 || comp > 2 || !eta1 || !eta2 || !(tol > 0)) return (cclr_status)fail(CCLR_EINVAL, "bad eta arguments");
  return (cclr_status)guarded_ctx(c, [&] {
    c->ensure_lambda(tol, 8, nullptr);
    c->alloc_full(c->fullA);
    c->unpack_to(c->eta_vec(comp), c->fullA.b.p, C128);
    from_dev(c, c->fullA.p1(), eta1, (size_t)c->n1 * 16);
    from_dev(c, c->fullA.p2(c->n1), eta2, (size_t)c->n2 * 16);
    CCLR_CUDA(cudaStreamSynchronize(c->st));
  });
}

cclr_status cc_lr_solve(cclr_ctx *c, int nomega, const double *omegas, int ncomp, const int *comps,
                        double tol, int diis_depth, double *alpha, cclr_stats *stats) {
  return solve_alpha(c, nomega, omegas, 0.0, ncomp, comps, tol, diis_depth, alpha, stats);
}

cclr_status cc_lr_solve_damped(cclr_ctx *c, int nomega, const double *omegas, double gamma, int ncomp,
                               const int *comps, double tol, int diis_depth, double *alpha, cclr_stats *stats) {
  return solve_alpha(c, nomega, omegas, gamma, ncomp, comps, tol, diis_depth, alpha, stats);
}

cclr_status cc_lr_ccsd_residual(cclr_ctx *c, int prec, const double *t1, const double *t2, double *r1,
                                double *r2, double *energy) {
  if (!c || !t1 || !t2 || !r1 || !r2) return (cclr_status)fail(CCLR_EINVAL, "bad ccsd_residual arguments");
  return (cclr_status)guarded_ctx(c, [&] {
    const int p = c->gs_prec(prec);
    c->alloc_full(c->fullB);
    AVec tv, rv;
    c->alloc_vec(tv);
    c->alloc_vec(rv);
    to_dev(c, t1, c->fullB.p1(), (size_t)c->n1 * 16);
    to_dev(c, t2, c->fullB.p2(c->n1), (size_t)c->n2 * 16);
    c->pack_from(c->fullB.b.p, C128, tv.b.p);
    c->ccsd_residual(p, tv.b.p, rv.b.p);
    if (energy) {
      const zd e = c->ccsd_energy(tv.b.p);
      energy[0] = e.real();
      energy[1] = e.imag();
    }
    c->unpack_to(rv.b.p, c->fullA.b.p, C128);
    from_dev(c, c->fullA.p1(), r1, (size_t)c->n1 * 16);
    from_dev(c, c->fullA.p2(c->n1), r2, (size_t)c->n2 * 16);
    CCLR_CUDA(cudaStreamSynchronize(c->st));
    c->M->release_set(c->gs);
    if (c->M->lean) c->release_scratch();
  });
}

cclr_status cc_lr_ccsd(cclr_ctx *c, int prec, double tol, int max_iterations, int diis_depth, double *energy,
                       double *res_norm, int *iterations) {
  if (!c || !(tol > 0.0) || max_iterations < 1) return (cclr_status)fail(CCLR_EINVAL, "bad ccsd arguments");
  bool conv = false;
  int st = guarded_ctx(c, [&] {
    const int p = c->gs_prec(prec);
    AVec tv;
    int its = 0;
    const double rn = c->ccsd_solve(p, tol, max_iterations, diis_depth, tv, &its);
    conv = rn < tol;
    c->set_amplitudes(tv.b.p);
    if (energy) {
      const zd e = c->ccsd_energy(tv.b.p);
      energy[0] = e.real();
      energy[1] = e.imag();
    }
    if (res_norm) *res_norm = rn;
    if (iterations) *iterations = its;
    if (c->M->lean) c->release_scratch();
  });
  if (st == CCLR_OK && !conv) return (cclr_status)fail(CCLR_ENOCONV, "ground-state CCSD did not reach the tolerance");
  return (cclr_status)st;
}

cclr_status cc_lr_get_t(cclr_ctx *c, double *t1, double *t2) {
  if (!c || !t1 || !t2) return (cclr_status)fail(CCLR_EINVAL, "bad get_t arguments");
  return (cclr_status)guarded_ctx(c, [&] {
    from_dev(c, c->M->t1.p, t1, (size_t)c->n1 * 16);
    from_dev(c, c->M->t2.p, t2, (size_t)c->n2 * 16);
    CCLR_CUDA(cudaStreamSynchronize(c->st));
  });
}

cclr_status cc_lr_set_precision(cclr_ctx *c, int prec) {
  if (!c || prec < 0 || prec > 4) return (cclr_status)fail(CCLR_EINVAL, "bad precision");
  return (cclr_status)guarded_ctx(c, [&] {
    c->M->prec = prec;
    if (prec != CCLR_FP64) c->M->cst_for(prec);
  });
}

cclr_status cc_lr_set_graphs(cclr_ctx *c, int on) {
  if (!c || (on != 0 && on != 1)) return (cclr_status)fail(CCLR_EINVAL, "graphs must be 0 or 1");
  if (on && (c->st == nullptr || c->st == cudaStreamLegacy || c->st == cudaStreamPerThread))
    return (cclr_status)fail(CCLR_EUNSUPPORTED, "CUDA graphs need a context created with its own (non-default) stream");
  return (cclr_status)guarded_ctx(c, [&] {
    CCLR_CUDA(cudaStreamSynchronize(c->st));
    c->M->graphs = on != 0;
    if (!on) c->M->clear_graphs();
  });
}

cclr_status cc_lr_graph_stats(cclr_ctx *c, int *captures, int *launches) {
  if (!c || !captures || !launches) return (cclr_status)fail(CCLR_EINVAL, "bad graph_stats arguments");
  *captures = c->M->graph_captures;
  *launches = c->M->graph_launches;
  return CCLR_OK;
}

cclr_status cc_lr_ladder_tuning(cclr_ctx *c, int prec, int *group_size, int cap, int *cand, double *ms, int *n) {
  if (!c || (prec != CCLR_C64_TF32 && prec != CCLR_C64_3XTF32 && prec != CCLR_BF16X3) || !group_size || !n || cap < 0 ||
      (cap > 0 && (!cand || !ms)))
    return (cclr_status)fail(CCLR_EINVAL, "bad ladder_tuning arguments");
  const LadderTC &l = c->M->ltc[prec == CCLR_C64_3XTF32 ? 1 : prec == CCLR_BF16X3 ? 2 : 0];
  *group_size = l.group_size();
  *n = (int)l.tune_log.size();
  for (int k = 0; k < cap && k < *n; ++k) {
    cand[k] = l.tune_log[k].first;
    ms[k] = l.tune_log[k].second;
  }
  return CCLR_OK;
}

cclr_status cc_lr_set_ladder_storage(cclr_ctx *c, int store) {
  if (!c || (store != 0 && store != 1)) return (cclr_status)fail(CCLR_EINVAL, "ladder storage must be 0 or 1");
  return (cclr_status)guarded_ctx(c, [&] {
    CCLR_CUDA(cudaStreamSynchronize(c->st));
    for (auto &l : c->M->ltc) l.set_store(store != 0);
  });
}

cclr_status cc_lr_set_refinement(cclr_ctx *c, int prec) {
  if (!c || (prec != CCLR_FP64 && prec != CCLR_C64_3XTF32))
    return (cclr_status)fail(CCLR_EINVAL, "refinement precision must be CCLR_FP64 or CCLR_C64_3XTF32");
  return (cclr_status)guarded_ctx(c, [&] {
    CCLR_CUDA(cudaStreamSynchronize(c->st));
    c->hi_prec = prec;
    if (prec != CCLR_FP64) {
      c->M->cst_for(prec);
      if (c->M->prec != CCLR_FP64) {
        c->M->oovv_packed();  // formed from the complex128 set while it exists
        // no FP64 product remains in this configuration: its set and buffers are freed (an FP64
        // product requested later rebuilds them; in a budgeted context the FP64 inputs go too,
        // and FP64 products are refused afterwards)
        c->M->release_fp64();
        c->xfs[C128].clear();
        c->sfs[C128].clear();
        c->M->release_set(c->shift);
        if (c->M->lean) c->M->release_fp64_inputs();
      }
    }
  });
}

cclr_status cc_lr_set_solver(cclr_ctx *c, int method, int subspace, int max_iterations) {
  if (!c || method < 0 || method > 2 || subspace < 0 || subspace > 100 || max_iterations < 0)
    return (cclr_status)fail(CCLR_EINVAL, "bad solver arguments");
  c->method = method;
  if (subspace >= 2) c->krylov = subspace;
  if (max_iterations > 0) c->maxit = max_iterations;
  return CCLR_OK;
}

cclr_status cc_lr_set_autotune(cclr_ctx *c, int on) {
  if (!c || (on != 0 && on != 1)) return (cclr_status)fail(CCLR_EINVAL, "autotune must be 0 or 1");
  c->M->autotune = on != 0;
  return CCLR_OK;
}

cclr_status cc_lr_gemm_tuning(cclr_ctx *c, int cap, int *n, double *rec) {
  if (!c || !n || cap < 0 || (cap > 0 && !rec)) return (cclr_status)fail(CCLR_EINVAL, "bad gemm_tuning arguments");
  return (cclr_status)guarded_ctx(c, [&] { *n = tc_tuning_table(cap, rec); });
}

cclr_status cc_lr_memory(cclr_ctx *c, size_t *in_use, size_t *peak, size_t *budget) {
  if (!c || !in_use || !peak || !budget) return (cclr_status)fail(CCLR_EINVAL, "bad memory arguments");
  *in_use = c->acct.used;
  *peak = c->acct.peak;
  *budget = c->acct.budget;
  return CCLR_OK;
}

cclr_status cc_lr_last_timings(cclr_ctx *c, double *ms, int n) {
  if (!c || !ms || n < 0) return (cclr_status)fail(CCLR_EINVAL, "bad timings arguments");
  for (int k = 0; k < n && k < 4; ++k) ms[k] = c->M->ms_last[k];
  if (n > 4) ms[4] = c->last_products;
  return CCLR_OK;
}

void cc_lr_free(cclr_ctx *c) {
  if (!c) return;
  try {
    if (c->st) cudaStreamSynchronize(c->st);
  } catch (...) {
  }
  delete c;
}

const char *cc_lr_strerror(cclr_status s) {
  switch (s) {
    case CCLR_OK: return "success";
    case CCLR_EINVAL: return "invalid argument";
    case CCLR_ENOMEM: return "out of device memory or HBM budget exceeded";
    case CCLR_ENOCONV: return "solver did not converge";
    case CCLR_EDEVICE: return "CUDA device error";
    case CCLR_ETIMEOUT: return "bounded device wait timed out";
    case CCLR_EUNSUPPORTED: return "unsupported on this device or build";
  }
  return "unknown status";
}

const char *cc_lr_last_error(void) { return g_last_error.c_str(); }

unsigned long long cc_lr_launch_count(void) { return cclr::launch_count(); }

int cc_lr_selftest_precond(int n, double omega, double omega_im, unsigned seed, double *max_rel_err) {
  if (n < 1 || n > (1 << 26) || !max_rel_err) return fail(CCLR_EINVAL, "bad selftest_precond arguments");
  return guarded([&] {
    std::mt19937_64 g(seed);
    std::uniform_real_distribution<double> ud(0.1, 20.0);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<double> D(n), r(2 * (size_t)n), out(2 * (size_t)n);
    for (auto &d : D) d = ud(g);
    for (auto &x : r) x = nd(g);
    cudaStream_t st;
    CCLR_CUDA(cudaStreamCreate(&st));
    DevBuf Dd((size_t)n * 8), rd((size_t)n * 16), od((size_t)n * 16);
    CCLR_CUDA(cudaMemcpyAsync(Dd.p, D.data(), Dd.bytes, cudaMemcpyHostToDevice, st));
    CCLR_CUDA(cudaMemcpyAsync(rd.p, r.data(), rd.bytes, cudaMemcpyHostToDevice, st));
    vec_precond(C128, n, Dd.as<double>(), omega, omega_im, rd.p, od.p, st);
    CCLR_CUDA(cudaMemcpyAsync(out.data(), od.p, od.bytes, cudaMemcpyDeviceToHost, st));
    CCLR_CUDA(cudaStreamSynchronize(st));
    CCLR_CUDA(cudaStreamDestroy(st));
    double mx = 0.0;
    for (int i = 0; i < n; ++i) {
      const std::complex<double> ref = std::complex<double>(r[2 * i], r[2 * i + 1]) /
                                       std::complex<double>(D[i] - omega, -omega_im);
      const std::complex<double> got(out[2 * i], out[2 * i + 1]);
      if (std::abs(ref) > 0) mx = std::max(mx, std::abs(got - ref) / std::abs(ref));
    }
    *max_rel_err = mx;
  });
}

int cc_lr_selftest_timeout(int timeout_us, int *flag) {
  if (timeout_us < 1 || timeout_us > 10000000 || !flag) return fail(CCLR_EINVAL, "bad selftest_timeout arguments");
  int st = guarded([&] {
    cudaStream_t s;
    CCLR_CUDA(cudaStreamCreate(&s));
    *flag = tc_selftest_timeout(timeout_us, s);
    CCLR_CUDA(cudaStreamDestroy(s));
  });
  if (st != CCLR_OK) return st;
  return *flag ? fail(CCLR_ETIMEOUT, "bounded device wait gave up (self-test)") : CCLR_OK;
}

int cc_lr_bench_gemm(int M, int N, int K, int mode, int reps, double *ms) {
  if (M < 1 || N < 1 || K < 1 || mode < 1 || mode > 3 || reps < 1 || !ms) return fail(CCLR_EINVAL, "bad bench_gemm arguments");
  return guarded([&] {
    cudaStream_t st;
    CCLR_CUDA(cudaStreamCreate(&st));
    const int seg = mode == 1 ? 1 : 3, kind = mode == 3 ? TC_BF16 : TC_TF32;
    const int64_t ld = 2 * tc_kpad(K) * seg, es = tc_esize(kind);
    DevBuf A((size_t)M * ld * es), B((size_t)2 * N * ld * es), C((size_t)M * N * 8);
    // deterministic small values (exact content is irrelevant for timing)
    CCLR_CUDA(cudaMemsetAsync(A.p, 0, A.bytes, st));
    CCLR_CUDA(cudaMemsetAsync(B.p, 0, B.bytes, st));
    CCLR_CUDA(cudaMemsetAsync(C.p, 0, C.bytes, st));
    cudaEvent_t e0, e1;
    CCLR_CUDA(cudaEventCreate(&e0));
    CCLR_CUDA(cudaEventCreate(&e1));
    tc_gemm_seg(A.p, ld, B.p, ld, M, 2 * N, 2 * tc_kpad(K), seg, kind, C.as<float>(), 2 * N, zc(1), false, st);
    CCLR_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r)
      tc_gemm_seg(A.p, ld, B.p, ld, M, 2 * N, 2 * tc_kpad(K), seg, kind, C.as<float>(), 2 * N, zc(1), false, st);
    CCLR_CUDA(cudaEventRecord(e1, st));
    CCLR_CUDA(cudaEventSynchronize(e1));
    float t = 0;
    CCLR_CUDA(cudaEventElapsedTime(&t, e0, e1));
    ms[0] = t / reps;
    ms[1] = 8.0 * M * (double)N * K / (ms[0] * 1e-3) / 1e12;
    if (tc_error(st)) throw Error(CCLR_ETIMEOUT, "tensor-core kernel gave up on a bounded wait");
    CCLR_CUDA(cudaEventDestroy(e0));
    CCLR_CUDA(cudaEventDestroy(e1));
    CCLR_CUDA(cudaStreamDestroy(st));
  });
}

int cc_lr_bench_hbm(int o, int v, int reps, double *out, int n) {
  if (o < 2 || v < 2 || reps < 1 || !out || n < 0) return fail(CCLR_EINVAL, "bad bench_hbm arguments");
  return guarded([&] {
    cudaStream_t st;
    CCLR_CUDA(cudaStreamCreate(&st));
    const int64_t nf = (int64_t)o * o * v * v, n1 = (int64_t)o * v;
    const int64_t np = (int64_t)o * (o - 1) / 2 * ((int64_t)v * (v - 1) / 2), nt = n1 + np;
    DevBuf S((size_t)nf * 8), R1((size_t)nf * 8), R2((size_t)nf * 8), R3((size_t)nf * 8);
    DevBuf P((size_t)nt * 16), Q((size_t)nt * 16), D((size_t)nt * 8), dots(sizeof(double2) * 576);
    for (DevBuf *b : {&S, &R1, &R2, &R3, &P, &Q, &D, &dots}) CCLR_CUDA(cudaMemsetAsync(b->p, 0, b->bytes, st));
    double2 *part = dots.as<double2>(), *res = part + 512;
    cudaEvent_t e0, e1;
    CCLR_CUDA(cudaEventCreate(&e0));
    CCLR_CUDA(cudaEventCreate(&e1));
    auto timeit = [&](auto &&fn) {
      fn();
      CCLR_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < reps; ++r) fn();
      CCLR_CUDA(cudaEventRecord(e1, st));
      CCLR_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      CCLR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return (double)ms / reps;
    };
    double res_[16];
    res_[0] = timeit([&] { antisym_apply(C64, o, v, +1, S.p, R1.p, R2.p, R3.p, st); });
    res_[1] = 5.0 * nf * 8;
    res_[2] = timeit([&] { antisym_project(C64, o, v, S.p, st); });
    res_[3] = 2.0 * nf * 8;
    res_[4] = timeit([&] { unpack_doubles(C128, C64, o, v, P.p, S.p, zc(1), false, st); });
    res_[5] = 16.0 * np + 8.0 * nf;
    res_[6] = timeit([&] { pack_doubles(C64, C128, o, v, S.p, P.p, st); });
    res_[7] = 8.0 * np + 16.0 * np;
    res_[8] = timeit([&] { vec_precond(C128, nt, D.as<double>(), 0.0, 0.0, P.p, Q.p, st); });
    res_[9] = 40.0 * nt;
    res_[10] = timeit([&] { vec_dot(C128, nt, P.p, Q.p, 1, part, res, 0, st); });
    res_[11] = 32.0 * nt;
    res_[12] = timeit([&] { vec_axpy(C128, nt, zc(0.5), P.p, Q.p, st); });
    res_[13] = 48.0 * nt;
    res_[14] = timeit([&] { ladder_unpack_sig_bench(o, v, R1.p, S.p, st); });
    res_[15] = 8.0 * np + 4 * 2 * 8.0 * np;
    for (int k = 0; k < 2 * std::min(n, 8); ++k) out[k] = res_[k];
    CCLR_CUDA(cudaEventDestroy(e0));
    CCLR_CUDA(cudaEventDestroy(e1));
    CCLR_CUDA(cudaStreamDestroy(st));
  });
}

int cc_lr_selftest_gemm(int M, int N, int K, int mode, unsigned seed, double *err) {
  if (M < 1 || N < 1 || K < 1 || mode < 1 || mode > 3 || !err) return fail(CCLR_EINVAL, "bad selftest arguments");
  return guarded([&] {
    std::mt19937_64 g(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<double> a((size_t)2 * M * K), b((size_t)2 * K * N);
    for (auto &x : a) x = nd(g);
    for (auto &x : b) x = nd(g);
    Engine E;
    CCLR_CUDA(cudaStreamCreate(&E.st));
    DevBuf A128((size_t)M * K * 16), B128((size_t)K * N * 16), C128b((size_t)M * N * 16);
    DevBuf A64((size_t)M * K * 8), B64((size_t)K * N * 8), Ct((size_t)M * N * 8), Cs((size_t)M * N * 8);
    CCLR_CUDA(cudaMemcpy(A128.p, a.data(), a.size() * 8, cudaMemcpyHostToDevice));
    CCLR_CUDA(cudaMemcpy(B128.p, b.data(), b.size() * 8, cudaMemcpyHostToDevice));
    Tens a128 = make_tens(A128.p, C128, {M, K}), b128 = make_tens(B128.p, C128, {K, N});
    Tens a64 = make_tens(A64.p, C64, {M, K}), b64 = make_tens(B64.p, C64, {K, N});
    Tens c128 = make_tens(C128b.p, C128, {M, N}), ct = make_tens(Ct.p, C64, {M, N}), cs = make_tens(Cs.p, C64, {M, N});
    E.permute(zc(1), a128, "mk", a64, "mk", false);
    E.permute(zc(1), b128, "kn", b64, "kn", false);
    E.zero(c128); E.zero(ct); E.zero(cs);
    E.contract(zc(1), a128, "mk", b128, "kn", c128, "mn");
    E.tc_mode = mode;
    E.tc_force = true;
    E.contract(zc(1), a64, "mk", b64, "kn", ct, "mn");
    E.tc_force = false;
    const bool used_tc = E.tc_calls > 0;
    E.tc_mode = 0;
    E.contract(zc(1), a64, "mk", b64, "kn", cs, "mn");
    CCLR_CUDA(cudaStreamSynchronize(E.st));
    if (tc_error(E.st)) throw Error(CCLR_ETIMEOUT, "tensor-core kernel gave up on a bounded wait");
    std::vector<double> r((size_t)2 * M * N);
    std::vector<float> t((size_t)2 * M * N), q((size_t)2 * M * N);
    CCLR_CUDA(cudaMemcpy(r.data(), C128b.p, r.size() * 8, cudaMemcpyDeviceToHost));
    CCLR_CUDA(cudaMemcpy(t.data(), Ct.p, t.size() * 4, cudaMemcpyDeviceToHost));
    CCLR_CUDA(cudaMemcpy(q.data(), Cs.p, q.size() * 4, cudaMemcpyDeviceToHost));
    double mx = 0, e1 = 0, e2 = 0;
    for (size_t i = 0; i < r.size(); ++i) {
      mx = std::max(mx, std::abs(r[i]));
      e1 = std::max(e1, std::abs(r[i] - (double)t[i]));
      e2 = std::max(e2, std::abs(r[i] - (double)q[i]));
    }
    err[0] = used_tc ? e1 / mx : -1.0;
    err[1] = e2 / mx;
    CCLR_CUDA(cudaStreamDestroy(E.st));
  });
}

}  // extern "C"
