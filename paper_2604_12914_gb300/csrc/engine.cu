// Contraction engine: classifies the modes of C += A*B into batch / M / N / K groups,
// views each operand as a strided batched matrix when its modes merge, and permutes it
// into a contiguous scratch layout otherwise.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <cstdio>
#include <cstdlib>

#include "engine.cuh"
#include "tc_gemm.cuh"

namespace cclr {

static std::atomic<size_t> g_bytes_in_use{0};

size_t device_bytes_in_use() { return g_bytes_in_use.load(); }

static std::atomic<unsigned long long> g_epoch{1};
unsigned long long state_epoch() { return g_epoch.load(); }
void bump_state_epoch() { ++g_epoch; }

MemAcct *&current_acct() {
  static thread_local MemAcct *a = nullptr;
  return a;
}

void DevBuf::alloc(size_t b) {
  release();
  if (b == 0) return;
  MemAcct *a = current_acct();
  if (a && a->budget && a->used + b > a->budget)
    throw Error(2, "HBM budget of " + std::to_string(a->budget) + " bytes exceeded: " + std::to_string(a->used) +
                       " bytes held, " + std::to_string(b) + " more requested");
  cudaError_t e = cudaMalloc(&p, b);
  if (e != cudaSuccess) {
    p = nullptr;
    (void)cudaGetLastError();
    throw Error(2, "cudaMalloc of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
  }
  bytes = b;
  acct = a;
  if (a) {
    a->used += b;
    a->peak = std::max(a->peak, a->used);
  }
  g_bytes_in_use += b;
}

void DevBuf::release() {
  if (p) {
    ++g_epoch;
    cudaFree(p);
    g_bytes_in_use -= bytes;
    if (acct) acct->used -= bytes;
  }
  p = nullptr;
  bytes = 0;
  acct = nullptr;
}

void *Engine::ws(int slot, size_t bytes) {
  if ((int)slots_.size() <= slot) slots_.resize(slot + 1);
  if (slots_[slot].bytes < bytes) {
    if (slots_[slot].p) CCLR_CUDA(cudaStreamSynchronize(st));
    slots_[slot].alloc(bytes + bytes / 8);
  }
  return slots_[slot].p;
}

double2 *Engine::dot_scratch() {
  if (!dots_.p) dots_.alloc(sizeof(double2) * (512 + 64));
  return dots_.as<double2>();
}
double2 *Engine::dot_results() { return dot_scratch() + 512; }

static int mode_pos(const std::string &m, char c) {
  auto k = m.find(c);
  return k == std::string::npos ? -1 : (int)k;
}

// View the modes `group` (outer to inner) of tensor t as one index with a single stride.
static bool group_view(const Tens &t, const std::string &modes, const std::string &group,
                       int64_t &size, int64_t &stride) {
  size = 1;
  stride = 0;
  int64_t expect = -1;
  for (int g = (int)group.size() - 1; g >= 0; --g) {
    int pos = mode_pos(modes, group[g]);
    int64_t d = t.dim[pos], s = t.str[pos];
    if (d == 1) continue;
    if (expect < 0) stride = s;
    else if (s != expect) return false;
    expect = s * d;
    size *= d;
  }
  return true;
}

// The same with up to two levels: index = outer * v.sout + inner * v.sin, inner < v.din.
static bool group_view2(const Tens &t, const std::string &modes, const std::string &group, View2 &v) {
  v = View2();
  int64_t expect = -1, size = 1;
  int levels = 0;
  for (int g = (int)group.size() - 1; g >= 0; --g) {
    int pos = mode_pos(modes, group[g]);
    int64_t d = t.dim[pos], s = t.str[pos];
    if (d == 1) continue;
    if (expect < 0) {
      v.sin = s;
      levels = 1;
    } else if (s != expect) {
      if (levels == 2) return false;
      v.din = size;
      v.sout = s;
      levels = 2;
    }
    expect = s * d;
    size *= d;
  }
  return true;
}

static int64_t prod_dims(const Tens &t, const std::string &modes, const std::string &group) {
  int64_t p = 1;
  for (char c : group) p *= t.dim[mode_pos(modes, c)];
  return p;
}

static Tens contiguous_like(void *p, int dt, const Tens &src, const std::string &smodes,
                            const std::string &order) {
  Tens t;
  t.p = p;
  t.dt = dt;
  t.rank = (int)order.size();
  for (int i = 0; i < t.rank; ++i) t.dim[i] = src.dim[mode_pos(smodes, order[i])];
  int64_t s = 1;
  for (int i = t.rank - 1; i >= 0; --i) {
    t.str[i] = s;
    s *= t.dim[i];
  }
  return t;
}

// CCLR_TRACE=1 prints one line per contraction (modes, sizes, path) to stderr.
static bool trace_on() {
  static const bool t = std::getenv("CCLR_TRACE") && std::getenv("CCLR_TRACE")[0] == '1';
  return t;
}

static std::string vstr(const View2 &v) {
  if (v.din == TC_ONE_LEVEL) return std::to_string(v.sin);
  return std::to_string(v.sout) + "/" + std::to_string(v.din) + "x" + std::to_string(v.sin);
}

void Engine::permute(zc alpha, const Tens &in, const std::string &mi, const Tens &out,
                     const std::string &mo, bool acc) {
  CCLR_REQUIRE((int)mi.size() == in.rank && (int)mo.size() == out.rank && in.rank == out.rank,
               "permute: rank / mode mismatch " + mi + " -> " + mo);
  PermArgs a;
  a.in = in.p;
  a.out = out.p;
  a.alr = alpha.re;
  a.ali = alpha.im;
  a.acc = acc ? 1 : 0;
  // drop unit modes, keep output order
  int r = 0;
  a.total = 1;
  for (int d = 0; d < out.rank; ++d) {
    int pi = mode_pos(mi, mo[d]);
    CCLR_REQUIRE(pi >= 0, "permute: mode missing in input");
    CCLR_REQUIRE(in.dim[pi] == out.dim[d], "permute: dimension mismatch for mode " + std::string(1, mo[d]));
    if (out.dim[d] == 1) continue;
    a.dim[r] = out.dim[d];
    a.sout[r] = out.str[d];
    a.sin[r] = in.str[pi];
    a.total *= out.dim[d];
    ++r;
  }
  a.rank = r;
  if (r == 0) {  // scalar
    a.rank = 1;
    a.dim[0] = 1;
    a.sin[0] = a.sout[0] = 0;
  }
  for (int d = 0; d < out.rank; ++d)
    if (out.dim[d] == 0) a.total = 0;
  launch_permute(a, in.dt, out.dt, st);
}

void Engine::zero(const Tens &t) {
  CCLR_REQUIRE(t.contiguous(), "zero: tensor is not contiguous");
  if (t.numel() > 0) CCLR_CUDA(cudaMemsetAsync(t.p, 0, t.numel() * dt_size(t.dt), st));
}

void Engine::contract(zc alpha, const Tens &A, const std::string &ma, const Tens &B,
                      const std::string &mb, const Tens &C, const std::string &mc) {
  CCLR_REQUIRE((int)ma.size() == A.rank && (int)mb.size() == B.rank && (int)mc.size() == C.rank,
               "contract: rank / mode mismatch " + ma + "," + mb + "->" + mc);
  CCLR_REQUIRE(A.dt == B.dt && B.dt == C.dt, "contract: dtype mismatch");
  const int dt = C.dt;
  std::string bat, Mm, Nm, Km;
  for (char c : mc) {
    int pa = mode_pos(ma, c), pb = mode_pos(mb, c);
    CCLR_REQUIRE(pa >= 0 || pb >= 0, std::string("contract: output mode only in C: ") + c);
    if (pa >= 0 && pb >= 0) bat += c;
    else if (pa >= 0) Mm += c;
    else Nm += c;
  }
  for (char c : ma) {
    if (mode_pos(mc, c) >= 0) continue;
    CCLR_REQUIRE(mode_pos(mb, c) >= 0, std::string("contract: mode only in A: ") + c);
    Km += c;
  }
  for (char c : mb)
    CCLR_REQUIRE(mode_pos(mc, c) >= 0 || mode_pos(ma, c) >= 0, std::string("contract: mode only in B: ") + c);
  for (char c : ma) {
    int pb = mode_pos(mb, c), pc = mode_pos(mc, c), pa = mode_pos(ma, c);
    if (pb >= 0) CCLR_REQUIRE(A.dim[pa] == B.dim[pb], std::string("contract: dim mismatch A/B for ") + c);
    if (pc >= 0) CCLR_REQUIRE(A.dim[pa] == C.dim[pc], std::string("contract: dim mismatch A/C for ") + c);
  }
  for (char c : mb) {
    int pc = mode_pos(mc, c), pb = mode_pos(mb, c);
    if (pc >= 0) CCLR_REQUIRE(B.dim[pb] == C.dim[pc], std::string("contract: dim mismatch B/C for ") + c);
  }
  const int64_t nb = prod_dims(C, mc, bat), M = prod_dims(C, mc, Mm), N = prod_dims(C, mc, Nm);
  const int64_t K = prod_dims(A, ma, Km);
  if (nb == 0 || M == 0 || N == 0) return;
  if (K == 0) return;
  const size_t es = dt_size(dt);

  // An o x o (at most 64 x 64) matrix acting on one index of a large tensor, X[p][k][q] -> Y[p][j][q]
  // with q unit-stride in both: one pass over X and Y on the CUDA cores (memory-bound; a GEMM tile
  // would be mostly padding in k and j and would stage X twice).
  if (bat.empty() && Km.size() == 1 && (Mm.size() == 1 || Nm.size() == 1) && !tc_force) {
    for (int side = 0; side < 2; ++side) {
      const Tens &Sm = side == 0 ? A : B, &Xt = side == 0 ? B : A;
      const std::string &ms = side == 0 ? ma : mb, &mx = side == 0 ? mb : ma;
      const std::string &jg = side == 0 ? Mm : Nm;
      if (jg.size() != 1 || ms.size() != 2) continue;
      const char k = Km[0], j = jg[0];
      const int pk = mode_pos(mx, k), pj = mode_pos(mc, j);
      const std::string prefX = mx.substr(0, pk), sufX = mx.substr(pk + 1);
      const std::string prefC = mc.substr(0, pj), sufC = mc.substr(pj + 1);
      if (prefX != prefC || sufX != sufC) continue;
      const int64_t Kd = Xt.dim[pk], Jd = C.dim[pj];
      if (Kd > 64 || Jd > 64) continue;
      int64_t P1, sXp, P2, sYp, Q1, sXq, Q2, sYq;
      if (!group_view(Xt, mx, prefX, P1, sXp) || !group_view(C, mc, prefC, P2, sYp)) continue;
      if (!group_view(Xt, mx, sufX, Q1, sXq) || !group_view(C, mc, sufC, Q2, sYq)) continue;
      if (Q1 < 32 || (sXq != 1 && Q1 > 1) || (sYq != 1 && Q2 > 1)) continue;
      if (trace_on())
        std::fprintf(stderr, "cclr contract smallk %s,%s->%s P=%lld K=%lld J=%lld Q=%lld dt=%d\n", ma.c_str(),
                     mb.c_str(), mc.c_str(), (long long)P1, (long long)Kd, (long long)Jd, (long long)Q1, dt);
      contract_smallk(dt, P1, (int)Kd, (int)Jd, Q1, Sm.p, Sm.str[mode_pos(ms, k)], Sm.str[mode_pos(ms, j)], Xt.p, sXp,
                      Xt.str[pk], C.p, sYp, C.str[pj], alpha, st);
      return;
    }
  }

  // A tensor of rank <= 4 contracted with a vector over some of its modes, y[r] = sum_c B[r, c] s[c]
  // (the small operand has no output mode): one coalesced pass over B (memory-bound).
  if (bat.empty() && (Mm.empty() || Nm.empty()) && !tc_force) {
    const bool small_a = Mm.empty();
    const Tens &Bt = small_a ? B : A, &Sv = small_a ? A : B;
    const std::string &mbig = small_a ? mb : ma, &msm = small_a ? ma : mb;
    bool ok = Bt.rank <= 4 && Bt.numel() >= (1 << 16);
    int64_t expect = 1;
    for (int q = Bt.rank - 1; q >= 0 && ok; --q) {  // contiguous row-major
      ok = Bt.str[q] == expect || Bt.dim[q] == 1;
      expect *= Bt.dim[q];
    }
    if (ok) {
      int64_t d[4] = {1, 1, 1, 1}, ss[4] = {0, 0, 0, 0}, ys[4] = {0, 0, 0, 0};
      int rmask = 0;
      const int off = 4 - Bt.rank;
      for (int q = 0; q < Bt.rank; ++q) {
        const char mch = mbig[q];
        d[off + q] = Bt.dim[q];
        const int pc = mode_pos(mc, mch);
        if (pc >= 0) {
          rmask |= 1 << (off + q);
          ys[off + q] = C.str[pc];
        } else {
          ss[off + q] = Sv.str[mode_pos(msm, mch)];
        }
      }
      if (!((rmask & 4) && (rmask & 8))) {
        if (trace_on())
          std::fprintf(stderr, "cclr contract gemv %s,%s->%s dims %lld %lld %lld %lld rmask %d dt=%d\n", ma.c_str(),
                       mb.c_str(), mc.c_str(), (long long)d[0], (long long)d[1], (long long)d[2], (long long)d[3],
                       rmask, dt);
        contract_slab_gemv(dt, d, rmask, Bt.p, Sv.p, ss, C.p, ys, alpha, st);
        return;
      }
    }
  }

  // complex64 on tensor cores: operands prepared straight from (two-level) strided views and
  // the result written as interleaved complex pairs into C through its own views; an operand
  // whose modes need more than two levels is first permuted into a contiguous temporary.
  if (dt == C64 && tc_mode && nb <= 16 &&
      (tc_force || ((double)M * N * K >= 3.0e7 && M >= 16 && K >= 8))) {
    // the tensor-core tile is 128 rows high and up to 256 columns wide: a short M side
    // goes to the columns (C^T = B^T A^T)
    // and, when the contraction is short in K (memory-bound), the larger operand goes to the
    // row side, which is read as is (the column side is stored twice as large, embedded)
    if ((M < 128 && N > M) || (N > M && K <= 2048))
      contract_tc(alpha, B, mb, A, ma, C, mc, bat, Nm, Mm, Km, nb, N, M, K);
    else
      contract_tc(alpha, A, ma, B, mb, C, mc, bat, Mm, Nm, Km, nb, M, N, K);
    return;
  }

  // An output mode that keeps the M or N group from being one strided index in both of its
  // operands is peeled off as a batch index (stride 0 in the operand that lacks it), so that
  // no operand is permuted; batch modes proper take precedence.
  if (bat.empty()) {
    auto merges = [&](const std::string &mm, const std::string &nn) {
      int64_t z, t;
      return group_view(A, ma, mm, z, t) && group_view(A, ma, Km, z, t) && group_view(B, mb, Km, z, t) &&
             group_view(B, mb, nn, z, t) && group_view(C, mc, mm, z, t) && group_view(C, mc, nn, z, t);
    };
    if (!merges(Mm, Nm)) {
      for (int side = 0; side < 2; ++side) {
        const std::string &grp = side == 0 ? Nm : Mm;
        for (size_t k = 0; k < grp.size() && grp.size() >= 2; ++k) {
          std::string rest = grp;
          const char pm = rest[k];
          rest.erase(k, 1);
          if (!(side == 0 ? merges(Mm, rest) : merges(rest, Nm))) continue;
          GemmArgs g;
          g.alr = alpha.re; g.ali = alpha.im;
          const int pc = mode_pos(mc, pm);
          g.batch = C.dim[pc];
          g.sCb = C.str[pc];
          if (side == 0) { g.sAb = 0; g.sBb = B.str[mode_pos(mb, pm)]; }
          else { g.sBb = 0; g.sAb = A.str[mode_pos(ma, pm)]; }
          const std::string &mm = side == 0 ? Mm : rest, &nn = side == 0 ? rest : Nm;
          int64_t z;
          group_view(A, ma, mm, z, g.sAm); group_view(A, ma, Km, z, g.sAk);
          group_view(B, mb, Km, z, g.sBk); group_view(B, mb, nn, z, g.sBn);
          group_view(C, mc, mm, z, g.sCm); group_view(C, mc, nn, z, g.sCn);
          g.M = prod_dims(C, mc, mm); g.N = prod_dims(C, mc, nn); g.K = K;
          if (!(g.M == 1 || K == 1 || g.sAm == 1 || g.sAk == 1) || !(K == 1 || g.N == 1 || g.sBk == 1 || g.sBn == 1))
            continue;
          g.A = A.p; g.B = B.p; g.C = C.p; g.overwrite = 0;
          if (trace_on())
            std::fprintf(stderr, "cclr contract simt %s,%s->%s batch over %c (%lld) M=%lld N=%lld K=%lld dt=%d\n",
                         ma.c_str(), mb.c_str(), mc.c_str(), pm, (long long)g.batch, (long long)g.M, (long long)g.N,
                         (long long)K, dt);
          launch_gemm(g, dt, st);
          return;
        }
      }
    }
  }
  GemmArgs g;
  g.M = M; g.N = N; g.K = K; g.batch = nb;
  g.alr = alpha.re; g.ali = alpha.im;
  // A as [batch][M][K]
  {
    int64_t s0, s1, s2, z;
    bool ok = group_view(A, ma, bat, z, s0) && group_view(A, ma, Mm, z, s1) &&
              group_view(A, ma, Km, z, s2);
    ok = ok && (M == 1 || K == 1 || s1 == 1 || s2 == 1);
    if (ok) {
      g.A = A.p; g.sAb = s0; g.sAm = s1; g.sAk = s2;
    } else {
      std::string order = bat + Mm + Km;
      Tens T = contiguous_like(ws(0, nb * M * K * es), dt, A, ma, order);
      permute(zc(1.0), A, ma, T, order, false);
      g.A = T.p; g.sAb = M * K; g.sAm = K; g.sAk = 1;
    }
  }
  // B as [batch][K][N]
  {
    int64_t s0, s1, s2, z;
    bool ok = group_view(B, mb, bat, z, s0) && group_view(B, mb, Km, z, s1) &&
              group_view(B, mb, Nm, z, s2);
    ok = ok && (K == 1 || N == 1 || s1 == 1 || s2 == 1);
    if (ok) {
      g.B = B.p; g.sBb = s0; g.sBk = s1; g.sBn = s2;
    } else {
      std::string order = bat + Km + Nm;
      Tens T = contiguous_like(ws(1, nb * K * N * es), dt, B, mb, order);
      permute(zc(1.0), B, mb, T, order, false);
      g.B = T.p; g.sBb = K * N; g.sBk = N; g.sBn = 1;
    }
  }
  if (trace_on())
    std::fprintf(stderr, "cclr contract simt %s,%s->%s nb=%lld M=%lld N=%lld K=%lld dt=%d\n", ma.c_str(),
                 mb.c_str(), mc.c_str(), (long long)nb, (long long)M, (long long)N, (long long)K, dt);
  // C as [batch][M][N]
  int64_t s0, s1, s2, z;
  bool ok = group_view(C, mc, bat, z, s0) && group_view(C, mc, Mm, z, s1) &&
            group_view(C, mc, Nm, z, s2);
  if (ok) {
    g.C = C.p; g.sCb = s0; g.sCm = s1; g.sCn = s2; g.overwrite = 0;
    launch_gemm(g, dt, st);
  } else {
    std::string order = bat + Mm + Nm;
    Tens T = contiguous_like(ws(2, nb * M * N * es), dt, C, mc, order);
    g.C = T.p; g.sCb = M * N; g.sCm = N; g.sCn = 1; g.overwrite = 1;
    launch_gemm(g, dt, st);
    permute(zc(1.0), T, order, C, mc, true);
  }
}

Engine::PrepEntry *Engine::prep_find(const std::string &key) {
  for (auto &e : prep_)
    if (e->key == key) return e->epoch == state_epoch() ? e.get() : nullptr;
  return nullptr;
}

Engine::PrepEntry *Engine::prep_get(const std::string &key, size_t bytes) {
  for (auto &e : prep_)
    if (e->key == key) return e->buf.bytes == bytes ? e.get() : nullptr;
  if (prep_bytes_ + bytes > prep_cache_cap) return nullptr;
  auto e = std::make_unique<PrepEntry>();
  e->key = key;
  e->buf.alloc(bytes);
  prep_bytes_ += bytes;
  prep_.push_back(std::move(e));
  return prep_.back().get();
}

void Engine::contract_tc(zc alpha, const Tens &A, const std::string &ma, const Tens &B,
                         const std::string &mb, const Tens &C, const std::string &mc,
                         const std::string &bat, const std::string &Mm, const std::string &Nm,
                         const std::string &Km, int64_t nb, int64_t M, int64_t N, int64_t K) {
  const size_t es = dt_size(C64);
  int64_t a0, b0, c0, z;
  View2 am, ak, bk, bn, cm, cn;
  const void *Ap = A.p, *Bp = B.p;
  // A view is read (or written) in place only if one of its two indices walks memory in
  // unit-stride runs of at least 8 elements (or the whole index, when shorter); otherwise
  // the accesses would be scattered and a coalesced permute into a temporary is cheaper.
  auto runs = [](const View2 &x, int64_t n) {
    if (x.sin != 1) return false;
    const int64_t run = x.din == TC_ONE_LEVEL ? n : x.din;
    return run >= std::min<int64_t>(8, n);
  };
  auto coalesced = [&](const View2 &x, int64_t nx, const View2 &y, int64_t ny) {
    return runs(x, nx) || runs(y, ny);
  };
  const int seg = tc_mode == 1 ? 1 : 3;
  const int kind = tc_mode == 3 ? TC_BF16 : TC_TF32;
  const int64_t ld = 2 * tc_kpad(K) * seg, tes = tc_esize(kind);
  const int64_t per_col = 2 * ld * tes, per_row = ld * tes, capb = 2ll << 30;
  // A constant operand (cst_hint) keeps its prepared form: "P" entries hold its permuted
  // contiguous copy, "R" entries its prepared rows (A) or columns (B) for every batch and chunk.
  const bool cache_a = prep_cache_cap && cst_hint && cst_hint == A.p;
  const bool cache_b = prep_cache_cap && cst_hint && cst_hint == B.p && !cache_a;
  std::string akey, bkey;
  if (cache_a || cache_b) {
    char h[96];
    std::snprintf(h, sizeof h, "%p|%d|%d|", cache_a ? A.p : B.p, seg, kind);
    if (cache_a) akey = std::string("A|") + h + ma + "|" + bat + "|" + Mm + "|" + Km + "|";
    else bkey = std::string("B|") + h + mb + "|" + bat + "|" + Km + "|" + Nm + "|";
  }
  PrepEntry *ra = cache_a ? prep_find(akey + "R") : nullptr;  // valid prepared rows of A
  PrepEntry *rb = cache_b ? prep_find(bkey + "R") : nullptr;  // valid prepared columns of B
  if (!(group_view(A, ma, bat, z, a0) && group_view2(A, ma, Mm, am) && group_view2(A, ma, Km, ak) &&
        coalesced(am, M, ak, K))) {
    std::string order = bat + Mm + Km;
    a0 = M * K; am = view1(K); ak = view1(1);
    if (!ra) {
      PrepEntry *pa = cache_a ? prep_find(akey + "P") : nullptr;
      if (pa) {
        Ap = pa->buf.p;
      } else {
        // (a permuted copy pays only where TF32 reads it in place; otherwise its rows are kept)
        PrepEntry *fa = cache_a && seg == 1 ? prep_get(akey + "P", (size_t)(nb * M * K * es)) : nullptr;
        Tens T = contiguous_like(fa ? fa->buf.p : ws(0, nb * M * K * es), C64, A, ma, order);
        permute(zc(1.0), A, ma, T, order, false);
        if (fa) fa->epoch = state_epoch();
        Ap = T.p;
      }
    }
  }
  if (!(group_view(B, mb, bat, z, b0) && group_view2(B, mb, Km, bk) && group_view2(B, mb, Nm, bn) &&
        coalesced(bk, K, bn, N))) {
    std::string order = bat + Km + Nm;
    b0 = K * N; bk = view1(N); bn = view1(1);
    if (!rb) {  // (B is always prepared: its prepared columns are what is kept)
      Tens T = contiguous_like(ws(1, nb * K * N * es), C64, B, mb, order);
      permute(zc(1.0), B, mb, T, order, false);
      Bp = T.p;
    }
  }
  const bool direct = group_view(C, mc, bat, z, c0) && group_view2(C, mc, Mm, cm) &&
                      group_view2(C, mc, Nm, cn) && coalesced(cm, M, cn, N);
  Tens T;
  if (!direct) {
    std::string order = bat + Mm + Nm;
    T = contiguous_like(ws(2, nb * M * N * es), C64, C, mc, order);
    c0 = M * N; cm = view1(N); cn = view1(1);
  }
  if (trace_on())
    std::fprintf(stderr, "cclr contract tc %s,%s->%s nb=%lld M=%lld N=%lld K=%lld A[%s|%s]%s B[%s|%s]%s C[%s|%s]%s%s\n",
                 ma.c_str(), mb.c_str(), mc.c_str(), (long long)nb, (long long)M, (long long)N, (long long)K,
                 vstr(am).c_str(), vstr(ak).c_str(), Ap == A.p ? "" : "(permuted)", vstr(bk).c_str(),
                 vstr(bn).c_str(), Bp == B.p ? "" : "(permuted)", vstr(cm).c_str(), vstr(cn).c_str(),
                 direct ? "" : "(temporary)", ra || rb ? " (cached operand)" : "");
  // prepared operands are bounded (2 GiB each): B in chunks of columns, A in chunks of rows,
  // each chunk starting on a whole block of a two-level view
  auto unit_of = [](const View2 &x, const View2 &y) {
    int64_t u = 1;
    if (x.din != TC_ONE_LEVEL) u = std::lcm(u, x.din);
    if (y.din != TC_ONE_LEVEL) u = std::lcm(u, y.din);
    return u;
  };
  int64_t Nc = N, Mc = M;
  {
    const int64_t u = unit_of(bn, cn);
    if (N * per_col > capb && u < N) Nc = std::max(u, capb / per_col / u * u);
  }
  {
    const int64_t u = unit_of(am, cm);
    if (M * per_row > capb && u < M) Mc = std::max(u, capb / per_row / u * u);
  }
  // TF32 reads A in place when its K index is contiguous and its rows are one strided level
  const bool a_direct = !ra && seg == 1 && ak.sin == 1 && ak.din == TC_ONE_LEVEL && am.din == TC_ONE_LEVEL &&
                        (M == 1 || tc_a_inplace_ok(Ap, am.sin, K)) && (nb == 1 || (a0 * es) % 16 == 0);
  // the constant's rows / columns prepared in this call for later ones (all batches and chunks)
  PrepEntry *wa = cache_a && !ra && !a_direct ? prep_get(akey + "R", (size_t)(nb * M * per_row)) : nullptr;
  PrepEntry *wb = cache_b && !rb ? prep_get(bkey + "R", (size_t)(nb * N * per_col)) : nullptr;
  char *Arows = ra ? (char *)ra->buf.p : wa ? (char *)wa->buf.p : nullptr;
  char *Bcols = rb ? (char *)rb->buf.p : wb ? (char *)wb->buf.p : nullptr;
  void *Ao = nullptr;
  void *Bo = Bcols ? nullptr : ws(4, (size_t)(Nc * per_col));
  bool used_direct = false;
  for (int64_t b = 0; b < nb; ++b) {
    const void *Ab = (const char *)Ap + b * a0 * es;
    const bool ad = a_direct && tc_a_inplace_ok(Ab, M == 1 ? (K + 1) / 2 * 2 : am.sin, K);
    used_direct |= ad;
    if (!ad && !Arows && !Ao) Ao = ws(3, (size_t)(Mc * per_row));
    float *Cb = (float *)((char *)(direct ? C.p : T.p) + b * c0 * es);
    for (int64_t n0 = 0; n0 < N; n0 += Nc) {
      const int64_t nn = std::min(Nc, N - n0);
      void *Bn = Bcols ? (void *)(Bcols + (b * N + n0) * per_col) : Bo;
      if (!rb) tc_prep_b2((const char *)Bp + (b * b0 + v2off(bn, n0)) * es, bk, bn, K, nn, seg, kind, Bn, ld, st);
      float *Cn = Cb + 2 * v2off(cn, n0);
      if (ad) {
        tc_gemm_a_inplace(Ab, M == 1 ? (K + 1) / 2 * 2 : am.sin, K, (const float *)Bn, ld, M, 2 * nn, Cn, cm, cn,
                          alpha, direct, st);
        continue;
      }
      for (int64_t m0 = 0; m0 < M; m0 += Mc) {
        const int64_t mm = std::min(Mc, M - m0);
        void *Am = Arows ? (void *)(Arows + (b * M + m0) * per_row) : Ao;
        if (Arows ? (!ra && n0 == 0) : (n0 == 0 || Mc < M))
          tc_prep_a2((const char *)Ab + v2off(am, m0) * es, am, ak, mm, K, seg, kind, Am, ld, st);
        tc_gemm_seg_v(Am, ld, Bn, ld, mm, 2 * nn, 2 * tc_kpad(K), seg, kind, Cn + 2 * v2off(cm, m0), cm, cn, alpha,
                      direct, st);
      }
    }
    ++tc_calls;
  }
  if (wa && !used_direct) wa->epoch = state_epoch();
  if (wb) wb->epoch = state_epoch();
  if (!direct) permute(zc(1.0), T, bat + Mm + Nm, C, mc, true);
}

}  // namespace cclr
