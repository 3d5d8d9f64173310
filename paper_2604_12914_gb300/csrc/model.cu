// Device-side LR-CCSD model: input upload, T1 dressing of the Cholesky vectors, the stored
// H-bar intermediates, the right-hand side xi, and the sigma / sigma^T interpreter.
//
// Notation (Sec. 2.2): i,j,m,n occupied; a,b,e,f virtual; P Cholesky index.  The exact
// two-body elements of H-bar = e^{-T2} H~ e^{T2}, with H~ the T1-dressed Hamiltonian
// (Cholesky vectors L~ = (1 - t) L (1 + t), t_ai = t_i^a), are
//   Fov = f~_ov, Foo = f~_oo + 1/2 <mn||ef> t_in^ef, Fvv = f~_vv - 1/2 <mn||ef> t_mn^af,
//   Woooo = <mn||ij>~ + 1/2 <mn||ef> t_ij^ef, Wovvo = <mb||ej>~ - <mn||ef> t_jn^fb,
//   Wooov = <mn||ie>~, Wovoo = <mb||ij>~ - Fov_me t_ij^be + 1/2 <mb||ef>~ t_ij^ef
//                               + P(ij) <mn||ie>~ t_jn^be,
// and the vvvv / vovv / vvvo elements are never stored: they enter sigma through L~_vv
// (the "higher-rank integrals evaluated on the fly" of Sec. 3).
#include <cstdio>
#include <cstdlib>

#include <chrono>
#include "model.cuh"
#include "tc_gemm.cuh"

namespace cclr {

Model::Model(int o_, int v_, int naux_, cudaStream_t st_)
    : o(o_), v(v_), naux(naux_), n(o_ + v_), st(st_) {
  E.st = st;
  prog = build_sigma_program(o, v, naux);
}

Model::~Model() {
  clear_graphs();
  if (tm.made)
    for (auto &e : tm.ev) cudaEventDestroy(e);
}

static void h2d_or_d2d(void *dst, const void *src, size_t bytes, int device_ptrs, cudaStream_t st) {
  (void)device_ptrs;  // unified addressing: the copy direction follows from the pointers
  CCLR_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
}

void Model::upload_inputs(const double *eps_h, const double *L, const double *mu_h,
                          const double *t1_h, const double *t2_h, int device_ptrs) {
  const int64_t nn = (int64_t)n * n;
  eps.alloc(sizeof(double) * n);
  h2d_or_d2d(eps.p, eps_h, sizeof(double) * n, device_ptrs, st);
  // full L staged once, split into contiguous blocks
  DevBuf Lfull((size_t)naux * nn * 16);
  h2d_or_d2d(Lfull.p, L, (size_t)naux * nn * 16, device_ptrs, st);
  Tens Lf = make_tens(Lfull.p, C128, {naux, n, n});
  Loo0.alloc((size_t)naux * o * o * 16);
  Lov0.alloc((size_t)naux * o * v * 16);
  Lvo0.alloc((size_t)naux * v * o * 16);
  Lvv0.alloc((size_t)naux * v * v * 16);
  E.permute(zc(1), Lf.slice(1, 0, o).slice(2, 0, o), "Ppq", T(Loo0, {naux, o, o}), "Ppq", false);
  E.permute(zc(1), Lf.slice(1, 0, o).slice(2, o, n), "Ppq", T(Lov0, {naux, o, v}), "Ppq", false);
  E.permute(zc(1), Lf.slice(1, o, n).slice(2, 0, o), "Ppq", T(Lvo0, {naux, v, o}), "Ppq", false);
  E.permute(zc(1), Lf.slice(1, o, n).slice(2, o, n), "Ppq", T(Lvv0, {naux, v, v}), "Ppq", false);
  mu.alloc((size_t)3 * nn * 16);
  h2d_or_d2d(mu.p, mu_h, (size_t)3 * nn * 16, device_ptrs, st);

  // one-body operator h = f - sum_k <pk||qk> with f = diag(eps):
  // sum_k <pk||qk> = sum_P L_pq tr_P - sum_P sum_k L_pk L_kq, tr_P = sum_k L_kk.
  h.alloc(nn * 16);
  Tens H = T(h, {n, n});
  E.zero(H);
  set_diag(n, eps.as<double>(), h.p, st);
  DevBuf Ioo((size_t)o * o * 16), tr((size_t)naux * 16);
  E.zero(T(Ioo, {o, o}));
  {
    std::vector<double> ones(o, 1.0);
    DevBuf od(sizeof(double) * o);
    CCLR_CUDA(cudaMemcpyAsync(od.p, ones.data(), sizeof(double) * o, cudaMemcpyHostToDevice, st));
    set_diag(o, od.as<double>(), Ioo.p, st);
    CCLR_CUDA(cudaStreamSynchronize(st));
  }
  E.zero(T(tr, {naux}));
  E.contract(zc(1), Lf.slice(1, 0, o).slice(2, 0, o), "Pkl", T(Ioo, {o, o}), "kl", T(tr, {naux}), "P");
  E.contract(zc(-1), Lf, "Ppq", T(tr, {naux}), "P", H, "pq");
  E.contract(zc(1), Lf.slice(2, 0, o), "Ppk", Lf.slice(1, 0, o), "Pkq", H, "pq");

  t1.alloc((size_t)o * v * 16);
  if (t1_h) h2d_or_d2d(t1.p, t1_h, (size_t)o * v * 16, device_ptrs, st);
  else E.zero(T(t1, {o, v}));
  t2.alloc((size_t)o * o * v * v * 16);
  Tens T2 = T(t2, {o, o, v, v});
  if (t2_h) {
    h2d_or_d2d(t2.p, t2_h, (size_t)o * o * v * v * 16, device_ptrs, st);
  } else {
    // first-order doubles t_ij^ab = <ab||ij> / (e_i + e_j - e_a - e_b), <ab|ij> = sum_P L_ai L_bj
    E.zero(T2);
    Tens Lvo = T(Lvo0, {naux, v, o});
    E.contract(zc(1), Lvo, "Pai", Lvo, "Pbj", T2, "ijab");
    E.contract(zc(-1), Lvo, "Paj", Lvo, "Pbi", T2, "ijab");
    apply_denominator(o, v, eps.as<double>(), t2.p, st);
  }
  CCLR_CUDA(cudaStreamSynchronize(st));
}

// Complex64 copies of the undressed inputs (made once, for complex64 rebuilds).
void Model::ensure_src64() {
  if (Loo64.p) return;
  auto conv = [&](const DevBuf &src, DevBuf &dst, int64_t ne) {
    dst.alloc((size_t)ne * 8);
    E.permute(zc(1), make_tens(src.p, C128, {ne}), "a", make_tens(dst.p, C64, {ne}), "a", false);
  };
  conv(Loo0, Loo64, (int64_t)naux * o * o);
  conv(Lov0, Lov64, (int64_t)naux * o * v);
  conv(Lvo0, Lvo64, (int64_t)naux * v * o);
  conv(Lvv0, Lvv64, (int64_t)naux * v * v);
  conv(h, h64, (int64_t)n * n);
}

void Model::build_set(const void *t1d, const void *t2d, CstSet &out, int dt, int tc) {
  // CCLR_OPTIME=1 also prints the wall time of every build (diagnostics)
  static const bool optime = std::getenv("CCLR_OPTIME") && std::getenv("CCLR_OPTIME")[0] == '1';
  const auto wall0 = std::chrono::steady_clock::now();
  out.dt = dt;
  const size_t es = dt_size(dt);
  const int P = naux;
  // complex64 builds run on the FP32 CUDA cores by default (FP32-accurate: the stored
  // intermediates enter every sigma, so their error is systematic), or in 3xTF32 (tc = 2)
  const int tc_saved = E.tc_mode;
  E.tc_mode = dt == C64 ? tc : 0;
  auto alloc = [&](int id, std::initializer_list<int64_t> dims) {
    int64_t ne = 1;
    for (auto d : dims) ne *= d;
    if (out.buf[id].bytes != (size_t)ne * es) out.buf[id].alloc((size_t)ne * es);
    out.t[id] = make_tens(out.buf[id].p, dt, dims);
    E.zero(out.t[id]);
    return out.t[id];
  };
  if (dt == C64) ensure_src64();
  auto src = [&](const DevBuf &b128, const DevBuf &b64, std::initializer_list<int64_t> dims) {
    return make_tens(dt == C128 ? b128.p : b64.p, dt, dims);
  };
  Tens Loo = src(Loo0, Loo64, {P, o, o}), Lov = src(Lov0, Lov64, {P, o, v}),
       Lvo = src(Lvo0, Lvo64, {P, v, o}), Lvv = src(Lvv0, Lvv64, {P, v, v});
  Tens Hf = src(h, h64, {n, n});
  // amplitudes in the build precision
  DevBuf t1b, t2b;
  Tens t1t = make_tens((void *)t1d, C128, {o, v});
  Tens t2t = make_tens((void *)t2d, C128, {o, o, v, v});
  if (dt == C64) {
    t1b.alloc((size_t)o * v * 8);
    t2b.alloc((size_t)o * o * v * v * 8);
    Tens a = make_tens(t1b.p, C64, {o, v}), b = make_tens(t2b.p, C64, {o, o, v, v});
    E.permute(zc(1), t1t, "ia", a, "ia", false);
    E.permute(zc(1), t2t, "ijab", b, "ijab", false);
    t1t = a;
    t2t = b;
  }

  // ---- T1 dressing of the Cholesky blocks: L~ = (1 - t) L (1 + t)
  DevBuf Ltoo_b((size_t)P * o * o * es);
  Tens Ltoo = make_tens(Ltoo_b.p, dt, {P, o, o});
  E.permute(zc(1), Loo, "Pij", Ltoo, "Pij", false);
  E.contract(zc(1), Lov, "Pib", t1t, "jb", Ltoo, "Pij");
  Tens Ltov = alloc(K_LOV, {P, o, v});
  E.permute(zc(1), Lov, "Pia", Ltov, "Pia", false);
  Tens Ltvv = alloc(K_LVV, {P, v, v});
  E.permute(zc(1), Lvv, "Pab", Ltvv, "Pab", false);
  E.contract(zc(-1), t1t, "ma", Lov, "Pmb", Ltvv, "Pab");
  Tens Ltvo = alloc(K_LVO, {P, v, o});
  E.permute(zc(1), Lvo, "Pai", Ltvo, "Pai", false);
  E.contract(zc(-1), t1t, "ma", Loo, "Pmi", Ltvo, "Pai");
  E.contract(zc(1), Ltvv, "Pab", t1t, "ib", Ltvo, "Pai");

  // ---- dressed Fock f~ = (1 - t) h (1 + t) + sum_k <pk||qk>~ (oo, ov, vv blocks)
  Tens hoo = Hf.slice(0, 0, o).slice(1, 0, o), hov = Hf.slice(0, 0, o).slice(1, o, n),
       hvv = Hf.slice(0, o, n).slice(1, o, n);
  Tens Foo = alloc(K_FOO, {o, o}), Fov = alloc(K_FOV, {o, v}), Fvv = alloc(K_FVV, {v, v});
  E.permute(zc(1), hoo, "ij", Foo, "ij", false);
  E.contract(zc(1), hov, "ib", t1t, "jb", Foo, "ij");
  E.permute(zc(1), hov, "ia", Fov, "ia", false);
  E.permute(zc(1), hvv, "ab", Fvv, "ab", false);
  E.contract(zc(-1), t1t, "ma", hov, "mb", Fvv, "ab");
  {
    DevBuf Ib((size_t)o * o * 16), Id((size_t)o * o * es), trb((size_t)P * es), ones(sizeof(double) * o);
    Tens I128 = T(Ib, {o, o}), I = make_tens(Id.p, dt, {o, o}), tr = make_tens(trb.p, dt, {P});
    E.zero(I128);
    std::vector<double> one(o, 1.0);
    CCLR_CUDA(cudaMemcpyAsync(ones.p, one.data(), sizeof(double) * o, cudaMemcpyHostToDevice, st));
    set_diag(o, ones.as<double>(), Ib.p, st);
    E.permute(zc(1), I128, "kl", I, "kl", false);
    E.zero(tr);
    E.contract(zc(1), Ltoo, "Pkl", I, "kl", tr, "P");
    E.contract(zc(1), Ltoo, "Pij", tr, "P", Foo, "ij");
    E.contract(zc(1), Ltov, "Pia", tr, "P", Fov, "ia");
    E.contract(zc(1), Ltvv, "Pab", tr, "P", Fvv, "ab");
    E.contract(zc(-1), Ltoo, "Pik", Ltoo, "Pkj", Foo, "ij");
    E.contract(zc(-1), Ltoo, "Pik", Ltov, "Pka", Fov, "ia");
    E.contract(zc(-1), Ltvo, "Pak", Ltov, "Pkb", Fvv, "ab");
    CCLR_CUDA(cudaStreamSynchronize(st));
  }

  // ---- amplitudes and <mn||ef>
  Tens T2 = alloc(K_T2, {o, o, v, v});
  E.permute(zc(1), t2t, "ijab", T2, "ijab", false);
  Tens oovv = alloc(K_OOVV, {o, o, v, v});
  E.contract(zc(1), Ltov, "Pme", Ltov, "Pnf", oovv, "mnef");
  E.contract(zc(-1), Ltov, "Pmf", Ltov, "Pne", oovv, "mnef");

  // ---- one-body H-bar elements
  E.contract(zc(0.5), T2, "inef", oovv, "mnef", Foo, "mi");
  E.contract(zc(-0.5), T2, "mnaf", oovv, "mnef", Fvv, "ae");

  // ---- Woooo = <mn||ij>~ + 1/2 <mn||ef> t_ij^ef
  Tens Woooo = alloc(K_WOOOO, {o, o, o, o});
  E.contract(zc(1), Ltoo, "Pmi", Ltoo, "Pnj", Woooo, "mnij");
  E.contract(zc(-1), Ltoo, "Pmj", Ltoo, "Pni", Woooo, "mnij");
  E.contract(zc(0.5), T2, "ijef", oovv, "mnef", Woooo, "mnij");

  // ---- Wovvo = <mb||ej>~ - <mn||ef> t_jn^fb
  Tens Wovvo = alloc(K_WOVVO, {o, v, v, o});
  E.contract(zc(1), Ltov, "Pme", Ltvo, "Pbj", Wovvo, "mbej");
  E.contract(zc(-1), Ltoo, "Pmj", Ltvv, "Pbe", Wovvo, "mbej");
  E.contract(zc(-1), T2, "jnfb", oovv, "mnef", Wovvo, "mbej");

  // ---- Wooov = <mn||ie>~
  Tens Wooov = alloc(K_WOOOV, {o, o, o, v});
  E.contract(zc(1), Ltoo, "Pmi", Ltov, "Pne", Wooov, "mnie");
  E.contract(zc(-1), Ltov, "Pme", Ltoo, "Pni", Wooov, "mnie");

  // ---- Wovoo = <mb||ij>~ - Fov t + 1/2 <mb||ef>~ t_ij^ef + P(ij) <mn||ie>~ t_jn^be
  Tens Wovoo = alloc(K_WOVOO, {o, v, o, o});
  E.contract(zc(1), Ltoo, "Pmi", Ltvo, "Pbj", Wovoo, "mbij");
  E.contract(zc(-1), Ltoo, "Pmj", Ltvo, "Pbi", Wovoo, "mbij");
  E.contract(zc(-1), Fov, "me", T2, "ijbe", Wovoo, "mbij");
  {
    DevBuf tb((size_t)o * v * o * o * es);
    Tens tmp = make_tens(tb.p, dt, {o, v, o, o});
    E.zero(tmp);
    E.contract(zc(1), Wooov, "mnie", T2, "jnbe", tmp, "mbij");
    E.permute(zc(1), tmp, "mbij", Wovoo, "mbij", true);
    E.permute(zc(-1), tmp, "mbij", Wovoo, "mbji", true);
    // 1/2 sum_ef <mb||ef>~ t_ij^ef = sum_ef <mb|ef>~ t_ij^ef, formed in chunks of b
    int64_t per_b = (int64_t)o * v * v * es;
    int64_t bc = std::max<int64_t>(1, std::min<int64_t>(v, (int64_t)(1ll << 30) / per_b));
    DevBuf Gb((size_t)(bc * per_b));
    for (int64_t b0 = 0; b0 < v; b0 += bc) {
      int64_t b1 = std::min<int64_t>(v, b0 + bc);
      Tens G = make_tens(Gb.p, dt, {o, b1 - b0, v, v});
      E.zero(G);
      E.contract(zc(1), Ltov, "Pme", Ltvv.slice(1, b0, b1), "Pbf", G, "mbef");
      E.contract(zc(1), G, "mbef", T2, "ijef", Wovoo.slice(1, b0, b1), "mbij");
    }
    CCLR_CUDA(cudaStreamSynchronize(st));
  }
  E.tc_mode = tc_saved;
  if (lean) E.release_ws();  // the builds' permuted operands are not needed by the products
  for (int k = 0; k < 3; ++k)  // a ladder prepared from this buffer is stale
    if (ltc_src[k] == out.t[K_LVV].p) ltc_src[k] = nullptr;
  bump_state_epoch();  // and so is any captured program that read the set
  E.clear_prep_cache();  // and every prepared constant operand
  out.valid = true;
  if (optime) {
    CCLR_CUDA(cudaStreamSynchronize(st));
    std::fprintf(stderr, "cclr build_set dt %d: %.3f ms\n", dt,
                 std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count());
  }
}

// H-bar of a one-body operator B (Hamiltonian without two-body part) with the T1 dressing
// B~ = (1 - t) B (1 + t): Fov = B~_ov, Foo = B~_oo, Fvv = B~_vv, Wovoo = -Fov_me t_ij^be; every
// element with a two-body integral (Woooo, Wovvo, Wooov, <mn||ef>, L~) vanishes.
void Model::build_set_onebody(const void *Bd, const void *t1d, const void *t2d, CstSet &out) {
  out.dt = C128;
  const int tc_saved = E.tc_mode;
  E.tc_mode = 0;
  Tens Bm = make_tens((void *)Bd, C128, {n, n});
  Tens t1t = make_tens((void *)t1d, C128, {o, v});
  Tens t2t = make_tens((void *)t2d, C128, {o, o, v, v});
  auto alloc = [&](int id, std::initializer_list<int64_t> dims) {
    int64_t ne = 1;
    for (auto d : dims) ne *= d;
    if (out.buf[id].bytes != (size_t)ne * 16) out.buf[id].alloc((size_t)ne * 16);
    out.t[id] = make_tens(out.buf[id].p, C128, dims);
    E.zero(out.t[id]);
    return out.t[id];
  };
  Tens boo = Bm.slice(0, 0, o).slice(1, 0, o), bov = Bm.slice(0, 0, o).slice(1, o, n),
       bvv = Bm.slice(0, o, n).slice(1, o, n);
  Tens Foo = alloc(K_FOO, {o, o}), Fov = alloc(K_FOV, {o, v}), Fvv = alloc(K_FVV, {v, v});
  E.permute(zc(1), boo, "ij", Foo, "ij", false);
  E.contract(zc(1), bov, "ib", t1t, "jb", Foo, "ij");
  E.permute(zc(1), bov, "ia", Fov, "ia", false);
  E.permute(zc(1), bvv, "ab", Fvv, "ab", false);
  E.contract(zc(-1), t1t, "ma", bov, "mb", Fvv, "ab");
  Tens T2 = alloc(K_T2, {o, o, v, v});
  E.permute(zc(1), t2t, "ijab", T2, "ijab", false);
  Tens Wovoo = alloc(K_WOVOO, {o, v, o, o});
  E.contract(zc(-1), Fov, "me", T2, "ijbe", Wovoo, "mbij");
  for (int k = 0; k < K_NCST; ++k) out.zero[k] = true;
  for (int k : {K_FOO, K_FOV, K_FVV, K_T2, K_WOVOO}) out.zero[k] = false;
  for (int k = 0; k < K_NCST; ++k)
    if (out.zero[k]) out.buf[k].release();
  E.tc_mode = tc_saved;
  CCLR_CUDA(cudaStreamSynchronize(st));
  bump_state_epoch();
  E.clear_prep_cache();
  out.valid = true;
}

void Model::build_diagonal() {
  D1.alloc(sizeof(double) * o * v);
  D2.alloc(sizeof(double) * std::max<size_t>(1, (size_t)o * (o - 1) / 2 * ((size_t)v * (v - 1) / 2)));
  const CstSet &C = c128.valid ? c128 : c64;
  DevBuf f((size_t)(o * o + v * v) * 16);
  Tens foo = make_tens(f.p, C128, {o, o}), fvv = make_tens((char *)f.p + (size_t)o * o * 16, C128, {v, v});
  E.permute(zc(1), C.t[K_FOO], "ij", foo, "ij", false);
  E.permute(zc(1), C.t[K_FVV], "ab", fvv, "ab", false);
  build_diag(o, v, foo.p, fvv.p, D1.as<double>(), D2.as<double>(), st);
  CCLR_CUDA(cudaStreamSynchronize(st));
}

// complex64 rounding of a complex128 set (same shapes, contiguous)
void Model::round_set(const CstSet &src, CstSet &dst) {
  CCLR_REQUIRE(src.valid && src.dt == C128, "round_set: source must be a valid complex128 set");
  dst.dt = C64;
  dst.zero = src.zero;
  for (int k = 0; k < K_NCST; ++k) {
    const Tens &s = src.t[k];
    const size_t bytes = (size_t)s.numel() * 8;
    if (dst.buf[k].bytes != bytes) dst.buf[k].alloc(bytes);
    Tens d = s;
    d.p = dst.buf[k].p;
    d.dt = C64;
    const std::string m = std::string("abcdefgh").substr(0, s.rank);
    E.permute(zc(1), s, m, d, m, false);
    dst.t[k] = d;
  }
  // a tensor-core ladder prepared from this set's L~_vv (same buffer) is now stale, and so is
  // any captured program that read it
  for (int k = 0; k < 3; ++k)
    if (ltc_src[k] == dst.t[K_LVV].p) ltc_src[k] = nullptr;
  bump_state_epoch();
  E.clear_prep_cache();
  CCLR_CUDA(cudaStreamSynchronize(st));
  dst.valid = true;
}

void Model::release_set(CstSet &s) {
  E.clear_prep_cache();
  for (int k = 0; k < 3; ++k)
    if (s.t[K_LVV].p && ltc_src[k] == s.t[K_LVV].p) ltc_src[k] = nullptr;
  for (auto &b : s.buf) b.release();
  s.valid = false;
}

void Model::release_fp64() {
  release_set(c128);
  tmp128.clear();
  x2bar[C128].clear();
  lcc.release();
}

void Model::release_product_buffers() {
  tmp64.clear();
  tmp128.clear();
  x2bar[0].clear();
  x2bar[1].clear();
  E.release_ws();
  E.clear_prep_cache();
  for (int k = 0; k < 3; ++k) {
    ltc[k].release();
    ltc_src[k] = nullptr;
  }
  lcc.release();
  clear_graphs();
}

void Model::release_fp64_inputs() {
  ensure_src64();
  oovv_packed();
  Loo0.release(); Lov0.release(); Lvo0.release(); Lvv0.release();
  fp64_gone = true;
}

// The FP64 mode reads intermediates built in FP64.  The complex64 modes read the rounding of
// those when they exist, else a set built in FP32 on the CUDA cores (this GPU's FP64 rate makes
// the FP64 build of the o^3 v^3 and o v^3 naux terms take minutes at o=56, v=480).
const CstSet &Model::cst_for(int p) {
  if (p == 0) {
    if (!c128.valid) {
      if (fp64_gone)
        throw Error(6, "FP64 products are unavailable: this budgeted context freed its FP64 inputs when 3xTF32 "
                       "refinement was set");
      build_set(t1.p, t2.p, c128, C128);
    }
    return c128;
  }
  if (!c64.valid) {
    if (c128.valid) round_set(c128, c64);
    else build_set(t1.p, t2.p, c64, C64);
  }
  return c64;
}

// <ij||ab> in complex128, packed (the T1-independent oovv block), for dE/dT and the F X stencil:
// from the complex128 set when it exists, else formed from the undressed L_ov (the ov block is
// unchanged by the T1 dressing) in a temporary full tensor.
const void *Model::oovv_packed() {
  if (!oovvp.p) {
    oovvp.alloc((size_t)std::max<int64_t>(1, (int64_t)o * (o - 1) / 2 * ((int64_t)v * (v - 1) / 2)) * 16);
    if (c128.valid) {
      pack_doubles(C128, C128, o, v, c128.t[K_OOVV].p, oovvp.p, st);
    } else {
      DevBuf full((size_t)o * o * v * v * 16);
      Tens F = make_tens(full.p, C128, {o, o, v, v});
      Tens Lov = T(Lov0, {naux, o, v});
      E.zero(F);
      E.contract(zc(1), Lov, "Pme", Lov, "Pnf", F, "mnef");
      E.contract(zc(-1), Lov, "Pmf", Lov, "Pne", F, "mnef");
      pack_doubles(C128, C128, o, v, full.p, oovvp.p, st);
      CCLR_CUDA(cudaStreamSynchronize(st));
    }
    CCLR_CUDA(cudaStreamSynchronize(st));
  }
  return oovvp.p;
}

std::vector<DevBuf> &Model::temps(int dt) {
  auto &tv = dt == C128 ? tmp128 : tmp64;
  if (tv.empty()) {
    tv.resize(prog.vars.size());
    for (size_t k = 0; k < prog.vars.size(); ++k) {
      if (k < 4) continue;  // x1, x2, s1, s2 (and their bars) live in per-RHS buffers
      int64_t ne = 1;
      for (auto d : prog.vars[k].dims) ne *= d;
      tv[k].alloc((size_t)ne * dt_size(dt));
    }
  }
  return tv;
}

Tens Model::var_tens(int id, int dt, void *p) const {
  Tens t;
  t.p = p;
  t.dt = dt;
  t.rank = (int)prog.vars[id].dims.size();
  int64_t s = 1;
  for (int k = t.rank - 1; k >= 0; --k) {
    t.dim[k] = prog.vars[id].dims[k];
    t.str[k] = s;
    s *= t.dim[k];
  }
  return t;
}

// pp-ladder: out[i,j,a,b] += alpha sum_ef <ab|ef>~ in[i,j,e,f] (dir +1), or the transpose
// in'[i,j,e,f] += alpha sum_ab <ab|ef>~ in[i,j,a,b] (dir -1), over packed pairs with <ab|ef>~
// formed per group of a from L~_vv and never stored whole: tcgen05 tensor cores in the TF32 /
// 3xTF32 modes, CUDA cores otherwise.
void Model::ladder(int dir, const CstSet &C, zc alpha, const std::vector<Tens> &in,
                   const std::vector<Tens> &out) {
  const int dt = C.dt;
  const int nr = (int)in.size();
  if (dt == C64 && E.tc_mode) {
    const int k = E.tc_mode - 1, seg = E.tc_mode == 1 ? 1 : 3, kind = E.tc_mode == 3 ? TC_BF16 : TC_TF32;
    if (lean)  // a budgeted context keeps one tensor-core ladder's buffers at a time
      for (int q = 0; q < 3; ++q)
        if (q != k && ltc_src[q]) {
          ltc[q].release();
          ltc_src[q] = nullptr;
        }
    if (!ltc[k].ready(seg, kind) || ltc_src[k] != C.t[K_LVV].p) {
      ltc[k].prepare(E, C.t[K_LVV], o, v, naux, seg, kind, lean);
      ltc_src[k] = C.t[K_LVV].p;
    }
    std::vector<const void *> ip(nr);
    std::vector<void *> outp(nr);
    for (int r = 0; r < nr; ++r) { ip[r] = in[r].p; outp[r] = out[r].p; }
    ltc[k].apply(E, dir, alpha, nr, ip.data(), outp.data());
    return;
  }
  // CUDA cores (FP64 DFMA or FP32 FFMA): the same packed algorithm
  std::vector<const void *> ip(nr);
  std::vector<void *> outp(nr);
  for (int r = 0; r < nr; ++r) { ip[r] = in[r].p; outp[r] = out[r].p; }
  lcc.apply(E, dt, C.t[K_LVV], o, v, naux, dir, alpha, nr, ip.data(), outp.data());
}

void Model::apply(int dir, const CstSet &C, const void *x1, const void *x2, void *s1, void *s2) {
  apply_batch(dir, C, 1, &x1, &x2, &s1, &s2);
}

void Model::apply_body(int dir, const CstSet &C, int nr, const void *const *x1, const void *const *x2,
                       void *const *s1, void *const *s2, bool timed, float &lad_ms, float &form_ms) {
  const int dt = C.dt;
  const int nv = (int)prog.vars.size();
  // One set of program temporaries serves every right-hand side in turn; only the ladder, which
  // forms each <ab||ef>~ block once for all of them, sees all right-hand sides at once.  Its
  // output (input, in the transpose) is a per-RHS buffer, so it can run first (last).
  auto &tv = temps(dt);
  std::vector<std::vector<void *>> ptr(nr, std::vector<void *>(nv, nullptr));
  for (int r = 0; r < nr; ++r)
    for (int k = 4; k < nv; ++k) ptr[r][k] = tv[k].p;
  auto V = [&](int r, int id) { return var_tens(id, dt, ptr[r][id]); };
  auto Cst = [&](int id) { return C.t[id]; };
  auto run_ladder = [&](int d, zc a, int in_id, int out_id) {
    if (C.zero[K_LVV]) return;
    std::vector<Tens> in(nr), out(nr);
    for (int r = 0; r < nr; ++r) { in[r] = V(r, in_id); out[r] = V(r, out_id); }
    if (!timed) {
      ladder(d, C, a, in, out);
      return;
    }
    CCLR_CUDA(cudaEventRecord(tm.ev[1], st));
    ladder(d, C, a, in, out);
    CCLR_CUDA(cudaEventRecord(tm.ev[2], st));
    CCLR_CUDA(cudaEventSynchronize(tm.ev[2]));
    float ms = 0.f;
    CCLR_CUDA(cudaEventElapsedTime(&ms, tm.ev[1], tm.ev[2]));
    lad_ms += ms;
    if (dt == C64 && E.tc_mode) form_ms += ltc[E.tc_mode - 1].formation_ms();
  };
  const Op *lad = nullptr;
  for (const Op &op : prog.ops)
    if (op.kind == OP_LADDER) lad = &op;
  if (dir > 0) {
    for (int r = 0; r < nr; ++r) {
      ptr[r][0] = (void *)x1[r]; ptr[r][1] = (void *)x2[r]; ptr[r][2] = s1[r]; ptr[r][3] = s2[r];
      E.zero(V(r, 2));
      E.zero(V(r, 3));
    }
    if (lad) run_ladder(+1, lad->alpha, lad->in, lad->out);
    // CCLR_OPTIME=1 prints the device time of every operation of the first RHS (diagnostics)
    static const bool optime = std::getenv("CCLR_OPTIME") && std::getenv("CCLR_OPTIME")[0] == '1';
    cudaEvent_t oe0 = nullptr, oe1 = nullptr;
    if (optime && timed) {
      CCLR_CUDA(cudaEventCreate(&oe0));
      CCLR_CUDA(cudaEventCreate(&oe1));
    }
    for (int r = 0; r < nr; ++r)
      for (size_t oi = 0; oi < prog.ops.size(); ++oi) {
        const Op &op = prog.ops[oi];
        if (op.kind == OP_LADDER || (op.kind == OP_CONTRACT && C.zero[op.cst])) continue;
        if (oe0 && r == 0) CCLR_CUDA(cudaEventRecord(oe0, st));
        switch (op.kind) {
          case OP_CONTRACT:
            E.cst_hint = Cst(op.cst).p;
            E.contract(op.alpha, Cst(op.cst), op.mc, V(r, op.in), op.mi, V(r, op.out), op.mo);
            E.cst_hint = nullptr;
            break;
          case OP_PERM: E.permute(op.alpha, V(r, op.in), op.mi, V(r, op.out), op.mo, true); break;
          case OP_ZERO: E.zero(V(r, op.out)); break;
          case OP_ANTISYM:
            antisym_apply(dt, o, v, +1, ptr[r][op.out], ptr[r][op.in], ptr[r][op.in2], ptr[r][op.in3], st);
            break;
          case OP_PROJECT: antisym_project(dt, o, v, ptr[r][op.out], st); break;
          default: break;
        }
        if (oe0 && r == 0) {
          CCLR_CUDA(cudaEventRecord(oe1, st));
          CCLR_CUDA(cudaEventSynchronize(oe1));
          float ms = 0.f;
          CCLR_CUDA(cudaEventElapsedTime(&ms, oe0, oe1));
          std::fprintf(stderr, "cclr op %zu kind %d cst %d %s,%s->%s dt %d tc %d: %.3f ms\n", oi, (int)op.kind, op.cst,
                       op.mc.c_str(), op.mi.c_str(), op.mo.c_str(), dt, E.tc_mode, ms);
        }
      }
    if (oe0) {
      cudaEventDestroy(oe0);
      cudaEventDestroy(oe1);
    }
  } else {
    // bars: s1-bar = y1 (the x1 argument), s2-bar = y2 / 4 (unique-amplitude weight), held in
    // the s2 output until the end; x1-bar accumulates in the s1 output and x2-bar in a per-RHS
    // buffer, which is projected onto antisymmetric tensors into s2 at the end
    auto &xb = x2bar[dt];
    if ((int)xb.size() < nr) xb.resize(nr);
    for (int r = 0; r < nr; ++r) {
      if (!xb[r].p) xb[r].alloc((size_t)o * o * v * v * dt_size(dt));
      ptr[r][2] = (void *)x1[r];
      ptr[r][3] = s2[r];
      ptr[r][0] = s1[r];
      ptr[r][1] = xb[r].p;
      E.permute(zc(0.25), var_tens(3, dt, (void *)x2[r]), "ijab", V(r, 3), "ijab", false);
      E.zero(V(r, 0));
      E.zero(V(r, 1));
    }
    for (int r = 0; r < nr; ++r) {
      for (int k = 4; k < nv; ++k) E.zero(V(r, k));
      for (auto it = prog.ops.rbegin(); it != prog.ops.rend(); ++it) {
        const Op &op = *it;
        if (op.kind == OP_LADDER || (op.kind == OP_CONTRACT && C.zero[op.cst])) continue;
        switch (op.kind) {
          case OP_CONTRACT:
            E.cst_hint = Cst(op.cst).p;
            E.contract(op.alpha, Cst(op.cst), op.mc, V(r, op.out), op.mo, V(r, op.in), op.mi);
            E.cst_hint = nullptr;
            break;
          case OP_PERM: E.permute(op.alpha, V(r, op.out), op.mo, V(r, op.in), op.mi, true); break;
          case OP_ZERO: E.zero(V(r, op.out)); break;
          case OP_ANTISYM:
            antisym_apply(dt, o, v, -1, ptr[r][op.out], ptr[r][op.in], ptr[r][op.in2], ptr[r][op.in3], st);
            break;
          case OP_PROJECT: antisym_project(dt, o, v, ptr[r][op.out], st); break;
          default: break;
        }
      }
    }
    // the transposed ladder reads only s2-bar, which is final once the projection (the first
    // transposed operation) has run, and adds into x2-bar
    if (lad) run_ladder(-1, lad->alpha, lad->out, lad->in);
    for (int r = 0; r < nr; ++r) {
      Tens out2 = var_tens(3, dt, s2[r]);
      Tens z2 = V(r, 1);
      E.permute(zc(1), z2, "ijab", out2, "ijab", false);
      E.permute(zc(-1), z2, "ijab", out2, "jiab", true);
      E.permute(zc(-1), z2, "ijab", out2, "ijba", true);
      E.permute(zc(1), z2, "ijab", out2, "jiba", true);
    }
  }
}

void Model::clear_graphs() {
  for (auto &g : gcache)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  gcache.clear();
  warm.clear();
}

void Model::apply_batch(int dir, const CstSet &C, int nr, const void *const *x1, const void *const *x2,
                        void *const *s1, void *const *s2) {
  const int dt = C.dt;
  // tensor cores for complex64: TF32 (prec 1), 3xTF32 (prec 2) or bf16x3 (prec 4); FP32 CUDA cores
  // for prec 3
  E.tc_mode = dt == C64 ? (prec == 1 ? 1 : prec == 2 ? 2 : prec == 4 ? 3 : 0) : 0;
  if (!tm.made) {
    for (auto &e : tm.ev) CCLR_CUDA(cudaEventCreate(&e));
    tm.made = true;
  }
  GraphKey key;
  if (graphs) {
    key.dir = dir; key.dt = dt; key.tc = E.tc_mode; key.nr = nr; key.set = &C;
    for (int r = 0; r < nr; ++r) {
      key.ptrs.push_back(x1[r]); key.ptrs.push_back(x2[r]);
      key.ptrs.push_back(s1[r]); key.ptrs.push_back(s2[r]);
    }
    const unsigned long long ep = state_epoch();
    GraphEntry *hit = nullptr;
    for (size_t g = 0; g < gcache.size(); ++g) {
      if (!(gcache[g].key == key)) continue;
      if (gcache[g].epoch == ep) {
        hit = &gcache[g];
      } else {  // memory it refers to was freed or constants rebuilt since the capture
        cudaGraphExecDestroy(gcache[g].exec);
        gcache.erase(gcache.begin() + g);
      }
      break;
    }
    bool was_warm = false;
    for (const auto &w : warm)
      if (w.key == key && w.epoch == ep) was_warm = true;
    if (!hit && was_warm) {
      // an eager call with these arguments ran since the last free or rebuild, so every buffer
      // the program touches is allocated and prepared: capture
      cudaGraph_t gr = nullptr;
      float l = 0.f, f = 0.f;
      CCLR_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      bool body_ok = true;
      try {
        apply_body(dir, C, nr, x1, x2, s1, s2, false, l, f);
      } catch (...) {
        body_ok = false;  // nothing of a capture executes: the eager path below redoes it all
      }
      const cudaError_t ec = cudaStreamEndCapture(st, &gr);
      cudaGraphExec_t ex = nullptr;
      if (body_ok && ec == cudaSuccess && gr && state_epoch() == ep &&
          cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess) {
        if (gcache.size() >= 8) {
          cudaGraphExecDestroy(gcache.front().exec);
          gcache.erase(gcache.begin());
        }
        GraphEntry e;
        e.key = key;
        e.exec = ex;
        e.epoch = ep;
        gcache.push_back(std::move(e));
        hit = &gcache.back();
        ++graph_captures;
      } else {
        (void)cudaGetLastError();
        graphs = false;  // this program cannot be captured here: stay eager from now on
        warm.clear();
      }
      if (gr) cudaGraphDestroy(gr);
    }
    if (hit) {
      CCLR_CUDA(cudaEventRecord(tm.ev[0], st));
      CCLR_CUDA(cudaGraphLaunch(hit->exec, st));
      CCLR_CUDA(cudaEventRecord(tm.ev[3], st));
      CCLR_CUDA(cudaEventSynchronize(tm.ev[3]));
      float tot = 0.f;
      CCLR_CUDA(cudaEventElapsedTime(&tot, tm.ev[0], tm.ev[3]));
      ms_last[0] = -1.f;  // the split is not measured inside a graph
      ms_last[1] = -1.f;
      ms_last[2] = tot;
      ms_last[3] = -1.f;
      ++graph_launches;
      if (E.tc_mode && tc_error(st)) throw Error(5, "a tensor-core kernel gave up on a bounded wait");
      return;
    }
  }
  float lad_ms = 0.f, form_ms = 0.f;
  tc_set_autotune(autotune && E.tc_mode != 0);
  try {
    CCLR_CUDA(cudaEventRecord(tm.ev[0], st));
    apply_body(dir, C, nr, x1, x2, s1, s2, true, lad_ms, form_ms);
  } catch (...) {
    tc_set_autotune(false);
    throw;
  }
  tc_set_autotune(false);
  if (lean) E.release_ws();  // a budgeted context does not keep the product's staging
  CCLR_CUDA(cudaEventRecord(tm.ev[3], st));
  CCLR_CUDA(cudaEventSynchronize(tm.ev[3]));
  float tot = 0.f;
  CCLR_CUDA(cudaEventElapsedTime(&tot, tm.ev[0], tm.ev[3]));
  ms_last[0] = lad_ms;
  ms_last[1] = tot - lad_ms;
  ms_last[2] = tot;
  ms_last[3] = form_ms;
  if (E.tc_mode && tc_error(st)) throw Error(5, "a tensor-core kernel gave up on a bounded wait");
  if (graphs) {
    for (size_t w = 0; w < warm.size(); ++w)
      if (warm[w].key == key) {
        warm.erase(warm.begin() + w);
        break;
      }
    if (warm.size() >= 8) warm.erase(warm.begin());
    GraphEntry e;
    e.key = key;
    e.epoch = state_epoch();
    warm.push_back(std::move(e));
  }
}

// xi^B_ia = mu~_ai + sum_me mu~_me t_im^ae ;
// xi^B_ijab = P(ab) sum_e mu~_be t_ij^ae - P(ij) sum_m mu~_mj t_im^ab ; mu~ = (1-t) mu (1+t).
void Model::xi(const void *mub, const void *t1d, const void *t2d, void *xi1, void *xi2) {
  Tens M = make_tens((void *)mub, C128, {n, n});
  Tens t1t = make_tens((void *)t1d, C128, {o, v});
  Tens t2t = make_tens((void *)t2d, C128, {o, o, v, v});
  Tens moo = M.slice(0, 0, o).slice(1, 0, o), mov = M.slice(0, 0, o).slice(1, o, n),
       mvo = M.slice(0, o, n).slice(1, 0, o), mvv = M.slice(0, o, n).slice(1, o, n);
  DevBuf b((size_t)(o * o + v * v + v * o) * 16);
  Tens Moo = make_tens(b.p, C128, {o, o});
  Tens Mvv = make_tens((char *)b.p + (size_t)o * o * 16, C128, {v, v});
  Tens Mvo = make_tens((char *)b.p + (size_t)(o * o + v * v) * 16, C128, {v, o});
  E.permute(zc(1), moo, "ij", Moo, "ij", false);
  E.contract(zc(1), mov, "ib", t1t, "jb", Moo, "ij");
  E.permute(zc(1), mvv, "ab", Mvv, "ab", false);
  E.contract(zc(-1), t1t, "ma", mov, "mb", Mvv, "ab");
  E.permute(zc(1), mvo, "ai", Mvo, "ai", false);
  E.contract(zc(-1), t1t, "ma", moo, "mi", Mvo, "ai");
  E.contract(zc(1), Mvv, "ab", t1t, "ib", Mvo, "ai");
  Tens X1 = make_tens(xi1, C128, {o, v});
  Tens X2 = make_tens(xi2, C128, {o, o, v, v});
  E.permute(zc(1), Mvo, "ai", X1, "ia", false);
  E.contract(zc(1), mov, "me", t2t, "imae", X1, "ia");
  // f = sum_e mu~_be t_ij^ae is antisymmetric in (i,j), g = sum_m mu~_mj t_im^ab in (a,b); the
  // projection onto tensors antisymmetric in both pairs maps f - g to (P(ab) f - P(ij) g) / 2,
  // so xi_2 = 2 project(f - g), formed in place (no temporary of o^2 v^2 entries)
  E.zero(X2);
  E.contract(zc(1), Mvv, "be", t2t, "ijae", X2, "ijab");
  E.contract(zc(-1), Moo, "mj", t2t, "imab", X2, "ijab");
  antisym_project(C128, o, v, X2.p, st);
  vec_scal(C128, X2.numel(), zc(2.0), X2.p, st);
  CCLR_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------------------
// The sigma program: <mu|(H-bar X)_c|Phi_0> as linear operations on X (Sec. 2.2 Jacobian).
// ---------------------------------------------------------------------------------------
Program build_sigma_program(int o, int v, int naux) {
  Program p;
  const int64_t O = o, Vv = v, P = naux;
  auto var = [&](std::vector<int64_t> d) { p.vars.push_back({d}); return (int)p.vars.size() - 1; };
  const int X1 = var({O, Vv}), X2 = var({O, O, Vv, Vv}), S1 = var({O, Vv}), S2 = var({O, O, Vv, Vv});
  const int Zt = var({P, O, Vv}), Rab = var({O, O, Vv, Vv}), Rij = var({O, O, Vv, Vv}),
            Rijab = var({O, O, Vv, Vv}), Zoo = var({O, O, O, O}), U = var({P, Vv, O}),
            sm = var({P, O, O}), Vm = var({O, Vv, O, Vv}), Xvv = var({Vv, Vv}), Xoo = var({O, O}),
            w = var({P});
  (void)S1;
  auto C = [&](double a, int cst, const char *mc, int in, const char *mi, int out, const char *mo) {
    p.ops.push_back(Op{OP_CONTRACT, zc(a), cst, mc, mi, mo, in, out});
  };
  auto Z = [&](int out) { p.ops.push_back(Op{OP_ZERO, zc(0), -1, "", "", "", -1, out}); };
  auto PM = [&](double a, int in, const char *mi, int out, const char *mo) {
    p.ops.push_back(Op{OP_PERM, zc(a), -1, "", mi, mo, in, out});
  };
  // ---- singles
  C(1, K_FVV, "ae", X1, "ie", S1, "ia");
  C(-1, K_FOO, "mi", X1, "ma", S1, "ia");
  C(1, K_WOVVO, "maei", X1, "me", S1, "ia");
  C(1, K_FOV, "me", X2, "imae", S1, "ia");
  Z(Zt);  // 1/2 sum <am||ef>~ X_im^ef = sum_P sum_e L~_ae (sum_mf L~_mf X_im^ef)
  C(1, K_LOV, "Pmf", X2, "imef", Zt, "Pie");
  C(1, K_LVV, "Pae", Zt, "Pie", S1, "ia");
  C(-0.5, K_WOOOV, "mnie", X2, "mnae", S1, "ia");
  // ---- doubles
  Z(Rab); Z(Rij); Z(Rijab);
  C(1, K_FVV, "be", X2, "ijae", Rab, "ijab");
  C(-1, K_FOO, "mj", X2, "imab", Rij, "ijab");
  C(0.5, K_WOOOO, "mnij", X2, "mnab", S2, "ijab");
  p.ops.push_back(Op{OP_LADDER, zc(1), -1, "", "ijef", "ijab", X2, S2});  // sum_ef <ab|ef>~ X
  Z(Zoo);  // vvvv element's T2 part: 1/2 t_mn^ab (1/2 <mn||ef> X_ij^ef)
  C(0.5, K_OOVV, "mnef", X2, "ijef", Zoo, "mnij");
  // and P(ij) 1/2 t_mn^ab <mn||ej>~ x_i^e: the o^4 matrix it contracts with t joins Zoo, already
  // antisymmetrised in (i,j), so one o^4 v^2 contraction serves both terms
  C(-1, K_WOOOV, "mnje", X1, "ie", Zoo, "mnij");
  C(1, K_WOOOV, "mnie", X1, "je", Zoo, "mnij");
  C(0.5, K_T2, "mnab", Zoo, "mnij", S2, "ijab");
  C(1, K_WOVVO, "mbej", X2, "imae", Rijab, "ijab");           // ring, P(ij)P(ab)
  // P(ij) sum_e Wvvvo_abej x_i^e, factorised through L~ (vvvo never stored)
  Z(U);
  C(1, K_LVV, "Pae", X1, "ie", U, "Pai");
  C(1, K_LVO, "Pbj", U, "Pai", Rijab, "ijab");               // <ab||ej>~ x_i^e
  Z(sm);
  C(1, K_LOV, "Pme", X1, "ie", sm, "Pmi");
  Z(Vm);                                                     // V_mbif = sum_e <mb||ef>~ x_i^e
  C(1, K_LVV, "Pbf", sm, "Pmi", Vm, "mbif");
  C(-1, K_LOV, "Pmf", U, "Pbi", Vm, "mbif");
  C(-1, K_T2, "mjaf", Vm, "mbif", Rijab, "ijab");
  C(-1, K_WOVOO, "mbij", X1, "ma", Rab, "ijab");             // -P(ab) Wovoo_mbij x_m^a
  // three-body parts of H-bar
  Z(w);
  C(1, K_LOV, "Pmf", X1, "mf", w, "P");
  Z(Xvv);
  C(1, K_LVV, "Pbe", w, "P", Xvv, "be");
  C(-1, K_LOV, "Pme", U, "Pbm", Xvv, "be");
  C(-0.5, K_OOVV, "mnef", X2, "mnbf", Xvv, "be");
  C(1, K_T2, "ijae", Xvv, "be", Rab, "ijab");
  Z(Xoo);
  // -P(ij) Fov_me t_mj^ab x_i^e = -P(ij) t_im^ab (Fov_me x_j^e) (t antisymmetric): one more
  // o x o matrix for the same contraction with t
  C(1, K_FOV, "me", X1, "je", Xoo, "mj");
  C(1, K_WOOOV, "mnje", X1, "ne", Xoo, "mj");
  C(0.5, K_OOVV, "mnef", X2, "jnef", Xoo, "mj");
  C(-1, K_T2, "imab", Xoo, "mj", Rij, "ijab");
  // antisymmetrisers P(ab), P(ij), P(ij)P(ab), applied in one pass
  {
    Op a{OP_ANTISYM, zc(1), -1, "", "", "", Rab, S2};
    a.in2 = Rij;
    a.in3 = Rijab;
    p.ops.push_back(a);
  }
  // exact projection onto antisymmetric doubles: the identity on exact results, it keeps the
  // rounding of the partial terms from leaving the antisymmetric subspace (self-adjoint)
  p.ops.push_back(Op{OP_PROJECT, zc(1), -1, "", "", "", -1, S2});
  (void)PM;
  return p;
}

}  // namespace cclr
