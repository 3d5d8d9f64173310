// Packed particle-particle ladder on tcgen05 tensor cores; see ladder_tc.cuh.
#include <vector>

#include "ladder_tc.cuh"
#include "tc_gemm.cuh"

namespace cclr {
namespace {

// Packed X as the contraction B operand over the pairs q0 .. q0 + nq - 1:
// B(k = (e<f) - q0, n = (i<j)) = X[i,j,e,f].
template <int KIND>
__global__ void pack_x_b(const float2 *X, int o, int v, const int2 *op, const int2 *vp, int64_t Po,
                         int64_t q0, int64_t nq, int64_t Kp, int seg, typename TcElem<KIND>::T *dst, int64_t ldd) {
  const int64_t total = Po * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = e / Kp, k = e % Kp;
    float2 val = make_float2(0.f, 0.f);
    if (k < nq) {
      const int2 ij = op[n], ef = vp[q0 + k];
      val = X[(((int64_t)ij.x * o + ij.y) * v + ef.x) * v + ef.y];
    }
    tc_put_b<KIND>(dst + (2 * n) * ldd, dst + (2 * n + 1) * ldd, k, Kp, seg, val);
  }
}

// Y (transpose direction) as the A operand over a group of (a<b) pairs:
// A(m = (i<j), k = r) = Y[i,j,a,b] - Y[j,i,a,b] - Y[i,j,b,a] + Y[j,i,b,a], (a,b) = pair(p0 + r).
template <int KIND>
__global__ void pack_y_a(const float2 *Y, int o, int v, const int2 *op, const int2 *vp, int64_t Po,
                         int64_t p0, int64_t np, int64_t Kp, int seg, typename TcElem<KIND>::T *dst, int64_t ldd) {
  const int64_t total = Po * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / Kp, k = e % Kp;
    float2 val = make_float2(0.f, 0.f);
    if (k < np) {
      const int2 ij = op[m], ab = vp[p0 + k];
      const int64_t i = ij.x, j = ij.y, a = ab.x, b = ab.y;
      const float2 y1 = Y[((i * o + j) * v + a) * v + b], y2 = Y[((j * o + i) * v + a) * v + b];
      const float2 y3 = Y[((i * o + j) * v + b) * v + a], y4 = Y[((j * o + i) * v + b) * v + a];
      val = make_float2(y1.x - y2.x - y3.x + y4.x, y1.y - y2.y - y3.y + y4.y);
    }
    tc_put_a<KIND>(dst + m * ldd, k, Kp, seg, val);
  }
}

// Antisymmetrised packed block of the group, from W[(b - a0) v + f][(a - a0) v + e] = <ab|ef>~:
//   <ab||ef>~ = W[(b-a0)v+f][(a-a0)v+e] - W[(b-a0)v+e][(a-a0)v+f],  a in group, b > a, e < f,
// for the (e<f) pairs q0 .. q0 + nq - 1 (q below is the pair's offset from q0).
// mode 0: A operand rows r = (a,b) pair - p0, K = q          (forward contraction)
// mode 1: B operand rows 2q, 2q+1, K = r                      (transpose contraction)
template <int KIND>
__global__ void pack_w(const float2 *W, int64_t ldw, int v, int a0, const int2 *vp, int64_t p0,
                       int64_t np, int64_t q0, int64_t nq, int64_t Kp, int seg, int mode, typename TcElem<KIND>::T *dst,
                       int64_t ldd) {
  const int64_t total = mode == 0 ? np * Kp : nq * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r, q;  // r: (a,b) pair within the group; q: (e<f) pair offset
    if (mode == 0) { r = e / Kp; q = e % Kp; } else { q = e / Kp; r = e % Kp; }
    const bool inside = mode == 0 ? (q < nq) : (r < np);
    float2 val = make_float2(0.f, 0.f);
    if (inside) {
      const int2 ab = vp[p0 + r], ef = vp[q0 + q];
      const int64_t rb = (int64_t)(ab.y - a0) * v, ca = (int64_t)(ab.x - a0) * v;
      const float2 w1 = W[(rb + ef.y) * ldw + ca + ef.x];
      const float2 w2 = W[(rb + ef.x) * ldw + ca + ef.y];
      val = make_float2(w1.x - w2.x, w1.y - w2.y);
    }
    if (mode == 0) tc_put_a<KIND>(dst + r * ldd, q, Kp, seg, val);
    else tc_put_b<KIND>(dst + (2 * q) * ldd, dst + (2 * q + 1) * ldd, r, Kp, seg, val);
  }
}

// out[i,j,a,b] += alpha * S[(ab) * lds + (ij)] with the four antisymmetric images (S rows (a<b),
// columns (i<j)).
// By orbit tiles: one block takes a 32 x 32 tile of (a, b) with a-block <= b-block and
// SIG_TN consecutive (i<j) pairs; it reads S[(ab)][(ij) .. (ij) + SIG_TN) (one 32-byte run per pair
// (ab)) into shared memory, then writes the four images out[i,j,a,b], out[j,i,a,b] (along b) and
// out[i,j,b,a], out[j,i,b,a] (along a, through the transposed shared tile), each coalesced.  Every
// unordered (a, b) belongs to one tile and every (i<j) to one chunk, so no two blocks touch one entry.
constexpr int SIG_TN = 4;
__global__ void __launch_bounds__(256) unpack_sig_tiled(const float2 *__restrict__ S, int64_t lds, int o, int v,
                                                        const int2 *__restrict__ op, int64_t Po, int nbv, float ar,
                                                        float ai, float2 *__restrict__ out) {
  __shared__ float2 T[SIG_TN][32][33];
  // tile (A, B), A <= B, from blockIdx.x in row order of the upper triangle of nbv x nbv blocks
  int A = 0, t = blockIdx.x;
  while (t >= nbv - A) { t -= nbv - A; ++A; }
  const int B = A + t;
  const int a0 = A * 32, b0 = B * 32, tx = threadIdx.x, ty = threadIdx.y;
  const int64_t n0 = (int64_t)blockIdx.y * SIG_TN;
  const int nn = Po - n0 < SIG_TN ? (int)(Po - n0) : SIG_TN;
  for (int al = ty; al < 32; al += 8) {
    const int a = a0 + al, b = b0 + tx;
    const bool in = a < b && b < v;
    const int64_t k = in ? ((int64_t)a * v - (int64_t)a * (a + 1) / 2 + b - a - 1) : 0;
    for (int q = 0; q < SIG_TN; ++q) {
      float2 s = make_float2(0.f, 0.f);
      if (in && q < nn) {
        const float2 z = S[k * lds + n0 + q];
        s = make_float2(ar * z.x - ai * z.y, ar * z.y + ai * z.x);
      }
      T[q][al][tx] = s;
    }
  }
  __syncthreads();
  for (int q = 0; q < nn; ++q) {
    const int2 ij = op[n0 + q];
    const int64_t rij = ((int64_t)ij.x * o + ij.y) * v, rji = ((int64_t)ij.y * o + ij.x) * v;
    for (int rl = ty; rl < 32; rl += 8) {
      {  // (a = a0 + rl, b = b0 + tx): images (ij, ab) and (ji, ab)
        const int a = a0 + rl, b = b0 + tx;
        if (a < b && b < v) {
          const float2 val = T[q][rl][tx];
          float2 *p = out + (rij + a) * v + b;
          float2 w = *p;
          w.x += val.x; w.y += val.y;
          *p = w;
          p = out + (rji + a) * v + b;
          w = *p;
          w.x -= val.x; w.y -= val.y;
          *p = w;
        }
      }
      {  // (b = b0 + rl, a = a0 + tx): images (ij, ba) and (ji, ba)
        const int b = b0 + rl, a = a0 + tx;
        if (a < b && b < v) {
          const float2 val = T[q][tx][rl];
          float2 *p = out + (rij + b) * v + a;
          float2 w = *p;
          w.x -= val.x; w.y -= val.y;
          *p = w;
          p = out + (rji + b) * v + a;
          w = *p;
          w.x += val.x; w.y += val.y;
          *p = w;
        }
      }
    }
  }
}

void launch_unpack_sig(const float2 *S, int64_t lds, int o, int v, const int2 *op, int64_t Po, float ar, float ai,
                       float2 *out, cudaStream_t st) {
  if (Po == 0 || v < 2) return;
  const int nbv = (v + 31) / 32;
  const int64_t ny = (Po + SIG_TN - 1) / SIG_TN;
  CCLR_REQUIRE(ny < 65536, "unpack_sig: too many occupied pairs for the grid");
  unpack_sig_tiled<<<dim3((unsigned)(nbv * (nbv + 1) / 2), (unsigned)ny), dim3(32, 8), 0, st>>>(S, lds, o, v, op, Po,
                                                                                              nbv, ar, ai, out);
  count_launch();
}

// out[i,j,e,f] += alpha * Z[(ij)][(ef)] for i<j, e<f only (Z rows of Pv).
__global__ void unpack_z(const float2 *Z, int o, int v, const int2 *op, const int2 *vp, int64_t Po,
                         int64_t Pv, float ar, float ai, float2 *out) {
  const int64_t total = Po * Pv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = e / Pv, k = e % Pv;
    const int2 ij = op[n], ef = vp[k];
    const float2 z = Z[n * Pv + k];
    float2 *p = out + (((int64_t)ij.x * o + ij.y) * v + ef.x) * v + ef.y;
    p->x += ar * z.x - ai * z.y;
    p->y += ar * z.y + ai * z.x;
  }
}

unsigned grid1d(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
}

std::vector<int2> pairs(int n) {
  std::vector<int2> t;
  t.reserve((size_t)n * (n - 1) / 2);
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q) t.push_back(make_int2(p, q));
  return t;
}

int64_t pair_start(int v, int a) { return (int64_t)a * v - (int64_t)a * (a + 1) / 2; }

}  // namespace

void ladder_unpack_sig_bench(int o, int v, const void *S, void *out, cudaStream_t st) {
  static thread_local DevBuf opairs, vpairs;
  static thread_local int po = -1, pv = -1;
  const int64_t Po = (int64_t)o * (o - 1) / 2, Pv = (int64_t)v * (v - 1) / 2;
  if (po != o || pv != v) {
    auto op = pairs(o), vp = pairs(v);
    opairs.alloc(op.size() * sizeof(int2));
    vpairs.alloc(vp.size() * sizeof(int2));
    CCLR_CUDA(cudaMemcpy(opairs.p, op.data(), op.size() * sizeof(int2), cudaMemcpyHostToDevice));
    CCLR_CUDA(cudaMemcpy(vpairs.p, vp.data(), vp.size() * sizeof(int2), cudaMemcpyHostToDevice));
    po = o;
    pv = v;
  }
  launch_unpack_sig((const float2 *)S, Po, o, v, opairs.as<int2>(), Po, 1.f, 0.f, (float2 *)out, st);
  CCLR_CUDA(cudaGetLastError());
}

void LadderTC::prepare(Engine &E, const Tens &Lvv, int o, int v, int naux, int seg, int kind, bool lean) {
  cudaStream_t st = E.st;
  wall_ready_ = false;  // a stored block belongs to the previous L~_vv
  o_ = o; v_ = v; naux_ = naux; seg_ = seg; kind_ = kind;
  Po_ = (int64_t)o * (o - 1) / 2;
  Pv_ = (int64_t)v * (v - 1) / 2;
  const int64_t ld = 2 * tc_kpad(naux) * seg, es = tc_esize(kind);
  const int64_t vv = (int64_t)v * v;
  Lvv_ = Lvv.p;
  LA.alloc((size_t)vv * ld * es);
  // A(m = (b,f), k = P) = L[P,b,f]
  tc_prep_a(Lvv.p, 1, vv, vv, naux, seg, kind, LA.p, ld, st);
  // B(k = P, n = (a,e)) = L[P,a,e], embedded (two rows per complex column): prepared here for every
  // a when it takes at most 3 GB (it is the same for every product with this L~_vv), else per group
  // inside each product
  const size_t lb_all = (size_t)2 * vv * ld * es;
  lb_all_ = !lean && lb_all <= (size_t)3 << 30;
  if (lb_all_) {
    if (LB.bytes != lb_all) LB.alloc(lb_all);
    tc_prep_b(Lvv.p, vv, 1, naux, vv, seg, kind, LB.p, ld, st);
  } else {
    LB.release();
  }
  auto op = pairs(o), vp = pairs(v);
  opairs.alloc(std::max<size_t>(1, op.size()) * sizeof(int2));
  vpairs.alloc(std::max<size_t>(1, vp.size()) * sizeof(int2));
  if (!op.empty()) CCLR_CUDA(cudaMemcpyAsync(opairs.p, op.data(), op.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  if (!vp.empty()) CCLR_CUDA(cudaMemcpyAsync(vpairs.p, vp.data(), vp.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  CCLR_CUDA(cudaStreamSynchronize(st));
  if (lean) {
    ga_ = 1;
    for (int cand : {2, 4, 8, 16, 32, 64})
      if ((double)v * v * std::min(cand, v) * v * 8 <= 4e9) ga_ = std::min(cand, v);
    tuned_ = true;
    tune_log.clear();
  } else if (!tuned_) {
    tune(E);
  }
}

void LadderTC::tune(Engine &E) {
  tuned_ = true;
  tune_log.clear();
  if (Po_ == 0 || Pv_ == 0) return;
  cudaStream_t st = E.st;
  const int64_t n2 = (int64_t)o_ * o_ * v_ * v_;
  DevBuf xin((size_t)n2 * 8), xout((size_t)n2 * 8);
  CCLR_CUDA(cudaMemsetAsync(xin.p, 0, xin.bytes, st));
  cudaEvent_t e0, e1;
  CCLR_CUDA(cudaEventCreate(&e0));
  CCLR_CUDA(cudaEventCreate(&e1));
  const void *in[1] = {xin.p};
  void *out[1] = {xout.p};
  int best = ga_;
  float best_ms = 1e30f;
  const bool store_saved = store_;
  store_ = false;  // the tuner times the on-the-fly formation
  for (int cand : {8, 16, 32, 64}) {
    const int ga = std::min(cand, v_);
    // the group block W [(v - a0) v][ga v] complex64: at most 8 GB (the smallest group always)
    const double wbytes = (double)v_ * v_ * ga * v_ * 8;
    if (cand > 8 && wbytes > 8e9) continue;
    if (!tune_log.empty() && tune_log.back().first == ga) continue;
    ga_ = ga;
    apply(E, +1, zc(1.0), 1, in, out);  // the first run allocates the group buffers
    CCLR_CUDA(cudaEventRecord(e0, st));
    apply(E, +1, zc(1.0), 1, in, out);
    CCLR_CUDA(cudaEventRecord(e1, st));
    CCLR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    CCLR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    tune_log.push_back({ga, ms});
    if (ms < best_ms) { best_ms = ms; best = ga; }
    // buffers sized for this candidate are released before the next one
    W.release(); Wp.release(); Xp.release(); sig.release();
  }
  ga_ = best;
  store_ = store_saved;
  CCLR_CUDA(cudaEventDestroy(e0));
  CCLR_CUDA(cudaEventDestroy(e1));
}

void LadderTC::apply(Engine &E, int dir, zc alpha, int nrhs, const void *const *in, void *const *out) {
  cudaStream_t st = E.st;
  const int o = o_, v = v_, seg = seg_, kind = kind_;
  const int64_t Po = Po_, Pv = Pv_;
  if (Po == 0 || Pv == 0 || nrhs < 1) return;
  const int64_t vv = (int64_t)v * v, es = tc_esize(kind);
  const int64_t ldL = 2 * tc_kpad(naux_) * seg;
  const int ga = std::min(ga_, v);
  const int64_t NR = (int64_t)nrhs;
  const bool use_wall = store_ && dir > 0;
  // buffers sized for the first (largest) group
  const int64_t maxpairs = pair_start(v, ga);
  const int64_t kpg = tc_kpad(maxpairs);
  // the (e<f) pairs in chunks of QC, so that a packed block (rows of the group's pairs, or
  // rows of the chunk's pairs in the transpose) stays within 2 GiB; the stored ablation keeps one
  const int64_t cap = 2ll << 30;
  int64_t QC = use_wall ? Pv : std::max<int64_t>(64, cap / (4 * std::max<int64_t>(kpg, 1) * seg * es) / 8 * 8);
  QC = std::min(QC, Pv);
  const int64_t nch = (Pv + QC - 1) / QC, Kc = tc_kpad(QC), ldc = 2 * Kc * seg;
  if (W.bytes < (size_t)vv * ga * v * 8) W.alloc((size_t)vv * ga * v * 8);
  if (!lb_all_ && LB.bytes < (size_t)2 * ga * v * ldL * es) LB.alloc((size_t)2 * ga * v * ldL * es);
  const size_t wp_bytes = dir > 0 ? (size_t)maxpairs * ldc * es : (size_t)2 * QC * (2 * kpg * seg) * es;
  if (Wp.bytes < wp_bytes) Wp.alloc(wp_bytes);
  const size_t xp_bytes = dir > 0 ? (size_t)nch * 2 * Po * NR * ldc * es : (size_t)Po * NR * (2 * kpg * seg) * es;
  if (Xp.bytes < xp_bytes) Xp.alloc(xp_bytes);
  if (sig.bytes < (size_t)Po * Pv * NR * 8) sig.alloc((size_t)Po * Pv * NR * 8);
  const int2 *op = opairs.as<int2>(), *vp = vpairs.as<int2>();
  char *LAb = (char *)LA.p, *LBb = (char *)LB.p, *Wpb = (char *)Wp.p, *Xpb = (char *)Xp.p;
  const size_t xchunk = (size_t)2 * Po * NR * ldc * es;  // bytes of one chunk of packed X
  nform_ = 0;
  if (dir > 0) {
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t q0 = c * QC, nq = std::min(QC, Pv - q0);
      for (int64_t r = 0; r < NR; ++r) {
        void *dst = Xpb + c * xchunk + 2 * Po * r * ldc * es;
        if (kind == TC_BF16)
          pack_x_b<TC_BF16><<<grid1d(Po * Kc), 256, 0, st>>>((const float2 *)in[r], o, v, op, vp, Po, q0, nq, Kc, seg,
                                                              (__nv_bfloat16 *)dst, ldc);
        else
          pack_x_b<TC_TF32><<<grid1d(Po * Kc), 256, 0, st>>>((const float2 *)in[r], o, v, op, vp, Po, q0, nq, Kc, seg,
                                                              (float *)dst, ldc);
        count_launch();
      }
    }
  } else {
    CCLR_CUDA(cudaMemsetAsync(sig.p, 0, (size_t)Po * Pv * NR * 8, st));
  }
  if (use_wall && !wall_ready_) {
    const size_t wall_bytes = (size_t)Pv * ldc * es;
    if (Wall.bytes != wall_bytes) Wall.alloc(wall_bytes);
  }
  // pack_w launch into dst (rows of ldd elements of the mode's operand type)
  auto packw = [&](int a0, int64_t p0, int64_t np, int64_t q0, int64_t nq, int64_t cols, int64_t Kp, int mode,
                   void *dst, int64_t ldd) {
    const int64_t total = mode == 0 ? np * Kp : nq * Kp;
    if (kind == TC_BF16)
      pack_w<TC_BF16><<<grid1d(total), 256, 0, st>>>(W.as<float2>(), cols, v, a0, vp, p0, np, q0, nq, Kp, seg, mode,
                                                     (__nv_bfloat16 *)dst, ldd);
    else
      pack_w<TC_TF32><<<grid1d(total), 256, 0, st>>>(W.as<float2>(), cols, v, a0, vp, p0, np, q0, nq, Kp, seg, mode,
                                                     (float *)dst, ldd);
    count_launch();
  };
  for (int a0 = 0; a0 < v - 1 && !(use_wall && wall_ready_); a0 += ga) {
    const int a1 = std::min(v, a0 + ga);
    const int64_t p0 = pair_start(v, a0), np = pair_start(v, a1) - p0;
    if (np == 0) continue;
    // formation: W[(b - a0, f)][(a - a0, e)] = sum_P L[P,b,f] L[P,a,e], b >= a0
    const int64_t rows = (int64_t)(v - a0) * v, cols = (int64_t)(a1 - a0) * v;
    if ((int)fev.size() < 2 * (nform_ + 1)) {
      fev.resize(2 * (nform_ + 1), nullptr);
      for (auto &e : fev)
        if (!e) CCLR_CUDA(cudaEventCreate(&e));
    }
    // B(k = P, n = (a,e)) = L[P,a,e] for the group's a values, embedded (already prepared for
    // every a when lb_all_)
    const char *LBg = LBb + (lb_all_ ? (size_t)2 * a0 * v * ldL * es : 0);
    if (!lb_all_) tc_prep_b((const char *)Lvv_ + (size_t)a0 * v * 8, vv, 1, naux_, cols, seg, kind, LBb, ldL, st);
    CCLR_CUDA(cudaEventRecord(fev[2 * nform_], st));
    tc_gemm_seg(LAb + (int64_t)a0 * v * ldL * es, ldL, LBg, ldL, rows, 2 * cols, ldL / seg, seg, kind, W.as<float>(),
                2 * cols, zc(1.0), false, st);
    CCLR_CUDA(cudaEventRecord(fev[2 * nform_ + 1], st));
    ++nform_;
    if (use_wall) {  // pack the group's rows into the stored block; contract once afterwards
      packw(a0, p0, np, 0, Pv, cols, Kc, 0, (char *)Wall.p + p0 * ldc * es, ldc);
    } else if (dir > 0) {
      // sigT[(ab)][(r, ij)] = sum_{e<f} <ab||ef>~ X_r[i,j,e,f] for the group's pairs, all RHS, summed
      // over the chunks of (e<f)
      for (int64_t c = 0; c < nch; ++c) {
        const int64_t q0 = c * QC, nq = std::min(QC, Pv - q0);
        packw(a0, p0, np, q0, nq, cols, Kc, 0, Wpb, ldc);
        tc_gemm_seg(Wpb, ldc, Xpb + c * xchunk, ldc, np, 2 * Po * NR, ldc / seg, seg, kind,
                    sig.as<float>() + 2 * p0 * Po * NR, 2 * Po * NR, zc(1.0), c > 0, st);
      }
    } else {
      const int64_t kg = tc_kpad(np), ldg = 2 * kg * seg;
      for (int64_t r = 0; r < NR; ++r) {
        void *dst = Xpb + Po * r * ldg * es;
        if (kind == TC_BF16)
          pack_y_a<TC_BF16><<<grid1d(Po * kg), 256, 0, st>>>((const float2 *)in[r], o, v, op, vp, Po, p0, np, kg, seg,
                                                              (__nv_bfloat16 *)dst, ldg);
        else
          pack_y_a<TC_TF32><<<grid1d(Po * kg), 256, 0, st>>>((const float2 *)in[r], o, v, op, vp, Po, p0, np, kg, seg,
                                                              (float *)dst, ldg);
        count_launch();
      }
      // Z[(r, ij)][(ef)] += sum_{(ab) in group} Y'_r[(ij)][(ab)] <ab||ef>~, a chunk of (e<f) at a time
      for (int64_t c = 0; c < nch; ++c) {
        const int64_t q0 = c * QC, nq = std::min(QC, Pv - q0);
        packw(a0, p0, np, q0, nq, cols, kg, 1, Wpb, ldg);
        tc_gemm_seg(Xpb, ldg, Wpb, ldg, Po * NR, 2 * nq, ldg / seg, seg, kind, sig.as<float>() + 2 * q0, 2 * Pv,
                    zc(1.0), true, st);
      }
    }
    CCLR_CUDA(cudaGetLastError());
  }
  if (use_wall) {
    wall_ready_ = true;
    // sigT[(ab)][(r, ij)] = sum_{e<f} <ab||ef>~ X_r[i,j,e,f] for every pair at once (one chunk)
    tc_gemm_seg(Wall.p, ldc, Xpb, ldc, Pv, 2 * Po * NR, ldc / seg, seg, kind, sig.as<float>(), 2 * Po * NR, zc(1.0),
                false, st);
    CCLR_CUDA(cudaGetLastError());
  }
  for (int64_t r = 0; r < NR; ++r) {
    if (dir > 0) {
      launch_unpack_sig(sig.as<float2>() + Po * r, Po * NR, o, v, op, Po, (float)alpha.re, (float)alpha.im,
                        (float2 *)out[r], st);
    } else {
      unpack_z<<<grid1d(Po * Pv), 256, 0, st>>>(sig.as<float2>() + Po * Pv * r, o, v, op, vp, Po, Pv,
                                                 (float)alpha.re, (float)alpha.im, (float2 *)out[r]);
      count_launch();
    }
  }
  CCLR_CUDA(cudaGetLastError());
}

float LadderTC::formation_ms() {
  float tot = 0.f;
  for (int g = 0; g < nform_; ++g) {
    float ms = 0.f;
    CCLR_CUDA(cudaEventElapsedTime(&ms, fev[2 * g], fev[2 * g + 1]));
    tot += ms;
  }
  return tot;
}

}  // namespace cclr
