// Packed particle-particle ladder on the CUDA cores; see ladder_cc.cuh.
#include <vector>

#include "ladder_cc.cuh"

namespace cclr {
namespace {

template <typename T> using C2 = typename cpx<T>::t;

unsigned grid1d(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
}

// Xp[q = (e<f)][r * Po + n] = X_r[i,j,e,f], n = (i<j)
template <typename T>
__global__ void cc_pack_x(const C2<T> *X, int o, int v, const int2 *op, const int2 *vp, int64_t Po, int64_t Pv,
                          int64_t ldx, C2<T> *dst) {
  const int64_t total = Po * Pv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / Po, n = e % Po;
    const int2 ij = op[n], ef = vp[q];
    dst[q * ldx + n] = X[(((int64_t)ij.x * o + ij.y) * v + ef.x) * v + ef.y];
  }
}

// Y'[r * Po + m][k] = Y[i,j,a,b] - Y[j,i,a,b] - Y[i,j,b,a] + Y[j,i,b,a], (a,b) = pair p0 + k
template <typename T>
__global__ void cc_pack_y(const C2<T> *Y, int o, int v, const int2 *op, const int2 *vp, int64_t Po, int64_t p0,
                          int64_t np, C2<T> *dst) {
  const int64_t total = Po * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / np, k = e % np;
    const int2 ij = op[m], ab = vp[p0 + k];
    const int64_t i = ij.x, j = ij.y, a = ab.x, b = ab.y;
    const C2<T> y1 = Y[((i * o + j) * v + a) * v + b], y2 = Y[((j * o + i) * v + a) * v + b];
    const C2<T> y3 = Y[((i * o + j) * v + b) * v + a], y4 = Y[((j * o + i) * v + b) * v + a];
    C2<T> r;
    r.x = y1.x - y2.x - y3.x + y4.x;
    r.y = y1.y - y2.y - y3.y + y4.y;
    dst[m * np + k] = r;
  }
}

// Wp[r][q] = W[(b-a0)v+f][(a-a0)v+e] - W[(b-a0)v+e][(a-a0)v+f], (a,b) = pair p0 + r, (e,f) = pair q
template <typename T>
__global__ void cc_pack_w(const C2<T> *W, int64_t ldw, int v, int a0, const int2 *vp, int64_t p0, int64_t np,
                          int64_t Pv, C2<T> *dst) {
  const int64_t total = np * Pv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Pv, q = e % Pv;
    const int2 ab = vp[p0 + r], ef = vp[q];
    const int64_t rb = (int64_t)(ab.y - a0) * v, ca = (int64_t)(ab.x - a0) * v;
    const C2<T> w1 = W[(rb + ef.y) * ldw + ca + ef.x], w2 = W[(rb + ef.x) * ldw + ca + ef.y];
    C2<T> d;
    d.x = w1.x - w2.x;
    d.y = w1.y - w2.y;
    dst[e] = d;
  }
}

// out[i,j,a,b] += alpha * S[(ab) * lds + (ij)] with the four antisymmetric images
template <typename T>
__global__ void cc_unpack_sig(const C2<T> *S, int64_t lds, int o, int v, const int2 *op, const int2 *vp, int64_t Po,
                              int64_t Pv, T ar, T ai, C2<T> *out) {
  const int64_t total = Po * Pv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = e / Pv, k = e % Pv;
    const int2 ij = op[n], ab = vp[k];
    const C2<T> s = S[k * lds + n];
    const T vr = ar * s.x - ai * s.y, vi = ar * s.y + ai * s.x;
    const int64_t i = ij.x, j = ij.y, a = ab.x, b = ab.y;
    C2<T> *p;
    p = out + ((i * o + j) * v + a) * v + b; p->x += vr; p->y += vi;
    p = out + ((j * o + i) * v + a) * v + b; p->x -= vr; p->y -= vi;
    p = out + ((i * o + j) * v + b) * v + a; p->x -= vr; p->y -= vi;
    p = out + ((j * o + i) * v + b) * v + a; p->x += vr; p->y += vi;
  }
}

// out[i,j,e,f] += alpha * Z[(r, ij)][(ef)] for i<j, e<f only
template <typename T>
__global__ void cc_unpack_z(const C2<T> *Z, int o, int v, const int2 *op, const int2 *vp, int64_t Po, int64_t Pv,
                            T ar, T ai, C2<T> *out) {
  const int64_t total = Po * Pv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = e / Pv, k = e % Pv;
    const int2 ij = op[n], ef = vp[k];
    const C2<T> z = Z[n * Pv + k];
    C2<T> *p = out + (((int64_t)ij.x * o + ij.y) * v + ef.x) * v + ef.y;
    p->x += ar * z.x - ai * z.y;
    p->y += ar * z.y + ai * z.x;
  }
}

std::vector<int2> pairs(int n) {
  std::vector<int2> t;
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q) t.push_back(make_int2(p, q));
  return t;
}

int64_t pair_start(int v, int a) { return (int64_t)a * v - (int64_t)a * (a + 1) / 2; }

}  // namespace

void LadderCC::apply(Engine &E, int dt, const Tens &Lvv, int o, int v, int naux, int dir, zc alpha, int nrhs,
                     const void *const *in, void *const *out) {
  cudaStream_t st = E.st;
  const int64_t Po = (int64_t)o * (o - 1) / 2, Pv = (int64_t)v * (v - 1) / 2;
  if (Po == 0 || Pv == 0 || nrhs < 1) return;
  if (o != o_ || v != v_) {
    auto op = pairs(o), vp = pairs(v);
    opairs.alloc(op.size() * sizeof(int2));
    vpairs.alloc(vp.size() * sizeof(int2));
    CCLR_CUDA(cudaMemcpyAsync(opairs.p, op.data(), op.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CCLR_CUDA(cudaMemcpyAsync(vpairs.p, vp.data(), vp.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CCLR_CUDA(cudaStreamSynchronize(st));
    o_ = o;
    v_ = v;
  }
  const size_t es = dt_size(dt);
  const int ga = std::min(kGroup, v);
  const int64_t NR = nrhs, vv = (int64_t)v * v;
  const int64_t maxpairs = pair_start(v, ga);
  if (W.bytes < (size_t)vv * ga * v * es) W.alloc((size_t)vv * ga * v * es);
  if (Wp.bytes < (size_t)maxpairs * Pv * es) Wp.alloc((size_t)maxpairs * Pv * es);
  const size_t xp = dir > 0 ? (size_t)Pv * NR * Po * es : (size_t)NR * Po * maxpairs * es;
  if (Xp.bytes < xp) Xp.alloc(xp);
  const size_t sg = dir > 0 ? (size_t)Pv * NR * Po * es : (size_t)NR * Po * Pv * es;
  if (sig.bytes < sg) sig.alloc(sg);
  const int2 *op = opairs.as<int2>(), *vp = vpairs.as<int2>();
  const bool f64 = dt == C128;
  if (dir > 0) {
    for (int64_t r = 0; r < NR; ++r) {
      if (f64)
        cc_pack_x<double><<<grid1d(Po * Pv), 256, 0, st>>>((const double2 *)in[r], o, v, op, vp, Po, Pv, NR * Po,
                                                         Xp.as<double2>() + r * Po);
      else
        cc_pack_x<float><<<grid1d(Po * Pv), 256, 0, st>>>((const float2 *)in[r], o, v, op, vp, Po, Pv, NR * Po,
                                                        Xp.as<float2>() + r * Po);
      count_launch();
    }
  } else {
    CCLR_CUDA(cudaMemsetAsync(sig.p, 0, sg, st));
  }
  for (int a0 = 0; a0 < v - 1; a0 += ga) {
    const int a1 = std::min(v, a0 + ga);
    const int64_t p0 = pair_start(v, a0), np = pair_start(v, a1) - p0;
    if (np == 0) continue;
    // formation: W[(b - a0, f)][(a - a0, e)] = sum_P L[P,b,f] L[P,a,e], b >= a0
    const int64_t rows = (int64_t)(v - a0) * v, cols = (int64_t)(a1 - a0) * v;
    GemmArgs g;
    g.A = (const char *)Lvv.p + (size_t)a0 * v * es;
    g.sAm = 1; g.sAk = vv;
    g.B = (const char *)Lvv.p + (size_t)a0 * v * es;
    g.sBk = vv; g.sBn = 1;
    g.C = W.p;
    g.sCm = cols; g.sCn = 1;
    g.M = rows; g.N = cols; g.K = naux;
    g.overwrite = 1;
    launch_gemm(g, dt, st);
    if (f64)
      cc_pack_w<double><<<grid1d(np * Pv), 256, 0, st>>>(W.as<double2>(), cols, v, a0, vp, p0, np, Pv, Wp.as<double2>());
    else
      cc_pack_w<float><<<grid1d(np * Pv), 256, 0, st>>>(W.as<float2>(), cols, v, a0, vp, p0, np, Pv, Wp.as<float2>());
    count_launch();
    if (dir > 0) {
      // sig[(ab)][(r, ij)] = sum_{e<f} <ab||ef>~ X_r[i,j,e,f] for the group's pairs
      GemmArgs c;
      c.A = Wp.p; c.sAm = Pv; c.sAk = 1;
      c.B = Xp.p; c.sBk = NR * Po; c.sBn = 1;
      c.C = (char *)sig.p + (size_t)p0 * NR * Po * es;
      c.sCm = NR * Po; c.sCn = 1;
      c.M = np; c.N = NR * Po; c.K = Pv;
      c.overwrite = 1;
      launch_gemm(c, dt, st);
    } else {
      for (int64_t r = 0; r < NR; ++r) {
        if (f64)
          cc_pack_y<double><<<grid1d(Po * np), 256, 0, st>>>((const double2 *)in[r], o, v, op, vp, Po, p0, np,
                                                             Xp.as<double2>() + r * Po * np);
        else
          cc_pack_y<float><<<grid1d(Po * np), 256, 0, st>>>((const float2 *)in[r], o, v, op, vp, Po, p0, np,
                                                            Xp.as<float2>() + r * Po * np);
        count_launch();
      }
      // Z[(r, ij)][(ef)] += sum_{(ab) in group} Y'_r[(ij)][(ab)] <ab||ef>~
      GemmArgs c;
      c.A = Xp.p; c.sAm = np; c.sAk = 1;
      c.B = Wp.p; c.sBk = Pv; c.sBn = 1;
      c.C = sig.p; c.sCm = Pv; c.sCn = 1;
      c.M = NR * Po; c.N = Pv; c.K = np;
      c.overwrite = 0;
      launch_gemm(c, dt, st);
    }
  }
  for (int64_t r = 0; r < NR; ++r) {
    if (dir > 0) {
      if (f64)
        cc_unpack_sig<double><<<grid1d(Po * Pv), 256, 0, st>>>(sig.as<double2>() + r * Po, NR * Po, o, v, op, vp, Po,
                                                              Pv, alpha.re, alpha.im, (double2 *)out[r]);
      else
        cc_unpack_sig<float><<<grid1d(Po * Pv), 256, 0, st>>>(sig.as<float2>() + r * Po, NR * Po, o, v, op, vp, Po, Pv,
                                                             (float)alpha.re, (float)alpha.im, (float2 *)out[r]);
    } else {
      if (f64)
        cc_unpack_z<double><<<grid1d(Po * Pv), 256, 0, st>>>(sig.as<double2>() + r * Po * Pv, o, v, op, vp, Po, Pv,
                                                            alpha.re, alpha.im, (double2 *)out[r]);
      else
        cc_unpack_z<float><<<grid1d(Po * Pv), 256, 0, st>>>(sig.as<float2>() + r * Po * Pv, o, v, op, vp, Po, Pv,
                                                           (float)alpha.re, (float)alpha.im, (float2 *)out[r]);
    }
    count_launch();
  }
  CCLR_CUDA(cudaGetLastError());
}

}  // namespace cclr
