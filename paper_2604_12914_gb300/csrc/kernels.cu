// Generic device kernels of libcclr: strided complex GEMM on CUDA cores (FP64 DFMA and
// FP32 FFMA), arbitrary-stride permute/accumulate, and the HBM-bound vector kernels of the
// solver (axpy, bilinear and Hermitian dot products with FP64 accumulation, diagonal
// preconditioner, precision conversion).
#include "kernels.cuh"

#include <atomic>

namespace cclr {

static std::atomic<unsigned long long> g_launches{0};
unsigned long long launch_count() { return g_launches.load(); }
void count_launch(unsigned long long n) { g_launches += n; }

// --------------------------------------------------------------------------------------
// Complex GEMM, C[b](m,n) (+)= alpha * sum_k A[b](m,k) B[b](k,n); arbitrary strides.
// Tile BM x BN x BK, each thread TM x TN outputs (interleaved rows/cols to spread banks).
// --------------------------------------------------------------------------------------
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    zgemm_simt(GemmArgs g, int64_t b0) {
  using C = typename cpx<T>::t;
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int RX = BN / TN;  // threads along n
  constexpr int RY = BM / TM;  // threads along m
  __shared__ C As[BK][BM + 1];
  __shared__ C Bs[BK][BN + 1];

  const int64_t nMt = (g.M + BM - 1) / BM;
  const int64_t tile = blockIdx.x;
  const int64_t m0 = (tile % nMt) * BM;
  const int64_t n0 = (tile / nMt) * BN;
  const int64_t b = b0 + blockIdx.z;
  const C *A = (const C *)g.A + b * g.sAb;
  const C *B = (const C *)g.B + b * g.sBb;
  C *Cp = (C *)g.C + b * g.sCb;

  const int tid = threadIdx.x;
  const int tx = tid % RX, ty = tid / RX;
  C acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = C{T(0), T(0)};

  const bool a_kfast = (g.sAk == 1);
  const bool b_nfast = (g.sBn == 1);
  for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      int64_t m = m0 + mm, k = k0 + kk;
      C val = C{T(0), T(0)};
      if (m < g.M && k < g.K) val = A[m * g.sAm + k * g.sAk];
      As[kk][mm] = val;
    }
#pragma unroll
    for (int e = tid; e < BN * BK; e += NT) {
      int nn, kk;
      if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      int64_t n = n0 + nn, k = k0 + kk;
      C val = C{T(0), T(0)};
      if (n < g.N && k < g.K) val = B[k * g.sBk + n * g.sBn];
      Bs[kk][nn] = val;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * RY];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + j * RX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          acc[i][j].x = fma(a[i].x, bb[j].x, acc[i][j].x);
          acc[i][j].x = fma(-a[i].y, bb[j].y, acc[i][j].x);
          acc[i][j].y = fma(a[i].x, bb[j].y, acc[i][j].y);
          acc[i][j].y = fma(a[i].y, bb[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }
  const T ar = (T)g.alr, ai = (T)g.ali;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t m = m0 + ty + i * RY;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t n = n0 + tx + j * RX;
      if (n >= g.N) continue;
      C *dst = Cp + m * g.sCm + n * g.sCn;
      C v = acc[i][j];
      C r;
      r.x = ar * v.x - ai * v.y;
      r.y = ar * v.y + ai * v.x;
      if (!g.overwrite) {
        C o = *dst;
        r.x += o.x;
        r.y += o.y;
      }
      *dst = r;
    }
  }
}

void launch_gemm(const GemmArgs &g, int dt, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return;
  if (g.K <= 0) {
    CCLR_REQUIRE(!g.overwrite, "gemm with K=0 and overwrite is not supported");
    return;
  }
  for (int64_t b0 = 0; b0 < g.batch; b0 += 65535) {
    int64_t nb = std::min<int64_t>(65535, g.batch - b0);
    if (dt == C128) {
      constexpr int BM = 64, BN = 64, BK = 8;
      int64_t tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
      dim3 grid((unsigned)tiles, 1, (unsigned)nb);
      zgemm_simt<double, BM, BN, BK, 4, 4><<<grid, 256, 0, st>>>(g, b0);
    } else {
      constexpr int BM = 64, BN = 64, BK = 16;
      int64_t tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
      dim3 grid((unsigned)tiles, 1, (unsigned)nb);
      zgemm_simt<float, BM, BN, BK, 4, 4><<<grid, 256, 0, st>>>(g, b0);
    }
    count_launch();
    CCLR_CUDA(cudaGetLastError());
  }
}

// --------------------------------------------------------------------------------------
// Permute / accumulate: out[idx] = alpha * in[perm idx] (+ out[idx]).  Iterates in the
// order of the output's own mode list (rank <= 8); strides in elements.
// --------------------------------------------------------------------------------------
template <typename TI, typename TO>
__global__ void permute_kernel(PermArgs a) {
  using CI = typename cpx<TI>::t;
  using CO = typename cpx<TO>::t;
  const CI *in = (const CI *)a.in;
  CO *out = (CO *)a.out;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e, oi = 0, oo = 0;
#pragma unroll
    for (int d = 7; d >= 0; --d) {
      if (d >= a.rank) continue;
      int64_t c = r % a.dim[d];
      r /= a.dim[d];
      oi += c * a.sin[d];
      oo += c * a.sout[d];
    }
    CI v = in[oi];
    double vr = (double)v.x, vi = (double)v.y;
    double wr = a.alr * vr - a.ali * vi;
    double wi = a.alr * vi + a.ali * vr;
    CO res;
    if (a.acc) {
      CO o = out[oo];
      res.x = (TO)(wr + (double)o.x);
      res.y = (TO)(wi + (double)o.y);
    } else {
      res.x = (TO)wr;
      res.y = (TO)wi;
    }
    out[oo] = res;
  }
}

void launch_permute(const PermArgs &a, int dt_in, int dt_out, cudaStream_t st) {
  if (a.total <= 0) return;
  int threads = 256;
  int64_t blocks = std::min<int64_t>((a.total + threads - 1) / threads, 152 * 32);
  if (dt_in == C128 && dt_out == C128) permute_kernel<double, double><<<(unsigned)blocks, threads, 0, st>>>(a);
  else if (dt_in == C64 && dt_out == C64) permute_kernel<float, float><<<(unsigned)blocks, threads, 0, st>>>(a);
  else if (dt_in == C128 && dt_out == C64) permute_kernel<double, float><<<(unsigned)blocks, threads, 0, st>>>(a);
  else permute_kernel<float, double><<<(unsigned)blocks, threads, 0, st>>>(a);
  count_launch();
    CCLR_CUDA(cudaGetLastError());
}

// --------------------------------------------------------------------------------------
// Vector kernels (contiguous complex arrays).
// --------------------------------------------------------------------------------------
template <typename T>
__global__ void axpy_kernel(int64_t n, double ar, double ai, const typename cpx<T>::t *x,
                            typename cpx<T>::t *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    auto xv = x[i];
    auto yv = y[i];
    yv.x += (T)(ar * xv.x - ai * xv.y);
    yv.y += (T)(ar * xv.y + ai * xv.x);
    y[i] = yv;
  }
}

template <typename T>
__global__ void scal_kernel(int64_t n, double ar, double ai, typename cpx<T>::t *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    auto v = y[i];
    typename cpx<T>::t r;
    r.x = (T)(ar * v.x - ai * v.y);
    r.y = (T)(ar * v.y + ai * v.x);
    y[i] = r;
  }
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

void vec_axpy(int dt, int64_t n, zc a, const void *x, void *y, cudaStream_t st) {
  if (n <= 0) return;
  if (dt == C128) axpy_kernel<double><<<grid_for(n), 256, 0, st>>>(n, a.re, a.im, (const double2 *)x, (double2 *)y);
  else axpy_kernel<float><<<grid_for(n), 256, 0, st>>>(n, a.re, a.im, (const float2 *)x, (float2 *)y);
  count_launch();
    CCLR_CUDA(cudaGetLastError());
}

void vec_scal(int dt, int64_t n, zc a, void *y, cudaStream_t st) {
  if (n <= 0) return;
  if (dt == C128) scal_kernel<double><<<grid_for(n), 256, 0, st>>>(n, a.re, a.im, (double2 *)y);
  else scal_kernel<float><<<grid_for(n), 256, 0, st>>>(n, a.re, a.im, (float2 *)y);
  count_launch();
    CCLR_CUDA(cudaGetLastError());
}

// Dot products with FP64 accumulation: mode 0 bilinear sum x*y, mode 1 Hermitian
// sum conj(x)*y.  Two passes (block partials, then one block) for a deterministic result.
template <typename T>
__global__ void dot_partial(int64_t n, const typename cpx<T>::t *x, const typename cpx<T>::t *y,
                            int herm, double2 *part) {
  double sr = 0.0, si = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double xr = x[i].x, xi = herm ? -(double)x[i].y : (double)x[i].y;
    double yr = y[i].x, yi = y[i].y;
    sr += xr * yr - xi * yi;
    si += xr * yi + xi * yr;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  __shared__ double rs[32], is[32];
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { rs[w] = sr; is[w] = si; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x / 32;
    sr = l < nw ? rs[l] : 0.0;
    si = l < nw ? is[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, o);
      si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (l == 0) part[blockIdx.x] = make_double2(sr, si);
  }
}

__global__ void dot_final(int nb, const double2 *part, double2 *out, int slot) {
  double sr = 0.0, si = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    sr += part[i].x;
    si += part[i].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  __shared__ double rs[32], is[32];
  int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { rs[w] = sr; is[w] = si; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x / 32;
    sr = l < nw ? rs[l] : 0.0;
    si = l < nw ? is[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, o);
      si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (l == 0) out[slot] = make_double2(sr, si);
  }
}

void vec_dot(int dt, int64_t n, const void *x, const void *y, int herm, double2 *part,
             double2 *out, int slot, cudaStream_t st) {
  const int nb = 304;
  if (n <= 0) {
    CCLR_CUDA(cudaMemsetAsync(out + slot, 0, sizeof(double2), st));
    return;
  }
  if (dt == C128) dot_partial<double><<<nb, 256, 0, st>>>(n, (const double2 *)x, (const double2 *)y, herm, part);
  else dot_partial<float><<<nb, 256, 0, st>>>(n, (const float2 *)x, (const float2 *)y, herm, part);
  dot_final<<<1, 256, 0, st>>>(nb, part, out, slot);
  count_launch(2);
    CCLR_CUDA(cudaGetLastError());
}

// Delta = r / (D - omega), D real; in place allowed.
template <typename T>
__global__ void precond_kernel(int64_t n, const double *D, double omega,
                               const typename cpx<T>::t *r, typename cpx<T>::t *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = D[i] - omega;
    if (fabs(d) < 1e-8) d = d < 0 ? -1e-8 : 1e-8;
    auto v = r[i];
    typename cpx<T>::t o;
    o.x = (T)(v.x / d);
    o.y = (T)(v.y / d);
    out[i] = o;
  }
}

void vec_precond(int dt, int64_t n, const double *D, double omega, const void *r, void *out,
                 cudaStream_t st) {
  if (n <= 0) return;
  if (dt == C128) precond_kernel<double><<<grid_for(n), 256, 0, st>>>(n, D, omega, (const double2 *)r, (double2 *)out);
  else precond_kernel<float><<<grid_for(n), 256, 0, st>>>(n, D, omega, (const float2 *)r, (float2 *)out);
  count_launch();
    CCLR_CUDA(cudaGetLastError());
}

// D1[i,a] = Fvv_aa - Foo_ii ; D2[i,j,a,b] = Fvv_aa + Fvv_bb - Foo_ii - Foo_jj (real parts).
__global__ void diag_kernel(int o, int v, const double2 *Foo, const double2 *Fvv, double *D1,
                            double *D2) {
  int64_t n1 = (int64_t)o * v, n2 = n1 * o * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n1 + n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < n1) {
      int i = (int)(e / v), a = (int)(e % v);
      D1[e] = Fvv[(int64_t)a * v + a].x - Foo[(int64_t)i * o + i].x;
    } else {
      int64_t r = e - n1;
      int b = (int)(r % v); r /= v;
      int a = (int)(r % v); r /= v;
      int j = (int)(r % o); r /= o;
      int i = (int)r;
      D2[e - n1] = Fvv[(int64_t)a * v + a].x + Fvv[(int64_t)b * v + b].x -
                   Foo[(int64_t)i * o + i].x - Foo[(int64_t)j * o + j].x;
    }
  }
}

void build_diag(int o, int v, const void *Foo, const void *Fvv, double *D1, double *D2,
                cudaStream_t st) {
  int64_t n = (int64_t)o * v * (1 + (int64_t)o * v);
  diag_kernel<<<grid_for(n), 256, 0, st>>>(o, v, (const double2 *)Foo, (const double2 *)Fvv, D1, D2);
  count_launch();
    CCLR_CUDA(cudaGetLastError());
}

// t2[i,j,a,b] = w[i,j,a,b] / (e_i + e_j - e_a - e_b)
__global__ void denom_kernel(int o, int v, const double *eps, double2 *t2) {
  int64_t n = (int64_t)o * o * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e;
    int b = (int)(r % v); r /= v;
    int a = (int)(r % v); r /= v;
    int j = (int)(r % o); r /= o;
    int i = (int)r;
    double d = eps[i] + eps[j] - eps[o + a] - eps[o + b];
    double2 x = t2[e];
    t2[e] = make_double2(x.x / d, x.y / d);
  }
}

void apply_denominator(int o, int v, const double *eps, void *t2, cudaStream_t st) {
  int64_t n = (int64_t)o * o * v * v;
  denom_kernel<<<grid_for(n), 256, 0, st>>>(o, v, eps, (double2 *)t2);
  count_launch();
    CCLR_CUDA(cudaGetLastError());
}

// out[p,q] = value on the diagonal (complex128 square matrix), used for diag(eps).
__global__ void set_diag_kernel(int n, const double *d, double2 *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[(int64_t)i * n + i] = make_double2(d[i], 0.0);
}

void set_diag(int n, const double *d, void *out, cudaStream_t st) {
  set_diag_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, d, (double2 *)out);
  count_launch();
    CCLR_CUDA(cudaGetLastError());
}

}  // namespace cclr
