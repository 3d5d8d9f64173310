// cc_lr_selftest_gemm_noalloc: the tensor-core GEMM self-test of cc_lr_selftest_gemm, run
// without allocating any device memory.
//
// Who needs it.  Some host programs give nearly all of a device's memory to their own
// caching pool when they start and account for every byte through it.  A library that calls
// cudaMalloc after that either fails for lack of room or takes memory behind the pool's back,
// and cudaFree makes the whole device wait for outstanding work.  Such a program still wants
// to check, on the device it was given, that this library's tensor-core GEMM gives correct
// numbers before it trusts the results.  This entry point does that with no cudaMalloc,
// cudaFree or allocating library call: every buffer lives in one fixed array in device
// global memory, declared below, whose size is the limit on M, N and K.
//
// Set-up: the first call on a device, with that device current, looks the array up with
// cudaGetSymbolAddress, fetches the tensor-map encoder and raises the GEMM kernel's
// shared-memory limit.  Later calls on that device reuse the result.  All calls on a device
// share the one array, so calls that overlap on the GPU (from two host threads at once) race
// and give wrong answers; the call itself is synchronous.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <random>
#include <string>

#include "../../include/cclr.h"
#include "../../include/cclr_testing.h"
#include "kernels.cuh"
#include "tc_gemm.cuh"

namespace cclr {
int record_error(int status, const std::string &msg);
}

using namespace cclr;

// The only memory this entry point uses on the device (one copy per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[CCLR_SELFTEST_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_base[kMaxDevices] = {};

// Base address of the array on the current device; the first call per device does the set-up.
unsigned char *device_scratch() {
  int dev = 0;
  CCLR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Error(CCLR_EUNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_base[dev]) {
    unsigned char *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      (void)cudaGetLastError();
      throw Error(CCLR_EDEVICE, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                    cudaGetErrorString(e));
    }
    tc_setup_device_flagged();
    g_base[dev] = ptr;
  }
  return g_base[dev];
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the buffers inside the array.
struct Layout {
  size_t flag, a128, b128, c128, a64, b64, ct, cs, ao, bo, total;
  int64_t ld;
};

Layout plan(int64_t M, int64_t N, int64_t K, int seg) {
  Layout l;
  l.ld = 2 * tc_kpad(K) * seg;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += up256(bytes);
    return at;
  };
  l.flag = take(sizeof(int));
  l.a128 = take((size_t)M * K * 16);
  l.b128 = take((size_t)K * N * 16);
  l.c128 = take((size_t)M * N * 16);
  l.a64 = take((size_t)M * K * 8);
  l.b64 = take((size_t)K * N * 8);
  l.ct = take((size_t)M * N * 8);
  l.cs = take((size_t)M * N * 8);
  l.ao = take((size_t)M * l.ld * 4);
  l.bo = take((size_t)2 * N * l.ld * 4);
  l.total = off;
  return l;
}

// Copies n doubles of the generator's stream to dst, a stack chunk at a time.
template <typename Gen, typename Dist>
void fill_normal(Gen &g, Dist &nd, double *dst, size_t n, cudaStream_t s) {
  double chunk[4096];
  for (size_t i = 0; i < n; i += 4096) {
    const size_t m = std::min<size_t>(4096, n - i);
    for (size_t k = 0; k < m; ++k) chunk[k] = nd(g);
    CCLR_CUDA(cudaMemcpyAsync(dst + i, chunk, m * sizeof(double), cudaMemcpyHostToDevice, s));
    CCLR_CUDA(cudaStreamSynchronize(s));
  }
}

void gemm_plain(int dt, const void *A, const void *B, void *C, int64_t M, int64_t N, int64_t K,
                cudaStream_t s) {
  GemmArgs g;
  g.A = A; g.B = B; g.C = C;
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.sAm = K; g.sAk = 1;
  g.sBk = N; g.sBn = 1;
  g.sCm = N; g.sCn = 1;
  g.overwrite = 0;
  launch_gemm(g, dt, s);
}

void narrow(const void *in, void *out, int64_t n, cudaStream_t s) {
  PermArgs a;
  a.in = in; a.out = out;
  a.rank = 1; a.dim[0] = n; a.sin[0] = 1; a.sout[0] = 1;
  a.total = n;
  launch_permute(a, C128, C64, s);
}

}  // namespace

extern "C" int cc_lr_selftest_gemm_noalloc(int M, int N, int K, int mode, unsigned seed, double *err) {
  if (M < 1 || N < 1 || K < 1 || (mode != 1 && mode != 2) || !err)
    return record_error(CCLR_EINVAL, "bad selftest_gemm_noalloc arguments");
  const int seg = mode == 2 ? 3 : 1;
  // the bound is checked in floating point first, so that huge sizes cannot overflow
  const double approx = 48.0 * ((double)M * K + (double)K * N) + 48.0 * (double)M * N +
                        24.0 * ((double)M + 2.0 * N) * ((double)K + 64.0) * seg + 4096.0;
  if (approx > 4.0 * (double)CCLR_SELFTEST_NOALLOC_SCRATCH_BYTES ||
      plan(M, N, K, seg).total > (size_t)CCLR_SELFTEST_NOALLOC_SCRATCH_BYTES) {
    char need[64];
    if (approx > 4.0 * (double)CCLR_SELFTEST_NOALLOC_SCRATCH_BYTES)
      snprintf(need, sizeof need, "%.4g", approx);
    else
      snprintf(need, sizeof need, "%zu", plan(M, N, K, seg).total);
    return record_error(CCLR_EINVAL, "selftest_gemm_noalloc: M=" + std::to_string(M) + " N=" + std::to_string(N) +
                                         " K=" + std::to_string(K) + " needs about " + need +
                                         " bytes of scratch; the fixed device array holds " +
                                         std::to_string((size_t)CCLR_SELFTEST_NOALLOC_SCRATCH_BYTES));
  }
  try {
    const Layout l = plan(M, N, K, seg);
    unsigned char *base = device_scratch();
    cudaStream_t s = cudaStreamPerThread;
    auto at = [&](size_t off) { return (void *)(base + off); };
    // inputs: the same seeded stream as cc_lr_selftest_gemm (A then B, row-major complex)
    std::mt19937_64 g(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    fill_normal(g, nd, (double *)at(l.a128), (size_t)2 * M * K, s);
    fill_normal(g, nd, (double *)at(l.b128), (size_t)2 * K * N, s);
    // what must start at zero on every call: the wait flag and the three accumulated products
    CCLR_CUDA(cudaMemsetAsync(at(l.flag), 0, sizeof(int), s));
    CCLR_CUDA(cudaMemsetAsync(at(l.c128), 0, (size_t)M * N * 16, s));
    CCLR_CUDA(cudaMemsetAsync(at(l.ct), 0, (size_t)M * N * 8, s));
    CCLR_CUDA(cudaMemsetAsync(at(l.cs), 0, (size_t)M * N * 8, s));
    narrow(at(l.a128), at(l.a64), (int64_t)M * K, s);
    narrow(at(l.b128), at(l.b64), (int64_t)K * N, s);
    gemm_plain(C128, at(l.a128), at(l.b128), at(l.c128), M, N, K, s);  // FP64 reference
    tc_prep_a(at(l.a64), K, 1, M, K, seg, TC_TF32, at(l.ao), l.ld, s);
    tc_prep_b(at(l.b64), N, 1, K, N, seg, TC_TF32, at(l.bo), l.ld, s);
    tc_gemm_seg_flagged((const float *)at(l.ao), l.ld, (const float *)at(l.bo), l.ld, M, 2 * (int64_t)N,
                        2 * tc_kpad(K), seg, (float *)at(l.ct), 2 * (int64_t)N, zc(1.0), true, (int *)at(l.flag), s);
    gemm_plain(C64, at(l.a64), at(l.b64), at(l.cs), M, N, K, s);  // FP32 CUDA cores
    int flag = 0;
    CCLR_CUDA(cudaMemcpyAsync(&flag, at(l.flag), sizeof(int), cudaMemcpyDeviceToHost, s));
    CCLR_CUDA(cudaStreamSynchronize(s));
    if (flag) throw Error(CCLR_ETIMEOUT, "tensor-core kernel gave up on a bounded wait");
    // max |C_x - C_ref| / max |C_ref| over real and imaginary parts, a stack chunk at a time
    double r[2048];
    float t[2048], q[2048];
    double mx = 0, e1 = 0, e2 = 0;
    const size_t n = (size_t)2 * M * N;
    for (size_t i = 0; i < n; i += 2048) {
      const size_t m = std::min<size_t>(2048, n - i);
      CCLR_CUDA(cudaMemcpyAsync(r, (const double *)at(l.c128) + i, m * 8, cudaMemcpyDeviceToHost, s));
      CCLR_CUDA(cudaMemcpyAsync(t, (const float *)at(l.ct) + i, m * 4, cudaMemcpyDeviceToHost, s));
      CCLR_CUDA(cudaMemcpyAsync(q, (const float *)at(l.cs) + i, m * 4, cudaMemcpyDeviceToHost, s));
      CCLR_CUDA(cudaStreamSynchronize(s));
      for (size_t k = 0; k < m; ++k) {
        mx = std::max(mx, std::abs(r[k]));
        e1 = std::max(e1, std::abs(r[k] - (double)t[k]));
        e2 = std::max(e2, std::abs(r[k] - (double)q[k]));
      }
    }
    err[0] = e1 / mx;
    err[1] = e2 / mx;
    return CCLR_OK;
  } catch (const Error &e) {
    return record_error(e.status, e.what());
  } catch (const std::exception &e) {
    return record_error(CCLR_EDEVICE, e.what());
  }
}
