// tcgen05 tensor-core GEMM (TF32 inputs, FP32 accumulation in TMEM) and the operand
// preparation that maps complex products onto it.
//
// Real kernel:   D[m][n] = sum_k A[m][k] * B[n][k]     (A, B row-major, K contiguous)
// Complex use:   C[M][N] = A[M][K] . B[K][N] (complex64) becomes one real GEMM with
//   A_real = A as interleaved (re, im) pairs, [M][2K]            (no transformation)
//   B_real rows 2n, 2n+1 = (Re b_kn, -Im b_kn), (Im b_kn, Re b_kn) over k, [2N][2K]
// so that D[m][2n] = Re C[m][n] and D[m][2n+1] = Im C[m][n]: the FP32 output is already
// the interleaved complex result (4 real multiplies per complex multiply-add).
// 3xTF32 (split) mode: x = hi + lo with hi rounded to TF32; A_real = [hi | hi | lo],
// B_real = [hi | lo | hi] along K gives hi.hi + hi.lo + lo.hi (about FP32 accuracy).
#pragma once
#include "kernels.cuh"

namespace cclr {

// Two-level strided index view: offset(i) = (i / din) * sout + (i % din) * sin (elements).
// One level: din = TC_ONE_LEVEL, sout = 0.
constexpr int64_t TC_ONE_LEVEL = (int64_t)1 << 62;
struct View2 {
  int64_t din = TC_ONE_LEVEL, sout = 0, sin = 1;
};
__host__ __device__ __forceinline__ int64_t v2off(const View2 &v, int64_t i) {
  if (v.din == TC_ONE_LEVEL) return i * v.sin;
  if (i < 0x7fffffff && v.din < 0x7fffffff) {  // 32-bit division where it suffices
    const uint32_t q = (uint32_t)i / (uint32_t)v.din, r = (uint32_t)i - q * (uint32_t)v.din;
    return (int64_t)q * v.sout + (int64_t)r * v.sin;
  }
  return (i / v.din) * v.sout + (i % v.din) * v.sin;
}
inline View2 view1(int64_t stride) {
  View2 v;
  v.sin = stride;
  return v;
}

// Complex K padded so that every operand row is a whole number of 16-byte units.
inline int64_t tc_kpad(int64_t K) { return (K + 1) / 2 * 2; }

// seg = 1 (TF32) or 3 (3xTF32 split).  dst rows have ldd floats (>= 2*tc_kpad(K)*seg).
void tc_prep_a(const void *A, int64_t sam, int64_t sak, int64_t M, int64_t K, int seg, float *dst,
               int64_t ldd, cudaStream_t st);
void tc_prep_b(const void *B, int64_t sbk, int64_t sbn, int64_t K, int64_t N, int seg, float *dst,
               int64_t ldd, cudaStream_t st);
// the same reading A(m, k) at v2off(mv, m) + v2off(kv, k) (B(k, n) likewise)
void tc_prep_a2(const void *A, View2 mv, View2 kv, int64_t M, int64_t K, int seg, float *dst, int64_t ldd,
                cudaStream_t st);
void tc_prep_b2(const void *B, View2 kv, View2 nv, int64_t K, int64_t N, int seg, float *dst, int64_t ldd,
                cudaStream_t st);

// Real tensor-core GEMM; C is written as complex pairs: C[m][n..n+1] (+)= alpha * D[m][n..n+1]
// for even n.  Nreal must be even; lda/ldb multiples of 4 floats; A, B 16-byte aligned.
void tc_gemm(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t M, int64_t Nreal,
             int64_t Kreal, float *C, int64_t ldc_floats, zc alpha, bool accumulate, cudaStream_t st);

// Complex GEMM on prepared operands with seg segments of Kseg floats each (Kseg = 2*Kp).
// seg = 1: one pass.  seg = 3: the correction terms hi.lo + lo.hi (segments 1-2) and the
// main term hi.hi (segment 0) run as two passes with separate TMEM accumulators, summed
// into C in FP32 by the epilogues.
void tc_gemm_seg(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t M, int64_t Nreal,
                 int64_t Kseg, int seg, float *C, int64_t ldc_floats, zc alpha, bool accumulate,
                 cudaStream_t st);
// TF32 GEMM whose A is read in place: complex64 rows of K contiguous elements, lda_cpx complex
// elements apart (no prepared copy; TF32 needs no split of A).  tc_a_inplace_ok tells whether
// the TMA rules allow it (16-byte aligned base, row pitch a multiple of 16 bytes).
bool tc_a_inplace_ok(const void *A, int64_t lda_cpx, int64_t K);
void tc_gemm_a_inplace(const void *A, int64_t lda_cpx, int64_t K, const float *B, int64_t ldb, int64_t M,
                       int64_t Nreal, float *C, View2 rv, View2 cv, zc alpha, bool accumulate, cudaStream_t st);

// The same GEMM for callers that hold their own device error flag (it must start at zero;
// a bounded wait that gives up sets it to 1).  Neither function allocates device memory:
// tc_setup_device_flagged fetches the tensor-map encoder and raises the kernel's dynamic
// shared-memory limit on the current device, and must be called once per device first.
void tc_setup_device_flagged();
void tc_gemm_seg_flagged(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t M, int64_t Nreal,
                         int64_t Kseg, int seg, float *C, int64_t ldc_floats, zc alpha, bool accumulate,
                         int *err, cudaStream_t st);
// the same with C addressed through views of its rows and its complex columns
// (complex element (m, n) at C + 2 * (v2off(rv, m) + v2off(cv, n)) floats)
void tc_gemm_seg_v(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t M, int64_t Nreal,
                   int64_t Kseg, int seg, float *C, View2 rv, View2 cv, zc alpha, bool accumulate,
                   cudaStream_t st);

// Reads (and clears) the device-side error flag of the tensor-core kernels: 0 = fine,
// 1 = a bounded wait gave up.
int tc_error(cudaStream_t st);

// Runs the bounded-wait give-up path once (a wait nothing completes); returns the flag.
int tc_selftest_timeout(int timeout_us, cudaStream_t st);

}  // namespace cclr
