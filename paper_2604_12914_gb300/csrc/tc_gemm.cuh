// tcgen05 tensor-core GEMM (TF32 or BF16 inputs, FP32 accumulation in TMEM) and the operand
// preparation that maps complex products onto it.
//
// Real kernel:   D[m][n] = sum_k A[m][k] * B[n][k]     (A, B row-major, K contiguous)
// Complex use:   C[M][N] = A[M][K] . B[K][N] (complex64) becomes one real GEMM with
//   A_real = A as interleaved (re, im) pairs, [M][2K]            (no transformation)
//   B_real rows 2n, 2n+1 = (Re b_kn, -Im b_kn), (Im b_kn, Re b_kn) over k, [2N][2K]
// so that D[m][2n] = Re C[m][n] and D[m][2n+1] = Im C[m][n]: the FP32 output is already
// the interleaved complex result (4 real multiplies per complex multiply-add).
// Split modes (seg = 3): x = hi + lo with hi the operand type's rounding of x and lo the
// rounding of x - hi; A_real = [hi | hi | lo], B_real = [hi | lo | hi] along K gives
// hi.hi + hi.lo + lo.hi.  With TF32 operands (3xTF32) that is about FP32 accuracy; with BF16
// operands (bf16x3, the three-product split of Henry, Tang and Heinecke, ARITH 2019) about
// 2^-16 relative, at the BF16 rate (twice the TF32 rate).
#pragma once
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace cclr {

// Operand type of the tensor-core GEMM: TF32 (kind::tf32, FP32 storage) or BF16 (kind::f16).
enum TcKind { TC_TF32 = 0, TC_BF16 = 1 };
inline int64_t tc_esize(int kind) { return kind == TC_BF16 ? 2 : 4; }

template <int KIND> struct TcElem;
template <> struct TcElem<TC_TF32> { using T = float; };
template <> struct TcElem<TC_BF16> { using T = __nv_bfloat16; };

// TF32 rounding: the 13 dropped mantissa bits rounded to nearest (ties away from zero)
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}

// one stored operand value (single pass) and the (hi, lo) split
template <int KIND> __device__ __forceinline__ typename TcElem<KIND>::T tc_one(float x);
template <> __device__ __forceinline__ float tc_one<TC_TF32>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 tc_one<TC_BF16>(float x) { return __float2bfloat16_rn(x); }
template <int KIND> __device__ __forceinline__ void tc_split(float x, typename TcElem<KIND>::T &h, typename TcElem<KIND>::T &l);
template <> __device__ __forceinline__ void tc_split<TC_TF32>(float x, float &h, float &l) {
  h = tf32_round(x);
  l = x - h;
}
template <> __device__ __forceinline__ void tc_split<TC_BF16>(float x, __nv_bfloat16 &h, __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));
}

// complex value v as element k of an A-format row (K-major; [hi | hi | lo] when seg = 3)
template <int KIND>
__device__ __forceinline__ void tc_put_a(typename TcElem<KIND>::T *row, int64_t k, int64_t Kp, int seg, float2 v) {
  if (seg == 1) {
    row[2 * k] = tc_one<KIND>(v.x);
    row[2 * k + 1] = tc_one<KIND>(v.y);
  } else {
    typename TcElem<KIND>::T hr, lr, hi, li;
    tc_split<KIND>(v.x, hr, lr);
    tc_split<KIND>(v.y, hi, li);
    row[2 * k] = hr; row[2 * k + 1] = hi;
    row[2 * Kp + 2 * k] = hr; row[2 * Kp + 2 * k + 1] = hi;
    row[4 * Kp + 2 * k] = lr; row[4 * Kp + 2 * k + 1] = li;
  }
}

// complex value v as element k of the embedded B rows r0 (re, -im), r1 (im, re) ([hi | lo | hi])
template <int KIND>
__device__ __forceinline__ void tc_put_b(typename TcElem<KIND>::T *r0, typename TcElem<KIND>::T *r1, int64_t k,
                                         int64_t Kp, int seg, float2 v) {
  if (seg == 1) {
    const auto re = tc_one<KIND>(v.x), im = tc_one<KIND>(v.y), mim = tc_one<KIND>(-v.y);
    r0[2 * k] = re; r0[2 * k + 1] = mim; r1[2 * k] = im; r1[2 * k + 1] = re;
  } else {
    typename TcElem<KIND>::T hr, lr, hi, li, nhi, nli;
    tc_split<KIND>(v.x, hr, lr);
    tc_split<KIND>(v.y, hi, li);
    tc_split<KIND>(-v.y, nhi, nli);
    r0[2 * k] = hr; r0[2 * k + 1] = nhi; r1[2 * k] = hi; r1[2 * k + 1] = hr;
    r0[2 * Kp + 2 * k] = lr; r0[2 * Kp + 2 * k + 1] = nli; r1[2 * Kp + 2 * k] = li; r1[2 * Kp + 2 * k + 1] = lr;
    r0[4 * Kp + 2 * k] = hr; r0[4 * Kp + 2 * k + 1] = nhi; r1[4 * Kp + 2 * k] = hi; r1[4 * Kp + 2 * k + 1] = hr;
  }
}

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

// Complex K padded so that every operand row is a whole number of 16-byte units for every
// operand type and split (2 K seg elements of 2 or 4 bytes: K a multiple of 4).
inline int64_t tc_kpad(int64_t K) { return (K + 3) / 4 * 4; }

// seg = 1 (one pass) or 3 (split); kind = TC_TF32 or TC_BF16.  dst rows have ldd elements of
// the operand type (>= 2*tc_kpad(K)*seg).
void tc_prep_a(const void *A, int64_t sam, int64_t sak, int64_t M, int64_t K, int seg, int kind, void *dst,
               int64_t ldd, cudaStream_t st);
void tc_prep_b(const void *B, int64_t sbk, int64_t sbn, int64_t K, int64_t N, int seg, int kind, void *dst,
               int64_t ldd, cudaStream_t st);
// the same reading A(m, k) at v2off(mv, m) + v2off(kv, k) (B(k, n) likewise)
void tc_prep_a2(const void *A, View2 mv, View2 kv, int64_t M, int64_t K, int seg, int kind, void *dst, int64_t ldd,
                cudaStream_t st);
void tc_prep_b2(const void *B, View2 kv, View2 nv, int64_t K, int64_t N, int seg, int kind, void *dst, int64_t ldd,
                cudaStream_t st);

// Real tensor-core GEMM; C is written as complex pairs: C[m][n..n+1] (+)= alpha * D[m][n..n+1]
// for even n.  Nreal must be even; lda/ldb multiples of 4 floats; A, B 16-byte aligned.
void tc_gemm(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t M, int64_t Nreal,
             int64_t Kreal, float *C, int64_t ldc_floats, zc alpha, bool accumulate, cudaStream_t st);

// Complex GEMM on prepared operands (elements of the operand type kind) with seg segments of
// Kseg elements each (Kseg = 2*Kp).  seg = 1: one pass.  seg = 3: the correction terms
// hi.lo + lo.hi (segments 1-2) and the main term hi.hi (segment 0) run as two passes with
// separate TMEM accumulators, summed into C in FP32 by the epilogues.
void tc_gemm_seg(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int64_t Nreal, int64_t Kseg,
                 int seg, int kind, float *C, int64_t ldc_floats, zc alpha, bool accumulate, cudaStream_t st);
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
void tc_gemm_seg_v(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int64_t Nreal, int64_t Kseg,
                   int seg, int kind, float *C, View2 rv, View2 cv, zc alpha, bool accumulate, cudaStream_t st);

// Tile autotuner: while on (per host thread), the first use of a GEMM shape (operand kind, M,
// real N, real K, epilogue layout) on a device times a handful of launch configurations (tile
// width, K splits, raster band) around the rules' choice and caches the fastest for that shape
// and device; later uses launch the cached configuration.  Never tunes inside a stream capture.
void tc_set_autotune(bool on);
// Rows of 10 doubles per tuned shape of the current device (kind, M, N, K, BN, splits, band,
// best ms, the rule's ms, candidates timed), up to cap rows; returns the number of shapes.
int tc_tuning_table(int cap, double *rec);

// Reads (and clears) the device-side error flag of the tensor-core kernels: 0 = fine,
// 1 = a bounded wait gave up.
int tc_error(cudaStream_t st);

// Runs the bounded-wait give-up path once (a wait nothing completes); returns the flag.
int tc_selftest_timeout(int timeout_us, cudaStream_t st);

}  // namespace cclr
