/*
 * cclr_testing.h -- self-test entry points of libcclr (not part of the response API).
 */
#ifndef CCLR_TESTING_H
#define CCLR_TESTING_H

#ifdef __cplusplus
extern "C" {
#endif

/* Complex64 GEMM C[M][N] = A[M][K] B[K][N] on seeded random data, computed three ways
 * on the current device: tcgen05 tensor cores (mode 1 TF32, mode 2 3xTF32, mode 3 bf16x3),
 * FP32 CUDA cores, and FP64 CUDA cores (reference).  Writes max|C_x - C_ref| / max|C_ref| for the
 * tensor-core (err[0]) and FP32 (err[1]) results.  Returns 0 on success, else a
 * cclr_status code. */
int cc_lr_selftest_gemm(int M, int N, int K, int mode, unsigned seed, double *err);

/* Times the tensor-core complex GEMM C[M][N] = A[M][K] B[K][N] (operand preparation
 * excluded) on seeded data: reps launches, CUDA events; ms[0] = mean milliseconds per
 * GEMM, ms[1] = the corresponding TFLOP/s at 8 real flops per complex multiply-add. */
int cc_lr_bench_gemm(int M, int N, int K, int mode, int reps, double *ms);

/* Times the HBM-bound kernels of the solver and the sigma program at o occupied and v virtual
 * spinors on device buffers of those sizes (contents: zeros; the time does not depend on them):
 * reps launches each, CUDA events.  Writes for k = 0..min(n, 8)-1 the pair
 * (out[2k] = milliseconds per launch, out[2k+1] = algorithmic bytes per launch), in the order
 *   0 antisym_apply    complex64 S += P(ab) Rab + P(ij) Rij + P(ij)P(ab) R4 (3 reads, S read+write)
 *   1 antisym_project  complex64 in-place projection of S (read + write)
 *   2 unpack_doubles   packed complex128 -> full complex64 (packed read, full write)
 *   3 pack_doubles     full complex64 -> packed complex128 (the i<j, a<b entries read, packed write)
 *   4 vec_precond      packed complex128 r / (D - w) (r and D read, result written)
 *   5 vec_dot          packed complex128 Hermitian dot, FP64 accumulation (two reads)
 *   6 vec_axpy         packed complex128 y += a x (x, y read, y written)
 *   7 unpack_sig       pp-ladder result scattered to the four antisymmetric images (complex64)
 * Returns 0 on success, else a cclr_status code. */
int cc_lr_bench_hbm(int o, int v, int reps, double *out, int n);

/* Size in bytes of the fixed device array that cc_lr_selftest_gemm_noalloc works in (32 MiB).
 * The array is part of the library's device code: loading the library reserves it on every
 * device the process uses, whether or not the entry point is ever called, and it is not part
 * of any context's HBM budget (cc_lr_memory does not count it). */
#define CCLR_SELFTEST_NOALLOC_SCRATCH_BYTES 33554432ull

/* cc_lr_selftest_gemm without any device allocation.  The paper has no counterpart: this
 * entry point exists for host programs that cannot let a library call cudaMalloc or cudaFree
 * -- typically because they hand nearly all device memory to their own caching pool at start-up
 * and account for every byte through it, so a stray cudaMalloc fails or escapes the pool, and
 * cudaFree would make the whole device wait.  It computes the same products on the same
 * seeded data and writes the same err[0] (tcgen05 tensor cores, mode 1 TF32 or 2 3xTF32) and
 * err[1] (FP32 CUDA cores), both relative to the FP64 result.
 *   Memory: every buffer (inputs in FP64 and complex64, the three products, the staged
 *   tensor-core operands and the bounded-wait flag) lives in one file-scope device array of
 *   CCLR_SELFTEST_NOALLOC_SCRATCH_BYTES; sizes that do not fit return CCLR_EINVAL (1) and a
 *   message naming the bytes needed (cc_lr_last_error).  About 24(MK + KN) + 32MN +
 *   8(M + 2N)(K + 1)s bytes are needed, s = 1 for TF32 and 3 for 3xTF32; M = N = K = 384
 *   fits with 3xTF32.  Nothing is allocated: no cudaMalloc, no cudaFree, no allocating
 *   library routine; host staging uses fixed stack buffers.
 *   Set-up: the first call on each device (with that device current) looks the array up with
 *   cudaGetSymbolAddress and prepares the tensor-core kernel; make that first call before
 *   any stream capture begins.
 *   Sharing: all calls on a device use the same array, and each call clears what must start
 *   at zero (the flag and the products) itself.  Calls that overlap on the GPU -- two host
 *   threads calling at once on one device -- race on the array and give wrong results;
 *   callers must serialise them.  The call is synchronous (it runs on the calling thread's
 *   per-thread default stream and waits for it).
 * Returns 0 on success, else a cclr_status code. */
int cc_lr_selftest_gemm_noalloc(int M, int N, int K, int mode, unsigned seed, double *err);

/* The diagonal preconditioner out = r / (D - (omega + i omega_im)) on n seeded complex128 entries
 * (D uniform in [0.1, 20], r normal), whose kernel forms the FP64 reciprocal by Newton-Raphson
 * iteration from the FP32 reciprocal: writes max |out - r/(D - z)| / |r/(D - z)| over the entries,
 * the reference quotient computed on the host in FP64 (IEEE division).  Returns 0 on success,
 * else a cclr_status code. */
int cc_lr_selftest_precond(int n, double omega, double omega_im, unsigned seed, double *max_rel_err);

/* Failure-detection self-test: launches one block that waits on an mbarrier phase that
 * nothing completes, with a limit of timeout_us microseconds (globaltimer).  The wait gives
 * up, raises the device error flag and returns; *flag receives the flag (1 expected) and the
 * call returns CCLR_ETIMEOUT (5).  No fault, trap or hang is involved. */
int cc_lr_selftest_timeout(int timeout_us, int *flag);

#ifdef __cplusplus
}
#endif
#endif
