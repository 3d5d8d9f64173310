/*
 * cclr_testing.h -- self-test entry points of libcclr (not part of the response API).
 */
#ifndef CCLR_TESTING_H
#define CCLR_TESTING_H

#ifdef __cplusplus
extern "C" {
#endif

/* Complex64 GEMM C[M][N] = A[M][K] B[K][N] on seeded random data, computed three ways
 * on the current device: tcgen05 tensor cores (mode 1 TF32, mode 2 3xTF32), FP32 CUDA
 * cores, and FP64 CUDA cores (reference).  Writes max|C_x - C_ref| / max|C_ref| for the
 * tensor-core (err[0]) and FP32 (err[1]) results.  Returns 0 on success, else a
 * cclr_status code. */
int cc_lr_selftest_gemm(int M, int N, int K, int mode, unsigned seed, double *err);

/* Times the tensor-core complex GEMM C[M][N] = A[M][K] B[K][N] (operand preparation
 * excluded) on seeded data: reps launches, CUDA events; ms[0] = mean milliseconds per
 * GEMM, ms[1] = the corresponding TFLOP/s at 8 real flops per complex multiply-add. */
int cc_lr_bench_gemm(int M, int N, int K, int mode, int reps, double *ms);

/* Failure-detection self-test: launches one block that waits on an mbarrier phase that
 * nothing completes, with a limit of timeout_us microseconds (globaltimer).  The wait gives
 * up, raises the device error flag and returns; *flag receives the flag (1 expected) and the
 * call returns CCLR_ETIMEOUT (5).  No fault, trap or hang is involved. */
int cc_lr_selftest_timeout(int timeout_us, int *flag);

#ifdef __cplusplus
}
#endif
#endif
