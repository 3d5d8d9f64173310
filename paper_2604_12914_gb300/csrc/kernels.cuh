// Declarations of the generic device kernels and their host launchers.
#pragma once
#include <algorithm>

#include "common.cuh"

namespace cclr {

struct GemmArgs {
  const void *A = nullptr;
  const void *B = nullptr;
  void *C = nullptr;
  int64_t M = 0, N = 0, K = 0, batch = 1;
  int64_t sAb = 0, sAm = 0, sAk = 0;
  int64_t sBb = 0, sBk = 0, sBn = 0;
  int64_t sCb = 0, sCm = 0, sCn = 0;
  double alr = 1.0, ali = 0.0;
  int overwrite = 0;  // 1: C = alpha A B ; 0: C += alpha A B
  int64_t kchunk = 0;  // set by launch_gemm: K range per block when K is split (atomic sums)
};

struct PermArgs {
  const void *in = nullptr;
  void *out = nullptr;
  int rank = 0;
  int64_t dim[8] = {0};
  int64_t sin[8] = {0};
  int64_t sout[8] = {0};
  double alr = 1.0, ali = 0.0;
  int acc = 0;
  int64_t total = 0;
};

// Number of kernels this library has launched (all streams, process lifetime).
unsigned long long launch_count();
void count_launch(unsigned long long n = 1);

void launch_gemm(const GemmArgs &g, int dt, cudaStream_t st);
void launch_permute(const PermArgs &a, int dt_in, int dt_out, cudaStream_t st);
// S += P(ab) Rab + P(ij) Rij + P(ij)P(ab) R4 (dir +1) or the transpose into Rab, Rij, R4
// (dir -1); all [o][o][v][v].
void antisym_apply(int dt, int o, int v, int dir, void *S, void *Rab, void *Rij, void *R4, cudaStream_t st);
// In-place projection of S [o][o][v][v] onto tensors antisymmetric in (i,j) and (a,b).
void antisym_project(int dt, int o, int v, void *S, cudaStream_t st);
void vec_axpy(int dt, int64_t n, zc a, const void *x, void *y, cudaStream_t st);
void vec_scal(int dt, int64_t n, zc a, void *y, cudaStream_t st);
void vec_dot(int dt, int64_t n, const void *x, const void *y, int herm, double2 *part,
             double2 *out, int slot, cudaStream_t st);
// out = r / (D - (omega + i omega_im))
void vec_precond(int dt, int64_t n, const double *D, double omega, double omega_im, const void *r, void *out,
                 cudaStream_t st);
// D1[i,a] = Fvv_aa - Foo_ii; D2p[(i<j),(a<b)] = Fvv_aa + Fvv_bb - Foo_ii - Foo_jj over the
// packed doubles (real parts of complex128 Foo, Fvv).
void build_diag(int o, int v, const void *Foo, const void *Fvv, double *D1, double *D2p,
                cudaStream_t st);

// Packed (unique-amplitude) doubles: P[(i<j) * P_v + (a<b)], pairs (p<q) of n indices numbered
// row by row, pair(p, q) = p n - p (p + 1) / 2 + q - p - 1.  The full tensor F[o][o][v][v] is
// antisymmetric in (i,j) and (a,b).
// F (+)= alpha * unpack(P): every entry of F is written (zero where i = j or a = b).
// dt_p / dt_f: C128 or C64 (conversion on the fly).
void unpack_doubles(int dt_p, int dt_f, int o, int v, const void *P, void *F, zc alpha, bool acc, cudaStream_t st);
// P = F[i<j, a<b] (dt_f -> dt_p).
void pack_doubles(int dt_f, int dt_p, int o, int v, const void *F, void *P, cudaStream_t st);
// out1[i,a] += alpha * sum_{j,b} W[i,j,a,b] x1[j,b] for W antisymmetric in (i,j) and (a,b), given
// packed (complex128; x1, out1 complex128 [o][v]).
void packed_doubles_dot_singles(int o, int v, const void *Wp, const void *x1, void *out1, zc alpha, cudaStream_t st);
// Y[p][j][q] += alpha * sum_k S[k sSk + j sSj] X[p sXp + k sXk + q] (q unit stride in X and Y,
// Y[p sYp + j sYj + q]); k and j extents 1..64; complex128 or complex64 (dt), FP64 / FP32 CUDA cores.
void contract_smallk(int dt, int64_t P, int K, int J, int64_t Q, const void *S, int64_t sSk, int64_t sSj,
                     const void *X, int64_t sXp, int64_t sXk, void *Y, int64_t sYp, int64_t sYj, zc alpha,
                     cudaStream_t st);
// y[r] += alpha * sum_c B[x0][x1][x2][x3] s[c] for a contiguous rank-4 B (dims d[4]) whose modes are
// output modes (bit k of rmask set; y stride ys[k]) or contracted modes (s stride ss[k]); at most one of
// modes 2 and 3 is an output mode.  Complex128 or complex64 (dt); atomics (order of summation varies).
void contract_slab_gemv(int dt, const int64_t *d, int rmask, const void *B, const void *S, const int64_t *ss,
                        void *Y, const int64_t *ys, zc alpha, cudaStream_t st);
// tau[(i<j),(a<b)] = t2p + t1[i,a] t1[j,b] - t1[i,b] t1[j,a] over the packed doubles (complex128;
// t1 [o][v]); the CCSD energy is sum over the packed doubles of <ij||ab> tau.
void tau_packed(int o, int v, const void *t1, const void *t2p, void *tau, cudaStream_t st);
// y = conj(x), n complex128 entries (y may be x)
void vec_conj(int64_t n, const void *x, void *y, cudaStream_t st);
void apply_denominator(int o, int v, const double *eps, void *t2, cudaStream_t st);
void set_diag(int n, const double *d, void *out, cudaStream_t st);

// Particle-particle ladder on tcgen05 tensor cores (complex64 operands in TF32):
// out[i,j,a,b] += alpha * sum_{e,f} <ab|ef>~ X[i,j,e,f] with <ab|ef>~ = sum_P L[P,a,e] L[P,b,f].
struct LadderTC;
bool ladder_tc_available();

}  // namespace cclr
