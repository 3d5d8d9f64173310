// Packed particle-particle ladder on the CUDA cores (FP64 DFMA for complex128, FP32 FFMA for
// complex64): the same packed algorithm as the tensor-core ladder (LadderTC), for the
// precision modes that do not use tensor cores.
//   out[i,j,a,b] += alpha * sum_{e<f} <ab||ef>~ X[i,j,e,f],   <ab|ef>~ = sum_P L~[P,a,e] L~[P,b,f]
// over packed pairs i<j, a<b, e<f, <ab|ef>~ formed on the fly for one group of a at a time
// (formation GEMM, K = naux), antisymmetrised and packed, then contracted with packed X; the
// transpose product (dir -1) contracts the same packed block over (a<b).
#pragma once
#include "engine.cuh"

namespace cclr {

class LadderCC {
 public:
  // a values per formed group block
  static constexpr int kGroup = 16;
  // out[r] += alpha * ladder(in[r]) (dir +1) or ladder^T(in[r]) (dir -1), r < nrhs; all
  // [o][o][v][v] of dtype dt (C128 or C64); Lvv [naux][v][v] of the same dtype (T1-dressed).
  void apply(Engine &E, int dt, const Tens &Lvv, int o, int v, int naux, int dir, zc alpha, int nrhs,
             const void *const *in, void *const *out);
  void release() { W.release(); Wp.release(); Xp.release(); sig.release(); }

 private:
  int o_ = -1, v_ = -1;
  DevBuf opairs, vpairs;       // pair tables (p, q), p < q
  DevBuf W, Wp, Xp, sig;       // group formation block, packed group block, packed X / Y', packed result
};

}  // namespace cclr
