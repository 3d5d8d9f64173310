// Particle-particle ladder on tcgen05 tensor cores (complex64 data; TF32, 3xTF32 or bf16x3):
//   out[i,j,a,b] += alpha * sum_{e<f} <ab||ef>~ X[i,j,e,f],   <ab|ef>~ = sum_P L~[P,a,e] L~[P,b,f]
// over packed pairs i<j, a<b, e<f (the four antisymmetric images of each output are written).
// <ab|ef>~ is formed on the fly from L~_vv for one group of a at a time and never stored
// whole: formation GEMM (rows (b,f), b >= a0; columns (a,e), a in the group; K = naux),
// antisymmetrise/pack to <ab||ef>~ over (a<b) x (e<f), contraction GEMM with packed X.
// The transpose product (dir -1) contracts the same packed block over (a<b) instead.
#pragma once
#include <vector>

#include "engine.cuh"

namespace cclr {

// Times nothing itself: runs the ladder's result scatter (unpack_sig) once on a packed result S
// [(a<b)][(i<j)] (complex64) into out [o][o][v][v] (complex64), with its own pair tables (for the
// HBM kernel benchmark).
void ladder_unpack_sig_bench(int o, int v, const void *S, void *out, cudaStream_t st);

class LadderTC {
 public:
  LadderTC() = default;
  LadderTC(const LadderTC &) = delete;
  LadderTC &operator=(const LadderTC &) = delete;
  ~LadderTC() {
    for (auto e : fev)
      if (e) cudaEventDestroy(e);
  }
  // Lvv: complex64 [naux][v][v] (T1-dressed).  seg = 1 (one pass) or 3 (split); kind = TC_TF32
  // or TC_BF16 (operand type of the tensor-core GEMMs).
  // lean: skip the group-size tuner and take the largest candidate whose block fits in 4 GB
  void prepare(Engine &E, const Tens &Lvv, int o, int v, int naux, int seg, int kind, bool lean = false);
  bool ready(int seg, int kind) const { return seg_ == seg && kind_ == kind && LA.p != nullptr; }
  // dir +1: out[r] += alpha * ladder(in[r]);  dir -1: out[r] += alpha * ladder^T(in[r]),
  // r = 0..nrhs-1, all complex64 [o][o][v][v].  Each <ab||ef>~ group block is formed once
  // and contracted with every right-hand side.
  void apply(Engine &E, int dir, zc alpha, int nrhs, const void *const *in, void *const *out);
  // device time (ms) of the formation GEMMs of the last apply(); call once its work has completed
  float formation_ms();
  // Autotuner: times one product for each candidate group size (a values per formed block:
  // 8, 16, 32, 64, those whose block fits in 8 GB) on zero input and keeps the fastest.  Runs
  // once per object, on its first preparation; group_size() and tune_log report the result.
  void tune(Engine &E);
  int group_size() const { return ga_; }
  // Ablation: keep the whole packed <ab||ef>~ (P_v x P_v, TF32 rows) once formed, so that later
  // sigma products (dir +1) skip the formation and run one contraction GEMM.  The transpose
  // product still forms the blocks on the fly.  Costs P_v^2 x 8 bytes (x 3 for 3xTF32, x 1.5 for
  // bf16x3).
  void set_store(bool on) {
    store_ = on;
    if (!on) { Wall.release(); wall_ready_ = false; }
  }
  bool stored() const { return store_; }
  // frees the per-product buffers and the prepared operands (prepare() is needed again)
  void release() {
    W.release(); Wp.release(); Xp.release(); sig.release(); LB.release(); LA.release();
    lb_all_ = false;
  }
  size_t stored_bytes() const { return Wall.bytes; }
  std::vector<std::pair<int, float>> tune_log;

 private:
  int o_ = 0, v_ = 0, naux_ = 0, seg_ = 0, kind_ = 0;
  int64_t Po_ = 0, Pv_ = 0;
  DevBuf LA, LB;            // formation operands: rows (b,f) (all), embedded rows (a,e) of one group; K = naux
  bool lb_all_ = false;     // LB holds the embedded rows (a,e) of every a (prepared once per L~_vv)
  const void *Lvv_ = nullptr;  // the complex64 L~_vv the operands are prepared from
  DevBuf opairs, vpairs;    // pair tables (p, q), p < q, row-major pair order
  DevBuf W, Wp, Xp, sig;    // group formation block, packed group block, packed X, packed result
  int ga_ = 32;             // a values per group (set by tune())
  bool tuned_ = false;
  bool store_ = false, wall_ready_ = false;
  DevBuf Wall;              // stored packed <ab||ef>~ (ablation)
  std::vector<cudaEvent_t> fev;  // formation start/stop events, two per group
  int nform_ = 0;                // groups timed in the last apply()
};

}  // namespace cclr
