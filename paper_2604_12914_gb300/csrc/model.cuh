// The LR-CCSD response model held on the device: inputs, T1-dressed Cholesky blocks,
// stored H-bar intermediates, and the sigma program (a list of linear operations on
// amplitude-shaped buffers that is run forward for sigma = A X and in reverse, with every
// operation transposed, for Y A).
#pragma once
#include <array>
#include <map>
#include <string>
#include <vector>

#include "engine.cuh"
#include "ladder_cc.cuh"
#include "ladder_tc.cuh"

namespace cclr {

// Constants a sigma program reads (one complete set per precision and per T).
enum CstId {
  K_FOV, K_FOO, K_FVV, K_WOOOO, K_WOVVO, K_WOOOV, K_WOVOO, K_T2, K_OOVV, K_LOV, K_LVO, K_LVV,
  K_NCST
};

struct CstSet {
  int dt = C128;
  std::array<DevBuf, K_NCST> buf;
  std::array<Tens, K_NCST> t;
  // constants known to be zero: the operations that read them are skipped (a set built for a
  // one-body operator alone has no two-body elements)
  std::array<bool, K_NCST> zero{};
  bool valid = false;
};

enum OpKind { OP_CONTRACT, OP_PERM, OP_ZERO, OP_LADDER, OP_ANTISYM, OP_PROJECT };

struct Op {
  OpKind kind;
  zc alpha;
  int cst = -1;
  std::string mc, mi, mo;
  int in = -1, out = -1;
  int in2 = -1, in3 = -1;  // OP_ANTISYM: in = R(ab), in2 = R(ij), in3 = R(ij)(ab)
};

struct VarSpec {
  std::vector<int64_t> dims;
};

struct Program {
  std::vector<VarSpec> vars;  // 0 x1, 1 x2, 2 s1, 3 s2, then temporaries
  std::vector<Op> ops;
};

Program build_sigma_program(int o, int v, int naux);

struct Timers {
  cudaEvent_t ev[8];
  bool made = false;
};

// A captured sigma / sigma^T program for one argument set (see Model::graphs).
struct GraphKey {
  int dir = 0, dt = 0, tc = 0, nr = 0;
  const void *set = nullptr;
  std::vector<const void *> ptrs;
  bool operator==(const GraphKey &k) const {
    return dir == k.dir && dt == k.dt && tc == k.tc && nr == k.nr && set == k.set && ptrs == k.ptrs;
  }
};
struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec = nullptr;
  unsigned long long epoch = 0;
};

class Model {
 public:
  Model(int o, int v, int naux, cudaStream_t st);
  ~Model();
  int o, v, naux, n;
  cudaStream_t st;
  Engine E;

  // inputs (complex128 / double)
  DevBuf eps;                       // [n]
  DevBuf Loo0, Lov0, Lvo0, Lvv0;    // undressed Cholesky blocks [P][.][.]
  DevBuf mu;                        // [3][n][n]
  DevBuf t1, t2;                    // [o][v], [o][o][v][v]
  DevBuf h;                         // one-body part of H, [n][n]
  DevBuf Loo64, Lov64, Lvo64, Lvv64, h64;  // complex64 copies (complex64 builds)
  DevBuf oovvp;                     // <ij||ab> packed [(i<j)][(a<b)], complex128 (T1-independent)

  CstSet c128, c64;                 // intermediates at the current T
  DevBuf D1, D2;                    // preconditioner diagonal (real): singles [o][v], packed doubles
  Program prog;
  std::vector<DevBuf> tmp128, tmp64;  // program temporaries per precision (shared by the RHS)
  std::vector<DevBuf> x2bar[2];       // per-RHS x2-bar of the transpose product, per precision
  int prec = 0;
  LadderCC lcc;                     // packed CUDA-core ladder (FP64 and FP32 modes)
  LadderTC ltc[3];                  // packed tensor-core ladder: [0] TF32, [1] 3xTF32, [2] bf16x3
  const void *ltc_src[3] = {nullptr, nullptr, nullptr};
  float ms_last[4] = {0, 0, 0, 0};  // last apply(): ladder, everything else, total, ladder formation (ms)
  Timers tm;
  // CUDA graphs: with graphs on, a sigma program whose arguments (direction, constant set,
  // precision, buffer addresses) repeat those of an earlier eager call, with no memory freed
  // or constants rebuilt since, is captured once and then replayed by cudaGraphLaunch.
  bool graphs = false;
  bool autotune = true;  // tensor-core GEMM shapes tuned on their first (eager) use
  bool lean = false;     // budgeted context: transient buffers are freed after use
  std::vector<GraphEntry> gcache;
  std::vector<GraphEntry> warm;  // recent eager calls (key, epoch after the call); no exec
  int graph_launches = 0, graph_captures = 0;
  void clear_graphs();

  void upload_inputs(const double *eps_h, const double *L, const double *mu_h,
                     const double *t1_h, const double *t2_h, int device_ptrs);
  // Build dressed blocks + intermediates for amplitudes (t1d, t2d; complex128 device) in
  // precision dt (complex64 on the tensor cores with the 3xTF32 split).
  // tc: tensor-core mode of a complex64 build's contractions (0: FP32 CUDA cores, the default;
  // 2: 3xTF32)
  void build_set(const void *t1d, const void *t2d, CstSet &out, int dt, int tc = 0);
  // The set of the one-body operator B alone (no two-body part; complex128) at amplitudes
  // (t1d, t2d): its sigma program is the Jacobian of xi^B(T) = Omega[B](T).
  void build_set_onebody(const void *Bd, const void *t1d, const void *t2d, CstSet &out);
  void ensure_src64();
  const void *oovv_packed();
  void build_diagonal();
  const CstSet &cst_for(int prec_) ;
  void round_set(const CstSet &src, CstSet &dst);
  // frees a set's buffers (it is rebuilt on its next use)
  void release_set(CstSet &s);
  // frees everything the FP64 products hold (the complex128 set, temporaries and the CUDA-core
  // ladder's blocks); an FP64 product afterwards rebuilds them
  void release_fp64();
  // frees what a product allocates for itself and keeps for the next one (program temporaries,
  // x2-bar, workspace, the ladders' blocks and prepared operands); the next product allocates
  // them again
  void release_product_buffers();
  // lean memory (a context with an HBM budget): also frees the undressed complex128 Cholesky
  // blocks once their complex64 copies exist; FP64 products are refused afterwards
  bool fp64_gone = false;
  void release_fp64_inputs();

  // sigma (dir = +1) or sigma^T (dir = -1) on device buffers of the given dtype.
  void apply(int dir, const CstSet &C, const void *x1, const void *x2, void *s1, void *s2);
  // the same for nr right-hand sides at once (the ladder's <ab||ef>~ is formed once for all)
  void apply_batch(int dir, const CstSet &C, int nr, const void *const *x1, const void *const *x2,
                   void *const *s1, void *const *s2);
  // xi^B (or at other amplitudes), complex128 device buffers.
  void xi(const void *mub, const void *t1d, const void *t2d, void *xi1, void *xi2);

  Tens T(const DevBuf &b, std::initializer_list<int64_t> dims, int dt = C128) const {
    return make_tens(b.p, dt, dims);
  }

 private:
  void ladder(int dir, const CstSet &C, zc alpha, const std::vector<Tens> &in, const std::vector<Tens> &out);
  // the program itself; timed = event timing of the ladder (not while capturing)
  void apply_body(int dir, const CstSet &C, int nr, const void *const *x1, const void *const *x2,
                  void *const *s1, void *const *s2, bool timed, float &lad_ms, float &form_ms);
  std::vector<DevBuf> &temps(int dt);
  Tens var_tens(int id, int dt, void *p) const;
};

}  // namespace cclr
