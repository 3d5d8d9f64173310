// Host-side tensor-contraction engine: device buffers, workspace, einsum-style
// contractions mapped onto the strided complex GEMM, permutes and vector helpers.
#pragma once
#include <memory>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace cclr {

// Device memory charged to one owner (a context): bytes held now, the most ever held, and
// an optional limit (0 = none) that every allocation charged to it is checked against.
struct MemAcct {
  size_t used = 0, peak = 0, budget = 0;
};
// The account that allocations made on this thread are charged to (nullptr: none).
MemAcct *&current_acct();
// Charges the allocations of a scope (one library call) to an account.
struct AcctScope {
  MemAcct *prev;
  explicit AcctScope(MemAcct *a) : prev(current_acct()) { current_acct() = a; }
  ~AcctScope() { current_acct() = prev; }
  AcctScope(const AcctScope &) = delete;
  AcctScope &operator=(const AcctScope &) = delete;
};

// Owning device allocation.  An allocation over the current account's budget throws status 2
// (CCLR_ENOMEM) before cudaMalloc is called; the bytes are returned to the same account when
// the buffer is released, whichever thread releases it.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  MemAcct *acct = nullptr;
  DevBuf() = default;
  explicit DevBuf(size_t b) { alloc(b); }
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), acct(o.acct) { o.p = nullptr; o.bytes = 0; o.acct = nullptr; }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; acct = o.acct;
      o.p = nullptr; o.bytes = 0; o.acct = nullptr;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t b);
  void release();
  template <typename T> T *as() const { return (T *)p; }
};

size_t device_bytes_in_use();
// Counter bumped whenever device memory is freed (and by callers that rewrite state a captured
// CUDA graph depends on): a graph captured at one value is valid while the counter keeps it.
unsigned long long state_epoch();
void bump_state_epoch();

class Engine {
 public:
  cudaStream_t st = nullptr;
  // complex64 contractions above a size threshold run on the tcgen05 tensor cores:
  // 0 = never (CUDA-core FP32), 1 = TF32, 2 = 3xTF32 split, 3 = bf16x3 split.
  int tc_mode = 0;
  bool tc_force = false;  // route every complex64 contraction to the tensor cores (self-test)
  int64_t tc_calls = 0;
  // Workspace slot s of at least `bytes` bytes (grown on demand, reused across calls).
  void *ws(int slot, size_t bytes);
  // frees the workspace slots (they grow again on demand)
  void release_ws() { slots_.clear(); }
  // C[mc] += alpha * sum A[ma] B[mb] over the modes not in mc (einsum semantics; every
  // mode must appear in exactly two operands or in all three).
  void contract(zc alpha, const Tens &A, const std::string &ma, const Tens &B,
                const std::string &mb, const Tens &C, const std::string &mc);
  // the complex64 tensor-core branch of contract (modes already classified)
  void contract_tc(zc alpha, const Tens &A, const std::string &ma, const Tens &B, const std::string &mb,
                   const Tens &C, const std::string &mc, const std::string &bat, const std::string &Mm,
                   const std::string &Nm, const std::string &Km, int64_t nb, int64_t M, int64_t N, int64_t K);
  // out[mo] (+)= alpha * in[mi]  (same mode set; dtypes may differ -> conversion).
  void permute(zc alpha, const Tens &in, const std::string &mi, const Tens &out,
               const std::string &mo, bool acc);
  void zero(const Tens &t);
  double2 *dot_scratch();  // device: partials [>=304] and results [64]
  double2 *dot_results();
  // Constant operands: while cst_hint points at one operand of a tensor-core contraction, the
  // prepared form of that operand (its permuted copy, or its TF32 / BF16 embedded rows or columns)
  // is kept and reused by later contractions of the same operand with the same modes and
  // precision, as long as state_epoch() has not moved (no device memory freed, no constants
  // rebuilt); at most prep_cache_cap bytes (0: off).
  const void *cst_hint = nullptr;
  size_t prep_cache_cap = 0;
  void clear_prep_cache() {
    prep_.clear();
    prep_bytes_ = 0;
  }
  size_t prep_cache_bytes() const { return prep_bytes_; }

 private:
  std::vector<DevBuf> slots_;
  DevBuf dots_;
  struct PrepEntry {
    std::string key;
    DevBuf buf;
    unsigned long long epoch = 0;  // the entry's content is valid while state_epoch() equals it
  };
  std::vector<std::unique_ptr<PrepEntry>> prep_;
  size_t prep_bytes_ = 0;
  // a valid entry, or nullptr
  PrepEntry *prep_find(const std::string &key);
  // the entry to (re)fill, created if needed; nullptr when it would exceed the cap
  PrepEntry *prep_get(const std::string &key, size_t bytes);
};

}  // namespace cclr
