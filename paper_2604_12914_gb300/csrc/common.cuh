// Shared definitions for libcclr: complex types, error handling, tensor views.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

namespace cclr {

struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string &m) : std::runtime_error(m), status(s) {}
};

#define CCLR_CUDA(x)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      throw ::cclr::Error(4, std::string(#x) + " failed: " + cudaGetErrorString(e_) +      \
                                 " at " + __FILE__ + ":" + std::to_string(__LINE__));     \
  } while (0)

#define CCLR_REQUIRE(cond, msg)                                                           \
  do {                                                                                    \
    if (!(cond)) throw ::cclr::Error(1, std::string(msg));                                \
  } while (0)

enum DType { C128 = 0, C64 = 1 };

inline size_t dt_size(int dt) { return dt == C128 ? 16 : 8; }

// Host-side complex scalar used for coefficients.
struct zc {
  double re, im;
  zc(double r = 0.0, double i = 0.0) : re(r), im(i) {}
};

// A strided view of a device tensor (element strides, up to 8 modes).
struct Tens {
  void *p = nullptr;
  int dt = C128;
  int rank = 0;
  int64_t dim[8] = {0};
  int64_t str[8] = {0};

  int64_t numel() const {
    int64_t n = 1;
    for (int i = 0; i < rank; ++i) n *= dim[i];
    return n;
  }
  bool contiguous() const {
    int64_t s = 1;
    for (int i = rank - 1; i >= 0; --i) {
      if (dim[i] != 1 && str[i] != s) return false;
      s *= dim[i];
    }
    return true;
  }
  // Sub-range [lo, hi) of mode m (same storage).
  Tens slice(int m, int64_t lo, int64_t hi) const {
    Tens t = *this;
    t.p = (char *)p + lo * str[m] * (int64_t)dt_size(dt);
    t.dim[m] = hi - lo;
    return t;
  }
};

inline Tens make_tens(void *p, int dt, std::initializer_list<int64_t> dims) {
  Tens t;
  t.p = p;
  t.dt = dt;
  t.rank = (int)dims.size();
  int i = 0;
  for (auto d : dims) t.dim[i++] = d;
  int64_t s = 1;
  for (int k = t.rank - 1; k >= 0; --k) {
    t.str[k] = s;
    s *= t.dim[k];
  }
  return t;
}

// Device-side complex helpers.
template <typename T> struct cpx;
template <> struct cpx<double> { using t = double2; };
template <> struct cpx<float> { using t = float2; };

template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

}  // namespace cclr
