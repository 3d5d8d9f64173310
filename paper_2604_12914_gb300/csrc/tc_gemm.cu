// tcgen05 GEMM (kind::tf32 on TF32 operands, kind::f16 on BF16 operands) for sm_103a,
// persistent and warp-specialised: one CTA per SM walks a
// static list of (tile, K split) work units.  Warp 0 streams A/B K blocks with TMA (128-byte
// swizzle) into a 4-stage shared-memory ring, warp 1 issues tcgen05.mma into one of two TMEM
// accumulators, and warps 2-9 drain the other accumulator (tcgen05.ld -> registers ->
// shared-memory staging -> coalesced global stores), so the epilogue of one tile overlaps
// the main loop of the next.  Every mbarrier wait is bounded (globaltimer); on timeout the
// kernel raises a device flag, stops every role, drains its own copies and MMAs with bounded
// waits, frees its TMEM and returns.
#include <cstdio>
#include <cstdlib>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "engine.cuh"
#include "tc_gemm.cuh"

namespace cclr {
namespace {

constexpr int BM = 128;      // UMMA M
constexpr int BKB = 128;     // bytes per K block = one 128-byte swizzle row (32 TF32 or 64 BF16)
constexpr int STAGES = 4;
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;  // 2 s per wait

struct TcParams {
  int M, N, K, BN;
  int nMt, nNt, band;   // tile counts; M tiles per raster band (N varies fastest inside a band)
  int kb_per_split;     // K blocks per split (splits of K are atomically summed)
  int splits;           // work units = tiles x splits, walked with stride gridDim.x
  int transposed;       // epilogue: 1 = lanes along columns (C columns contiguous), 0 = lane per row
  float *C;
  View2 rv, cv;         // C rows and complex columns
  float ar, ai;
  int accumulate;       // add to C (always true when split)
  int atomic;           // split-K: combine partial tiles with atomicAdd
  int *err;
};

__device__ __forceinline__ uint32_t su32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (gtime() - t0 > TIMEOUT_NS) {
      atomicExch(err, 1);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      :
      : "r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused with 128B swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return d;
}

// Instruction descriptor of kind::tf32 / kind::f16: D FP32 (bits 4-5), A and B type (bits 7-9
// and 10-12: TF32 = 2, BF16 = 1), both K-major, N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_mma(int kind, int M, int N) {
  return (1u << 4) | ((kind == TC_BF16 ? 1u : 2u) << 7) | ((kind == TC_BF16 ? 1u : 2u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// one MMA of K = 32 bytes per row (8 TF32 or 16 BF16), D (+)= A B^T in TMEM
template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (KIND == TC_BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Bounded wait that also gives up when another role of the CTA has aborted.
__device__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, int *err, volatile int *abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtime() - t0 > TIMEOUT_NS) {
      atomicExch(err, 1);
      *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// work unit -> (m tile, n tile, split); banded rasterisation: consecutive units share one B
// tile column across a band of M tiles, so the band's A tiles and the current B tiles stay in L2
__device__ __forceinline__ void unit_coords(const TcParams &p, int u, int &m_tile, int &n_tile, int &split) {
  const int tiles = p.nMt * p.nNt;
  split = u / tiles;
  const int id = u - split * tiles;
  const int per_band = p.band * p.nNt;
  const int b = id / per_band;
  const int local = id - b * per_band;
  const int mb = min(p.band, p.nMt - b * p.band);
  m_tile = b * p.band + local % mb;
  n_tile = local / mb;
}

constexpr int EPI_PITCH = 18;  // floats per staged row (16 + 2): conflict-free float2 traffic

template <int KIND>
__global__ void __launch_bounds__(320, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int BK = BKB / (KIND == TC_BF16 ? 2 : 4);  // operand elements per K block
  const int BN = p.BN;
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * BM * BKB;
  float *stage = (float *)(smem + STAGES * (BM + BN) * BKB);  // 8 warps x 32 rows x EPI_PITCH
  // barriers: full[S], empty[S], tfull[2], tempty[2], drain
  uint64_t *bars = (uint64_t *)(stage + 8 * 32 * EPI_PITCH);
  uint64_t *full = bars, *empty = bars + STAGES, *tfull = bars + 2 * STAGES, *tempty = tfull + 2,
           *drain = tempty + 2;
  uint32_t *tslot = (uint32_t *)(drain + 1);
  int *issued = (int *)(tslot + 1);  // K blocks loaded (producer)
  int *consumed = issued + 1;        // K blocks whose full barrier the MMA warp passed
  volatile int *abort_flag = issued + 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = p.nMt * p.nNt * p.splits;
  const int nk_all = (p.K + BK - 1) / BK;
  // accumulator columns: one buffer per power of two >= BN, two buffers
  const uint32_t half = BN <= 32 ? 32u : BN <= 64 ? 64u : BN <= 128 ? 128u : 256u;
  const uint32_t tcols = 2 * half;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(full + s)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(empty + s)) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(tfull + b)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(su32(tempty + b)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(drain)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    issued[0] = 0;
    consumed[0] = 0;
    *abort_flag = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: K blocks of every unit of this CTA, through the ring
      const uint32_t bytes = (uint32_t)(BM + BN) * BKB;
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        int mt, nt, sp;
        unit_coords(p, u, mt, nt, sp);
        const int kb0 = sp * p.kb_per_split;
        const int nk = max(0, min(nk_all - kb0, p.kb_per_split));
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (!mbar_wait_ab(su32(empty + s), ph ^ 1u, p.err, abort_flag)) { ok = false; break; }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(full + s)), "r"(bytes)
                       : "memory");
          tma_load_2d(sA + s * BM * BKB, &tmA, (kb0 + kb) * BK, mt * BM, su32(full + s));
          tma_load_2d(sB + s * BN * BKB, &tmB, (kb0 + kb) * BK, nt * BN, su32(full + s));
          issued[0] = g + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: accumulator buffer it & 1 for the it-th unit of this CTA
      const uint32_t idesc = idesc_mma(KIND, BM, BN);
      int g = 0, it = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x, ++it) {
        int mt, nt, sp;
        unit_coords(p, u, mt, nt, sp);
        const int kb0 = sp * p.kb_per_split;
        const int nk = max(0, min(nk_all - kb0, p.kb_per_split));
        const int buf = it & 1;
        if (!mbar_wait_ab(su32(tempty + buf), ((uint32_t)(it >> 1) & 1u) ^ 1u, p.err, abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)buf * half;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (!mbar_wait_ab(su32(full + s), ph, p.err, abort_flag)) { ok = false; break; }
          consumed[0] = g + 1;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da = sw128_desc(su32(sA + s * BM * BKB));
          const uint64_t db = sw128_desc(su32(sB + s * BN * BKB));
#pragma unroll
          for (int kk = 0; kk < BKB / 32; ++kk)  // 32 bytes of K per instruction (+2 in 16-byte units)
            mma_issue<KIND>(dacc, da + 2 * kk, db + 2 * kk, idesc, (kb | kk) != 0 ? 1u : 0u);
          mma_commit(su32(empty + s));
        }
        if (ok) mma_commit(su32(tfull + buf));  // arrives once this unit's MMAs have completed
      }
      // every MMA issued above has completed once this arrives
      mma_commit(su32(drain));
      mbar_wait(su32(drain), 0, p.err);
    }
    __syncwarp();
  } else {
    // epilogue warps 2..9: warps w and w + 4 share TMEM lane quarter w % 4 (rows 32 (w % 4)
    // .. + 31 of the tile) and take alternate 16-column chunks
    const int q = warp & 3, h = (warp - 2) >> 2;
    float *stg = stage + (warp - 2) * 32 * EPI_PITCH;
    int it = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x, ++it) {
      int mt, nt, sp;
      unit_coords(p, u, mt, nt, sp);
      const int buf = it & 1;
      bool ok = mbar_wait_ab(su32(tfull + buf), (uint32_t)(it >> 1) & 1u, p.err, abort_flag);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m0 = mt * BM, n0 = nt * BN;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * half;
      const int row = m0 + q * 32 + lane;
      if (16 * h >= BN) {  // no chunk for this warp: release the buffer at once
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(su32(tempty + buf));
        continue;
      }
      for (int c0 = 16 * h; c0 < BN; c0 += 32) {
        uint32_t r[16];
        tmem_ld16(tbase + (uint32_t)c0, r);
        if (c0 + 32 >= BN) {
          // the accumulator buffer is free for the next unit once every warp has read its part
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(su32(tempty + buf));
        }
        // eight complex values per lane: destinations first, then all loads, then all stores
        // (independent accesses in flight instead of one read-modify-write at a time)
        float *dst[8];
        float2 val[8];
        if (p.transposed) {
          // stage rows, then 4 rows x 8 complex per instruction (64 contiguous bytes per row)
          float2 *srow = reinterpret_cast<float2 *>(stg + lane * EPI_PITCH);
#pragma unroll
          for (int j = 0; j < 8; ++j) srow[j] = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
          __syncwarp();
          const int jj = lane & 7, rs = lane >> 3;
          const int n = n0 + c0 + 2 * jj;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int rl = 4 * k + rs, grow = m0 + q * 32 + rl;
            val[k] = reinterpret_cast<const float2 *>(stg + rl * EPI_PITCH)[jj];
            dst[k] = (grow < p.M && n < p.N) ? p.C + 2 * (v2off(p.rv, grow) + v2off(p.cv, n >> 1)) : nullptr;
          }
          __syncwarp();
        } else {
          const float *crow = p.C + 2 * v2off(p.rv, row < p.M ? row : 0);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int n = n0 + c0 + 2 * k;
            val[k] = make_float2(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
            dst[k] = (row < p.M && n < p.N) ? const_cast<float *>(crow) + 2 * v2off(p.cv, n >> 1) : nullptr;
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
          val[k] = make_float2(p.ar * val[k].x - p.ai * val[k].y, p.ar * val[k].y + p.ai * val[k].x);
        if (p.atomic) {
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (dst[k]) {
              atomicAdd(dst[k], val[k].x);
              atomicAdd(dst[k] + 1, val[k].y);
            }
        } else {
          if (p.accumulate) {
            float2 old[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              old[k] = dst[k] ? *reinterpret_cast<const float2 *>(dst[k]) : make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 8; ++k) val[k] = make_float2(val[k].x + old[k].x, val[k].y + old[k].y);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (dst[k]) *reinterpret_cast<float2 *>(dst[k]) = val[k];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && consumed[0] < issued[0]) {
    // error path: drain TMA copies issued but never consumed (bounded)
    for (int g = consumed[0]; g < issued[0]; ++g)
      mbar_wait(su32(full + g % STAGES), (uint32_t)(g / STAGES) & 1u, p.err);
  }
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// A wait that nothing completes, bounded by timeout_ns (self-test of the give-up path).
__global__ void wait_never_kernel(unsigned long long timeout_ns, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t0 = gtime();
    while (!mbar_try(su32(&bar), 0)) {
      if (gtime() - t0 > timeout_ns) {
        atomicExch(err, 1);
        break;
      }
    }
  }
  __syncthreads();
}

// ---------------- operand preparation ----------------
template <int KIND>
__global__ void prep_a_kernel(const float2 *A, View2 mv, View2 kv, int64_t M, int64_t K, int64_t Kp, int seg,
                              typename TcElem<KIND>::T *dst, int64_t ldd) {
  const int64_t total = M * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t m, k;
    if (kv.sin == 1 || mv.sin != 1) { k = e % Kp; m = e / Kp; } else { m = e % M; k = e / M; }
    float2 v = make_float2(0.f, 0.f);
    if (k < K) v = A[v2off(mv, m) + v2off(kv, k)];
    tc_put_a<KIND>(dst + m * ldd, k, Kp, seg, v);
  }
}

template <int KIND>
__global__ void prep_b_kernel(const float2 *B, View2 kv, View2 nv, int64_t K, int64_t N, int64_t Kp, int seg,
                              typename TcElem<KIND>::T *dst, int64_t ldd) {
  const int64_t total = N * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t n, k;
    if (kv.sin == 1 || nv.sin != 1) { k = e % Kp; n = e / Kp; } else { n = e % N; k = e / N; }
    float2 v = make_float2(0.f, 0.f);
    if (k < K) v = B[v2off(kv, k) + v2off(nv, n)];
    tc_put_b<KIND>(dst + (2 * n) * ldd, dst + (2 * n + 1) * ldd, k, Kp, seg, v);
  }
}

// Transposing preparation: the source is contiguous along m (A) or n (B) and strided along
// k; 32 x 32 tiles through shared memory so that reads and writes are both coalesced.
template <int KIND>
__global__ void prep_tiled_kernel(const float2 *src, View2 mnv, View2 kv, int64_t MN, int64_t K, int64_t Kp, int seg,
                                  int isB, typename TcElem<KIND>::T *dst, int64_t ldd) {
  __shared__ float2 tile[32][33];
  const int64_t tmn = (MN + 31) / 32, tk = (Kp + 31) / 32;
  for (int64_t t = blockIdx.x; t < tmn * tk; t += gridDim.x) {
    const int64_t mn0 = (t % tmn) * 32, k0 = (t / tmn) * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int64_t mn = mn0 + threadIdx.x, k = k0 + r;
      float2 v = make_float2(0.f, 0.f);
      if (mn < MN && k < K) v = src[v2off(mnv, mn) + v2off(kv, k)];
      tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int64_t mn = mn0 + r, k = k0 + threadIdx.x;
      if (mn < MN && k < Kp) {
        const float2 v = tile[threadIdx.x][r];
        if (!isB) tc_put_a<KIND>(dst + mn * ldd, k, Kp, seg, v);
        else tc_put_b<KIND>(dst + (2 * mn) * ldd, dst + (2 * mn + 1) * ldd, k, Kp, seg, v);
      }
    }
    __syncthreads();
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
constexpr int kMaxDevs = 64;
int *g_err_dev[kMaxDevs] = {};  // bounded-wait flag, one per device
std::mutex g_dev_mu;

std::once_flag g_enc_once;

void fetch_encoder() {
  // the driver entry point is fetched through the runtime, so the library does not link
  // against libcuda itself (it still loads on machines without a driver)
  cudaDriverEntryPointQueryResult q;
  void *fn = nullptr;
  CCLR_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !fn) throw Error(4, "cuTensorMapEncodeTiled not available");
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

int current_device() {
  int dev = 0;
  CCLR_CUDA(cudaGetDevice(&dev));
  CCLR_REQUIRE(dev >= 0 && dev < kMaxDevs, "device ordinal beyond 63");
  return dev;
}

// raises the dynamic shared-memory limit of every kernel instantiation on the current device
void set_smem_limits() {
  CCLR_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<TC_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  CCLR_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
}

// The current device's wait flag; the first use on a device allocates and clears it and raises
// the kernel's shared-memory limit there.
int *device_err() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_dev_mu);
  if (!g_err_dev[dev]) {
    std::call_once(g_enc_once, fetch_encoder);
    int *p = nullptr;
    CCLR_CUDA(cudaMalloc(&p, sizeof(int)));
    CCLR_CUDA(cudaMemset(p, 0, sizeof(int)));
    set_smem_limits();
    g_err_dev[dev] = p;
  }
  return g_err_dev[dev];
}

// 2-D tensor map over a row-major operand (rows x cols elements, ld elements apart), boxes of
// one 128-byte K block by box_rows rows, 128-byte swizzle
CUtensorMap make_map(const void *base, int64_t rows, int64_t cols, int64_t ld, int box_rows, int kind) {
  CUtensorMap m;
  const int64_t es = tc_esize(kind);
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(BKB / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(&m, kind == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        (void *)base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(4, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

int pick_bn(int64_t N) {
  if (N <= 256) return (int)((N + 15) / 16 * 16);
  int best = 256;
  int64_t best_waste = -1;
  for (int bn = 256; bn >= 128; bn -= 16) {
    int64_t tiles = (N + bn - 1) / bn;
    int64_t waste = tiles * bn - N;
    if (best_waste < 0 || waste < best_waste) {
      best = bn;
      best_waste = waste;
    }
  }
  return best;
}

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n <= 0) {
    (void)cudaGetLastError();
    return 152;
  }
  return n;
}

unsigned grid1d(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
}

template <int KIND>
void prep_launch(const void *src, View2 mv, View2 kv, int64_t MN, int64_t K, int seg, int isB, void *dst, int64_t ldd,
                 cudaStream_t st) {
  using T = typename TcElem<KIND>::T;
  const int64_t Kp = tc_kpad(K);
  const bool tiled = kv.sin != 1 && mv.sin == 1 && MN >= 8;
  if (tiled) {
    const int64_t nt = ((MN + 31) / 32) * ((Kp + 31) / 32);
    prep_tiled_kernel<KIND><<<(unsigned)std::min<int64_t>(nt, 152 * 64), dim3(32, 8), 0, st>>>(
        (const float2 *)src, mv, kv, MN, K, Kp, seg, isB, (T *)dst, ldd);
  } else if (!isB) {
    prep_a_kernel<KIND><<<grid1d(MN * Kp), 256, 0, st>>>((const float2 *)src, mv, kv, MN, K, Kp, seg, (T *)dst, ldd);
  } else {
    prep_b_kernel<KIND><<<grid1d(MN * Kp), 256, 0, st>>>((const float2 *)src, kv, mv, K, MN, Kp, seg, (T *)dst, ldd);
  }
}

}  // namespace

void tc_prep_a2(const void *A, View2 mv, View2 kv, int64_t M, int64_t K, int seg, int kind, void *dst, int64_t ldd,
                cudaStream_t st) {
  CCLR_REQUIRE(ldd >= 2 * tc_kpad(K) * seg, "tc_prep_a: row too short");
  if (kind == TC_BF16) prep_launch<TC_BF16>(A, mv, kv, M, K, seg, 0, dst, ldd, st);
  else prep_launch<TC_TF32>(A, mv, kv, M, K, seg, 0, dst, ldd, st);
  count_launch();
  CCLR_CUDA(cudaGetLastError());
}

void tc_prep_b2(const void *B, View2 kv, View2 nv, int64_t K, int64_t N, int seg, int kind, void *dst, int64_t ldd,
                cudaStream_t st) {
  CCLR_REQUIRE(ldd >= 2 * tc_kpad(K) * seg, "tc_prep_b: row too short");
  if (kind == TC_BF16) prep_launch<TC_BF16>(B, nv, kv, N, K, seg, 1, dst, ldd, st);
  else prep_launch<TC_TF32>(B, nv, kv, N, K, seg, 1, dst, ldd, st);
  count_launch();
  CCLR_CUDA(cudaGetLastError());
}

void tc_prep_a(const void *A, int64_t sam, int64_t sak, int64_t M, int64_t K, int seg, int kind, void *dst,
               int64_t ldd, cudaStream_t st) {
  tc_prep_a2(A, view1(sam), view1(sak), M, K, seg, kind, dst, ldd, st);
}

void tc_prep_b(const void *B, int64_t sbk, int64_t sbn, int64_t K, int64_t N, int seg, int kind, void *dst,
               int64_t ldd, cudaStream_t st) {
  tc_prep_b2(B, view1(sbk), view1(sbn), K, N, seg, kind, dst, ldd, st);
}

// Launch configuration: tile width BN, K splits and raster band (0 = the rule's choice).
struct TcCfg {
  int BN = 0, splits = 0, band = 0;
};

struct TuneKey {
  int dev, kind, transposed;
  int64_t M, N, K;
  bool operator<(const TuneKey &o) const {
    return std::tie(dev, kind, transposed, M, N, K) < std::tie(o.dev, o.kind, o.transposed, o.M, o.N, o.K);
  }
};
struct TuneRec {
  TcCfg cfg, rule;
  float ms_best = 0.f, ms_rule = 0.f;
  int tried = 0;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneRec> g_tune;
thread_local bool g_tune_on = false;

// a_cols: operand elements A actually holds per row (<= Kreal; the rest reads as zero).
// lda, ldb, Kreal in elements of the operand type.  cfg overrides the rules; *used receives the
// configuration launched.
static void tc_launch(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int64_t Nreal, int64_t Kreal,
                      int kind, float *C, View2 rv, View2 cv, zc alpha, bool accumulate, int max_kb_per_split,
                      int *err, cudaStream_t st, int64_t a_cols, TcCfg cfg, TcCfg *used) {
  const int64_t es = tc_esize(kind), BK = BKB / es;
  const int BN = cfg.BN > 0 ? cfg.BN : pick_bn(Nreal);
  const CUtensorMap ma = make_map(A, M, a_cols < 0 ? Kreal : a_cols, lda, BM, kind);
  const CUtensorMap mb = make_map(B, Nreal, Kreal, ldb, BN, kind);
  TcParams p;
  p.M = (int)M;
  p.N = (int)Nreal;
  p.K = (int)Kreal;
  p.BN = BN;
  p.nMt = (int)((M + BM - 1) / BM);
  p.nNt = (int)((Nreal + BN - 1) / BN);
  // band of M tiles whose A rows (about 32 MB) stay in L2 while N sweeps
  p.band = cfg.band > 0 ? std::min(cfg.band, p.nMt)
                        : (int)std::max<int64_t>(1, std::min<int64_t>(p.nMt, (32ll << 20) / (BM * Kreal * es + 1)));
  const int nk = (int)((Kreal + BK - 1) / BK);
  const int64_t tiles = (int64_t)p.nMt * p.nNt;
  const int nsm = num_sms();
  // split K when the tile list cannot fill the GPU (two units per SM), at least 16 K blocks
  // per split
  int splits = 1;
  if (cfg.splits > 0) splits = std::min(cfg.splits, nk);
  else if (tiles < 2 * nsm && nk >= 32)
    splits = (int)std::max<int64_t>(1, std::min<int64_t>((2 * nsm + tiles - 1) / tiles, nk / 16));
  // bound the length of each accumulation chain (accuracy of the split-precision passes)
  if (max_kb_per_split > 0) splits = std::max(splits, (nk + max_kb_per_split - 1) / max_kb_per_split);
  splits = std::min(splits, 65535);
  p.kb_per_split = (nk + splits - 1) / splits;
  splits = (nk + p.kb_per_split - 1) / p.kb_per_split;  // every split has at least one K block
  p.splits = splits;
  p.C = C;
  p.rv = rv;
  p.cv = cv;
  // lanes along columns when C's columns run contiguously, one lane per row otherwise
  p.transposed = (cv.sin == 1 && (cv.din == TC_ONE_LEVEL || cv.din >= 8)) ? 1 : 0;
  p.ar = (float)alpha.re;
  p.ai = (float)alpha.im;
  p.atomic = splits > 1 ? 1 : 0;
  p.accumulate = (accumulate || splits > 1) ? 1 : 0;
  p.err = err;
  if (splits > 1 && !accumulate) {
    CCLR_REQUIRE(rv.din == TC_ONE_LEVEL && cv.din == TC_ONE_LEVEL && cv.sin == 1,
                 "tc_gemm: split K without accumulation needs a plain C layout");
    CCLR_CUDA(cudaMemset2DAsync(C, (size_t)rv.sin * 8, 0, (size_t)Nreal * 4, (size_t)M, st));
  }
  const int64_t units = tiles * splits;
  CCLR_REQUIRE(units < (1ll << 31), "tc_gemm: too many work units");
  static const bool trace = std::getenv("CCLR_TRACE") && std::getenv("CCLR_TRACE")[0] == '1';
  if (trace)
    std::fprintf(stderr, "cclr tc_gemm kind=%d M=%lld N=%lld K=%lld BN=%d tiles=%lld splits=%d band=%d atomic=%d transposed=%d\n",
                 kind, (long long)M, (long long)Nreal, (long long)Kreal, BN, (long long)tiles, splits, p.band, p.atomic,
                 p.transposed);
  const size_t smem = 1024 + (size_t)STAGES * (BM + BN) * BKB + (size_t)8 * 32 * EPI_PITCH * 4 +
                      (2 * STAGES + 5) * 8 + 16;
  const unsigned grid = (unsigned)std::min<int64_t>(units, nsm);
  if (kind == TC_BF16) tc_gemm_kernel<TC_BF16><<<grid, 320, smem, st>>>(ma, mb, p);
  else tc_gemm_kernel<TC_TF32><<<grid, 320, smem, st>>>(ma, mb, p);
  count_launch();
  CCLR_CUDA(cudaGetLastError());
  if (used) {
    used->BN = BN;
    used->splits = splits;
    used->band = p.band;
  }
}

// Candidate configurations around the rule's choice: other tile widths for wide outputs, more or
// fewer K splits where the tile list is short, and the two extreme raster bands.
static std::vector<TcCfg> candidates(const TcCfg &rule, int64_t M, int64_t Nreal, int64_t Kreal, int kind,
                                     bool allow_split) {
  std::vector<TcCfg> c{rule};
  auto add = [&](TcCfg x) {
    for (const auto &y : c)
      if (y.BN == x.BN && y.splits == x.splits && y.band == x.band) return;
    c.push_back(x);
  };
  if (Nreal > 256)
    for (int bn : {128, 192, 256}) { TcCfg x = rule; x.BN = bn; add(x); }
  const int64_t nk = (Kreal + BKB / tc_esize(kind) - 1) / (BKB / tc_esize(kind));
  if (!allow_split) {
  } else if (rule.splits > 1) {
    TcCfg x = rule; x.splits = std::max(1, rule.splits / 2); add(x);
    x.splits = (int)std::min<int64_t>(nk, 2 * rule.splits); add(x);
  } else if (nk >= 16) {
    TcCfg x = rule; x.splits = 2; add(x);
  }
  const int nMt = (int)((M + BM - 1) / BM);
  if (nMt > 1) {
    TcCfg x = rule; x.band = 1; add(x);
    x.band = nMt; add(x);
  }
  return c;
}

static void tc_gemm_core(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int64_t Nreal,
                         int64_t Kreal, int kind, float *C, View2 rv, View2 cv, zc alpha, bool accumulate,
                         int max_kb_per_split, int *err, cudaStream_t st, int64_t a_cols = -1) {
  if (M <= 0 || Nreal <= 0) return;
  const int64_t es = tc_esize(kind);
  CCLR_REQUIRE(Nreal % 2 == 0, "tc_gemm: real N must be even (complex pairs)");
  CCLR_REQUIRE((lda * es) % 16 == 0 && (ldb * es) % 16 == 0, "tc_gemm: row pitches must be multiples of 16 bytes");
  CCLR_REQUIRE(((uintptr_t)A % 16) == 0 && ((uintptr_t)B % 16) == 0, "tc_gemm: operands must be 16-byte aligned");
  CCLR_REQUIRE(M < (1ll << 31) && Nreal < (1ll << 31) && Kreal < (1ll << 31), "tc_gemm: dimension too large");
  const int transposed = (cv.sin == 1 && (cv.din == TC_ONE_LEVEL || cv.din >= 8)) ? 1 : 0;
  const TuneKey key{current_device(), kind, transposed, M, Nreal, Kreal};
  TcCfg cfg;
  bool have = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      cfg = it->second.cfg;
      have = true;
    }
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CCLR_CUDA(cudaStreamIsCapturing(st, &cap));
  // Autotuning (first use of a shape while tuning is on, never inside a capture): every candidate
  // is timed with CUDA events on the real operands.  Outputs that are overwritten are tuned in
  // place (the launch below rewrites them); accumulated ones into a scratch block of the same
  // shape when it fits in 512 MB, else the rule stands.
  if (!have && g_tune_on && cap == cudaStreamCaptureStatusNone) {
    const size_t cbytes = (size_t)M * Nreal * 4;
    DevBuf scratch;
    float *Ct = C;
    View2 trv = rv, tcv = cv;
    bool ok = true;
    if (accumulate) {
      if (cbytes <= (512ull << 20)) {
        scratch.alloc(cbytes);
        Ct = scratch.as<float>();
        trv = view1(Nreal / 2);
        tcv = view1(1);
      } else {
        ok = false;
      }
    }
    TuneRec rec;
    if (ok) {
      TcCfg rule;
      tc_launch(A, lda, B, ldb, M, Nreal, Kreal, kind, Ct, trv, tcv, alpha, false, max_kb_per_split, err, st, a_cols,
                TcCfg(), &rule);
      rec.rule = rule;
      cudaEvent_t e0, e1;
      CCLR_CUDA(cudaEventCreate(&e0));
      CCLR_CUDA(cudaEventCreate(&e1));
      float best = 1e30f;
      // K splits need an accumulating or plain output (split partial tiles are added atomically)
      const bool plain = trv.din == TC_ONE_LEVEL && tcv.din == TC_ONE_LEVEL && tcv.sin == 1;
      for (const TcCfg &cand : candidates(rule, M, Nreal, Kreal, kind, accumulate || plain)) {
        TcCfg used;
        CCLR_CUDA(cudaEventRecord(e0, st));
        tc_launch(A, lda, B, ldb, M, Nreal, Kreal, kind, Ct, trv, tcv, alpha, false, max_kb_per_split, err, st, a_cols,
                  cand, &used);
        CCLR_CUDA(cudaEventRecord(e1, st));
        CCLR_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        CCLR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rec.tried == 0) rec.ms_rule = ms;  // the first candidate is the rule's configuration
        ++rec.tried;
        if (ms < best) {
          best = ms;
          rec.cfg = used;
        }
      }
      rec.ms_best = best;
      CCLR_CUDA(cudaEventDestroy(e0));
      CCLR_CUDA(cudaEventDestroy(e1));
    } else {
      rec.cfg = TcCfg();
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = rec;
    cfg = rec.cfg;
  }
  tc_launch(A, lda, B, ldb, M, Nreal, Kreal, kind, C, rv, cv, alpha, accumulate, max_kb_per_split, err, st, a_cols, cfg,
            nullptr);
}

void tc_gemm(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t M, int64_t Nreal,
             int64_t Kreal, float *C, int64_t ldc_floats, zc alpha, bool accumulate, cudaStream_t st) {
  tc_gemm_core(A, lda, B, ldb, M, Nreal, Kreal, TC_TF32, C, view1(ldc_floats / 2), view1(1), alpha, accumulate, 0,
               device_err(), st);
}

// The tensor-core accumulation error was measured to grow linearly with the chain length,
// so the split passes keep every accumulator to at most 64 K blocks (2048 real K in TF32, 4096
// in BF16) and sum the partial tiles in FP32.
void tc_gemm_seg_v(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int64_t Nreal, int64_t Kseg,
                   int seg, int kind, float *C, View2 rv, View2 cv, zc alpha, bool accumulate, cudaStream_t st) {
  int *err = device_err();
  if (seg == 1) {
    tc_gemm_core(A, lda, B, ldb, M, Nreal, Kseg, kind, C, rv, cv, alpha, accumulate, 0, err, st);
    return;
  }
  const int64_t es = tc_esize(kind);
  tc_gemm_core((const char *)A + Kseg * es, lda, (const char *)B + Kseg * es, ldb, M, Nreal, 2 * Kseg, kind, C, rv,
               cv, alpha, accumulate, 64, err, st);
  tc_gemm_core(A, lda, B, ldb, M, Nreal, Kseg, kind, C, rv, cv, alpha, true, 64, err, st);
}

void tc_gemm_a_inplace(const void *A, int64_t lda_cpx, int64_t K, const float *B, int64_t ldb, int64_t M,
                       int64_t Nreal, float *C, View2 rv, View2 cv, zc alpha, bool accumulate, cudaStream_t st) {
  tc_gemm_core(A, 2 * lda_cpx, B, ldb, M, Nreal, 2 * tc_kpad(K), TC_TF32, C, rv, cv, alpha, accumulate, 0,
               device_err(), st, 2 * K);
}

bool tc_a_inplace_ok(const void *A, int64_t lda_cpx, int64_t K) {
  return ((uintptr_t)A % 16) == 0 && lda_cpx % 2 == 0 && lda_cpx >= K && 8 * lda_cpx < (1ll << 40);
}

void tc_gemm_seg(const void *A, int64_t lda, const void *B, int64_t ldb, int64_t M, int64_t Nreal, int64_t Kseg,
                 int seg, int kind, float *C, int64_t ldc_floats, zc alpha, bool accumulate, cudaStream_t st) {
  tc_gemm_seg_v(A, lda, B, ldb, M, Nreal, Kseg, seg, kind, C, view1(ldc_floats / 2), view1(1), alpha, accumulate, st);
}

void tc_setup_device_flagged() {
  std::call_once(g_enc_once, fetch_encoder);
  set_smem_limits();
}

void tc_gemm_seg_flagged(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t M, int64_t Nreal,
                         int64_t Kseg, int seg, float *C, int64_t ldc_floats, zc alpha, bool accumulate,
                         int *err, cudaStream_t st) {
  CCLR_REQUIRE(g_encode != nullptr, "tc_gemm_seg_flagged: tc_setup_device_flagged was not called");
  const View2 rv = view1(ldc_floats / 2), cv = view1(1);
  if (seg == 1) {
    tc_gemm_core(A, lda, B, ldb, M, Nreal, Kseg, TC_TF32, C, rv, cv, alpha, accumulate, 0, err, st);
    return;
  }
  tc_gemm_core(A + Kseg, lda, B + Kseg, ldb, M, Nreal, 2 * Kseg, TC_TF32, C, rv, cv, alpha, accumulate, 64, err, st);
  tc_gemm_core(A, lda, B, ldb, M, Nreal, Kseg, TC_TF32, C, rv, cv, alpha, true, 64, err, st);
}

int tc_selftest_timeout(int timeout_us, cudaStream_t st) {
  wait_never_kernel<<<1, 32, 0, st>>>((unsigned long long)timeout_us * 1000ull, device_err());
  count_launch();
  CCLR_CUDA(cudaGetLastError());
  return tc_error(st);
}

void tc_set_autotune(bool on) { g_tune_on = on; }

int tc_tuning_table(int cap, double *rec) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lock(g_tune_mu);
  int n = 0;
  for (const auto &kv : g_tune) {
    if (kv.first.dev != dev) continue;
    if (n < cap && rec) {
      double *r = rec + 10 * n;
      const TuneKey &k = kv.first;
      const TuneRec &t = kv.second;
      r[0] = k.kind; r[1] = (double)k.M; r[2] = (double)k.N; r[3] = (double)k.K;
      r[4] = t.cfg.BN; r[5] = t.cfg.splits; r[6] = t.cfg.band;
      r[7] = t.ms_best; r[8] = t.ms_rule; r[9] = t.tried;
    }
    ++n;
  }
  return n;
}

int tc_error(cudaStream_t st) {
  int *g_err = nullptr;
  {
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_dev_mu);
    g_err = g_err_dev[dev];
  }
  if (!g_err) return 0;
  int h = 0;
  CCLR_CUDA(cudaMemcpyAsync(&h, g_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CCLR_CUDA(cudaStreamSynchronize(st));
  if (h) CCLR_CUDA(cudaMemsetAsync(g_err, 0, sizeof(int), st));
  return h;
}

}  // namespace cclr
