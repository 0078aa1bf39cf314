// Multi-right-hand-side complex matrix product Y = A X on the tcgen05 tensor cores (step a11).
//
// The complex matrix A (n x n, re/im interleaved) is read as a real n x 2n matrix that is contiguous along
// K, and the block X (nrhs <= 64 columns) becomes a real K-major operand Bt of 128 rows:
// Bt[s] = (Re x_s, -Im x_s) pairs and Bt[64+s] = (Im x_s, Re x_s) pairs, so that one real GEMM
// D = A_real Bt^T gives D[r][s] = Re y_s[r] and D[r][64+s] = Im y_s[r].
//
// Precision: FP16 x 3 with power-of-two scaling.  Row r of A is scaled by 2^-e_r so that its largest
// magnitude lies in [1/2, 1); each scaled value v is written as hi = fp16(v) and lo = fp16(2^11 (v - hi)),
// 22 significant bits in all.  Bt is split the same way with one scale per right-hand side.  The tensor
// cores accumulate D1 = A_hi B_hi and D2 = A_lo B_hi + A_hi B_lo in FP32 (two TMEM accumulators; the
// lo x lo term is below the FP32 rounding of the result) and the epilogue forms
// (D1 + 2^-11 D2) / (2^-e_r t_s).  Values far below a row's largest entry fall into FP16's subnormal range,
// where hi and lo still hold them to an absolute error of ~1e-11 of that largest entry.  A's split is made
// once per assembled matrix (tc_prepare_a) and costs no more memory traffic per product than complex FP32:
// 2 x 2 bytes per real entry.  FP16 operands move half the bytes of TF32 ones through shared memory and run
// at twice the rate, so the product is bound by streaming A from HBM.
//
// Work split (stream-K): the (row tile, K-step) pairs of the whole product are cut into G equal contiguous
// ranges, G a multiple of the SM count with G >= row tiles, so every CTA does the same amount of work and
// touches at most two row tiles.  Each CTA writes one partial 128 x 128 tile per row tile it touches
// (column-major, tc_operand.cuh); a reduction kernel, or the GMRES iteration kernel as it stages w, adds the
// partials of each tile in CTA order (deterministic) and applies the scales.
//
// CTA roles (256 threads): warp 0 = TMA producer, warp 1 = TMEM owner and MMA issuer, warps 4-7 =
// accumulator readers (TMEM lanes 0-127).  3 pipeline stages of 64 KB (A_hi, A_lo, B_hi, B_lo tiles of
// 128 x 64 FP16, 128-byte swizzle).  TMEM holds two buffers of (D1, D2), 512 columns; every kSeg K-steps (and
// at a row-tile boundary) the MMA warp switches buffers and the readers fold the finished one into FP32
// registers, which bounds the length of each tensor-core accumulation chain.
//
// Every mbarrier wait is bounded by the global timer; on expiry the kernel records an error code, stops
// issuing work, waits (bounded) for its own in-flight copies and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <atomic>
#include <cstdio>

#include "internal.cuh"
#include "tc_operand.cuh"

namespace bem {

namespace {

constexpr int kM = kTcM;             // rows per tile (UMMA M)
constexpr int kN = kTcN;             // Bt rows: 64 real parts + 64 imaginary parts
constexpr int kKs = 64;              // FP16 elements per K-step = 128 bytes = one swizzle row
constexpr int kStages = 3;
constexpr int kSeg = 4;              // K-steps per accumulation segment (256 K values)
constexpr int kTile = kM * kKs * 2;  // 16 KB
constexpr int kStage = 4 * kTile;    // A_hi, A_lo, B_hi, B_lo
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 512;  // two buffers x (D1, D2) x 128 FP32 columns
constexpr int kMaxRhs = 64;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s
constexpr int kMaxDev = 64;

struct Bars {
  unsigned long long full[kStages];
  unsigned long long empty[kStages];
  unsigned long long accf[2];
  unsigned long long acce[2];
  unsigned long long fin;
  uint32_t tmem;
};
constexpr int kSmemBytes = kStages * kStage + 1024 + (int)sizeof(Bars) + 64;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error code recorded) if the phase does not complete within limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* err, int code,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_try(a, parity)) return true;
    if (gtime() - t0 > limit_ns) {
      atomicCAS(err, 0, code);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B FP16, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(kIdesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Row stride (FP16 elements) of the split copies of A and of Bt: 2n rounded up to 8 (16-byte TMA strides).
inline size_t ld16(int n) { return ((size_t)2 * n + 7) & ~(size_t)7; }

// The accumulation schedule of one CTA's range [kb, kb + nk) of global K-steps (kpt K-steps per row tile):
// a segment ends after kSeg K-steps, at the end of a row tile and at the end of the range.  MMA issuer and
// readers walk it identically.
struct SegWalk {
  int kb, nk, kpt;
  int it = 0;                  // next K-step (relative to kb)
  __device__ bool next(int& beg, int& end, bool& tile_end) {
    if (it >= nk) return false;
    beg = it;
    const int g = kb + it;
    const int to_tile_end = kpt - g % kpt;
    int len = kSeg < to_tile_end ? kSeg : to_tile_end;
    if (len > nk - it) len = nk - it;
    end = it + len;
    tile_end = (len == to_tile_end) || (end == nk);
    it = end;
    return true;
  }
};

// One CTA per stream-K range.  partial: G x 2 x kM x kN FP32 (slot 0 = first row tile of the range, 1 = the
// next one).  wait_ns bounds the waits of the main loop (normally kWaitNs); the waits that drain this CTA's
// own copies and MMAs before it releases TMEM always keep kWaitNs.
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
              const __grid_constant__ CUtensorMap mapBh, const __grid_constant__ CUtensorMap mapBl, int n,
              int kpt, long long total, float* partial, int* err, const int* gate, unsigned long long wait_ns,
              const int* relax) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Bars* bars = reinterpret_cast<Bars*>(smem + kStages * kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, c = blockIdx.x;
  int kb, nk;
  if ((unsigned long long)total * (unsigned long long)G < (1ull << 32)) {   // 32-bit divisions where they fit
    const unsigned t = (unsigned)total, g = (unsigned)G;
    kb = (int)(t * (unsigned)c / g);
    nk = (int)(t * (unsigned)(c + 1) / g) - kb;
  } else {
    const long long gb = total * c / G, ge = total * (c + 1) / G;
    kb = (int)gb;
    nk = (int)(ge - gb);
  }
  const int tile0 = kb / kpt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(su32(&bars->full[s]), 1);
      mbar_init(su32(&bars->empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(su32(&bars->accf[b]), 1);
      mbar_init(su32(&bars->acce[b]), 128);
    }
    mbar_init(su32(&bars->fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&bars->tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem;
  // The set-up above overlaps the previous kernel's tail; its outputs (the B operand, the gate) are read only
  // from here on.
  pdl_enter();
  if (gate && *gate == 0) {   // every system of the block has converged (uniform for the grid)
    if (warp == 1)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    return;
  }
  // relaxed product: the FP16 remainders of A and of Bt are neither loaded nor multiplied, only hi x hi (uniform
  // for the grid); counted in the word after the error word
  const bool hi_only = relax && *relax == 0;
  if (hi_only && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(err + 1, 1);
  int issued = 0;   // TMA stages issued by the producer thread

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int st = it % kStages;
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        if (!mbar_wait(su32(&bars->empty[st]), ph ^ 1u, err, 1, wait_ns)) break;
        if (*(volatile int*)err) break;
        unsigned char* base = smem + st * kStage;
        const uint32_t fb = su32(&bars->full[st]);
        mbar_expect_tx(fb, (hi_only ? 2 : 4) * kTile);
        const int g = kb + it;
        const int x = (g % kpt) * kKs, y = (g / kpt) * kM;
        tma_load_2d(su32(base), &mapAh, x, y, fb);
        if (!hi_only) tma_load_2d(su32(base + kTile), &mapAl, x, y, fb);
        tma_load_2d(su32(base + 2 * kTile), &mapBh, x, 0, fb);
        if (!hi_only) tma_load_2d(su32(base + 3 * kTile), &mapBl, x, 0, fb);
        issued = it + 1;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      SegWalk w{kb, nk, kpt};
      int beg, end, seg = 0;
      bool tile_end;
      while (ok && w.next(beg, end, tile_end)) {
        const int b = seg & 1;
        // the buffer must have been drained by the readers (segments seg-2, seg-4, ...)
        if (!mbar_wait(su32(&bars->acce[b]), (uint32_t)(((seg >> 1) & 1) ^ 1), err, 2, wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d1 = tmem + (uint32_t)(b * 2 * kN), d2 = d1 + (uint32_t)kN;
        for (int it = beg; it < end; ++it) {
          const int st = it % kStages;
          const uint32_t ph = (uint32_t)((it / kStages) & 1);
          if (!mbar_wait(su32(&bars->full[st]), ph, err, 3, wait_ns)) { ok = false; break; }
          tc_fence_after();
          unsigned char* base = smem + st * kStage;
          const uint64_t dah = sdesc(su32(base)), dal = sdesc(su32(base + kTile));
          const uint64_t dbh = sdesc(su32(base + 2 * kTile)), dbl = sdesc(su32(base + 3 * kTile));
#pragma unroll
          for (int k = 0; k < kKs / 16; ++k) {
            const uint64_t off = (uint64_t)((k * 32) >> 4);   // 16 FP16 = 32 bytes along the swizzled row
            const uint32_t acc0 = (it == beg && k == 0) ? 0u : 1u;
            mma_f16(d1, dah + off, dbh + off, acc0);
            if (!hi_only) {
              mma_f16(d2, dal + off, dbh + off, acc0);
              mma_f16(d2, dah + off, dbl + off, 1u);
            }
          }
          mma_commit(su32(&bars->empty[st]));
        }
        if (!ok) break;
        mma_commit(su32(&bars->accf[b]));
        ++seg;
      }
      // all MMAs issued by this thread complete before `fin` arrives
      mma_commit(su32(&bars->fin));
    }
  } else if (warp >= 4) {
    // ---------------- accumulator readers (128 threads, TMEM lanes 0..127) ----------------
    const int q = warp - 4;
    float acc[kN];
#pragma unroll
    for (int j = 0; j < kN; ++j) acc[j] = 0.f;
    bool ok = true;
    SegWalk w{kb, nk, kpt};
    int beg, end, seg = 0, slot = 0;
    bool tile_end;
    while (ok && w.next(beg, end, tile_end)) {
      const int b = seg & 1;
      // the TMEM loads below are warp-collective: the whole warp proceeds or stops together
      ok = __all_sync(0xffffffffu, mbar_wait(su32(&bars->accf[b]), (uint32_t)((seg >> 1) & 1), err, 5, wait_ns));
      if (!ok) break;
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 2 * kN);
#pragma unroll
      for (int cc = 0; cc < kN / 32; ++cc) {
        float v[32];
        tmem_ld32(ta + (uint32_t)(cc * 32), v);                  // D1
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[cc * 32 + i] += v[i];
        if (!hi_only) {   // D2 (lo terms times 2^11) is not written by a relaxed product
          tmem_ld32(ta + (uint32_t)(kN + cc * 32), v);
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[cc * 32 + i] = fmaf(v[i], 1.f / kTcLoScale, acc[cc * 32 + i]);
        }
      }
      tc_fence_before();
      mbar_arrive(su32(&bars->acce[b]));
      ++seg;
      if (tile_end) {
        // column-major partial tile: for each column the warp's 32 rows are 128 contiguous bytes
        float* dst = partial + ((size_t)c * 2 + slot) * kM * kN + q * 32 + lane;
#pragma unroll
        for (int j = 0; j < kN; ++j) {
          dst[(size_t)j * kM] = acc[j];
          acc[j] = 0.f;
        }
        ++slot;
      }
    }
  }

  // make sure no copy or MMA of this CTA is still in flight before TMEM is released
  __syncwarp();
  if (warp == 1 && lane == 0) mbar_wait(su32(&bars->fin), 0u, err, 6);
  if (warp == 0 && lane == 0 && *(volatile int*)err) {
    // drain TMA loads that were issued but possibly not consumed (the last kStages issues); a phase that
    // the MMA warp already consumed reads as complete because nothing newer was issued on it
    for (int it = (issued > kStages ? issued - kStages : 0); it < issued; ++it)
      mbar_wait(su32(&bars->full[it % kStages]), (uint32_t)((it / kStages) & 1), err, 7);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  (void)tile0;
}

// Largest |value| of each column block of X (one per right-hand side), as float bits for atomicMax
// (non-negative floats order like their bit patterns).
__global__ void k_tc_colmax(const float2* __restrict__ x, int n, int nrhs, unsigned* __restrict__ cmax,
                            const int* gate) {
  if (gate && *gate == 0) return;
  const int s = blockIdx.y;
  float m = 0.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const float2 v = x[(size_t)s * n + c];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(cmax + s, __float_as_uint(m));
}

// 2^-e with m 2^e = v, m in [1/2, 1) (1 for v = 0): the power-of-two scale that maps v into [1/2, 1).
__device__ __forceinline__ float pow2_scale(float v) {
  if (!(v > 0.f)) return 1.f;
  int e;
  frexpf(v, &e);
  return ldexpf(1.f, -e);
}

// Bt rows (K-major, ld16(n) FP16 each): row s < 64: (Re x_s[c], -Im x_s[c]); row 64+s: (Im x_s[c], Re x_s[c]),
// scaled by t_s = pow2_scale(max |x_s|) and split into hi and lo; rows of absent columns are zero.
__global__ void k_tc_prep_b(const float2* __restrict__ x, int n, int nrhs, const unsigned* __restrict__ cmax,
                            __half* __restrict__ bhi, __half* __restrict__ blo, size_t ldb, float* __restrict__ tsc,
                            const int* gate) {
  if (gate && *gate == 0) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;   // complex column index along K
  const int s = blockIdx.y;                               // 0..63
  if (c >= n) return;
  float re = 0.f, im = 0.f, t = 1.f;
  if (s < nrhs) {
    t = pow2_scale(__uint_as_float(cmax[s]));
    const float2 xv = x[(size_t)s * n + c];
    re = xv.x * t;
    im = xv.y * t;
  }
  if (c == 0) tsc[s] = t;
  tc_write_b(bhi, blo, ldb, s, c, re, im);
}

// Split copy of A: one CTA per row; row scale 2^-e_r from the row's largest |real entry|.
__global__ void __launch_bounds__(256) k_tc_prep_a(const float2* __restrict__ A, int n, __half* __restrict__ ahi,
                                                   __half* __restrict__ alo, size_t lda16, float* __restrict__ rsc) {
  __shared__ float red[8];
  const int r = blockIdx.x;
  const float2* row = A + (size_t)r * n;
  float m = 0.f;
  for (int c = threadIdx.x; c < n; c += 256) m = fmaxf(m, fmaxf(fabsf(row[c].x), fabsf(row[c].y)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
  const float sc = pow2_scale(m);
  if (threadIdx.x == 0) rsc[r] = sc;
  __half* hr = ahi + (size_t)r * lda16;
  __half* lr = alo + (size_t)r * lda16;
  for (int c = threadIdx.x; c < n; c += 256) {
    const float2 v = row[c];
    __half2 h, l;
    tc_split16x2(v.x * sc, v.y * sc, h, l);
    *reinterpret_cast<__half2*>(hr + 2 * c) = h;
    *reinterpret_cast<__half2*>(lr + 2 * c) = l;
  }
}

// Y[s][r] = (sum of the partials of r's row tile) / (rsc[r] tsc[s]), the real part from column s of D and
// the imaginary part from column 64 + s.  One CTA per kRedRows rows of one row tile; lane = row, so every load
// of a partial column and every store of Y is 128 contiguous bytes; warp w takes systems w, w + 8, ...; the
// partials are summed in CTA order (deterministic).
constexpr int kRedRows = 32;
__global__ void __launch_bounds__(256) k_tc_reduce(const float* __restrict__ partial, int n, int nrhs, int kpt,
                                                   long long total, int G, const float* __restrict__ rsc,
                                                   const float* __restrict__ tsc, float2* __restrict__ y,
                                                   const int* gate) {
  pdl_enter();
  if (gate && *gate == 0) return;
  __shared__ int src[kTcMaxCover];   // partial tiles covering this row tile, in CTA order (2 c + slot)
  __shared__ int nsrc;
  const int r0 = blockIdx.x * kRedRows;
  if (threadIdx.x == 0) nsrc = tc_cover(r0 / kM, kpt, total, G, src, kTcMaxCover);
  __syncthreads();
  const int ns = nsrc;
  const int r = r0 + (threadIdx.x & 31);
  if (r >= n) return;
  const int rr = r % kM;
  const float rs = rsc[r];
  for (int sidx = threadIdx.x >> 5; sidx < nrhs; sidx += 8) {
    float re = 0.f, im = 0.f;
    for (int q = 0; q < ns; ++q) {
      const float* t = partial + (size_t)src[q] * kM * kN + rr;
      re += t[(size_t)sidx * kM];
      im += t[(size_t)(64 + sidx) * kM];
    }
    const float inv = 1.f / (rs * (tsc ? tsc[sidx] : 1.f));   // a power of two: exact
    y[(size_t)sidx * n + r] = make_float2(re * inv, im * inv);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// rows x cols FP16 (row stride ld16 elements), box 64 x 128, 128-byte swizzle, zero fill out of bounds
bool make_map16(CUtensorMap* m, const void* base, int cols, size_t ld, int rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kKs, (cuuint32_t)kM};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
  int s = cache[dev].load(std::memory_order_relaxed);
  if (s > 0) return s;
  if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) s = 1;
  cache[dev].store(s, std::memory_order_relaxed);
  return s;
}

// Stream-K grid: a multiple of the SM count, at least the number of row tiles (so a range spans at most two
// tiles), and at most one CTA per K-step.
int grid_of(int n) {
  const int tiles = (n + kM - 1) / kM;
  const long long total = (long long)tiles * (((long long)2 * n + kKs - 1) / kKs);
  const int sms = num_sms();
  long long g = (long long)sms * ((tiles + sms - 1) / sms);
  if (g > total) g = total;
  return (int)g;
}

size_t b_bytes(int n) { return (size_t)kN * ld16(n) * 2; }

// Main-loop wait limit of the kernels launched from now on (graphs keep the value they were recorded with).
std::atomic<unsigned long long> g_wait_ns{kWaitNs};

bool smem_attr_set() {
  static std::atomic<int> done[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return false;
  if (done[dev].load(std::memory_order_relaxed)) return true;
  if (cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
    return false;
  done[dev].store(1, std::memory_order_relaxed);
  return true;
}

// workspace layout: B_hi | B_lo | partials | column max (64 u32) | column scales (64 f32) | error word
size_t off_part(int n) { return (2 * b_bytes(n) + 255) & ~(size_t)255; }
size_t off_cmax(int n) { return off_part(n) + (size_t)grid_of(n) * 2 * kM * kN * 4; }
size_t off_tsc(int n) { return off_cmax(n) + 256; }
size_t off_err(int n) { return off_tsc(n) + 256; }

}  // namespace

bool matvec_tc_supported(int n, int nrhs) {
  return nrhs >= 2 && nrhs <= kMaxRhs && n >= kM && (n % 2) == 0 && encode_fn() != nullptr;
}

size_t matvec_tc_workspace_bytes(int n, int nrhs) {
  if (nrhs < 2 || nrhs > kMaxRhs || n < kM) return 0;
  return off_err(n) + 64;
}

bool matvec_tc_partials(const void* a16, int n, int nrhs, void* ws, TcPartials* out) {
  if (!matvec_tc_supported(n, nrhs) || !out) return false;
  const size_t ld = ld16(n);
  out->part = reinterpret_cast<const float*>(static_cast<const char*>(ws) + off_part(n));
  out->rsc = reinterpret_cast<const float*>(static_cast<const char*>(a16) +
                                            ((2 * (size_t)n * ld * 2 + 255) & ~(size_t)255));
  out->kpt = (2 * n + kKs - 1) / kKs;
  out->total = (long long)((n + kM - 1) / kM) * out->kpt;
  out->G = grid_of(n);
  return true;
}

int* matvec_tc_error_word(void* ws, int n, int nrhs) {
  if (nrhs < 2 || nrhs > kMaxRhs || n < kM) return nullptr;
  return reinterpret_cast<int*>(static_cast<char*>(ws) + off_err(n));
}

cudaError_t matvec_tc_clear_error(void* ws, int n, int nrhs, cudaStream_t s) {
  int* err = matvec_tc_error_word(ws, n, nrhs);
  if (!err) return cudaErrorInvalidValue;
  return cudaMemsetAsync(err, 0, 2 * sizeof(int), s);   // the error word and the relaxed-launch count
}

size_t matvec_tc_a16_bytes(int n) { return ((2 * (size_t)n * ld16(n) * 2 + 255) & ~(size_t)255) + (size_t)n * 4; }

cudaError_t launch_tc_prepare_a(const float2* A, int n, void* a16, cudaStream_t s) {
  if (n < kM || (n % 2) != 0) return cudaErrorInvalidValue;
  const size_t ld = ld16(n);
  __half* ahi = static_cast<__half*>(a16);
  __half* alo = ahi + (size_t)n * ld;
  float* rsc = reinterpret_cast<float*>(static_cast<char*>(a16) + ((2 * (size_t)n * ld * 2 + 255) & ~(size_t)255));
  k_tc_prep_a<<<n, 256, 0, s>>>(A, n, ahi, alo, ld, rsc);
  return cudaGetLastError();
}

cudaError_t launch_matvec_tc(const void* a16, int n, int nrhs, const float2* x, float2* y, void* ws,
                             size_t ws_bytes, cudaStream_t s, const int* gate, int stage, const int* relax) {
  if (!matvec_tc_supported(n, nrhs)) return cudaErrorNotSupported;
  if (ws_bytes < matvec_tc_workspace_bytes(n, nrhs)) return cudaErrorInvalidValue;
  const size_t ld = ld16(n);
  const __half* ahi = static_cast<const __half*>(a16);
  const __half* alo = ahi + (size_t)n * ld;
  const float* rsc =
      reinterpret_cast<const float*>(static_cast<const char*>(a16) + ((2 * (size_t)n * ld * 2 + 255) & ~(size_t)255));
  char* w = static_cast<char*>(ws);
  __half* bhi = reinterpret_cast<__half*>(w);
  __half* blo = reinterpret_cast<__half*>(w + b_bytes(n));
  float* part = reinterpret_cast<float*>(w + off_part(n));
  unsigned* cmax = reinterpret_cast<unsigned*>(w + off_cmax(n));
  float* tsc = reinterpret_cast<float*>(w + off_tsc(n));
  int* err = reinterpret_cast<int*>(w + off_err(n));
  const int cols = 2 * n;
  const int tiles = (n + kM - 1) / kM;
  const int kpt = (cols + kKs - 1) / kKs;
  const long long total = (long long)tiles * kpt;
  const int G = grid_of(n);
  if (stage == 2)   // the reduction alone (its partials come from a stage-1 call with the same arguments)
    return launch_pdl(k_tc_reduce, dim3((n + kRedRows - 1) / kRedRows), dim3(256), 0, s, part, n, nrhs, kpt, total,
                      G, rsc, x ? tsc : static_cast<const float*>(nullptr), y, gate);
  CUtensorMap mAh, mAl, mBh, mBl;
  if (!make_map16(&mAh, ahi, cols, ld, n) || !make_map16(&mAl, alo, cols, ld, n) ||
      !make_map16(&mBh, bhi, cols, ld, kN) || !make_map16(&mBl, blo, cols, ld, kN))
    return cudaErrorInvalidValue;
  if (!smem_attr_set()) return cudaErrorInvalidValue;
  if (x) {
    cudaError_t e = cudaMemsetAsync(cmax, 0, 64 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
  }
  if (x) {
    k_tc_colmax<<<dim3(8, nrhs), 256, 0, s>>>(x, n, nrhs, cmax, gate);
    k_tc_prep_b<<<dim3((n + 255) / 256, kMaxRhs), 256, 0, s>>>(x, n, nrhs, cmax, bhi, blo, ld, tsc, gate);
  }
  cudaError_t e = launch_pdl(k_gemm_tc, dim3(G), dim3(kThreads), kSmemBytes, s, mAh, mAl, mBh, mBl, n, kpt, total,
                             part, err, gate, g_wait_ns.load(std::memory_order_relaxed), relax);
  if (e != cudaSuccess || stage == 1) return e;
  return launch_pdl(k_tc_reduce, dim3((n + kRedRows - 1) / kRedRows), dim3(256), 0, s, part, n, nrhs, kpt, total, G,
                    rsc, x ? tsc : static_cast<const float*>(nullptr), y, gate);
}

void matvec_tc_b_operand(void* ws, int n, void** bhi, void** blo, size_t* ldb) {
  *bhi = ws;
  *blo = static_cast<char*>(ws) + b_bytes(n);
  *ldb = ld16(n);
}

size_t matvec_tc_b_bytes(int n) { return 2 * b_bytes(n); }

cudaError_t matvec_tc_setup() { return smem_attr_set() && encode_fn() ? cudaSuccess : cudaErrorNotSupported; }

void matvec_tc_set_wait_ns(unsigned long long ns) { g_wait_ns.store(ns ? ns : kWaitNs, std::memory_order_relaxed); }

}  // namespace bem
