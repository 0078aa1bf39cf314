// Multi-right-hand-side complex matrix product Y = A X on the tcgen05 tensor cores (step a11).
//
// The complex FP32 matrix A (n x n, row-major, re/im interleaved) is read as a real n x 2n matrix that
// is contiguous along K, and the block X (nrhs <= 64 columns) becomes a real K-major operand Bt of 128
// rows:  Bt[s] = (Re x_s, -Im x_s) pairs and Bt[64+s] = (Im x_s, Re x_s) pairs, so that one real GEMM
// D = A_real Bt^T gives D[r][s] = Re y_s[r] and D[r][64+s] = Im y_s[r].
//
// Precision: 3xTF32 split.  Each FP32 value v is written as hi + lo with hi = v with its 13 low mantissa
// bits cleared (exactly representable in TF32) and lo = v - hi; D accumulates A_hi B_hi + A_hi B_lo +
// A_lo B_hi in FP32, which keeps the products at about FP32 accuracy.  B is split once by a prep kernel;
// A is split inside the GEMM: TMA brings an FP32 tile into shared memory and two converter warps rewrite
// it in place as hi and write lo beside it (same swizzled positions, so the same descriptors apply).
//
// Tiling: one CTA per (128-row tile, K split); 3 pipeline stages of 64 KB (A, A_lo, B_hi, B_lo tiles of
// 128 x 32 FP32, 128-byte swizzle).  Warp roles: 0 = TMA producer, 1 = TMEM owner and MMA issuer,
// 2-3 = split converters, 4-7 = accumulator readers.  The accumulator lives in TMEM as two 128 x 128 FP32
// buffers; every kSeg K-steps the MMA warp switches buffers and the reader warps add the finished buffer
// into FP32 registers, which bounds the length of each tensor-core accumulation chain.  Partial results
// of the K splits are summed by a small reduction kernel that also writes Y in complex layout.
//
// Every mbarrier wait is bounded by the global timer; on expiry the kernel records an error code, stops
// issuing work, waits (bounded) for its own in-flight copies and MMAs, frees its TMEM and returns.
#include <cuda.h>

#include <cstdio>

#include "internal.cuh"

namespace bem {

namespace {

constexpr int kM = 128;              // rows per CTA (UMMA M)
constexpr int kN = 128;              // Bt rows: 64 real parts + 64 imaginary parts
constexpr int kKs = 32;              // FP32 elements per K-step = 128 bytes = one swizzle row
constexpr int kStages = 3;
constexpr int kSeg = 8;              // K-steps per accumulation segment
constexpr int kTile = kM * kKs * 4;  // 16 KB
constexpr int kStage = 4 * kTile;    // A, A_lo, B_hi, B_lo
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 256;  // two 128-column FP32 accumulators
constexpr int kMaxRhs = 64;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

struct Bars {
  unsigned long long full[kStages];
  unsigned long long conv[kStages];
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
// Bounded wait: false (and the error code recorded) if the phase does not complete within kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* err, int code) {
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = gtime();
  while (true) {
    if (mbar_try(a, parity)) return true;
    if (gtime() - t0 > kWaitNs) {
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

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
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

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBhi,
              const __grid_constant__ CUtensorMap mapBlo, int n, int ksteps_total, int nsplit, float* partial,
              int* err, const int* gate) {
  if (gate && *gate == 0) return;   // every system of the block has converged (uniform for the grid)
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Bars* bars = reinterpret_cast<Bars*>(smem + kStages * kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, split = blockIdx.y;
  const int kb = (int)(((long long)ksteps_total * split) / nsplit);
  const int ke = (int)(((long long)ksteps_total * (split + 1)) / nsplit);
  const int nk = ke - kb;
  const int nseg = (nk + kSeg - 1) / kSeg;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(su32(&bars->full[s]), 1);
      mbar_init(su32(&bars->conv[s]), 64);
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
  int issued = 0;   // TMA stages issued by the producer thread

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      for (int it = 0; it < nk; ++it) {
        const int st = it % kStages;
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        if (!mbar_wait(su32(&bars->empty[st]), ph ^ 1u, err, 1)) break;
        if (*(volatile int*)err) break;
        unsigned char* base = smem + st * kStage;
        const uint32_t fb = su32(&bars->full[st]);
        mbar_expect_tx(fb, 3 * kTile);
        const int x = (kb + it) * kKs;
        tma_load_2d(su32(base), &mapA, x, tile * kM, fb);
        tma_load_2d(su32(base + 2 * kTile), &mapBhi, x, 0, fb);
        tma_load_2d(su32(base + 3 * kTile), &mapBlo, x, 0, fb);
        issued = it + 1;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      for (int it = 0; it < nk && ok; ++it) {
        const int st = it % kStages;
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        const int seg = it / kSeg;
        const int b = seg & 1;
        const bool seg_first = (it % kSeg) == 0;
        const bool seg_last = ((it % kSeg) == kSeg - 1) || (it == nk - 1);
        if (seg_first) {
          // the accumulator buffer must have been drained by the readers (segments seg-2, seg-4, ...)
          if (!mbar_wait(su32(&bars->acce[b]), (uint32_t)(((seg >> 1) & 1) ^ 1), err, 2)) { ok = false; break; }
          tc_fence_after();
        }
        if (!mbar_wait(su32(&bars->conv[st]), ph, err, 3)) { ok = false; break; }
        tc_fence_after();
        unsigned char* base = smem + st * kStage;
        const uint64_t da = sdesc(su32(base)), dal = sdesc(su32(base + kTile));
        const uint64_t dbh = sdesc(su32(base + 2 * kTile)), dbl = sdesc(su32(base + 3 * kTile));
        const uint32_t dt = tmem + (uint32_t)(b * kN);
#pragma unroll
        for (int k = 0; k < kKs / 8; ++k) {
          const uint64_t off = (uint64_t)((k * 32) >> 4);   // 8 TF32 = 32 bytes along the swizzled row
          const uint32_t acc0 = (seg_first && k == 0) ? 0u : 1u;
          mma_tf32(dt, da + off, dbh + off, acc0);
          mma_tf32(dt, da + off, dbl + off, 1u);
          mma_tf32(dt, dal + off, dbh + off, 1u);
        }
        mma_commit(su32(&bars->empty[st]));
        if (seg_last) mma_commit(su32(&bars->accf[b]));
      }
      // all MMAs issued by this thread complete before `fin` arrives
      mma_commit(su32(&bars->fin));
    }
  } else if (warp < 4) {
    // ---------------- split converters (64 threads) ----------------
    const int t = threadIdx.x - 64;
    for (int it = 0; it < nk; ++it) {
      const int st = it % kStages;
      const uint32_t ph = (uint32_t)((it / kStages) & 1);
      if (!mbar_wait(su32(&bars->full[st]), ph, err, 4)) break;
      float4* a = reinterpret_cast<float4*>(smem + st * kStage);
      float4* al = reinterpret_cast<float4*>(smem + st * kStage + kTile);
#pragma unroll 4
      for (int i = 0; i < kTile / 16 / 64; ++i) {
        const int idx = i * 64 + t;
        const float4 v = a[idx];
        float4 h, l;
        h.x = tf32_hi(v.x); h.y = tf32_hi(v.y); h.z = tf32_hi(v.z); h.w = tf32_hi(v.w);
        l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
        a[idx] = h;
        al[idx] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(su32(&bars->conv[st]));
    }
  } else {
    // ---------------- accumulator readers (128 threads, TMEM lanes 0..127) ----------------
    const int q = warp - 4;
    float acc[kN];
#pragma unroll
    for (int c = 0; c < kN; ++c) acc[c] = 0.f;
    bool ok = true;
    for (int seg = 0; seg < nseg && ok; ++seg) {
      const int b = seg & 1;
      // the TMEM loads below are warp-collective: the whole warp proceeds or stops together
      ok = __all_sync(0xffffffffu, mbar_wait(su32(&bars->accf[b]), (uint32_t)((seg >> 1) & 1), err, 5));
      if (!ok) break;
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kN);
#pragma unroll
      for (int c = 0; c < kN / 32; ++c) {
        float v[32];
        tmem_ld32(ta + (uint32_t)(c * 32), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[c * 32 + i] += v[i];
      }
      tc_fence_before();
      mbar_arrive(su32(&bars->acce[b]));
    }
    const int row = tile * kM + q * 32 + lane;
    if (ok && row < n) {
      float4* dst = reinterpret_cast<float4*>(partial + ((size_t)split * n + row) * kN);
#pragma unroll
      for (int c = 0; c < kN / 4; ++c) dst[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
    }
  }

  // make sure no copy or MMA of this CTA is still in flight before TMEM is released
  __syncwarp();
  if (warp == 1 && lane == 0) mbar_wait(su32(&bars->fin), 0u, err, 6);
  if (warp == 0 && lane == 0 && *(volatile int*)err) {
    // drain TMA loads that were issued but possibly not consumed (the last kStages issues); a phase that
    // the converters already consumed reads as complete because nothing newer was issued on it
    for (int it = (issued > kStages ? issued - kStages : 0); it < issued; ++it)
      mbar_wait(su32(&bars->full[it % kStages]), (uint32_t)((it / kStages) & 1), err, 7);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Bt rows (K-major, 2n FP32 each): row s < 64: (Re x_s[c], -Im x_s[c]); row 64+s: (Im x_s[c], Re x_s[c]);
// rows of absent columns are zero.  Written as TF32-exact hi and lo = v - hi.
__global__ void k_tc_prep_b(const float2* __restrict__ x, int n, int nrhs, float* __restrict__ bhi,
                            float* __restrict__ blo, const int* gate) {
  if (gate && *gate == 0) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;   // complex column index along K
  const int row = blockIdx.y;                             // 0..127
  if (c >= n) return;
  const int s = row & 63;
  float v0 = 0.f, v1 = 0.f;
  if (s < nrhs) {
    const float2 xv = x[(size_t)s * n + c];
    if (row < 64) { v0 = xv.x; v1 = -xv.y; }
    else { v0 = xv.y; v1 = xv.x; }
  }
  const size_t o = (size_t)row * 2 * n + 2 * c;
  const float h0 = tf32_hi(v0), h1 = tf32_hi(v1);
  bhi[o] = h0; bhi[o + 1] = h1;
  blo[o] = v0 - h0; blo[o + 1] = v1 - h1;
}

// Y[s][r] = (sum_k P[k][r][s], sum_k P[k][r][64+s]) in FP32.
__global__ void k_tc_reduce(const float* __restrict__ partial, int n, int nrhs, int nsplit, float2* __restrict__ y,
                            const int* gate) {
  if (gate && *gate == 0) return;
  const int s = threadIdx.x & 63;
  const int r = blockIdx.x * (blockDim.x >> 6) + (threadIdx.x >> 6);
  if (r >= n || s >= nrhs) return;
  float re = 0.f, im = 0.f;
  for (int k = 0; k < nsplit; ++k) {
    const float* p = partial + ((size_t)k * n + r) * kN;
    re += p[s];
    im += p[64 + s];
  }
  y[(size_t)s * n + r] = make_float2(re, im);
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

// rows x (2n) FP32, box 32 x 128, 128-byte swizzle, zero fill out of bounds
bool make_map(CUtensorMap* m, const void* base, int n2real, int rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n2real, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)n2real * 4};
  cuuint32_t box[2] = {(cuuint32_t)kKs, (cuuint32_t)kM};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int choose_split(int n) {
  const int tiles = (n + kM - 1) / kM;
  int s = num_sms() / tiles;
  const int ksteps = (2 * n + kKs - 1) / kKs;
  if (s < 1) s = 1;
  if (s > ksteps / kSeg) s = ksteps / kSeg > 0 ? ksteps / kSeg : 1;
  return s;
}

}  // namespace

bool matvec_tc_supported(int n, int nrhs) {
  return nrhs >= 2 && nrhs <= kMaxRhs && n >= kM && (n % 2) == 0 && encode_fn() != nullptr;
}

size_t matvec_tc_workspace_bytes(int n, int nrhs) {
  if (nrhs < 2 || nrhs > kMaxRhs || n < kM) return 0;
  const size_t b = (size_t)kN * 2 * n * 4;                              // one of B_hi / B_lo
  const size_t part = (size_t)choose_split(n) * n * kN * 4;            // split partials
  return 2 * b + part + 256 + 64;                                      // + error word
}

int* matvec_tc_error_word(void* ws, int n, int nrhs) {
  if (nrhs < 2 || nrhs > kMaxRhs || n < kM) return nullptr;
  char* w = static_cast<char*>(ws);
  return reinterpret_cast<int*>(w + 2 * (size_t)kN * 2 * n * 4 + (size_t)choose_split(n) * n * kN * 4);
}

cudaError_t matvec_tc_clear_error(void* ws, int n, int nrhs, cudaStream_t s) {
  int* err = matvec_tc_error_word(ws, n, nrhs);
  if (!err) return cudaErrorInvalidValue;
  return cudaMemsetAsync(err, 0, sizeof(int), s);
}

cudaError_t launch_matvec_tc(const float2* A, size_t lda, int n, int nrhs, const float2* x, float2* y, void* ws,
                             size_t ws_bytes, cudaStream_t s, const int* gate) {
  if (!matvec_tc_supported(n, nrhs) || lda != (size_t)n) return cudaErrorNotSupported;
  if (ws_bytes < matvec_tc_workspace_bytes(n, nrhs)) return cudaErrorInvalidValue;
  const int n2 = 2 * n;
  char* w = static_cast<char*>(ws);
  float* bhi = reinterpret_cast<float*>(w);
  float* blo = reinterpret_cast<float*>(w + (size_t)kN * n2 * 4);
  float* part = reinterpret_cast<float*>(w + 2 * (size_t)kN * n2 * 4);
  const int nsplit = choose_split(n);
  int* err = matvec_tc_error_word(ws, n, nrhs);
  CUtensorMap mA, mBh, mBl;
  if (!make_map(&mA, A, n2, n) || !make_map(&mBh, bhi, n2, kN) || !make_map(&mBl, blo, n2, kN))
    return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_tc_prep_b<<<dim3((n + 255) / 256, kN), 256, 0, s>>>(x, n, nrhs, bhi, blo, gate);
  const int tiles = (n + kM - 1) / kM;
  const int ksteps = (n2 + kKs - 1) / kKs;
  k_gemm_tc<<<dim3(tiles, nsplit), kThreads, kSmemBytes, s>>>(mA, mBh, mBl, n, ksteps, nsplit, part, err, gate);
  k_tc_reduce<<<(n + 3) / 4, 256, 0, s>>>(part, n, nrhs, nsplit, y, gate);
  return cudaGetLastError();
}


}  // namespace bem
