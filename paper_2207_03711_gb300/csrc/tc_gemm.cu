// Real GEMM on the fifth-generation tensor cores of sm_103a (tcgen05 + TMEM + TMA)
// with compensated TF32 splits, the contraction primitive of the environment sweeps.
//
// C (M x N, FP32) = A (M x K) . B (N x K)^T, both FP32 operands K-major (row-major with K
// contiguous). Inside the kernel every loaded tile is split into hi = tf32(x) and
// lo = tf32(x - hi), and the product is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi,
// which recovers the bits a single TF32 product drops (relative error ~2^-21 instead of
// ~2^-11). Splitting after the load keeps the traffic from L2 at one FP32 plane per
// operand.
//
// The tensor core's FP32 accumulation rounds toward zero: measured on a GB300 with
// positive operands, the mean relative error grows linearly with K (-5e-6 at K = 512,
// -9e-5 at K = 8192) where a cuBLAS SGEMM stays unbiased. Chained through the dozens of
// levels of an environment sweep that bias, not the split, set the error. So each
// 32-wide K tile is accumulated in TMEM from zero (12 MMAs), and the epilogue warps add
// the finished tile to a running sum kept in registers with ordinary round-to-nearest
// FP32 additions; two TMEM buffers alternate so that the MMAs of tile k+1 run while the
// epilogue reads tile k.
//
// A persistent grid (at most one CTA per SM) walks the 128 x 128 tiles of C; each CTA
// runs 448 threads:
//   warp 0, lane 0  TMA producer: K-major 128-byte-swizzled 128 x 32 FP32 tiles of A and
//                   B per stage, three stages
//   warp 1          allocates 256 TMEM columns (two 128-column accumulators); lane 0
//                   issues tcgen05.mma (M 128, N 128, K 8) three times per K step,
//                   frees each stage back to the producer and hands each finished
//                   K tile to the epilogue through mbarriers
//   warps 2..9      epilogue: tcgen05.ld of the tile (warp w reads TMEM lanes
//                   32 (w mod 4) .. and half of the 128 columns), FP32 running sums in
//                   registers, bounds-checked stores of C
//   warps 10..13    split each loaded stage in shared memory: hi over the loaded tile,
//                   lo beside it (same swizzled offsets), then a proxy fence so the
//                   tensor core sees the stores
// The pipeline counters run on across a CTA's tiles, so the loads and MMAs of the next
// tile overlap the epilogue of the previous one. Every mbarrier wait is bounded: a wait
// that runs out records an error code in *err, and the kernel still passes its final
// barrier, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <algorithm>

#include "kernels.cuh"
#include "tc_gemm.cuh"

namespace mpsvqe {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 32;            // BK fp32 = 128 bytes = one swizzle row
constexpr int STAGES = 3;
constexpr int TILE_A = BM * BK * 4;                   // 16 KB
constexpr int TILE_B = BN * BK * 4;                   // 16 KB
constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;  // hi and lo of both operands: 64 KB
constexpr int NBARS = 3 * STAGES + 4;                 // full, split, empty per stage; ready, free per buffer
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 8 * NBARS + 16;
constexpr int NTHREADS = 448;
constexpr int NEPI = 256;                             // epilogue threads (warps 2..9)
constexpr int EPI_COLS = BN / 2;                      // columns per epilogue thread
constexpr int CONV_WARP0 = 10;                        // split threads (warps 10..13)
constexpr int NCONV = 128;
constexpr int TMEM_COLS = 2 * BN;                     // two accumulators
constexpr long long kWaitCycles = 4000000000LL;       // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on the phase with the given parity; false (and *err set) on time-out.
// backoff: the many-thread waiters (split and epilogue warps) sleep briefly between
// polls, so that their polling does not take shared-memory bandwidth from the split and
// the TMA writes; the single-thread producer and MMA issuer poll without sleeping.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code,
                                          bool backoff = false) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(err, code);
      return false;
    }
    if (backoff) __nanosleep(64);
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile stored as rows of 128 bytes with the
// 128-byte swizzle (the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_128B): 8-row core
// groups 1024 bytes apart (stride byte offset); the leading byte offset is not used by
// this layout; version 1 (tcgen05); layout type 2 = SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
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

__device__ __forceinline__ float tf32_rna(float v) {
  uint32_t b;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(v));
  return __uint_as_float(b);
}

__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm_tf32x3(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float* C,
                  int64_t ldc, int M, int N, int K, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // barriers: full[s] (TMA), split[s] (hi/lo written), empty[s] (MMAs done), ready[b], freed[b]
  uint64_t* bars = (uint64_t*)(base + STAGES * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* split = bars + STAGES;
  uint64_t* empty = bars + 2 * STAGES;
  uint64_t* ready = bars + 3 * STAGES;
  uint64_t* freed = bars + 3 * STAGES + 2;
  uint32_t* tmem_slot = (uint32_t*)(bars + NBARS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = (K + BK - 1) / BK;
  const int tiles_n = (N + BN - 1) / BN, tiles = tiles_n * ((M + BM - 1) / BM);
  // persistent: this CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...; the
  // pipeline counters (stage and accumulator phases) run on across its tiles
  const int my_tiles = blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int total = my_tiles * nk;

  if (tid == 0) {
    for (int s = 0; s < 3 * STAGES + 2; ++s) mbar_init(smem_u32(&bars[s]), 1);
    for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&freed[b]), NEPI);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: the FP32 tiles of A and B, into the hi slots of the stage
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    int g = 0;
    bool ok = true;
    for (int n = 0; n < my_tiles && ok; ++n) {
      const int tile = blockIdx.x + n * gridDim.x;
      const int m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
      for (int kt = 0; kt < nk; ++kt, ++g) {
        const int s = g % STAGES;
        if (g >= STAGES && !mbar_wait(smem_u32(&empty[s]), ((g / STAGES) & 1) ^ 1, err, 1)) {
          ok = false;
          break;
        }
        unsigned char* st = base + s * STAGE_BYTES;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_arrive_expect_tx(fb, TILE_A + TILE_B);
        tma_load_2d(smem_u32(st), &tmA, kt * BK, m0, fb);
        tma_load_2d(smem_u32(st + 2 * TILE_A), &tmB, kt * BK, n0, fb);
      }
    }
    // no copy may still be landing in shared memory when the CTA exits: wait (bounded)
    // for the last load of each stage (already complete unless a consumer gave up)
    for (int gl = g - 1; gl >= 0 && gl >= g - STAGES; --gl)
      mbar_wait(smem_u32(&full[gl % STAGES]), (gl / STAGES) & 1, err, 6);
  } else if (warp >= CONV_WARP0) {
    // ---- split: hi = tf32(x) over the loaded tile, lo = tf32(x - hi) beside it
    const int ct = tid - CONV_WARP0 * 32;
    for (int g = 0; g < total; ++g) {
      const int s = g % STAGES;
      const bool got = mbar_wait(smem_u32(&full[s]), (g / STAGES) & 1, err, 5, true);
      // all split threads leave together if any wait ran out (none is left at a barrier)
      uint32_t all_ok;
      asm volatile(
          "{\n"
          " .reg .pred p, q;\n"
          " setp.ne.u32 p, %1, 0;\n"
          " bar.red.and.pred q, 1, %2, p;\n"
          " selp.u32 %0, 1, 0, q;\n"
          "}\n"
          : "=r"(all_ok)
          : "r"((uint32_t)got), "n"(NCONV)
          : "memory");
      if (!all_ok) break;
      unsigned char* st = base + s * STAGE_BYTES;
      float4* ah = (float4*)st;
      float4* al = (float4*)(st + TILE_A);
      float4* bh = (float4*)(st + 2 * TILE_A);
      float4* bl = (float4*)(st + 2 * TILE_A + TILE_B);
#pragma unroll 4
      for (int v = ct; v < TILE_A / 16; v += NCONV) {
        const float4 x = ah[v];
        float4 h, l;
        h.x = tf32_rna(x.x); l.x = tf32_rna(x.x - h.x);
        h.y = tf32_rna(x.y); l.y = tf32_rna(x.y - h.y);
        h.z = tf32_rna(x.z); l.z = tf32_rna(x.z - h.z);
        h.w = tf32_rna(x.w); l.w = tf32_rna(x.w - h.w);
        ah[v] = h;
        al[v] = l;
      }
#pragma unroll 4
      for (int v = ct; v < TILE_B / 16; v += NCONV) {
        const float4 x = bh[v];
        float4 h, l;
        h.x = tf32_rna(x.x); l.x = tf32_rna(x.x - h.x);
        h.y = tf32_rna(x.y); l.y = tf32_rna(x.y - h.y);
        h.z = tf32_rna(x.z); l.z = tf32_rna(x.z - h.z);
        h.w = tf32_rna(x.w); l.w = tf32_rna(x.w - h.w);
        bh[v] = h;
        bl[v] = l;
      }
      // the generic-proxy stores must be visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 2, %0;" ::"n"(NCONV) : "memory");
      if (ct == 0) mbar_arrive(smem_u32(&split[s]));
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: K tile g goes to accumulator g & 1, from zero
    constexpr uint32_t idesc = idesc_tf32(BM, BN);
    for (int g = 0; g < total; ++g) {
      const int s = g % STAGES, b = g & 1;
      if (!mbar_wait(smem_u32(&split[s]), (g / STAGES) & 1, err, 2)) break;
      if (g >= 2 && !mbar_wait(smem_u32(&freed[b]), ((g >> 1) & 1) ^ 1, err, 4)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = smem_u32(base + s * STAGE_BYTES);
      const uint32_t acc = tmem + (uint32_t)(b * BN);
#pragma unroll
      for (int ks = 0; ks < BK / 8; ++ks) {
        // K step of 8 TF32 = 32 bytes inside each 128-byte swizzled row
        const uint64_t ah = sw128_kmajor_desc(st + ks * 32);
        const uint64_t al = sw128_kmajor_desc(st + TILE_A + ks * 32);
        const uint64_t bh = sw128_kmajor_desc(st + 2 * TILE_A + ks * 32);
        const uint64_t bl = sw128_kmajor_desc(st + 2 * TILE_A + TILE_B + ks * 32);
        mma_tf32(acc, ah, bh, idesc, ks > 0 ? 1u : 0u);
        mma_tf32(acc, ah, bl, idesc, 1u);
        mma_tf32(acc, al, bh, idesc, 1u);
      }
      mma_commit(smem_u32(&empty[s]));   // stage s free once these finish
      mma_commit(smem_u32(&ready[b]));   // K tile g complete in accumulator b
    }
  } else if (warp >= 2) {
    // ---- epilogue: round-to-nearest FP32 sums of the K tiles; warp w reads TMEM lanes
    // 32 (w mod 4) .. (its rows) and one half of the columns
    const int q = warp & 3, c_lo = ((warp - 2) >> 2) * EPI_COLS;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const bool vec = ((ldc & 3) == 0) && (((uintptr_t)C & 15) == 0);
    bool ok = true;
    int g = 0;
    for (int n = 0; n < my_tiles && ok; ++n) {
      const int tile = blockIdx.x + n * gridDim.x;
      const int m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN + c_lo;
      float sum[EPI_COLS];
#pragma unroll
      for (int c = 0; c < EPI_COLS; ++c) sum[c] = 0.f;
      for (int kt = 0; kt < nk && ok; ++kt, ++g) {
        const int b = g & 1;
        // tcgen05.ld is warp-collective: the whole warp goes on or stops together
        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ready[b]), (g >> 1) & 1, err, 3, true));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) {
#pragma unroll
          for (int c0 = 0; c0 < EPI_COLS; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + lane_off + (uint32_t)(b * BN + c_lo + c0), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) sum[c0 + j] = __fadd_rn(sum[c0 + j], v[j]);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&freed[b]));
      }
      const int row = m0 + q * 32 + lane;
      if (ok && row < M) {
        float* out = C + (size_t)row * ldc + n0;
        if (vec && n0 + EPI_COLS <= N) {
#pragma unroll
          for (int c = 0; c < EPI_COLS; c += 4)
            *reinterpret_cast<float4*>(out + c) = make_float4(sum[c], sum[c + 1], sum[c + 2], sum[c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < EPI_COLS; ++c)
            if (n0 + c < N) out[c] = sum[c];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Copy of an M x K row-major plane (leading dimension ld_in) into one of leading
// dimension ld_out (a multiple of 4 floats, so TMA rows start on 16-byte boundaries);
// columns K..ld_out-1 are written as zero.
__global__ void k_pad_rows(const float* x, int64_t ld_in, int M, int K, float* out, int64_t ld_out) {
  const int64_t total = (int64_t)M * ld_out;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld_out, c = i - r * ld_out;
    out[i] = c < K ? x[r * ld_in + c] : 0.f;
  }
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_status = cudaSuccess;
}  // namespace

static cudaError_t get_encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    g_encode_status = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (g_encode_status == cudaSuccess && (q != cudaDriverEntryPointSuccess || !fn))
      g_encode_status = cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  return g_encode_status;
}

// 2-D FP32 tensor map of a rows x K plane with leading dimension ld (floats): boxes of
// 32 x box_rows, 128-byte swizzle, out-of-range elements read as zero.
static cudaError_t make_map(CUtensorMap* map, const float* p, int rows, int K, int64_t ld, int box_rows) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_pad_rows(const float* x, int64_t ld_in, int M, int K, float* out, int64_t ld_out,
                            cudaStream_t st) {
  if (M <= 0 || ld_out <= 0) return cudaSuccess;
  const int64_t total = (int64_t)M * ld_out;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_pad_rows<<<blocks, 256, 0, st>>>(x, ld_in, M, K, out, ld_out);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tf32x3(const Plane& A, const Plane& B, int M, int N, int K, float* C, int64_t ldc, int* err,
                               cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if ((A.ld & 3) || (B.ld & 3) || ((uintptr_t)A.p & 15) || ((uintptr_t)B.p & 15)) return cudaErrorInvalidValue;
  CUtensorMap am, bm;
  cudaError_t e;
  if ((e = make_map(&am, A.p, M, K, A.ld, BM)) != cudaSuccess) return e;
  if ((e = make_map(&bm, B.p, N, K, B.ld, BN)) != cudaSuccess) return e;
  static std::once_flag once[64];
  static cudaError_t attr[64];
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::call_once(once[dev], [dev] {
    attr[dev] = cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  if (attr[dev] != cudaSuccess) return attr[dev];
  // persistent grid: one CTA per SM at most (197 KB of shared memory each)
  static int sm_count[64] = {0};
  if (!sm_count[dev] && (e = cudaDeviceGetAttribute(&sm_count[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int64_t tiles = (int64_t)((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  const int grid = (int)std::min<int64_t>(tiles, sm_count[dev]);
  k_gemm_tf32x3<<<grid, NTHREADS, SMEM_BYTES, st>>>(am, bm, C, ldc, M, N, K, err);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace mpsvqe

// ------------------------------------------------------------------ C ABI
#include "../../include/mpsvqe.h"

extern "C" int mps_tc_gemm_tf32x3(int M, int N, int K, const float* A, int64_t lda, const float* B, int64_t ldb,
                                  float* C, int64_t ldc, void* cuda_stream) {
  using namespace mpsvqe;
  if (M < 0 || N < 0 || K < 1 || !A || !B || !C || lda < K || ldb < K || ldc < N) {
    set_error_message("mps_tc_gemm_tf32x3: needs M, N >= 0, K >= 1, lda, ldb >= K, ldc >= N and non-null pointers");
    return MPS_EINVAL;
  }
  if (M == 0 || N == 0) return MPS_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // TMA wants 16-byte-aligned rows: operands that are not get a padded copy
  const bool pad_a = (lda & 3) || ((uintptr_t)A & 15), pad_b = (ldb & 3) || ((uintptr_t)B & 15);
  const int64_t ldk = ((int64_t)K + 3) & ~(int64_t)3;
  float* buf = nullptr;
  int* err = nullptr;
  const size_t na = pad_a ? (size_t)M * ldk : 0, nb = pad_b ? (size_t)N * ldk : 0;
  if (cudaMallocAsync((void**)&buf, (na + nb + 4) * sizeof(float), st) != cudaSuccess ||
      cudaMallocAsync((void**)&err, sizeof(int), st) != cudaSuccess) {
    set_error_message("mps_tc_gemm_tf32x3: cudaMallocAsync of the work buffers failed");
    return MPS_ENOMEM;
  }
  int rc = MPS_OK;
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess && pad_a) e = tc::launch_pad_rows(A, lda, M, K, buf, ldk, st);
  if (e == cudaSuccess && pad_b) e = tc::launch_pad_rows(B, ldb, N, K, buf + na, ldk, st);
  if (e == cudaSuccess)
    e = tc::launch_gemm_tf32x3(pad_a ? tc::Plane{buf, ldk} : tc::Plane{A, lda},
                               pad_b ? tc::Plane{buf + na, ldk} : tc::Plane{B, ldb}, M, N, K, C, ldc, err, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(buf, st);
  cudaFreeAsync(err, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error_message((std::string("mps_tc_gemm_tf32x3: ") + cudaGetErrorString(e)).c_str());
    rc = MPS_ECUDA;
  } else if (herr) {
    set_error_message("mps_tc_gemm_tf32x3: a bounded tensor-core pipeline wait ran out");
    rc = MPS_ETIMEOUT;
  }
  return rc;
}
