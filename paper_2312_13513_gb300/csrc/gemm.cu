// BF16 GEMM on the 5th-generation tensor cores (tcgen05) for sm_103a:
//   C[M x N] (FP32) = A[M x K] * B[N x K]^T (+ bias[N]),  A and B BF16 with K contiguous,
// or, with the activation epilogue, C[M x N] (BF16) = bf16(GELU(A B^T + bias)) (the erf form of
// GELU to 5e-7, gelu.cuh; round to nearest even): the layer-by-layer inference of the per-species
// networks.
//
// A training forward layer can take both outputs at once: the FP32 pre-activation and the BF16
// GELU of it (gemm_bf16_gelu2).
//
// Used by the surrogate's training (forward and backward products of §2's MLP, trained with
// Adam) and by the per-species networks' inference; the single network's inference uses the
// fused kernel in surrogate.cu built from the same primitives.  One persistent kernel
// (gemm_bf16_persistent): warp 0 (one lane) streams 128 x 64 tiles of A and B with TMA (128-byte
// swizzle) through an mbarrier ring, warp 1 (one lane) issues tcgen05.mma.cta_group::1.kind::f16
// (M = 128, N = BN, K = 16) into one of two TMEM accumulators, and sixteen warps read the other
// accumulator back with tcgen05.ld for the epilogue.  Every wait is bounded: a timeout sets a
// device error flag and the kernel drains and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "chem_internal.h"
#include "gelu.cuh"
#include "sm100.h"

namespace chem {

using namespace sm100;

// ---------------------------------------------------------------------------------------
// tensor maps (driver entry point fetched through the runtime; no link-time libcuda)
// ---------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// 2D BF16 row-major matrix [rows x cols] (cols contiguous, row pitch ld elements); box
// box_cols x box_rows with 128-byte swizzle (box_cols * 2 must be 128).
int make_tmap_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                   int box_rows, int box_cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) { set_error("cuTensorMapEncodeTiled unavailable"); return CHEM_ECUDA; }
  if (((uintptr_t)base & 15) || (ld * 2) % 16) {
    set_error("TMA operand must be 16-byte aligned with a 16-byte multiple row pitch");
    return CHEM_EINVAL;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return CHEM_ECUDA; }
  return CHEM_OK;
}

namespace {

constexpr int BM = 128, BN = 128, BK = 64;      // tile rows, the narrower tile width, K step

struct GemmArgs {
  float* C;
  __nv_bfloat16* Cb;       // non-null: BF16 output of the activation epilogue instead of C
  float* Cz;               // with Cb (persistent kernel): also the FP32 pre-activation, same pitch
  int gelu;                // activation epilogue: apply GELU before rounding
  int vec;                 // output base and row pitch allow 16-byte stores
  const float* bias;
  int M, N, K;
  int64_t ldc;
  int* err;
  // split-K (FP32 output C only, no bias): the K steps of every output tile are dealt to `splits`
  // tiles of the queue, split s writing its partial sum to C + s * split_stride
  int splits = 1;
  int64_t split_stride = 0;
};


// ---------------------------------------------------------------------------------------
// Persistent form: one CTA per SM walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... (N-fastest
// within a row block, so consecutive tiles share their A rows in L2) with a 128 x BN_ tile and
// two TMEM accumulators: the epilogue of one tile runs while the MMAs of the next fill the other
// accumulator.  Warp 0 (one lane): TMA producer over a STAGES_P-stage ring; warp 1 (one lane):
// MMA issuer; warps 2-17: epilogue (warp w reads TMEM lanes 32 (w % 4) .. + 31 and the columns of
// quarter (w - 2) / 4 of the tile: four warps per scheduler hide the latency of the bias, GELU and
// store chain), storing each row's 32-column pieces straight to global memory.
// ---------------------------------------------------------------------------------------
constexpr int kPersistThreads = 576;     // TMA warp, MMA warp, sixteen epilogue warps

template <int BN_>
struct PersistCfg {
  static constexpr int STAGES_P = BN_ == 256 ? 4 : 6;
  static constexpr int TA = BM * BK * 2;                   // 16 KB
  static constexpr int TB = BN_ * BK * 2;                  // 16 or 32 KB
  static constexpr int SMEM = STAGES_P * (TA + TB) + 1024 + 256;
};

// SPLITK_: the split-K decode is compiled in (training's weight gradients); without it every tile
// takes all K steps, as the inference products do
template <int BN_, bool SPLITK_>
__global__ void __launch_bounds__(kPersistThreads, 1)
    gemm_bf16_persistent(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         const GemmArgs a) {
  using Cfg = PersistCfg<BN_>;
  constexpr int NS = Cfg::STAGES_P;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + NS * Cfg::TA;
  uint64_t* full = (uint64_t*)(sB + NS * Cfg::TB);
  uint64_t* empty = full + NS;
  uint64_t* acc_full = empty + NS;        // [2]: the MMAs of a tile into accumulator b are done
  uint64_t* acc_empty = acc_full + 2;     // [2]: the epilogue has read accumulator b
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntm = (a.M + BM - 1) / BM, ntn = (a.N + BN_ - 1) / BN_;
  const int splits = SPLITK_ ? a.splits : 1;
  const long long ntiles = (long long)ntm * ntn * splits;
  // K steps of one split (the host makes splits divide the step count)
  const int nk = (a.K + BK - 1) / BK / splits;
  // queue entry t: output tile t / splits (N-fastest within a row block), split t % splits
  auto decode = [&](long long t, int& m0, int& n0, int& kb0, int& split) {
    const long long mn = SPLITK_ ? t / splits : t;
    split = SPLITK_ ? (int)(t % splits) : 0;
    m0 = (int)(mn / ntn) * BM;
    n0 = (int)(mn % ntn) * BN_;
    kb0 = split * nk;
  };
  const long long rounds = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], kPersistThreads - 64); }
    fence_barrier_init();
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  if (warp == 0) tmem_alloc(tmem_slot, 2 * BN_);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer
      long long it = 0;
      bool ok = true;
      for (long long rd = 0; rd < rounds && ok; ++rd) {
        int m0, n0, kb0, split;
        decode(blockIdx.x + rd * gridDim.x, m0, n0, kb0, split);
        for (int kb = kb0; kb < kb0 + nk; ++kb, ++it) {
          const int s = (int)(it % NS);
          if (!mbar_wait(&empty[s], (uint32_t)((it / NS) & 1) ^ 1u, a.err)) { ok = false; break; }
          mbar_arrive_expect_tx(&full[s], Cfg::TA + Cfg::TB);
          tma_load_2d(sA + s * Cfg::TA, &tmA, &full[s], kb * BK, m0);
          tma_load_2d(sB + s * Cfg::TB, &tmB, &full[s], kb * BK, n0);
        }
      }
      // drain: every issued stage has been consumed by the MMAs
      const long long first = it > NS ? it - NS : 0;
      for (long long k = first; k < it; ++k) mbar_wait(&empty[k % NS], (uint32_t)((k / NS) & 1), a.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = idesc_bf16_f32(BM, BN_);
      long long it = 0;
      bool ok = true;
      for (long long rd = 0; rd < rounds && ok; ++rd) {
        const int b = (int)(rd & 1);
        // the epilogue has drained this accumulator (its use two tiles ago)
        if (rd >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)(((rd - 2) >> 1) & 1), a.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * BN_);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int s = (int)(it % NS);
          if (!mbar_wait(&full[s], (uint32_t)((it / NS) & 1), a.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t abase = smem_addr(sA + s * Cfg::TA), bbase = smem_addr(sB + s * Cfg::TB);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_bf16(d, sdesc_k128(abase + kk * 32), sdesc_k128(bbase + kk * 32), idesc,
                     (kb > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full[b]);
      }
    }
  } else {
    // epilogue warps 2-17
    const int quarter = warp & 3, part = (warp - 2) >> 2;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    constexpr int HW = BN_ / 4;                              // columns per epilogue warp
    bool ok = true;
    for (long long rd = 0; rd < rounds && ok; ++rd) {
      int m0, n0, kb0, split;
      decode(blockIdx.x + rd * gridDim.x, m0, n0, kb0, split);
      const int b = (int)(rd & 1);
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)((rd >> 1) & 1), a.err))) { ok = false; break; }
      tc_fence_after();
      const int row = m0 + quarter * 32 + lane;
      const bool rv = row < a.M;
      const uint32_t tb = trow + (uint32_t)(b * BN_ + part * HW);
#pragma unroll 1
      for (int cc = 0; cc < HW; cc += 32) {
        uint32_t r[32];
        tmem_ld32(tb + cc, r);
        tmem_ld_wait(r);
        const int col = n0 + part * HW + cc;
        if (a.Cb) {
          if (a.Cz) {
            // the pre-activation z = acc + bias, kept in r for the activation below
#pragma unroll
            for (int j = 0; j < 32; ++j)
              r[j] = __float_as_uint(__uint_as_float(r[j]) + (a.bias && col + j < a.N ? a.bias[col + j] : 0.0f));
            if (rv) {
              float* outz = a.Cz + (int64_t)row * a.ldc + col;
              if (a.vec && col + 32 <= a.N) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                  reinterpret_cast<float4*>(outz)[q] =
                      make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                  __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
              } else {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                  if (col + j < a.N) outz[j] = __uint_as_float(r[j]);
              }
            }
          }
          const bool add_bias = a.bias && !a.Cz;
          uint32_t pk[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int cj = col + 2 * j;
            float v0 = __uint_as_float(r[2 * j]) + (add_bias && cj < a.N ? a.bias[cj] : 0.0f);
            float v1 = __uint_as_float(r[2 * j + 1]) + (add_bias && cj + 1 < a.N ? a.bias[cj + 1] : 0.0f);
            if (a.gelu) gelu2(v0, v1);
            __nv_bfloat162 hv = __floats2bfloat162_rn(v0, v1);
            pk[j] = *reinterpret_cast<uint32_t*>(&hv);
          }
          if (rv) {
            __nv_bfloat16* out = a.Cb + (int64_t)row * a.ldc + col;
            if (a.vec && col + 32 <= a.N) {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                reinterpret_cast<uint4*>(out)[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                if (col + j < a.N) {
                  const uint32_t w = pk[j >> 1];
                  reinterpret_cast<uint16_t*>(out)[j] = (uint16_t)((j & 1) ? (w >> 16) : (w & 0xffffu));
                }
              }
            }
          }
        } else if (rv) {
          float* out = a.C + (SPLITK_ ? split * a.split_stride : 0) + (int64_t)row * a.ldc + col;
          float v[32];
#pragma unroll
          for (int j = 0; j < 32; ++j)
            v[j] = __uint_as_float(r[j]) + (a.bias && col + j < a.N ? a.bias[col + j] : 0.0f);
          if (a.vec && col + 32 <= a.N) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              reinterpret_cast<float4*>(out)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (col + j < a.N) out[j] = v[j];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * BN_);
}

}  // namespace

template <int BN_, bool SPLITK_>
static int launch_persistent(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, unsigned grid,
                             cudaStream_t stream) {
  static bool attr = false;
  if (!attr) {
    CHEM_CUDA_TRY(cudaFuncSetAttribute(gemm_bf16_persistent<BN_, SPLITK_>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, PersistCfg<BN_>::SMEM));
    attr = true;
  }
  gemm_bf16_persistent<BN_, SPLITK_><<<grid, kPersistThreads, PersistCfg<BN_>::SMEM, stream>>>(ta, tb, g);
  return CHEM_OK;
}

static int gemm_launch(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, void* Cb, int gelu,
                       int64_t ldc, const float* bias, int M, int N, int K, int* err, cudaStream_t stream,
                       float* Cz = nullptr, int splits = 1, int64_t split_stride = 0) {
  if (M < BM || N < BN || K <= 0 || !A || !B || (!C && !Cb) || !err) {
    set_error("gemm_bf16: bad arguments (M=%d N=%d K=%d; M and N must be >= 128)", M, N, K);
    return CHEM_EINVAL;
  }
  CUtensorMap ta, tb;
  int rc = make_tmap_bf16(&ta, A, M, K, lda, BM, BK);
  if (rc) return rc;
  rc = make_tmap_bf16(&tb, B, N, K, ldb, BN, BK);
  if (rc) return rc;
  const uintptr_t obase = C ? (uintptr_t)C : (uintptr_t)Cb;
  const int64_t opitch = ldc * (C ? 4 : 2);
  int vec = (obase % 16 == 0 && opitch % 16 == 0) ? 1 : 0;
  if (Cz && ((uintptr_t)Cz % 16 != 0 || (ldc * 4) % 16 != 0)) vec = 0;
  GemmArgs g{C, (__nv_bfloat16*)Cb, Cz, gelu, vec, bias, M, N, K, ldc, err};
  g.splits = splits;
  g.split_stride = split_stride;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    CHEM_CUDA_TRY(cudaGetDevice(&dev));
    CHEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  // persistent kernel, 256-column tiles unless 128-column tiles pad N less, or unless 256-column
  // tiles would leave SMs without a tile (small products: more, smaller tiles finish sooner)
  const int pad128 = (N + 127) / 128 * 128 - N, pad256 = (N + 255) / 256 * 256 - N;
  int bn = (N >= 256 && pad256 <= pad128) ? 256 : 128;
  if (bn == 256 && (long long)((M + BM - 1) / BM) * ((N + 255) / 256) * splits < sms) bn = 128;
  const long long ntiles = (long long)((M + BM - 1) / BM) * ((N + bn - 1) / bn) * splits;
  const unsigned grid = (unsigned)std::min<long long>(ntiles, sms);
  if (bn == 256) {
    CUtensorMap tb2;
    rc = make_tmap_bf16(&tb2, B, N, K, ldb, 256, BK);
    if (rc) return rc;
    rc = splits > 1 ? launch_persistent<256, true>(ta, tb2, g, grid, stream)
                    : launch_persistent<256, false>(ta, tb2, g, grid, stream);
  } else {
    rc = splits > 1 ? launch_persistent<128, true>(ta, tb, g, grid, stream)
                    : launch_persistent<128, false>(ta, tb, g, grid, stream);
  }
  if (rc) return rc;
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

int gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
              const float* bias, int M, int N, int K, int* err, cudaStream_t stream) {
  return gemm_launch(A, lda, B, ldb, C, nullptr, 0, ldc, bias, M, N, K, err, stream);
}

// Split-K product for short, deep shapes (training's weight gradients: a few output tiles, K =
// the batch): split s of `splits` multiplies over K steps [s, s + 1) * K / splits and writes its
// FP32 partial [M x N] (pitch ldc) to Cparts + s * split_stride; the caller adds the partials.
// The number of 64-wide K steps must be a multiple of splits.
int gemm_bf16_splitk(const void* A, int64_t lda, const void* B, int64_t ldb, float* Cparts, int64_t ldc,
                     int64_t split_stride, int splits, int M, int N, int K, int* err, cudaStream_t stream) {
  if (splits < 1 || ((K + BK - 1) / BK) % splits != 0 || split_stride < (int64_t)M * ldc) {
    set_error("gemm_bf16_splitk: splits must divide the K steps (%d) and the stride hold M x ldc", (K + BK - 1) / BK);
    return CHEM_EINVAL;
  }
  return gemm_launch(A, lda, B, ldb, Cparts, nullptr, 0, ldc, nullptr, M, N, K, err, stream, nullptr, splits,
                     split_stride);
}

int gemm_bf16_act(const void* A, int64_t lda, const void* B, int64_t ldb, void* Cb, int64_t ldc,
                  const float* bias, int gelu, int M, int N, int K, int* err, cudaStream_t stream) {
  return gemm_launch(A, lda, B, ldb, nullptr, Cb, gelu, ldc, bias, M, N, K, err, stream);
}

// C = A B^T + bias twice: the FP32 pre-activation into Cz and GELU of it, rounded to BF16, into Cb
// (both [M x N] with row pitch ldc elements): a training forward layer in one launch
int gemm_bf16_gelu2(const void* A, int64_t lda, const void* B, int64_t ldb, float* Cz, void* Cb, int64_t ldc,
                    const float* bias, int M, int N, int K, int* err, cudaStream_t stream) {
  if (!Cz || !Cb) { set_error("gemm_bf16_gelu2: both outputs are required"); return CHEM_EINVAL; }
  return gemm_launch(A, lda, B, ldb, nullptr, Cb, 1, ldc, bias, M, N, K, err, stream, Cz);
}

}  // namespace chem

using namespace chem;

extern "C" int chem_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C,
                              int64_t ldc, const float* bias, int M, int N, int K, int* err,
                              chem_stream_t stream) {
  return gemm_bf16(A, lda, B, ldb, C, ldc, bias, M, N, K, err, (cudaStream_t)stream);
}

extern "C" int chem_gemm_bf16_act(const void* A, int64_t lda, const void* B, int64_t ldb, void* Cb,
                                  int64_t ldc, const float* bias, int gelu, int M, int N, int K, int* err,
                                  chem_stream_t stream) {
  return gemm_bf16_act(A, lda, B, ldb, Cb, ldc, bias, gelu, M, N, K, err, (cudaStream_t)stream);
}
