// BF16 MLP surrogate of the chemistry step (the paper's DNN chemistry, §2 / §3.1) on sm_103a.
//
// Network: x = z-scored [T, ln p, BC(Y_1..Y_ns)] (BC = Box-Cox, lambda = 0.1) -> 512 -> 512 ->
// 512 -> 512 -> ns, GELU (exact erf form) after each hidden layer, BF16 weights and activations,
// FP32 accumulation.  Outputs are z-scored increments of BC(Y) over the training step dt.
// The first layer is compensated: its input and weights are each split into a BF16 pair,
// x = x_hi + x_lo and W = W_hi + W_lo, and one K = 64 product over the input row
// [x_hi | x_lo | x_hi] with the weight row [W_hi | W_hi | W_lo] sums W_hi x_hi + W_hi x_lo +
// W_lo x_hi (the W_lo x_lo term is below FP32 accumulation noise).  Reaction rates depend
// exponentially on T, and a plain BF16 T feature (8-bit mantissa) is off by several kelvin.
//
// surrogate_forward_kernel (persistent, one CTA per SM, 18 warps; a layer's 512 outputs are two
// accumulator halves of 256 TMEM columns):
//   warps 0-15 epilogue: after every hidden layer read the FP32 accumulator from TMEM
//              (tcgen05.ld), add the bias, apply GELU, round to BF16 and write the next layer's
//              input tile in place (128-byte swizzled K-major layout).  Warp w reads TMEM lanes
//              32 (w % 4) .. + 31 (its cells) and 128 columns of half w / 8, so four warps per SM
//              sub-partition share a layer's 512 columns.
//              Warps 8-11 also build the next tile's input (FP64 state -> features -> BF16) right
//              after its first layer and, after the last layer, apply the inverse transform
//              (de-normalise, add to BC(Y0), invert Box-Cox) and write Y' (FP32).  The
//              trust-region test (training box) is done on the features.
//   warp 16    one lane streams weight tiles (256 x 64 BF16, 32 KB) with TMA into a 3-stage ring.
//   warp 17    one lane issues tcgen05.mma (M = 128, N = 256 or 16, K = 16) into 512 TMEM columns.
// surrogate_post_kernel (FP64, one thread per cell): element-conservation projection, clip,
//   temperature from enthalpy by Newton (the paper's Thermo class, §3.1), acceptance tests, and
//   compaction of rejected cells into a fallback list that the FP64 integrator then advances
//   (indexed mode, count read from device memory).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <vector>

#include "chem_internal.h"
#include "sm100.h"
#include "gelu.cuh"
#include "surrogate_model.h"
#include "thermo.cuh"

namespace chem {

using namespace sm100;

int make_tmap_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld,
                   int box_rows, int box_cols);

constexpr int TM = 128;            // cells per tile
constexpr int HID = 512;           // hidden width
constexpr int KIN = SUR_KIN;       // padded input width (one 128-byte K chunk)
constexpr int NOUT = 16;           // padded output width
constexpr int MAXNS = SUR_MAXNS;   // outputs supported
static_assert(3 * (MAXNS + 2) <= KIN, "the compensated first layer needs 3 n_in <= KIN");
constexpr int WSTAGES = 3;
constexpr int WSTAGE_BYTES = 256 * 64 * 2;
constexpr int ACT_CHUNK = TM * 128;                  // 16 KB: 128 rows x 64 bf16
constexpr int ACT_BYTES = 8 * ACT_CHUNK;             // 128 KB
constexpr int FWD_SMEM = ACT_BYTES + WSTAGES * WSTAGE_BYTES + 1024 + 256;
constexpr float BC_LAMBDA = SUR_BC_LAMBDA;

// rows of SurParams::st: feature statistics and box, target statistics, output bias
enum { ST_XMU, ST_XSD, ST_LO, ST_HI, ST_YMU, ST_YSD, ST_B5, ST_ROWS };

struct SurParams {
  float hb[4][HID];     // hidden-layer biases by value: read from the parameter (constant) bank
  float st[ST_ROWS][MAXNS + 2];   // statistics, box and output bias, also from the parameter bank
  int ns, nin;
  const double* T;
  const double* p;
  const double* Y;
  int64_t ld, ncells;
  float* ynet;          // [ns][ncells]
  float* zout;          // [ns][ncells] raw network output (nullable)
  uint8_t* outbox;      // [ncells] 1 = features outside the training box
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Bias, GELU and BF16 rounding of 32 accumulator columns (c0 .. c0 + 31) of one row, written as
// half of a 128-byte K chunk of the next layer's input (128-byte swizzled K-major layout).  The
// 32 biases are warp-uniform reads of the kernel's parameter bank.
__device__ __forceinline__ void epilogue_block(const uint32_t (&a)[32], const float* bias, int c0,
                                               unsigned char* arow, int r) {
  unsigned char* chunk = arow + (c0 >> 6) * ACT_CHUNK;
  const int part = (c0 >> 5) & 1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float* bq = bias + c0 + 8 * q;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      // the bias of a pair of columns in one packed add (each half rounds like the scalar add)
      const unsigned long long s2 = add_x2(f32x2(__uint_as_float(a[8 * q + e]), __uint_as_float(a[8 * q + e + 1])),
                                           f32x2(bq[e], bq[e + 1]));
      f32x2_split(s2, v[e], v[e + 1]);
      gelu2(v[e], v[e + 1]);
    }
    uint4 pk;
    pk.x = pack_bf16(v[0], v[1]); pk.y = pack_bf16(v[2], v[3]);
    pk.z = pack_bf16(v[4], v[5]); pk.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(chunk + (((part * 4 + q) ^ (r & 7)) << 4)) = pk;
  }
}

// the per-tile chunk schedule shared by the producer and the MMA issuer
// layer 0: 2 chunks (rows 0-255, 256-511 of W1, K = 64); layers 1-3: 8 K-chunks x 2 halves;
// layer 4: 8 K-chunks of W5 (16 rows)
constexpr int CHUNKS_PER_TILE = 2 + 3 * 16 + 8;

// Epilogue warps: two per TMEM lane quarter and accumulator half, each draining 128 of the
// half's 256 columns (four 32-column blocks)
constexpr int kEpiParts = 2;
constexpr int kEpiWarps = 8 * kEpiParts;
constexpr int kFwdThreads = 32 * (kEpiWarps + 2);
constexpr int kTmaWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;

// Input features of one cell (x = [T, ln p, BC(Y)], z-scored, split into BF16 hi and lo parts:
// [x_hi | x_lo | x_hi | 0], packed two per word), with its Box-Cox values bc (the output transform
// adds the network's increments to them); outside = the features leave the training box.
template <int NS_>
struct CellFeatures {
  static constexpr int AS = NS_ > 0 ? NS_ : MAXNS;
  static constexpr int KP = NS_ > 0 ? (3 * (NS_ + 2) + 1) / 2 : KIN / 2;   // packed words in use
  uint32_t xp[KP];
};

template <int NS_>
__device__ __forceinline__ void cell_features(const SurParams& P, double tv, double pv,
                                              const double (&yv)[CellFeatures<NS_>::AS], CellFeatures<NS_>& F,
                                              float (&bc)[CellFeatures<NS_>::AS], bool& outside) {
  constexpr int AS = CellFeatures<NS_>::AS;
  const int ns = NS_ > 0 ? NS_ : P.ns, nin = ns + 2;
  float x[2 * CellFeatures<NS_>::KP];
#pragma unroll
  for (int i = 0; i < 2 * CellFeatures<NS_>::KP; ++i) x[i] = 0.0f;
  float f[2 + AS];
  f[0] = (float)tv;
  f[1] = logf((float)pv);
#pragma unroll
  for (int k = 0; k < AS; ++k) {
    if (k < ns) {
      const float yf = fmaxf((float)yv[k], 0.0f);
      bc[k] = (powf(yf, BC_LAMBDA) - 1.0f) / BC_LAMBDA;
      f[2 + k] = bc[k];
    }
  }
  outside = false;
#pragma unroll
  for (int i = 0; i < 2 + AS; ++i) {
    if (i < nin) {
      if (!(f[i] >= P.st[ST_LO][i] && f[i] <= P.st[ST_HI][i])) outside = true;
      const float v = (f[i] - P.st[ST_XMU][i]) / P.st[ST_XSD][i];
      const float vh = __bfloat162float(__float2bfloat16_rn(v));
      if (NS_ > 0) {
        x[i] = vh;
        x[nin + i] = v - vh;
        x[2 * nin + i] = vh;
      } else {
        // runtime widths: place the three parts with compile-time indices
#pragma unroll
        for (int j = 0; j < KIN; ++j) {
          if (j == i) x[j] = vh;
          if (j == nin + i) x[j] = v - vh;
          if (j == 2 * nin + i) x[j] = vh;
        }
      }
    }
  }
#pragma unroll
  for (int w = 0; w < CellFeatures<NS_>::KP; ++w) F.xp[w] = pack_bf16(x[2 * w], x[2 * w + 1]);
}

// the packed features of row r into activation chunk 0 (128-byte swizzled K-major row)
template <int NS_>
__device__ __forceinline__ void put_features(const CellFeatures<NS_>& F, unsigned char* arow, int r) {
  constexpr int KP = CellFeatures<NS_>::KP;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    uint4 v;
    v.x = 4 * u + 0 < KP ? F.xp[4 * u + 0] : 0u;
    v.y = 4 * u + 1 < KP ? F.xp[4 * u + 1] : 0u;
    v.z = 4 * u + 2 < KP ? F.xp[4 * u + 2] : 0u;
    v.w = 4 * u + 3 < KP ? F.xp[4 * u + 3] : 0u;
    *reinterpret_cast<uint4*>(arow + ((u ^ (r & 7)) << 4)) = v;
  }
}

// NS_ = the number of species when it is fixed at compile time (every per-cell array in
// registers), 0 for any count up to MAXNS.
template <int NS_>
__global__ void __launch_bounds__(kFwdThreads, 1)
    surrogate_forward_kernel(const __grid_constant__ CUtensorMap tW1, const __grid_constant__ CUtensorMap tW2,
                             const __grid_constant__ CUtensorMap tW3, const __grid_constant__ CUtensorMap tW4,
                             const __grid_constant__ CUtensorMap tW5, const __grid_constant__ SurParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* act = smem;
  unsigned char* wst = smem + ACT_BYTES;
  uint64_t* full = (uint64_t*)(wst + WSTAGES * WSTAGE_BYTES);
  uint64_t* empty = full + WSTAGES;
  // acc_full[h]: the MMAs into accumulator half h (TMEM columns 256 h .. + 255) of a layer are
  // done; chunk_free[c] (c < 4): the layer's second-half MMAs have read activation chunk c, which
  // the first half's epilogue then overwrites (it starts on its accumulator at once and waits
  // only before writing each chunk); act_ready[h]: the epilogue of half h has drained its
  // accumulator and written activation chunks 4 h .. 4 h + 3
  uint64_t* acc_full = empty + WSTAGES;
  uint64_t* chunk_free = acc_full + 2;
  uint64_t* act_ready = chunk_free + 4;
  // feat_ready: the tile's features are in chunk 0 and the previous tile's output (TMEM columns
  // 256 .. 271) has been read
  uint64_t* feat_ready = act_ready + 2;
  uint32_t* tmem_slot = (uint32_t*)(feat_ready + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = (P.ncells + TM - 1) / TM;
  // tiles blockIdx.x, blockIdx.x + gridDim.x, ...: every role of the CTA walks the same sequence
  const long long rounds = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < WSTAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(&acc_full[0], 1);
    mbar_init(&acc_full[1], 1);
    for (int c = 0; c < 4; ++c) mbar_init(&chunk_free[c], 1);
    mbar_init(&act_ready[0], 32 * kEpiWarps / 2);
    mbar_init(&act_ready[1], 32 * kEpiWarps / 2);
    mbar_init(feat_ready, 32 * 4);
    fence_barrier_init();
  }
  if (warp == kTmaWarp) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      // weight stages in the order the MMA issuer consumes them: layer 0 (rows 0-255, then
      // 256-511 of W1), layers 1-3 (first output half: K chunks 0-7, then the second half), layer 4
      prefetch_tmap(&tW1); prefetch_tmap(&tW2); prefetch_tmap(&tW3); prefetch_tmap(&tW4); prefetch_tmap(&tW5);
      long long it = 0;
      bool ok = true;
      for (long long rd = 0; rd < rounds && ok; ++rd) {
        for (int c = 0; c < CHUNKS_PER_TILE; ++c, ++it) {
          const int s = (int)(it % WSTAGES);
          if (!mbar_wait(&empty[s], (uint32_t)((it / WSTAGES) & 1) ^ 1u, P.err)) { ok = false; break; }
          unsigned char* dst = wst + s * WSTAGE_BYTES;
          if (c < 2) {
            mbar_arrive_expect_tx(&full[s], WSTAGE_BYTES);
            tma_load_2d(dst, &tW1, &full[s], 0, c * 256);
          } else if (c < 2 + 48) {
            const int l = (c - 2) / 16, r = (c - 2) % 16, nh = r / 8, kc = r % 8;
            const CUtensorMap* tm = l == 0 ? &tW2 : (l == 1 ? &tW3 : &tW4);
            mbar_arrive_expect_tx(&full[s], WSTAGE_BYTES);
            tma_load_2d(dst, tm, &full[s], kc * 64, nh * 256);
          } else {
            const int kc = c - 50;
            mbar_arrive_expect_tx(&full[s], NOUT * 128);
            tma_load_2d(dst, &tW5, &full[s], kc * 64, 0);
          }
        }
      }
      // drain: every issued stage has been read by the MMAs (their commits have landed)
      const long long first = it > WSTAGES ? it - WSTAGES : 0;
      for (long long k = first; k < it; ++k) mbar_wait(&empty[k % WSTAGES], (uint32_t)((k / WSTAGES) & 1), P.err);
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t id256 = idesc_bf16_f32(128, 256);
      constexpr uint32_t id16 = idesc_bf16_f32(128, NOUT);
      long long it = 0;
      long long n_ready[2] = {0, 0};
      bool ok = true;
      const uint32_t abase = smem_addr(act);
      // one weight stage: A chunk kc (128 x 64) times the stage's B (N x 64) into d
      auto stage = [&](int kc, uint32_t d, uint32_t idesc, bool accumulate) -> bool {
        const int s = (int)(it % WSTAGES);
        if (!mbar_wait(&full[s], (uint32_t)((it / WSTAGES) & 1), P.err)) return false;
        tc_fence_after();
        const uint32_t bbase = smem_addr(wst + s * WSTAGE_BYTES);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16(d, sdesc_k128(abase + kc * ACT_CHUNK + kk * 32), sdesc_k128(bbase + kk * 32), idesc,
                   (accumulate || kk > 0) ? 1u : 0u);
        mma_commit(&empty[s]);                               // frees the stage
        ++it;
        return true;
      };
      auto wait_ready = [&](int h) -> bool {
        if (!mbar_wait(&act_ready[h], (uint32_t)(n_ready[h] & 1), P.err)) return false;
        ++n_ready[h];
        tc_fence_after();
        return true;
      };
      long long n_feat = 0;
      for (long long rd = 0; rd < rounds && ok; ++rd) {
        // layer 0: the features (chunk 0) into both halves
        ok = mbar_wait(feat_ready, (uint32_t)(n_feat & 1), P.err);
        ++n_feat;
        tc_fence_after();
        if (ok) ok = stage(0, tmem, id256, false);
        if (ok) { mma_commit(&acc_full[0]); ok = stage(0, tmem + 256, id256, false); }
        if (ok) {
          for (int c = 0; c < 4; ++c) mma_commit(&chunk_free[c]);
          mma_commit(&acc_full[1]);
        }
        // hidden layers: the first half starts on chunks 0-3 while the second half's epilogue of
        // the previous layer still runs
        for (int l = 1; l < 4 && ok; ++l) {
          ok = wait_ready(0);
          for (int kc = 0; kc < 4 && ok; ++kc) ok = stage(kc, tmem, id256, kc > 0);
          if (ok) ok = wait_ready(1);
          for (int kc = 4; kc < 8 && ok; ++kc) ok = stage(kc, tmem, id256, true);
          if (!ok) break;
          mma_commit(&acc_full[0]);
          for (int kc = 0; kc < 4 && ok; ++kc) {
            ok = stage(kc, tmem + 256, id256, kc > 0);
            if (ok) mma_commit(&chunk_free[kc]);
          }
          if (!ok) break;
          for (int kc = 4; kc < 8 && ok; ++kc) ok = stage(kc, tmem + 256, id256, true);
          if (ok) mma_commit(&acc_full[1]);
        }
        // output layer into columns 256-271 (the second half): the next tile's first-half MMAs
        // need not wait for the output transform
        if (ok) ok = wait_ready(0);
        if (ok) ok = wait_ready(1);
        for (int kc = 0; kc < 8 && ok; ++kc) ok = stage(kc, tmem + 256, id16, kc > 0);
        if (ok) mma_commit(&acc_full[1]);
      }
    }
  } else {
    // ---------------- epilogue warps ----------------
    // Warp w reads TMEM lanes 32 (w % 4) .. + 31 (its cells) of accumulator half w / 8, columns
    // 256 (w / 8) + 128 ((w / 4) % 2) .. + 127 (two 64-column K chunks of the next layer's input):
    // warps 0-7 drain the first half while the second half's MMAs still run, warps 8-15 the second
    // half while the next layer's first-half MMAs start.  Warps 8-11, which wait longer between
    // their blocks, also build the input tiles (the next tile's features right after the current
    // tile's first layer, written once the output layer has read chunk 0) and apply the output
    // transform.
    constexpr int AS = CellFeatures<NS_>::AS;
    const int quarter = warp & 3, half = warp / (kEpiWarps / 2), part = (warp >> 2) % kEpiParts;
    const int r = quarter * 32 + lane;                 // cell row of the tile = TMEM lane
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    unsigned char* arow = act + r * 128;               // row r inside each 16 KB chunk
    const bool io = half == 1 && part == 0;
    const int ns = NS_ > 0 ? NS_ : P.ns;
    long long n_full = 0, n_lo = 0;
    bool ok = true;
    CellFeatures<NS_> F;          // the next tile's features
    auto tile_cell = [&](long long rd) { return (blockIdx.x + rd * gridDim.x) * TM + r; };
    // features of tile rd from the cell's state; the box flag is stored at once, and the Box-Cox
    // values wait in the cell's output slots ynet[k][cell], which the output transform reads and
    // overwrites (this keeps them out of registers for the whole tile)
    auto make_features = [&](long long rd) {
      const long long c = tile_cell(rd);
      if (c < P.ncells) {
        double yv[AS];
#pragma unroll
        for (int k = 0; k < AS; ++k) yv[k] = k < ns ? P.Y[(int64_t)k * P.ld + c] : 0.0;
        bool outside;
        float bc[AS];
        cell_features<NS_>(P, P.T[c], P.p[c], yv, F, bc, outside);
        P.outbox[c] = outside ? 1 : 0;
#pragma unroll
        for (int k = 0; k < AS; ++k)
          if (k < ns) P.ynet[(int64_t)k * P.ncells + c] = bc[k];
      } else {
#pragma unroll
        for (int w = 0; w < CellFeatures<NS_>::KP; ++w) F.xp[w] = 0u;
      }
    };
    if (io && rounds > 0) {
      make_features(0);
      put_features<NS_>(F, arow, r);
      fence_async_smem();
      mbar_arrive(feat_ready);
    }
    for (long long rd = 0; rd < rounds && ok; ++rd) {
      const long long cell = tile_cell(rd);
      const bool valid = cell < P.ncells;
      // ---- hidden layers: this warp's half of the layer's columns ----
      for (int l = 0; l < 4 && ok; ++l) {
        const float* bias = P.hb[l];
        // tcgen05.ld is warp-collective: the warp agrees on the wait's outcome
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[half], (uint32_t)(n_full & 1), P.err))) { ok = false; break; }
        ++n_full;
        tc_fence_after();
        // blocks of 32 columns, one TMEM load at a time (four warps per scheduler hide its latency);
        // the first half's columns overwrite activation chunks 0-3, each once the second half's
        // MMAs have read it
        constexpr int NBLK = 8 / kEpiParts;
        const int col0 = half * 256 + part * (256 / kEpiParts);
        bool fine = true;
        for (int blk = 0; blk < NBLK; ++blk) {
          if (half == 0 && (blk & 1) == 0 &&
              !__all_sync(0xffffffffu, mbar_wait(&chunk_free[(col0 + blk * 32) >> 6], (uint32_t)(n_lo & 1), P.err))) {
            fine = false;
            break;
          }
          uint32_t a[32];
          tmem_ld32(trow + col0 + blk * 32, a);
          tmem_ld_wait(a);
          epilogue_block(a, bias, col0 + blk * 32, arow, r);
        }
        if (!fine) { ok = false; break; }
        ++n_lo;
        tc_fence_before();
        fence_async_smem();
        mbar_arrive(&act_ready[half]);
        if (io && l == 0 && rd + 1 < rounds) make_features(rd + 1);
      }
      if (!ok) break;
      // ---- output layer (columns 256-271), the next tile's input, the output transform ----
      // Every second-half warp follows each phase of acc_full[1] (its parity must not run ahead):
      // the others only wait for the output layer's phase.
      if (half == 1 && !io) {
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[1], (uint32_t)(n_full & 1), P.err))) { ok = false; break; }
        ++n_full;
      }
      if (io) {
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[1], (uint32_t)(n_full & 1), P.err))) { ok = false; break; }
        ++n_full;
        tc_fence_after();
        uint32_t o[16];
        tmem_ld16(trow + 256, o);
        tmem_ld_wait();
        tc_fence_before();
        if (rd + 1 < rounds) {
          put_features<NS_>(F, arow, r);
          fence_async_smem();
          mbar_arrive(feat_ready);
        }
        if (valid) {
#pragma unroll
          for (int k = 0; k < AS; ++k) {
            if (k < ns) {
              const float z = __uint_as_float(o[k]) + P.st[ST_B5][k];
              if (P.zout) P.zout[(int64_t)k * P.ncells + cell] = z;
              const float d = z * P.st[ST_YSD][k] + P.st[ST_YMU][k];
              float* yk = P.ynet + (int64_t)k * P.ncells + cell;
              const float b1 = *yk + d;                // the cell's Box-Cox value, left by make_features
              *yk = powf(fmaxf(1.0f + BC_LAMBDA * b1, 0.0f), 1.0f / BC_LAMBDA);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kTmaWarp) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------------------
// FP64 post-processing
// ---------------------------------------------------------------------------------------
constexpr int NEMAX = 8;

struct PostParams {
  const unsigned char* blob;   // mechanism blob (global memory)
  MechLayout lay;
  const double* Aem;           // [ne][ns] element mass fractions a_ek M_e / W_k, then the pair
                               // products A_ek A_fk, e >= f ([ne (ne + 1) / 2][ns])
  int ne;
  double* T;
  const double* p;
  double* Y;
  int64_t ld, ncells;
  const float* ynet;
  const uint8_t* outbox;
  int8_t* route;
  int32_t* fb_idx;
  unsigned int* fb_count;
};


// The mixture's NASA-7 polynomials of one temperature range for a register-resident
// composition (the sums of mixture_nasa, with the species loop unrolled to the array extent).
template <int AS>
__device__ __forceinline__ void mixture_poly(const double (&Y)[AS], int ns, int rg, const double* hcoef,
                                             const double* ccoef, const double* invW, double (&Ah)[6],
                                             double (&Ac)[5]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) Ah[i] = 0.0;
#pragma unroll
  for (int i = 0; i < 5; ++i) Ac[i] = 0.0;
#pragma unroll
  for (int k = 0; k < AS; ++k) {
    if (k < ns) {
      const double yw = Y[k] * __ldg(invW + k);
      const double* a = hcoef + (rg * ns + k) * 6;
      const double* c = ccoef + (rg * ns + k) * 5;
#pragma unroll
      for (int i = 0; i < 6; ++i) Ah[i] = fma(yw, a[i], Ah[i]);
#pragma unroll
      for (int i = 0; i < 5; ++i) Ac[i] = fma(yw, c[i], Ac[i]);
    }
  }
}

// One cell's post-processing for a mechanism of NS_ species and NE_ elements known at compile
// time: every per-cell array lives in registers (no local-memory frame).
template <int NS_, int NE_>
__global__ void __launch_bounds__(256) surrogate_post_kernel(const PostParams P) {
  constexpr int AS = NS_ > 0 ? NS_ : MAXNS;          // array extents
  constexpr int AE = NE_ > 0 ? NE_ : NEMAX;
  const int ns = NS_ > 0 ? NS_ : P.lay.ns;
  const int ne = NE_ > 0 ? NE_ : P.ne;
  const double* hcoef = (const double*)(P.blob + P.lay.o_hc);
  const double* ccoef = (const double*)(P.blob + P.lay.o_cpc);
  const double* invW = (const double*)(P.blob + P.lay.o_invW);
  for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < P.ncells;
       cell += (int64_t)gridDim.x * blockDim.x) {
    bool pass = P.outbox[cell] == 0;
    double Y0[AS], Y1[AS];
    const double T0 = P.T[cell];
#pragma unroll
    for (int k = 0; k < AS; ++k) {
      if (k < ns) {
        Y0[k] = P.Y[(int64_t)k * P.ld + cell];
        Y1[k] = (double)P.ynet[(int64_t)k * P.ncells + cell];
        if (!isfinite(Y1[k])) pass = false;
      }
    }
    double Tn = T0;
    if (pass) {
      // element-conservation projection: Y'' = Y' - D A^T (A D A^T)^-1 (A Y' - b), D = diag(Y' + 1e-12)
      double b[AE], lam[AE], G[AE][AE];
#pragma unroll
      for (int e = 0; e < AE; ++e) {
        if (e < ne) {
          double sb = 0.0, sr = 0.0;
#pragma unroll
          for (int k = 0; k < AS; ++k) {
            if (k < ns) {
              const double a = P.Aem[e * ns + k];
              sb += a * Y0[k];
              sr += a * Y1[k];
            }
          }
          b[e] = sb;
          lam[e] = sr - sb;
        }
      }
      const double* AA = P.Aem + ne * ns;
#pragma unroll
      for (int e = 0; e < AE; ++e)
#pragma unroll
        for (int f = 0; f <= e; ++f) {
          if (e < ne) {
            double sg = 0.0;
#pragma unroll
            for (int k = 0; k < AS; ++k)
              if (k < ns) sg = fma(AA[k], Y1[k] + 1e-12, sg);
            AA += ns;
            G[e][f] = sg;
            G[f][e] = sg;
          }
        }
      // Gaussian elimination with partial pivoting on the small SPD system; one reciprocal per
      // pivot serves the elimination below it and the back substitution
      double inv_piv[AE];
#pragma unroll
      for (int k = 0; k < AE; ++k) {
        if (k < ne && pass) {
          // pivot search on values (no runtime index into the register array)
          int pr = k;
          double gmax = fabs(G[k][k]);
#pragma unroll
          for (int i = k + 1; i < AE; ++i)
            if (i < ne && fabs(G[i][k]) > gmax) { pr = i; gmax = fabs(G[i][k]); }
          if (gmax == 0.0) {
            pass = false;
          } else {
            if (pr != k) {
#pragma unroll
              for (int j = 0; j < AE; ++j) {
                if (j < ne) {
                  double gk = G[k][j], gp = 0.0;
#pragma unroll
                  for (int i = k + 1; i < AE; ++i) if (i == pr) gp = G[i][j];
                  G[k][j] = gp;
#pragma unroll
                  for (int i = k + 1; i < AE; ++i) if (i == pr) G[i][j] = gk;
                }
              }
              double lk = lam[k], lp = 0.0;
#pragma unroll
              for (int i = k + 1; i < AE; ++i) if (i == pr) lp = lam[i];
              lam[k] = lp;
#pragma unroll
              for (int i = k + 1; i < AE; ++i) if (i == pr) lam[i] = lk;
            }
            inv_piv[k] = 1.0 / G[k][k];
#pragma unroll
            for (int i = k + 1; i < AE; ++i) {
              if (i < ne) {
                const double l = G[i][k] * inv_piv[k];
#pragma unroll
                for (int j = k; j < AE; ++j)
                  if (j < ne) G[i][j] -= l * G[k][j];
                lam[i] -= l * lam[k];
              }
            }
          }
        }
      }
      if (pass) {
#pragma unroll
        for (int i = AE - 1; i >= 0; --i) {
          if (i < ne) {
            double sl = lam[i];
#pragma unroll
            for (int j = i + 1; j < AE; ++j)
              if (j < ne) sl -= G[i][j] * lam[j];
            lam[i] = sl * inv_piv[i];
          }
        }
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int k = 0; k < AS; ++k) {
          if (k < ns) {
            double c = 0.0;
#pragma unroll
            for (int e = 0; e < AE; ++e)
              if (e < ne) c += P.Aem[e * ns + k] * lam[e];
            Y1[k] = fmax(Y1[k] - (Y1[k] + 1e-12) * c, 0.0);
            s0 += Y0[k];
            s1 += Y1[k];
          }
        }
        double res = 0.0;
#pragma unroll
        for (int e = 0; e < AE; ++e) {
          if (e < ne) {
            double sr = 0.0;
#pragma unroll
            for (int k = 0; k < AS; ++k)
              if (k < ns) sr += P.Aem[e * ns + k] * Y1[k];
            res = fmax(res, fabs(sr - b[e]));
          }
        }
        if (!(res <= 1e-9) || !(fabs(s1 - s0) <= 1e-9)) pass = false;
      }
      if (pass) {
        // temperature from enthalpy conservation: h(T, Y'') = h(T0, Y0); the new composition is
        // fixed during the iteration, so its mixture NASA-7 polynomial is formed once per
        // temperature range visited
        double h0;
        {
          // h / R = a5 + a0 T + ... + a4 T^5 per species (no division by T)
          const int rg0 = T0 < TMID ? 0 : 1;
          double hs = 0.0;
#pragma unroll
          for (int k = 0; k < AS; ++k) {
            if (k < ns) {
              const double* a = hcoef + (rg0 * ns + k) * 6;
              const double hR = a[5] + T0 * (a[0] + T0 * (a[1] + T0 * (a[2] + T0 * (a[3] + T0 * a[4]))));
              hs += Y0[k] * hR * __ldg(invW + k);
            }
          }
          h0 = RU * hs;
        }
        double Ah[6], Ac[5];
        int rg = Tn < TMID ? 0 : 1;
        mixture_poly<AS>(Y1, ns, rg, hcoef, ccoef, invW, Ah, Ac);
        bool conv = false;
        for (int it = 0; it < 50; ++it) {
          const int r = Tn < TMID ? 0 : 1;
          if (r != rg) { rg = r; mixture_poly<AS>(Y1, ns, rg, hcoef, ccoef, invW, Ah, Ac); }
          double hh, cp;
          h_cp_from_mixture(Ah, Ac, Tn, &hh, &cp);
          const double dT = (hh - h0) / cp;
          Tn -= dT;
          if (!(Tn >= 200.0 && Tn <= 6000.0)) break;
          if (fabs(dT) < 1e-9 * Tn) { conv = true; break; }
        }
        if (!conv) pass = false;
      }
    }
    if (pass) {
      P.T[cell] = Tn;
#pragma unroll
      for (int k = 0; k < AS; ++k)
        if (k < ns) P.Y[(int64_t)k * P.ld + cell] = Y1[k];
    } else {
      const unsigned slot = atomicAdd(P.fb_count, 1u);
      P.fb_idx[slot] = (int32_t)cell;
    }
    if (P.route) P.route[cell] = pass ? 0 : 1;
  }
}

// The same post-processing for any species and element counts (runtime loops; per-cell arrays
// sized for the maxima, in local memory).
__global__ void surrogate_post_general(const PostParams P) {
  const int ns = P.lay.ns;
  for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < P.ncells;
       cell += (int64_t)gridDim.x * blockDim.x) {
    bool pass = P.outbox[cell] == 0;
    double Y0[MAXNS], Y1[MAXNS];
    double T0 = P.T[cell];
    for (int k = 0; k < ns; ++k) {
      Y0[k] = P.Y[(int64_t)k * P.ld + cell];
      Y1[k] = (double)P.ynet[(int64_t)k * P.ncells + cell];
      if (!isfinite(Y1[k])) pass = false;
    }
    double Tn = T0;
    if (pass) {
      // element-conservation projection: Y'' = Y' - D A^T (A D A^T)^-1 (A Y' - b)
      const int ne = P.ne;
      double b[NEMAX], rr[NEMAX], G[NEMAX][NEMAX], lam[NEMAX];
      for (int e = 0; e < ne; ++e) {
        double sb = 0.0, sr = 0.0;
        for (int k = 0; k < ns; ++k) {
          const double a = P.Aem[e * ns + k];
          sb += a * Y0[k];
          sr += a * Y1[k];
        }
        b[e] = sb;
        rr[e] = sr - sb;
      }
      double Yp[MAXNS];
      for (int k = 0; k < ns; ++k) Yp[k] = Y1[k] + 1e-12;
      const double* AA = P.Aem + ne * ns;
      for (int e = 0; e < ne; ++e)
        for (int f = 0; f <= e; ++f, AA += ns) {
          double s = 0.0;
          for (int k = 0; k < ns; ++k) s = fma(AA[k], Yp[k], s);
          G[e][f] = s;
          G[f][e] = s;
        }
      // Gaussian elimination with partial pivoting on the small SPD system; one reciprocal per
      // pivot serves the elimination below it and the back substitution
      double inv_piv[NEMAX];
      for (int e = 0; e < ne; ++e) lam[e] = rr[e];
      for (int k = 0; k < ne; ++k) {
        int pr = k;
        for (int i = k + 1; i < ne; ++i)
          if (fabs(G[i][k]) > fabs(G[pr][k])) pr = i;
        if (G[pr][k] == 0.0) { pass = false; break; }
        if (pr != k) {
          for (int j = 0; j < ne; ++j) { const double t = G[k][j]; G[k][j] = G[pr][j]; G[pr][j] = t; }
          const double t = lam[k]; lam[k] = lam[pr]; lam[pr] = t;
        }
        inv_piv[k] = 1.0 / G[k][k];
        for (int i = k + 1; i < ne; ++i) {
          const double l = G[i][k] * inv_piv[k];
          for (int j = k; j < ne; ++j) G[i][j] -= l * G[k][j];
          lam[i] -= l * lam[k];
        }
      }
      if (pass) {
        for (int i = ne - 1; i >= 0; --i) {
          double s = lam[i];
          for (int j = i + 1; j < ne; ++j) s -= G[i][j] * lam[j];
          lam[i] = s * inv_piv[i];
        }
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < ns; ++k) {
          double c = 0.0;
          for (int e = 0; e < ne; ++e) c += P.Aem[e * ns + k] * lam[e];
          Y1[k] = fmax(Y1[k] - (Y1[k] + 1e-12) * c, 0.0);
          s0 += Y0[k];
          s1 += Y1[k];
        }
        double res = 0.0;
        for (int e = 0; e < ne; ++e) {
          double s = 0.0;
          for (int k = 0; k < ns; ++k) s += P.Aem[e * ns + k] * Y1[k];
          res = fmax(res, fabs(s - b[e]));
        }
        if (!(res <= 1e-9) || !(fabs(s1 - s0) <= 1e-9)) pass = false;
      }
      if (pass) {
        // temperature from enthalpy conservation: h(T, Y'') = h(T0, Y0)
        const double h0 = h_mass(P.blob, P.lay, T0, Y0);
        // the new composition is fixed during the iteration: its mixture polynomial once per
        // temperature range visited
        double Ah[6], Ac[5];
        int rg = Tn < TMID ? 0 : 1;
        mixture_nasa(P.blob, P.lay, rg, Y1, Ah, Ac);
        bool conv = false;
        for (int it = 0; it < 50; ++it) {
          const int r = Tn < TMID ? 0 : 1;
          if (r != rg) { rg = r; mixture_nasa(P.blob, P.lay, rg, Y1, Ah, Ac); }
          double hh, cp;
          h_cp_from_mixture(Ah, Ac, Tn, &hh, &cp);
          const double dT = (hh - h0) / cp;
          Tn -= dT;
          if (!(Tn >= 200.0 && Tn <= 6000.0)) break;
          if (fabs(dT) < 1e-9 * Tn) { conv = true; break; }
        }
        if (!conv) pass = false;
      }
    }
    if (pass) {
      P.T[cell] = Tn;
      for (int k = 0; k < ns; ++k) P.Y[(int64_t)k * P.ld + cell] = Y1[k];
    } else {
      const unsigned slot = atomicAdd(P.fb_count, 1u);
      P.fb_idx[slot] = (int32_t)cell;
    }
    if (P.route) P.route[cell] = pass ? 0 : 1;
  }
}

// heat-release rate of a step: q = -rho0 sum_k h_k(T0) (Y1_k - Y0_k) / (W_k dt), h_k molar
__global__ void heat_release_kernel(const unsigned char* blob, MechLayout L, const double* T0, const double* p,
                                    const double* Y0, const double* Y1, int64_t ld, int64_t n, double dt,
                                    double* q) {
  const int ns = L.ns;
  const double* hc = (const double*)(blob + L.o_hc);
  const double* invW = (const double*)(blob + L.o_invW);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const double T = T0[c], invT = 1.0 / T;
    const int rg = T < TMID ? 0 : 1;
    double S = 0.0, acc = 0.0;
    for (int k = 0; k < ns; ++k) {
      const double* a = hc + (rg * ns + k) * 6;
      const double hRT = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4]))) + a[5] * invT;
      const double y0 = Y0[(int64_t)k * ld + c];
      S += y0 * __ldg(invW + k);
      acc += hRT * (Y1[(int64_t)k * ld + c] - y0) * __ldg(invW + k);
    }
    const double rho = p[c] / (RU * T * S);
    q[c] = -rho * RU * T * acc / dt;
  }
}

}  // namespace chem

extern "C" int chem_heat_release(chem_mech_t m, const double* T0, const double* p, const double* Y0,
                                 const double* Y1, int64_t ld, int64_t ncells, double dt, double* q,
                                 chem_stream_t stream) {
  using namespace chem;
  if (!m || !T0 || !p || !Y0 || !Y1 || !q || ncells < 0 || ld < ncells || !(dt > 0.0)) {
    set_error("bad arguments");
    return CHEM_EINVAL;
  }
  if (ncells == 0) return CHEM_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((ncells + 255) / 256, 8192);
  heat_release_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const unsigned char*)m->d_blob, m->lay, T0, p,
                                                                  Y0, Y1, ld, ncells, dt, q);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

namespace chem {}

// ---------------------------------------------------------------------------------------
// model object and entry points
// ---------------------------------------------------------------------------------------

namespace chem {

static uint16_t f2bf(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  const uint32_t bias = ((u >> 16) & 1u) + 0x7fffu;
  return (uint16_t)((u + bias) >> 16);
}

int surrogate_forward(chem_model_s* md, const double* T, const double* p, const double* Y, int64_t ld,
                      int64_t ncells, float* ynet, float* zout, uint8_t* outbox, int* err,
                      cudaStream_t stream) {
  if (md->kind == 1) return surrogate_forward_ps(md, T, p, Y, ld, ncells, ynet, zout, outbox, err, stream);
  static bool attr = false;
  if (!attr) {
    CHEM_CUDA_TRY(cudaFuncSetAttribute(surrogate_forward_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       FWD_SMEM));
    CHEM_CUDA_TRY(cudaFuncSetAttribute(surrogate_forward_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       FWD_SMEM));
    attr = true;
  }
  SurParams P;
  memcpy(P.hb, md->hbias, sizeof(P.hb));
  memcpy(P.st, md->hstat, sizeof(P.st));
  P.ns = md->ns; P.nin = md->nin; P.T = T; P.p = p; P.Y = Y; P.ld = ld; P.ncells = ncells;
  P.ynet = ynet; P.zout = zout; P.outbox = outbox; P.err = err;
  // persistent grid: as many CTAs as can be resident at once (one per SM), no more than the tiles
  static int max_ctas = 0;
  if (max_ctas == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    CHEM_CUDA_TRY(cudaGetDevice(&dev));
    CHEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CHEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, surrogate_forward_kernel<0>, kFwdThreads,
                                                                FWD_SMEM));
    if (per_sm < 1) { set_error("surrogate kernel does not fit on an SM"); return CHEM_ECUDA; }
    max_ctas = sms * per_sm;
  }
  if (ncells < 1) return CHEM_OK;
  const long long ntiles = (ncells + TM - 1) / TM;
  const long long grid = std::min<long long>(ntiles, max_ctas);
  if (md->ns == 9)
    surrogate_forward_kernel<9><<<(unsigned)grid, kFwdThreads, FWD_SMEM, stream>>>(md->tw[0], md->tw[1], md->tw[2],
                                                                                  md->tw[3], md->tw[4], P);
  else
    surrogate_forward_kernel<0><<<(unsigned)grid, kFwdThreads, FWD_SMEM, stream>>>(md->tw[0], md->tw[1], md->tw[2],
                                                                                  md->tw[3], md->tw[4], P);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

int launch_advance_counted(chem_mech_s* m, double* T, const double* p, double* Y, int64_t ld,
                           double dt, int64_t capacity, const unsigned int* count_dev, double rtol,
                           double atol, const int32_t* idx, cudaStream_t stream);

}  // namespace chem

using namespace chem;

// Element mass fractions A[e][k] = a_ek M_e / W_k ([ne][ns]), followed by the products
// A[e][k] A[f][k] of every pair e <= f ([ne (ne + 1) / 2][ns], pairs in row order), which the
// projection's normal matrix sum_k A_ek A_fk (Y_k + 1e-12) needs per cell.
static std::vector<double> element_matrices(chem_mech_t mech, int ns) {
  const int ne = mech->ne;
  std::vector<double> A((size_t)ne * ns + (size_t)ne * (ne + 1) / 2 * ns);
  for (int e = 0; e < ne; ++e)
    for (int k = 0; k < ns; ++k)
      A[(size_t)e * ns + k] = mech->comp[(size_t)k * ne + e] * mech->elem_mass[e] / mech->W[k];
  size_t o = (size_t)ne * ns;
  for (int e = 0; e < ne; ++e)
    for (int f = 0; f <= e; ++f, o += ns)
      for (int k = 0; k < ns; ++k) A[o + k] = A[(size_t)e * ns + k] * A[(size_t)f * ns + k];
  return A;
}

extern "C" int chem_surrogate_create(const chem_surrogate_desc* d, chem_mech_t mech, chem_model_t* out) {
  if (!d || !mech || !out) { set_error("NULL argument"); return CHEM_EINVAL; }
  *out = nullptr;
  const int ns = d->n_species, nin = ns + 2;
  if (ns != mech->ns || ns < 1 || ns > MAXNS || d->hidden != HID || nin > KIN || mech->ne > NEMAX) {
    set_error("surrogate shape unsupported (ns=%d, mechanism ns=%d, hidden=%d, ne=%d)", ns, mech->ns,
              d->hidden, mech->ne);
    return CHEM_EINVAL;
  }
  if (!(d->dt > 0.0)) { set_error("surrogate dt must be positive"); return CHEM_EINVAL; }
  for (int l = 0; l < 5; ++l)
    if (!d->W[l] || !d->b[l]) { set_error("NULL weight or bias"); return CHEM_EINVAL; }
  if (!d->x_mean || !d->x_std || !d->y_mean || !d->y_std || !d->box_lo || !d->box_hi) {
    set_error("NULL normalisation statistics");
    return CHEM_EINVAL;
  }
  chem_model_s* md = new chem_model_s();
  md->ns = ns; md->nin = nin; md->ne = mech->ne; md->dt = d->dt;
  // BF16 weights, zero padded: W1 [512 x 64] as [W_hi | W_hi | W_lo], W2..W4 [512 x 512],
  // W5 [16 x 512]
  const size_t n1 = (size_t)HID * KIN, nh = (size_t)HID * HID, n5 = (size_t)NOUT * HID;
  std::vector<uint16_t> wb(n1 + 3 * nh + n5, 0);
  for (int o = 0; o < HID; ++o)
    for (int i = 0; i < nin; ++i) {
      const float w = d->W[0][(size_t)o * nin + i];
      const uint16_t hi = f2bf(w);
      const uint32_t hbits = (uint32_t)hi << 16;
      float wh;
      memcpy(&wh, &hbits, 4);
      wb[(size_t)o * KIN + i] = hi;
      wb[(size_t)o * KIN + nin + i] = hi;
      wb[(size_t)o * KIN + 2 * nin + i] = f2bf(w - wh);
    }
  for (int l = 1; l < 4; ++l)
    for (size_t e = 0; e < nh; ++e) wb[n1 + (l - 1) * nh + e] = f2bf(d->W[l][e]);
  for (int o = 0; o < ns; ++o)
    for (int i = 0; i < HID; ++i) wb[n1 + 3 * nh + (size_t)o * HID + i] = f2bf(d->W[4][(size_t)o * HID + i]);
  // FP32: 4 hidden biases, padded output bias, statistics
  std::vector<float> fb(4 * HID + NOUT + 6 * KIN, 0.0f);
  for (int l = 0; l < 4; ++l) memcpy(&fb[l * HID], d->b[l], HID * sizeof(float));
  for (int l = 0; l < 4; ++l) memcpy(md->hbias[l], d->b[l], HID * sizeof(float));
  memcpy(&fb[4 * HID], d->b[4], ns * sizeof(float));
  float* st = &fb[4 * HID + NOUT];
  for (int i = 0; i < nin; ++i) {
    st[i] = d->x_mean[i];
    st[KIN + i] = d->x_std[i] > 0.0f ? d->x_std[i] : 1.0f;
    st[4 * KIN + i] = d->box_lo[i];
    st[5 * KIN + i] = d->box_hi[i];
  }
  for (int k = 0; k < ns; ++k) {
    st[2 * KIN + k] = d->y_mean[k];
    st[3 * KIN + k] = d->y_std[k];
  }
  for (int i = 0; i < nin; ++i) {
    md->hstat[ST_XMU][i] = st[i];
    md->hstat[ST_XSD][i] = st[KIN + i];
    md->hstat[ST_LO][i] = st[4 * KIN + i];
    md->hstat[ST_HI][i] = st[5 * KIN + i];
  }
  for (int k = 0; k < ns; ++k) {
    md->hstat[ST_YMU][k] = st[2 * KIN + k];
    md->hstat[ST_YSD][k] = st[3 * KIN + k];
    md->hstat[ST_B5][k] = d->b[4][k];
  }
  std::vector<double> A = element_matrices(mech, ns);
  auto fail = [&](int rc) { chem_surrogate_free(md); return rc; };
  if (cudaGetDevice(&md->device) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "cudaGetDevice"));
  cudaError_t e1 = cudaMalloc(&md->d_w, wb.size() * 2);
  cudaError_t e2 = cudaMalloc(&md->d_f, fb.size() * 4);
  cudaError_t e3 = cudaMalloc((void**)&md->d_A, A.size() * 8);
  if (e1 || e2 || e3) return fail(cuda_fail(e1 ? e1 : (e2 ? e2 : e3), "cudaMalloc(surrogate)"));
  if (cudaMemcpy(md->d_w, wb.data(), wb.size() * 2, cudaMemcpyHostToDevice) ||
      cudaMemcpy(md->d_f, fb.data(), fb.size() * 4, cudaMemcpyHostToDevice) ||
      cudaMemcpy(md->d_A, A.data(), A.size() * 8, cudaMemcpyHostToDevice))
    return fail(cuda_fail(cudaGetLastError(), "cudaMemcpy(surrogate)"));
  const uint16_t* w = (const uint16_t*)md->d_w;
  const float* f = (const float*)md->d_f;
  for (int l = 0; l < 4; ++l) md->bias[l] = f + l * HID;
  md->bias[4] = f + 4 * HID;
  const float* sd = f + 4 * HID + NOUT;
  md->xmu = sd; md->xsd = sd + KIN; md->ymu = sd + 2 * KIN; md->ysd = sd + 3 * KIN;
  md->lo = sd + 4 * KIN; md->hi = sd + 5 * KIN;
  // hidden-layer weight boxes are one 256-row x 64-column stage (32 KB)
  int rc = make_tmap_bf16(&md->tw[0], w, HID, KIN, KIN, 256, 64);
  for (int l = 1; l < 4 && !rc; ++l)
    rc = make_tmap_bf16(&md->tw[l], w + n1 + (l - 1) * nh, HID, HID, HID, 256, 64);
  if (!rc) rc = make_tmap_bf16(&md->tw[4], w + n1 + 3 * nh, NOUT, HID, HID, NOUT, 64);
  if (rc) return fail(rc);
  *out = md;
  return CHEM_OK;
}

extern "C" int chem_surrogate_create_per_species(const chem_surrogate_ps_desc* d, chem_mech_t mech,
                                                 chem_model_t* out) {
  if (!d || !mech || !out) { set_error("NULL argument"); return CHEM_EINVAL; }
  *out = nullptr;
  const int ns = d->n_species, nin = ns + 2;
  if (ns != mech->ns || ns < 1 || ns > MAXNS || 3 * nin > KIN || mech->ne > NEMAX) {
    set_error("surrogate shape unsupported (ns=%d, mechanism ns=%d, ne=%d)", ns, mech->ns, mech->ne);
    return CHEM_EINVAL;
  }
  const int h1 = d->hidden[0], h2 = d->hidden[1], h3 = d->hidden[2];
  for (int i = 0; i < 3; ++i)
    if (d->hidden[i] < 128 || d->hidden[i] > 8192 || d->hidden[i] % 8) {
      set_error("per-species hidden widths must be multiples of 8 in [128, 8192] (got %d)", d->hidden[i]);
      return CHEM_EINVAL;
    }
  if (!(d->dt > 0.0)) { set_error("surrogate dt must be positive"); return CHEM_EINVAL; }
  if (!d->x_mean || !d->x_std || !d->y_mean || !d->y_std || !d->box_lo || !d->box_hi) {
    set_error("NULL normalisation statistics");
    return CHEM_EINVAL;
  }
  chem_model_s* md = new chem_model_s();
  md->kind = 1; md->ns = ns; md->nin = nin; md->ne = mech->ne; md->dt = d->dt;
  md->h[0] = h1; md->h[1] = h2; md->h[2] = h3;
  // BF16: the first layers of all networks stacked, [nnet h1 x 64] (compensated; one GEMM feeds
  // every network from the shared features), then per network W2 [h2 x h1], W3 [h3 x h2], w4 [h3];
  // FP32: the stacked b1 [nnet h1], then per network b2 [h2], b3 [h3], b4 (4 slots); then the
  // statistics block
  const size_t nw1 = (size_t)h1 * KIN, nw2 = (size_t)h2 * h1, nw3 = (size_t)h3 * h2, nw4 = (size_t)h3;
  const size_t per_w = nw2 + nw3 + nw4, per_f = (size_t)h2 + h3 + 4;
  std::vector<int> sp;
  for (int k = 0; k < ns; ++k) {
    const bool any = d->W[k][0] || d->W[k][1] || d->W[k][2] || d->W[k][3];
    if (!any) continue;
    for (int l = 0; l < 4; ++l)
      if (!d->W[k][l] || !d->b[k][l]) { set_error("species %d: NULL weight or bias", k); delete md; return CHEM_EINVAL; }
    sp.push_back(k);
  }
  md->nnet = (int)sp.size();
  const size_t nsp = sp.size();
  std::vector<uint16_t> wb(nw1 * nsp + per_w * std::max<size_t>(nsp, 1), 0);
  std::vector<float> fb((size_t)h1 * nsp + per_f * nsp + 6 * KIN, 0.0f);
  for (size_t s = 0; s < sp.size(); ++s) {
    const int k = sp[s];
    uint16_t* w1 = &wb[s * nw1];
    uint16_t* w = &wb[nw1 * nsp + s * per_w];
    for (int o = 0; o < h1; ++o)
      for (int i = 0; i < nin; ++i) {
        const float v = d->W[k][0][(size_t)o * nin + i];
        const uint16_t hi = f2bf(v);
        const uint32_t hbits = (uint32_t)hi << 16;
        float vh;
        memcpy(&vh, &hbits, 4);
        w1[(size_t)o * KIN + i] = hi;
        w1[(size_t)o * KIN + nin + i] = hi;
        w1[(size_t)o * KIN + 2 * nin + i] = f2bf(v - vh);
      }
    for (size_t e = 0; e < nw2; ++e) w[e] = f2bf(d->W[k][1][e]);
    for (size_t e = 0; e < nw3; ++e) w[nw2 + e] = f2bf(d->W[k][2][e]);
    for (size_t e = 0; e < nw4; ++e) w[nw2 + nw3 + e] = f2bf(d->W[k][3][e]);
    memcpy(&fb[s * h1], d->b[k][0], h1 * sizeof(float));
    float* f = &fb[(size_t)h1 * nsp + s * per_f];
    memcpy(f, d->b[k][1], h2 * sizeof(float));
    memcpy(f + h2, d->b[k][2], h3 * sizeof(float));
    f[h2 + h3] = d->b[k][3][0];
  }
  float* st = &fb[(size_t)h1 * nsp + per_f * nsp];
  for (int i = 0; i < nin; ++i) {
    st[i] = d->x_mean[i];
    st[KIN + i] = d->x_std[i] > 0.0f ? d->x_std[i] : 1.0f;
    st[4 * KIN + i] = d->box_lo[i];
    st[5 * KIN + i] = d->box_hi[i];
  }
  for (int k = 0; k < ns; ++k) {
    st[2 * KIN + k] = d->y_mean[k];
    st[3 * KIN + k] = d->y_std[k];
  }
  std::vector<double> A = element_matrices(mech, ns);
  auto fail = [&](int rc) { chem_surrogate_free(md); return rc; };
  if (cudaGetDevice(&md->device) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "cudaGetDevice"));
  cudaError_t e1 = cudaMalloc(&md->d_w, wb.size() * 2);
  cudaError_t e2 = cudaMalloc(&md->d_f, fb.size() * 4);
  cudaError_t e3 = cudaMalloc((void**)&md->d_A, A.size() * 8);
  if (e1 || e2 || e3) return fail(cuda_fail(e1 ? e1 : (e2 ? e2 : e3), "cudaMalloc(surrogate)"));
  if (cudaMemcpy(md->d_w, wb.data(), wb.size() * 2, cudaMemcpyHostToDevice) ||
      cudaMemcpy(md->d_f, fb.data(), fb.size() * 4, cudaMemcpyHostToDevice) ||
      cudaMemcpy(md->d_A, A.data(), A.size() * 8, cudaMemcpyHostToDevice))
    return fail(cuda_fail(cudaGetLastError(), "cudaMemcpy(surrogate)"));
  const uint16_t* w = (const uint16_t*)md->d_w;
  const float* f = (const float*)md->d_f;
  for (size_t s = 0; s < sp.size(); ++s) {
    PsNet& n = md->net[s];
    n.species = sp[s];
    const uint16_t* ws = w + nw1 * nsp + s * per_w;
    n.W1 = w + s * nw1; n.W2 = ws; n.W3 = ws + nw2; n.w4 = ws + nw2 + nw3;
    const float* fs = f + (size_t)h1 * nsp + s * per_f;
    n.b1 = f + s * h1; n.b2 = fs; n.b3 = fs + h2; n.b4 = fs + h2 + h3;
  }
  const float* sd = f + (size_t)h1 * nsp + per_f * nsp;
  md->xmu = sd; md->xsd = sd + KIN; md->ymu = sd + 2 * KIN; md->ysd = sd + 3 * KIN;
  md->lo = sd + 4 * KIN; md->hi = sd + 5 * KIN;
  *out = md;
  return CHEM_OK;
}

// CHEMSUR2 (per-species networks): magic, int32 ns, int32 h1, h2, h3, double dt, int32 nnet,
// int32 species[nnet], then per network W1, b1, W2, b2, W3, b3, W4, b4, then the statistics
static int load_per_species(std::ifstream& f, const char* path, chem_mech_t mech, chem_model_t* out) {
  int32_t ns = 0, h[3] = {0, 0, 0}, nnet = 0;
  double dt = 0.0;
  f.read((char*)&ns, 4);
  f.read((char*)h, 12);
  f.read((char*)&dt, 8);
  f.read((char*)&nnet, 4);
  if (!f || ns < 1 || ns > MAXNS || nnet < 0 || nnet > ns) {
    set_error("%s: not a per-species surrogate model file", path);
    return CHEM_EINVAL;
  }
  for (int i = 0; i < 3; ++i)
    if (h[i] < 128 || h[i] > 8192) { set_error("%s: bad hidden width", path); return CHEM_EINVAL; }
  std::vector<int32_t> sp(nnet);
  f.read((char*)sp.data(), 4 * (size_t)nnet);
  const int nin = ns + 2;
  const size_t wsz[4] = {(size_t)h[0] * nin, (size_t)h[1] * h[0], (size_t)h[2] * h[1], (size_t)h[2]};
  const size_t bsz[4] = {(size_t)h[0], (size_t)h[1], (size_t)h[2], 1};
  std::vector<std::vector<float>> W(4 * (size_t)nnet), b(4 * (size_t)nnet);
  chem_surrogate_ps_desc d{};
  d.n_species = ns; d.hidden[0] = h[0]; d.hidden[1] = h[1]; d.hidden[2] = h[2]; d.dt = dt;
  for (int s = 0; s < nnet; ++s) {
    if (sp[s] < 0 || sp[s] >= ns) { set_error("%s: bad species index", path); return CHEM_EINVAL; }
    for (int l = 0; l < 4; ++l) {
      W[4 * s + l].resize(wsz[l]);
      b[4 * s + l].resize(bsz[l]);
      f.read((char*)W[4 * s + l].data(), wsz[l] * 4);
      f.read((char*)b[4 * s + l].data(), bsz[l] * 4);
      d.W[sp[s]][l] = W[4 * s + l].data();
      d.b[sp[s]][l] = b[4 * s + l].data();
    }
  }
  std::vector<float> xm(nin), xs(nin), ym(ns), ys(ns), lo(nin), hi(nin);
  f.read((char*)xm.data(), nin * 4); f.read((char*)xs.data(), nin * 4);
  f.read((char*)ym.data(), ns * 4); f.read((char*)ys.data(), ns * 4);
  f.read((char*)lo.data(), nin * 4); f.read((char*)hi.data(), nin * 4);
  if (!f) { set_error("%s: truncated surrogate model file", path); return CHEM_EINVAL; }
  d.x_mean = xm.data(); d.x_std = xs.data(); d.y_mean = ym.data(); d.y_std = ys.data();
  d.box_lo = lo.data(); d.box_hi = hi.data();
  return chem_surrogate_create_per_species(&d, mech, out);
}

extern "C" int chem_surrogate_load(const char* path, chem_mech_t mech, chem_model_t* out) {
  if (!path || !mech || !out) { set_error("NULL argument"); return CHEM_EINVAL; }
  std::ifstream f(path, std::ios::binary);
  if (!f) { set_error("cannot open %s", path); return CHEM_ENOTFOUND; }
  char magic[8];
  int32_t ns = 0, hid = 0;
  double dt = 0.0;
  f.read(magic, 8);
  if (f && memcmp(magic, "CHEMSUR2", 8) == 0) return load_per_species(f, path, mech, out);
  f.read((char*)&ns, 4);
  f.read((char*)&hid, 4);
  f.read((char*)&dt, 8);
  if (!f || memcmp(magic, "CHEMSUR1", 8) != 0 || ns < 1 || ns > MAXNS || hid != HID) {
    set_error("%s: not a surrogate model file", path);
    return CHEM_EINVAL;
  }
  const int nin = ns + 2;
  const size_t sizes[5] = {(size_t)HID * nin, (size_t)HID * HID, (size_t)HID * HID, (size_t)HID * HID,
                           (size_t)ns * HID};
  const size_t bsz[5] = {HID, HID, HID, HID, (size_t)ns};
  std::vector<float> W[5], b[5], xm(nin), xs(nin), ym(ns), ys(ns), lo(nin), hi(nin);
  for (int l = 0; l < 5; ++l) {
    W[l].resize(sizes[l]);
    b[l].resize(bsz[l]);
    f.read((char*)W[l].data(), sizes[l] * 4);
    f.read((char*)b[l].data(), bsz[l] * 4);
  }
  f.read((char*)xm.data(), nin * 4); f.read((char*)xs.data(), nin * 4);
  f.read((char*)ym.data(), ns * 4); f.read((char*)ys.data(), ns * 4);
  f.read((char*)lo.data(), nin * 4); f.read((char*)hi.data(), nin * 4);
  if (!f) { set_error("%s: truncated surrogate model file", path); return CHEM_EINVAL; }
  chem_surrogate_desc d{};
  d.n_species = ns; d.hidden = hid; d.dt = dt;
  for (int l = 0; l < 5; ++l) { d.W[l] = W[l].data(); d.b[l] = b[l].data(); }
  d.x_mean = xm.data(); d.x_std = xs.data(); d.y_mean = ym.data(); d.y_std = ys.data();
  d.box_lo = lo.data(); d.box_hi = hi.data();
  return chem_surrogate_create(&d, mech, out);
}

extern "C" int chem_surrogate_free(chem_model_t md) {
  if (!md) { set_error("NULL model"); return CHEM_EINVAL; }
  if (md->d_w) cudaFree(md->d_w);
  if (md->d_f) cudaFree(md->d_f);
  if (md->d_A) cudaFree(md->d_A);
  delete md;
  return CHEM_OK;
}

extern "C" int chem_surrogate_forward(chem_model_t md, const double* T, const double* p, const double* Y,
                                      int64_t ld, int64_t ncells, float* ynet, float* zout,
                                      uint8_t* out_of_box, chem_stream_t stream) {
  if (!md) { set_error("NULL model"); return CHEM_EINVAL; }
  if (ncells < 0 || ld < ncells) { set_error("bad ncells / ld"); return CHEM_EINVAL; }
  if (ncells == 0) return CHEM_OK;
  if (!T || !p || !Y || !ynet || !out_of_box) { set_error("NULL pointer"); return CHEM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  CHEM_CUDA_TRY(cudaMallocAsync((void**)&err, sizeof(int), st));
  CHEM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  int rc = surrogate_forward(md, T, p, Y, ld, ncells, ynet, zout, out_of_box, err, st);
  int herr = 0;
  if (!rc) {
    // the timeout flag is checked once the stream reaches this point
    CHEM_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CHEM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(err, st);
  if (rc) return rc;
  if (herr) { set_error("surrogate forward kernel: a pipeline wait timed out"); return CHEM_ECUDA; }
  return CHEM_OK;
}

// ---------------------------------------------------------------------------------------
// several solvers' states in one surrogate pass: gathered into one contiguous state, advanced by
// one forward launch, one post-processing launch and one FP64 fallback launch, scattered back
// ---------------------------------------------------------------------------------------
namespace chem {

struct GatherSeg {
  double* T;
  const double* p;
  double* Y;
  int64_t ld;
  int64_t begin;        // first gathered cell of the segment
  int8_t* route;        // nullable
};

struct GatherParams {
  GatherSeg seg[kMaxSegsPerLaunch];
  int nseg, ns;
  int64_t n;            // gathered cells (also the gathered arrays' leading dimension)
  double* T;
  double* p;
  double* Y;
  const int8_t* route;
};

__device__ __forceinline__ int seg_of(const GatherParams& P, int64_t i) {
  int s = 0;
  while (s + 1 < P.nseg && P.seg[s + 1].begin <= i) ++s;
  return s;
}

__global__ void gather_kernel(const __grid_constant__ GatherParams P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    const GatherSeg& g = P.seg[seg_of(P, i)];
    const int64_t c = i - g.begin;
    P.T[i] = g.T[c];
    P.p[i] = g.p[c];
    for (int k = 0; k < P.ns; ++k) P.Y[(int64_t)k * P.n + i] = g.Y[(int64_t)k * g.ld + c];
  }
}

__global__ void scatter_kernel(const __grid_constant__ GatherParams P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    const GatherSeg& g = P.seg[seg_of(P, i)];
    const int64_t c = i - g.begin;
    g.T[c] = P.T[i];
    for (int k = 0; k < P.ns; ++k) g.Y[(int64_t)k * g.ld + c] = P.Y[(int64_t)k * P.n + i];
    if (g.route) g.route[c] = P.route[i];
  }
}

}  // namespace chem

extern "C" int chem_surrogate_advance(chem_model_t md, chem_mech_t mech, double* T, const double* p,
                                      double* Y, int64_t ld, double dt, int64_t ncells, double rtol,
                                      double atol, int8_t* route_out, chem_stream_t stream);

extern "C" int chem_surrogate_advance_batch(chem_model_t md, chem_mech_t mech, const chem_segment* segs, int nseg,
                                            chem_stream_t stream) {
  if (!md || !mech || !segs || nseg < 1) { set_error("bad batch arguments"); return CHEM_EINVAL; }
  for (int i = 0; i < nseg; ++i) {
    const chem_segment& a = segs[i];
    if (a.ncells < 0 || (a.ncells > 0 && (!a.T || !a.p || !a.Y)) || a.ld < a.ncells || a.idx ||
        !(fabs(a.dt - md->dt) <= 1e-12 * md->dt) || a.rtol != segs[0].rtol || a.atol != segs[0].atol ||
        !(a.rtol > 0.0) || !(a.atol > 0.0)) {
      set_error("segment %d: invalid (indexed segment, bad sizes, a dt other than the model's, or "
                "tolerances that differ from the first segment's)", i);
      return CHEM_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int ns = md->ns;
  for (int first = 0; first < nseg; first += kMaxSegsPerLaunch) {
    const int cnt = std::min(kMaxSegsPerLaunch, nseg - first);
    GatherParams P{};
    int64_t n = 0;
    bool any_route = false;
    for (int i = 0; i < cnt; ++i) {
      const chem_segment& a = segs[first + i];
      P.seg[i] = GatherSeg{a.T, a.p, a.Y, a.ld, n, a.status};
      any_route = any_route || a.status;
      n += a.ncells;
    }
    if (n == 0) continue;
    P.nseg = cnt; P.ns = ns; P.n = n;
    unsigned char* ws = nullptr;
    const size_t bT = (size_t)n * 8, bY = (size_t)n * ns * 8, bR = ((size_t)n + 15) & ~(size_t)15;
    CHEM_CUDA_TRY(cudaMallocAsync((void**)&ws, 2 * bT + bY + bR, st));
    P.T = (double*)ws; P.p = (double*)(ws + bT); P.Y = (double*)(ws + 2 * bT);
    int8_t* route = (int8_t*)(ws + 2 * bT + bY);
    P.route = route;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    gather_kernel<<<blocks, 256, 0, st>>>(P);
    cudaError_t le = cudaGetLastError();
    int rc = le == cudaSuccess ? CHEM_OK : cuda_fail(le, "gather_kernel");
    if (!rc)
      rc = chem_surrogate_advance(md, mech, P.T, P.p, P.Y, n, segs[first].dt, n, segs[first].rtol, segs[first].atol,
                                  any_route ? route : nullptr, stream);
    if (!rc) {
      scatter_kernel<<<blocks, 256, 0, st>>>(P);
      le = cudaGetLastError();
      if (le != cudaSuccess) rc = cuda_fail(le, "scatter_kernel");
    }
    cudaError_t fe = cudaFreeAsync(ws, st);
    if (rc) return rc;
    CHEM_CUDA_TRY(fe);
  }
  return CHEM_OK;
}

extern "C" int chem_surrogate_advance(chem_model_t md, chem_mech_t mech, double* T, const double* p,
                                      double* Y, int64_t ld, double dt, int64_t ncells, double rtol,
                                      double atol, int8_t* route_out, chem_stream_t stream) {
  if (!md || !mech) { set_error("NULL model or mechanism"); return CHEM_EINVAL; }
  if (md->ns != mech->ns) { set_error("model and mechanism disagree on the species count"); return CHEM_EINVAL; }
  if (ncells < 0 || ld < ncells || !(rtol > 0.0) || !(atol > 0.0)) { set_error("bad arguments"); return CHEM_EINVAL; }
  if (!(fabs(dt - md->dt) <= 1e-12 * md->dt)) {
    set_error("dt %g differs from the surrogate's training step %g", dt, md->dt);
    return CHEM_EINVAL;
  }
  if (ncells == 0) return CHEM_OK;
  if (!T || !p || !Y) { set_error("NULL state pointer"); return CHEM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  // per-call temporaries from the stream-ordered allocator: net output, box flags, fallback list
  const size_t b_ynet = (size_t)ncells * md->ns * 4, b_box = ((size_t)ncells + 15) & ~(size_t)15;
  const size_t b_idx = (size_t)ncells * 4;
  unsigned char* ws = nullptr;
  CHEM_CUDA_TRY(cudaMallocAsync((void**)&ws, b_ynet + b_box + b_idx + 64, st));
  float* ynet = (float*)ws;
  uint8_t* box = ws + b_ynet;
  int32_t* fb_idx = (int32_t*)(ws + b_ynet + b_box);
  unsigned int* fb_count = (unsigned int*)(ws + b_ynet + b_box + b_idx);
  int* err = (int*)(fb_count + 4);
  CHEM_CUDA_TRY(cudaMemsetAsync(fb_count, 0, 64, st));
  int rc = surrogate_forward(md, T, p, Y, ld, ncells, ynet, nullptr, box, err, st);
  if (!rc) {
    PostParams Q;
    Q.blob = (const unsigned char*)mech->d_blob; Q.lay = mech->lay; Q.Aem = md->d_A; Q.ne = md->ne;
    Q.T = T; Q.p = p; Q.Y = Y; Q.ld = ld; Q.ncells = ncells; Q.ynet = ynet; Q.outbox = box;
    Q.route = route_out; Q.fb_idx = fb_idx; Q.fb_count = fb_count;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = std::min<long long>((ncells + 255) / 256, (long long)sms * 16);
    if (md->ns == 9 && md->ne == 3) surrogate_post_kernel<9, 3><<<(unsigned)blocks, 256, 0, st>>>(Q);
    else surrogate_post_general<<<(unsigned)blocks, 256, 0, st>>>(Q);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) rc = cuda_fail(le, "surrogate_post_kernel");
  }
  if (!rc)
    rc = launch_advance_counted(mech, T, p, Y, ld, dt, ncells, fb_count, rtol, atol, fb_idx, st);
  cudaError_t fe = cudaFreeAsync(ws, st);
  if (rc) return rc;
  CHEM_CUDA_TRY(fe);
  return CHEM_OK;
}
