// The paper's own surrogate variant (§2): one network per species (inert species have none and
// keep their mass fraction), each n_in -> 1600 -> 800 -> 400 -> 1 with GELU, on the same features,
// normalisation and trust box as the single network.
//
// The widths do not fit the fused single-network kernel (a 128 x 1600 BF16 activation tile alone
// is 400 KB), so the networks run layer by layer on the tcgen05 GEMM with its activation epilogue
// (bias, exact-erf GELU and BF16 rounding fused into the accumulator read-back): per chunk of
// 16384 cells, one feature kernel; one grouped GEMM for the first layers of all networks (they
// share the input, so their weights stack into one [nnet h1 x 64] operand); then for every species
// two GEMMs reading its column block of that output and an output dot product; then one
// inverse-transform kernel.  A species' later activations (26 + 13 MB) stay in the 129 MB L2.  The output layer (400 -> 1) is a warp-per-cell dot
// product of BF16 values with FP32 accumulation, the precision of the single network's output MMA.
// Everything after the network (projection, Newton on T, fallback) is shared with the single
// network (surrogate.cu).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "chem_internal.h"
#include "surrogate_model.h"

namespace chem {

int gemm_bf16_act(const void* A, int64_t lda, const void* B, int64_t ldb, void* Cb, int64_t ldc,
                  const float* bias, int gelu, int M, int N, int K, int* err, cudaStream_t stream);

namespace {

// cells per pass of the layer-by-layer schedule: 65536 rows give the GEMMs enough tiles to fill
// the GPU several times over; the stacked first-layer output of a pass is 65536 x (networks x h1)
// BF16 (1.7 GB for eight 1600-wide networks, stream-ordered workspace)
constexpr int64_t kPsChunk = 65536;

struct PsFeatParams {
  const double *T, *p, *Y;
  int64_t ld, nc, M;
  int ns, nin;
  const float *xmu, *xsd, *lo, *hi;
  __nv_bfloat16* X;          // [M x 64]
  uint8_t* outbox;           // [nc]
};

// features of one cell, exactly as the single network's feature warps form them: T, ln p and the
// Box-Cox transformed mass fractions in FP32, z-scored, split into [x_hi | x_lo | x_hi | 0]
__global__ void k_ps_features(const PsFeatParams P) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.M) return;
  float x[SUR_KIN];
#pragma unroll
  for (int i = 0; i < SUR_KIN; ++i) x[i] = 0.0f;
  if (c < P.nc) {
    float f[2 + SUR_MAXNS];
    f[0] = (float)P.T[c];
    f[1] = logf((float)P.p[c]);
    for (int k = 0; k < P.ns; ++k) {
      const float yf = fmaxf((float)P.Y[(int64_t)k * P.ld + c], 0.0f);
      f[2 + k] = (powf(yf, SUR_BC_LAMBDA) - 1.0f) / SUR_BC_LAMBDA;
    }
    bool outside = false;
    for (int i = 0; i < P.nin; ++i) {
      if (!(f[i] >= P.lo[i] && f[i] <= P.hi[i])) outside = true;
      const float v = (f[i] - P.xmu[i]) / P.xsd[i];
      const float vh = __bfloat162float(__float2bfloat16_rn(v));
      x[i] = vh;
      x[P.nin + i] = v - vh;
      x[2 * P.nin + i] = vh;
    }
    P.outbox[c] = outside ? 1 : 0;
  }
  uint4* row = reinterpret_cast<uint4*>(P.X + c * SUR_KIN);
#pragma unroll
  for (int u = 0; u < SUR_KIN / 8; ++u) {
    __nv_bfloat162 q[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) q[j] = __floats2bfloat162_rn(x[8 * u + 2 * j], x[8 * u + 2 * j + 1]);
    row[u] = *reinterpret_cast<uint4*>(q);
  }
}

// output layer: z[c] = sum_i A3[c, i] w4[i] + b4 (BF16 products, FP32 sums), one warp per cell
__global__ void k_ps_out(const __nv_bfloat16* A3, int h3, const __nv_bfloat16* w4, const float* b4, int64_t nc,
                         float* z) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nc) return;
  const __nv_bfloat16* a = A3 + c * h3;
  float acc = 0.0f;
  for (int i = lane; i < h3; i += 32) acc = fmaf(__bfloat162float(a[i]), __bfloat162float(w4[i]), acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) z[c] = acc + b4[0];
}

struct PsInvParams {
  const double* Y;
  int64_t ld, nc, Mp, ldo;
  int ns;
  int8_t net_of[SUR_MAXNS];  // network index of each species, -1: none (the species is unchanged)
  const float *ymu, *ysd;
  const float* z;            // [nnet x Mp]
  float* ynet;               // [ns x ldo], this chunk's columns
  float* zout;               // nullable, same layout
};

// inverse transform: Y' = BC^-1(BC(Y0) + z sd + mu), as the single network's epilogue
__global__ void k_ps_inverse(const PsInvParams P) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.nc) return;
  for (int k = 0; k < P.ns; ++k) {
    const float yf = fmaxf((float)P.Y[(int64_t)k * P.ld + c], 0.0f);
    const float bc0 = (powf(yf, SUR_BC_LAMBDA) - 1.0f) / SUR_BC_LAMBDA;
    const int s = P.net_of[k];
    const float zz = s >= 0 ? P.z[(int64_t)s * P.Mp + c] : 0.0f;
    if (P.zout) P.zout[(int64_t)k * P.ldo + c] = zz;
    const float d = zz * P.ysd[k] + P.ymu[k];
    const float b1 = bc0 + d;
    P.ynet[(int64_t)k * P.ldo + c] = powf(fmaxf(1.0f + SUR_BC_LAMBDA * b1, 0.0f), 1.0f / SUR_BC_LAMBDA);
  }
}

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

int surrogate_forward_ps(chem_model_s* md, const double* T, const double* p, const double* Y, int64_t ld,
                         int64_t ncells, float* ynet, float* zout, uint8_t* outbox, int* err,
                         cudaStream_t st) {
  const int h1 = md->h[0], h2 = md->h[1], h3 = md->h[2];
  const int64_t chunk = std::min<int64_t>(ncells, kPsChunk);
  const int64_t Mp = std::max<int64_t>(chunk, 128);           // a GEMM needs at least one 128-row tile
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const int nnet = std::max(md->nnet, 1), ld1 = nnet * h1;     // A1 holds every network's first layer
  const size_t bX = al((size_t)Mp * SUR_KIN * 2), bA1 = al((size_t)Mp * ld1 * 2), bA2 = al((size_t)Mp * h2 * 2);
  const size_t bA3 = al((size_t)Mp * h3 * 2), bz = al((size_t)std::max(md->nnet, 1) * Mp * 4);
  unsigned char* ws = nullptr;
  CHEM_CUDA_TRY(cudaMallocAsync((void**)&ws, bX + bA1 + bA2 + bA3 + bz, st));
  __nv_bfloat16* X = (__nv_bfloat16*)ws;
  __nv_bfloat16* A1 = (__nv_bfloat16*)(ws + bX);
  __nv_bfloat16* A2 = (__nv_bfloat16*)(ws + bX + bA1);
  __nv_bfloat16* A3 = (__nv_bfloat16*)(ws + bX + bA1 + bA2);
  float* z = (float*)(ws + bX + bA1 + bA2 + bA3);
  PsInvParams Q{};
  Q.ld = ld; Q.Mp = Mp; Q.ldo = ncells; Q.ns = md->ns; Q.ymu = md->ymu; Q.ysd = md->ysd; Q.z = z;
  for (int k = 0; k < SUR_MAXNS; ++k) Q.net_of[k] = -1;
  for (int s = 0; s < md->nnet; ++s) Q.net_of[md->net[s].species] = (int8_t)s;
  int rc = CHEM_OK;
  for (int64_t c0 = 0; c0 < ncells && !rc; c0 += chunk) {
    const int64_t nc = std::min<int64_t>(chunk, ncells - c0);
    const int M = (int)std::max<int64_t>(nc, 128);
    PsFeatParams F;
    F.T = T + c0; F.p = p + c0; F.Y = Y + c0; F.ld = ld; F.nc = nc; F.M = M;
    F.ns = md->ns; F.nin = md->nin; F.xmu = md->xmu; F.xsd = md->xsd; F.lo = md->lo; F.hi = md->hi;
    F.X = X; F.outbox = outbox + c0;
    k_ps_features<<<blocks_for(M, 256), 256, 0, st>>>(F);
    if (md->nnet > 0)   // stacked first layers: net s's weights and biases follow net s - 1's
      rc = gemm_bf16_act(X, SUR_KIN, md->net[0].W1, SUR_KIN, A1, ld1, md->net[0].b1, 1, M, md->nnet * h1, SUR_KIN,
                         err, st);
    for (int s = 0; s < md->nnet && !rc; ++s) {
      const PsNet& n = md->net[s];
      rc = gemm_bf16_act(A1 + (size_t)s * h1, ld1, n.W2, h1, A2, h2, n.b2, 1, M, h2, h1, err, st);
      if (!rc) rc = gemm_bf16_act(A2, h2, n.W3, h2, A3, h3, n.b3, 1, M, h3, h2, err, st);
      if (!rc) k_ps_out<<<blocks_for(nc * 32, 256), 256, 0, st>>>(A3, h3, (const __nv_bfloat16*)n.w4, n.b4, nc,
                                                                  z + (int64_t)s * Mp);
    }
    if (rc) break;
    Q.Y = Y + c0; Q.nc = nc; Q.ynet = ynet + c0; Q.zout = zout ? zout + c0 : nullptr;
    k_ps_inverse<<<blocks_for(nc, 256), 256, 0, st>>>(Q);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) rc = cuda_fail(le, "per-species surrogate kernels");
  }
  cudaError_t fe = cudaFreeAsync(ws, st);
  if (rc) return rc;
  CHEM_CUDA_TRY(fe);
  return CHEM_OK;
}

}  // namespace chem
