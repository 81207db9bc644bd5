// Training of the BF16 MLP surrogate on the GPU (§2: the paper's networks use GELU and are
// trained with Adam).  Every product runs on the tcgen05 GEMM (gemm.cu); the rest are small
// elementwise / reduction kernels here.
//
// Layer l maps in_pad[l] -> out_pad[l] features; training pads the input to 128 columns, the
// output layer to 128 rows and every hidden width to at least 128 (a multiple of 8) so that every
// GEMM dimension is at least one 128-wide tile (padding is zero and stays zero: its gradients
// vanish).  The hidden widths are the caller's: 4 x 512 for the single network, 1600/800/400 for
// the paper's per-species networks.  Per step, with batch B:
//   forward   Z_l = A_l W_l^T + b_l (FP32), A_{l+1} = bf16(GELU(Z_l))
//   loss      L = mean over B x n_out of (Z_4 - target)^2,  dZ_4 = 2 (Z_4 - target) / (B n_out)
//   backward  dW_l = dZ_l^T A_l,  db_l = sum_b dZ_l,  dA_{l-1} = dZ_l W_l,
//             dZ_{l-1} = dA_{l-1} * GELU'(Z_{l-1})
//   Adam      FP32 master weights with bias correction (Kingma & Ba), then BF16 copies of W and
//             W^T for the next step's products.
// The first layer is compensated as in the inference kernel: an input row holds
// [x_hi | x_lo | x_hi | 0] (n_in columns each) and the BF16 copy of W_1 holds
// [W_hi | W_hi | W_lo | 0], so one product yields W_hi x_hi + W_hi x_lo + W_lo x_hi.  Its weight
// gradient with respect to the FP32 master W_1 is dZ^T (x_hi + x_lo): the sum of the first two
// column blocks of the product's gradient.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "chem_internal.h"

namespace chem {
int gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
              const float* bias, int M, int N, int K, int* err, cudaStream_t stream);
int gemm_bf16_gelu2(const void* A, int64_t lda, const void* B, int64_t ldb, float* Cz, void* Cb, int64_t ldc,
                    const float* bias, int M, int N, int K, int* err, cudaStream_t stream);
int gemm_bf16_splitk(const void* A, int64_t lda, const void* B, int64_t ldb, float* Cparts, int64_t ldc,
                     int64_t split_stride, int splits, int M, int N, int K, int* err, cudaStream_t stream);
}

using namespace chem;

namespace {

constexpr int HID = 512;
constexpr int PADIO = 128;
constexpr int MAXL = 8;          // layers at most (hidden layers + output)

__device__ __forceinline__ float gelu_grad(float v) {
  return 0.5f * (1.0f + erff(v * 0.70710678118654752f)) + v * 0.3989422804014327f * expf(-0.5f * v * v);
}

__global__ void k_gelu_bwd(const float* dA, const float* Z, float* dZf, __nv_bfloat16* dZb, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = dA[i] * gelu_grad(Z[i]);
    dZf[i] = g;
    dZb[i] = __float2bfloat16_rn(g);
  }
}

// out, dZ: [B x ld] (ld = 128); target: [B x nout]
__global__ void k_mse_grad(const float* out, const float* target, float* dZf, __nv_bfloat16* dZb, double* loss,
                           int B, int nout, int ld) {
  double part = 0.0;
  const float scale = 2.0f / ((float)B * (float)nout);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B * ld;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / ld), c = (int)(i % ld);
    float g = 0.0f;
    if (c < nout) {
      const float d = out[i] - target[(int64_t)b * nout + c];
      part += (double)d * d;
      g = scale * d;
    }
    dZf[i] = g;
    dZb[i] = __float2bfloat16_rn(g);
  }
  // one atomic per block: the warps' sums through shared memory
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (warp == 0) {
    part = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0 && loss) atomicAdd(loss, part / ((double)B * nout));
  }
}

// several BF16 transposes in one launch: blockIdx.z selects the job (out[c * R + r] = in[r * C + c])
struct TransposeJob {
  const __nv_bfloat16* in;
  __nv_bfloat16* out;
  int R, C;
};
struct TransposeSet {
  TransposeJob j[MAXL];
  int n;
};

__global__ void k_transpose_set(const __grid_constant__ TransposeSet S) {
  if ((int)blockIdx.z >= S.n) return;
  const TransposeJob& J = S.j[blockIdx.z];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  if (r0 >= J.R || c0 >= J.C) return;                // the whole block: before the barrier
  __shared__ __nv_bfloat16 t[32][33];
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < J.R && c < J.C) t[i][threadIdx.x] = J.in[(int64_t)r * J.C + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < J.R && c < J.C) J.out[(int64_t)c * J.R + r] = t[threadIdx.x][i];
  }
}

void launch_transposes(const TransposeSet& S, cudaStream_t st) {
  int gx = 1, gy = 1;
  for (int k = 0; k < S.n; ++k) {
    gx = std::max(gx, (S.j[k].C + 31) / 32);
    gy = std::max(gy, (S.j[k].R + 31) / 32);
  }
  k_transpose_set<<<dim3(gx, gy, S.n), dim3(32, 8), 0, st>>>(S);
}

// column sums of a [R x C] FP32 matrix, in two deterministic passes spread over the whole GPU:
// block (x, y) sums rows [y * kColRows, ...) of 32 columns (8 thread rows, FP32, then the 8
// partials in FP64) into part[y][c]; k_colsum_finish adds the row-block partials of a column.
constexpr int kColRows = 64;
__global__ void k_colsum_part(const float* A, double* part, int R, int C) {
  __shared__ double red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int r0 = blockIdx.y * kColRows;
  float acc = 0.0f;
  if (c < C)
    for (int r = r0 + threadIdx.y; r < min(R, r0 + kColRows); r += 8) acc += A[(int64_t)r * C + c];
  red[threadIdx.y][threadIdx.x] = (double)acc;
  __syncthreads();
  if (threadIdx.y == 0 && c < C) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
    part[(int64_t)blockIdx.y * C + c] = t;
  }
}

// out[i] = sum over s of parts[s * stride + i], in the order s = 0, 1, ...: the split-K partial
// products of a weight gradient added deterministically
__global__ void k_sum_parts(const float* parts, float* out, int64_t n, int splits, int64_t stride) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float v = parts[i];
    for (int s = 1; s < splits; ++s) v += parts[s * stride + i];
    out[i] = v;
  }
}

// one warp per column: the lanes sum strided partials, then a shuffle reduction
__global__ void k_colsum_finish(const double* part, float* s, int nparts, int C) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= C) return;                                // whole warps leave together
  double t = 0.0;
  for (int i = lane; i < nparts; i += 32) t += part[(int64_t)i * C + c];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) s[c] = (float)t;
}

// Adam on a [rows x cols] parameter block (cols = 1 for biases); writes the BF16 copy of W if given
// (its transpose follows by the tiled k_transpose)
// Adam over every parameter block of the network in one launch: block b of the grid serves the
// segment whose first block is the last one <= b; each segment is one weight matrix or bias
// vector (W, its gradient G, moments m and v; Wb: the BF16 copy of W to write, or null).
struct AdamSeg {
  float* W;
  const float* G;
  float* m;
  float* v;
  __nv_bfloat16* Wb;
  int64_t n;
  int block0;
};
struct AdamSet {
  AdamSeg s[2 * MAXL];
  int n;
};

__global__ void k_adam_set(const __grid_constant__ AdamSet S, const float* coef, float b1, float b2, float eps) {
  int k = 0;
  while (k + 1 < S.n && S.s[k + 1].block0 <= (int)blockIdx.x) ++k;
  const AdamSeg& q = S.s[k];
  const int nb = (k + 1 < S.n ? S.s[k + 1].block0 : (int)gridDim.x) - q.block0;
  const float lr = coef[0], c1 = coef[1], c2 = coef[2];
  for (int64_t i = (int64_t)(blockIdx.x - q.block0) * blockDim.x + threadIdx.x; i < q.n;
       i += (int64_t)nb * blockDim.x) {
    const float g = q.G[i];
    const float mi = b1 * q.m[i] + (1.0f - b1) * g;
    const float vi = b2 * q.v[i] + (1.0f - b2) * g * g;
    q.m[i] = mi;
    q.v[i] = vi;
    const float w = q.W[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    q.W[i] = w;
    if (q.Wb) q.Wb[i] = __float2bfloat16_rn(w);
  }
}

// One Adam step's scalars on the device: step += 1, coef = {lr, 1 - b1^step, 1 - b2^step}, with lr
// from lr_dev when given (a captured training step reads its learning rate from device memory)
__global__ void k_adam_prep(int64_t* step, float* coef, const float* lr_dev, float lr, float b1, float b2) {
  const int64_t s = *step + 1;
  *step = s;
  coef[0] = lr_dev ? *lr_dev : lr;
  coef[1] = (float)(1.0 - pow((double)b1, (double)s));
  coef[2] = (float)(1.0 - pow((double)b2, (double)s));
}

// compensated BF16 copy of the first layer: Wb row = [W_hi | W_hi | W_lo | 0] from master W[:, :nin]
__global__ void k_split_bf16(const float* W, __nv_bfloat16* Wb, int rows, int ld, int nin) {
  const int64_t n = (int64_t)rows * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / ld), c = (int)(i % ld);
    float v = 0.0f;
    if (c < 3 * nin) {
      const float w = W[(int64_t)r * ld + c % nin];
      const float wh = __bfloat162float(__float2bfloat16_rn(w));
      v = c < 2 * nin ? wh : w - wh;
    }
    Wb[i] = __float2bfloat16_rn(v);
  }
}

// fold the first layer's block gradient into the master's columns: dW[:, c] += dW[:, nin + c]
// for c < nin, zero elsewhere (one thread per row: the row is read before it is written)
__global__ void k_fold_split_grad(float* dW, int rows, int ld, int nin) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float* row = dW + (int64_t)r * ld;
  for (int c = 0; c < nin; ++c) row[c] += row[nin + c];
  for (int c = nin; c < ld; ++c) row[c] = 0.0f;
}

__global__ void k_to_bf16(const float* W, __nv_bfloat16* Wb, __nv_bfloat16* Wt, int rows, int cols) {
  const int64_t n = (int64_t)rows * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const __nv_bfloat16 wb = __float2bfloat16_rn(W[i]);
    Wb[i] = wb;
    const int r = (int)(i / cols), c = (int)(i % cols);
    Wt[(int64_t)c * rows + r] = wb;
  }
}

// dst[r * ld + c] = scale * src[r * cols + c] for the real block of a padded gradient buffer
// (the padding of dst keeps its zeros)
__global__ void k_unpack_scaled(const float* src, float* dst, int rows, int cols, int ld, float scale) {
  const int64_t n = (int64_t)rows * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i % cols);
    dst[(int64_t)r * ld + c] = scale * src[i];
  }
}

// ---- training data: raw features and targets, statistics, normalisation ----------------
__global__ void k_train_features(const double* T0, const double* p, const double* Y0, const double* Y1,
                                 int64_t ld, int64_t n, int ns, float* x, float* t) {
  const int nin = ns + 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i * nin + 0] = (float)T0[i];
    x[i * nin + 1] = (float)log(p[i]);
    for (int k = 0; k < ns; ++k) {
      // the increment is formed in FP64: an FP32 difference of two Box-Cox values near -1/lambda
      // is rounding noise for a species whose mass fraction barely moves over dt
      const double y0 = fmax(Y0[(int64_t)k * ld + i], 0.0);
      const double y1 = fmax(Y1[(int64_t)k * ld + i], 0.0);
      const double b0 = (pow(y0, 0.1) - 1.0) / 0.1;
      const double b1 = (pow(y1, 0.1) - 1.0) / 0.1;
      x[i * nin + 2 + k] = (float)b0;
      t[i * ns + k] = (float)(b1 - b0);
    }
  }
}

// per-column sum, sum of squares, min and max of a [n x c] FP32 matrix (c <= 64)
__global__ void k_col_stats(const float* A, int64_t n, int c, double* acc /*[4][c]*/) {
  __shared__ double s1[64], s2[64], mn[64], mx[64];
  for (int j = threadIdx.x; j < c; j += blockDim.x) { s1[j] = 0; s2[j] = 0; mn[j] = 1e300; mx[j] = -1e300; }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * c; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % c);
    const double v = A[i];
    atomicAdd(&s1[j], v);
    atomicAdd(&s2[j], v * v);
    // min / max through CAS on the bit patterns of doubles
    unsigned long long* pm = (unsigned long long*)&mn[j];
    unsigned long long old = *pm, assumed;
    while (v < __longlong_as_double(old)) {
      assumed = old;
      old = atomicCAS(pm, assumed, __double_as_longlong(v));
      if (old == assumed) break;
    }
    unsigned long long* px = (unsigned long long*)&mx[j];
    old = *px;
    while (v > __longlong_as_double(old)) {
      assumed = old;
      old = atomicCAS(px, assumed, __double_as_longlong(v));
      if (old == assumed) break;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < c; j += blockDim.x) {
    atomicAdd(&acc[j], s1[j]);
    atomicAdd(&acc[c + j], s2[j]);
    unsigned long long* pm = (unsigned long long*)&acc[2 * c + j];
    unsigned long long old = *pm, assumed;
    while (mn[j] < __longlong_as_double(old)) {
      assumed = old;
      old = atomicCAS(pm, assumed, __double_as_longlong(mn[j]));
      if (old == assumed) break;
    }
    unsigned long long* px = (unsigned long long*)&acc[3 * c + j];
    old = *px;
    while (mx[j] > __longlong_as_double(old)) {
      assumed = old;
      old = atomicCAS(px, assumed, __double_as_longlong(mx[j]));
      if (old == assumed) break;
    }
  }
}

__global__ void k_init_stats(double* acc, int c) {
  const int j = threadIdx.x;
  if (j < c) { acc[j] = 0; acc[c + j] = 0; acc[2 * c + j] = 1e300; acc[3 * c + j] = -1e300; }
}

// v = (x - mean) / std;  X[i, :] = [bf16(v_hi) | bf16(v - v_hi) | bf16(v_hi) | 0] (c columns each,
// zero up to ldx);  T[i, :] = (t - tmean) / tstd
__global__ void k_normalize(const float* x, int64_t n, int c, const float* mean, const float* sd,
                            __nv_bfloat16* X, int ldx, const float* t, int ct, const float* tmean,
                            const float* tsd, float* Tn) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int j = 0; j < ldx; ++j) {
      float o = 0.0f;
      if (j < 3 * c) {
        const int jj = j % c;
        const float v = (x[i * c + jj] - mean[jj]) / sd[jj];
        const float vh = __bfloat162float(__float2bfloat16_rn(v));
        o = (j >= c && j < 2 * c) ? v - vh : vh;
      }
      X[i * ldx + j] = __float2bfloat16_rn(o);
    }
    if (t)
      for (int j = 0; j < ct; ++j) Tn[i * ct + j] = (t[i * ct + j] - tmean[j]) / tsd[j];
  }
}

inline unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace

struct chem_trainer_s {
  int nin, nout, B, nl;
  int real_in[MAXL], real_out[MAXL], in_pad[MAXL], out_pad[MAXL];
  float *W[MAXL], *b[MAXL], *mW[MAXL], *vW[MAXL], *mb[MAXL], *vb[MAXL], *dW[MAXL], *db[MAXL];
  __nv_bfloat16 *Wb[MAXL], *Wt[MAXL];
  float* Z[MAXL];                  // pre-activations [B x out_pad]
  __nv_bfloat16* A[MAXL];          // A[0] = caller's input, A[l] = bf16(GELU(Z[l-1]))
  float *dA, *dZf;
  float* dWparts;                  // split-K partials of the weight gradients (null: no layer splits)
  int splitsW[MAXL];               // K splits of each layer's weight-gradient product
  double* colpart;                 // row-block partial column sums [B / 64 x max width]
  __nv_bfloat16 *dZb, *dZt, *At;
  int* err;
  double* loss;
  int64_t* d_step;                 // Adam steps taken (device: a captured step advances it)
  float* d_coef;                   // the current step's lr, 1 - b1^step, 1 - b2^step
  std::vector<void*> allocs;
};

static int tr_alloc(chem_trainer_s* t, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(trainer)");
  t->allocs.push_back(*p);
  CHEM_CUDA_TRY(cudaMemset(*p, 0, bytes));
  return CHEM_OK;
}

extern "C" int chem_mlp_trainer_free(chem_trainer_t t) {
  if (!t) { set_error("NULL trainer"); return CHEM_EINVAL; }
  for (void* p : t->allocs) cudaFree(p);
  delete t;
  return CHEM_OK;
}

extern "C" int chem_mlp_trainer_create(int n_in, int n_out, int batch, const float* const* W_init,
                                       const float* const* b_init, uint64_t seed, chem_trainer_t* out) {
  const int hidden[4] = {HID, HID, HID, HID};
  return chem_mlp_trainer_create_layers(n_in, n_out, 4, hidden, batch, W_init, b_init, seed, out);
}

extern "C" int chem_mlp_trainer_create_layers(int n_in, int n_out, int n_hidden, const int* hidden, int batch,
                                              const float* const* W_init, const float* const* b_init,
                                              uint64_t seed, chem_trainer_t* out) {
  if (!out || n_in < 1 || 3 * n_in > PADIO || n_out < 1 || n_out > PADIO || batch < 128 || batch % 128 ||
      n_hidden < 1 || n_hidden + 1 > MAXL || !hidden) {
    set_error("trainer: n_in in [1, 42], n_out in [1, 128], 1..%d hidden layers, batch a positive "
              "multiple of 128 required", MAXL - 1);
    return CHEM_EINVAL;
  }
  for (int h = 0; h < n_hidden; ++h)
    if (hidden[h] < 1 || hidden[h] > 8192) { set_error("trainer: hidden width %d out of range", hidden[h]); return CHEM_EINVAL; }
  *out = nullptr;
  chem_trainer_s* t = new chem_trainer_s();
  t->nin = n_in; t->nout = n_out; t->B = batch; t->nl = n_hidden + 1;
  const int NL = t->nl;
  auto pad = [](int w) { return std::max(128, (w + 7) / 8 * 8); };
  int ins[MAXL], outs[MAXL];
  for (int l = 0; l < NL; ++l) {
    t->real_in[l] = l == 0 ? n_in : hidden[l - 1];
    t->real_out[l] = l == NL - 1 ? n_out : hidden[l];
    ins[l] = l == 0 ? PADIO : pad(hidden[l - 1]);
    outs[l] = l == NL - 1 ? PADIO : pad(hidden[l]);
  }
  const int* real_in = t->real_in;
  const int* real_out = t->real_out;
  int maxw = PADIO;
  for (int l = 0; l < NL; ++l) maxw = std::max(maxw, std::max(ins[l], outs[l]));
  int rc = CHEM_OK;
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.0f, 1.0f);
  for (int l = 0; l < NL && !rc; ++l) {
    t->in_pad[l] = ins[l];
    t->out_pad[l] = outs[l];
    const size_t nw = (size_t)ins[l] * outs[l];
    void* p;
    if ((rc = tr_alloc(t, &p, nw * 4))) break; t->W[l] = (float*)p;
    if ((rc = tr_alloc(t, &p, outs[l] * 4))) break; t->b[l] = (float*)p;
    if ((rc = tr_alloc(t, &p, nw * 4))) break; t->mW[l] = (float*)p;
    if ((rc = tr_alloc(t, &p, nw * 4))) break; t->vW[l] = (float*)p;
    if ((rc = tr_alloc(t, &p, outs[l] * 4))) break; t->mb[l] = (float*)p;
    if ((rc = tr_alloc(t, &p, outs[l] * 4))) break; t->vb[l] = (float*)p;
    if ((rc = tr_alloc(t, &p, nw * 4))) break; t->dW[l] = (float*)p;
    if ((rc = tr_alloc(t, &p, outs[l] * 4))) break; t->db[l] = (float*)p;
    if ((rc = tr_alloc(t, &p, nw * 2))) break; t->Wb[l] = (__nv_bfloat16*)p;
    if ((rc = tr_alloc(t, &p, nw * 2))) break; t->Wt[l] = (__nv_bfloat16*)p;
    if ((rc = tr_alloc(t, &p, (size_t)batch * outs[l] * 4))) break; t->Z[l] = (float*)p;
    if (l > 0) {
      if ((rc = tr_alloc(t, &p, (size_t)batch * ins[l] * 2))) break;
      t->A[l] = (__nv_bfloat16*)p;
    }
    // initial weights: caller's, else scaled Gaussian (1/sqrt(fan_in)); padding stays zero
    std::vector<float> hw(nw, 0.0f), hb(outs[l], 0.0f);
    const float sc = 1.0f / sqrtf((float)real_in[l]);
    for (int o = 0; o < real_out[l]; ++o) {
      for (int i = 0; i < real_in[l]; ++i)
        hw[(size_t)o * ins[l] + i] = W_init && W_init[l] ? W_init[l][(size_t)o * real_in[l] + i] : sc * nd(rng);
      hb[o] = b_init && b_init[l] ? b_init[l][o] : 0.0f;
    }
    if (cudaMemcpy(t->W[l], hw.data(), nw * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t->b[l], hb.data(), outs[l] * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "cudaMemcpy(trainer)");
      break;
    }
    if (l == 0) k_split_bf16<<<grid_for(nw), 256>>>(t->W[0], t->Wb[0], outs[0], ins[0], n_in);
    else k_to_bf16<<<grid_for(nw), 256>>>(t->W[l], t->Wb[l], t->Wt[l], outs[l], ins[l]);
  }
  void* p;
  if (!rc) rc = tr_alloc(t, &p, (size_t)batch * maxw * 4), t->dA = (float*)p;
  // weight gradients dW = dZ^T A have few output tiles and K = batch: split K over the SMs (a
  // power of two dividing the 64-wide K steps, splits x tiles at most the SM count) and add the
  // partials in a fixed order
  if (!rc) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nk = (batch + 63) / 64;
    size_t parts = 0;
    for (int l = 0; l < NL; ++l) {
      const long long tiles = (long long)((t->out_pad[l] + 127) / 128) * ((t->in_pad[l] + 127) / 128);
      int sp = 1;
      while (nk % (2 * sp) == 0 && tiles * 2 * sp <= sms) sp *= 2;
      t->splitsW[l] = sp;
      if (sp > 1) parts = std::max(parts, (size_t)sp * t->out_pad[l] * t->in_pad[l]);
    }
    t->dWparts = nullptr;
    if (parts) rc = tr_alloc(t, &p, parts * 4), t->dWparts = (float*)p;
  }
  if (!rc) rc = tr_alloc(t, &p, (size_t)batch * maxw * 4), t->dZf = (float*)p;
  if (!rc) rc = tr_alloc(t, &p, (size_t)batch * maxw * 2), t->dZb = (__nv_bfloat16*)p;
  if (!rc) rc = tr_alloc(t, &p, (size_t)batch * maxw * 2), t->dZt = (__nv_bfloat16*)p;
  if (!rc) rc = tr_alloc(t, &p, (size_t)batch * maxw * 2), t->At = (__nv_bfloat16*)p;
  if (!rc) rc = tr_alloc(t, &p, (size_t)((batch + kColRows - 1) / kColRows) * maxw * 8), t->colpart = (double*)p;
  if (!rc) rc = tr_alloc(t, &p, 16), t->err = (int*)p;
  if (!rc) rc = tr_alloc(t, &p, 16), t->loss = (double*)p;
  if (!rc) rc = tr_alloc(t, &p, 16), t->d_step = (int64_t*)p;
  if (!rc) rc = tr_alloc(t, &p, 16), t->d_coef = (float*)p;
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "trainer init");
  if (rc) { chem_mlp_trainer_free(t); return rc; }
  *out = t;
  return CHEM_OK;
}

extern "C" int chem_mlp_forward(chem_trainer_t t, const void* X, float* out, chem_stream_t stream) {
  if (!t || !X) { set_error("NULL argument"); return CHEM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  t->A[0] = (__nv_bfloat16*)X;
  const int B = t->B, NL = t->nl;
  for (int l = 0; l < NL; ++l) {
    // hidden layers keep the pre-activation Z (for the backward pass) and write the next
    // layer's BF16 input GELU(Z) from the same epilogue
    const int rc = l < NL - 1
                       ? gemm_bf16_gelu2(t->A[l], t->in_pad[l], t->Wb[l], t->in_pad[l], t->Z[l], t->A[l + 1],
                                         t->out_pad[l], t->b[l], B, t->out_pad[l], t->in_pad[l], t->err, st)
                       : gemm_bf16(t->A[l], t->in_pad[l], t->Wb[l], t->in_pad[l], t->Z[l], t->out_pad[l], t->b[l],
                                   B, t->out_pad[l], t->in_pad[l], t->err, st);
    if (rc) return rc;
  }
  if (out) {
    CHEM_CUDA_TRY(cudaMemcpy2DAsync(out, t->nout * 4, t->Z[NL - 1], PADIO * 4, t->nout * 4, B,
                                    cudaMemcpyDeviceToDevice, st));
  }
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_mlp_backward(chem_trainer_t t, const float* target, double* loss_out,
                                 chem_stream_t stream) {
  if (!t || !target) { set_error("NULL argument"); return CHEM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const int B = t->B, NL = t->nl;
  CHEM_CUDA_TRY(cudaMemsetAsync(t->loss, 0, sizeof(double), st));
  k_mse_grad<<<std::min(grid_for((int64_t)B * PADIO), 1024u), 256, 0, st>>>(t->Z[NL - 1], target, t->dZf, t->dZb,
                                                                         t->loss, B, t->nout, PADIO);
  for (int l = NL - 1; l >= 0; --l) {
    const int nout = t->out_pad[l], nin = t->in_pad[l];
    // dZ^T and A^T (batch contiguous) for the weight gradient
    {
      TransposeSet T{};
      T.j[0] = TransposeJob{t->dZb, t->dZt, B, nout};
      T.j[1] = TransposeJob{t->A[l], t->At, B, nin};
      T.n = 2;
      launch_transposes(T, st);
    }
    int rc;
    if (t->splitsW[l] > 1) {
      const int64_t n = (int64_t)nout * nin;
      rc = gemm_bf16_splitk(t->dZt, B, t->At, B, t->dWparts, nin, n, t->splitsW[l], nout, nin, B, t->err, st);
      if (rc) return rc;
      k_sum_parts<<<grid_for(n), 256, 0, st>>>(t->dWparts, t->dW[l], n, t->splitsW[l], n);
    } else {
      rc = gemm_bf16(t->dZt, B, t->At, B, t->dW[l], nin, nullptr, nout, nin, B, t->err, st);
      if (rc) return rc;
    }
    if (l == 0) k_fold_split_grad<<<(nout + 127) / 128, 128, 0, st>>>(t->dW[0], nout, nin, t->nin);
    {
      const int nparts = (B + kColRows - 1) / kColRows;
      k_colsum_part<<<dim3((nout + 31) / 32, nparts), dim3(32, 8), 0, st>>>(t->dZf, t->colpart, B, nout);
      k_colsum_finish<<<(nout + 7) / 8, 256, 0, st>>>(t->colpart, t->db[l], nparts, nout);
    }
    if (l > 0) {
      rc = gemm_bf16(t->dZb, nout, t->Wt[l], nout, t->dA, nin, nullptr, B, nin, nout, t->err, st);
      if (rc) return rc;
      const int64_t n = (int64_t)B * nin;
      k_gelu_bwd<<<grid_for(n), 256, 0, st>>>(t->dA, t->Z[l - 1], t->dZf, t->dZb, n);
    }
  }
  if (loss_out) CHEM_CUDA_TRY(cudaMemcpyAsync(loss_out, t->loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

static int adam_step(chem_trainer_t t, const float* lr_dev, float lr, float beta1, float beta2, float eps,
                     cudaStream_t st) {
  k_adam_prep<<<1, 1, 0, st>>>(t->d_step, t->d_coef, lr_dev, lr, beta1, beta2);
  // every weight matrix and bias vector in one launch (BF16 copies of the hidden weights written
  // on the way), then the transposed copies the backward pass multiplies with and the first
  // layer's split copy
  AdamSet A{};
  int blocks = 0;
  auto add = [&](float* W, const float* G, float* m, float* v, __nv_bfloat16* Wb, int64_t n) {
    A.s[A.n] = AdamSeg{W, G, m, v, Wb, n, blocks};
    blocks += (int)std::min<int64_t>((n + 255) / 256, 1024);
    ++A.n;
  };
  for (int l = 0; l < t->nl; ++l) {
    const int r = t->out_pad[l], c = t->in_pad[l];
    add(t->W[l], t->dW[l], t->mW[l], t->vW[l], l == 0 ? nullptr : t->Wb[l], (int64_t)r * c);
    add(t->b[l], t->db[l], t->mb[l], t->vb[l], nullptr, r);
  }
  k_adam_set<<<blocks, 256, 0, st>>>(A, t->d_coef, beta1, beta2, eps);
  TransposeSet T{};
  for (int l = 1; l < t->nl; ++l) T.j[T.n++] = TransposeJob{t->Wb[l], t->Wt[l], t->out_pad[l], t->in_pad[l]};
  if (T.n) launch_transposes(T, st);
  k_split_bf16<<<grid_for((int64_t)t->out_pad[0] * t->in_pad[0]), 256, 0, st>>>(t->W[0], t->Wb[0], t->out_pad[0],
                                                                                 t->in_pad[0], t->nin);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_mlp_adam_step(chem_trainer_t t, float lr, float beta1, float beta2, float eps,
                                  chem_stream_t stream) {
  if (!t || !(lr > 0.0f)) { set_error("bad Adam arguments"); return CHEM_EINVAL; }
  return adam_step(t, nullptr, lr, beta1, beta2, eps, (cudaStream_t)stream);
}

extern "C" int chem_mlp_adam_step_dev(chem_trainer_t t, const float* lr, float beta1, float beta2, float eps,
                                      chem_stream_t stream) {
  if (!t || !lr) { set_error("NULL argument"); return CHEM_EINVAL; }
  return adam_step(t, lr, 0.0f, beta1, beta2, eps, (cudaStream_t)stream);
}

// copy parameters (which = 0) or gradients (which = 1) of the real (unpadded) layers to host
extern "C" int chem_mlp_trainer_get(chem_trainer_t t, int which, float* const* W, float* const* b) {
  if (!t || !W || !b) { set_error("NULL argument"); return CHEM_EINVAL; }
  CHEM_CUDA_TRY(cudaDeviceSynchronize());
  const int* real_in = t->real_in;
  const int* real_out = t->real_out;
  for (int l = 0; l < t->nl; ++l) {
    const float* sw = which ? t->dW[l] : t->W[l];
    const float* sb = which ? t->db[l] : t->b[l];
    if (W[l])
      CHEM_CUDA_TRY(cudaMemcpy2D(W[l], real_in[l] * 4, sw, t->in_pad[l] * 4, real_in[l] * 4, real_out[l],
                                 cudaMemcpyDeviceToHost));
    if (b[l]) CHEM_CUDA_TRY(cudaMemcpy(b[l], sb, real_out[l] * 4, cudaMemcpyDeviceToHost));
  }
  int herr = 0;
  CHEM_CUDA_TRY(cudaMemcpy(&herr, t->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) { set_error("a GEMM pipeline wait timed out during training"); return CHEM_ECUDA; }
  return CHEM_OK;
}

// ---- data-parallel gradient exchange ---------------------------------------------------
// Flat layout of the real (unpadded) gradients: for each layer l in order, dW_l [real_out x
// real_in] row-major, then db_l [real_out].
static int64_t flat_count(const chem_trainer_s* t) {
  int64_t n = 0;
  for (int l = 0; l < t->nl; ++l) n += (int64_t)t->real_out[l] * t->real_in[l] + t->real_out[l];
  return n;
}

extern "C" int chem_mlp_grad_count(chem_trainer_t t, int64_t* n) {
  if (!t || !n) { set_error("NULL argument"); return CHEM_EINVAL; }
  *n = flat_count(t);
  return CHEM_OK;
}

extern "C" int chem_mlp_grad_pack(chem_trainer_t t, float* flat, chem_stream_t stream) {
  if (!t || !flat) { set_error("NULL argument"); return CHEM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  int64_t o = 0;
  for (int l = 0; l < t->nl; ++l) {
    const int ro = t->real_out[l], ri = t->real_in[l];
    CHEM_CUDA_TRY(cudaMemcpy2DAsync(flat + o, (size_t)ri * 4, t->dW[l], (size_t)t->in_pad[l] * 4, (size_t)ri * 4, ro,
                                    cudaMemcpyDeviceToDevice, st));
    o += (int64_t)ro * ri;
    CHEM_CUDA_TRY(cudaMemcpyAsync(flat + o, t->db[l], (size_t)ro * 4, cudaMemcpyDeviceToDevice, st));
    o += ro;
  }
  return CHEM_OK;
}

extern "C" int chem_mlp_grad_unpack(chem_trainer_t t, const float* flat, float scale, chem_stream_t stream) {
  if (!t || !flat || !std::isfinite(scale)) { set_error("bad arguments"); return CHEM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  int64_t o = 0;
  for (int l = 0; l < t->nl; ++l) {
    const int ro = t->real_out[l], ri = t->real_in[l];
    k_unpack_scaled<<<grid_for((int64_t)ro * ri), 256, 0, st>>>(flat + o, t->dW[l], ro, ri, t->in_pad[l], scale);
    o += (int64_t)ro * ri;
    k_unpack_scaled<<<grid_for(ro), 256, 0, st>>>(flat + o, t->db[l], ro, 1, 1, scale);
    o += ro;
  }
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

// ---- checkpoint / resume ---------------------------------------------------------------
// CHEMTRN1 file: magic, int32 nl, n_in, n_out, real_in[nl], real_out[nl], int64 Adam step,
// then per layer (real shapes, FP32): W, b, first moments of W and b, second moments of W and b.
namespace {
constexpr char kTrnMagic[8] = {'C', 'H', 'E', 'M', 'T', 'R', 'N', '1'};

// one [rows x cols] block of a padded device buffer (leading dimension ld) to / from host
int block_io(float* dev, int rows, int cols, int ld, std::vector<float>& host, bool to_host) {
  host.resize((size_t)rows * cols);
  if (to_host)
    CHEM_CUDA_TRY(cudaMemcpy2D(host.data(), (size_t)cols * 4, dev, (size_t)ld * 4, (size_t)cols * 4, rows,
                               cudaMemcpyDeviceToHost));
  else
    CHEM_CUDA_TRY(cudaMemcpy2D(dev, (size_t)ld * 4, host.data(), (size_t)cols * 4, (size_t)cols * 4, rows,
                               cudaMemcpyHostToDevice));
  return CHEM_OK;
}
}  // namespace

extern "C" int chem_mlp_trainer_save(chem_trainer_t t, const char* path) {
  if (!t || !path) { set_error("NULL argument"); return CHEM_EINVAL; }
  CHEM_CUDA_TRY(cudaDeviceSynchronize());
  FILE* f = fopen(path, "wb");
  if (!f) { set_error("cannot open %s for writing", path); return CHEM_ENOTFOUND; }
  bool ok = fwrite(kTrnMagic, 1, 8, f) == 8;
  const int32_t hdr[3] = {t->nl, t->nin, t->nout};
  ok = ok && fwrite(hdr, 4, 3, f) == 3;
  ok = ok && fwrite(t->real_in, 4, t->nl, f) == (size_t)t->nl && fwrite(t->real_out, 4, t->nl, f) == (size_t)t->nl;
  int64_t step = 0;
  if (cudaMemcpy(&step, t->d_step, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
    fclose(f);
    return cuda_fail(cudaGetLastError(), "cudaMemcpy(trainer step)");
  }
  ok = ok && fwrite(&step, 8, 1, f) == 1;
  std::vector<float> h;
  for (int l = 0; l < t->nl && ok; ++l) {
    const int ro = t->real_out[l], ri = t->real_in[l], ld = t->in_pad[l];
    float* blocks[6] = {t->W[l], t->b[l], t->mW[l], t->mb[l], t->vW[l], t->vb[l]};
    for (int k = 0; k < 6 && ok; ++k) {
      const bool w = (k % 2) == 0;
      int rc = block_io(blocks[k], w ? ro : 1, w ? ri : ro, w ? ld : ro, h, true);
      if (rc) { fclose(f); return rc; }
      ok = fwrite(h.data(), 4, h.size(), f) == h.size();
    }
  }
  if (fclose(f) != 0) ok = false;
  if (!ok) { set_error("write error on %s", path); return CHEM_EINVAL; }
  return CHEM_OK;
}

extern "C" int chem_mlp_trainer_load(chem_trainer_t t, const char* path) {
  if (!t || !path) { set_error("NULL argument"); return CHEM_EINVAL; }
  FILE* f = fopen(path, "rb");
  if (!f) { set_error("cannot open %s", path); return CHEM_ENOTFOUND; }
  char magic[8];
  int32_t hdr[3];
  std::vector<int32_t> ri(t->nl), ro(t->nl);
  int64_t step = 0;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kTrnMagic, 8) == 0 && fread(hdr, 4, 3, f) == 3 &&
            hdr[0] == t->nl && hdr[1] == t->nin && hdr[2] == t->nout &&
            fread(ri.data(), 4, t->nl, f) == (size_t)t->nl && fread(ro.data(), 4, t->nl, f) == (size_t)t->nl;
  for (int l = 0; l < t->nl && ok; ++l) ok = ri[l] == t->real_in[l] && ro[l] == t->real_out[l];
  ok = ok && fread(&step, 8, 1, f) == 1 && step >= 0;
  if (!ok) { fclose(f); set_error("%s: not a trainer state of this network's shape", path); return CHEM_EINVAL; }
  // read everything first: a truncated file leaves the trainer unchanged
  std::vector<std::vector<float>> blocks((size_t)t->nl * 6);
  for (int l = 0; l < t->nl && ok; ++l)
    for (int k = 0; k < 6 && ok; ++k) {
      std::vector<float>& h = blocks[(size_t)l * 6 + k];
      h.resize(k % 2 == 0 ? (size_t)t->real_out[l] * t->real_in[l] : (size_t)t->real_out[l]);
      ok = fread(h.data(), 4, h.size(), f) == h.size();
    }
  fclose(f);
  if (!ok) { set_error("%s: truncated trainer state", path); return CHEM_EINVAL; }
  CHEM_CUDA_TRY(cudaDeviceSynchronize());
  for (int l = 0; l < t->nl; ++l) {
    const int r = t->real_out[l], c = t->real_in[l], ld = t->in_pad[l];
    float* dst[6] = {t->W[l], t->b[l], t->mW[l], t->mb[l], t->vW[l], t->vb[l]};
    for (int k = 0; k < 6; ++k) {
      const bool w = (k % 2) == 0;
      int rc = block_io(dst[k], w ? r : 1, w ? c : r, w ? ld : r, blocks[(size_t)l * 6 + k], false);
      if (rc) return rc;
    }
    const int64_t nw = (int64_t)t->out_pad[l] * t->in_pad[l];
    if (l == 0) k_split_bf16<<<grid_for(nw), 256>>>(t->W[0], t->Wb[0], t->out_pad[0], t->in_pad[0], t->nin);
    else k_to_bf16<<<grid_for(nw), 256>>>(t->W[l], t->Wb[l], t->Wt[l], t->out_pad[l], t->in_pad[l]);
  }
  CHEM_CUDA_TRY(cudaMemcpy(t->d_step, &step, 8, cudaMemcpyHostToDevice));
  CHEM_CUDA_TRY(cudaDeviceSynchronize());
  return CHEM_OK;
}

extern "C" int chem_mlp_trainer_step(chem_trainer_t t, int64_t* step) {
  if (!t || !step) { set_error("NULL argument"); return CHEM_EINVAL; }
  CHEM_CUDA_TRY(cudaMemcpy(step, t->d_step, 8, cudaMemcpyDeviceToHost));
  return CHEM_OK;
}

extern "C" int chem_train_features(const double* T0, const double* p, const double* Y0, const double* Y1,
                                   int64_t ld, int64_t n, int ns, float* x_raw, float* t_raw,
                                   chem_stream_t stream) {
  if (!T0 || !p || !Y0 || !Y1 || !x_raw || !t_raw || n < 0 || ld < n || ns < 1 || ns > 62) {
    set_error("bad arguments");
    return CHEM_EINVAL;
  }
  if (n == 0) return CHEM_OK;
  k_train_features<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(T0, p, Y0, Y1, ld, n, ns, x_raw, t_raw);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_column_stats(const float* A, int64_t n, int c, double* stats, chem_stream_t stream) {
  if (!A || !stats || n < 1 || c < 1 || c > 64) { set_error("bad arguments"); return CHEM_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  k_init_stats<<<1, 64, 0, st>>>(stats, c);
  k_col_stats<<<grid_for(n * c), 256, 0, st>>>(A, n, c, stats);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_train_normalize(const float* x, int64_t n, int c, const float* mean, const float* sd,
                                    void* X, int ldx, const float* t, int ct, const float* tmean,
                                    const float* tsd, float* Tn, chem_stream_t stream) {
  if (!x || !mean || !sd || !X || n < 0 || c < 1 || ldx < 3 * c || (t && (!tmean || !tsd || !Tn))) {
    set_error("bad arguments");
    return CHEM_EINVAL;
  }
  if (n == 0) return CHEM_OK;
  k_normalize<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(x, n, c, mean, sd, (__nv_bfloat16*)X, ldx, t, ct,
                                                             tmean, tsd, Tn);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}
