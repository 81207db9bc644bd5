// The surrogate model object, shared by the single-network path (surrogate.cu: one fused
// tcgen05 kernel for all species) and the per-species path (surrogate_ps.cu: the paper's one
// network per species, §2, run layer by layer on the tcgen05 GEMM).
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "chem_internal.h"

namespace chem {

constexpr int SUR_KIN = 64;            // padded input width of a first layer (one 128-byte K chunk)
constexpr int SUR_MAXNS = 16;          // species supported
constexpr float SUR_BC_LAMBDA = 0.1f;  // Box-Cox exponent of the species features

// one species' network on the device (per-species models)
struct PsNet {
  int species = -1;
  const uint16_t* W1 = nullptr;   // BF16 [h1 x 64]: [W_hi | W_hi | W_lo | 0] (compensated first layer)
  const uint16_t* W2 = nullptr;   // BF16 [h2 x h1]
  const uint16_t* W3 = nullptr;   // BF16 [h3 x h2]
  const uint16_t* w4 = nullptr;   // BF16 [h3] (output row)
  const float *b1 = nullptr, *b2 = nullptr, *b3 = nullptr, *b4 = nullptr;
};

int surrogate_forward_ps(chem_model_s* md, const double* T, const double* p, const double* Y, int64_t ld,
                         int64_t ncells, float* ynet, float* zout, uint8_t* outbox, int* err,
                         cudaStream_t stream);

}  // namespace chem

struct chem_model_s {
  int kind = 0;              // 0: one network for all species; 1: one network per species
  int ns = 0, nin = 0, ne = 0;
  double dt = 0.0;
  int device = 0;
  void* d_w = nullptr;       // all BF16 weights
  void* d_f = nullptr;       // FP32 biases and statistics
  double* d_A = nullptr;     // element mass-fraction matrix
  const float* bias[5] = {};
  const float *xmu = nullptr, *xsd = nullptr, *ymu = nullptr, *ysd = nullptr, *lo = nullptr, *hi = nullptr;
  CUtensorMap tw[5];
  float hbias[4][512];       // host copy of the hidden-layer biases (single network)
  float hstat[7][chem::SUR_MAXNS + 2] = {};   // host copy of the statistics, box and output bias (single network)
  // per-species networks (kind 1)
  int h[3] = {0, 0, 0};
  int nnet = 0;
  chem::PsNet net[chem::SUR_MAXNS];
};
