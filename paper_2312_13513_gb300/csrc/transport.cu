// Thermophysical and transport properties per cell on sm_103a (the paper's Thermo class, §3.1:
// "Newton's method and high-order temperature polynomials", compute bound).
//
// * chem_mixture_thermo: mixture h and cp from the NASA-7 polynomials (one thread per cell).
// * chem_temperature_from_enthalpy: T from h by Newton on the same polynomials (one thread per
//   cell; |dT| < 1e-9 T within 50 iterations and T in [200, 6000] K, else status 1 and T
//   unchanged).
// * chem_transport_eval: mixture-averaged viscosity (Wilke), conductivity (Mathur-Saxena) and
//   diffusion coefficients D_km = (1 - Y_k) / sum_{j != k} X_j / D_jk from cubic fits in ln T.
//   A group of G threads owns a cell (G = 4 for small mechanisms, 32 for CH4-sized ones): lanes
//   first evaluate the inverse binary diffusion coefficients once per unordered species pair
//   (one exponential each, kept in shared memory), then split the species rows of the Wilke and
//   diffusion sums (ns^2 terms); the per-cell scalars are formed once per group.  Fits, the
//   pair list and the Wilke weight tables stay in global memory behind the read-only cache.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "chem_internal.h"
#include "fastexp.cuh"
#include "thermo.cuh"

using namespace chem;

struct chem_transport_s {
  chem_mech_s* mech = nullptr;
  int ns = 0;
  double* d = nullptr;                 // one device allocation holding the tables below
  const double* mu_poly = nullptr;     // [ns][4]
  const double* lam_poly = nullptr;    // [ns][4]
  const double* diff_poly = nullptr;   // [ns][ns][4]
  const double* invW = nullptr;        // [ns]
  const double* wq = nullptr;          // [ns][ns]: (W_j / W_k)^(1/4) at [j * ns + k]
  const double* cw = nullptr;          // [ns][ns]: (8 (1 + W_k / W_j))^(-1/2) at [k * ns + j]
  const int* pairs = nullptr;          // [ns (ns - 1) / 2]: j | k << 16, j < k, row-major upper triangle
};

namespace {

constexpr double kPatm = 1.01325e6;

__global__ void mixture_thermo_kernel(const unsigned char* blob, MechLayout L, const double* T, const double* Y,
                                      int64_t ld, int64_t n, double* h, double* cp) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    double hh, cc;
    h_cp_mass(blob, L, T[c], Y, ld, c, nullptr, &hh, &cc);
    if (h) h[c] = hh;
    if (cp) cp[c] = cc;
  }
}

__global__ void temperature_from_h_kernel(const unsigned char* blob, MechLayout L, const double* h0,
                                          const double* Y, int64_t ld, int64_t n, double* T, int8_t* status) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const double target = h0[c];
    double Tn = T[c];
    bool conv = false;
    if (isfinite(target) && Tn >= 200.0 && Tn <= 6000.0) {
      for (int it = 0; it < 50; ++it) {
        double hh, cp;
        h_cp_mass(blob, L, Tn, Y, ld, c, nullptr, &hh, &cp);
        const double dT = (hh - target) / cp;
        Tn -= dT;
        if (!(Tn >= 200.0 && Tn <= 6000.0)) break;
        if (fabs(dT) < 1e-9 * Tn) { conv = true; break; }
      }
    }
    if (conv) T[c] = Tn;
    if (status) status[c] = conv ? 0 : 1;
  }
}

template <int G>
struct TGrp {
  int tid, gid;
  unsigned mask;
  __device__ void init() {
    tid = threadIdx.x % G;
    gid = threadIdx.x / G;
    mask = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  }
  __device__ void sync() const { __syncwarp(mask); }
  __device__ double sum(double v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
  }
};

struct TrParams {
  const double *T, *p, *Y;
  int64_t ld, n;
  double *mu, *lam, *Dm;
  const double *mu_poly, *lam_poly, *diff_poly, *invW, *wq, *cw;
  const int* pairs;
  int ns;
};

// index of the unordered pair (j, k), j < k, in the row-major upper triangle
__device__ __forceinline__ int pair_index(int j, int k, int ns) { return j * ns - (j * (j + 1)) / 2 + (k - j - 1); }

__device__ __forceinline__ double poly3(const double* c, double x) {
  return __ldg(c) + x * (__ldg(c + 1) + x * (__ldg(c + 2) + x * __ldg(c + 3)));
}

// G <= 32: a group lives inside one warp, so its synchronisation is a warp-level one
template <int G>
__global__ void __launch_bounds__(256) transport_kernel(const TrParams P) {
  extern __shared__ double tsm[];
  double* etab = tsm;                        // 2^(j/64) of the table-driven exponential
  stage_exp_table(etab);
  __syncthreads();
  TGrp<G> g;
  g.init();
  const int ns = P.ns;
  const int gpb = blockDim.x / G;
  const int npair = ns * (ns - 1) / 2;
  double* X = tsm + 64 + (size_t)g.gid * (4 * ns + npair);   // mole fractions
  double* s = X + ns;                        // mu_k^(1/2)
  double* is = s + ns;                       // mu_k^(-1/2)
  double* Yc = is + ns;                      // mass fractions of the cell
  double* E = Yc + ns;                       // 1 / D_jk(p_atm) per unordered pair
  for (int64_t c = (int64_t)blockIdx.x * gpb + g.gid; c < P.n; c += (int64_t)gridDim.x * gpb) {
    const double T = P.T[c];
    const double lnT = log(T);
    const double pr = P.p[c] / kPatm;          // D_jk(p) = D_jk(p_atm) / pr
    // pure-species properties, mole fractions, Mathur sums
    double yw = 0.0;
    for (int k = g.tid; k < ns; k += G) {
      const double y = P.Y[(int64_t)k * P.ld + c];
      Yc[k] = y;
      const double a = 0.5 * poly3(P.mu_poly + 4 * k, lnT);
      s[k] = exp_tab(a, etab);
      is[k] = exp_tab(-a, etab);
      X[k] = y * __ldg(P.invW + k);
      yw += X[k];
    }
    const double S = g.sum(yw);
    double lx = 0.0, lxi = 0.0;
    for (int k = g.tid; k < ns; k += G) {
      const double x = X[k] / S;
      X[k] = x;
      const double pl = poly3(P.lam_poly + 4 * k, lnT);
      lx += x * exp_tab(pl, etab);
      lxi += x * exp_tab(-pl, etab);
    }
    lx = g.sum(lx);
    lxi = g.sum(lxi);
    if (P.Dm)
      for (int q = g.tid; q < npair; q += G) {
        const int jk = __ldg(P.pairs + q);
        E[q] = exp_tab(-poly3(P.diff_poly + 4 * ((jk & 0xffff) * ns + (jk >> 16)), lnT), etab);
      }
    g.sync();
    // Wilke viscosity and mixture-averaged diffusion: row k per lane
    double num = 0.0;
    for (int k = g.tid; k < ns; k += G) {
      double den = 0.0, dsum = 0.0;
      const double sk = s[k];
      for (int j = 0; j < ns; ++j) {
        const double xj = X[j];
        const double t = 1.0 + sk * is[j] * __ldg(P.wq + j * ns + k);
        den += xj * t * t * __ldg(P.cw + k * ns + j);
        if (P.Dm && j != k) dsum += xj * E[j < k ? pair_index(j, k, ns) : pair_index(k, j, ns)];
      }
      num += X[k] * sk * sk / den;
      if (P.Dm) {
        // 1 / D_jk(p) = pr / D_jk(p_atm); a cell holding species k alone takes the self-diffusion fit
        const double D = dsum > 0.0 ? (1.0 - Yc[k]) / (dsum * pr) : exp(poly3(P.diff_poly + 4 * (k * ns + k), lnT)) / pr;
        P.Dm[(int64_t)k * P.ld + c] = D;
      }
    }
    num = g.sum(num);
    if (g.tid == 0) {
      if (P.mu) P.mu[c] = num;
      if (P.lam) P.lam[c] = 0.5 * (lx + 1.0 / lxi);
    }
    g.sync();
  }
}

inline unsigned grid_cells(int64_t n, int per_block) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, 152 * 16));
}

}  // namespace

extern "C" int chem_mixture_thermo(chem_mech_t m, const double* T, const double* Y, int64_t ld, int64_t ncells,
                                   double* h, double* cp, chem_stream_t stream) {
  if (!m || ncells < 0 || ld < ncells) { set_error("bad arguments"); return CHEM_EINVAL; }
  if (ncells == 0) return CHEM_OK;
  if (!T || !Y || (!h && !cp)) { set_error("NULL pointer"); return CHEM_EINVAL; }
  mixture_thermo_kernel<<<grid_cells(ncells, 256), 256, 0, (cudaStream_t)stream>>>(
      (const unsigned char*)m->d_blob, m->lay, T, Y, ld, ncells, h, cp);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_temperature_from_enthalpy(chem_mech_t m, const double* h, const double* Y, int64_t ld,
                                              int64_t ncells, double* T, int8_t* status, chem_stream_t stream) {
  if (!m || ncells < 0 || ld < ncells) { set_error("bad arguments"); return CHEM_EINVAL; }
  if (ncells == 0) return CHEM_OK;
  if (!h || !Y || !T) { set_error("NULL pointer"); return CHEM_EINVAL; }
  temperature_from_h_kernel<<<grid_cells(ncells, 256), 256, 0, (cudaStream_t)stream>>>(
      (const unsigned char*)m->d_blob, m->lay, h, Y, ld, ncells, T, status);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_transport_free(chem_transport_t t) {
  if (!t) { set_error("NULL transport"); return CHEM_EINVAL; }
  if (t->d) cudaFree(t->d);
  delete t;
  return CHEM_OK;
}

extern "C" int chem_transport_create(chem_mech_t m, const chem_transport_desc* d, chem_transport_t* out) {
  if (!m || !d || !out) { set_error("NULL argument"); return CHEM_EINVAL; }
  *out = nullptr;
  const int ns = d->n_species;
  if (ns != m->ns || !d->mu_poly || !d->lambda_poly || !d->diff_poly) {
    set_error("transport data do not match the mechanism (ns %d vs %d) or a table is NULL", ns, m->ns);
    return CHEM_EINVAL;
  }
  const size_t n1 = (size_t)ns * 4, n2 = (size_t)ns * ns * 4, nw = (size_t)ns * ns;
  const size_t npair = (size_t)ns * (ns - 1) / 2;
  std::vector<double> h(2 * n1 + n2 + ns + 2 * nw + (npair + 1) / 2);   // the pair list rides along as ints
  double* p = h.data();
  for (size_t i = 0; i < n1; ++i) {
    if (!std::isfinite(d->mu_poly[i]) || !std::isfinite(d->lambda_poly[i])) {
      set_error("non-finite transport fit");
      return CHEM_EINVAL;
    }
  }
  std::copy(d->mu_poly, d->mu_poly + n1, p);
  std::copy(d->lambda_poly, d->lambda_poly + n1, p + n1);
  std::copy(d->diff_poly, d->diff_poly + n2, p + 2 * n1);
  double* invW = p + 2 * n1 + n2;
  double* wq = invW + ns;
  double* cw = wq + nw;
  for (int k = 0; k < ns; ++k) invW[k] = 1.0 / m->W[k];
  for (int j = 0; j < ns; ++j)
    for (int k = 0; k < ns; ++k) {
      wq[j * ns + k] = std::pow(m->W[j] / m->W[k], 0.25);
      cw[k * ns + j] = 1.0 / std::sqrt(8.0 * (1.0 + m->W[k] / m->W[j]));
    }
  int* pairs = reinterpret_cast<int*>(cw + nw);
  for (int j = 0, q = 0; j < ns; ++j)
    for (int k = j + 1; k < ns; ++k) pairs[q++] = j | (k << 16);
  chem_transport_s* t = new chem_transport_s();
  t->mech = m;
  t->ns = ns;
  cudaError_t e = cudaMalloc((void**)&t->d, h.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(t->d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    const int rc = cuda_fail(e, "transport tables");
    chem_transport_free(t);
    return rc;
  }
  t->mu_poly = t->d;
  t->lam_poly = t->d + n1;
  t->diff_poly = t->d + 2 * n1;
  t->invW = t->d + 2 * n1 + n2;
  t->wq = t->invW + ns;
  t->cw = t->wq + nw;
  t->pairs = reinterpret_cast<const int*>(t->cw + nw);
  *out = t;
  return CHEM_OK;
}

extern "C" int chem_transport_eval(chem_transport_t t, const double* T, const double* p, const double* Y,
                                   int64_t ld, int64_t ncells, double* mu, double* lambda, double* Dmix,
                                   chem_stream_t stream) {
  if (!t || ncells < 0 || ld < ncells) { set_error("bad arguments"); return CHEM_EINVAL; }
  if (ncells == 0) return CHEM_OK;
  if (!T || !p || !Y || (!mu && !lambda && !Dmix)) { set_error("NULL pointer"); return CHEM_EINVAL; }
  TrParams P;
  P.T = T; P.p = p; P.Y = Y; P.ld = ld; P.n = ncells; P.mu = mu; P.lam = lambda; P.Dm = Dmix;
  P.mu_poly = t->mu_poly; P.lam_poly = t->lam_poly; P.diff_poly = t->diff_poly; P.invW = t->invW;
  P.wq = t->wq; P.cw = t->cw; P.pairs = t->pairs; P.ns = t->ns;
  const int G = t->ns + 1 <= 16 ? 4 : 32;
  const int threads = 256, gpb = threads / G;
  const size_t per_group = (size_t)(4 * t->ns + t->ns * (t->ns - 1) / 2) * sizeof(double);
  const size_t smem = 64 * sizeof(double) + (size_t)gpb * per_group;
  static size_t smem_set = 48 * 1024;
  if (smem > smem_set) {
    if (smem > 200 * 1024) { set_error("mechanism too large for the transport kernel"); return CHEM_EINVAL; }
    CHEM_CUDA_TRY(cudaFuncSetAttribute(transport_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CHEM_CUDA_TRY(cudaFuncSetAttribute(transport_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    smem_set = smem;
  }
  const unsigned grid = grid_cells(ncells, gpb);
  if (G == 4) transport_kernel<4><<<grid, threads, smem, (cudaStream_t)stream>>>(P);
  else transport_kernel<32><<<grid, threads, smem, (cudaStream_t)stream>>>(P);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}
