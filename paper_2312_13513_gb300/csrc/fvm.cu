// Implicit finite-volume assembly of a species equation (the paper's species PDE, §3.1, with the
// Laplacian term of Alg. 1) and the PaSR factor of the LES closure (§2), for sm_103a.
//
// Equation of one species over one step dt, for the new value Y of every cell P:
//   (rho_P Y_P - rho_P^old Y_P^old) V_P / dt + sum_f F_f(Y) - sum_f a_f (Y_N - Y_P)
//     - sum_{fixed-value b} a_b (Y_b - Y_P) = V_P kappa_P S_P
// with a_f = gamma_f |S_f| delta_f, gamma_f = w_f gamma_owner + (1 - w_f) gamma_neighbour (Alg. 1)
// and upwind convection F_f by the face mass flux.  The result is the paper's ldu matrix (lower
// and upper per internal face, diag per cell) plus a source per cell, and on request the same
// matrix in CSR form for a linear solver (the paper converts ldu to CSR for AmgX).
//
// Design.  Alg. 1 assembles face by face and accumulates the diagonal with atomicAdd, with one
// kernel per boundary patch captured in a CUDA graph.  Here one kernel does everything: a thread
// per cell walks the cell's faces through a cell-to-face index built once per mesh, computes each
// face coefficient itself (an internal face is evaluated by both of its cells, identically), sums
// the diagonal in registers and writes the upper entry of the faces it owns and the lower entry of
// the faces it neighbours.  No atomics, one launch whatever the patch count, and results that are
// bitwise reproducible run to run.  On GB300 the FP64 pipe, not HBM, bounds this gather (ncu: FP64
// pipe 85 % busy at 20 % of DRAM bandwidth), so the FP64 work per face visit is kept small: the
// geometric factor |S_f| delta_f is multiplied once per mesh, the interpolation is one FMA
// (gamma_f = gamma_n + w (gamma_o - gamma_n)), the upwind choice tests the flux's sign bit with
// integer arithmetic, and 1/dt is formed once per launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "chem_internal.h"

struct chem_fvmesh_s {
  int64_t n_cells = 0, n_faces = 0, n_bfaces = 0, nnz = 0;
  int32_t *owner = nullptr, *neighbour = nullptr;
  double *weight = nullptr, *sd = nullptr;            // sd = |S_f| delta_f
  int32_t* b_cell = nullptr;
  int8_t* b_type = nullptr;
  double *b_sd = nullptr, *volume = nullptr;
  int32_t *cell_ptr = nullptr, *cell_face = nullptr;   // per cell: codes f<<2 | 0 (owner), f<<2 | 1 (neighbour), b<<2 | 2
  int32_t *row_ptr = nullptr, *col_idx = nullptr, *csr_src = nullptr;   // CSR pattern; src: -1 diag, 2f upper, 2f+1 lower
  std::vector<void*> allocs;
};

namespace chem {
namespace {

struct FvmArgs {
  int64_t n;
  const int32_t *owner, *neighbour, *cell_ptr, *cell_face, *b_cell;
  const int8_t* b_type;
  const double *weight, *sd, *b_sd, *volume;
  double inv_dt;                                       // 1 / dt, 0: no time term
  const double *rho, *rho_old, *Y_old, *phi, *phi_b, *gamma, *gamma_b, *Y_b, *S, *kappa;
  double *lower, *upper, *diag, *source;
};

__global__ void fvm_assemble_kernel(const FvmArgs a) {
  for (int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; P < a.n; P += (int64_t)gridDim.x * blockDim.x) {
    const double V = a.volume[P];
    double dg = 0.0, src = 0.0;
    if (a.inv_dt > 0.0) {
      const double vdt = V * a.inv_dt;
      dg = a.rho[P] * vdt;
      src = a.rho_old[P] * a.Y_old[P] * vdt;
    }
    const double gP = a.gamma ? a.gamma[P] : 0.0;
    const int e1 = a.cell_ptr[P + 1];
    for (int e = a.cell_ptr[P]; e < e1; ++e) {
      const int code = a.cell_face[e];
      const int kind = code & 3, f = code >> 2;
      if (kind < 2) {                                        // internal face; kind 0: P owns it
        double off = 0.0;
        if (a.phi) {
          // mass flux out of P (the sign flip and the upwind test are bit operations)
          const double F = a.phi[f];
          const double Fout = __hiloint2double(__double2hiint(F) ^ (kind == 0 ? 0 : (int)0x80000000),
                                               __double2loint(F));
          if (__double2hiint(Fout) >= 0) dg += Fout; else off += Fout;   // outflow carries Y_P
        }
        if (a.gamma) {
          const int other = kind == 0 ? a.neighbour[f] : a.owner[f];
          const double gO = a.gamma[other];
          const double g_own = kind == 0 ? gP : gO, g_nei = kind == 0 ? gO : gP;
          const double gf = fma(a.weight[f], g_own - g_nei, g_nei);     // w g_own + (1 - w) g_nei
          const double c = gf * a.sd[f];
          dg += c;
          off -= c;
        }
        if (kind == 0) a.upper[f] = off; else a.lower[f] = off;
      } else {                                               // boundary face
        if (a.phi_b) {
          const double Fb = a.phi_b[f];
          if (__double2hiint(Fb) >= 0) dg += Fb; else src -= Fb * a.Y_b[f];
        }
        if (a.gamma && a.b_type[f] == 1) {
          const double c = a.gamma_b[f] * a.b_sd[f];
          dg += c;
          src += c * a.Y_b[f];
        }
      }
    }
    if (a.S) src += V * (a.kappa ? a.kappa[P] : 1.0) * a.S[P];
    a.diag[P] = dg;
    if (a.source) a.source[P] = src;
  }
}

__global__ void fvm_to_csr_kernel(int64_t nnz, const int32_t* row_of, const int32_t* src, const double* lower,
                                  const double* upper, const double* diag, double* vals) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = src[e];
    vals[e] = s < 0 ? diag[row_of[e]] : ((s & 1) ? lower[s >> 1] : upper[s >> 1]);
  }
}

// kappa = tau_c / (tau_c + tau_mix), tau_mix = C_mix sqrt(mu_eff / (rho eps)),
// nu_sgs = (C_s Delta)^2 |S|, mu_eff = mu + rho nu_sgs, eps = nu_sgs |S|^2; kappa = 1 without
// sub-grid turbulence (eps = 0)
__global__ void pasr_kernel(int64_t n, const double* tau_c, const double* rho, const double* mu,
                            const double* strain, const double* delta, double c_s, double c_mix, double* kappa) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double cd = c_s * delta[i];
    const double s = strain[i];
    const double nu = cd * cd * s;
    const double eps = nu * s * s;
    double k = 1.0;
    if (eps > 0.0) {
      const double tmix = c_mix * sqrt((mu[i] + rho[i] * nu) / (rho[i] * eps));
      k = tau_c[i] / (tau_c[i] + tmix);
    }
    kappa[i] = k;
  }
}

inline unsigned grid_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)std::max(sms, 1) * 16));
}

template <class T>
int upload(chem_fvmesh_s* m, T** dst, const T* src, size_t count) {
  if (count == 0) { *dst = nullptr; return CHEM_OK; }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(mesh)");
  m->allocs.push_back(p);
  e = cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(mesh)");
  *dst = (T*)p;
  return CHEM_OK;
}

}  // namespace
}  // namespace chem

using namespace chem;

extern "C" int chem_fvmesh_free(chem_fvmesh_t m) {
  if (!m) { set_error("NULL mesh"); return CHEM_EINVAL; }
  for (void* p : m->allocs) cudaFree(p);
  delete m;
  return CHEM_OK;
}

extern "C" int chem_fvmesh_create(const chem_fvmesh_desc* d, chem_fvmesh_t* out) {
  if (!d || !out) { set_error("NULL argument"); return CHEM_EINVAL; }
  *out = nullptr;
  const int64_t n = d->n_cells, nf = d->n_faces, nb = d->n_bfaces;
  if (n < 1 || nf < 0 || nb < 0 || n > INT32_MAX || nf >= (1ll << 29) || nb >= (1ll << 29) ||
      (nf && (!d->owner || !d->neighbour || !d->weight || !d->delta || !d->mag_sf)) ||
      (nb && (!d->b_cell || !d->b_type || !d->b_delta || !d->b_mag_sf)) || !d->volume) {
    set_error("bad mesh description");
    return CHEM_EINVAL;
  }
  if (n + 2 * nf > INT32_MAX) {      // the CSR pattern's row pointers are 32-bit
    set_error("mesh too large: %lld matrix entries exceed 2^31 - 1", (long long)(n + 2 * nf));
    return CHEM_EINVAL;
  }
  for (int64_t f = 0; f < nf; ++f)
    if (d->owner[f] < 0 || d->neighbour[f] >= n || d->owner[f] >= d->neighbour[f]) {
      set_error("face %lld: owner must be below neighbour, both cells of the mesh", (long long)f);
      return CHEM_EINVAL;
    }
  for (int64_t b = 0; b < nb; ++b)
    if (d->b_cell[b] < 0 || d->b_cell[b] >= n || (d->b_type[b] != 0 && d->b_type[b] != 1)) {
      set_error("boundary face %lld: bad cell or patch type", (long long)b);
      return CHEM_EINVAL;
    }
  // cell -> face index (faces in mesh order within each cell) and the CSR pattern of the matrix
  std::vector<int32_t> cnt(n + 1, 0), nnz_row(n, 1);
  for (int64_t f = 0; f < nf; ++f) { cnt[d->owner[f] + 1]++; cnt[d->neighbour[f] + 1]++; nnz_row[d->owner[f]]++; nnz_row[d->neighbour[f]]++; }
  for (int64_t b = 0; b < nb; ++b) cnt[d->b_cell[b] + 1]++;
  std::vector<int32_t> cell_ptr(n + 1, 0);
  for (int64_t c = 0; c < n; ++c) cell_ptr[c + 1] = cell_ptr[c] + cnt[c + 1];
  std::vector<int32_t> fill(cell_ptr.begin(), cell_ptr.end() - 1), cell_face(cell_ptr[n]);
  for (int64_t f = 0; f < nf; ++f) {
    cell_face[fill[d->owner[f]]++] = (int32_t)(f << 2);
    cell_face[fill[d->neighbour[f]]++] = (int32_t)((f << 2) | 1);
  }
  for (int64_t b = 0; b < nb; ++b) cell_face[fill[d->b_cell[b]]++] = (int32_t)((b << 2) | 2);
  std::vector<int32_t> row_ptr(n + 1, 0);
  for (int64_t c = 0; c < n; ++c) row_ptr[c + 1] = row_ptr[c] + nnz_row[c];
  const int64_t nnz = row_ptr[n];
  std::vector<std::pair<int32_t, int32_t>> row;      // (column, source) of one row
  std::vector<int32_t> col_idx(nnz), csr_src(nnz);
  for (int64_t c = 0; c < n; ++c) {
    row.clear();
    row.push_back({(int32_t)c, -1});
    for (int e = cell_ptr[c]; e < cell_ptr[c + 1]; ++e) {
      const int code = cell_face[e], kind = code & 3, f = code >> 2;
      if (kind == 0) row.push_back({d->neighbour[f], 2 * f});        // upper: (owner row, neighbour col)
      else if (kind == 1) row.push_back({d->owner[f], 2 * f + 1});   // lower: (neighbour row, owner col)
    }
    std::sort(row.begin(), row.end());
    for (size_t k = 0; k < row.size(); ++k) {
      col_idx[row_ptr[c] + k] = row[k].first;
      csr_src[row_ptr[c] + k] = row[k].second;
    }
  }
  std::vector<double> sd(nf), b_sd(nb);
  for (int64_t f = 0; f < nf; ++f) sd[f] = d->mag_sf[f] * d->delta[f];
  for (int64_t b = 0; b < nb; ++b) b_sd[b] = d->b_mag_sf[b] * d->b_delta[b];
  chem_fvmesh_s* m = new chem_fvmesh_s();
  m->n_cells = n; m->n_faces = nf; m->n_bfaces = nb; m->nnz = nnz;
  int rc = CHEM_OK;
  if (!rc) rc = upload(m, &m->owner, d->owner, nf);
  if (!rc) rc = upload(m, &m->neighbour, d->neighbour, nf);
  if (!rc) rc = upload(m, &m->weight, d->weight, nf);
  if (!rc) rc = upload(m, &m->sd, sd.data(), nf);
  if (!rc) rc = upload(m, &m->b_cell, d->b_cell, nb);
  if (!rc) rc = upload(m, &m->b_type, d->b_type, nb);
  if (!rc) rc = upload(m, &m->b_sd, b_sd.data(), nb);
  if (!rc) rc = upload(m, &m->volume, d->volume, n);
  if (!rc) rc = upload(m, &m->cell_ptr, cell_ptr.data(), n + 1);
  if (!rc) rc = upload(m, &m->cell_face, cell_face.data(), cell_face.size());
  if (!rc) rc = upload(m, &m->row_ptr, row_ptr.data(), n + 1);
  if (!rc) rc = upload(m, &m->col_idx, col_idx.data(), nnz);
  if (!rc) rc = upload(m, &m->csr_src, csr_src.data(), nnz);
  if (rc) { chem_fvmesh_free(m); return rc; }
  *out = m;
  return CHEM_OK;
}

extern "C" int chem_fvmesh_csr(chem_fvmesh_t m, int64_t* nnz, const int32_t** row_ptr, const int32_t** col_idx) {
  if (!m || !nnz || !row_ptr || !col_idx) { set_error("NULL argument"); return CHEM_EINVAL; }
  *nnz = m->nnz; *row_ptr = m->row_ptr; *col_idx = m->col_idx;
  return CHEM_OK;
}

extern "C" int chem_fvm_assemble(chem_fvmesh_t m, const chem_fvm_terms* t, double* lower, double* upper,
                                 double* diag, double* source, chem_stream_t stream) {
  if (!m || !t || !diag || (m->n_faces && (!lower || !upper))) { set_error("NULL argument"); return CHEM_EINVAL; }
  if (t->dt > 0.0 && (!t->rho || !t->rho_old || !t->Y_old)) { set_error("the time term needs rho, rho_old, Y_old"); return CHEM_EINVAL; }
  if (t->phi_b && !t->Y_b) { set_error("boundary fluxes need boundary values"); return CHEM_EINVAL; }
  if (t->gamma && m->n_bfaces && (!t->gamma_b || !t->Y_b)) { set_error("the Laplacian needs gamma_b and Y_b"); return CHEM_EINVAL; }
  FvmArgs a;
  a.n = m->n_cells; a.owner = m->owner; a.neighbour = m->neighbour; a.cell_ptr = m->cell_ptr;
  a.cell_face = m->cell_face; a.b_cell = m->b_cell; a.b_type = m->b_type; a.weight = m->weight;
  a.sd = m->sd; a.b_sd = m->b_sd; a.volume = m->volume;
  a.inv_dt = t->dt > 0.0 ? 1.0 / t->dt : 0.0; a.rho = t->rho; a.rho_old = t->rho_old; a.Y_old = t->Y_old; a.phi = t->phi; a.phi_b = t->phi_b;
  a.gamma = t->gamma; a.gamma_b = t->gamma_b; a.Y_b = t->Y_b; a.S = t->S; a.kappa = t->kappa;
  a.lower = lower; a.upper = upper; a.diag = diag; a.source = source;
  fvm_assemble_kernel<<<grid_for(a.n), 256, 0, (cudaStream_t)stream>>>(a);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_fvm_to_csr(chem_fvmesh_t m, const double* lower, const double* upper, const double* diag,
                               double* vals, chem_stream_t stream) {
  if (!m || !diag || !vals || (m->n_faces && (!lower || !upper))) { set_error("NULL argument"); return CHEM_EINVAL; }
  // the row of each nonzero, for the diagonal entries: col_idx holds the row there
  fvm_to_csr_kernel<<<grid_for(m->nnz), 256, 0, (cudaStream_t)stream>>>(m->nnz, m->col_idx, m->csr_src, lower,
                                                                         upper, diag, vals);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_pasr_kappa(int64_t n, const double* tau_c, const double* rho, const double* mu,
                               const double* strain, const double* delta, double c_s, double c_mix,
                               double* kappa, chem_stream_t stream) {
  if (n < 0) { set_error("negative n"); return CHEM_EINVAL; }
  if (n == 0) return CHEM_OK;
  if (!tau_c || !rho || !mu || !strain || !delta || !kappa || !(c_s >= 0.0) || !(c_mix >= 0.0)) {
    set_error("bad arguments");
    return CHEM_EINVAL;
  }
  pasr_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, tau_c, rho, mu, strain, delta, c_s, c_mix, kappa);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}
