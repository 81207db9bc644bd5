// Internal declarations shared by the libchem translation units (host + device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/chem.h"

namespace chem {

constexpr double RU = 8.314462618e7;    // erg / (mol K)
constexpr double RC = RU / 4.184e7;     // cal / (mol K)
constexpr double PATM = 1.01325e6;      // dyn / cm^2
constexpr double TMID = 1000.0;

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define CHEM_CUDA_TRY(call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::chem::cuda_fail(e_, #call); \
  } while (0)

// Byte offsets of the arrays inside the mechanism blob that each CTA stages into shared memory.
// All arrays are 16-byte aligned.  Doubles first, then 16-bit and 32-bit integers.
struct MechLayout {
  int ns, nr, N, ntb, ntroe, nprod;     // nprod: entries of the species production lists
  int npieces;                          // balanced pieces of the production lists
  int bytes;                            // total blob size (multiple of 16)
  int o_W, o_invW;                      // [ns]
  int o_hc;                             // [2][ns][6]  h/RT:  a1, a2/2, a3/3, a4/4, a5/5, a6
  int o_sc;                             // [2][ns][6]  s/R:   a1 (x lnT), a2, a3/2, a4/3, a5/4, a7
  int o_cpc;                            // [2][ns][5]  cp/R:  a1..a5
  int o_lnA, o_beta, o_Ta;              // [nr]
  int o_troe;                           // [ntroe][8]: lnA0, b0, Ta0, a, 1/T3, 1/T1, T2, has_T2
  int o_effv;                           // [neff] efficiency - 1 (sparse, per third-body set)
  int o_const;                          // [kConsts] doubles, see kC_*
  int o_reac, o_prod;                   // [nr][4] int16 species (-1 pad), 4th entry unused
  int o_rinfo;                          // [nr][4] int16: type, dnu, third-body set, troe index
  int o_effidx;                         // [neff] int16 species
  int o_wpk;                            // [nprod] int32 production term: reaction << 4 | (nu + 8)
  int o_effoff;                         // [ntb + 1] int32
  int o_woff;                           // [ns + 1] int32
  int o_pterm;                          // [npieces + 1] int32: term range of each piece
  int o_poff;                           // [ns + 1] int32: pieces of each species
};

// constants block of the blob: the stoichiometric-coefficient table indexed by the 4-bit code of
// a production term (value = code - 8), ln(p_atm / R), 1 / ns, and the 64-entry table 2^(j / 64)
// of the table-driven exponential (fastexp.cuh)
constexpr int kC_NU = 0;
constexpr int kC_LNPR0 = 16;
constexpr int kC_INVNS = 17;
constexpr int kC_EXPTAB = 18;
constexpr int kConsts = 82;

// Jacobian-assembly program of d(wdot)/dC (global memory, read-only): entry e covers row
// ent_row[e], column ent_col[e]; its value is sum over terms t in [ent_off[e], ent_off[e+1]) of
// term_coef[t] * d_t.  Per reaction j the rate pass keeps three numbers: a_j = mult kf,
// b_j = -mult kr and the collision-partner factor X_j.  term_src[t] = j << 3 | c: for c = 7,
// d_t = X_j; for a reactant slot c < 3 (product slot c - 3), d_t = a_j (b_j) times the
// concentrations of the other two species of that side, term_oth[t] = o1 | o2 << 16 (ns for an
// empty slot, whose concentration reads as 1).
struct JacProgram {
  int nent = 0, nterm = 0;
  int* ent_off = nullptr;       // [nent + 1]
  int16_t* ent_row = nullptr;   // [nent]
  int16_t* ent_col = nullptr;   // [nent]
  int* term_src = nullptr;      // [nterm]
  int* term_oth = nullptr;      // [nterm]
  double* term_coef = nullptr;  // [nterm]
};

}  // namespace chem

struct chem_mech_s {
  int ns = 0, ne = 0, nr = 0;
  std::vector<double> W, elem_mass;
  std::vector<int> comp;
  std::vector<double> nasa_lo, nasa_hi;   // host copies (used by the surrogate set-up)
  chem::MechLayout lay{};
  int device = 0;
  void* d_blob = nullptr;                 // device copy of the shared-memory blob
  void* d_jac = nullptr;                  // device allocation holding the JacProgram arrays
  chem::JacProgram jac{};
};

namespace chem {
// integrator launch (used by the public entry points, the surrogate fallback and the server)
int launch_advance_batch(chem_mech_s* m, const chem_segment* segs, int nseg, cudaStream_t stream);
constexpr int kMaxSegsPerLaunch = 32;
int launch_advance_slice(chem_mech_s* m, const chem_segment* segs, int nseg, unsigned long long budget_ns,
                         unsigned long long* counter, long long* seg_end, cudaStream_t stream,
                         const unsigned int* stop = nullptr, unsigned long long min_ns = 0);
long long advance_queue_chunks(chem_mech_s* m, int64_t ncells);
int launch_advance(chem_mech_s* m, double* T, const double* p, double* Y, int64_t ld, double dt,
                   int64_t ncells, double rtol, double atol, const int32_t* idx, int8_t* status,
                   int32_t* nsub, int32_t* nrej, const chem_options* opt, cudaStream_t stream,
                   unsigned int* queue_counter);
}
