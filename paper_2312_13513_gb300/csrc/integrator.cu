// FP64 per-cell chemistry integrator for sm_103a.
//
// Each cell is an adiabatic constant-pressure reactor (the finite-rate chemistry step of §2,
// which the paper integrates with CVODE on the CPU).  It is advanced over one CFD step with the
// L-stable Rosenbrock method Rodas4 (Hairer & Wanner, Solving ODEs II, §IV.7): analytic Jacobian,
// dense LU with partial pivoting, six stages, embedded error estimate, adaptive sub-steps.
//
// Work decomposition ("group per cell"): a group of G threads owns one cell at a time.
//   G = 2   (sixteen cells per warp, sub-warp groups) for small mechanisms (N = ns + 1 <= 16,
//           H2-sized): FP64 instructions issue warp-wide whatever the active mask, so a warp per
//           10-unknown cell would leave most FP64 lanes idle; two lanes split a 10-long loop
//           into 5 full rounds (four lanes would idle half a round) and halve the lanes that
//           sit out per-cell scalar work;
//   G = 128 (a CTA-sized group per cell, named barriers) for CH4-sized ones (N ~ 54).
// Inside a group, threads split the species, the reactions, the Jacobian entries, the LU
// trailing updates and the triangular solves; sums use warp shuffles.  The mechanism (NASA-7
// coefficients, Arrhenius, fall-off, efficiency lists) is staged once per CTA into shared memory
// and shared by all groups of the CTA (§3.2 keeps constant coefficients in fast on-chip memory).
// The kernel is persistent: groups claim chunks of consecutive cells from a device work queue
// (one atomicAdd), load them species-row by species-row (coalesced 64-byte rows of the SoA
// state, §3.2), integrate them one after another and store them back, so cells needing many
// sub-steps do not stall the rest of the grid.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "chem_internal.h"
#include "fastexp.cuh"

namespace chem {

// Cells claimed per work-queue access: two consecutive cells for sub-warp groups (16 bytes per
// row of the SoA state: the state traffic is far below HBM bandwidth, shared memory per cell is
// what limits residency), one cell for groups of a warp or more, whose cells take milliseconds
// each
// (a time-sliced launch then overruns its budget by at most one cell).
__host__ __device__ constexpr int chunk_cells(int G) { return G >= 32 ? 1 : 2; }

// Threads per CTA at most.  Two-thread groups are few per CTA (shared memory per cell bounds
// them near 80), so their kernels are compiled for 256 threads and one CTA per SM, which lifts
// the register cap from 128 to 255 per thread: the inlined rate evaluation does not spill.
__host__ __device__ constexpr int max_threads(int G) { return G == 2 ? 256 : 512; }

// Rodas4 coefficients, transformed (u-variable) form:
//   (I/(gamma h) - J) u_s = f(y + sum_j A[s][j] u_j) + sum_j (C[s][j]/h) u_j,
//   y_new = y + sum_s M[s] u_s,  error = u_5.
__constant__ double kRA[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.544, 0, 0, 0, 0, 0},
    {0.9466785280815826, 0.2557011698983284, 0, 0, 0, 0},
    {3.314825187068521, 2.896124015972201, 0.9986419139977817, 0, 0, 0},
    {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.6878860361058950, 0, 0},
    {1.221224509226641, 6.019134481288629, 12.53708332932087, -0.6878860361058950, 1.0, 0}};
__constant__ double kRC[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {-5.6688, 0, 0, 0, 0, 0},
    {-2.430093356833875, -0.2063599157091915, 0, 0, 0, 0},
    {-0.1073529058151375, -9.594562251023355, -20.47028614809616, 0, 0, 0},
    {7.496443313967647, -10.24680431464352, -33.99990352819905, 11.70890893206160, 0, 0},
    {8.083246795921522, -7.981132988064893, -31.52159432874371, 16.31930543123136,
     -6.058818238834054, 0}};
__constant__ double kRM[6] = {1.221224509226641, 6.019134481288629, 12.53708332932087,
                              -0.6878860361058950, 1.0, 1.0};
constexpr double kGamma = 0.25;

// ---------------------------------------------------------------------------------------
// mechanism view (shared memory)
// ---------------------------------------------------------------------------------------
struct MechView {
  int ns, nr, N, npieces;
  const double *W, *invW, *hc, *sc, *cpc, *lnA, *beta, *Ta, *troe, *effv, *cst;
  const short4 *reac, *prod, *rinfo;
  const int16_t* effidx;
  const int *wpk, *effoff, *woff, *pterm, *poff;
};

__device__ __forceinline__ MechView bind_mech(const unsigned char* s, const MechLayout& L) {
  MechView m;
  m.ns = L.ns; m.nr = L.nr; m.N = L.N; m.npieces = L.npieces;
  m.W = (const double*)(s + L.o_W);
  m.invW = (const double*)(s + L.o_invW);
  m.hc = (const double*)(s + L.o_hc);
  m.sc = (const double*)(s + L.o_sc);
  m.cpc = (const double*)(s + L.o_cpc);
  m.lnA = (const double*)(s + L.o_lnA);
  m.beta = (const double*)(s + L.o_beta);
  m.Ta = (const double*)(s + L.o_Ta);
  m.troe = (const double*)(s + L.o_troe);
  m.effv = (const double*)(s + L.o_effv);
  m.cst = (const double*)(s + L.o_const);
  m.reac = (const short4*)(s + L.o_reac);
  m.prod = (const short4*)(s + L.o_prod);
  m.rinfo = (const short4*)(s + L.o_rinfo);
  m.effidx = (const int16_t*)(s + L.o_effidx);
  m.wpk = (const int*)(s + L.o_wpk);
  m.effoff = (const int*)(s + L.o_effoff);
  m.woff = (const int*)(s + L.o_woff);
  m.pterm = (const int*)(s + L.o_pterm);
  m.poff = (const int*)(s + L.o_poff);
  return m;
}

// Per-cell scalars that a multi-warp group evaluates on its first warp only and shares through
// the workspace (slot indices into w.sc).
enum : int {
  S_LNT, S_INVT, S_RHO, S_INVRHO, S_GSHIFT, S_EP1, S_IEP1, S_S, S_CP, S_DCP, S_Q, S_IRCP,
  S_RS, S_QOR2R, S_RHS, S_CPS, S_J00, S_IG, S_INVH, S_EN, S_FAC, S_NSC
};

// per-group workspace layout (doubles unless noted); offsets in doubles.  The Jacobian is
// assembled (negated) straight into the iteration-matrix buffer M and re-evaluated at every
// attempt, so a group holds one N x N matrix.
struct WsLayout {
  int LD;                  // leading dimension of the N x N matrix
  int y, ynew, ys, fs, f0, u, M, invd, tmp;
  int C, hRT, gRT, cpR, wdot, dwdT, rk, Hm;
  int q, dqdT, dq, wpart, dwpart, red, sc, stage, ctl, perm;
  int total;               // doubles
};

inline WsLayout make_ws(int ns, int nr, int npieces, int G) {
  WsLayout w{};
  const int N = ns + 1;
  // a group wider than a warp reads matrix columns across rows: an odd leading dimension keeps
  // those rows in different banks; sub-warp groups have at most 4 rows in flight and no padding
  w.LD = (G > 32 && N % 2 == 0) ? N + 1 : N;
  int o = 0;
  auto take = [&](int n) { int r = o; o += (n + 1) & ~1; return r; };   // keep 16-byte alignment
  // ys (a stage argument) is dead while a stage's solve runs and after the last stage, so the
  // solve's scratch and the new state share its storage
  w.y = take(N); w.f0 = take(N); w.ys = take(N); w.ynew = w.ys; w.tmp = w.ys; w.fs = take(N);
  w.u = take(6 * N); w.M = take(N * w.LD); w.invd = take(N);
  w.C = take(ns + 1); w.hRT = take(ns); w.gRT = take(ns); w.cpR = take(ns);
  w.wdot = take(ns); w.dwdT = take(ns); w.rk = take(ns); w.Hm = take(ns);
  // dq/dT per reaction is only needed inside a Jacobian evaluation, before the assembly writes the
  // matrix buffer (whose previous content, the last LU, is dead by then): it borrows that buffer
  w.q = take(nr); w.dqdT = nr <= N * w.LD ? w.M : take(nr);
  // the per-reaction derivative numbers live from the rate pass to the assembly of one Jacobian
  // evaluation, at the start of an attempt, when the stage buffers ys, fs and u (contiguous
  // above) are dead: small mechanisms keep them there
  const int stage_span = w.M - w.ys;
  w.dq = 3 * nr <= stage_span ? w.ys : take(3 * nr);
  // partial production sums of the balanced pieces (groups wider than a warp)
  w.wpart = take(G > 32 ? npieces : 0); w.dwpart = take(G > 32 ? npieces : 0);
  // cross-warp reductions and shared scalars exist only for groups wider than a warp
  w.red = take(G > 32 ? 8 * (G / 32) + 8 : 0);
  w.sc = take(G > 32 ? S_NSC : 0);
  w.stage = take(chunk_cells(G) * (N + 1));
  w.ctl = take(2);
  w.perm = take((N + 1) / 2);      // ints
  w.total = o;
  return w;
}

struct WsPtr {
  double *y, *ynew, *ys, *fs, *f0, *u, *M, *invd, *tmp;
  double *C, *hRT, *gRT, *cpR, *wdot, *dwdT, *rk, *Hm;
  double *q, *dqdT, *dq, *wpart, *dwpart, *red, *sc, *stage;
  unsigned long long* ctl;
  int* perm;
};

__device__ __forceinline__ WsPtr bind_ws(double* b, const WsLayout& w) {
  WsPtr p;
  p.y = b + w.y; p.ynew = b + w.ynew; p.ys = b + w.ys; p.fs = b + w.fs; p.f0 = b + w.f0;
  p.u = b + w.u; p.M = b + w.M; p.invd = b + w.invd; p.tmp = b + w.tmp;
  p.C = b + w.C; p.hRT = b + w.hRT; p.gRT = b + w.gRT; p.cpR = b + w.cpR;
  p.wdot = b + w.wdot; p.dwdT = b + w.dwdT; p.rk = b + w.rk; p.Hm = b + w.Hm;
  p.q = b + w.q; p.dqdT = b + w.dqdT; p.dq = b + w.dq; p.red = b + w.red; p.sc = b + w.sc;
  p.wpart = b + w.wpart; p.dwpart = b + w.dwpart;
  p.stage = b + w.stage;
  p.ctl = (unsigned long long*)(b + w.ctl);
  p.perm = (int*)(b + w.perm);
  return p;
}

// ---------------------------------------------------------------------------------------
// group primitives
// ---------------------------------------------------------------------------------------
template <int G>
struct Grp {
  int tid, gid;
  unsigned mask;      // lanes of this group within its warp (G <= 32)
  __device__ __forceinline__ void init() {
    tid = threadIdx.x % G;
    gid = threadIdx.x / G;
    if constexpr (G >= 32) {
      mask = 0xffffffffu;
    } else {
      const unsigned lane = threadIdx.x & 31u;
      mask = ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
  }
  __device__ __forceinline__ void sync() const {
    if (G < 32) {
      __syncwarp(mask);
    } else if (G == 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "n"(G) : "memory");
    }
  }
};

template <int G>
__device__ __forceinline__ double sub_sum(double v, unsigned mask) {
  constexpr int W = G < 32 ? G : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Sum of K values over the group; every thread receives bitwise-identical results (a butterfly
// adds the same two partial sums in every lane).
template <int G, int K>
__device__ __forceinline__ void gsum(const Grp<G>& g, double (&v)[K], double* red) {
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = sub_sum<G>(v[i], g.mask);
  if (G <= 32) return;
  constexpr int NW = G / 32;
  if ((g.tid & 31) == 0)
#pragma unroll
    for (int i = 0; i < K; ++i) red[i * NW + (g.tid >> 5)] = v[i];
  g.sync();
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double s = red[i * NW];
    for (int w = 1; w < NW; ++w) s += red[i * NW + w];
    v[i] = s;
  }
  g.sync();
}

// First warp of a multi-warp group (every thread of a group of at most one warp).  Per-cell
// scalar work runs there only: FP64 instructions are issued per warp whatever the number of
// active lanes, so each extra warp that repeats a logarithm or a division costs as much as a warp
// doing useful work.
template <int G>
__device__ __forceinline__ bool is_lead(const Grp<G>& g) { return G <= 32 || g.tid < 32; }

// Sum of K values over the group, delivered to the lead threads only (all threads for G <= 32).
// Only threads below nact hold non-zero values: warps entirely above it skip the reduction.
// Ends with the group synchronised once (G > 32); the caller publishes derived scalars through
// w.sc and synchronises again.
template <int G, int K>
__device__ __forceinline__ void gsum_lead(const Grp<G>& g, double (&v)[K], double* red, int nact) {
  if (G <= 32) {
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = sub_sum<G>(v[i], g.mask);
    return;
  }
  constexpr int NW = G / 32;
  const int nw = min(NW, (nact + 31) >> 5);
  if ((g.tid >> 5) < nw) {
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = sub_sum<G>(v[i], g.mask);
    if ((g.tid & 31) == 0)
#pragma unroll
      for (int i = 0; i < K; ++i) red[i * NW + (g.tid >> 5)] = v[i];
  }
  g.sync();
  if (g.tid < 32) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      double s = red[i * NW];
      for (int w = 1; w < nw; ++w) s += red[i * NW + w];
      v[i] = s;
    }
  }
}

// Division of a flat index by a run-time row length d without the integer divide: q = e / d is
// the high word of e * ceil(2^32 / d) (div_magic, formed in 32 bits; it wraps to 0 for d = 1,
// where only e = 0 occurs), exact while e * d < 2^32: the loops below have e < d^2, so any row
// length up to 1625, far beyond a matrix that fits in shared memory.
__device__ __forceinline__ unsigned div_magic(unsigned d) { return 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int div_by(int e, unsigned magic) { return (int)__umulhi((unsigned)e, magic); }

// Pivot key of a matrix entry: the bit pattern of |a| read as an unsigned integer.  For
// non-negative doubles the integer order is the numeric order, so the pivot search runs on the
// integer pipes instead of FP64 compares (the FP64 pipe is the scarce one).  NaN maps to 0.
__device__ __forceinline__ unsigned long long pivot_key(double a) {
  const unsigned long long k = (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
  return k > 0x7ff0000000000000ull ? 0ull : k;
}

__device__ __forceinline__ void argmax_merge(unsigned long long& best, int& bi, unsigned long long ob, int oi) {
  if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
}

// argmax (largest key, ties to the lowest index) across the lanes of a group within its warp
template <int G>
__device__ __forceinline__ void warp_argmax(const Grp<G>& g, unsigned long long& best, int& bi) {
  constexpr int W = G < 32 ? G : 32;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(g.mask, best, o);
    const int oi = __shfl_xor_sync(g.mask, bi, o);
    argmax_merge(best, bi, ob, oi);
  }
}

// ---------------------------------------------------------------------------------------
// right-hand side and analytic Jacobian at state y (group-cooperative)
// ---------------------------------------------------------------------------------------
struct JacArgs {
  int nent;
  const int* ent_off;
  const int16_t* ent_row;
  const int16_t* ent_col;
  const int* term_src;
  const int* term_oth;
  const double* term_coef;
};

// Right-hand side f(y) and, when Jneg is given, the NEGATED analytic Jacobian -df/dy written into
// Jneg (N x N, leading dimension LD): the iteration matrix I/(gamma h) - J then only needs its
// diagonal.  Ends with the group synchronised.
template <int G>
__device__ __forceinline__ void eval_fj(const Grp<G>& g, const MechView& m, const WsPtr& w,
                                     const JacArgs& jp, int LD, const double* y, double p,
                                     double* f, double* Jneg) {
  constexpr bool kMulti = G > 32;
  const bool lead = is_lead(g);
  const bool jac = Jneg != nullptr;
  const int ns = m.ns, nr = m.nr;
  const double* etab = m.cst + kC_EXPTAB;     // the table-driven exponential's 2^(j/64)
  const double T = y[0];
  double lnT = 0.0, invT = 0.0;
  if (lead) { lnT = log(T); invT = 1.0 / T; }
  if (kMulti) {
    if (g.tid == 0) { w.sc[S_LNT] = lnT; w.sc[S_INVT] = invT; }
    g.sync();
    lnT = w.sc[S_LNT]; invT = w.sc[S_INVT];
  }
  const int rg = (T < TMID) ? 0 : 1;

  // species thermo (A2): NASA-7 cp/R, h/RT, g/RT sharing T powers and ln T
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = g.tid; k < ns; k += G) {
    const double* hc = m.hc + (rg * ns + k) * 6;
    const double* sc = m.sc + (rg * ns + k) * 6;
    const double* cc = m.cpc + (rg * ns + k) * 5;
    const double h = hc[0] + T * (hc[1] + T * (hc[2] + T * (hc[3] + T * hc[4]))) + hc[5] * invT;
    const double s = sc[0] * lnT + T * (sc[1] + T * (sc[2] + T * (sc[3] + T * sc[4]))) + sc[5];
    const double cp = cc[0] + T * (cc[1] + T * (cc[2] + T * (cc[3] + T * cc[4])));
    w.hRT[k] = h;
    w.gRT[k] = h - s;
    w.cpR[k] = cp;
    acc[3] += h - s;
    const double yw = y[1 + k] * m.invW[k];
    acc[0] += yw;
    acc[1] += yw * cp;
    if (jac) {
      // d(cp/R)/dT = a2 + 2 a3 T + 3 a4 T^2 + 4 a5 T^3
      const double d = cc[1] + T * (2.0 * cc[2] + T * (3.0 * cc[3] + T * (4.0 * cc[4])));
      acc[2] += yw * d;
    }
  }
  gsum_lead<G, 4>(g, acc, w.red, ns);
  // mixture scalars: sum Y/W, cp, d(cp)/dT, mean g/RT (keeps exp(g/RT - gshift) in range),
  // density, and exp(gshift - ln(p_atm / (R T))) for the equilibrium constants
  double S = 0.0, cp = 0.0, dcpdT = 0.0, gshift = 0.0, rho = 0.0, invrho = 0.0, ep1 = 0.0, iep1 = 0.0;
  if (lead) {
    S = acc[0];
    cp = RU * acc[1];
    dcpdT = RU * acc[2];
    gshift = acc[3] * m.cst[kC_INVNS];
    rho = p / (RU * T * S);
    invrho = 1.0 / rho;
    ep1 = exp_tab(gshift - (m.cst[kC_LNPR0] - lnT), etab);
    iep1 = 1.0 / ep1;
  }
  if (kMulti) {
    if (g.tid == 0) {
      w.sc[S_S] = S; w.sc[S_CP] = cp; w.sc[S_DCP] = dcpdT; w.sc[S_GSHIFT] = gshift;
      w.sc[S_RHO] = rho; w.sc[S_INVRHO] = invrho; w.sc[S_EP1] = ep1; w.sc[S_IEP1] = iep1;
    }
    g.sync();
    S = w.sc[S_S]; cp = w.sc[S_CP]; dcpdT = w.sc[S_DCP]; gshift = w.sc[S_GSHIFT];
    rho = w.sc[S_RHO]; invrho = w.sc[S_INVRHO]; ep1 = w.sc[S_EP1]; iep1 = w.sc[S_IEP1];
  }
  // concentrations; per-species exp(g/RT - gshift) and its inverse: 1/Kc of every reaction
  // becomes a product (w.rk / w.Hm are free until the Jacobian section)
  double* eg = w.rk;
  double* ieg = w.Hm;
  if (g.tid == 0) w.C[ns] = 1.0;           // the concentration of an empty reaction slot
  for (int k = g.tid; k < ns; k += G) {
    w.C[k] = rho * y[1 + k] * m.invW[k];
    const double e = exp_tab(w.gRT[k] - gshift, etab);
    eg[k] = e;
    ieg[k] = 1.0 / e;
  }
  g.sync();

  // rates of progress (A3)
  const double Ctot = rho * S;
  const double lnPR = m.cst[kC_LNPR0] - lnT;     // ln(p_atm / (R T)), range fallback only
  for (int j = g.tid; j < nr; j += G) {
    const short4 ri = m.rinfo[j];
    const short4 re = m.reac[j];
    const short4 pr = m.prod[j];
    double kf = exp_tab(m.lnA[j] + m.beta[j] * lnT - m.Ta[j] * invT, etab);
    double Pf = 1.0, Pr = 1.0, dG = 0.0, dH = 0.0;
    const double cr0 = re.x >= 0 ? w.C[re.x] : 1.0;
    const double cr1 = re.y >= 0 ? w.C[re.y] : 1.0;
    const double cr2 = re.z >= 0 ? w.C[re.z] : 1.0;
    const double cp0 = pr.x >= 0 ? w.C[pr.x] : 1.0;
    const double cp1 = pr.y >= 0 ? w.C[pr.y] : 1.0;
    const double cp2 = pr.z >= 0 ? w.C[pr.z] : 1.0;
    Pf = cr0 * cr1 * cr2;
    Pr = cp0 * cp1 * cp2;
    double Mc = 0.0;
    if (ri.x != 0) {
      Mc = Ctot;
      for (int e = m.effoff[ri.z]; e < m.effoff[ri.z + 1]; ++e) Mc += m.effv[e] * w.C[m.effidx[e]];
    }
    double dlnkf = jac ? m.beta[j] * invT + m.Ta[j] * invT * invT : 0.0;
    double dkfdM = 0.0;
    if (ri.x == 2) {
      // Troe fall-off (Gilbert, Luther & Troe 1983): k = kinf Pr/(1+Pr) F(T, Pr)
      const double* tr = m.troe + 8 * ri.w;
      const double kinf = kf;
      const double k0 = exp_tab(tr[0] + tr[1] * lnT - tr[2] * invT, etab);
      if (kinf == 0.0 || k0 == 0.0) {
        kf = 0.0; dlnkf = 0.0; dkfdM = 0.0;
      } else {
        const double e3 = exp_tab(-T * tr[4], etab), e1 = exp_tab(-T * tr[5], etab);
        double Fc = (1.0 - tr[3]) * e3 + tr[3] * e1;
        double dFc = -(1.0 - tr[3]) * tr[4] * e3 - tr[3] * tr[5] * e1;
        if (tr[7] != 0.0) {
          const double e2 = exp_tab(-tr[6] * invT, etab);
          Fc += e2;
          dFc += tr[6] * invT * invT * e2;
        }
        if (Mc == 0.0) {
          kf = 0.0;
          dkfdM = k0 * pow(Fc, 1.0 / (1.0 + 1.0 / (0.14 * 0.14)));
          dlnkf = 0.0;
        } else {
          const double Prr = k0 * Mc / kinf;
          const double L = log10(Fc);
          const double c = -0.4 - 0.67 * L;
          const double n = 0.75 - 1.27 * L;
          const double u = log10(Prr) + c;
          const double d = n - 0.14 * u;
          const double f1 = u / d;
          const double den = 1.0 + f1 * f1;
          const double F = exp_tab(2.302585092994046 * (L / den), etab);
          const double opr = 1.0 / (1.0 + Prr);
          kf = kinf * (Prr * opr) * F;
          if (jac) {
            const double dGdlogPr = -2.0 * L * f1 / (den * den) * (n / (d * d));
            const double df1dL = (-0.67 * d - u * (-1.27 + 0.14 * 0.67)) / (d * d);
            const double dGdL = 1.0 / den - 2.0 * L * f1 / (den * den) * df1dL;
            const double dLdT = dFc / (Fc * 2.302585092994046);
            const double dlnk0 = tr[1] * invT + tr[2] * invT * invT;
            const double dlnPr = dlnk0 - dlnkf;
            dlnkf = dlnkf + dlnPr * (opr + dGdlogPr) + 2.302585092994046 * dGdL * dLdT;
            dkfdM = k0 * F * opr * (opr + dGdlogPr);
          }
        }
      }
    }
    double invKc = 1.0;                                   // 1 / Kc
    if (re.x >= 0) invKc *= ieg[re.x];
    if (re.y >= 0) invKc *= ieg[re.y];
    if (re.z >= 0) invKc *= ieg[re.z];
    if (pr.x >= 0) invKc *= eg[pr.x];
    if (pr.y >= 0) invKc *= eg[pr.y];
    if (pr.z >= 0) invKc *= eg[pr.z];
    for (int d = ri.y; d > 0; --d) invKc *= ep1;
    for (int d = ri.y; d < 0; ++d) invKc *= iep1;
    // range fallback (exp of dG directly) unless invKc is a positive normal number below 2^995;
    // the test reads the exponent bits (integer work, no FP64 compare)
    if ((unsigned)__double2hiint(invKc) - 0x00100000u >= 0x7e200000u - 0x00100000u) {
      if (re.x >= 0) dG -= w.gRT[re.x];
      if (re.y >= 0) dG -= w.gRT[re.y];
      if (re.z >= 0) dG -= w.gRT[re.z];
      if (pr.x >= 0) dG += w.gRT[pr.x];
      if (pr.y >= 0) dG += w.gRT[pr.y];
      if (pr.z >= 0) dG += w.gRT[pr.z];
      invKc = exp(dG - (double)ri.y * lnPR);
    }
    const double mult = (ri.x == 1) ? Mc : 1.0;
    if (!jac) {
      // q = kf (Pf - Pr / Kc): one FMA for the difference of the two directions
      w.q[j] = kf * fma(-invKc, Pr, Pf) * mult;
      continue;
    }
    const double kr = kf * invKc;
    const double fwd = kf * Pf, rev = kr * Pr;
    w.q[j] = (fwd - rev) * mult;
    {                                                     // the Jacobian's per-reaction numbers
      if (re.x >= 0) dH -= w.hRT[re.x];
      if (re.y >= 0) dH -= w.hRT[re.y];
      if (re.z >= 0) dH -= w.hRT[re.z];
      if (pr.x >= 0) dH += w.hRT[pr.x];
      if (pr.y >= 0) dH += w.hRT[pr.y];
      if (pr.z >= 0) dH += w.hRT[pr.z];
      const double dlnKc = (dH - (double)ri.y) * invT;
      w.dqdT[j] = mult * (fwd * dlnkf - rev * (dlnkf - dlnKc));
      // slot derivatives dq/dC = a (b) times the other concentrations of the side, formed by
      // the assembly program; the collision-partner factor X completes the reaction's share
      double* dq = w.dq + 3 * j;
      dq[0] = mult * kf;
      dq[1] = -mult * kr;
      dq[2] = (ri.x == 1) ? (fwd - rev) : (ri.x == 2 ? dkfdM * (Pf - Pr * invKc) : 0.0);
    }
  }
  g.sync();

  // production rates and right-hand side (A4).  A multi-warp group first sums balanced pieces
  // of the production lists (similar loop lengths in every lane), then adds each species' pieces.
  if (kMulti) {
    for (int pc = g.tid; pc < m.npieces; pc += G) {
      double a = 0.0, b = 0.0;
      for (int e = m.pterm[pc]; e < m.pterm[pc + 1]; ++e) {
        const int pk = m.wpk[e];
        const double nu = m.cst[kC_NU + (pk & 15)];
        const int j = pk >> 4;
        a += nu * w.q[j];
        if (jac) b += nu * w.dqdT[j];
      }
      w.wpart[pc] = a;
      if (jac) w.dwpart[pc] = b;
    }
    g.sync();
  }
  double r3[3] = {0.0, 0.0, 0.0};
  const double RT = RU * T;
  for (int k = g.tid; k < ns; k += G) {
    double wk = 0.0, dwk = 0.0;
    if (kMulti) {
      for (int pc = m.poff[k]; pc < m.poff[k + 1]; ++pc) {
        wk += w.wpart[pc];
        if (jac) dwk += w.dwpart[pc];
      }
    } else {
      for (int e = m.woff[k]; e < m.woff[k + 1]; ++e) {
        const int pk = m.wpk[e];
        const double nu = m.cst[kC_NU + (pk & 15)];
        const int j = pk >> 4;
        wk += nu * w.q[j];
        if (jac) dwk += nu * w.dqdT[j];
      }
    }
    w.wdot[k] = wk;
    const double hk = RT * w.hRT[k];
    r3[0] += hk * wk;
    f[1 + k] = m.W[k] * wk * invrho;
    if (jac) {
      w.dwdT[k] = dwk;
      r3[1] += w.cpR[k] * wk;
      r3[2] += hk * dwk;
    }
  }
  if (!jac) {
    double q1[1] = {r3[0]};
    gsum_lead<G, 1>(g, q1, w.red, ns);
    if (g.tid == 0) f[0] = -q1[0] / (rho * cp);
    g.sync();
    return;
  }
  gsum_lead<G, 3>(g, r3, w.red, ns);
  const double Q = r3[0];
  const double rcp = rho * cp;
  double ircp = 0.0;
  if (lead) ircp = 1.0 / rcp;
  if (g.tid == 0) f[0] = -Q / rcp;

  // analytic Jacobian (A5): d(wdot)/dC by the precomputed assembly program ...
  double* Jm = Jneg;
  const unsigned mns = div_magic((unsigned)ns);
  for (int e = g.tid; e < ns * ns; e += G) {
    const int k = div_by(e, mns);
    Jm[(1 + k) * LD + 1 + (e - k * ns)] = 0.0;
  }
  g.sync();
  for (int e = g.tid; e < jp.nent; e += G) {
    double s = 0.0;
    const int t1 = __ldg(jp.ent_off + e + 1);
    for (int t = __ldg(jp.ent_off + e); t < t1; ++t) {
      const int src = __ldg(jp.term_src + t);
      const double* dq = w.dq + 3 * (src >> 3);
      double d;
      if ((src & 7) == 7) {
        d = dq[2];
      } else {
        const int oth = __ldg(jp.term_oth + t);
        d = dq[(src & 7) >= 3 ? 1 : 0] * w.C[oth & 0xffff] * w.C[oth >> 16];
      }
      s += __ldg(jp.term_coef + t) * d;
    }
    Jm[(1 + __ldg(jp.ent_row + e)) * LD + 1 + __ldg(jp.ent_col + e)] = s;
  }
  if (kMulti && g.tid == 0) w.sc[S_IRCP] = ircp;
  g.sync();
  if (kMulti) ircp = w.sc[S_IRCP];
  // ... then the chain rule through C(T, Y) and rho(T, Y):
  //   r_k = sum_m dw_k/dC_m C_m,  H_m = RT sum_k h_k/RT dw_k/dC_m,  R_h = RT sum_k h_k/RT r_k
  //   J_km = W_k / W_m (dw_k/dC_m - (r_k - w_k) rho^-1 / S)              (species rows)
  //   J_k0 = W_k / rho (dw_k/dT - (r_k - w_k) / T)
  //   J_0m = (-(rho H_m - R_h / S) / (rho cp) + Q / (rho cp)^2 rho (R cp_m/R - cp / S)) / W_m
  const double rS = invrho / S;
  double rh[1] = {0.0};
  for (int k = g.tid; k < ns; k += G) {
    double s = 0.0;
    for (int mm = 0; mm < ns; ++mm) s += Jm[(1 + k) * LD + 1 + mm] * w.C[mm];
    rh[0] += RT * w.hRT[k] * s;
    const double dk = s - w.wdot[k];
    w.rk[k] = dk * rS;                               // (r_k - w_k) / (rho S)
    Jm[(1 + k) * LD] = -(m.W[k] * invrho * (w.dwdT[k] - dk * invT));
  }
  for (int mm = g.tid; mm < ns; mm += G) {
    double s = 0.0;
    for (int k = 0; k < ns; ++k) s += w.hRT[k] * Jm[(1 + k) * LD + 1 + mm];
    w.Hm[mm] = RT * s;
  }
  gsum_lead<G, 1>(g, rh, w.red, ns);
  double RhS = 0.0, cpS = 0.0, QoR2r = 0.0;
  if (lead) {
    const double Rh = rh[0];
    RhS = Rh / S;
    cpS = cp / S;
    QoR2r = Q * ircp * ircp * rho;
    if (g.tid == 0)
      Jm[0] = (RU * r3[1] + r3[2] - Rh * invT) * ircp - QoR2r * (-cp * invT + dcpdT);
  }
  if (kMulti) {
    if (g.tid == 0) { w.sc[S_RHS] = RhS; w.sc[S_CPS] = cpS; w.sc[S_QOR2R] = QoR2r; }
    g.sync();
    RhS = w.sc[S_RHS]; cpS = w.sc[S_CPS]; QoR2r = w.sc[S_QOR2R];
  } else {
    g.sync();
  }
  for (int e = g.tid; e < ns * ns; e += G) {
    const int k = div_by(e, mns), mm = e - k * ns;
    double* Jkm = Jm + (1 + k) * LD + 1 + mm;
    *Jkm = m.W[k] * m.invW[mm] * (w.rk[k] - *Jkm);
  }
  for (int mm = g.tid; mm < ns; mm += G)
    Jm[1 + mm] = m.invW[mm] * ((rho * w.Hm[mm] - RhS) * ircp - QoR2r * (RU * w.cpR[mm] - cpS));
  g.sync();
}

// ---------------------------------------------------------------------------------------
// dense LU with partial pivoting (A6) and triangular solves
// ---------------------------------------------------------------------------------------
// LU factorisation with partial pivoting, rows pivoted implicitly: perm[i] is the physical row
// of logical row i.  On return, for logical row i and column j, L[i][j] = M[perm[i]][j] (j < i,
// unit diagonal implied) and U[i][j] = M[perm[i]][j] (j >= i); invd[j] = 1 / U[j][j].
// Step k: (1) every thread merges the per-warp pivot candidates of column k; (2) the first warp
// forms the reciprocal of the pivot and the multipliers of column k and records the row swap in
// perm; (3) all threads update the trailing block and, on the way, collect the candidates of
// column k + 1.  Two group barriers per step.  Returns false on an exactly singular matrix.
template <int G>
__device__ bool lu_factor(const Grp<G>& g, double* M, int N, int LD, int* perm, double* invd,
                          double* red) {
  constexpr int NW = G > 32 ? G / 32 : 1;
  constexpr int W = G < 32 ? G : 32;
  unsigned long long* rkey = (unsigned long long*)red;
  int* ridx = (int*)(red + NW);
  for (int i = g.tid; i < N; i += G) perm[i] = i;
  unsigned long long best = 0ull;
  int bi = 0;
  for (int i = g.tid; i < N; i += G) argmax_merge(best, bi, pivot_key(M[i * LD]), i);
  warp_argmax<G>(g, best, bi);
  if (G > 32 && (g.tid & 31) == 0) { rkey[g.tid >> 5] = best; ridx[g.tid >> 5] = bi; }
  g.sync();
  for (int k = 0; k < N; ++k) {
    if (G > 32) {
      best = rkey[0];
      bi = ridx[0];
      for (int w = 1; w < NW; ++w) argmax_merge(best, bi, rkey[w], ridx[w]);
    }
    if (best == 0ull) return false;
    if (is_lead(g)) {
      const int pk = perm[bi], pb = perm[k];
      const double ip = 1.0 / M[pk * LD + k];
      for (int i = k + 1 + g.tid; i < N; i += W) {
        const int ph = (i == bi) ? pb : perm[i];
        M[ph * LD + k] *= ip;
      }
      if (G <= 32) __syncwarp(g.mask); else __syncwarp();
      if (g.tid == 0) {
        invd[k] = ip;
        perm[k] = pk;
        perm[bi] = pb;
      }
    }
    g.sync();
    const int n = N - k - 1;
    if (n == 0) break;
    const int pk = perm[k];
    best = 0ull;
    bi = k + 1;
    const unsigned magic = div_magic((unsigned)n);
    for (int e = g.tid; e < n * n; e += G) {
      const int q = div_by(e, magic);
      const int i = k + 1 + q, j = k + 1 + (e - q * n);
      const int ph = perm[i];
      const double v = fma(-M[ph * LD + k], M[pk * LD + j], M[ph * LD + j]);
      M[ph * LD + j] = v;
      if (j == k + 1) argmax_merge(best, bi, pivot_key(v), i);
    }
    warp_argmax<G>(g, best, bi);
    if (G > 32 && (g.tid & 31) == 0) { rkey[g.tid >> 5] = best; ridx[g.tid >> 5] = bi; }
    g.sync();
  }
  return true;
}

// LU factorisation for a group of several warps and at most 64 unknowns, one group barrier per
// step: in step k the first warp (the panel warp) finishes column k + 1 of the trailing update,
// chooses the pivot of step k + 1 among those values, forms its reciprocal and the multipliers
// of column k + 1, while the other warps update columns k + 2 .. N - 1 (the panel warp takes the
// last part of those elements once its pivot work is done).  The logical-to-physical
// row map is double-buffered (pbuf[0 .. N) for even steps, pbuf[N .. 2N) for odd ones), so the
// panel warp writes the next step's row swap while the other warps still read this step's map;
// the singular flag is double-buffered the same way.  Each element sees the same operations as
// in lu_factor (explicit FMAs in both) and the pivot choice is the same (largest magnitude, the
// lowest logical row on ties), so the factors, perm and invd are bitwise lu_factor's.
// Elements [0, E1) of a step's update of columns k + 2 .. go to the warps other than the panel
// warp, [E1, E) to the panel warp after its pivot work: its per-lane share of a balanced split
// less 8 elements per lane, the pivot work's measured worth (less 3, 12, 16 or 24 per lane
// measured slower on the CH4 LES field).
__device__ __forceinline__ int panel_split(int E, int G) {
  return max(E - max((E * 32) / G - 32 * 8, 0), 0);
}

template <int G>
__device__ bool lu_factor_panel(const Grp<G>& g, double* M, int N, int LD, int* perm,
                                double* invd, int* pbuf, int* sing) {
  static_assert(G > 32, "groups of several warps");
  constexpr unsigned F = 0xffffffffu;
  const bool panel = g.tid < 32;
  const int l = g.tid;
  if (panel) {                                      // the pivot of step 0
    unsigned long long best = 0ull;
    int bi = 0;
    for (int i = l; i < N; i += 32) argmax_merge(best, bi, pivot_key(M[i * LD]), i);
    warp_argmax<G>(g, best, bi);
    for (int i = l; i < N; i += 32) pbuf[i] = i == 0 ? bi : (i == bi ? 0 : i);
    if (best != 0ull) {
      const double ip = 1.0 / M[bi * LD];
      for (int i = 1 + l; i < N; i += 32) {
        const int ph = i == bi ? 0 : i;
        M[ph * LD] *= ip;
      }
      if (l == 0) { invd[0] = ip; perm[0] = bi; }
    }
    if (l == 0) sing[1] = best == 0ull;
  }
  g.sync();
  if (sing[1]) return false;
  for (int k = 0; k < N - 1; ++k) {
    const int* Pk = pbuf + (k & 1) * N;
    const int pk = Pk[k];
    const int n = N - k - 1;
    if (panel) {
      int* Pn = pbuf + ((k + 1) & 1) * N;
      const int i0 = k + 1 + l, i1 = k + 33 + l;
      const double ukj = M[pk * LD + k + 1];
      unsigned long long best = 0ull;
      int bi = k + 1;
      double v0 = 0.0, v1 = 0.0;
      int ph0 = -1, ph1 = -1;
      if (i0 < N) {
        ph0 = Pk[i0];
        v0 = fma(-M[ph0 * LD + k], ukj, M[ph0 * LD + k + 1]);
        argmax_merge(best, bi, pivot_key(v0), i0);
      }
      if (i1 < N) {
        ph1 = Pk[i1];
        v1 = fma(-M[ph1 * LD + k], ukj, M[ph1 * LD + k + 1]);
        argmax_merge(best, bi, pivot_key(v1), i1);
      }
      warp_argmax<G>(g, best, bi);
      const int pnew = Pk[bi], pold = Pk[k + 1];
      for (int i = k + 1 + l; i < N; i += 32) Pn[i] = i == k + 1 ? pnew : (i == bi ? pold : Pk[i]);
      if (best != 0ull) {
        const int src = bi - (k + 1);
        const double piv = __shfl_sync(F, src < 32 ? v0 : v1, src & 31);
        const double ip = 1.0 / piv;
        if (ph0 >= 0) M[ph0 * LD + k + 1] = ph0 == pnew ? v0 : v0 * ip;
        if (ph1 >= 0) M[ph1 * LD + k + 1] = ph1 == pnew ? v1 : v1 * ip;
        if (l == 0) { invd[k + 1] = ip; perm[k + 1] = pnew; }
      }
      if (l == 0) sing[k & 1] = best == 0ull;
      if (n > 1) {                                  // then its share of the other columns
        const int m = n - 1, E = n * m;
        const int E1 = panel_split(E, G);
        const unsigned magic = div_magic((unsigned)m);
        for (int e = E1 + l; e < E; e += 32) {
          const int q = div_by(e, magic);
          const int ph = Pk[k + 1 + q], j = k + 2 + (e - q * m);
          M[ph * LD + j] = fma(-M[ph * LD + k], M[pk * LD + j], M[ph * LD + j]);
        }
      }
    } else if (n > 1) {                             // columns k + 2 .. N - 1
      const int m = n - 1, E = n * m;
      const int E1 = panel_split(E, G);
      const unsigned magic = div_magic((unsigned)m);
      for (int e = g.tid - 32; e < E1; e += G - 32) {
        const int q = div_by(e, magic);
        const int ph = Pk[k + 1 + q], j = k + 2 + (e - q * m);
        M[ph * LD + j] = fma(-M[ph * LD + k], M[pk * LD + j], M[ph * LD + j]);
      }
    }
    g.sync();
    if (sing[k & 1]) return false;
  }
  return true;
}

// The two triangular sweeps of lu_solve for a group of one or more whole warps and at most 64
// unknowns: the group's first warp alone runs them with the rows in registers, two per lane, and
// hands each finished unknown to the other lanes by a shuffle, so no row ends in a group barrier;
// the other warps wait at one barrier at the end.  The forward sweep keeps the last min(N, 32)
// rows in one register (lane l: row N - 32 + l) and the backward sweep the first 32 (lane l: row
// l), so that while at most 32 rows are open each step is one FMA instruction.  Every row sees
// the same operations in the same order as in the shared-memory sweeps below (both write the
// updates as explicit FMAs), so the two sweeps give bitwise the same solution.
template <int G>
__device__ void lu_solve_regs(const Grp<G>& g, const double* M, int N, int LD, const int* perm,
                              const double* invd, double* b, double* t) {
  if (g.tid < 32) {
    constexpr unsigned F = 0xffffffffu;
    const int l = g.tid;
    // forward sweep, L y = P b (unit diagonal): set B rows [0, nb), set A rows [nb, N)
    const int nb = N > 32 ? N - 32 : 0, na = N - nb;
    const bool hb = l < nb, ha = l < na;
    const int rb = hb ? perm[l] : 0, ra = ha ? perm[nb + l] : 0;
    const double* Lb = M + rb * LD;
    const double* La = M + ra * LD;
    double tb = hb ? b[rb] : 0.0;
    double ta = ha ? b[ra] : 0.0;
    for (int k = 0; k < nb - 1; ++k) {             // rows of both sets still open
      const double xk = __shfl_sync(F, tb, k);
      if (hb && l > k) tb = fma(-Lb[k], xk, tb);
      if (ha) ta = fma(-La[k], xk, ta);
    }
    if (nb > 0) {                                  // the last row of set B
      const double xk = __shfl_sync(F, tb, nb - 1);
      if (ha) ta = fma(-La[nb - 1], xk, ta);
    }
#pragma unroll 4
    for (int k = nb; k < N - 1; ++k) {
      const double xk = __shfl_sync(F, ta, k - nb);
      if (ha && nb + l > k) ta = fma(-La[k], xk, ta);
    }
    // the backward sweep's layout: set 1 rows [0, min(N, 32)), set 2 rows [32, N)
    if (hb) t[l] = tb;
    if (ha) t[nb + l] = ta;
    __syncwarp();
    const int n1 = N < 32 ? N : 32;
    const bool h1 = l < n1, h2 = 32 + l < N;
    double u1 = h1 ? t[l] : 0.0;
    double u2 = h2 ? t[32 + l] : 0.0;
    const double* U1 = M + (h1 ? perm[l] : 0) * LD;
    const double* U2 = M + (h2 ? perm[32 + l] : 0) * LD;
    const double d1 = h1 ? invd[l] : 0.0, d2 = h2 ? invd[32 + l] : 0.0;
    // U x = y, column by column; a row is final once scaled by the reciprocal of its pivot
    if (N > 32) {
      if (32 + l == N - 1) u2 *= d2;
    } else {
      if (l == N - 1) u1 *= d1;
    }
    for (int k = N - 1; k > 32; --k) {             // rows of both sets still open
      const double xk = __shfl_sync(F, u2, k - 32);
      if (32 + l < k) {
        double v = fma(-U2[k], xk, u2);
        if (32 + l == k - 1) v *= d2;
        u2 = v;
      }
      u1 = fma(-U1[k], xk, u1);
    }
    if (N > 32) {                                  // the first row of set 2
      const double xk = __shfl_sync(F, u2, 0);
      double v = fma(-U1[32], xk, u1);
      if (l == 31) v *= d1;
      u1 = v;
    }
#pragma unroll 4
    for (int k = n1 - 1; k > 0; --k) {
      const double xk = __shfl_sync(F, u1, k);
      if (l < k) {
        double v = fma(-U1[k], xk, u1);
        if (l == k - 1) v *= d1;
        u1 = v;
      }
    }
    if (h1) b[l] = u1;
    if (h2) b[32 + l] = u2;
  }
  g.sync();
}

// Solves A x = b with the factors of lu_factor; b (length N) is overwritten with x.  t: N-double
// scratch holding the permuted right-hand side during the two triangular sweeps.  The division
// by the diagonal of U happens once per row, in the thread that finishes that row.
template <int G>
__device__ void lu_solve(const Grp<G>& g, const double* M, int N, int LD, const int* perm,
                         const double* invd, double* b, double* t) {
  if constexpr (G >= 32) {
    if (N <= 64) {
      lu_solve_regs<G>(g, M, N, LD, perm, invd, b, t);
      return;
    }
  }
  for (int i = g.tid; i < N; i += G) t[i] = b[perm[i]];
  g.sync();
  for (int k = 0; k < N - 1; ++k) {          // L y = P b (unit diagonal)
    const double xk = t[k];
    for (int i = k + 1 + g.tid; i < N; i += G) t[i] = fma(-M[perm[i] * LD + k], xk, t[i]);
    g.sync();
  }
  if (g.tid == 0) t[N - 1] *= invd[N - 1];
  g.sync();
  for (int k = N - 1; k >= 0; --k) {         // U x = y, column by column
    const double xk = t[k];
    if (g.tid == 0) b[k] = xk;
    for (int i = g.tid; i < k; i += G) {
      double v = fma(-M[perm[i] * LD + k], xk, t[i]);
      if (i == k - 1) v *= invd[i];
      t[i] = v;
    }
    g.sync();
  }
}

// ---------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------
// One independent set of cells advanced by a launch: its own state arrays, step and
// tolerances, optional index list and outputs.  A launch walks the chunks of all its segments
// through one work queue (iteration-level batching of several requests).
struct Segment {
  double* T;
  const double* p;
  double* Y;
  int64_t ld, ncells;
  const int32_t* idx;
  int8_t* status;
  int32_t* nsub;
  int32_t* nrej;
  double dt, rtol, atol;
  long long chunk_begin;           // first queue entry of this segment
};

constexpr int kMaxSegs = kMaxSegsPerLaunch;   // segments per launch (kernel-parameter space)

struct AdvanceParams {
  MechLayout lay;
  WsLayout ws;
  JacArgs jp;
  const unsigned char* blob;
  Segment segs[kMaxSegs];
  int nseg;
  long long total_chunks;
  int max_steps;
  unsigned long long* counter;
  const unsigned int* ncells_dev;  // single segment: cell count read from device memory
  unsigned long long budget_ns = 0;  // > 0: stop claiming chunks this long after the group started
  // time-sliced launches: a nonzero *stop (device memory, set by the caller while the slice runs)
  // also stops the claiming, once the group has run min_ns
  const unsigned int* stop = nullptr;
  unsigned long long min_ns = 0;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void stage_mech(const unsigned char* src, unsigned char* dst, int bytes) {
  const int4* s = (const int4*)src;
  int4* d = (int4*)dst;
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

// One Rodas4 attempt from w.y with step h (f and J re-evaluated at w.y).  Returns false on an
// exactly singular iteration matrix; otherwise *en receives the error norm and *fac the step-size
// factor 0.9 en^(-1/4) (clamped below at 0.2; 0.2 for a non-finite norm), evaluated once per
// group.
template <int G>
__device__ bool rodas4_attempt(const Grp<G>& g, const MechView& m, const WsPtr& w,
                               const AdvanceParams& P, double p, double h, double rtol, double atol,
                               double* en, double* fac) {
  constexpr bool kMulti = G > 32;
  const int N = m.N, LD = P.ws.LD;
  double ig = 0.0, invh = 0.0;
  if (is_lead(g)) { ig = 1.0 / (kGamma * h); invh = 1.0 / h; }
  if (kMulti && g.tid == 0) { w.sc[S_IG] = ig; w.sc[S_INVH] = invh; }
  eval_fj<G>(g, m, w, P.jp, LD, w.y, p, w.f0, w.M);      // M = -J; synchronises
  if (kMulti) { ig = w.sc[S_IG]; invh = w.sc[S_INVH]; }
  for (int i = g.tid; i < N; i += G) w.M[i * LD + i] += ig;   // M = I / (gamma h) - J
  g.sync();
  bool regular;
  if constexpr (G > 32) {
    regular = N <= 64 ? lu_factor_panel<G>(g, w.M, N, LD, w.perm, w.invd, (int*)w.ys, (int*)w.red)
                      : lu_factor<G>(g, w.M, N, LD, w.perm, w.invd, w.red);
  } else {
    regular = lu_factor<G>(g, w.M, N, LD, w.perm, w.invd, w.red);
  }
  if (!regular) return false;
  for (int s = 0; s < 6; ++s) {
    const double* src = w.f0;
    if (s > 0) {
      for (int i = g.tid; i < N; i += G) {
        double v = w.y[i];
        for (int j = 0; j < s; ++j) v += kRA[s][j] * w.u[j * N + i];
        w.ys[i] = v;
      }
      g.sync();
      eval_fj<G>(g, m, w, P.jp, LD, w.ys, p, w.fs, nullptr);
      src = w.fs;
    }
    double* us = w.u + s * N;
    for (int i = g.tid; i < N; i += G) {
      double v = src[i];
      for (int j = 0; j < s; ++j) v += (kRC[s][j] * invh) * w.u[j * N + i];
      us[i] = v;
    }
    g.sync();
    lu_solve<G>(g, w.M, N, LD, w.perm, w.invd, us, w.tmp);
  }
  double acc[1] = {0.0};
  for (int i = g.tid; i < N; i += G) {
    double v = w.y[i];
#pragma unroll
    for (int s = 0; s < 6; ++s) v += kRM[s] * w.u[s * N + i];
    w.ynew[i] = v;
    const double sc = atol + rtol * fmax(fabs(w.y[i]), fabs(v));
    const double r = w.u[5 * N + i] / sc;
    acc[0] += r * r;
  }
  gsum_lead<G, 1>(g, acc, w.red, N);
  double e = 0.0, f = 0.0;
  if (is_lead(g)) {
    e = sqrt(acc[0] / (double)N);
    f = 0.2;
    if (isfinite(e)) {
      f = 0.9 * pow(e, -0.25);
      if (f < 0.2) f = 0.2;
    }
  }
  if (kMulti) {
    if (g.tid == 0) { w.sc[S_EN] = e; w.sc[S_FAC] = f; }
    g.sync();
    e = w.sc[S_EN]; f = w.sc[S_FAC];
  }
  *en = e;
  *fac = f;
  return true;
}

// Chunk bookkeeping of one group: the current chunk of up to chunk_cells(G) consecutive cells of one
// segment, staged in shared memory, and the position of the cell being integrated.
struct ChunkPos {
  const Segment* seg;
  long long base;
  int nloc, c;
  bool exhausted;
  long long total;      // queue entries (chunks) of the launch
  unsigned long long t0;  // group start time (time-sliced launches)
};

__device__ __forceinline__ int64_t cell_of(const Segment* S, long long base, int c) {
  return S->idx ? (int64_t)S->idx[base + c] : (int64_t)(base + c);
}

__device__ __forceinline__ const Segment* segment_of(const AdvanceParams& P, long long chunk) {
  int s = 0;
  while (s + 1 < P.nseg && P.segs[s + 1].chunk_begin <= chunk) ++s;
  return &P.segs[s];
}

// Move to the next cell: store a finished chunk, claim and load the next one when needed.
// Loads the cell's state into w.y and returns its pressure; false when the queue is empty.
template <int G>
__device__ bool next_cell(const Grp<G>& g, const MechView& m, const WsPtr& w,
                          const AdvanceParams& P, ChunkPos& q, double* p) {
  constexpr int CHUNK = chunk_cells(G);
  const int N = m.N;
  for (;;) {
    if (q.c + 1 < q.nloc) {
      ++q.c;
      for (int i = g.tid; i < N; i += G) w.y[i] = w.stage[i * CHUNK + q.c];
      *p = w.stage[N * CHUNK + q.c];
      g.sync();
      return true;
    }
    if (q.nloc > 0) {
      // coalesced store of the finished chunk (rows T, Y_1..Y_ns)
      const Segment* S = q.seg;
      for (int e = g.tid; e < N * CHUNK; e += G) {
        const int row = e / CHUNK, c = e % CHUNK;
        if (c >= q.nloc) continue;
        const int64_t cell = cell_of(S, q.base, c);
        const double v = w.stage[row * CHUNK + c];
        if (row == 0) S->T[cell] = v;
        else S->Y[(int64_t)(row - 1) * S->ld + cell] = v;
      }
      q.nloc = 0;
      g.sync();
    }
    if (q.exhausted) return false;
    // a time-sliced launch stops claiming once its budget is spent or its caller asks it to stop:
    // the chunks claimed so far are exactly the prefix [0, counter) of the queue, and the next
    // slice continues from there
    if (g.tid == 0) {
      bool stop = false;
      if (P.budget_ns > 0) {
        const unsigned long long el = global_ns() - q.t0;
        stop = el > P.budget_ns || (P.stop && el > P.min_ns && *(const volatile unsigned int*)P.stop != 0u);
      }
      w.ctl[0] = stop ? ~0ull : atomicAdd(P.counter, 1ull);
    }
    g.sync();
    const unsigned long long claimed = w.ctl[0];      // ~0 when the time budget is spent
    g.sync();
    if (claimed >= (unsigned long long)q.total) {
      q.exhausted = true;
      return false;
    }
    const long long chunk = (long long)claimed;
    const Segment* S = segment_of(P, chunk);
    const long long ncs = P.ncells_dev ? min((long long)*P.ncells_dev, (long long)S->ncells)
                                       : (long long)S->ncells;
    q.seg = S;
    q.base = (chunk - S->chunk_begin) * CHUNK;
    q.nloc = (int)min((long long)CHUNK, ncs - q.base);
    q.c = -1;
    // coalesced load of the chunk: rows T, Y_1..Y_ns, p; each row CHUNK consecutive cells
    for (int e = g.tid; e < (N + 1) * CHUNK; e += G) {
      const int row = e / CHUNK, c = e % CHUNK;
      if (c >= q.nloc) continue;
      const int64_t cell = cell_of(S, q.base, c);
      double v;
      if (row == 0) v = S->T[cell];
      else if (row <= m.ns) v = S->Y[(int64_t)(row - 1) * S->ld + cell];
      else v = S->p[cell];
      w.stage[row * CHUNK + c] = v;
    }
    g.sync();
  }
}

// Persistent integrator.  Each loop iteration performs at most one Rodas4 attempt per group;
// cell changes happen between iterations.  For sub-warp groups every group of a warp executes
// the attempt body each iteration (an idle group works on a dummy state whose results are
// discarded), so the warp's FP64 instructions stay converged across its groups.
template <int G>
__global__ void __launch_bounds__(max_threads(G), 1) advance_kernel(const __grid_constant__ AdvanceParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (blockDim.x % G != 0 || blockDim.x < G) return;   // a block of whole groups only
  stage_mech(P.blob, smem, P.lay.bytes);
  __syncthreads();
  const MechView m = bind_mech(smem, P.lay);
  Grp<G> g;
  g.init();
  double* wbase = (double*)(smem + P.lay.bytes) + (size_t)g.gid * P.ws.total;
  const WsPtr w = bind_ws(wbase, P.ws);
  const int N = m.N;
  // benign dummy state for groups without a cell
  for (int i = g.tid; i < N; i += G) w.y[i] = i == 0 ? 1000.0 : 1.0 / m.ns;
  g.sync();

  constexpr int CHUNK = chunk_cells(G);
  long long total = P.total_chunks;
  if (P.ncells_dev)
    total = (min((long long)*P.ncells_dev, (long long)P.segs[0].ncells) + CHUNK - 1) / CHUNK;
  ChunkPos q{&P.segs[0], 0, 0, 0, false, total, P.budget_ns > 0 ? global_ns() : 0ull};
  bool active = false;
  double dt = 1.0, rtol = 1e-6, atol = 1e-10;
  double p = 1.0e6, t = 0.0, h = dt, facmax = 6.0;
  int attempts = 0, nacc = 0, nrej = 0;

  for (;;) {
    // ---- cell management (group-local) ----
    while (!active) {
      if (!next_cell<G>(g, m, w, P, q, &p)) break;
      double bad[1] = {0.0};
      for (int i = g.tid; i < N; i += G) {
        const double v = w.y[i];
        if (!isfinite(v) || (i == 0 && !(v > 0.0))) bad[0] += 1.0;
      }
      if (g.tid == 0 && (!isfinite(p) || !(p > 0.0))) bad[0] += 1.0;
      gsum<G, 1>(g, bad, w.red);
      if (bad[0] != 0.0) {
        if (g.tid == 0) {
          const Segment* S = q.seg;
          const int64_t cell = cell_of(S, q.base, q.c);
          if (S->status) S->status[cell] = (int8_t)CHEM_CELL_NONFINITE;
          if (S->nsub) S->nsub[cell] = 0;
          if (S->nrej) S->nrej[cell] = 0;
        }
        for (int i = g.tid; i < N; i += G) w.y[i] = i == 0 ? 1000.0 : 1.0 / m.ns;
        g.sync();
        continue;
      }
      active = true;
      dt = q.seg->dt; rtol = q.seg->rtol; atol = q.seg->atol;
      t = 0.0; h = dt; facmax = 6.0;
      attempts = 0; nacc = 0; nrej = 0;
    }
    if (G >= 32) {
      if (!active) break;
    } else {
      if (__all_sync(0xffffffffu, !active)) break;
    }

    // ---- one attempt ----
    int status = CHEM_CELL_OK;
    bool stop = false, last = false;
    if (active) {
      if (attempts >= P.max_steps) {
        stop = true; status = CHEM_CELL_MAX_STEPS;
      } else {
        if (h >= dt - t) { h = dt - t; last = true; }
        if (h < 1e-12 * dt) { stop = true; status = CHEM_CELL_H_UNDERFLOW; }
      }
    }
    const bool run = active && !stop;
    bool finished = false;
    if (run || G < 32) {
      double en = 0.0, fac = 0.2;
      const bool ok = rodas4_attempt<G>(g, m, w, P, p, run ? h : dt, rtol, atol, &en, &fac);
      if (run) {
        if (!ok) {
          stop = true; status = CHEM_CELL_SINGULAR_LU;
        } else {
          ++attempts;
          if (en <= 1.0) {
            for (int i = g.tid; i < N; i += G) w.y[i] = w.ynew[i];
            g.sync();
            ++nacc;
            if (last) {
              finished = true;
            } else {
              t += h;
              h = h * fmin(fac, facmax);
              facmax = 6.0;
            }
          } else {
            ++nrej;
            h = h * fac;
            facmax = 1.0;
          }
        }
      }
    }
    if (active && (stop || finished)) {
      // the last accepted state goes back into the chunk staging area
      for (int i = g.tid; i < N; i += G) w.stage[i * CHUNK + q.c] = w.y[i];
      if (g.tid == 0) {
        const Segment* S = q.seg;
        const int64_t cell = cell_of(S, q.base, q.c);
        if (S->status) S->status[cell] = (int8_t)status;
        if (S->nsub) S->nsub[cell] = nacc;
        if (S->nrej) S->nrej[cell] = nrej;
      }
      g.sync();
      active = false;
    }
    if (G < 32) __syncwarp();
  }
}

struct EvalParams {
  MechLayout lay;
  WsLayout ws;
  JacArgs jp;
  const unsigned char* blob;
  const double* T;
  const double* p;
  const double* Y;
  int64_t ld, ncells;
  double* f;
  double* J;
};

template <int G>
__global__ void __launch_bounds__(max_threads(G)) eval_kernel(const EvalParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (blockDim.x % G != 0 || blockDim.x < G) return;   // a block of whole groups only
  stage_mech(P.blob, smem, P.lay.bytes);
  __syncthreads();
  const MechView m = bind_mech(smem, P.lay);
  Grp<G> g;
  g.init();
  const int gpb = blockDim.x / G;
  double* wbase = (double*)(smem + P.lay.bytes) + (size_t)g.gid * P.ws.total;
  const WsPtr w = bind_ws(wbase, P.ws);
  const int N = m.N, LD = P.ws.LD;
  for (int64_t c = (int64_t)blockIdx.x * gpb + g.gid; c < P.ncells; c += (int64_t)gridDim.x * gpb) {
    for (int i = g.tid; i < N; i += G) w.y[i] = i == 0 ? P.T[c] : P.Y[(int64_t)(i - 1) * P.ld + c];
    g.sync();
    eval_fj<G>(g, m, w, P.jp, LD, w.y, P.p[c], w.f0, P.J ? w.M : nullptr);
    for (int i = g.tid; i < N; i += G) P.f[(int64_t)i * P.ld + c] = w.f0[i];
    if (P.J)     // the kernel assembles -J (exact negation back)
      for (int e = g.tid; e < N * N; e += G)
        P.J[(int64_t)e * P.ld + c] = -w.M[(e / N) * LD + e % N];
    g.sync();
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
namespace {

struct LaunchShape {
  int G, groups, threads;
  size_t smem;
  WsLayout ws;
};


int pick_shape(const chem_mech_s* m, const chem_options* opt, LaunchShape* s) {
  const int N = m->ns + 1;
  int G = (opt && opt->group_threads) ? opt->group_threads : (N <= 16 ? 2 : 128);
  if (G != 2 && G != 4 && G != 8 && G != 16 && G != 32 && G != 64 && G != 128 && G != 256) {
    set_error("group_threads must be 2, 4, 8, 16, 32, 64, 128 or 256 (got %d)", G);
    return CHEM_EINVAL;
  }
  s->G = G;
  s->ws = make_ws(m->ns, m->nr, m->lay.npieces, G);
  int dev = 0;
  CHEM_CUDA_TRY(cudaGetDevice(&dev));
  int smem_max = 0;
  CHEM_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t per_group = (size_t)s->ws.total * 8;
  const size_t fixed = (size_t)m->lay.bytes;
  const int unit = G < 32 ? 32 / G : 1;          // groups per warp: whole warps only
  int groups = (opt && opt->groups_per_cta) ? opt->groups_per_cta : max_threads(G) / G;
  groups = std::min(groups, max_threads(G) / G);
  if (G > 32) groups = std::min(groups, 15);     // named barriers 1..15
  while (groups > unit && fixed + per_group * groups > (size_t)smem_max) groups -= unit;
  groups = std::max(unit, (groups / unit) * unit);
  if (fixed + per_group * groups > (size_t)smem_max) {
    set_error("mechanism too large for shared memory (%zu bytes needed, %d available)",
              fixed + per_group * groups, smem_max);
    return CHEM_EINVAL;
  }
  s->groups = groups;
  s->threads = G * groups;
  s->smem = fixed + per_group * groups;
  return CHEM_OK;
}

template <int G>
int launch_adv_t(const LaunchShape& s, const AdvanceParams& P, const chem_options* opt,
                 cudaStream_t stream) {
  CHEM_CUDA_TRY(cudaFuncSetAttribute(advance_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)s.smem));
  int dev = 0, sms = 0, per_sm = 0;
  CHEM_CUDA_TRY(cudaGetDevice(&dev));
  CHEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CHEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, advance_kernel<G>, s.threads, s.smem));
  if (per_sm < 1) { set_error("kernel does not fit on an SM"); return CHEM_EINVAL; }
  int64_t chunks = P.total_chunks;     // an upper bound when the count is read on the device
  int64_t grid = (int64_t)sms * per_sm;
  int threads = s.threads;
  size_t smem = s.smem;
  const bool shaped = opt && (opt->groups_per_cta > 0 || opt->max_ctas > 0);
  if (!shaped && chunks < grid * s.groups) {
    // fewer chunks than group slots: spread the groups over every SM (fewer groups per CTA)
    // rather than filling a few SMs, so that a cell shares its SM's FP64 pipe with fewer others
    const int unit = G < 32 ? 32 / G : 1;
    int64_t gpc = (chunks + grid - 1) / grid;
    gpc = std::max<int64_t>(unit, (gpc + unit - 1) / unit * unit);
    gpc = std::min<int64_t>(gpc, s.groups);
    threads = G * (int)gpc;
    smem = s.smem - (size_t)s.ws.total * 8 * (size_t)(s.groups - gpc);
    grid = (chunks + gpc - 1) / gpc;
  } else {
    if (opt && opt->max_ctas > 0) grid = std::min<int64_t>(grid, opt->max_ctas);
    grid = std::min<int64_t>(grid, (chunks + s.groups - 1) / s.groups);
  }
  if (grid < 1) grid = 1;
  advance_kernel<G><<<(unsigned)grid, threads, smem, stream>>>(P);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

template <int G>
int launch_eval_t(const LaunchShape& s, const EvalParams& P, cudaStream_t stream) {
  CHEM_CUDA_TRY(cudaFuncSetAttribute(eval_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)s.smem));
  int64_t grid = (P.ncells + s.groups - 1) / s.groups;
  grid = std::min<int64_t>(grid, 65535);
  eval_kernel<G><<<(unsigned)grid, s.threads, s.smem, stream>>>(P);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

int dispatch_adv(const LaunchShape& s, const AdvanceParams& P, const chem_options* opt,
                 cudaStream_t stream) {
  switch (s.G) {
    case 2: return launch_adv_t<2>(s, P, opt, stream);
    case 4: return launch_adv_t<4>(s, P, opt, stream);
    case 8: return launch_adv_t<8>(s, P, opt, stream);
    case 16: return launch_adv_t<16>(s, P, opt, stream);
    case 32: return launch_adv_t<32>(s, P, opt, stream);
    case 64: return launch_adv_t<64>(s, P, opt, stream);
    case 128: return launch_adv_t<128>(s, P, opt, stream);
    case 256: return launch_adv_t<256>(s, P, opt, stream);
    default: set_error("no kernel for group_threads %d", s.G); return CHEM_EINVAL;
  }
}

JacArgs jac_args(const chem_mech_s* m) {
  JacArgs j;
  j.nent = m->jac.nent;
  j.ent_off = m->jac.ent_off;
  j.ent_row = m->jac.ent_row;
  j.ent_col = m->jac.ent_col;
  j.term_src = m->jac.term_src;
  j.term_oth = m->jac.term_oth;
  j.term_coef = m->jac.term_coef;
  return j;
}

}  // namespace

int launch_advance(chem_mech_s* m, double* T, const double* p, double* Y, int64_t ld, double dt,
                   int64_t ncells, double rtol, double atol, const int32_t* idx, int8_t* status,
                   int32_t* nsub, int32_t* nrej, const chem_options* opt, cudaStream_t stream,
                   unsigned int* /*unused*/) {
  if (!m) { set_error("NULL mechanism"); return CHEM_EINVAL; }
  if (ncells < 0 || !(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0) || !std::isfinite(dt)) {
    set_error("invalid arguments (ncells=%lld dt=%g rtol=%g atol=%g)", (long long)ncells, dt, rtol, atol);
    return CHEM_EINVAL;
  }
  if (ncells == 0) return CHEM_OK;
  if (!T || !p || !Y) { set_error("NULL state pointer"); return CHEM_EINVAL; }
  if (!idx && ld < ncells) { set_error("ld (%lld) < ncells (%lld)", (long long)ld, (long long)ncells); return CHEM_EINVAL; }
  LaunchShape s;
  int rc = pick_shape(m, opt, &s);
  if (rc) return rc;
  unsigned long long* counter = nullptr;
  CHEM_CUDA_TRY(cudaMallocAsync((void**)&counter, sizeof(unsigned long long), stream));
  CHEM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream));
  AdvanceParams P;
  P.lay = m->lay; P.ws = s.ws; P.jp = jac_args(m); P.blob = (const unsigned char*)m->d_blob;
  P.segs[0] = Segment{T, p, Y, ld, ncells, idx, status, nsub, nrej, dt, rtol, atol, 0};
  P.nseg = 1;
  P.total_chunks = (ncells + chunk_cells(s.G) - 1) / chunk_cells(s.G);
  P.max_steps = (opt && opt->max_steps > 0) ? opt->max_steps : 100000;
  P.counter = counter;
  P.ncells_dev = nullptr;
  P.budget_ns = 0;
  rc = dispatch_adv(s, P, opt, stream);
  cudaError_t fe = cudaFreeAsync(counter, stream);
  if (rc) return rc;
  CHEM_CUDA_TRY(fe);
  return CHEM_OK;
}

// Indexed integrator launch whose cell count (<= capacity) is read from device memory by the
// kernel: the surrogate's fallback pass runs without a host round trip.
int launch_advance_counted(chem_mech_s* m, double* T, const double* p, double* Y, int64_t ld,
                           double dt, int64_t capacity, const unsigned int* count_dev, double rtol,
                           double atol, const int32_t* idx, cudaStream_t stream) {
  if (!m || !count_dev || !idx) { set_error("NULL argument"); return CHEM_EINVAL; }
  if (capacity <= 0) return CHEM_OK;
  LaunchShape s;
  int rc = pick_shape(m, nullptr, &s);
  if (rc) return rc;
  unsigned long long* counter = nullptr;
  CHEM_CUDA_TRY(cudaMallocAsync((void**)&counter, sizeof(unsigned long long), stream));
  CHEM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream));
  AdvanceParams P;
  P.lay = m->lay; P.ws = s.ws; P.jp = jac_args(m); P.blob = (const unsigned char*)m->d_blob;
  P.segs[0] = Segment{T, p, Y, ld, capacity, idx, nullptr, nullptr, nullptr, dt, rtol, atol, 0};
  P.nseg = 1;
  P.total_chunks = (capacity + chunk_cells(s.G) - 1) / chunk_cells(s.G);
  P.max_steps = 100000;
  P.counter = counter;
  P.ncells_dev = count_dev;
  P.budget_ns = 0;
  rc = dispatch_adv(s, P, nullptr, stream);
  cudaError_t fe = cudaFreeAsync(counter, stream);
  if (rc) return rc;
  CHEM_CUDA_TRY(fe);
  return CHEM_OK;
}

// Batched launch: the chunks of all segments go through one work queue of one persistent
// launch (segment descriptors travel in the kernel parameters, kMaxSegs per launch; a larger
// batch becomes consecutive launches on the stream).
int launch_advance_batch(chem_mech_s* m, const chem_segment* segs, int nseg, cudaStream_t stream) {
  if (!m || !segs || nseg < 1) { set_error("bad batch arguments"); return CHEM_EINVAL; }
  for (int i = 0; i < nseg; ++i) {
    const chem_segment& a = segs[i];
    if (a.ncells < 0 || !(a.dt > 0.0) || !(a.rtol > 0.0) || !(a.atol > 0.0) || !std::isfinite(a.dt) ||
        (a.ncells > 0 && (!a.T || !a.p || !a.Y)) || (!a.idx && a.ld < a.ncells)) {
      set_error("segment %d: invalid arguments", i);
      return CHEM_EINVAL;
    }
  }
  LaunchShape s;
  int rc = pick_shape(m, nullptr, &s);
  if (rc) return rc;
  for (int first = 0; first < nseg; first += kMaxSegs) {
    const int cnt = std::min(kMaxSegs, nseg - first);
    AdvanceParams P;
    P.lay = m->lay; P.ws = s.ws; P.jp = jac_args(m); P.blob = (const unsigned char*)m->d_blob;
    long long total = 0;
    for (int i = 0; i < cnt; ++i) {
      const chem_segment& a = segs[first + i];
      P.segs[i] = Segment{a.T, a.p, a.Y, a.ld, a.ncells, a.idx, a.status, a.nsub, a.nrej, a.dt, a.rtol, a.atol, total};
      total += (a.ncells + chunk_cells(s.G) - 1) / chunk_cells(s.G);
    }
    if (total == 0) continue;
    P.nseg = cnt;
    P.total_chunks = total;
    P.max_steps = 100000;
    P.ncells_dev = nullptr;
    P.budget_ns = 0;
    unsigned long long* counter = nullptr;
    CHEM_CUDA_TRY(cudaMallocAsync((void**)&counter, sizeof(unsigned long long), stream));
    CHEM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream));
    P.counter = counter;
    rc = dispatch_adv(s, P, nullptr, stream);
    cudaError_t fe = cudaFreeAsync(counter, stream);
    if (rc) return rc;
    CHEM_CUDA_TRY(fe);
  }
  return CHEM_OK;
}

// Work-queue entries (chunks) of ncells cells in a default-shape launch for mechanism m: the
// queue end of a segment appended to a time-sliced job
long long advance_queue_chunks(chem_mech_s* m, int64_t ncells) {
  LaunchShape s;
  if (pick_shape(m, nullptr, &s) != CHEM_OK) return -1;
  return (ncells + chunk_cells(s.G) - 1) / chunk_cells(s.G);
}

// One time slice of a batched launch whose work-queue counter the caller owns (zeroed before the
// first slice).  Groups stop claiming chunks budget_ns after they start; the chunks claimed so far
// form the prefix [0, counter) of the queue, so re-issuing the same slice continues the work and
// a segment is complete once the counter reaches seg_end[i] (its last chunk + 1, written here).
// A slice issued after the counter reached the total returns at once.  stop (nullable, device
// memory): a nonzero value ends the slice early the same way, for groups that have run min_ns.
int launch_advance_slice(chem_mech_s* m, const chem_segment* segs, int nseg, unsigned long long budget_ns,
                         unsigned long long* counter, long long* seg_end, cudaStream_t stream,
                         const unsigned int* stop, unsigned long long min_ns) {
  if (!m || !segs || nseg < 1 || nseg > kMaxSegs || !counter) { set_error("bad slice arguments"); return CHEM_EINVAL; }
  LaunchShape s;
  int rc = pick_shape(m, nullptr, &s);
  if (rc) return rc;
  AdvanceParams P;
  P.lay = m->lay; P.ws = s.ws; P.jp = jac_args(m); P.blob = (const unsigned char*)m->d_blob;
  long long total = 0;
  for (int i = 0; i < nseg; ++i) {
    const chem_segment& a = segs[i];
    if (a.ncells < 0 || !(a.dt > 0.0) || !(a.rtol > 0.0) || !(a.atol > 0.0) || !std::isfinite(a.dt) ||
        (a.ncells > 0 && (!a.T || !a.p || !a.Y)) || (!a.idx && a.ld < a.ncells)) {
      set_error("segment %d: invalid arguments", i);
      return CHEM_EINVAL;
    }
    P.segs[i] = Segment{a.T, a.p, a.Y, a.ld, a.ncells, a.idx, a.status, a.nsub, a.nrej, a.dt, a.rtol, a.atol, total};
    total += (a.ncells + chunk_cells(s.G) - 1) / chunk_cells(s.G);
    if (seg_end) seg_end[i] = total;
  }
  if (total == 0) return CHEM_OK;
  P.nseg = nseg;
  P.total_chunks = total;
  P.max_steps = 100000;
  P.counter = counter;
  P.ncells_dev = nullptr;
  P.budget_ns = budget_ns;
  P.stop = stop;
  P.min_ns = min_ns;
  return dispatch_adv(s, P, nullptr, stream);
}

// FP64 FMA throughput probe: 8 independent dependency chains per thread
__global__ void fma_peak_kernel(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
  double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 12345.678) out[0] = s;     // keeps the chains live
}

// The integrator's table-driven exponential applied elementwise (testing and measurement)
__global__ void fast_exp_kernel(const double* x, double* y, int64_t n) {
  __shared__ double tab[64];
  stage_exp_table(tab);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = exp_tab(x[i], tab);
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the integrator launch.
//
// The work queue of the persistent kernel needs one zeroed 8-byte counter per launch; the
// regular entry points draw it from the stream-ordered allocator.  Callers that may not
// allocate device memory (a flow solver that has already claimed the device memory for its own
// fields and pools, code running under a hard allocation budget, or a latency-critical loop that
// must not touch the allocator) use chem_advance_noalloc instead, which takes the counter from
// this file-scope array.  Every GPU that loads the library holds the array until the process
// exits.  All calls share it, so calls that overlap on the GPU race on the counter.
// ---------------------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = 256;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocScratchBytes / 8];

namespace {
constexpr int kMaxDevices = 64;

// Device address of g_noalloc_scratch per device, remembered together with the context it was
// looked up in.  In host code the array's name is only a host-side stand-in, so the address must
// come from cudaGetSymbolAddress with the device current.  A context reset (cudaDeviceReset, a
// destroyed primary context) reloads the module at another address: a call made in a context
// other than the remembered one looks the address up again.  The lock makes first calls from
// several host threads safe.
struct NoallocCache {
  std::mutex mu;
  CUcontext ctx[kMaxDevices] = {};
  void* ptr[kMaxDevices] = {};
};
NoallocCache g_noalloc;

// cuCtxGetCurrent through the runtime's driver entry-point query: the library does not link the
// driver library itself (it loads on hosts without a GPU driver)
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn ctx_get_current_fn() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  });
  return fn;
}

int noalloc_scratch(void** out) {
  int dev = 0;
  CHEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d out of range for the allocation-free entry point", dev);
    return CHEM_EINVAL;
  }
  CtxGetCurrentFn get_ctx = ctx_get_current_fn();
  if (!get_ctx) {
    set_error("allocation-free entry point: cuCtxGetCurrent unavailable");
    return CHEM_ECUDA;
  }
  CUcontext ctx = nullptr;
  if (get_ctx(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  std::lock_guard<std::mutex> lk(g_noalloc.mu);
  if (!ctx || g_noalloc.ctx[dev] != ctx || !g_noalloc.ptr[dev]) {
    // the look-up also initialises the device's primary context when nothing else has yet
    void* ptr = nullptr;
    CHEM_CUDA_TRY(cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch));
    if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) {
      set_error("allocation-free entry point: no current CUDA context");
      return CHEM_ECUDA;
    }
    g_noalloc.ptr[dev] = ptr;
    g_noalloc.ctx[dev] = ctx;
  }
  *out = g_noalloc.ptr[dev];
  return CHEM_OK;
}
}  // namespace

int launch_advance_noalloc(chem_mech_s* m, double* T, const double* p, double* Y, int64_t ld,
                           double dt, int64_t ncells, double rtol, double atol, int8_t* status,
                           int32_t* nsub, int32_t* nrej, cudaStream_t stream) {
  if (!m) { set_error("NULL mechanism"); return CHEM_EINVAL; }
  if (ncells < 0 || !(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0) || !std::isfinite(dt)) {
    set_error("invalid arguments (ncells=%lld dt=%g rtol=%g atol=%g)", (long long)ncells, dt, rtol, atol);
    return CHEM_EINVAL;
  }
  if (!T || !p || !Y) { set_error("NULL state pointer"); return CHEM_EINVAL; }
  if (ld < ncells) { set_error("ld (%lld) < ncells (%lld)", (long long)ld, (long long)ncells); return CHEM_EINVAL; }
  // scratch needed by one launch: the work-queue counter, independent of ncells
  const size_t need = sizeof(unsigned long long);
  if (need > kNoAllocScratchBytes) {
    set_error("allocation-free integrator needs %zu scratch bytes, only %zu available", need,
              kNoAllocScratchBytes);
    return CHEM_EINVAL;
  }
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  if (ncells == 0) return CHEM_OK;
  LaunchShape s;
  rc = pick_shape(m, nullptr, &s);
  if (rc) return rc;
  unsigned long long* counter = (unsigned long long*)scratch;
  CHEM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream));
  AdvanceParams P;
  P.lay = m->lay; P.ws = s.ws; P.jp = jac_args(m); P.blob = (const unsigned char*)m->d_blob;
  P.segs[0] = Segment{T, p, Y, ld, ncells, nullptr, status, nsub, nrej, dt, rtol, atol, 0};
  P.nseg = 1;
  P.total_chunks = (ncells + chunk_cells(s.G) - 1) / chunk_cells(s.G);
  P.max_steps = 100000;
  P.counter = counter;
  P.ncells_dev = nullptr;
  P.budget_ns = 0;
  return dispatch_adv(s, P, nullptr, stream);
}

}  // namespace chem

using namespace chem;

extern "C" int chem_advance_noalloc(chem_mech_t m, double* T, const double* p, double* Y,
                                    int64_t ld, double dt, int64_t ncells, double rtol,
                                    double atol, int8_t* status, int32_t* nsub, int32_t* nrej,
                                    chem_stream_t stream) {
  return launch_advance_noalloc(m, T, p, Y, ld, dt, ncells, rtol, atol, status, nsub, nrej,
                                (cudaStream_t)stream);
}

extern "C" int chem_advance(chem_mech_t m, double* T, const double* p, double* Y, double dt,
                            int64_t ncells, double rtol, double atol, chem_stream_t stream) {
  return launch_advance(m, T, p, Y, ncells, dt, ncells, rtol, atol, nullptr, nullptr, nullptr,
                        nullptr, nullptr, (cudaStream_t)stream, nullptr);
}

extern "C" int chem_advance_ex(chem_mech_t m, double* T, const double* p, double* Y, int64_t ld,
                               double dt, int64_t ncells, double rtol, double atol,
                               const int32_t* idx, int8_t* status, int32_t* nsub, int32_t* nrej,
                               const chem_options* opt, chem_stream_t stream) {
  return launch_advance(m, T, p, Y, ld, dt, ncells, rtol, atol, idx, status, nsub, nrej, opt,
                        (cudaStream_t)stream, nullptr);
}

extern "C" int chem_advance_batch(chem_mech_t m, const chem_segment* segs, int nseg,
                                  chem_stream_t stream) {
  return launch_advance_batch(m, segs, nseg, (cudaStream_t)stream);
}

extern "C" int chem_eval_rhs_jac(chem_mech_t m, const double* T, const double* p, const double* Y,
                                 int64_t ld, int64_t ncells, double* f, double* J,
                                 chem_stream_t stream) {
  if (!m) { set_error("NULL mechanism"); return CHEM_EINVAL; }
  if (ncells < 0 || ld < ncells) { set_error("bad ncells/ld"); return CHEM_EINVAL; }
  if (ncells == 0) return CHEM_OK;
  if (!T || !p || !Y || !f) { set_error("NULL pointer"); return CHEM_EINVAL; }
  LaunchShape s;
  int rc = pick_shape(m, nullptr, &s);
  if (rc) return rc;
  EvalParams P;
  P.lay = m->lay; P.ws = s.ws; P.jp = jac_args(m); P.blob = (const unsigned char*)m->d_blob;
  P.T = T; P.p = p; P.Y = Y; P.ld = ld; P.ncells = ncells; P.f = f; P.J = J;
  cudaStream_t st = (cudaStream_t)stream;
  switch (s.G) {
    case 2: return launch_eval_t<2>(s, P, st);
    case 4: return launch_eval_t<4>(s, P, st);
    case 8: return launch_eval_t<8>(s, P, st);
    case 16: return launch_eval_t<16>(s, P, st);
    case 32: return launch_eval_t<32>(s, P, st);
    case 64: return launch_eval_t<64>(s, P, st);
    case 128: return launch_eval_t<128>(s, P, st);
    case 256: return launch_eval_t<256>(s, P, st);
    default: set_error("no kernel for group_threads %d", s.G); return CHEM_EINVAL;
  }
}

extern "C" int chem_fast_exp(const double* x, double* y, int64_t n, chem_stream_t stream) {
  if (n < 0) { set_error("negative n"); return CHEM_EINVAL; }
  if (n == 0) return CHEM_OK;
  if (!x || !y) { set_error("NULL pointer"); return CHEM_EINVAL; }
  int dev = 0, sms = 0;
  CHEM_CUDA_TRY(cudaGetDevice(&dev));
  CHEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t grid = std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  fast_exp_kernel<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(x, y, n);
  CHEM_CUDA_TRY(cudaGetLastError());
  return CHEM_OK;
}

extern "C" int chem_fp64_fma_peak(double* tflops) {
  if (!tflops) { set_error("NULL output"); return CHEM_EINVAL; }
  int dev = 0, sms = 0;
  CHEM_CUDA_TRY(cudaGetDevice(&dev));
  CHEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* out = nullptr;
  CHEM_CUDA_TRY(cudaMalloc(&out, sizeof(double)));
  cudaEvent_t e0, e1;
  CHEM_CUDA_TRY(cudaEventCreate(&e0));
  CHEM_CUDA_TRY(cudaEventCreate(&e1));
  const int threads = 256, blocks = sms * 8, iters = 4096;
  fma_peak_kernel<<<blocks, threads>>>(out, 64, 1.0000001, 1e-7);     // warm-up
  CHEM_CUDA_TRY(cudaEventRecord(e0));
  fma_peak_kernel<<<blocks, threads>>>(out, iters, 1.0000001, 1e-7);
  CHEM_CUDA_TRY(cudaEventRecord(e1));
  CHEM_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  CHEM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const double flops = 2.0 * 8.0 * (double)iters * threads * (double)blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return CHEM_OK;
}
