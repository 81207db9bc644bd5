// Mechanism loading: text parser, validation, device blob and Jacobian-assembly program.
//
// The kinetics model is the one §2 of the paper delegates to Cantera: NASA-7 species thermo
// with two ranges split at 1000 K, modified-Arrhenius rate constants, third-body collision
// partners with per-species efficiencies, Troe fall-off, and reverse rates from equilibrium
// constants.  This file precomputes everything that does not depend on the state (scaled
// polynomial coefficients, Ta = Ea/Rc, ln A, sparse efficiency lists, species production lists)
// into one blob that every CTA stages into shared memory once.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "chem_internal.h"
#include "exp_table.h"

namespace chem {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? CHEM_ENOMEM : CHEM_ECUDA;
}

namespace {

int align16(int x) { return (x + 15) & ~15; }

struct Builder {
  std::vector<unsigned char> buf;
  int add(int bytes) {
    int off = (int)buf.size();
    buf.resize(off + align16(bytes), 0);
    return off;
  }
  template <class T> T* at(int off) { return reinterpret_cast<T*>(buf.data() + off); }
};

// Copy of a mechanism description whose reactions are reordered fall-off first, then
// third-body, then elementary (stable within each class).  The rate loop hands consecutive
// reactions to consecutive threads, so the long fall-off branch runs in as few warps as possible.
struct Reordered {
  chem_mech_desc d{};
  std::vector<int> rtype, reac, prod, has_t2;
  std::vector<double> A, b, Ea, troe, eff;
};

void reorder_reactions(const chem_mech_desc* in, Reordered* o) {
  const int ns = in->n_species, nr = in->n_reactions;
  std::vector<int> order;
  for (int cls : {2, 1, 0})
    for (int j = 0; j < nr; ++j)
      if (in->rtype[j] == cls) order.push_back(j);
  o->d = *in;
  o->rtype.resize(nr); o->reac.resize(3 * nr); o->prod.resize(3 * nr); o->has_t2.resize(nr);
  o->A.resize(nr); o->b.resize(nr); o->Ea.resize(nr); o->troe.resize(7 * (size_t)nr);
  o->eff.resize((size_t)nr * ns);
  for (int jn = 0; jn < nr; ++jn) {
    const int j = order[jn];
    o->rtype[jn] = in->rtype[j];
    for (int i = 0; i < 3; ++i) { o->reac[3 * jn + i] = in->reac[3 * j + i]; o->prod[3 * jn + i] = in->prod[3 * j + i]; }
    o->has_t2[jn] = in->has_t2[j];
    o->A[jn] = in->A[j]; o->b[jn] = in->b[j]; o->Ea[jn] = in->Ea[j];
    for (int i = 0; i < 7; ++i) o->troe[7 * (size_t)jn + i] = in->troe[7 * (size_t)j + i];
    for (int k = 0; k < ns; ++k) o->eff[(size_t)jn * ns + k] = in->eff[(size_t)j * ns + k];
  }
  if (nr > 0) {
    o->d.rtype = o->rtype.data(); o->d.reac = o->reac.data(); o->d.prod = o->prod.data();
    o->d.has_t2 = o->has_t2.data(); o->d.A = o->A.data(); o->d.b = o->b.data(); o->d.Ea = o->Ea.data();
    o->d.troe = o->troe.data(); o->d.eff = o->eff.data();
  }
}

int build(const chem_mech_desc* din, chem_mech_s* m) {
  Reordered ro;
  reorder_reactions(din, &ro);
  const chem_mech_desc* d = &ro.d;
  const int ns = d->n_species, ne = d->n_elements, nr = d->n_reactions;
  m->ns = ns; m->ne = ne; m->nr = nr;
  m->elem_mass.assign(d->elem_mass, d->elem_mass + ne);
  m->comp.assign(d->comp, d->comp + (size_t)ns * ne);
  m->W.assign(ns, 0.0);
  for (int k = 0; k < ns; ++k)
    for (int e = 0; e < ne; ++e) m->W[k] += d->comp[(size_t)k * ne + e] * d->elem_mass[e];
  m->nasa_lo.assign(d->nasa_lo, d->nasa_lo + 7 * ns);
  m->nasa_hi.assign(d->nasa_hi, d->nasa_hi + 7 * ns);

  // third-body sets and troe parameters
  std::vector<int> tb_of(nr, -1), troe_of(nr, -1);
  std::vector<int> eff_off(1, 0);
  std::vector<int16_t> eff_idx;
  std::vector<double> eff_val;
  int ntb = 0, ntroe = 0;
  for (int j = 0; j < nr; ++j) {
    if (d->rtype[j] == 0) continue;
    tb_of[j] = ntb++;
    for (int k = 0; k < ns; ++k) {
      double e = d->eff[(size_t)j * ns + k];
      if (e != 1.0) { eff_idx.push_back((int16_t)k); eff_val.push_back(e - 1.0); }
    }
    eff_off.push_back((int)eff_idx.size());
    if (d->rtype[j] == 2) troe_of[j] = ntroe++;
  }
  // species production lists: (reaction, net stoichiometric coefficient), ascending reaction
  std::vector<std::vector<std::pair<int, int>>> plist(ns);
  std::vector<std::vector<int>> nu(nr, std::vector<int>(ns, 0));
  for (int j = 0; j < nr; ++j) {
    for (int i = 0; i < 3; ++i) {
      if (d->reac[3 * j + i] >= 0) nu[j][d->reac[3 * j + i]] -= 1;
      if (d->prod[3 * j + i] >= 0) nu[j][d->prod[3 * j + i]] += 1;
    }
    for (int k = 0; k < ns; ++k)
      if (nu[j][k] != 0) plist[k].push_back({j, nu[j][k]});
  }
  std::vector<int> woff(ns + 1, 0);
  for (int k = 0; k < ns; ++k) woff[k + 1] = woff[k] + (int)plist[k].size();
  const int nprod = woff[ns];
  // Balanced pieces of the production lists for groups wider than a warp: each species' list
  // is cut into pieces of at most plen terms, plen the smallest that gives at most kPieceTarget
  // pieces, so that one pass of a 128-thread group covers them with similar loop lengths.
  constexpr int kPieceTarget = 128;
  int plen = 1;
  auto count_pieces = [&](int len) {
    int c = 0;
    for (int k = 0; k < ns; ++k) c += std::max(1, ((int)plist[k].size() + len - 1) / len);
    return c;
  };
  while (count_pieces(plen) > kPieceTarget && plen < std::max(1, nprod)) ++plen;
  std::vector<int> pterm(1, 0), poff(ns + 1, 0);
  for (int k = 0; k < ns; ++k) {
    const int len = (int)plist[k].size();
    const int np = std::max(1, (len + plen - 1) / plen);
    for (int i = 0; i < np; ++i) pterm.push_back(woff[k] + std::min(len, (i + 1) * plen));
    poff[k + 1] = poff[k] + np;
  }
  const int npieces = poff[ns];
  const int neff = (int)eff_idx.size();

  MechLayout L{};
  L.ns = ns; L.nr = nr; L.N = ns + 1; L.ntb = ntb; L.ntroe = ntroe; L.nprod = nprod;
  L.npieces = npieces;
  Builder B;
  L.o_W = B.add(8 * ns);
  L.o_invW = B.add(8 * ns);
  L.o_hc = B.add(8 * 2 * ns * 6);
  L.o_sc = B.add(8 * 2 * ns * 6);
  L.o_cpc = B.add(8 * 2 * ns * 5);
  L.o_lnA = B.add(8 * nr);
  L.o_beta = B.add(8 * nr);
  L.o_Ta = B.add(8 * nr);
  L.o_troe = B.add(8 * 8 * ntroe);
  L.o_effv = B.add(8 * neff);
  L.o_const = B.add(8 * kConsts);
  L.o_reac = B.add(2 * 4 * nr);
  L.o_prod = B.add(2 * 4 * nr);
  L.o_rinfo = B.add(2 * 4 * nr);
  L.o_effidx = B.add(2 * neff);
  L.o_wpk = B.add(4 * nprod);
  L.o_effoff = B.add(4 * (ntb + 1));
  L.o_woff = B.add(4 * (ns + 1));
  L.o_pterm = B.add(4 * (npieces + 1));
  L.o_poff = B.add(4 * (ns + 1));
  L.bytes = (int)B.buf.size();

  double* W = B.at<double>(L.o_W);
  double* invW = B.at<double>(L.o_invW);
  for (int k = 0; k < ns; ++k) { W[k] = m->W[k]; invW[k] = 1.0 / m->W[k]; }
  for (int r = 0; r < 2; ++r) {
    const double* src = r == 0 ? d->nasa_lo : d->nasa_hi;
    for (int k = 0; k < ns; ++k) {
      const double* a = src + 7 * k;
      double* hc = B.at<double>(L.o_hc) + (r * ns + k) * 6;
      double* sc = B.at<double>(L.o_sc) + (r * ns + k) * 6;
      double* cc = B.at<double>(L.o_cpc) + (r * ns + k) * 5;
      hc[0] = a[0]; hc[1] = a[1] / 2.0; hc[2] = a[2] / 3.0; hc[3] = a[3] / 4.0; hc[4] = a[4] / 5.0; hc[5] = a[5];
      sc[0] = a[0]; sc[1] = a[1]; sc[2] = a[2] / 2.0; sc[3] = a[3] / 3.0; sc[4] = a[4] / 4.0; sc[5] = a[6];
      for (int i = 0; i < 5; ++i) cc[i] = a[i];
    }
  }
  for (int j = 0; j < nr; ++j) {
    B.at<double>(L.o_lnA)[j] = std::log(d->A[j]);      // A = 0 gives -inf: kf = 0 exactly
    B.at<double>(L.o_beta)[j] = d->b[j];
    B.at<double>(L.o_Ta)[j] = d->Ea[j] / RC;
    int16_t* re = B.at<int16_t>(L.o_reac) + 4 * j;
    int16_t* pr = B.at<int16_t>(L.o_prod) + 4 * j;
    int dnu = 0;
    for (int i = 0; i < 3; ++i) {
      re[i] = (int16_t)d->reac[3 * j + i];
      pr[i] = (int16_t)d->prod[3 * j + i];
      dnu += (d->prod[3 * j + i] >= 0) - (d->reac[3 * j + i] >= 0);
    }
    re[3] = pr[3] = -1;
    int16_t* ri = B.at<int16_t>(L.o_rinfo) + 4 * j;
    ri[0] = (int16_t)d->rtype[j]; ri[1] = (int16_t)dnu; ri[2] = (int16_t)tb_of[j];
    ri[3] = (int16_t)troe_of[j];
    if (troe_of[j] >= 0) {
      const double* t = d->troe + 7 * j;
      double* o = B.at<double>(L.o_troe) + 8 * troe_of[j];
      o[0] = std::log(t[0]); o[1] = t[1]; o[2] = t[2] / RC; o[3] = t[3];
      o[4] = 1.0 / t[4]; o[5] = 1.0 / t[5]; o[6] = t[6]; o[7] = d->has_t2[j] ? 1.0 : 0.0;
    }
  }
  for (int i = 0; i < neff; ++i) {
    B.at<double>(L.o_effv)[i] = eff_val[i];
    B.at<int16_t>(L.o_effidx)[i] = eff_idx[i];
  }
  for (int i = 0; i <= ntb; ++i) B.at<int>(L.o_effoff)[i] = eff_off[i];
  for (int k = 0; k <= ns; ++k) B.at<int>(L.o_woff)[k] = woff[k];
  for (int i = 0; i <= npieces; ++i) B.at<int>(L.o_pterm)[i] = pterm[i];
  for (int k = 0; k <= ns; ++k) B.at<int>(L.o_poff)[k] = poff[k];
  for (int k = 0; k < ns; ++k)
    for (int i = 0; i < (int)plist[k].size(); ++i) {
      const int nuk = plist[k][i].second;
      if (nuk < -8 || nuk > 7) {
        set_error("reaction %d: stoichiometric coefficient %d of species %d out of range", plist[k][i].first, nuk, k);
        return CHEM_EINVAL;
      }
      B.at<int>(L.o_wpk)[woff[k] + i] = (plist[k][i].first << 4) | (nuk + 8);
    }
  double* cst = B.at<double>(L.o_const);
  for (int c = 0; c < 16; ++c) cst[kC_NU + c] = (double)(c - 8);
  cst[kC_LNPR0] = std::log(PATM / RU);
  cst[kC_INVNS] = 1.0 / ns;
  for (int j = 0; j < 64; ++j) cst[kC_EXPTAB + j] = kExpTable[j];
  m->lay = L;

  // Jacobian-assembly program for d(wdot_k)/dC_m; a term is (src, oth, coef)
  struct Term { int src, oth; double coef; };
  std::map<std::pair<int, int>, std::vector<Term>> ent;
  for (int j = 0; j < nr; ++j) {
    for (int k = 0; k < ns; ++k) {
      if (nu[j][k] == 0) continue;
      for (int s = 0; s < 6; ++s) {
        const int* side = s < 3 ? d->reac + 3 * j : d->prod + 3 * j;
        const int sl = s % 3;
        const int sp = side[sl];
        if (sp < 0) continue;
        // the other two slots of the same side, in slot order
        const int a1 = sl == 0 ? 1 : 0, a2 = sl == 2 ? 1 : 2;
        const int o1 = side[a1] >= 0 ? side[a1] : ns, o2 = side[a2] >= 0 ? side[a2] : ns;
        ent[{k, sp}].push_back({(j << 3) | s, o1 | (o2 << 16), (double)nu[j][k]});
      }
      if (d->rtype[j] != 0)
        for (int mm = 0; mm < ns; ++mm) {
          double e = d->eff[(size_t)j * ns + mm];
          if (e != 0.0) ent[{k, mm}].push_back({(j << 3) | 7, 0, nu[j][k] * e});
        }
    }
  }
  JacProgram& P = m->jac;
  P.nent = (int)ent.size();
  std::vector<int> off(1, 0);
  std::vector<int16_t> rows, cols;
  std::vector<int> src, oth;
  std::vector<double> coef;
  // entries with many terms first: threads take consecutive entries, so a warp's entries have
  // similar term counts and its lanes stay busy for the same number of iterations
  std::vector<const std::pair<const std::pair<int, int>, std::vector<Term>>*> order;
  for (auto& kv : ent) order.push_back(&kv);
  std::stable_sort(order.begin(), order.end(),
                   [](const auto* a, const auto* b) { return a->second.size() > b->second.size(); });
  for (auto* kvp : order) {
    const auto& kv = *kvp;
    rows.push_back((int16_t)kv.first.first);
    cols.push_back((int16_t)kv.first.second);
    for (auto& t : kv.second) { src.push_back(t.src); oth.push_back(t.oth); coef.push_back(t.coef); }
    off.push_back((int)src.size());
  }
  P.nterm = (int)src.size();

  CHEM_CUDA_TRY(cudaGetDevice(&m->device));
  CHEM_CUDA_TRY(cudaMalloc(&m->d_blob, L.bytes));
  CHEM_CUDA_TRY(cudaMemcpy(m->d_blob, B.buf.data(), L.bytes, cudaMemcpyHostToDevice));
  size_t o_off = 0;
  size_t o_row = align16((int)(o_off + 4 * (P.nent + 1)));
  size_t o_col = o_row + align16(2 * P.nent);
  size_t o_src = o_col + align16(2 * P.nent);
  size_t o_oth = o_src + align16(4 * P.nterm);
  size_t o_coef = o_oth + align16(4 * P.nterm);
  size_t tot = o_coef + 8 * (size_t)P.nterm + 16;
  std::vector<unsigned char> jb(tot, 0);
  memcpy(jb.data() + o_off, off.data(), 4 * off.size());
  if (P.nent) {
    memcpy(jb.data() + o_row, rows.data(), 2 * rows.size());
    memcpy(jb.data() + o_col, cols.data(), 2 * cols.size());
  }
  if (P.nterm) {
    memcpy(jb.data() + o_src, src.data(), 4 * src.size());
    memcpy(jb.data() + o_oth, oth.data(), 4 * oth.size());
    memcpy(jb.data() + o_coef, coef.data(), 8 * coef.size());
  }
  CHEM_CUDA_TRY(cudaMalloc(&m->d_jac, tot));
  CHEM_CUDA_TRY(cudaMemcpy(m->d_jac, jb.data(), tot, cudaMemcpyHostToDevice));
  unsigned char* base = (unsigned char*)m->d_jac;
  P.ent_off = (int*)(base + o_off);
  P.ent_row = (int16_t*)(base + o_row);
  P.ent_col = (int16_t*)(base + o_col);
  P.term_src = (int*)(base + o_src);
  P.term_oth = (int*)(base + o_oth);
  P.term_coef = (double*)(base + o_coef);
  return CHEM_OK;
}

int validate(const chem_mech_desc* d) {
  if (!d) { set_error("NULL mechanism description"); return CHEM_EINVAL; }
  const int ns = d->n_species, ne = d->n_elements, nr = d->n_reactions;
  if (ns < 1 || ns > 4096 || ne < 1 || ne > 64 || nr < 0 || nr > 30000) {
    set_error("mechanism sizes out of range (ns=%d ne=%d nr=%d)", ns, ne, nr);
    return CHEM_EINVAL;
  }
  if (!d->elem_mass || !d->comp || !d->nasa_lo || !d->nasa_hi ||
      (nr > 0 && (!d->rtype || !d->reac || !d->prod || !d->A || !d->b || !d->Ea || !d->troe ||
                  !d->has_t2 || !d->eff))) {
    set_error("NULL array in mechanism description");
    return CHEM_EINVAL;
  }
  for (int e = 0; e < ne; ++e)
    if (!(d->elem_mass[e] > 0.0) || !std::isfinite(d->elem_mass[e])) {
      set_error("element %d has a non-positive or non-finite atomic mass", e);
      return CHEM_EINVAL;
    }
  for (int k = 0; k < ns; ++k) {
    double W = 0.0;
    for (int e = 0; e < ne; ++e) {
      if (d->comp[(size_t)k * ne + e] < 0) { set_error("species %d has a negative element count", k); return CHEM_EINVAL; }
      W += d->comp[(size_t)k * ne + e] * d->elem_mass[e];
    }
    if (!(W > 0.0)) { set_error("species %d has non-positive molar mass", k); return CHEM_EINVAL; }
    for (int i = 0; i < 7; ++i)
      if (!std::isfinite(d->nasa_lo[7 * k + i]) || !std::isfinite(d->nasa_hi[7 * k + i])) {
        set_error("species %d has non-finite NASA coefficients", k);
        return CHEM_EINVAL;
      }
  }
  for (int j = 0; j < nr; ++j) {
    if (d->rtype[j] < 0 || d->rtype[j] > 2) { set_error("reaction %d: bad type", j); return CHEM_EINVAL; }
    int nre = 0, npr = 0;
    for (int i = 0; i < 3; ++i) {
      int a = d->reac[3 * j + i], b = d->prod[3 * j + i];
      if (a < -1 || a >= ns || b < -1 || b >= ns) {
        set_error("reaction %d: species index out of range", j);
        return CHEM_EINVAL;
      }
      nre += a >= 0; npr += b >= 0;
    }
    if (nre == 0 || npr == 0) { set_error("reaction %d: empty side", j); return CHEM_EINVAL; }
    if (!(d->A[j] >= 0.0) || !std::isfinite(d->b[j]) || !std::isfinite(d->Ea[j])) {
      set_error("reaction %d: bad Arrhenius parameters", j);
      return CHEM_EINVAL;
    }
    if (d->rtype[j] != 0)
      for (int k = 0; k < ns; ++k) {
        const double e = d->eff[(size_t)j * ns + k];
        if (!(e >= 0.0) || !std::isfinite(e)) {
          set_error("reaction %d: third-body efficiency of species %d is negative or not finite", j, k);
          return CHEM_EINVAL;
        }
      }
    if (d->rtype[j] == 2) {
      const double* t = d->troe + 7 * j;
      bool finite = true;
      for (int i = 0; i < 7; ++i) finite = finite && std::isfinite(t[i]);
      if (!finite || !(t[0] >= 0.0) || !(t[4] > 0.0) || !(t[5] > 0.0) ||
          (d->has_t2[j] != 0 && d->has_t2[j] != 1)) {
        set_error("reaction %d: bad Troe parameters", j);
        return CHEM_EINVAL;
      }
    }
  }
  return CHEM_OK;
}

}  // namespace
}  // namespace chem

using namespace chem;

extern "C" int chem_load_mechanism_desc(const chem_mech_desc* desc, chem_mech_t* out) {
  if (!out) { set_error("NULL output handle"); return CHEM_EINVAL; }
  *out = nullptr;
  int rc = validate(desc);
  if (rc) return rc;
  chem_mech_s* m = new (std::nothrow) chem_mech_s();
  if (!m) { set_error("out of host memory"); return CHEM_ENOMEM; }
  rc = build(desc, m);
  if (rc) { chem_free_mechanism(m); return rc; }
  *out = m;
  return CHEM_OK;
}

extern "C" int chem_load_mechanism(const char* path, chem_mech_t* out) {
  if (!path || !out) { set_error("NULL argument"); return CHEM_EINVAL; }
  std::ifstream f(path);
  if (!f) { set_error("cannot open %s", path); return CHEM_ENOTFOUND; }
  std::stringstream ss;
  ss << f.rdbuf();
  std::istringstream in(ss.str());
  std::string tok;
  auto expect = [&](const char* w) { return (in >> tok) && tok == w; };
  int ne = 0, ns = 0, nr = 0, ver = 0;
  std::string name;
  if (!expect("CHEMMECH") || !(in >> ver) || ver != 1 || !expect("name") || !(in >> name) ||
      !expect("elements") || !(in >> ne) || ne < 1 || ne > 64) {
    set_error("%s: bad CHEMMECH header", path);
    return CHEM_EINVAL;
  }
  std::vector<double> emass(ne);
  for (int e = 0; e < ne; ++e)
    if (!(in >> tok >> emass[e])) { set_error("%s: bad element line", path); return CHEM_EINVAL; }
  if (!expect("species") || !(in >> ns) || ns < 1 || ns > 4096) {
    set_error("%s: bad species header", path);
    return CHEM_EINVAL;
  }
  std::vector<int> comp((size_t)ns * ne);
  std::vector<double> lo(7 * ns), hi(7 * ns);
  for (int k = 0; k < ns; ++k) {
    in >> tok;
    for (int e = 0; e < ne; ++e) in >> comp[(size_t)k * ne + e];
    for (int i = 0; i < 7; ++i) in >> lo[7 * k + i];
    for (int i = 0; i < 7; ++i) in >> hi[7 * k + i];
    if (!in) { set_error("%s: bad species %d", path, k); return CHEM_EINVAL; }
  }
  if (!expect("reactions") || !(in >> nr) || nr < 0 || nr > 30000) {
    set_error("%s: bad reactions header", path);
    return CHEM_EINVAL;
  }
  std::vector<int> rtype(nr), reac(3 * nr), prod(3 * nr), has_t2(nr, 0);
  std::vector<double> A(nr), b(nr), Ea(nr), troe(7 * (size_t)nr, 0.0), eff((size_t)nr * ns, 1.0);
  for (int j = 0; j < nr; ++j) {
    in >> rtype[j];
    for (int i = 0; i < 3; ++i) in >> reac[3 * j + i];
    for (int i = 0; i < 3; ++i) in >> prod[3 * j + i];
    in >> A[j] >> b[j] >> Ea[j];
    if (rtype[j] == 2) {
      for (int i = 0; i < 7; ++i) in >> troe[7 * j + i];
      in >> has_t2[j];
    }
    if (rtype[j] != 0) {
      int n = 0;
      in >> n;
      for (int i = 0; i < n && in; ++i) {
        int k = -1;
        double v = 0;
        in >> k >> v;
        if (k < 0 || k >= ns) { set_error("%s: reaction %d efficiency index", path, j); return CHEM_EINVAL; }
        eff[(size_t)j * ns + k] = v;
      }
    }
    if (!in) { set_error("%s: bad reaction %d", path, j); return CHEM_EINVAL; }
  }
  if (!expect("end")) { set_error("%s: missing end", path); return CHEM_EINVAL; }
  chem_mech_desc d{};
  d.n_species = ns; d.n_elements = ne; d.n_reactions = nr;
  d.elem_mass = emass.data(); d.comp = comp.data(); d.nasa_lo = lo.data(); d.nasa_hi = hi.data();
  d.rtype = rtype.data(); d.reac = reac.data(); d.prod = prod.data(); d.A = A.data();
  d.b = b.data(); d.Ea = Ea.data(); d.troe = troe.data(); d.has_t2 = has_t2.data();
  d.eff = eff.data();
  return chem_load_mechanism_desc(&d, out);
}

extern "C" int chem_free_mechanism(chem_mech_t m) {
  if (!m) { set_error("NULL mechanism"); return CHEM_EINVAL; }
  if (m->d_blob) cudaFree(m->d_blob);
  if (m->d_jac) cudaFree(m->d_jac);
  delete m;
  return CHEM_OK;
}

extern "C" int chem_mechanism_info(chem_mech_t m, int* n_species, int* n_reactions,
                                   int* n_elements) {
  if (!m) { set_error("NULL mechanism"); return CHEM_EINVAL; }
  if (n_species) *n_species = m->ns;
  if (n_reactions) *n_reactions = m->nr;
  if (n_elements) *n_elements = m->ne;
  return CHEM_OK;
}

extern "C" const char* chem_last_error(void) { return chem::g_err.c_str(); }
