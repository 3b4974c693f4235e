// Host-side RelRes parameter preparation (no GPU needed).
//
// Builds, for every type pair, the quantities of Section 2 of Chaimovich &
// Chaimovich (arXiv:2104.10231): mixed FG LJ parameters, CG LJ parameters from
// the zero-order multipole sum rule (Eq. 13), the three quartic smoothing
// polynomials (Eq. 16 with the coefficients of Eq. 17 and Eq. 18) and the
// shift constants (Eq. 19).  Two outputs: the FP64 export table documented in
// relres.h (relres_prepare_table) and the kernel tables used by the pair
// kernels (relres::KernelTable).
#include "relres_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace relres {

namespace {

// u(r) = 4 eps [(s/r)^12 - (s/r)^6] with u' and u'' (Eq. 11 / Eq. 12).
void lj3(double r, double eps, double sig, double* u, double* du, double* d2u) {
  const double q = sig / r;
  const double q6 = q * q * q * q * q * q;
  const double q12 = q6 * q6;
  *u = 4.0 * eps * (q12 - q6);
  *du = 4.0 * eps * (6.0 * q6 - 12.0 * q12) / r;
  *d2u = 4.0 * eps * (156.0 * q12 - 42.0 * q6) / (r * r);
}

// Eq. 17: polynomial that leaves u with value, slope and curvature at the
// inner edge and arrives flat (zero slope and curvature) at the outer edge.
void coeffs_off(double u, double du, double d2u, double w, double g[5]) {
  g[0] = u;
  g[1] = du;
  g[2] = 0.5 * d2u;
  g[3] = 0.0;
  g[4] = 0.0;
  if (w > 0.0) {
    g[3] = -(du / (w * w)) - (2.0 * d2u) / (3.0 * w);
    g[4] = du / (2.0 * w * w * w) + d2u / (4.0 * w * w);
  }
}

// Eq. 18, with gamma_4 taken from the conditions of Eq. 8 (flat at the inner
// edge, meeting u, u', u'' at the outer edge); the printed sign of its u''
// term does not satisfy f''(w) = u''.
void coeffs_on(double u, double du, double d2u, double w, double g[5]) {
  g[0] = u - 0.5 * du * w + d2u * w * w / 12.0;
  g[1] = 0.0;
  g[2] = 0.0;
  g[3] = 0.0;
  g[4] = 0.0;
  if (w > 0.0) {
    g[3] = du / (w * w) - d2u / (3.0 * w);
    g[4] = d2u / (4.0 * w * w) - du / (2.0 * w * w * w);
  }
}

double horner5(const double g[5], double d) {
  return (((g[4] * d + g[3]) * d + g[2]) * d + g[1]) * d + g[0];
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

void mix_pair(int mixing, double ea, double sa, double eb, double sb, double* e, double* s) {
  *e = std::sqrt(ea * eb);
  *s = (mixing == RELRES_MIX_LB) ? 0.5 * (sa + sb) : std::sqrt(sa * sb);
}

// Eq. 13: A_k = sum over the FG sites of both groups of eps_{mu nu} sig_{mu nu}^k;
// sig^CG = (A12/A6)^(1/6), eps^CG = A6^2 / A12.
bool sum_rule(int nt, const double* eps, const double* sig, int mixing, const int* ci,
              const int* cj, double* eps_cg, double* sig_cg) {
  double a6 = 0.0, a12 = 0.0;
  for (int m = 0; m < nt; ++m) {
    if (ci[m] < 0 || cj[m] < 0) return false;
    for (int n = 0; n < nt; ++n) {
      const double mult = double(ci[m]) * double(cj[n]);
      if (mult == 0.0) continue;
      double e, s;
      mix_pair(mixing, eps[m], sig[m], eps[n], sig[n], &e, &s);
      const double s6 = s * s * s * s * s * s;
      a6 += mult * e * s6;
      a12 += mult * e * s6 * s6;
    }
  }
  if (!(a6 > 0.0) || !(a12 > 0.0)) {
    *eps_cg = 0.0;
    *sig_cg = 0.0;
    return true;
  }
  *sig_cg = std::pow(a12 / a6, 1.0 / 6.0);
  *eps_cg = a6 * a6 / a12;
  return true;
}

std::string build_pair_records(const relres_params* p, std::vector<PairRecord>* out) {
  if (!p) return "params is NULL";
  const int nt = p->n_types;
  if (nt < 1 || nt > RELRES_MAX_TYPES) return "n_types must be in 1..RELRES_MAX_TYPES";
  if (!p->eps_fg || !p->sig_fg || !p->is_hybrid) return "eps_fg, sig_fg and is_hybrid are required";
  if (p->mixing != RELRES_MIX_GEOMETRIC && p->mixing != RELRES_MIX_LB) return "unknown mixing rule";
  if (p->precision != RELRES_PREC_FP64 && p->precision != RELRES_PREC_FP32) return "unknown precision";
  if (!(p->skin >= 0.0) || !std::isfinite(p->skin)) return "skin must be finite and >= 0";
  for (int a = 0; a < nt; ++a) {
    if (!(p->eps_fg[a] >= 0.0) || !std::isfinite(p->eps_fg[a])) return "eps_fg must be finite and >= 0";
    if (!finite_pos(p->sig_fg[a])) return "sig_fg must be finite and > 0";
    if (p->is_hybrid[a] != 0 && p->is_hybrid[a] != 1) return "is_hybrid must be 0 or 1";
  }
  if (!p->eps_cg && !p->group_comp) {
    // no CG data: every pair is FG only (allowed, e.g. the FG reference)
  }
  if ((p->eps_cg == nullptr) != (p->sig_cg == nullptr)) return "eps_cg and sig_cg go together";
  out->assign(size_t(nt) * nt, PairRecord{});
  for (int a = 0; a < nt; ++a) {
    for (int b = 0; b < nt; ++b) {
      PairRecord& r = (*out)[size_t(a) * nt + b];
      mix_pair(p->mixing, p->eps_fg[a], p->sig_fg[a], p->eps_fg[b], p->sig_fg[b], &r.eps_fg, &r.sig_fg);
      const bool hh = p->is_hybrid[a] && p->is_hybrid[b];
      if (p->eps_cg) {
        const double e = p->eps_cg[a * nt + b], s = p->sig_cg[a * nt + b];
        if (!(e >= 0.0) || !std::isfinite(e) || !(s >= 0.0) || !std::isfinite(s))
          return "eps_cg/sig_cg must be finite and >= 0";
        if (!hh && e != 0.0) return "eps_cg must be 0 for pairs with an ordinary type (Eq. 14)";
        if (e > 0.0 && !(s > 0.0)) return "sig_cg must be > 0 where eps_cg > 0";
        if (e != p->eps_cg[b * nt + a] || s != p->sig_cg[b * nt + a]) return "eps_cg/sig_cg must be symmetric";
        r.eps_cg = e;
        r.sig_cg = s;
      } else if (p->group_comp && hh) {
        if (!sum_rule(nt, p->eps_fg, p->sig_fg, p->mixing, p->group_comp + a * nt,
                      p->group_comp + b * nt, &r.eps_cg, &r.sig_cg))
          return "group_comp entries must be >= 0";
      } else {
        r.eps_cg = 0.0;
        r.sig_cg = 0.0;
      }
      const double* rad = p->radii_pair ? p->radii_pair + 4 * (a * nt + b) : nullptr;
      r.rsm = rad ? rad[0] : p->r_si;
      r.rsp = rad ? rad[1] : p->r_so;
      r.rcm = rad ? rad[2] : p->r_ci;
      r.rcp = rad ? rad[3] : p->r_co;
      if (!(r.rsm > 0.0 && r.rsm <= r.rsp && r.rsp <= r.rcm && r.rcm <= r.rcp) ||
          !std::isfinite(r.rcp))
        return "radii must satisfy 0 < r_s- <= r_s+ <= r_c- <= r_c+";
      if (rad) {
        const double* rt = p->radii_pair + 4 * (b * nt + a);
        for (int k = 0; k < 4; ++k)
          if (rt[k] != rad[k]) return "radii_pair must be symmetric";
      }
      const double ws = r.rsp - r.rsm, wc = r.rcp - r.rcm;
      double u, du, d2u;
      // f_{s-}^{FG}: switch the FG term off over [r_s-, r_s+]
      lj3(r.rsm, r.eps_fg, r.sig_fg, &u, &du, &d2u);
      coeffs_off(u, du, d2u, ws, r.g_fg_m);
      if (r.eps_cg > 0.0) {
        // f_{s+}^{CG}: switch the CG term on over [r_s-, r_s+]
        lj3(r.rsp, r.eps_cg, r.sig_cg, &u, &du, &d2u);
        coeffs_on(u, du, d2u, ws, r.g_cg_p);
        // f_{c-}^{CG}: switch the CG term off over [r_c-, r_c+]
        lj3(r.rcm, r.eps_cg, r.sig_cg, &u, &du, &d2u);
        coeffs_off(u, du, d2u, wc, r.g_cg_m);
      } else {
        for (int m = 0; m < 5; ++m) r.g_cg_p[m] = r.g_cg_m[m] = 0.0;
      }
      // Eq. 19
      r.gam_cm = p->shift ? horner5(r.g_cg_m, wc) : 0.0;
      r.gam_sp = r.gam_cm + horner5(r.g_fg_m, ws);
      r.gam_sm = r.gam_sp - r.g_cg_p[0];
    }
  }
  return "";
}

template <typename R>
static void fill_kernel_row(const PairRecord& r, PairTab<R>* t) {
  std::memset(t, 0, sizeof(*t));
  const double s6f = std::pow(r.sig_fg, 6.0), s6c = std::pow(r.sig_cg, 6.0);
  t->c12f = R(4.0 * r.eps_fg * s6f * s6f);
  t->c6f = R(4.0 * r.eps_fg * s6f);
  t->rsm = R(r.rsm);
  t->rsm2 = R(r.rsm * r.rsm);
  t->rsp2 = R(r.rsp * r.rsp);
  t->f12f = R(12.0 * 4.0 * r.eps_fg * s6f * s6f);
  t->f6f = R(6.0 * 4.0 * r.eps_fg * s6f);
  for (int m = 0; m < 5; ++m) t->fg[m] = R(r.g_fg_m[m]);
  for (int m = 1; m < 5; ++m) t->fgd[m - 1] = R(m * r.g_fg_m[m]);
  // FG part of the exact split: u^FG - f_{s-}^{FG}(dr_s) below r_s-, the
  // polynomial minus the same constant on the shell, zero beyond.
  t->e_fg_shift = R(horner5(r.g_fg_m, r.rsp - r.rsm));
  t->c12c = R(4.0 * r.eps_cg * s6c * s6c);
  t->c6c = R(4.0 * r.eps_cg * s6c);
  t->f12c = R(12.0 * 4.0 * r.eps_cg * s6c * s6c);
  t->f6c = R(6.0 * 4.0 * r.eps_cg * s6c);
  t->rcm = R(r.rcm);
  t->rcm2 = R(r.rcm * r.rcm);
  t->rcp2 = R(r.rcp * r.rcp);
  t->on0 = R(r.g_cg_p[0]);
  t->on3 = R(r.g_cg_p[3]);
  t->on4 = R(r.g_cg_p[4]);
  t->ond3 = R(3.0 * r.g_cg_p[3]);
  t->ond4 = R(4.0 * r.g_cg_p[4]);
  for (int m = 0; m < 5; ++m) t->cgo[m] = R(r.g_cg_m[m]);
  for (int m = 1; m < 5; ++m) t->cgod[m - 1] = R(m * r.g_cg_m[m]);
  t->gam_cm = R(r.gam_cm);
  // CG part below r_s-: the constant f_{s+}^{CG}(0) - Gamma_{c-}
  t->e_cg_close = R(r.g_cg_p[0] - r.gam_cm);
}

void build_kernel_tables(const std::vector<PairRecord>& recs, std::vector<PairTab<float>>* tf,
                         std::vector<PairTab<double>>* td) {
  tf->resize(recs.size());
  td->resize(recs.size());
  for (size_t k = 0; k < recs.size(); ++k) {
    fill_kernel_row(recs[k], &(*tf)[k]);
    fill_kernel_row(recs[k], &(*td)[k]);
  }
}

namespace {
// r^-k and its first two derivatives
void powk3(double r, int k, double* u, double* du, double* d2u) {
  const double v = std::pow(r, -double(k));
  *u = v;
  *du = -k * v / r;
  *d2u = k * (k + 1.0) * v / (r * r);
}
}  // namespace

template <typename R>
static void fill_basis_row(const PairRecord& r, int shift, BasisTab<R>* t) {
  std::memset(t, 0, sizeof(*t));
  t->rsm = R(r.rsm);
  t->rsp = R(r.rsp);
  t->rcm = R(r.rcm);
  t->rcp = R(r.rcp);
  const double ws = r.rsp - r.rsm, wc = r.rcp - r.rcm;
  const int kk[2] = {12, 6};
  for (int b = 0; b < 2; ++b) {
    double u, du, d2u, g[5];
    powk3(r.rsm, kk[b], &u, &du, &d2u);
    coeffs_off(u, du, d2u, ws, g);
    for (int m = 0; m < 5; ++m) t->fg[b][m] = R(g[m]);
    t->fg_sh[b] = R(horner5(g, ws));
    powk3(r.rsp, kk[b], &u, &du, &d2u);
    coeffs_on(u, du, d2u, ws, g);
    for (int m = 0; m < 5; ++m) t->on[b][m] = R(g[m]);
    powk3(r.rcm, kk[b], &u, &du, &d2u);
    coeffs_off(u, du, d2u, wc, g);
    for (int m = 0; m < 5; ++m) t->off[b][m] = R(g[m]);
    t->gam[b] = R(shift ? horner5(g, wc) : 0.0);
  }
  const double s6f = std::pow(r.sig_fg, 6.0), s6c = std::pow(r.sig_cg, 6.0);
  t->c12f = R(4.0 * r.eps_fg * s6f * s6f);
  t->c6f = R(4.0 * r.eps_fg * s6f);
  t->c12c = R(4.0 * r.eps_cg * s6c * s6c);
  t->c6c = R(4.0 * r.eps_cg * s6c);
}

void build_basis_tables(const std::vector<PairRecord>& recs, int shift, std::vector<BasisTab<float>>* tf,
                        std::vector<BasisTab<double>>* td) {
  tf->resize(recs.size());
  td->resize(recs.size());
  for (size_t k = 0; k < recs.size(); ++k) {
    fill_basis_row(recs[k], shift, &(*tf)[k]);
    fill_basis_row(recs[k], shift, &(*td)[k]);
  }
}

}  // namespace relres

using namespace relres;

extern "C" relres_status relres_prepare_table(const relres_params* p, double* out, int out_len) {
  std::vector<PairRecord> recs;
  const std::string err = build_pair_records(p, &recs);
  if (!err.empty()) return RELRES_ERR_ARG;
  const int need = int(recs.size()) * RELRES_PAIR_FIELDS;
  if (!out || out_len < need) return RELRES_ERR_ARG;
  for (size_t k = 0; k < recs.size(); ++k) {
    const PairRecord& r = recs[k];
    double* o = out + k * RELRES_PAIR_FIELDS;
    o[0] = r.eps_fg;
    o[1] = r.sig_fg;
    o[2] = r.eps_cg;
    o[3] = r.sig_cg;
    o[4] = r.rsm;
    o[5] = r.rsp;
    o[6] = r.rcm;
    o[7] = r.rcp;
    for (int m = 0; m < 5; ++m) {
      o[8 + m] = r.g_fg_m[m];
      o[13 + m] = r.g_cg_p[m];
      o[18 + m] = r.g_cg_m[m];
    }
    o[23] = r.gam_cm;
    o[24] = r.gam_sp;
    o[25] = r.gam_sm;
  }
  return RELRES_OK;
}

namespace relres {
namespace {

// Vector-Jacobian product of Eq. 13 for one group pair: adds to g_eps[t],
// g_sig[t] the derivatives of ge * eps^CG + gs * sig^CG with respect to the
// per-type FG eps_t, sig_t.  With A_k = sum n_mu n_nu eps_{mu nu} sig_{mu nu}^k,
// eps^CG = A6^2 / A12 and sig^CG = (A12 / A6)^(1/6):
//   d eps^CG = (2 A6 / A12) dA6 - (A6 / A12)^2 dA12,
//   d sig^CG = sig^CG / 6 (dA12 / A12 - dA6 / A6),
// and each mixed pair passes its share back through eps_{mu nu} =
// sqrt(eps_mu eps_nu) (no eps derivative where either is 0) and the sigma rule.
// Zero CG parameters (A6 or A12 not positive) depend on nothing.
void sum_rule_vjp(int nt, const double* eps, const double* sig, int mixing, const int* ci, const int* cj,
                  double ge, double gs, double* g_eps, double* g_sig) {
  double a6 = 0.0, a12 = 0.0;
  for (int m = 0; m < nt; ++m)
    for (int n = 0; n < nt; ++n) {
      const double mult = double(ci[m]) * double(cj[n]);
      if (mult == 0.0) continue;
      double e, s;
      mix_pair(mixing, eps[m], sig[m], eps[n], sig[n], &e, &s);
      const double s6 = s * s * s * s * s * s;
      a6 += mult * e * s6;
      a12 += mult * e * s6 * s6;
    }
  if (!(a6 > 0.0) || !(a12 > 0.0)) return;
  const double sig_cg = std::pow(a12 / a6, 1.0 / 6.0);
  const double g6 = ge * 2.0 * a6 / a12 - gs * sig_cg / (6.0 * a6);
  const double g12 = -ge * (a6 / a12) * (a6 / a12) + gs * sig_cg / (6.0 * a12);
  for (int m = 0; m < nt; ++m)
    for (int n = 0; n < nt; ++n) {
      const double mult = double(ci[m]) * double(cj[n]);
      if (mult == 0.0) continue;
      double e, s;
      mix_pair(mixing, eps[m], sig[m], eps[n], sig[n], &e, &s);
      const double s5 = s * s * s * s * s, s6 = s5 * s, s11 = s6 * s5;
      const double de = mult * (g6 * s6 + g12 * s6 * s6);               // d / d eps_{mu nu}
      const double ds = mult * e * (6.0 * g6 * s5 + 12.0 * g12 * s11);  // d / d sig_{mu nu}
      if (eps[m] > 0.0 && eps[n] > 0.0) {
        g_eps[m] += de * 0.5 * std::sqrt(eps[n] / eps[m]);
        g_eps[n] += de * 0.5 * std::sqrt(eps[m] / eps[n]);
      }
      if (mixing == RELRES_MIX_LB) {
        g_sig[m] += 0.5 * ds;
        g_sig[n] += 0.5 * ds;
      } else {
        g_sig[m] += ds * 0.5 * std::sqrt(sig[n] / sig[m]);
        g_sig[n] += ds * 0.5 * std::sqrt(sig[m] / sig[n]);
      }
    }
}

}  // namespace
}  // namespace relres

extern "C" relres_status relres_chain_cg_grads(const relres_params* p, const double* g_eps_cg,
                                               const double* g_sig_cg, double* g_eps_fg, double* g_sig_fg) {
  using namespace relres;
  if (!p || !g_eps_cg || !g_sig_cg || !g_eps_fg || !g_sig_fg || !p->group_comp || p->eps_cg) return RELRES_ERR_ARG;
  std::vector<PairRecord> recs;
  if (!build_pair_records(p, &recs).empty()) return RELRES_ERR_ARG;
  const int nt = p->n_types;
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      if (!(p->is_hybrid[a] && p->is_hybrid[b])) continue;
      const double ge = g_eps_cg[a * nt + b], gs = g_sig_cg[a * nt + b];
      if (!std::isfinite(ge) || !std::isfinite(gs)) return RELRES_ERR_ARG;
      sum_rule_vjp(nt, p->eps_fg, p->sig_fg, p->mixing, p->group_comp + a * nt, p->group_comp + b * nt, ge, gs,
                   g_eps_fg, g_sig_fg);
    }
  return RELRES_OK;
}

extern "C" relres_status relres_cg_params(int n_types, const double* eps_fg, const double* sig_fg,
                                          int mixing, const int* comp_i, const int* comp_j,
                                          double* eps_cg, double* sig_cg) {
  if (n_types < 1 || n_types > RELRES_MAX_TYPES || !eps_fg || !sig_fg || !comp_i || !comp_j ||
      !eps_cg || !sig_cg)
    return RELRES_ERR_ARG;
  if (mixing != RELRES_MIX_GEOMETRIC && mixing != RELRES_MIX_LB) return RELRES_ERR_ARG;
  for (int a = 0; a < n_types; ++a)
    if (!(eps_fg[a] >= 0.0) || !finite_pos(sig_fg[a])) return RELRES_ERR_ARG;
  if (!sum_rule(n_types, eps_fg, sig_fg, mixing, comp_i, comp_j, eps_cg, sig_cg)) return RELRES_ERR_ARG;
  return RELRES_OK;
}
