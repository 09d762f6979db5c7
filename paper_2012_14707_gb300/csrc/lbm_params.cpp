// Host-side FP64 precompute of the slip boundary parameters (Sec. 3.B) and
// of the per-link coefficients the step kernel consumes.
#include <cmath>
#include <cstdio>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace lbm {
namespace {

const double kPi = 3.14159265358979323846;
const int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const double kW[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                      1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

std::string fmt(const char *f, double a, double b = 0.0) {
  char buf[256];
  std::snprintf(buf, sizeof buf, f, a, b);
  return buf;
}

}  // namespace

std::string compute_case_params(double Kn, double H, const lbm_params_t &p, CaseParams *cp) {
  const double s6 = std::sqrt(6.0 / kPi);  // sqrt(6/pi), Eq. tKnrela
  // Eq. tKnrela: tau_s from the Knudsen number and the length H (lattice units).
  double ts = std::isnan(p.tau_s) ? 0.5 + s6 * Kn * H : p.tau_s;
  if (!(ts > 0.5) || !std::isfinite(ts)) return fmt("tau_s = %g must exceed 1/2", ts);
  // Sec. 4: L1 = (2 - sigma)(1 - 0.1817 sigma)/sigma, L2 = 1/pi + L1^2/2.
  const double sg = p.sigma;
  if (!(sg > 0.0) || sg > 2.0) return fmt("sigma = %g outside (0, 2]", sg);
  double L1 = std::isnan(p.L1) ? (2.0 - sg) * (1.0 - 0.1817 * sg) / sg : p.L1;
  double L2 = std::isnan(p.L2) ? 1.0 / kPi + 0.5 * L1 * L1 : p.L2;
  const double a = 2.0 * ts - 1.0;
  // Eq. EqECond: tau_q > 1/2 requires E < E_max.
  double Emax = (kPi * ts * L2 - 3.0 * std::sqrt(kPi / 6.0) * L1) * a / (12.0 * ts) - 0.5;
  double E = std::isnan(p.E) ? std::fmin(-0.65, Emax - 0.1) : p.E;
  double tau_fix[4] = {p.tau_rho, p.tau_j, p.tau_e, p.tau_eps};
  if (p.collision != 0 && p.collision != 1)
    return fmt("collision must be 0 (MRT) or 1 (BGK), got %g", static_cast<double>(p.collision));
  const bool bgk = p.collision == 1;
  if (bgk) {
    // BGK reading of Sec. 3.B: tau_q = tau_s in Eq. NSliCoertstq, solved for E.
    E = (a * (ts * std::sqrt(6.0 * kPi) * L2 - L1) - 2.0 * s6 * ts -
         ts * (8.0 * s6 * ts + 4.0 * L1 * a)) / (12.0 * s6 * ts);
    for (double &t : tau_fix) t = ts;
  }
  // Eq. NSliCoertstq: the gamma-independent tau_q.
  double tq = bgk ? std::numeric_limits<double>::quiet_NaN() : p.tau_q;
  if (std::isnan(tq)) {
    double num = a * (ts * std::sqrt(6.0 * kPi) * L2 - L1) - 2.0 * s6 * ts * (1.0 + 6.0 * E);
    tq = num / (8.0 * s6 * ts + 4.0 * L1 * a);
  }
  if (!(tq > 0.5) || !std::isfinite(tq))
    return fmt("tau_q = %g must exceed 1/2 (E = %g; see the E bound of Eq. EqECond)", tq, E);
  for (double t : tau_fix)
    if (!(t > 0.5) || !std::isfinite(t)) return fmt("fixed relaxation time %g must exceed 1/2", t);
  cp->tau_s = ts;
  cp->tau_q = tq;
  cp->tau_rho = tau_fix[0];
  cp->tau_j = tau_fix[1];
  cp->tau_e = tau_fix[2];
  cp->tau_eps = tau_fix[3];
  cp->L1 = L1;
  cp->L2 = L2;
  cp->E = E;
  cp->E_max = Emax;
  cp->n_clamped = 0;
  return "";
}

std::string compute_link_coefs(const CaseParams &cp, const lbm_params_t &p, size_t n,
                               const int32_t *dir, const double *q, const double *ubx,
                               const double *uby, double *r_out, double *l_out, double *coef8,
                               int64_t *n_clamped) {
  // the D2Q9 quantities of each link, then the lattice-independent part
  std::vector<double> cub(n), w(n), uu(n);
  for (size_t k = 0; k < n; k++) {
    const int i = dir[k];
    if (i < 1 || i > 8) return fmt("link direction %g outside 1..8", static_cast<double>(i));
    cub[k] = kCx[i] * ubx[k] + kCy[i] * uby[k];
    w[k] = kW[i];
    uu[k] = ubx[k] * ubx[k] + uby[k] * uby[k];
  }
  return compute_link_coefs_general(cp, p, n, q, cub.data(), w.data(), uu.data(), r_out, l_out,
                                    coef8, n_clamped);
}

std::string compute_link_coefs_general(const CaseParams &cp, const lbm_params_t &p, size_t n,
                                       const double *q, const double *cub_in, const double *w_in,
                                       const double *uu_in, double *r_out, double *l_out,
                                       double *coef8, int64_t *n_clamped) {
  const double s6 = std::sqrt(6.0 / kPi);
  const double ts = cp.tau_s, a = 2.0 * ts - 1.0, L1 = cp.L1;
  // one link: "" or an error text; sets *cl when the clamp applied
  auto one = [&](size_t k, int *cl) -> std::string {
    const double g = q[k];
    double l;
    switch (p.l_mode) {
      case LBM_L_PAPER: {
        // Eq. Eqexlva, then the clamp of Sec. 3.B.
        l = (s6 * g * g + g * a * (L1 + s6)) / (s6 * a) + cp.E;
        if (l < p.l_clamp) {
          l = 0.0;
          *cl = 1;
        }
        break;
      }
      case LBM_L_ZERO: l = 0.0; break;
      case LBM_L_GAMMA: l = g; break;
      case LBM_L_2GAMMA: l = 2.0 * g; break;
      case LBM_L_GAMMA2: l = g * g; break;
      case LBM_L_GAMMA2_GAMMA: l = g * g + g; break;
      case LBM_L_FIXED: l = p.l_value; break;
      default: return fmt("unknown l_mode %g", static_cast<double>(p.l_mode));
    }
    if (!(l > -1.0) || !std::isfinite(l)) return fmt("free parameter l = %g must exceed -1", l);
    // Eq. SliCoeffrtsr with the l actually used.
    double r = p.r_value;
    if (std::isnan(r)) {
      const double t = s6 * ts * (1.0 + l);
      r = t / (L1 * a + t);
    }
    if (!(r >= 0.0 && r <= 1.0)) return fmt("combination parameter r = %g outside [0, 1]", r);
    r_out[k] = r;
    l_out[k] = l;
    // Eq. EqNewBDSC split into bounce-back weights, wall term and Maxwell part.
    const double inv = 1.0 / (1.0 + l);
    const double k1 = r * (1.0 + l - 2.0 * g) * inv;
    const double k2 = r * l * inv;
    const double k3 = r * (2.0 * g - l) * inv;
    const double cub = cub_in[k], wi = w_in[k];
    double alpha = 2.0 * r * inv * wi * 3.0 * cub;  // multiplies rho_f
    double beta;                                      // multiplies f_eq(rho_f, u_f)
    if (p.diffuse_mode == 0) {
      beta = 1.0 - r;
    } else {
      alpha += (1.0 - r) * wi * (1.0 + 3.0 * cub + 4.5 * cub * cub - 1.5 * uu_in[k]);
      beta = 0.0;
    }
    (void)beta;  // implied by diffuse_mode and r = k1 + k2 + k3 in the kernel
    double *c = coef8 + 8 * k;
    c[0] = k1;
    c[1] = k2;
    c[2] = k3;
    c[3] = alpha;
    c[4] = c[5] = c[6] = c[7] = 0.0;
    return "";
  };
  // links in parallel; the lowest-numbered failing link's message wins
  std::mutex mu;
  int64_t clamped = 0, first_bad = -1;
  std::string first_msg;
  parallel_for(static_cast<int64_t>(n), [&](int64_t k0, int64_t k1) {
    int64_t cl_sum = 0;
    for (int64_t k = k0; k < k1; k++) {
      int cl = 0;
      std::string m = one(static_cast<size_t>(k), &cl);
      cl_sum += cl;
      if (!m.empty()) {
        std::lock_guard<std::mutex> lock(mu);
        if (first_bad < 0 || k < first_bad) {
          first_bad = k;
          first_msg = m;
        }
        break;
      }
    }
    std::lock_guard<std::mutex> lock(mu);
    clamped += cl_sum;
  });
  if (first_bad >= 0) return first_msg;
  *n_clamped = clamped;
  return "";
}

}  // namespace lbm
