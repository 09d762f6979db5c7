// Internal declarations shared by the host side and the kernels of liblbm.so.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace lbm {

// Node flag byte: bits 0..7 = unknown incoming directions 1..8 (x - c_i is
// solid); kSolid marks a solid (or padding) node that is never updated.
constexpr uint8_t kSolid = 0xFF;

// Relaxation rates and forcing of one case, as the kernels consume them.
template <typename C>
struct StepConst {
  C s_e, s_eps, s_q, s_s, s_j;  // 1/tau of the non-conserved moments and of j
  C h_e, h_eps, h_q, h_s, h_j;  // 1 - s/2: weights of the forcing moments (Eq. MomentPost)
  C sc, inv_sc;                 // storage scale of the 16-bit types (1 otherwise)
  C ax, ay;                     // body acceleration
  int32_t nx, ny, pitch;        // lattice size and row pitch (elements)
  int32_t periodic_x, periodic_y;
  int32_t diffuse_mode;         // reading of the Maxwell part, see LinkCoef
  int64_t plane;                // elements per population plane = ny * pitch
};

// Coefficients of one link in the kernels' folded form of Eq. EqNewBDSC,
// in deviation variables d = f - w:
//   d_i(x_f, t+1) = k1 d_ib + k2 d'_i + k3 d'_ib + c0 + c1 drho
//                   + c2 (drho + rho P_i(u_f)),
//   P_i(u) = 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u,
// with r = k1 + k2 + k3 and, for the Maxwell part at the fluid velocity
// (diffuse_mode 0): c0 = c1 = alpha, c2 = (1 - r) w_i; at the wall velocity
// (diffuse_mode 1): c0 = alpha + (r - 1) w_i, c1 = alpha, c2 = 0.  alpha
// collects every term proportional to rho_f (wall-velocity terms).  One
// 16-byte record per link.
template <typename C>
struct alignas(sizeof(C) * 4) LinkCoef {
  C k1, k2, k3, alpha;
};

// Case parameters after the FP64 precompute of Sec. 3.B.
struct CaseParams {
  double tau_s, tau_q, tau_rho, tau_j, tau_e, tau_eps;
  double L1, L2, E, E_max;
  int64_t n_clamped;
};

// One validated case laid out for the device (host copy): node flags, the
// first link of every node, and the node-sorted link coefficients
// (k1, k2, k3, alpha per link, FP64).
struct HostCase {
  int32_t nx = 0, ny = 0, pitch = 0, px = 0, py = 0;
  int64_t plane = 0, n_fluid = 0, n_links = 0;
  double ax = 0.0, ay = 0.0, scale = 1.0;
  CaseParams cp{};
  lbm_params_t params{};
  std::vector<uint8_t> flags;
  std::vector<int32_t> lbase;
  std::vector<double> coef;
  std::vector<double> link_r, link_l;  // per link in input order
};

// Kernel constants of one case in arithmetic type C.
template <typename C>
StepConst<C> make_step_const(const CaseParams &cp, int32_t nx, int32_t ny, int32_t pitch,
                             int64_t plane, int32_t px, int32_t py, double ax, double ay,
                             int32_t diffuse_mode, double scale) {
  StepConst<C> k;
  k.s_e = static_cast<C>(1.0 / cp.tau_e);
  k.s_eps = static_cast<C>(1.0 / cp.tau_eps);
  k.s_q = static_cast<C>(1.0 / cp.tau_q);
  k.s_s = static_cast<C>(1.0 / cp.tau_s);
  k.s_j = static_cast<C>(1.0 / cp.tau_j);
  k.h_e = static_cast<C>(1.0 - 0.5 / cp.tau_e);
  k.h_eps = static_cast<C>(1.0 - 0.5 / cp.tau_eps);
  k.h_q = static_cast<C>(1.0 - 0.5 / cp.tau_q);
  k.h_s = static_cast<C>(1.0 - 0.5 / cp.tau_s);
  k.h_j = static_cast<C>(1.0 - 0.5 / cp.tau_j);
  k.sc = static_cast<C>(scale);
  k.inv_sc = static_cast<C>(1.0 / scale);
  k.ax = static_cast<C>(ax);
  k.ay = static_cast<C>(ay);
  k.nx = nx;
  k.ny = ny;
  k.pitch = pitch;
  k.periodic_x = px;
  k.periodic_y = py;
  k.diffuse_mode = diffuse_mode;
  k.plane = plane;
  return k;
}

// Validation and layout of one case (lbm_api.cu).
int build_host_case(const lbm_domain_t *dom, const uint8_t *solid, size_t n_links,
                    const int32_t *link_x, const int32_t *link_y, const int32_t *link_dir,
                    const double *link_q, const double *link_ubx, const double *link_uby,
                    double Kn, const lbm_params_t *params, HostCase *hc, std::string *err);

// Host-side FP64 precompute (lbm_params.cpp).  Returns "" or an error text.
std::string compute_case_params(double Kn, double H, const lbm_params_t &p, CaseParams *out);
// Per-link l and r (Sec. 3.B) and the folded coefficients above.
std::string compute_link_coefs(const CaseParams &cp, const lbm_params_t &p, size_t n,
                               const int32_t *dir, const double *q, const double *ubx,
                               const double *uby, double *r_out, double *l_out,
                               double *coef8_out /* n x 8 */, int64_t *n_clamped);

// Step kernel geometry: one thread per node, kStepThreads nodes of a row
// per CTA, registers bounded for kStepMinBlocks resident CTAs per SM.
constexpr int kStepThreads = 256;
template <typename T>
struct StepOcc {
  static constexpr int min_blocks = 6;  // FP32: 40 registers, no spills
};
template <>
struct StepOcc<double> {
  static constexpr int min_blocks = 2;
};

// Kernel launchers (lbm_kernels.cu).  All return the launch error code.
template <typename T, typename C>
cudaError_t launch_step(const T *src, T *dst, const uint8_t *flags, const int32_t *lbase,
                        const LinkCoef<C> *links, const StepConst<C> &k, cudaStream_t s);

template <typename T>
cudaError_t launch_residual(const T *cur, const T *prev, const uint8_t *flags, int32_t nx,
                            int32_t ny, int32_t pitch, int64_t plane, double ax, double ay,
                            double scale, double *partials, double *result, cudaStream_t s);

template <typename T>
cudaError_t launch_fields(const T *f, const uint8_t *flags, int32_t nx, int32_t ny,
                          int32_t pitch, int64_t plane, double ax, double ay, double scale,
                          double *rho, double *ux, double *uy, cudaStream_t s);

template <typename T>
cudaError_t launch_export_f(const T *f, const uint8_t *flags, int32_t nx, int32_t ny, int32_t pitch, int64_t plane,
                            double scale, double *out, cudaStream_t s);

template <typename T>
cudaError_t launch_set_fields(const double *rho, const double *ux, const double *uy,
                              const uint8_t *flags, int32_t nx, int32_t ny, int32_t pitch,
                              int64_t plane, int32_t px, int32_t py, double ax, double ay,
                              double tau_s, double scale, T *f0, T *f1, cudaStream_t s);

template <typename T>
cudaError_t launch_import_f(const double *in, int32_t nx, int32_t ny, int32_t pitch,
                            int64_t plane, double scale, T *f, cudaStream_t s);

// Fixed reduction geometry: deterministic partial order on every device.
constexpr int kResidualBlocks = 1024;
constexpr int kResidualThreads = 256;
constexpr int kPartialStride = 4;  // num, den, mass deviation, non-finite count

}  // namespace lbm
