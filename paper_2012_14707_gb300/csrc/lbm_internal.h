// Internal declarations shared by the host side and the kernels of liblbm.so.
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <thread>
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
  // Relaxation rates s = 1/tau of e, eps, q and the stress (p_xx, p_xy),
  // as the collide function consumes them: s and the forcing weight 1 - s/2
  // (Eq. MomentPost), each times the moment's entry of
  // diag(1/36, 1/36, 1/12, 1/4) in M^-1 (x3 = 2 (1 - s_s/2) / 4); the
  // forcing weights also times the storage scale S (1 but for FP16).  The
  // momentum rows need no rate (collide): j6 = S / 6.  w3c = 3 S.
  C e2, e3, p2, p3, q2, q3, x2, x3, y3, j6, w3c;
  C sc, inv_sc;                 // storage scale of the 16-bit types (1 otherwise)
  C ax, ay;                     // body acceleration
  int32_t nx, ny, pitch;        // lattice size; row pitch (unused by the compacted lattice)
  int32_t periodic_x, periodic_y;
  int32_t diffuse_mode;         // reading of the Maxwell part, see LinkCoef
  int32_t n_fluid;              // fluid nodes (compacted lattice)
  int64_t plane;                // elements per population plane (padded fluid-node count)
  uint32_t sr_seed;             // seed of this time step's random bits (step_seed)
  int32_t exact;                // 1: the exact-mass variant (FP32 storage, moving walls)
  int32_t residual_mode;        // params.residual_mode (the batched reduction reads it)
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

// The FP64 coefficients k1, k2, k3, alpha of a link as pairs of FP32 values
// (hi + lo, lo the FP32 rounding of what hi leaves): the exact-mass variant
// evaluates its links in double-FP32 arithmetic.
struct alignas(16) LinkCoefDF {
  float hi[4], lo[4];
};
inline LinkCoefDF link_coef_df(const double *c) {
  LinkCoefDF r;
  for (int i = 0; i < 4; i++) {
    r.hi[i] = static_cast<float>(c[i]);
    r.lo[i] = static_cast<float>(c[i] - static_cast<double>(r.hi[i]));
  }
  return r;
}

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
  bool moving_walls = false;           // some link has a nonzero wall velocity
};
// FP32 storage runs the exact-mass variant of the step (collide,
// link_epilogue_pull: double-FP32 link values and rest-population closure,
// each with a carry of what FP32 storage dropped) always with
// params.mass_mode = 1, never with -1, and by default where a wall moves or
// the lattice has no boundary links (a periodic lattice whose flow tends to
// be uniform, so that every node rounds the same values the same way and
// nothing averages out).
inline bool exact_mass(const HostCase &hc) {
  if (hc.params.precision != LBM_FP32 || hc.params.mass_mode < 0) return false;
  return hc.params.mass_mode > 0 || hc.moving_walls || hc.n_links == 0;
}

// Bits above the flag byte in a compacted lattice's node word (.x; the
// full layout is described at CompactCase).
constexpr uint32_t kMetaWrapE = 1u << 8;  // x = nx - 1 on a periodic x axis
constexpr uint32_t kMetaWrapW = 1u << 9;  // x = 0 on a periodic x axis
constexpr uint32_t kNodeMeta = 0x3FFu;    // flag byte and the two seam bits
constexpr int kGroup = 32;                // nodes per group record (CompactCase::grp)
constexpr int kMaxGroupRows = 1 << 14;    // rows a group may span (14-bit row offset)

// Row offset of a node from its group's first row, and the offset of its
// first link from the group's first link (node word bits .x 10..15 with
// .y 24..31, and .y 16..23).
__host__ __device__ inline int node_dy(uint2 nw) {
  return static_cast<int>(((nw.x >> 10) & 63u) | ((nw.y >> 24) << 6));
}
__host__ __device__ inline uint32_t node_loff(uint2 nw) { return (nw.y >> 16) & 255u; }

// Rows of the compacted lattice above and below row y (wrapped where y is
// periodic; a non-periodic axis has solid edge rows, so fluid rows never
// need the wrap).
__host__ __device__ inline int row_above(int y, int ny, int periodic_y) {
  return y + 1 < ny ? y + 1 : (periodic_y ? 0 : y);
}
__host__ __device__ inline int row_below(int y, int ny, int periodic_y) {
  return y > 0 ? y - 1 : (periodic_y ? ny - 1 : y);
}

// n_lb and s_lb of fluid node i in row y (see CompactCase) from its node
// word, which holds n_lb - i and i - s_lb, each plus the fluid count n
// where the row above (below) is reached across a periodic y axis: both
// are then in [0, nx], and no row table is read.
__host__ __device__ inline void neighbour_rows(uint2 nw, uint32_t i, uint32_t n, int y, int ny,
                                               int periodic_y, uint32_t &nb, uint32_t &sb) {
  const uint32_t dn = nw.x >> 16, ds = nw.y & 0xFFFFu;
  nb = i + dn - ((periodic_y && y == ny - 1) ? n : 0u);
  sb = i - ds + ((periodic_y && y == 0) ? n : 0u);
}

// Compacted indices of the neighbours x + c_q (q = 1..8, tq[0] = i) of
// fluid node i in row y, from its node word m, n_lb / s_lb and rowstart
// (pull_slots gathers direction q from the neighbour x - c_q = x + c_opp(q)).
// Neighbours in the own row are i +- 1; in the rows above and below n_lb or
// s_lb, +1 past a fluid (x, y +- 1) (bits 3 and 1 of the flag byte clear),
// -1 for x - 1; across the periodic seam of x the row's first or last fluid
// node.  Only targets that are fluid (bit opp(q) - 1 of the flag byte
// clear) are meaningful.  Shared by the kernels and host-side checks.
__host__ __device__ inline void compact_targets(uint32_t m, uint32_t i, uint32_t nb, uint32_t sb,
                                                int y, int ny, int periodic_y,
                                                const int32_t *rowstart, uint32_t (&tq)[9]) {
  tq[0] = i;
  tq[1] = i + 1;
  tq[2] = nb;
  tq[3] = i - 1;
  tq[4] = sb;
  tq[5] = nb + ((m & (1u << 3)) ? 0u : 1u);
  tq[6] = nb - 1;
  tq[7] = sb - 1;
  tq[8] = sb + ((m & (1u << 1)) ? 0u : 1u);
  if (m & (kMetaWrapE | kMetaWrapW)) {
    // the seam exists only on a periodic x axis
    const int yn = row_above(y, ny, periodic_y);
    const int ys = row_below(y, ny, periodic_y);
    if (m & kMetaWrapE) {
      tq[1] = static_cast<uint32_t>(rowstart[y]);
      tq[5] = static_cast<uint32_t>(rowstart[yn]);
      tq[8] = static_cast<uint32_t>(rowstart[ys]);
    }
    if (m & kMetaWrapW) {
      tq[3] = static_cast<uint32_t>(rowstart[y + 1] - 1);
      tq[6] = static_cast<uint32_t>(rowstart[yn + 1] - 1);
      tq[7] = static_cast<uint32_t>(rowstart[ys + 1] - 1);
    }
  }
}

// Where a lattice keeps node i's populations (pull layout).
// A step stores f'_q(x, t) in x's own slot q * P + i, so that its stores
// are aligned and coalesced, and the next step gathers
// f_q(x, t + 1) = f'_q(x - c_q, t) from the slot of x - c_q, which is the
// push target of direction opp(q) (compact_targets).  Where x - c_q is
// solid (a boundary link), f_q(x, t + 1) is Eq. EqNewBDSC, which x itself
// evaluates during step t (every input is x's own) and keeps in the
// lattice's link tail: element 9 P + (index of the link), links sorted by
// node, then direction.  Every slot holds one population of one node, so
// the gather below is also the scatter that writes a state.
struct PullGeom {
  const uint2 *node = nullptr;      // node words (CompactCase::node)
  const int2 *grp = nullptr;        // group records (CompactCase::grp)
  const int32_t *rowstart = nullptr;
  const uint32_t *jbslot = nullptr; // per link (x, j): pull slot of f_jb(x) (link_jb_slots)
  const uint16_t *ldesc = nullptr;  // per link (x, j): (x mod 64) << 4 | j (link_descriptors)
  int32_t ny = 0, periodic_y = 0;
  uint32_t plane = 0;               // P
  uint32_t n_fluid = 0;
  uint32_t pf_dist = 0;             // step kernel: CTAs ahead whose data it prefetches to L2
  // the exact-mass variant (FP32 storage): FP64 link coefficients and, per
  // link and per node (rest population), the remainder of its values that
  // FP32 storage has not yet taken
  const LinkCoefDF *links64 = nullptr;
  float *carry = nullptr;
  float *carry0 = nullptr;
};

// s[q] = element of the pre-collision f_q of fluid node i, q = 0..8.
__host__ __device__ inline void pull_slots(uint2 nw, int2 grp, uint32_t i, uint32_t P,
                                           uint32_t n_fluid, int ny, int periodic_y,
                                           const int32_t *rowstart, uint32_t (&s)[9]) {
  const uint32_t m = nw.x & kNodeMeta;
  const int y = grp.x + node_dy(nw);
  uint32_t nb, sb;
  neighbour_rows(nw, i, n_fluid, y, ny, periodic_y, nb, sb);
  uint32_t tq[9];
  compact_targets(m, i, nb, sb, y, ny, periodic_y, rowstart, tq);
  uint32_t li = 9u * P + static_cast<uint32_t>(grp.y) + node_loff(nw);
  // bit q - 1 of the flag byte set <=> x - c_q solid; opp = {0, 3, 4, 1, 2, 7, 8, 5, 6}
  s[0] = i;
  s[1] = (m & 0x01u) ? li++ : 1u * P + tq[3];
  s[2] = (m & 0x02u) ? li++ : 2u * P + tq[4];
  s[3] = (m & 0x04u) ? li++ : 3u * P + tq[1];
  s[4] = (m & 0x08u) ? li++ : 4u * P + tq[2];
  s[5] = (m & 0x10u) ? li++ : 5u * P + tq[7];
  s[6] = (m & 0x20u) ? li++ : 6u * P + tq[8];
  s[7] = (m & 0x40u) ? li++ : 7u * P + tq[5];
  s[8] = (m & 0x80u) ? li : 8u * P + tq[6];
}

// Where node (x, y) of a case lives in its compacted lattice: the index
// map y * nx + x -> compacted index, -1 for solid nodes.  at() returns the
// compacted index, or -1 for a solid node; slots() the elements of its nine
// populations: q * plane + i in the push layout of the batched solver's
// arena (pull.node null), pull_slots in the pull layout of a single case.
struct NodeMap {
  const int32_t *index = nullptr;
  int32_t nx = 0, ny = 0;
  PullGeom pull{};
  __host__ __device__ int64_t at(int x, int y) const {
    return index[static_cast<int64_t>(y) * nx + x];
  }
  __host__ __device__ void slots(uint32_t i, uint32_t plane, uint32_t (&s)[9]) const {
    if (pull.node) {
      pull_slots(pull.node[i], pull.grp[i / kGroup], i, plane, pull.n_fluid, pull.ny,
                 pull.periodic_y, pull.rowstart, s);
    } else {
      for (int q = 0; q < 9; q++) s[q] = static_cast<uint32_t>(q) * plane + i;
    }
  }
};


// Compacted lattice of one case (host copy): only fluid nodes, in
// row-major order, each population plane padded to `plane` elements.
//   node     one 8-byte word per node, what the step kernels read:
//            .x bits 0..7   flag byte (bit q - 1: x - c_q solid)
//               bits 8, 9   kMetaWrapE / kMetaWrapW (periodic seam of x)
//               bits 10..15 row offset dy from the group's row, low 6 bits
//               bits 16..31 n_lb - i (+ n_fluid across a periodic y axis)
//            .y bits 0..15  i - s_lb (+ n_fluid across a periodic y axis)
//               bits 16..23 first link of the node - first link of its group
//               bits 24..31 dy, high 8 bits
//            n_lb / s_lb = compacted index of the first fluid node at or
//            after (x, y+1) / (x, y-1) (rows wrapped where periodic); both
//            differences are at most nx <= 65535 (neighbour_rows)
//   grp      one record per group of kGroup consecutive nodes (node i is in
//            group i / kGroup): .x = row of the group's first node,
//            .y = first link of the group's first node with links; a group
//            spans fewer than kMaxGroupRows rows, and holds at most
//            kGroup * 8 links, so the offsets fit the node word
//   lbase    first link of the node (links sorted by node, then direction)
//   rowstart compacted index of every row's first fluid node (ny + 1)
//   index    y * nx + x -> compacted index or -1 (conversions only)
struct CompactCase {
  int64_t n_fluid = 0, plane = 0;
  std::vector<int32_t> lbase, rowstart, index;
  std::vector<uint2> node;
  std::vector<int2> grp;
};
// Returns "" or the reason the case does not fit the node word.
std::string build_compact(const HostCase &hc, CompactCase *cc);
// For every link (node x, direction j) of a compacted case, in link-table
// order: the pull slot of f_jb(x, t) (jb = opp(j)), the pre-collision value
// Eq. EqNewBDSC takes from x.  The step kernel's link epilogue reads it
// there instead of recomputing the neighbour's index.
std::vector<uint32_t> link_jb_slots(const CompactCase &cc, int ny, int periodic_y,
                                    int64_t n_links);

// For every link (node x, direction j) of a compacted case, in link-table
// order: (x mod 64) << 4 | j.  A warp of the paired 16-bit step runs the 64
// nodes of one 64-aligned block (x mod 64 is the node's place in it), so
// each lane finds its link's node and direction from this one entry.
std::vector<uint16_t> link_descriptors(const CompactCase &cc, int64_t n_links);

// Kernel constants of one case in arithmetic type C.
template <typename C>
StepConst<C> make_step_const(const CaseParams &cp, int32_t nx, int32_t ny, int32_t pitch,
                             int64_t plane, int64_t n_fluid, int32_t px, int32_t py, double ax,
                             double ay, int32_t diffuse_mode, double scale) {
  StepConst<C> k;
  {
    const double se = 1.0 / cp.tau_e, sp = 1.0 / cp.tau_eps, sq = 1.0 / cp.tau_q,
                 ss = 1.0 / cp.tau_s;
    k.e2 = static_cast<C>(se / 36.0);
    k.e3 = static_cast<C>(scale * (1.0 - 0.5 * se) / 36.0);
    k.p2 = static_cast<C>(sp / 36.0);
    k.p3 = static_cast<C>(scale * (1.0 - 0.5 * sp) / 36.0);
    k.q2 = static_cast<C>(sq / 12.0);
    k.q3 = static_cast<C>(scale * (1.0 - 0.5 * sq) / 12.0);
    k.x2 = static_cast<C>(ss / 4.0);
    k.x3 = static_cast<C>(scale * (1.0 - 0.5 * ss) / 2.0);
    k.y3 = static_cast<C>(scale * (1.0 - 0.5 * ss) / 4.0);
    k.j6 = static_cast<C>(scale / 6.0);
    k.w3c = static_cast<C>(3.0 * scale);
  }
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
  k.n_fluid = static_cast<int32_t>(n_fluid);
  k.sr_seed = 0;
  k.exact = 0;
  k.residual_mode = 0;
  return k;
}

// Host-side preparation runs over rows or links in parallel: f(begin, end)
// on contiguous ranges of [0, n), one per hardware thread.  Every index is
// handled independently, so the result does not depend on the split.
template <typename F>
void parallel_for(int64_t n, F &&f, int64_t min_per_thread = 1 << 14) {
  const int64_t hw = std::max<int64_t>(1, static_cast<int64_t>(std::thread::hardware_concurrency()));
  const int64_t T = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(hw, 64), n / min_per_thread));
  if (T <= 1) {
    f(int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(static_cast<size_t>(T));
  for (int64_t t = 0; t < T; t++) {
    const int64_t b = n * t / T, e = n * (t + 1) / T;
    th.emplace_back([&f, b, e] { f(b, e); });
  }
  for (auto &t : th) t.join();
}

// Validation and layout of one case (lbm_api.cu).
int build_host_case(const lbm_domain_t *dom, const uint8_t *solid, size_t n_links,
                    const int32_t *link_x, const int32_t *link_y, const int32_t *link_dir,
                    const double *link_q, const double *link_ubx, const double *link_uby,
                    double Kn, const lbm_params_t *params, HostCase *hc, std::string *err);

// Host-side FP64 precompute (lbm_params.cpp).  Returns "" or an error text.
std::string compute_case_params(double Kn, double H, const lbm_params_t &p, CaseParams *out);
// Per-link l and r (Sec. 3.B) and the folded coefficients above, from the
// link's c_i . u_b, weight w_i and |u_b|^2 (any lattice; the D2Q9 entry
// below computes them from the direction).
std::string compute_link_coefs_general(const CaseParams &cp, const lbm_params_t &p, size_t n,
                                       const double *q, const double *cub, const double *w,
                                       const double *uu, double *r_out, double *l_out,
                                       double *coef8_out /* n x 8 */, int64_t *n_clamped);
// Per-link l and r (Sec. 3.B) and the folded coefficients above.
std::string compute_link_coefs(const CaseParams &cp, const lbm_params_t &p, size_t n,
                               const int32_t *dir, const double *q, const double *ubx,
                               const double *uby, double *r_out, double *l_out,
                               double *coef8_out /* n x 8 */, int64_t *n_clamped);

// Step kernel geometry (single case and batch): one thread per fluid
// node; the single-case kernel runs kPullThreads consecutive fluid nodes per
// CTA.  PullOcc<T>::min_blocks CTAs of kPullThreads threads per SM bound
// the registers (the batch scales it to its CTA width).
constexpr int kPullThreads = 128;
template <typename T>
struct PullOcc {
  // FP32: 32 registers, 64 warps per SM -- more warps hide the load latency
  // better than 40 registers without spills (one spilled register stays in L1)
  static constexpr int min_blocks = 16;
};
template <>
struct PullOcc<double> {
  static constexpr int min_blocks = 4;
};
// 16-bit storage: the conversions need more registers; 40 (12 CTAs/SM, no
// spills) beat 32 (16 CTAs, spills) and 48 or 64 (fewer warps).
template <>
struct PullOcc<__half> {
  static constexpr int min_blocks = 12;
};
template <>
struct PullOcc<__nv_bfloat16> {
  static constexpr int min_blocks = 12;
};

// The 16-bit step runs fluid-node pairs (step_pair_pull): kPairThreads
// threads per CTA, two nodes each; PairOcc bounds the registers.
constexpr int kPairThreads = 128;
struct PairOcc {
  static constexpr int min_blocks = 8;
};

// Kernel launchers (lbm_kernels.cu).  All return the launch error code.
// CTAs of step_kernel_pull<T, C> resident at once on the current device.
template <typename T, typename C>
int pull_resident_ctas();
template <typename T, typename C>
cudaError_t launch_step_pull(const T *src, T *dst, const PullGeom &g, int64_t n_fluid,
                             const LinkCoef<C> *links, const StepConst<C> &k, cudaStream_t s);

// Residual and mass of the states in cur and prev (the lattices of two
// consecutive steps), nodes in the layout of map.
template <typename T>
cudaError_t launch_residual_compact(const T *cur, const T *prev, const NodeMap &map,
                                    int64_t n_fluid, int64_t plane, double ax, double ay,
                                    double scale, double *partials, double *result, cudaStream_t s);

// The interval residual (params.residual_mode 1): num, den, mass deviation
// and non-finite count of the state in cur against the velocity snapshot
// snap (two values of the storage's arithmetic type per fluid node), which
// it then replaces with the state's velocity; partials and result as
// launch_residual_compact.
template <typename T>
cudaError_t launch_residual_interval(const T *cur, const NodeMap &map, int64_t n_fluid,
                                     int64_t plane, double ax, double ay, double scale, void *snap,
                                     double *partials, double *result, cudaStream_t s);

// Conversions between a compacted lattice (see NodeMap) and
// caller arrays over the nx x ny nodes (row-major, y * nx + x).
template <typename T>
cudaError_t launch_fields(const T *f, const NodeMap &map, int64_t plane, double ax, double ay,
                          double scale, double *rho, double *ux, double *uy, cudaStream_t s);

template <typename T>
cudaError_t launch_export_f(const T *f, const NodeMap &map, int64_t plane, double scale,
                            double *out, cudaStream_t s);

template <typename T>
cudaError_t launch_set_fields(const double *rho, const double *ux, const double *uy,
                              const NodeMap &map, int64_t plane, int32_t px, int32_t py,
                              double ax, double ay, double tau_s, double scale, T *f0, T *f1,
                              cudaStream_t s);

template <typename T>
cudaError_t launch_import_f(const double *in, const NodeMap &map, int64_t plane, double scale,
                            T *f, cudaStream_t s);

// Fixed reduction geometry: deterministic partial order on every device.
constexpr int kResidualBlocks = 4096;
constexpr int kResidualThreads = 256;
constexpr int kPartialStride = 4;  // num, den, mass deviation, non-finite count

}  // namespace lbm
