// C ABI of liblbm.so (declared in include/lbm.h): validation, the host-side
// layout build, device memory, and the step / residual / field calls.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm_device.cuh"
#include "lbm_internal.h"

struct lbm_handle {
  int precision = LBM_FP32;
  cudaStream_t stream = nullptr;
  int device = 0;
  int32_t nx = 0, ny = 0, pitch = 0, px = 0, py = 0;
  int64_t plane = 0;
  double ax = 0.0, ay = 0.0;
  double scale = 1.0;  // storage scale of the 16-bit types
  lbm::CaseParams cp{};
  lbm_params_t params{};
  void *f[2] = {nullptr, nullptr};
  int cur = 0;
  // compacted lattice in the pull layout (see lbm::CompactCase, lbm::pull_slots);
  // f[b] holds 9 planes of `plane` elements, then the link tail
  uint2 *node = nullptr;  // per fluid node: flags, seam bits, row and link offsets
  int2 *grp = nullptr;    // per group of lbm::kGroup nodes: first row, first link
  uint32_t *jbslot = nullptr;  // per link: slot of f_jb(x, t) (lbm::link_jb_slots)
  uint16_t *ldesc = nullptr;   // per link: (x mod 64) << 4 | j (lbm::link_descriptors)
  uint32_t pf_dist = 0;        // L2 prefetch distance of the step kernel, in CTAs
  int32_t *rowstart = nullptr;
  int32_t *index = nullptr;  // y * nx + x -> compacted index or -1
  void *links = nullptr;
  // the exact-mass variant (FP32 storage with moving walls): FP64 link
  // records and the per-link carry (see lbm::link_epilogue_pull)
  int exact = 0;
  lbm::LinkCoefDF *links64 = nullptr;
  float *carry = nullptr;   // per link
  float *carry0 = nullptr;  // per fluid node (rest population)
  // interval residual (params.residual_mode 1): velocity of every fluid
  // node at the step snap_steps (two values of the arithmetic type)
  void *snap = nullptr;
  int64_t snap_steps = 0;
  double *partials = nullptr;
  double *result = nullptr;
  double *h_result = nullptr;  // pinned, 4 doubles
  int64_t n_fluid = 0, n_links = 0, steps = 0, dev_bytes = 0;
  size_t fbytes = 0;          // bytes of one lattice (nine planes + link tail)
  uint64_t fingerprint = 0;   // of the case's inputs (checkpoint files)
  std::vector<double> link_r, link_l;
  std::string err;
};

namespace {

thread_local std::string g_create_error;

const int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

int fail(lbm_handle_t *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(lbm_handle_t *h, cudaError_t e, const char *what) {
  return fail(h, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CK(h, call)                                 \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

// FNV-1a over 8-byte words (the tail byte by byte): a fingerprint of a
// case's inputs for checkpoint files, not a cryptographic hash.
struct Fnv64 {
  uint64_t h = 1469598103934665603ull;
  void bytes(const void *p, size_t n) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
      uint64_t w;
      std::memcpy(&w, c + i, 8);
      h = (h ^ w) * 1099511628211ull;
    }
    for (; i < n; i++) h = (h ^ c[i]) * 1099511628211ull;
  }
  template <typename V>
  void value(const V &v) {
    bytes(&v, sizeof(v));
  }
  // Large arrays: 1 MiB chunks hashed on all host threads, then the chunk
  // hashes in order (the result does not depend on the thread count).
  void big(const void *p, size_t n) {
    constexpr size_t kChunkBytes = size_t(1) << 20;
    const size_t nc = (n + kChunkBytes - 1) / kChunkBytes;
    std::vector<uint64_t> part(nc);
    const unsigned char *c = static_cast<const unsigned char *>(p);
    lbm::parallel_for(static_cast<int64_t>(nc), [&](int64_t k0, int64_t k1) {
      for (int64_t k = k0; k < k1; k++) {
        Fnv64 f;
        const size_t off = static_cast<size_t>(k) * kChunkBytes;
        f.bytes(c + off, std::min(kChunkBytes, n - off));
        part[static_cast<size_t>(k)] = f.h;
      }
    }, 4);
    value(n);
    bytes(part.data(), part.size() * sizeof(uint64_t));
  }
};

size_t elem_size(int precision) {
  return precision == LBM_FP64 ? 8 : (precision == LBM_FP32 ? 4 : 2);
}

// Calls f(T*, C*) with null pointers whose types name the storage type T and
// the arithmetic type C of `precision`.
template <typename F>
cudaError_t dispatch(int precision, F &&f) {
  switch (precision) {
    case LBM_FP64: return f(static_cast<double *>(nullptr), static_cast<double *>(nullptr));
    case LBM_FP32: return f(static_cast<float *>(nullptr), static_cast<float *>(nullptr));
    case LBM_BF16: return f(static_cast<__nv_bfloat16 *>(nullptr), static_cast<float *>(nullptr));
    default: return f(static_cast<__half *>(nullptr), static_cast<float *>(nullptr));
  }
}
#define LBM_TYPES(tT, tC)                              \
  using T = std::remove_pointer_t<decltype(tT)>;       \
  using C = std::remove_pointer_t<decltype(tC)>;       \
  (void)sizeof(T);                                     \
  (void)sizeof(C)

void release(lbm_handle_t *h) {
  if (!h) return;
  cudaStream_t s = h->stream;
  cudaStreamSynchronize(s);
  for (void *p : {h->f[0], h->f[1], static_cast<void *>(h->node), static_cast<void *>(h->grp),
                  static_cast<void *>(h->jbslot), static_cast<void *>(h->ldesc),
                  static_cast<void *>(h->rowstart), static_cast<void *>(h->index), h->links,
                  static_cast<void *>(h->links64), static_cast<void *>(h->carry), h->snap,
                  static_cast<void *>(h->partials), static_cast<void *>(h->result)})
    if (p) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  if (h->h_result) cudaFreeHost(h->h_result);
  delete h;
}

template <typename C>
lbm::StepConst<C> step_const(const lbm_handle_t *h) {
  lbm::StepConst<C> k = lbm::make_step_const<C>(h->cp, h->nx, h->ny, 0, h->plane, h->n_fluid,
                                                h->px, h->py, h->ax, h->ay,
                                                h->params.diffuse_mode, h->scale);
  k.sr_seed = lbm::dev::step_seed(h->steps);
  k.exact = h->exact;
  return k;
}

lbm::PullGeom pull_geom(const lbm_handle_t *h) {
  lbm::PullGeom g;
  g.node = h->node;
  g.grp = h->grp;
  g.rowstart = h->rowstart;
  g.jbslot = h->jbslot;
  g.ldesc = h->ldesc;
  g.ny = h->ny;
  g.periodic_y = h->py;
  g.plane = static_cast<uint32_t>(h->plane);
  g.n_fluid = static_cast<uint32_t>(h->n_fluid);
  g.pf_dist = h->pf_dist;
  g.links64 = h->links64;
  g.carry = h->carry;
  g.carry0 = h->carry0;
  return g;
}

// Bytes of the exact-mass variant's carries (per link, then per node).
size_t carry_bytes(const lbm_handle_t *h) {
  return h->exact ? static_cast<size_t>(std::max<int64_t>(1, h->n_links) + h->plane) * sizeof(float)
                  : 0;
}

// Zero the carries of the exact-mass variant (a new state owes nothing).
cudaError_t clear_carry(lbm_handle_t *h) {
  if (!h->exact) return cudaSuccess;
  return cudaMemsetAsync(h->carry, 0, carry_bytes(h), h->stream);
}

// The interval residual's kernel on the current state: partials, result
// and the new velocity snapshot (the previous one is read first).
cudaError_t interval_residual_launch(lbm_handle_t *h);

// Start a new interval at the current state (the snapshot becomes its
// velocity field).
cudaError_t reset_interval(lbm_handle_t *h) {
  if (!h->snap) return cudaSuccess;
  const cudaError_t e = interval_residual_launch(h);
  h->snap_steps = h->steps;
  return e;
}

lbm::NodeMap node_map(const lbm_handle_t *h) {
  lbm::NodeMap m;
  m.index = h->index;
  m.nx = h->nx;
  m.ny = h->ny;
  m.pull = pull_geom(h);
  return m;
}

cudaError_t interval_residual_launch(lbm_handle_t *h) {
  return dispatch(h->precision, [&](auto tT, auto tC) {
    LBM_TYPES(tT, tC);
    return lbm::launch_residual_interval<T>(static_cast<const T *>(h->f[h->cur]), node_map(h),
                                            h->n_fluid, h->plane, h->ax, h->ay, h->scale, h->snap,
                                            h->partials, h->result, h->stream);
  });
}

cudaError_t do_step(lbm_handle_t *h) {
  const int src = h->cur, dst = 1 - h->cur;
  cudaError_t e = dispatch(h->precision, [&](auto tT, auto tC) {
    LBM_TYPES(tT, tC);
    return lbm::launch_step_pull<T, C>(static_cast<const T *>(h->f[src]),
                                       static_cast<T *>(h->f[dst]), pull_geom(h), h->n_fluid,
                                       static_cast<const lbm::LinkCoef<C> *>(h->links),
                                       step_const<C>(h), h->stream);
  });
  if (e == cudaSuccess) {
    h->cur = dst;
    h->steps++;
  }
  return e;
}

}  // namespace

namespace lbm {
// Validation and host-side layout of one case: flags, link-table bases and
// the node-sorted link coefficients (used by lbm_create and
// lbm_batch_create).  Returns a status code; *err gets the message.
int build_host_case(const lbm_domain_t *dom, const uint8_t *solid, size_t n_links,
                    const int32_t *link_x, const int32_t *link_y, const int32_t *link_dir,
                    const double *link_q, const double *link_ubx, const double *link_uby,
                    double Kn, const lbm_params_t *params, lbm::HostCase *hc,
                    std::string *err) {
  auto bad = [err](int code, const std::string &m) {
    *err = m;
    return code;
  };
  if (!dom || !solid || !params) return bad(LBM_EINVAL, "null argument");
  if (n_links && (!link_x || !link_y || !link_dir || !link_q || !link_ubx || !link_uby))
    return bad(LBM_EINVAL, "null link array");
  const lbm_params_t &p = *params;
  if (dom->nx < 1 || dom->ny < 1) return bad(LBM_EINVAL, "nx and ny must be >= 1");
  if (p.precision < LBM_FP64 || p.precision > LBM_FP16)
    return bad(LBM_EINVAL, "precision must be LBM_FP64, LBM_FP32, LBM_BF16 or LBM_FP16");
  if (!(p.storage_scale >= 0.0) || !std::isfinite(p.storage_scale))
    return bad(LBM_EINVAL, "storage_scale must be 0 (default) or a positive power of two");
  if (p.diffuse_mode != 0 && p.diffuse_mode != 1) return bad(LBM_EINVAL, "diffuse_mode must be 0 or 1");
  if (p.residual_every < 1) return bad(LBM_EINVAL, "residual_every must be >= 1");
  if (p.mass_mode < -1 || p.mass_mode > 1) return bad(LBM_EINVAL, "mass_mode must be -1, 0 or 1");
  if (p.residual_mode != 0 && p.residual_mode != 1)
    return bad(LBM_EINVAL, "residual_mode must be 0 or 1");
  if (!std::isfinite(dom->ax) || !std::isfinite(dom->ay)) return bad(LBM_EINVAL, "non-finite force");
  const int32_t nx = dom->nx, ny = dom->ny;
  // 32-bit element offsets in the kernels: 9 planes of the padded lattice < 2^31.
  if ((static_cast<int64_t>(nx) + 31) / 32 * 32 * ny * 9 >= (int64_t(1) << 31))
    return bad(LBM_EINVAL, "lattice too large: 9 * pitch * ny must stay below 2^31");
  // the node word keeps n_lb - i and i - s_lb (at most nx) in 16 bits
  if (nx > 65535) return bad(LBM_EINVAL, "rows longer than 65535 nodes are not supported");
  if (n_links > static_cast<size_t>(std::numeric_limits<int32_t>::max()))
    return bad(LBM_EINVAL, "too many links");
  const int px = dom->periodic_x ? 1 : 0, py = dom->periodic_y ? 1 : 0;
  // Non-periodic axes need solid edges so that no fluid node streams off the lattice.
  if (!px)
    for (int32_t y = 0; y < ny; y++)
      if (!solid[(size_t)y * nx] || !solid[(size_t)y * nx + nx - 1])
        return bad(LBM_EINVAL, "non-periodic x needs solid first and last columns");
  if (!py)
    for (int32_t x = 0; x < nx; x++)
      if (!solid[x] || !solid[(size_t)(ny - 1) * nx + x])
        return bad(LBM_EINVAL, "non-periodic y needs solid first and last rows");

  lbm::CaseParams cp;
  std::string msg = lbm::compute_case_params(Kn, dom->H, p, &cp);
  if (!msg.empty()) return bad(LBM_EINVAL, msg);

  const int32_t align = 32;
  const int32_t pitch = (nx + align - 1) / align * align;
  const int64_t plane = static_cast<int64_t>(pitch) * ny;
  std::vector<uint8_t> flags(static_cast<size_t>(plane), lbm::kSolid);
  std::vector<int64_t> row_fluid(static_cast<size_t>(ny), 0);
  lbm::parallel_for(ny, [&](int64_t y0, int64_t y1) {
    for (int64_t y = y0; y < y1; y++) {
      int64_t c = 0;
      for (int32_t x = 0; x < nx; x++)
        if (!solid[(size_t)y * nx + x]) {
          flags[(size_t)y * pitch + x] = 0;
          c++;
        }
      row_fluid[y] = c;
    }
  }, 64);
  int64_t n_fluid = 0;
  for (int64_t c : row_fluid) n_fluid += c;
  auto wrapped = [&](int32_t x, int32_t y, int dx, int dy, int32_t *xo, int32_t *yo) {
    int32_t a = x + dx, b = y + dy;
    if (a < 0 || a >= nx) {
      if (!px) return false;
      a = (a + nx) % nx;
    }
    if (b < 0 || b >= ny) {
      if (!py) return false;
      b = (b + ny) % ny;
    }
    *xo = a;
    *yo = b;
    return true;
  };
  for (size_t k = 0; k < n_links; k++) {
    const int32_t x = link_x[k], y = link_y[k], i = link_dir[k];
    char buf[200];
    if (x < 0 || x >= nx || y < 0 || y >= ny || i < 1 || i > 8) {
      std::snprintf(buf, sizeof buf, "link %zu: node or direction out of range", k);
      return bad(LBM_EINVAL, buf);
    }
    if (!(link_q[k] > 0.0 && link_q[k] <= 1.0) || !std::isfinite(link_ubx[k]) ||
        !std::isfinite(link_uby[k])) {
      std::snprintf(buf, sizeof buf, "link %zu: gamma must lie in (0, 1], wall velocity finite", k);
      return bad(LBM_EINVAL, buf);
    }
    uint8_t &fl = flags[(size_t)y * pitch + x];
    int32_t xr, yr;
    if (solid[(size_t)y * nx + x] || !wrapped(x, y, -kCx[i], -kCy[i], &xr, &yr) ||
        !solid[(size_t)yr * nx + xr]) {
      std::snprintf(buf, sizeof buf, "link %zu: node must be fluid and x - c_i solid", k);
      return bad(LBM_EINVAL, buf);
    }
    if (fl & (1u << (i - 1))) {
      std::snprintf(buf, sizeof buf, "link %zu: duplicate (node, direction)", k);
      return bad(LBM_EINVAL, buf);
    }
    fl |= static_cast<uint8_t>(1u << (i - 1));
    if (link_ubx[k] != 0.0 || link_uby[k] != 0.0) hc->moving_walls = true;
  }
  // Every unknown direction of every fluid node needs its link (rows in
  // parallel; the first offending node in row-major order is reported).
  std::vector<int64_t> row_bad(static_cast<size_t>(ny), -1);  // x * 16 + kind (0: enclosed) or dir
  lbm::parallel_for(ny, [&](int64_t y0, int64_t y1) {
    for (int64_t y = y0; y < y1; y++)
      for (int32_t x = 0; x < nx && row_bad[y] < 0; x++) {
        if (solid[(size_t)y * nx + x]) continue;
        const uint8_t fl = flags[(size_t)y * pitch + x];
        if (fl == lbm::kSolid) {
          row_bad[y] = static_cast<int64_t>(x) * 16;
          break;
        }
        for (int i = 1; i < 9; i++) {
          int32_t xr, yr;
          const bool unknown = !wrapped(x, static_cast<int32_t>(y), -kCx[i], -kCy[i], &xr, &yr) ||
                               solid[(size_t)yr * nx + xr];
          if (unknown != static_cast<bool>(fl & (1u << (i - 1)))) {
            row_bad[y] = static_cast<int64_t>(x) * 16 + i;
            break;
          }
        }
      }
  }, 64);
  for (int32_t y = 0; y < ny; y++)
    if (row_bad[y] >= 0) {
      const int32_t x = static_cast<int32_t>(row_bad[y] / 16), i = static_cast<int32_t>(row_bad[y] % 16);
      if (i == 0) return bad(LBM_EINVAL, "fluid node enclosed on all eight sides");
      char buf[200];
      std::snprintf(buf, sizeof buf, "node (%d, %d) direction %d: no link for an unknown population",
                    x, y, i);
      return bad(LBM_EINVAL, buf);
    }

  // Per-link parameters (input order), then the node-sorted table.
  hc->link_r.assign(n_links, 0.0);
  hc->link_l.assign(n_links, 0.0);
  std::vector<double> coef(8 * n_links);
  msg = lbm::compute_link_coefs(cp, p, n_links, link_dir, link_q, link_ubx, link_uby,
                                hc->link_r.data(), hc->link_l.data(), coef.data(), &cp.n_clamped);
  if (!msg.empty()) return bad(LBM_EINVAL, msg);
  // Node-sorted table without a sort: the links of a node are its unknown
  // directions in order, so a link's slot is the node's first link (a
  // prefix sum of the per-node link counts in row-major order) plus the
  // number of the node's unknown directions below its own.
  std::vector<int64_t> row_links(static_cast<size_t>(ny) + 1, 0);
  lbm::parallel_for(ny, [&](int64_t y0, int64_t y1) {
    for (int64_t y = y0; y < y1; y++) {
      int64_t c = 0;
      for (int32_t x = 0; x < nx; x++) {
        const uint8_t fl = flags[(size_t)y * pitch + x];
        if (fl != lbm::kSolid) c += __builtin_popcount(fl);
      }
      row_links[y + 1] = c;
    }
  }, 64);
  for (int32_t y = 0; y < ny; y++) row_links[y + 1] += row_links[y];
  hc->lbase.assign(static_cast<size_t>(plane), -1);
  lbm::parallel_for(ny, [&](int64_t y0, int64_t y1) {
    for (int64_t y = y0; y < y1; y++) {
      int64_t c = row_links[y];
      for (int32_t x = 0; x < nx; x++) {
        const uint8_t fl = flags[(size_t)y * pitch + x];
        if (fl != lbm::kSolid && fl) {
          hc->lbase[(size_t)y * pitch + x] = static_cast<int32_t>(c);
          c += __builtin_popcount(fl);
        }
      }
    }
  }, 64);
  std::vector<int64_t> order(n_links);
  lbm::parallel_for(static_cast<int64_t>(n_links), [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; k++) {
      const size_t node = (size_t)link_y[k] * pitch + link_x[k];
      const uint32_t below = flags[node] & ((1u << (link_dir[k] - 1)) - 1u);
      order[hc->lbase[node] + __builtin_popcount(below)] = k;
    }
  });
  hc->coef.resize(4 * n_links);
  lbm::parallel_for(static_cast<int64_t>(n_links), [&](int64_t q0, int64_t q1) {
    for (int64_t q = q0; q < q1; q++)
      for (int j = 0; j < 4; j++) hc->coef[4 * q + j] = coef[8 * order[q] + j];
  });
  hc->flags.swap(flags);
  hc->nx = nx;
  hc->ny = ny;
  hc->pitch = pitch;
  hc->plane = plane;
  hc->px = px;
  hc->py = py;
  hc->ax = dom->ax;
  hc->ay = dom->ay;
  // only FP16 storage is scaled (BF16 keeps FP32's exponent range; its
  // kernels assume scale 1)
  hc->scale = p.precision == LBM_FP16 ? (p.storage_scale > 0.0 ? p.storage_scale : 4096.0) : 1.0;
  hc->cp = cp;
  hc->params = p;
  hc->n_fluid = n_fluid;
  hc->n_links = static_cast<int64_t>(n_links);
  return LBM_OK;

}

}  // namespace lbm

namespace lbm {

std::string build_compact(const HostCase &hc, CompactCase *cc) {
  const int32_t nx = hc.nx, ny = hc.ny, pitch = hc.pitch;
  const int64_t nn = static_cast<int64_t>(nx) * ny;
  auto fluid = [&](int32_t x, int32_t y) {
    return hc.flags[static_cast<size_t>(y) * pitch + x] != kSolid;
  };
  cc->rowstart.assign(static_cast<size_t>(ny) + 1, 0);
  parallel_for(ny, [&](int64_t y0, int64_t y1) {
    for (int64_t y = y0; y < y1; y++) {
      int32_t c = 0;
      for (int32_t x = 0; x < nx; x++) c += fluid(x, static_cast<int32_t>(y));
      cc->rowstart[y + 1] = c;
    }
  }, 64);
  for (int32_t y = 0; y < ny; y++) cc->rowstart[y + 1] += cc->rowstart[y];
  const int32_t n = cc->rowstart[ny];
  cc->n_fluid = n;
  cc->plane = (std::max<int64_t>(n, 1) + 31) / 32 * 32;
  const size_t P = static_cast<size_t>(cc->plane);
  cc->index.resize(static_cast<size_t>(nn));
  cc->lbase.assign(P, 0);
  cc->node.assign(P, uint2{0u, 0u});
  parallel_for(ny, [&](int64_t y0, int64_t y1) {
    // ahead_n[x] / ahead_s[x]: fluid nodes of the row above / below before
    // column x, so that (x, y +- 1), or the next fluid node after it, has
    // the compacted index rowstart[y +- 1] + ahead
    std::vector<int32_t> ahead_n(nx), ahead_s(nx);
    for (int64_t yy = y0; yy < y1; yy++) {
      const int32_t y = static_cast<int32_t>(yy);
      const int32_t yn = row_above(y, ny, hc.py);
      const int32_t ys = row_below(y, ny, hc.py);
      int32_t cn = 0, cs = 0;
      for (int32_t x = 0; x < nx; x++) {
        ahead_n[x] = cn;
        ahead_s[x] = cs;
        cn += fluid(x, yn);
        cs += fluid(x, ys);
      }
      int32_t i = cc->rowstart[y];
      for (int32_t x = 0; x < nx; x++) {
        if (!fluid(x, y)) {
          cc->index[static_cast<size_t>(y) * nx + x] = -1;
          continue;
        }
        cc->index[static_cast<size_t>(y) * nx + x] = i;
        uint32_t m = hc.flags[static_cast<size_t>(y) * pitch + x];
        if (hc.px && x == nx - 1) m |= kMetaWrapE;
        if (hc.px && x == 0) m |= kMetaWrapW;
        // n_lb - i and i - s_lb (see neighbour_rows): at most nx <= 65535
        const int64_t nl = cc->rowstart[yn] + ahead_n[x], sl = cc->rowstart[ys] + ahead_s[x];
        const int64_t dn = nl - i + ((hc.py && y == ny - 1) ? n : 0);
        const int64_t ds = i - sl + ((hc.py && y == 0) ? n : 0);
        cc->node[i].x = m | (static_cast<uint32_t>(dn) << 16);
        cc->node[i].y = static_cast<uint32_t>(ds);
        const int32_t lb = hc.lbase[static_cast<size_t>(y) * pitch + x];
        cc->lbase[i] = lb < 0 ? 0 : lb;
        i++;
      }
    }
  }, 64);
  // Group records and the node words' row and link offsets.  Links are
  // sorted by node, so a group's links follow its first node with links.
  const int64_t n_groups = (static_cast<int64_t>(n) + kGroup - 1) / kGroup;
  cc->grp.assign(static_cast<size_t>(n_groups), int2{0, 0});
  std::vector<char> group_bad(static_cast<size_t>(n_groups), 0);
  parallel_for(n_groups, [&](int64_t g0, int64_t g1) {
    for (int64_t g = g0; g < g1; g++) {
      const int32_t i0 = static_cast<int32_t>(g * kGroup);
      const int32_t i1 = std::min<int32_t>(n, i0 + kGroup);
      int32_t y = static_cast<int32_t>(
          std::upper_bound(cc->rowstart.begin(), cc->rowstart.end(), i0) - cc->rowstart.begin() - 1);
      const int32_t y0 = y;
      int32_t l0 = -1;
      for (int32_t i = i0; i < i1; i++)
        if (cc->node[i].x & 0xFFu) {
          l0 = cc->lbase[i];
          break;
        }
      cc->grp[g] = int2{y0, l0 < 0 ? 0 : l0};
      for (int32_t i = i0; i < i1; i++) {
        while (cc->rowstart[y + 1] <= i) y++;
        const uint32_t dy = static_cast<uint32_t>(y - y0);
        const int32_t loff = (cc->node[i].x & 0xFFu) ? cc->lbase[i] - l0 : 0;
        if (dy >= static_cast<uint32_t>(kMaxGroupRows) || loff < 0 || loff > 255) {
          group_bad[g] = 1;
          continue;
        }
        cc->node[i].x |= (dy & 63u) << 10;
        cc->node[i].y |= (static_cast<uint32_t>(loff) << 16) | ((dy >> 6) << 24);
      }
    }
  }, 1024);
  for (char b : group_bad)
    if (b)
      return "more than 16383 solid rows between two fluid nodes " + std::to_string(kGroup) +
             " places apart in row-major order";
  return std::string();
}

std::vector<uint32_t> link_jb_slots(const CompactCase &cc, int ny, int periodic_y,
                                    int64_t n_links) {
  std::vector<uint32_t> out(static_cast<size_t>(n_links), 0u);
  const uint32_t P = static_cast<uint32_t>(cc.plane);
  static const int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  parallel_for(cc.n_fluid, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; i++) {
      const uint2 nw = cc.node[static_cast<size_t>(i)];
      const uint32_t fl = nw.x & 0xFFu;
      if (!fl) continue;
      uint32_t s[9];
      pull_slots(nw, cc.grp[static_cast<size_t>(i / kGroup)], static_cast<uint32_t>(i), P,
                 static_cast<uint32_t>(cc.n_fluid), ny, periodic_y, cc.rowstart.data(), s);
      int64_t l = cc.lbase[static_cast<size_t>(i)];
      for (int j = 1; j < 9; j++)
        if (fl & (1u << (j - 1))) out[static_cast<size_t>(l++)] = s[opp[j]];
    }
  });
  return out;
}

std::vector<uint16_t> link_descriptors(const CompactCase &cc, int64_t n_links) {
  std::vector<uint16_t> out(static_cast<size_t>(n_links), 0u);
  parallel_for(cc.n_fluid, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; i++) {
      const uint32_t fl = cc.node[static_cast<size_t>(i)].x & 0xFFu;
      int64_t l = cc.lbase[static_cast<size_t>(i)];
      for (int j = 1; j < 9; j++)
        if (fl & (1u << (j - 1)))
          out[static_cast<size_t>(l++)] = static_cast<uint16_t>(((i & 63) << 4) | j);
    }
  });
  return out;
}

// Error text for handle-less calls, read back by lbm_last_error(NULL).
const char *set_thread_error(const std::string &msg) {
  g_create_error = msg;
  return g_create_error.c_str();
}
}  // namespace lbm

extern "C" {

void lbm_params_default(lbm_params_t *p) {
  if (!p) return;
  const double nan = std::numeric_limits<double>::quiet_NaN();
  std::memset(p, 0, sizeof(*p));
  p->sigma = 1.0;
  p->L1 = nan;
  p->L2 = nan;
  p->E = nan;
  p->l_clamp = -0.4;
  p->tau_rho = 1.0;
  p->tau_j = 1.0;
  p->tau_e = 1.1;
  p->tau_eps = 1.2;
  p->tau_s = nan;
  p->tau_q = nan;
  p->r_value = nan;
  p->l_value = 0.0;
  p->l_mode = LBM_L_PAPER;
  p->diffuse_mode = 0;
  p->precision = LBM_FP32;
  p->residual_every = 100;
  p->stream = nullptr;
  p->mass_mode = 0;
  p->residual_mode = 0;
}

int lbm_create(const lbm_domain_t *dom, const uint8_t *solid, size_t n_links,
               const int32_t *link_x, const int32_t *link_y, const int32_t *link_dir,
               const double *link_q, const double *link_ubx, const double *link_uby, double Kn,
               const lbm_params_t *params, lbm_handle_t **out) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "null argument";
    return LBM_EINVAL;
  }
  *out = nullptr;
  lbm::HostCase hc;
  int rc = lbm::build_host_case(dom, solid, n_links, link_x, link_y, link_dir, link_q, link_ubx,
                                link_uby, Kn, params, &hc, &g_create_error);
  if (rc != LBM_OK) return rc;
  lbm_handle_t *h = new (std::nothrow) lbm_handle_t();
  if (!h) {
    g_create_error = "host allocation failed";
    return LBM_ENOMEM;
  }
  const lbm_params_t &p = *params;
  {
    Fnv64 f;
    f.value(dom->nx);
    f.value(dom->ny);
    f.value(dom->periodic_x);
    f.value(dom->periodic_y);
    f.value(dom->H);
    f.value(dom->ax);
    f.value(dom->ay);
    f.value(Kn);
    f.big(solid, static_cast<size_t>(dom->nx) * static_cast<size_t>(dom->ny));
    f.value(n_links);
    f.big(link_x, n_links * sizeof(int32_t));
    f.big(link_y, n_links * sizeof(int32_t));
    f.big(link_dir, n_links * sizeof(int32_t));
    f.big(link_q, n_links * sizeof(double));
    f.big(link_ubx, n_links * sizeof(double));
    f.big(link_uby, n_links * sizeof(double));
    f.value(p.precision);
    // the per-link coefficients carry every parameter that shapes the scheme
    f.big(hc.coef.data(), hc.coef.size() * sizeof(double));
    f.value(hc.cp.tau_s);
    f.value(hc.cp.tau_q);
    f.value(hc.cp.tau_e);
    f.value(hc.cp.tau_eps);
    f.value(hc.scale);
    f.value(p.diffuse_mode);
    h->fingerprint = f.h;
  }
  h->link_r.swap(hc.link_r);
  h->link_l.swap(hc.link_l);
  const size_t n_links_sz = static_cast<size_t>(hc.n_links);
  h->precision = p.precision;
  h->scale = hc.scale;
  h->stream = static_cast<cudaStream_t>(p.stream);
  lbm::CompactCase cc;
  const std::string cerr = lbm::build_compact(hc, &cc);
  // pull slots are 32-bit: nine planes and the link tail below 2^32
  if (cerr.empty() && 9 * cc.plane + hc.n_links >= (int64_t(1) << 32)) {
    delete h;
    g_create_error = "lattice too large: 9 x fluid nodes + links must stay below 2^32";
    return LBM_EINVAL;
  }
  if (!cerr.empty()) {
    delete h;
    g_create_error = cerr;
    return LBM_EINVAL;
  }
  h->nx = hc.nx;
  h->ny = hc.ny;
  h->pitch = 0;
  h->plane = cc.plane;
  h->px = hc.px;
  h->py = hc.py;
  h->ax = hc.ax;
  h->ay = hc.ay;
  h->cp = hc.cp;
  h->params = p;
  h->n_fluid = hc.n_fluid;
  h->n_links = hc.n_links;
  cudaGetDevice(&h->device);
  // half the step kernel's resident CTAs (see lbm::step_kernel_pull)
  int resident = 0;
  switch (p.precision) {
    case LBM_FP64: resident = lbm::pull_resident_ctas<double, double>(); break;
    case LBM_FP32: resident = lbm::pull_resident_ctas<float, float>(); break;
    case LBM_BF16: resident = lbm::pull_resident_ctas<__nv_bfloat16, float>(); break;
    default: resident = lbm::pull_resident_ctas<__half, float>(); break;
  }
  h->pf_dist = static_cast<uint32_t>(resident / 2);

  const size_t es = elem_size(p.precision);
  // nine planes, then the link tail (rounded up to whole 128-byte lines)
  const size_t fbytes = (9 * static_cast<size_t>(cc.plane) + (n_links_sz + 63) / 64 * 64) * es;
  const size_t ces = p.precision == LBM_FP64 ? 8 : 4;  // link coefficients: FP64 or FP32
  const size_t lbytes = std::max<size_t>(1, n_links_sz) * 4 * ces;
  const size_t pbytes = lbm::kResidualBlocks * lbm::kPartialStride * sizeof(double);
  std::vector<unsigned char> lhost(lbytes, 0);
  for (size_t s = 0; s < n_links_sz; s++) {
    const double *c = &hc.coef[4 * s];
    if (ces == 8) {
      std::memcpy(&lhost[s * 32], c, 32);
    } else {
      float cf[4];
      for (int j = 0; j < 4; j++) cf[j] = static_cast<float>(c[j]);
      std::memcpy(&lhost[s * 16], cf, 16);
    }
  }
  auto alloc = [&](void **ptr, size_t bytes) {
    cudaError_t e = cudaMallocAsync(ptr, bytes, h->stream);
    if (e == cudaSuccess) h->dev_bytes += static_cast<int64_t>(bytes);
    return e;
  };
  cudaError_t e = cudaSuccess;
  h->fbytes = fbytes;
  if (e == cudaSuccess) e = alloc(&h->f[0], fbytes);
  if (e == cudaSuccess) e = alloc(&h->f[1], fbytes);
  const size_t P = static_cast<size_t>(cc.plane);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->node), P * sizeof(uint2));
  if (e == cudaSuccess)
    e = alloc(reinterpret_cast<void **>(&h->grp), std::max<size_t>(1, cc.grp.size()) * sizeof(int2));
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->rowstart), cc.rowstart.size() * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->index), cc.index.size() * 4);
  const std::vector<uint32_t> jbs = lbm::link_jb_slots(cc, hc.ny, hc.py, hc.n_links);
  if (e == cudaSuccess)
    e = alloc(reinterpret_cast<void **>(&h->jbslot), std::max<size_t>(1, jbs.size()) * 4);
  const std::vector<uint16_t> lds = lbm::link_descriptors(cc, hc.n_links);
  if (e == cudaSuccess)
    e = alloc(reinterpret_cast<void **>(&h->ldesc), std::max<size_t>(1, lds.size()) * 2);
  if (e == cudaSuccess) e = alloc(&h->links, lbytes);
  h->exact = lbm::exact_mass(hc) ? 1 : 0;
  // the exact-mass variant's link coefficients as FP32 pairs (alive until
  // the stream synchronises below)
  std::vector<lbm::LinkCoefDF> ldf;
  if (h->exact) {
    ldf.resize(n_links_sz);
    for (size_t l = 0; l < n_links_sz; l++) ldf[l] = lbm::link_coef_df(&hc.coef[4 * l]);
  }
  if (h->exact) {
    // one allocation: the per-link carries, then the per-node ones
    const size_t nl = std::max<size_t>(1, n_links_sz);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->links64), nl * 32);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->carry), carry_bytes(h));
    if (e == cudaSuccess) h->carry0 = h->carry + nl;
    if (e == cudaSuccess && n_links_sz)
      e = cudaMemcpyAsync(h->links64, ldf.data(), n_links_sz * sizeof(lbm::LinkCoefDF),
                          cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = clear_carry(h);
  }
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->partials), pbytes);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->result), 4 * sizeof(double));
  if (e == cudaSuccess && p.residual_mode == 1)
    e = alloc(&h->snap, std::max<size_t>(1, static_cast<size_t>(hc.n_fluid)) * 2 *
                            (p.precision == LBM_FP64 ? sizeof(double) : sizeof(float)));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&h->h_result), 4 * sizeof(double));

  if (e == cudaSuccess) e = cudaMemsetAsync(h->f[0], 0, fbytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->f[1], 0, fbytes, h->stream);
  auto up = [&](void *dst, const void *src, size_t bytes) {
    if (e == cudaSuccess && bytes)
      e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream);
  };
  up(h->node, cc.node.data(), P * sizeof(uint2));
  up(h->grp, cc.grp.data(), cc.grp.size() * sizeof(int2));
  up(h->jbslot, jbs.data(), jbs.size() * 4);
  up(h->ldesc, lds.data(), lds.size() * 2);
  up(h->rowstart, cc.rowstart.data(), cc.rowstart.size() * 4);
  up(h->index, cc.index.data(), cc.index.size() * 4);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->links, lhost.data(), lbytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = reset_interval(h);  // the rest state starts the first interval
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    g_create_error = std::string("device setup: ") + cudaGetErrorString(e);
    const int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    release(h);
    return code;
  }
  *out = h;
  return LBM_OK;
}

int lbm_step(lbm_handle_t *h, int64_t n) {
  if (!h) return LBM_EINVAL;
  if (n < 0) return fail(h, LBM_EINVAL, "negative step count");
  for (int64_t s = 0; s < n; s++) {
    cudaError_t e = do_step(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
  }
  return LBM_OK;
}

int lbm_residual(lbm_handle_t *h, double *residual, double *mass) {
  if (!h) return LBM_EINVAL;
  const int c = h->cur, pv = 1 - h->cur;
  int64_t span = 1;
  cudaError_t e;
  if (h->snap) {
    span = h->steps - h->snap_steps;
    e = interval_residual_launch(h);
    h->snap_steps = h->steps;
  } else {
    e = dispatch(h->precision, [&](auto tT, auto tC) {
      LBM_TYPES(tT, tC);
      return lbm::launch_residual_compact<T>(static_cast<const T *>(h->f[c]),
                                             static_cast<const T *>(h->f[pv]), node_map(h),
                                             h->n_fluid, h->plane, h->ax, h->ay, h->scale,
                                             h->partials, h->result, h->stream);
    });
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "residual kernel launch");
  LBM_CK(h, cudaMemcpyAsync(h->h_result, h->result, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  LBM_CK(h, cudaStreamSynchronize(h->stream));
  const double num = h->h_result[0], den = h->h_result[1];
  double res;
  if (std::isnan(num) || std::isnan(den))
    res = std::numeric_limits<double>::quiet_NaN();
  else if (span <= 0)
    res = 0.0;  // no step since the interval began
  else
    res = (den > 0.0 ? std::sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0)) /
          static_cast<double>(span);
  if (residual) *residual = res;
  if (mass) *mass = static_cast<double>(h->n_fluid) + h->h_result[2];
  if (h->h_result[3] > 0.0) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "%.0f fluid nodes with non-finite density or velocity",
                  h->h_result[3]);
    return fail(h, LBM_EUNSTABLE, buf);
  }
  return LBM_OK;
}

int lbm_run_to(lbm_handle_t *h, double tol, int64_t max_steps, int64_t *steps_done,
               double *residual) {
  if (!h) return LBM_EINVAL;
  if (max_steps < 0) return fail(h, LBM_EINVAL, "negative max_steps");
  int64_t done = 0;
  double res = INFINITY;
  while (done < max_steps) {
    const int64_t n = std::min<int64_t>(h->params.residual_every, max_steps - done);
    int rc = lbm_step(h, n);
    if (rc) return rc;
    done += n;
    rc = lbm_residual(h, &res, nullptr);
    if (rc) {
      if (steps_done) *steps_done = done;
      if (residual) *residual = res;
      return rc;
    }
    if (res < tol) break;
  }
  if (steps_done) *steps_done = done;
  if (residual) *residual = res;
  return LBM_OK;
}

int lbm_fields(lbm_handle_t *h, double *rho, double *ux, double *uy, int on_device) {
  if (!h) return LBM_EINVAL;
  const int64_t n = static_cast<int64_t>(h->nx) * h->ny;
  double *d = nullptr;
  double *r = rho, *u = ux, *v = uy;
  if (!on_device) {
    LBM_CK(h, cudaMallocAsync(reinterpret_cast<void **>(&d), 3 * n * sizeof(double), h->stream));
    r = rho ? d : nullptr;
    u = ux ? d + n : nullptr;
    v = uy ? d + 2 * n : nullptr;
  }
  cudaError_t e = dispatch(h->precision, [&](auto tT, auto tC) {
    LBM_TYPES(tT, tC);
    return lbm::launch_fields<T>(static_cast<const T *>(h->f[h->cur]), node_map(h), h->plane, h->ax,
                                 h->ay, h->scale, r, u, v, h->stream);
  });
  if (e == cudaSuccess && !on_device) {
    if (rho && e == cudaSuccess)
      e = cudaMemcpyAsync(rho, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (ux && e == cudaSuccess)
      e = cudaMemcpyAsync(ux, d + n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (uy && e == cudaSuccess)
      e = cudaMemcpyAsync(uy, d + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "lbm_fields");
  return LBM_OK;
}

int lbm_get_f(lbm_handle_t *h, double *f) {
  if (!h || !f) return h ? fail(h, LBM_EINVAL, "null output") : LBM_EINVAL;
  const int64_t n = 9 * static_cast<int64_t>(h->nx) * h->ny;
  double *d = nullptr;
  LBM_CK(h, cudaMallocAsync(reinterpret_cast<void **>(&d), n * sizeof(double), h->stream));
  cudaError_t e = dispatch(h->precision, [&](auto tT, auto tC) {
    LBM_TYPES(tT, tC);
    return lbm::launch_export_f<T>(static_cast<const T *>(h->f[h->cur]), node_map(h), h->plane,
                                   h->scale, d, h->stream);
  });
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaFreeAsync(d, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "lbm_get_f");
  return LBM_OK;
}

int lbm_set_f(lbm_handle_t *h, const double *f) {
  if (!h || !f) return h ? fail(h, LBM_EINVAL, "null input") : LBM_EINVAL;
  const int64_t n = 9 * static_cast<int64_t>(h->nx) * h->ny;
  double *d = nullptr;
  LBM_CK(h, cudaMallocAsync(reinterpret_cast<void **>(&d), n * sizeof(double), h->stream));
  cudaError_t e = cudaMemcpyAsync(d, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  for (int b = 0; b < 2 && e == cudaSuccess; b++)
    e = dispatch(h->precision, [&](auto tT, auto tC) {
      LBM_TYPES(tT, tC);
      return lbm::launch_import_f<T>(d, node_map(h), h->plane, h->scale, static_cast<T *>(h->f[b]),
                                     h->stream);
    });
  cudaFreeAsync(d, h->stream);
  if (e == cudaSuccess) e = clear_carry(h);
  h->steps = 0;
  if (e == cudaSuccess) e = reset_interval(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "lbm_set_f");
  return LBM_OK;
}

int lbm_set_fields(lbm_handle_t *h, const double *rho, const double *ux, const double *uy,
                   int on_device) {
  if (!h || !rho || !ux || !uy) return h ? fail(h, LBM_EINVAL, "null field") : LBM_EINVAL;
  const int64_t n = static_cast<int64_t>(h->nx) * h->ny;
  double *d = nullptr;
  const double *r = rho, *u = ux, *v = uy;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    LBM_CK(h, cudaMallocAsync(reinterpret_cast<void **>(&d), 3 * n * sizeof(double), h->stream));
    e = cudaMemcpyAsync(d, rho, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + n, ux, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 2 * n, uy, n * 8, cudaMemcpyHostToDevice, h->stream);
    r = d;
    u = d + n;
    v = d + 2 * n;
  }
  if (e == cudaSuccess)
    e = dispatch(h->precision, [&](auto tT, auto tC) {
      LBM_TYPES(tT, tC);
      return lbm::launch_set_fields<T>(r, u, v, node_map(h), h->plane, h->px, h->py, h->ax, h->ay,
                                       h->cp.tau_s, h->scale,
                                       static_cast<T *>(h->f[0]), static_cast<T *>(h->f[1]),
                                       h->stream);
    });
  if (d) cudaFreeAsync(d, h->stream);
  if (e == cudaSuccess) e = clear_carry(h);
  h->steps = 0;
  if (e == cudaSuccess) e = reset_interval(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "lbm_set_fields");
  return LBM_OK;
}

int lbm_link_params(const lbm_handle_t *h, double *r, double *l) {
  if (!h) return LBM_EINVAL;
  if (r) std::copy(h->link_r.begin(), h->link_r.end(), r);
  if (l) std::copy(h->link_l.begin(), h->link_l.end(), l);
  return LBM_OK;
}

int lbm_get_info(const lbm_handle_t *h, lbm_info_t *info) {
  if (!h || !info) return LBM_EINVAL;
  info->n_nodes = static_cast<int64_t>(h->nx) * h->ny;
  info->n_fluid = h->n_fluid;
  info->n_links = h->n_links;
  info->steps = h->steps;
  info->tau_s = h->cp.tau_s;
  info->tau_q = h->cp.tau_q;
  info->E = h->cp.E;
  info->E_max = h->cp.E_max;
  info->L1 = h->cp.L1;
  info->L2 = h->cp.L2;
  info->n_clamped = h->cp.n_clamped;
  info->device_bytes = h->dev_bytes;
  info->precision = h->precision;
  info->pitch = h->pitch;
  info->exact_mass = h->exact;
  return LBM_OK;
}

int lbm_precompute(double Kn, double H, const lbm_params_t *params, size_t n, const int32_t *dir,
                   const double *q, const double *ubx, const double *uby, double *r, double *l,
                   lbm_info_t *info) {
  g_create_error.clear();
  if (!params || (n && (!dir || !q || !ubx || !uby))) {
    g_create_error = "null argument";
    return LBM_EINVAL;
  }
  for (size_t k = 0; k < n; k++)
    if (dir[k] < 1 || dir[k] > 8 || !(q[k] > 0.0 && q[k] <= 1.0)) {
      g_create_error = "direction outside 1..8 or gamma outside (0, 1]";
      return LBM_EINVAL;
    }
  lbm::CaseParams cp;
  std::string msg = lbm::compute_case_params(Kn, H, *params, &cp);
  std::vector<double> rr(n), ll(n), coef(8 * n);
  if (msg.empty())
    msg = lbm::compute_link_coefs(cp, *params, n, dir, q, ubx, uby, rr.data(), ll.data(),
                                  coef.data(), &cp.n_clamped);
  if (!msg.empty()) {
    g_create_error = msg;
    return LBM_EINVAL;
  }
  if (r) std::copy(rr.begin(), rr.end(), r);
  if (l) std::copy(ll.begin(), ll.end(), l);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->n_links = static_cast<int64_t>(n);
    info->tau_s = cp.tau_s;
    info->tau_q = cp.tau_q;
    info->E = cp.E;
    info->E_max = cp.E_max;
    info->L1 = cp.L1;
    info->L2 = cp.L2;
    info->n_clamped = cp.n_clamped;
    info->precision = params->precision;
  }
  return LBM_OK;
}

namespace {
struct CheckpointHeader {
  char magic[8];
  int32_t version, precision, nx, ny;
  int64_t n_fluid, n_links, elems, steps;
  uint64_t fingerprint;
};
static_assert(sizeof(CheckpointHeader) == 64, "64-byte header");
constexpr char kCheckpointMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', '1'};

CheckpointHeader checkpoint_header(const lbm_handle_t *h) {
  CheckpointHeader hd{};
  std::memcpy(hd.magic, kCheckpointMagic, 8);
  hd.version = 2;
  hd.precision = h->precision;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.n_fluid = h->n_fluid;
  hd.n_links = h->n_links;
  hd.elems = static_cast<int64_t>(h->fbytes / elem_size(h->precision));
  hd.steps = h->steps;
  hd.fingerprint = h->fingerprint;
  return hd;
}
}  // namespace

int lbm_save(lbm_handle_t *h, const char *path) {
  if (!h) return LBM_EINVAL;
  if (!path) return fail(h, LBM_EINVAL, "null path");
  std::vector<unsigned char> buf;
  const size_t cbytes = carry_bytes(h);
  try {
    buf.resize(2 * h->fbytes + cbytes);
  } catch (...) {
    return fail(h, LBM_ENOMEM, "host buffer for the checkpoint");
  }
  LBM_CK(h, cudaMemcpyAsync(buf.data(), h->f[h->cur], h->fbytes, cudaMemcpyDeviceToHost, h->stream));
  LBM_CK(h, cudaMemcpyAsync(buf.data() + h->fbytes, h->f[1 - h->cur], h->fbytes,
                            cudaMemcpyDeviceToHost, h->stream));
  if (cbytes)
    LBM_CK(h, cudaMemcpyAsync(buf.data() + 2 * h->fbytes, h->carry, cbytes, cudaMemcpyDeviceToHost,
                              h->stream));
  LBM_CK(h, cudaStreamSynchronize(h->stream));
  const CheckpointHeader hd = checkpoint_header(h);
  FILE *f = std::fopen(path, "wb");
  if (!f) return fail(h, LBM_EIO, std::string("cannot open ") + path + " for writing");
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                  std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) return fail(h, LBM_EIO, std::string("cannot write ") + path);
  return LBM_OK;
}

int lbm_load(lbm_handle_t *h, const char *path) {
  if (!h) return LBM_EINVAL;
  if (!path) return fail(h, LBM_EINVAL, "null path");
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(h, LBM_EIO, std::string("cannot open ") + path);
  CheckpointHeader hd{};
  if (std::fread(&hd, sizeof(hd), 1, f) != 1) {
    std::fclose(f);
    return fail(h, LBM_EIO, std::string("cannot read the header of ") + path);
  }
  const CheckpointHeader want = checkpoint_header(h);
  std::string why;
  if (std::memcmp(hd.magic, kCheckpointMagic, 8) != 0) why = "not a checkpoint file";
  else if (hd.version != 2) why = "unknown checkpoint version";
  else if (hd.precision != want.precision) why = "checkpoint of another precision";
  else if (hd.nx != want.nx || hd.ny != want.ny || hd.n_fluid != want.n_fluid ||
           hd.n_links != want.n_links || hd.elems != want.elems ||
           hd.fingerprint != want.fingerprint)
    why = "checkpoint of another case";
  else if (hd.steps < 0) why = "negative step count";
  if (!why.empty()) {
    std::fclose(f);
    return fail(h, LBM_EINVAL, why + ": " + path);
  }
  std::vector<unsigned char> buf;
  const size_t cbytes = carry_bytes(h);
  try {
    buf.resize(2 * h->fbytes + cbytes);
  } catch (...) {
    std::fclose(f);
    return fail(h, LBM_ENOMEM, "host buffer for the checkpoint");
  }
  const bool ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return fail(h, LBM_EIO, std::string("checkpoint file too short: ") + path);
  LBM_CK(h, cudaMemcpyAsync(h->f[h->cur], buf.data(), h->fbytes, cudaMemcpyHostToDevice, h->stream));
  LBM_CK(h, cudaMemcpyAsync(h->f[1 - h->cur], buf.data() + h->fbytes, h->fbytes,
                            cudaMemcpyHostToDevice, h->stream));
  if (cbytes)
    LBM_CK(h, cudaMemcpyAsync(h->carry, buf.data() + 2 * h->fbytes, cbytes, cudaMemcpyHostToDevice,
                              h->stream));
  h->steps = hd.steps;
  LBM_CK(h, reset_interval(h));
  LBM_CK(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

void lbm_destroy(lbm_handle_t *h) { release(h); }

const char *lbm_last_error(const lbm_handle_t *h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
