// Three-dimensional solver of liblbm.so (lbm3d_*): the D3Q19 lattice with
// the same multiple-relaxation-time collision, Guo forcing and curved slip
// boundary scheme (Eq. EqNewBDSC) per link as the two-dimensional solver --
// the extension the paper names as future work (Sec. 5).
//
// The paper's parameters (Sec. 3.B: tau_s from Kn, per-link l and r, the
// uniform tau_q) come from a two-dimensional analysis.  Carried out for
// D3Q19 (a flow u_x(z) between walls normal to z), that analysis involves
// the x-odd moments j_x, q_x, p_xz and the third-order m_x, and reaches
// exactly the wall relation of Eq. u1u0Coeff when m relaxes with tau_q; so
// m takes tau_q here, and the two-dimensional closed forms hold for the 3-D
// flat channel (tested against the oracle).
//
// Layout: a dense lattice (every node has slots; solid ones are never
// touched), populations stored as deviations d_q = f_q - w_q in FP64 or
// FP32, plane q of N elements (N = nodes rounded up to 32), then a link
// tail.  Pull scheme as in 2-D: step t stores f'_q(x, t) in x's own slot
// q N + x and step t+1 gathers f_q(x, t+1) = f'_q(x - c_q, t) from the slot
// of x - c_q, or, where x - c_q is solid (a boundary link), from the link's
// tail element 19 N + k, which Eq. EqNewBDSC (local to x) filled during
// step t.  Per node: a flag word (bit q: x - c_q solid; kSolid3 for solid
// nodes) and the index of its first link (links sorted by node, then
// direction).  The collision works in moment space with the D3Q19 basis
// built here from its defining polynomials (d'Humieres et al. 2002):
// m - m_eq = M (d - d_eq), M Fbar, then f' - f = M^T diag(1/|M_k|^2) (m' -
// m) (the basis is orthogonal), and the rest population closes the mass.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm3 {

constexpr int Q = 19;
constexpr uint32_t kSolid3 = 0xFFFFFFFFu;
constexpr int kThreads3 = 128;
constexpr int kResBlocks3 = 2048;
constexpr int kResThreads3 = 256;

// velocities: rest, the six axes (+x, -x, +y, -y, +z, -z), then the
// diagonals of the xy, xz and yz planes, each (+, +), (+, -), (-, +), (-, -)
struct Lattice {
  int c[Q][3];
  int opp[Q];
  double w[Q];
  double M[Q][Q];  // moment basis, rows = moments
  double norm[Q];  // |M_k|^2
  Lattice() {
    int k = 0;
    c[k][0] = c[k][1] = c[k][2] = 0;
    w[k++] = 1.0 / 3.0;
    for (int a = 0; a < 3; a++)
      for (int s = 1; s >= -1; s -= 2) {
        for (int b = 0; b < 3; b++) c[k][b] = b == a ? s : 0;
        w[k++] = 1.0 / 18.0;
      }
    const int pa[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (auto &pr : pa)
      for (int s1 = 1; s1 >= -1; s1 -= 2)
        for (int s2 = 1; s2 >= -1; s2 -= 2) {
          for (int b = 0; b < 3; b++) c[k][b] = 0;
          c[k][pr[0]] = s1;
          c[k][pr[1]] = s2;
          w[k++] = 1.0 / 36.0;
        }
    for (int i = 0; i < Q; i++)
      for (int j = 0; j < Q; j++)
        if (c[j][0] == -c[i][0] && c[j][1] == -c[i][1] && c[j][2] == -c[i][2]) opp[i] = j;
    for (int r = 0; r < Q; r++) {
      norm[r] = 0.0;
      for (int i = 0; i < Q; i++) {
        const double x = c[i][0], y = c[i][1], z = c[i][2], c2 = x * x + y * y + z * z;
        double v;
        switch (r) {
          case 0: v = 1.0; break;
          case 1: v = 19.0 * c2 - 30.0; break;
          case 2: v = (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0; break;
          case 3: v = x; break;
          case 4: v = (5.0 * c2 - 9.0) * x; break;
          case 5: v = y; break;
          case 6: v = (5.0 * c2 - 9.0) * y; break;
          case 7: v = z; break;
          case 8: v = (5.0 * c2 - 9.0) * z; break;
          case 9: v = 3.0 * x * x - c2; break;
          case 10: v = (3.0 * c2 - 5.0) * (3.0 * x * x - c2); break;
          case 11: v = y * y - z * z; break;
          case 12: v = (3.0 * c2 - 5.0) * (y * y - z * z); break;
          case 13: v = x * y; break;
          case 14: v = y * z; break;
          case 15: v = x * z; break;
          case 16: v = (y * y - z * z) * x; break;
          case 17: v = (z * z - x * x) * y; break;
          default: v = (x * x - y * y) * z; break;
        }
        M[r][i] = v;
        norm[r] += v * v;
      }
    }
  }
};

const Lattice &lattice() {
  static const Lattice L;
  return L;
}

// Kernel constants of one case (passed by value): the relaxation rates
// s_k and forcing weights 1 - s_k/2 of the 19 moments, each divided by
// |M_k|^2 (the scale of M^-1 = M^T diag(1/|M_k|^2)).  The lattice itself
// (velocities, weights, M) is the same for every case and sits in constant
// memory.
template <typename C>
struct Const3 {
  C s_scaled[Q], f_scaled[Q];
  C ax, ay, az;
  int32_t nx, ny, nz, px, py, pz;
  int32_t diffuse_mode;
  int64_t plane;  // N
};

// per link: k1, k2, k3, alpha of the folded form of Eq. EqNewBDSC (LinkCoef)
template <typename C>
struct Link3 {
  C k1, k2, k3, alpha;
};

// Slot of f_q(x, t) for node p (pull layout): the neighbour x - c_q's own
// slot, or the node's tail element when x - c_q is solid.  rank = links of
// the node in lower directions.
template <typename C>
__device__ __forceinline__ int64_t pull_slot3(const Const3<C> &k, const int cq[3], int x, int y,
                                              int z, uint32_t fl, int q, int64_t lbase,
                                              int64_t N) {
  if (fl & (1u << q)) return 19 * N + lbase + __popc(fl & ((1u << q) - 1u));
  int xs = x - cq[0], ys = y - cq[1], zs = z - cq[2];
  if (k.px) xs = (xs + k.nx) % k.nx;
  if (k.py) ys = (ys + k.ny) % k.ny;
  if (k.pz) zs = (zs + k.nz) % k.nz;
  return static_cast<int64_t>(q) * N + (static_cast<int64_t>(zs) * k.ny + ys) * k.nx + xs;
}

// the velocities and opposites in the order of Lattice, for device code
// (compile-time tables: unrolled loops index registers with them)
#define LBM3_CX {0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 0, 0, 0, 0}
#define LBM3_CY {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1}
#define LBM3_CZ {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1}
#define LBM3_OPP {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15}
__constant__ int c_c3[Q][3];
__constant__ double c_M3d[Q][Q];
__constant__ float c_M3f[Q][Q];
__constant__ double c_w3d[Q];
__constant__ float c_w3f[Q];

template <typename C>
__device__ __forceinline__ C mval(int r, int q) {
  if constexpr (std::is_same<C, double>::value) return c_M3d[r][q];
  else return c_M3f[r][q];
}
template <typename C>
__device__ __forceinline__ C wval(int q) {
  if constexpr (std::is_same<C, double>::value) return c_w3d[q];
  else return c_w3f[q];
}

template <typename C>
__global__ void __launch_bounds__(kThreads3)
step3_kernel(const C *__restrict__ src, C *__restrict__ dst, const uint32_t *__restrict__ flags,
             const int64_t *__restrict__ lbase, const Link3<C> *__restrict__ links,
             const Const3<C> k, int64_t n_nodes) {
  const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= n_nodes) return;
  const uint32_t fl = flags[p];
  if (fl == kSolid3) return;
  const int64_t N = k.plane;
  const int x = static_cast<int>(p % k.nx), y = static_cast<int>((p / k.nx) % k.ny),
            z = static_cast<int>(p / (static_cast<int64_t>(k.nx) * k.ny));
  constexpr int cx[Q] = LBM3_CX, cy[Q] = LBM3_CY, cz[Q] = LBM3_CZ, opp[Q] = LBM3_OPP;
  const int64_t lb = lbase[p];
  C d[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const int cq[3] = {cx[q], cy[q], cz[q]};
    d[q] = src[pull_slot3(k, cq, x, y, z, fl, q, lb, N)];
  }
  // Eq. FluidMacr
  C drho = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
  for (int q = 0; q < Q; q++) {
    drho += d[q];
    jx += C(cx[q]) * d[q];
    jy += C(cy[q]) * d[q];
    jz += C(cz[q]) * d[q];
  }
  const C rho = C(1) + drho;
  const C ux = (jx + C(0.5) * rho * k.ax) / rho, uy = (jy + C(0.5) * rho * k.ay) / rho,
          uz = (jz + C(0.5) * rho * k.az) / rho;
  const C uu = ux * ux + uy * uy + uz * uz, ua = ux * k.ax + uy * k.ay + uz * k.az;
  // d - d_eq and Fbar (Eq. LBEequi, Eq. LBEforce), then the moments
  C neq[Q], F[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const C cu = C(cx[q]) * ux + C(cy[q]) * uy + C(cz[q]) * uz;
    const C ca = C(cx[q]) * k.ax + C(cy[q]) * k.ay + C(cz[q]) * k.az;
    neq[q] = d[q] - wval<C>(q) * (drho + rho * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu));
    F[q] = wval<C>(q) * rho * (C(3) * ca + C(9) * (cu * ca - ua / C(3)));
  }
  // m' - m = -s (m - m_eq) + (1 - s/2) M Fbar, scaled by 1/|M_k|^2
  C dm[Q];
#pragma unroll
  for (int r = 0; r < Q; r++) {
    C a = C(0), b = C(0);
#pragma unroll
    for (int q = 0; q < Q; q++) {
      a += mval<C>(r, q) * neq[q];
      b += mval<C>(r, q) * F[q];
    }
    dm[r] = k.f_scaled[r] * b - k.s_scaled[r] * a;
  }
  // f' - f = M^T dm; f'_0 closes the mass from the stored changes
  C o[Q];
  C sum = C(0);
#pragma unroll
  for (int q = 1; q < Q; q++) {
    C ch = C(0);
#pragma unroll
    for (int r = 0; r < Q; r++) ch += mval<C>(r, q) * dm[r];
    o[q] = d[q] + ch;
    sum += o[q] - d[q];
  }
  o[0] = d[0] - sum;
#pragma unroll
  for (int q = 0; q < Q; q++) dst[q * N + p] = o[q];
  // Eq. EqNewBDSC for each unknown direction j of the node, to the tail
  if (fl) {
    int rank = 0;
#pragma unroll
    for (int j = 1; j < Q; j++) {
      if (!(fl & (1u << j))) continue;
      const Link3<C> c = links[lb + rank];
      const int jb = opp[j];
      const C r = c.k1 + c.k2 + c.k3;
      C c0, c2;
      if (k.diffuse_mode == 0) {
        c0 = c.alpha;
        c2 = (C(1) - r) * wval<C>(j);
      } else {
        c0 = c.alpha + (r - C(1)) * wval<C>(j);
        c2 = C(0);
      }
      const C cu = C(cx[j]) * ux + C(cy[j]) * uy + C(cz[j]) * uz;
      const C pj = C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu;
      dst[19 * N + lb + rank] = c.k1 * d[jb] + c.k2 * o[j] + c.k3 * o[jb] + c0 + c.alpha * drho +
                                c2 * (drho + rho * pj);
      rank++;
    }
  }
}

// Residual pass (FP64 sums, fixed grid and order): num, den, mass
// deviation, non-finite count of the states in cur and prev.
template <typename C>
__global__ void __launch_bounds__(kResThreads3)
residual3_kernel(const C *__restrict__ cur, const C *__restrict__ prev,
                 const uint32_t *__restrict__ flags, const int64_t *__restrict__ lbase,
                 const Const3<C> k, int64_t n_nodes, double *__restrict__ partials) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t G = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_nodes;
       p += G) {
    const uint32_t fl = flags[p];
    if (fl == kSolid3) continue;
    const int x = static_cast<int>(p % k.nx), y = static_cast<int>((p / k.nx) % k.ny),
              z = static_cast<int>(p / (static_cast<int64_t>(k.nx) * k.ny));
    double r1 = 1.0, r0 = 1.0, j1[3] = {0, 0, 0}, j0[3] = {0, 0, 0}, dm = 0.0;
    const int64_t lb = lbase[p];
    for (int q = 0; q < Q; q++) {
      const int64_t s = pull_slot3(k, c_c3[q], x, y, z, fl, q, lb, k.plane);
      const double a = static_cast<double>(cur[s]), b = static_cast<double>(prev[s]);
      r1 += a;
      r0 += b;
      dm += a;
      for (int e = 0; e < 3; e++) {
        j1[e] += c_c3[q][e] * a;
        j0[e] += c_c3[q][e] * b;
      }
    }
    const double acc3[3] = {static_cast<double>(k.ax), static_cast<double>(k.ay),
                            static_cast<double>(k.az)};
    double num = 0.0, den = 0.0;
    for (int e = 0; e < 3; e++) {
      const double u1 = (j1[e] + 0.5 * r1 * acc3[e]) / r1, u0 = (j0[e] + 0.5 * r0 * acc3[e]) / r0;
      num += (u1 - u0) * (u1 - u0);
      den += u1 * u1;
    }
    if (!(isfinite(num) && isfinite(den) && isfinite(dm))) {
      acc[3] += 1.0;
      continue;
    }
    acc[0] += num;
    acc[1] += den;
    acc[2] += dm;
  }
  __shared__ double sh[kResThreads3 / 32][4];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < 4; c++) {
    const double v = lbm::dev::warp_sum(acc[c]);
    if (lane == 0) sh[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int i = 0; i < kResThreads3 / 32; i++) t += sh[i][threadIdx.x];
    partials[blockIdx.x * 4 + threadIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) residual3_final(const double *partials, double *out) {
  __shared__ double sh[32][4];
  double v[4];
  for (int c = 0; c < 4; c++) {
    double t = 0.0;
    for (int b = threadIdx.x; b < kResBlocks3; b += 1024) t += partials[b * 4 + c];
    v[c] = lbm::dev::warp_sum(t);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int c = 0; c < 4; c++) sh[w][c] = v[c];
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int i = 0; i < 32; i++) s += sh[i][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// Conversions between the lattice and caller arrays of full populations
// f[19][nz][ny][nx] (export: solid nodes as the rest state w_q; import:
// solid entries ignored).
template <typename C>
__global__ void export3_kernel(const C *__restrict__ f, const uint32_t *__restrict__ flags,
                               const int64_t *__restrict__ lbase, const Const3<C> k,
                               int64_t n_nodes, double *out) {
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < Q * n_nodes;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(t / n_nodes);
    const int64_t p = t - static_cast<int64_t>(q) * n_nodes;
    const uint32_t fl = flags[p];
    double v = c_w3d[q];
    if (fl != kSolid3) {
      const int x = static_cast<int>(p % k.nx), y = static_cast<int>((p / k.nx) % k.ny),
                z = static_cast<int>(p / (static_cast<int64_t>(k.nx) * k.ny));
      v += static_cast<double>(f[pull_slot3(k, c_c3[q], x, y, z, fl, q, lbase[p], k.plane)]);
    }
    out[t] = v;
  }
}

// Eq. FluidMacr at every node (solid nodes 0): rho, ux, uy, uz arrays of
// nx*ny*nz doubles.
template <typename C>
__global__ void fields3_kernel(const C *__restrict__ f, const uint32_t *__restrict__ flags,
                               const int64_t *__restrict__ lbase, const Const3<C> k,
                               int64_t n_nodes, double *__restrict__ out) {
  constexpr int cx[Q] = LBM3_CX, cy[Q] = LBM3_CY, cz[Q] = LBM3_CZ;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_nodes;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t fl = flags[p];
    double r = 0.0, u[3] = {0.0, 0.0, 0.0};
    if (fl != kSolid3) {
      const int x = static_cast<int>(p % k.nx), y = static_cast<int>((p / k.nx) % k.ny),
                z = static_cast<int>(p / (static_cast<int64_t>(k.nx) * k.ny));
      double dr = 0.0, j[3] = {0.0, 0.0, 0.0};
      const int64_t lb = lbase[p];
#pragma unroll
      for (int q = 0; q < Q; q++) {
        const int cq[3] = {cx[q], cy[q], cz[q]};
        const double v = static_cast<double>(f[pull_slot3(k, cq, x, y, z, fl, q, lb, k.plane)]);
        dr += v;
        j[0] += cx[q] * v;
        j[1] += cy[q] * v;
        j[2] += cz[q] * v;
      }
      r = 1.0 + dr;
      const double a[3] = {static_cast<double>(k.ax), static_cast<double>(k.ay),
                           static_cast<double>(k.az)};
      for (int e = 0; e < 3; e++) u[e] = (j[e] + 0.5 * r * a[e]) / r;
    }
    out[p] = r;
    out[n_nodes + p] = u[0];
    out[2 * n_nodes + p] = u[1];
    out[3 * n_nodes + p] = u[2];
  }
}

template <typename C>
__global__ void import3_kernel(const double *__restrict__ in, const uint32_t *__restrict__ flags,
                               const int64_t *__restrict__ lbase, const Const3<C> k,
                               int64_t n_nodes, C *f) {
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < Q * n_nodes;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int q = static_cast<int>(t / n_nodes);
    const int64_t p = t - static_cast<int64_t>(q) * n_nodes;
    const uint32_t fl = flags[p];
    if (fl == kSolid3) continue;
    const int x = static_cast<int>(p % k.nx), y = static_cast<int>((p / k.nx) % k.ny),
              z = static_cast<int>(p / (static_cast<int64_t>(k.nx) * k.ny));
    f[pull_slot3(k, c_c3[q], x, y, z, fl, q, lbase[p], k.plane)] =
        static_cast<C>(in[t] - c_w3d[q]);
  }
}

// a case's constants in both arithmetic types (the one of its precision is set)
struct Const3Both {
  Const3<double> d;
  Const3<float> f;
  Const3<double> &get(double *) { return d; }
  Const3<float> &get(float *) { return f; }
  const Const3<double> &get(double *) const { return d; }
  const Const3<float> &get(float *) const { return f; }
};

int grid_for3(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return static_cast<int>(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace lbm3

using lbm3::Const3Both;
struct lbm3d {
  int precision = LBM_FP32;
  cudaStream_t stream = nullptr;
  int32_t nx = 0, ny = 0, nz = 0;
  int64_t n_nodes = 0, plane = 0, n_fluid = 0, n_links = 0, steps = 0;
  double ax = 0.0, ay = 0.0, az = 0.0;
  lbm::CaseParams cp{};
  void *f[2] = {nullptr, nullptr};
  int cur = 0;
  uint32_t *flags = nullptr;
  int64_t *lbase = nullptr;
  void *links = nullptr;
  Const3Both kc;
  double *partials = nullptr, *result = nullptr;
  std::vector<double> link_r, link_l;
  std::string err;
};

namespace {

thread_local std::string g_err3;

int fail3(lbm3d_t *h, int code, const std::string &m) {
  if (h) h->err = m;
  else g_err3 = m;
  return code;
}

void release3(lbm3d_t *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (void *p : {h->f[0], h->f[1], static_cast<void *>(h->flags), static_cast<void *>(h->lbase),
                  h->links, static_cast<void *>(h->partials),
                  static_cast<void *>(h->result)})
    if (p) cudaFree(p);
  delete h;
}

template <typename F>
cudaError_t dispatch3(int precision, F &&fn) {
  if (precision == LBM_FP64) return fn(static_cast<double *>(nullptr));
  return fn(static_cast<float *>(nullptr));
}

}  // namespace

extern "C" {

int lbm3d_create(const lbm3d_domain_t *dom, const uint8_t *solid, size_t n_links,
                 const int32_t *link_x, const int32_t *link_y, const int32_t *link_z,
                 const int32_t *link_dir, const double *link_q, const double *link_ub, double Kn,
                 const lbm_params_t *params, lbm3d_t **out) {
  using namespace lbm3;
  g_err3.clear();
  if (!out) return fail3(nullptr, LBM_EINVAL, "null output");
  *out = nullptr;
  if (!dom || !solid || !params) return fail3(nullptr, LBM_EINVAL, "null argument");
  if (n_links && (!link_x || !link_y || !link_z || !link_dir || !link_q || !link_ub))
    return fail3(nullptr, LBM_EINVAL, "null link array");
  const lbm_params_t &p = *params;
  if (p.precision != LBM_FP64 && p.precision != LBM_FP32)
    return fail3(nullptr, LBM_EINVAL, "the 3-D solver stores LBM_FP64 or LBM_FP32");
  if (p.diffuse_mode != 0 && p.diffuse_mode != 1)
    return fail3(nullptr, LBM_EINVAL, "diffuse_mode must be 0 or 1");
  if (p.collision != 0) return fail3(nullptr, LBM_EINVAL, "the 3-D solver is MRT only");
  const int32_t nx = dom->nx, ny = dom->ny, nz = dom->nz;
  if (nx < 1 || ny < 1 || nz < 1) return fail3(nullptr, LBM_EINVAL, "nx, ny, nz must be >= 1");
  const int64_t n = static_cast<int64_t>(nx) * ny * nz;
  if (n >= (int64_t(1) << 31)) return fail3(nullptr, LBM_EINVAL, "lattice too large");
  if (!std::isfinite(dom->ax) || !std::isfinite(dom->ay) || !std::isfinite(dom->az))
    return fail3(nullptr, LBM_EINVAL, "non-finite force");
  const int per[3] = {dom->periodic_x ? 1 : 0, dom->periodic_y ? 1 : 0, dom->periodic_z ? 1 : 0};
  const Lattice &L = lattice();
  auto node = [&](int64_t x, int64_t y, int64_t z) { return (z * ny + y) * nx + x; };
  // neighbour x + s c_q, or -1 outside a non-periodic axis
  auto nbr = [&](int x, int y, int z, int q, int s) -> int64_t {
    int a[3] = {x + s * L.c[q][0], y + s * L.c[q][1], z + s * L.c[q][2]};
    const int d[3] = {nx, ny, nz};
    for (int e = 0; e < 3; e++) {
      if (a[e] < 0 || a[e] >= d[e]) {
        if (!per[e]) return -1;
        a[e] = (a[e] + d[e]) % d[e];
      }
    }
    return node(a[0], a[1], a[2]);
  };
  // flags: unknown directions of fluid nodes
  std::vector<uint32_t> flags(static_cast<size_t>(n), kSolid3);
  int64_t n_fluid = 0;
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        const int64_t pn = node(x, y, z);
        if (solid[pn]) continue;
        n_fluid++;
        uint32_t fl = 0;
        for (int q = 1; q < Q; q++) {
          const int64_t r = nbr(x, y, z, q, -1);
          if (r < 0 || solid[r]) fl |= 1u << q;
        }
        flags[pn] = fl;
      }
  // links: validate, one per unknown (node, direction), sorted by node then direction
  std::vector<int64_t> lbase(static_cast<size_t>(n), 0);
  int64_t total = 0;
  for (int64_t pn = 0; pn < n; pn++) {
    lbase[pn] = total;
    if (flags[pn] != kSolid3) total += __builtin_popcount(flags[pn]);
  }
  if (static_cast<int64_t>(n_links) != total)
    return fail3(nullptr, LBM_EINVAL,
                 "links must cover every unknown (node, direction) once: " +
                     std::to_string(total) + " unknown, " + std::to_string(n_links) + " given");
  std::vector<int64_t> slot(n_links);
  std::vector<uint8_t> seen(static_cast<size_t>(total), 0);
  std::vector<double> cub(n_links), wq(n_links), uu(n_links);
  for (size_t k = 0; k < n_links; k++) {
    const int x = link_x[k], y = link_y[k], z = link_z[k], q = link_dir[k];
    if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz || q < 1 || q >= Q)
      return fail3(nullptr, LBM_EINVAL, "link " + std::to_string(k) + ": out of range");
    if (!(link_q[k] > 0.0 && link_q[k] <= 1.0))
      return fail3(nullptr, LBM_EINVAL, "link " + std::to_string(k) + ": gamma outside (0, 1]");
    const int64_t pn = node(x, y, z);
    const uint32_t fl = flags[pn];
    if (fl == kSolid3 || !(fl & (1u << q)))
      return fail3(nullptr, LBM_EINVAL,
                   "link " + std::to_string(k) + ": node must be fluid and x - c_i solid");
    const int64_t s = lbase[pn] + __builtin_popcount(fl & ((1u << q) - 1u));
    if (seen[s]) return fail3(nullptr, LBM_EINVAL, "link " + std::to_string(k) + ": duplicate");
    seen[s] = 1;
    slot[k] = s;
    const double *ub = link_ub + 3 * k;
    cub[k] = L.c[q][0] * ub[0] + L.c[q][1] * ub[1] + L.c[q][2] * ub[2];
    wq[k] = L.w[q];
    uu[k] = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
  }
  // Sec. 3.B parameters (the two-dimensional closed forms) and the folded
  // per-link coefficients
  lbm::CaseParams cp;
  std::string msg = lbm::compute_case_params(Kn, dom->H, p, &cp);
  if (!msg.empty()) return fail3(nullptr, LBM_EINVAL, msg);
  std::vector<double> r(n_links), l(n_links), coef(8 * n_links);
  msg = lbm::compute_link_coefs_general(cp, p, n_links, link_q, cub.data(), wq.data(), uu.data(),
                                        r.data(), l.data(), coef.data(), &cp.n_clamped);
  if (!msg.empty()) return fail3(nullptr, LBM_EINVAL, msg);

  lbm3d_t *h = new (std::nothrow) lbm3d_t();
  if (!h) return fail3(nullptr, LBM_ENOMEM, "host allocation failed");
  h->precision = p.precision;
  h->stream = static_cast<cudaStream_t>(p.stream);
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->n_nodes = n;
  h->plane = (n + 31) / 32 * 32;
  h->n_fluid = n_fluid;
  h->n_links = static_cast<int64_t>(n_links);
  h->ax = dom->ax;
  h->ay = dom->ay;
  h->az = dom->az;
  h->cp = cp;
  h->link_r = r;
  h->link_l = l;
  // relaxation times of the 19 moments: rho, e, eps, j_x, q_x, j_y, q_y,
  // j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z
  const double tau[Q] = {cp.tau_rho, cp.tau_e, cp.tau_eps, cp.tau_j, cp.tau_q, cp.tau_j,
                         cp.tau_q,   cp.tau_j, cp.tau_q,   cp.tau_s, cp.tau_eps, cp.tau_s,
                         cp.tau_eps, cp.tau_s, cp.tau_s,   cp.tau_s, cp.tau_q,   cp.tau_q,
                         cp.tau_q};
  cudaError_t e = cudaSuccess;
  int cc[Q][3];
  for (int q = 0; q < Q; q++)
    for (int a = 0; a < 3; a++) cc[q][a] = L.c[q][a];
  e = cudaMemcpyToSymbol(c_c3, cc, sizeof cc);
  {
    // the device's compile-time tables must be the lattice built here
    const int tx[Q] = LBM3_CX, ty[Q] = LBM3_CY, tz[Q] = LBM3_CZ, to[Q] = LBM3_OPP;
    for (int q = 0; q < Q; q++)
      if (tx[q] != L.c[q][0] || ty[q] != L.c[q][1] || tz[q] != L.c[q][2] || to[q] != L.opp[q])
        return fail3(nullptr, LBM_EINVAL, "internal: D3Q19 velocity tables disagree");
  }
  {
    float mf[Q][Q], wf[Q];
    for (int a = 0; a < Q; a++) {
      for (int b = 0; b < Q; b++) mf[a][b] = static_cast<float>(L.M[a][b]);
      wf[a] = static_cast<float>(L.w[a]);
    }
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_M3d, L.M, sizeof L.M);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w3d, L.w, sizeof L.w);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_M3f, mf, sizeof mf);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w3f, wf, sizeof wf);
  }
  const size_t es = p.precision == LBM_FP64 ? 8 : 4;
  const size_t fbytes = (19 * static_cast<size_t>(h->plane) + (n_links + 63) / 64 * 64) * es;
  auto alloc = [&](void **ptr, size_t bytes) {
    return cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  };
  if (e == cudaSuccess) e = alloc(&h->f[0], fbytes);
  if (e == cudaSuccess) e = alloc(&h->f[1], fbytes);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->flags), n * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->lbase), n * 8);
  if (e == cudaSuccess) e = alloc(&h->links, std::max<size_t>(1, n_links) * 4 * es);
  if (e == cudaSuccess)
    e = alloc(reinterpret_cast<void **>(&h->partials), kResBlocks3 * 4 * sizeof(double));
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->result), 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->f[0], 0, fbytes);
  if (e == cudaSuccess) e = cudaMemset(h->f[1], 0, fbytes);
  if (e == cudaSuccess) e = cudaMemcpy(h->flags, flags.data(), n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->lbase, lbase.data(), n * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = dispatch3(h->precision, [&](auto tag) {
      using C = std::remove_pointer_t<decltype(tag)>;
      std::vector<Link3<C>> lk(std::max<size_t>(1, n_links));
      for (size_t k = 0; k < n_links; k++) {
        const double *cf = &coef[8 * k];
        lk[slot[k]] = Link3<C>{static_cast<C>(cf[0]), static_cast<C>(cf[1]), static_cast<C>(cf[2]),
                               static_cast<C>(cf[3])};
      }
      Const3<C> &kc = h->kc.get(tag);
      for (int a = 0; a < Q; a++) {
        const double s = 1.0 / tau[a];
        kc.s_scaled[a] = static_cast<C>(s / L.norm[a]);
        kc.f_scaled[a] = static_cast<C>((1.0 - 0.5 * s) / L.norm[a]);
      }
      kc.ax = static_cast<C>(dom->ax);
      kc.ay = static_cast<C>(dom->ay);
      kc.az = static_cast<C>(dom->az);
      kc.nx = nx;
      kc.ny = ny;
      kc.nz = nz;
      kc.px = per[0];
      kc.py = per[1];
      kc.pz = per[2];
      kc.diffuse_mode = p.diffuse_mode;
      kc.plane = h->plane;
      return cudaMemcpy(h->links, lk.data(), lk.size() * sizeof(Link3<C>), cudaMemcpyHostToDevice);
    });
  if (e != cudaSuccess) {
    const int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    g_err3 = std::string("device setup: ") + cudaGetErrorString(e);
    release3(h);
    return code;
  }
  *out = h;
  return LBM_OK;
}

int lbm3d_step(lbm3d_t *h, int64_t n) {
  using namespace lbm3;
  if (!h) return LBM_EINVAL;
  if (n < 0) return fail3(h, LBM_EINVAL, "negative step count");
  for (int64_t s = 0; s < n; s++) {
    const int src = h->cur, dst = 1 - h->cur;
    cudaError_t e = dispatch3(h->precision, [&](auto tag) {
      using C = std::remove_pointer_t<decltype(tag)>;
      step3_kernel<C><<<static_cast<unsigned>((h->n_nodes + kThreads3 - 1) / kThreads3), kThreads3,
                        0, h->stream>>>(static_cast<const C *>(h->f[src]),
                                        static_cast<C *>(h->f[dst]), h->flags, h->lbase,
                                        static_cast<const Link3<C> *>(h->links), h->kc.get(tag),
                                        h->n_nodes);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return fail3(h, LBM_ECUDA, std::string("step: ") + cudaGetErrorString(e));
    h->cur = dst;
    h->steps++;
  }
  return LBM_OK;
}

int lbm3d_residual(lbm3d_t *h, double *residual, double *mass) {
  using namespace lbm3;
  if (!h) return LBM_EINVAL;
  double tot[4];
  cudaError_t e = dispatch3(h->precision, [&](auto tag) {
    using C = std::remove_pointer_t<decltype(tag)>;
    residual3_kernel<C><<<kResBlocks3, kResThreads3, 0, h->stream>>>(
        static_cast<const C *>(h->f[h->cur]), static_cast<const C *>(h->f[1 - h->cur]), h->flags,
        h->lbase, h->kc.get(tag), h->n_nodes, h->partials);
    residual3_final<<<1, 1024, 0, h->stream>>>(h->partials, h->result);
    return cudaGetLastError();
  });
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot, h->result, sizeof tot, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail3(h, LBM_ECUDA, std::string("residual: ") + cudaGetErrorString(e));
  double res;
  if (std::isnan(tot[0]) || std::isnan(tot[1])) res = std::numeric_limits<double>::quiet_NaN();
  else res = tot[1] > 0.0 ? std::sqrt(tot[0] / tot[1]) : (tot[0] > 0.0 ? INFINITY : 0.0);
  if (residual) *residual = res;
  if (mass) *mass = static_cast<double>(h->n_fluid) + tot[2];
  if (tot[3] > 0.0) return fail3(h, LBM_EUNSTABLE, "fluid nodes with non-finite density or velocity");
  return LBM_OK;
}

int lbm3d_get_f(lbm3d_t *h, double *f) {
  using namespace lbm3;
  if (!h || !f) return h ? fail3(h, LBM_EINVAL, "null output") : LBM_EINVAL;
  double *d = nullptr;
  const size_t bytes = static_cast<size_t>(Q) * h->n_nodes * sizeof(double);
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e == cudaSuccess)
    e = dispatch3(h->precision, [&](auto tag) {
      using C = std::remove_pointer_t<decltype(tag)>;
      export3_kernel<C><<<grid_for3(Q * h->n_nodes, 256), 256, 0, h->stream>>>(
          static_cast<const C *>(h->f[h->cur]), h->flags, h->lbase, h->kc.get(tag), h->n_nodes, d);
      return cudaGetLastError();
    });
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(f, d, bytes, cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail3(h, LBM_ECUDA, std::string("get_f: ") + cudaGetErrorString(e));
  return LBM_OK;
}

int lbm3d_set_f(lbm3d_t *h, const double *f) {
  using namespace lbm3;
  if (!h || !f) return h ? fail3(h, LBM_EINVAL, "null input") : LBM_EINVAL;
  double *d = nullptr;
  const size_t bytes = static_cast<size_t>(Q) * h->n_nodes * sizeof(double);
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(d, f, bytes, cudaMemcpyHostToDevice);
  for (int b = 0; b < 2 && e == cudaSuccess; b++)
    e = dispatch3(h->precision, [&](auto tag) {
      using C = std::remove_pointer_t<decltype(tag)>;
      import3_kernel<C><<<grid_for3(Q * h->n_nodes, 256), 256, 0, h->stream>>>(
          d, h->flags, h->lbase, h->kc.get(tag), h->n_nodes, static_cast<C *>(h->f[b]));
      return cudaGetLastError();
    });
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail3(h, LBM_ECUDA, std::string("set_f: ") + cudaGetErrorString(e));
  h->steps = 0;
  return LBM_OK;
}

int lbm3d_fields(lbm3d_t *h, double *rho, double *ux, double *uy, double *uz) {
  using namespace lbm3;
  if (!h) return LBM_EINVAL;
  double *d = nullptr;
  const size_t n = static_cast<size_t>(h->n_nodes);
  cudaError_t e = cudaMalloc(&d, 4 * n * sizeof(double));
  if (e == cudaSuccess)
    e = dispatch3(h->precision, [&](auto tag) {
      using C = std::remove_pointer_t<decltype(tag)>;
      fields3_kernel<C><<<grid_for3(h->n_nodes, 256), 256, 0, h->stream>>>(
          static_cast<const C *>(h->f[h->cur]), h->flags, h->lbase, h->kc.get(tag), h->n_nodes, d);
      return cudaGetLastError();
    });
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  double *outs[4] = {rho, ux, uy, uz};
  for (int a = 0; a < 4 && e == cudaSuccess; a++)
    if (outs[a]) e = cudaMemcpy(outs[a], d + a * n, n * sizeof(double), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail3(h, LBM_ECUDA, std::string("fields: ") + cudaGetErrorString(e));
  return LBM_OK;
}

int lbm3d_link_params(const lbm3d_t *h, double *r, double *l) {
  if (!h) return LBM_EINVAL;
  if (r) std::copy(h->link_r.begin(), h->link_r.end(), r);
  if (l) std::copy(h->link_l.begin(), h->link_l.end(), l);
  return LBM_OK;
}

void lbm3d_destroy(lbm3d_t *h) { release3(h); }

const char *lbm3d_last_error(const lbm3d_t *h) { return h ? h->err.c_str() : g_err3.c_str(); }

}  // extern "C"
