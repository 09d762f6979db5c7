// Device kernels of liblbm.so: the fused collide-stream-boundary step, the
// FP64 residual/mass reduction, and field/population conversion.
//
// Populations are stored as deviations d_i = f_i - w_i (rest state rho = 1,
// u = 0 is d = 0), one plane per direction, over the fluid nodes only, in
// row-major order (compacted lattice: every thread of the step kernel owns
// a fluid node, no sector holds solid slots).  A single case's step kernel
// is a pull scheme (pull_slots): each fluid node gathers f(x, t) from the
// post-collision values its neighbours stored in the previous step,
// collides in moment space (Sec. 2), and stores f'(x, t) in its own slots
// of the other lattice: every store is aligned and coalesced.  Unknown
// populations of a boundary node (x_f - c_i solid) come from Eq. EqNewBDSC,
// which is local (f_ib(x_f, t), f'_i(x_f, t), f'_ib(x_f, t) and rho_f all
// belong to x_f): the node evaluates them in the same step and keeps them
// in the lattice's link tail, where its next gather finds them.  The
// batched solver (lbm_batch.cu) runs the same per-node update on each case
// of its arena.
#include <cstdint>
#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

using namespace dev;

// One time step of a single case (pull layout): thread t of CTA b runs
// fluid node b * kPullThreads + t.
//
// Each node waits out two dependent memory latencies (its node word, then
// the gathers it addresses), which 64 warps per SM do not hide.  So every
// CTA first asks L2 for the data of the CTA g.pf_dist blocks ahead (half
// the CTAs resident at once: it starts about half a CTA lifetime from now
// on some SM): its node words, group record and own slots in the nine
// planes.  A prefetch holds no register and never waits; the later loads
// then find their lines in L2 (the gathers from the rows above and below
// mostly hit lines that the neighbouring rows' CTAs brought in).
//
// kExact: the exact-mass variant of FP32 storage (cases with moving walls;
// see collide and link_epilogue_pull), with 64 registers per thread.
template <typename T, typename C, bool kExact>
__global__ void __launch_bounds__(kPullThreads, kExact ? 8 : PullOcc<T>::min_blocks)
step_kernel_pull(const T *__restrict__ src, T *__restrict__ dst, __grid_constant__ const PullGeom g,
                 const uint32_t n_fluid, const LinkCoef<C> *__restrict__ links,
                 __grid_constant__ const StepConst<C> k) {
  {
    constexpr uint32_t kNodeLines = kPullThreads * sizeof(uint2) / 128;
    constexpr uint32_t kPlaneLines = kPullThreads * sizeof(T) / 128;
    constexpr uint32_t kPerLine = 128 / sizeof(T);
    const uint32_t base = (blockIdx.x + g.pf_dist) * kPullThreads;
    const uint32_t t = threadIdx.x;
    // whole warps: the others skip the block without diverging
    constexpr uint32_t kPfThreads = (kNodeLines + 9 * kPlaneLines + 1 + 31) / 32 * 32;
    static_assert(kPfThreads <= kPullThreads, "one prefetch per thread");
    if (t < kPfThreads && g.pf_dist && base < n_fluid) {
      if (t < kNodeLines) {
        if (base + t * 16 < n_fluid)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(g.node + base + t * 16));
      } else if (t < kNodeLines + 9 * kPlaneLines) {
        const uint32_t q = (t - kNodeLines) / kPlaneLines, l = (t - kNodeLines) % kPlaneLines;
        if (base + l * kPerLine < n_fluid)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(src + q * g.plane + base + l * kPerLine));
      } else if (t == kNodeLines + 9 * kPlaneLines) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(g.grp + base / kGroup));
      }
    }
  }
  const uint32_t i = blockIdx.x * kPullThreads + threadIdx.x;
  if (i >= n_fluid) return;
  if constexpr (kExact)
    step_node_exact(src, dst, g, links, k, i, k.sr_seed);
  else
    step_node_pull<T, C, false, kPullThreads / 32>(src, dst, g, links, k, i, k.sr_seed);
}

// One time step of a single case in 16-bit storage: thread t of CTA b runs
// the fluid-node pair 2 (b kPairThreads + t), 2 (b kPairThreads + t) + 1
// (step_pair_pull; a lone last node takes the one-node step), after the
// same L2 prefetch of the data of the CTA g.pf_dist blocks ahead as
// step_kernel_pull.
template <typename T>
__global__ void __launch_bounds__(kPairThreads, PairOcc::min_blocks)
step_kernel_pair(const T *__restrict__ src, T *__restrict__ dst, const PullGeom g,
                 const uint32_t n_fluid, const LinkCoef<float> *__restrict__ links,
                 const StepConst<float> k) {
  constexpr uint32_t kNodes = 2 * kPairThreads;  // per CTA
  {
    constexpr uint32_t kNodeLines = kNodes * sizeof(uint2) / 128;
    constexpr uint32_t kPlaneLines = kNodes * sizeof(T) / 128;
    constexpr uint32_t kPerLine = 128 / sizeof(T);
    constexpr uint32_t kGrpLines = (kNodes / kGroup * sizeof(int2) + 127) / 128;
    const uint32_t base = (blockIdx.x + g.pf_dist) * kNodes;
    const uint32_t t = threadIdx.x;
    constexpr uint32_t kPfThreads = (kNodeLines + 9 * kPlaneLines + kGrpLines + 31) / 32 * 32;
    static_assert(kPfThreads <= kPairThreads, "one prefetch per thread");
    if (t < kPfThreads && g.pf_dist && base < n_fluid) {
      if (t < kNodeLines) {
        if (base + t * 16 < n_fluid)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(g.node + base + t * 16));
      } else if (t < kNodeLines + 9 * kPlaneLines) {
        const uint32_t q = (t - kNodeLines) / kPlaneLines, l = (t - kNodeLines) % kPlaneLines;
        if (base + l * kPerLine < n_fluid)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(src + q * g.plane + base + l * kPerLine));
      } else if (t < kNodeLines + 9 * kPlaneLines + kGrpLines) {
        const uint32_t l = t - kNodeLines - 9 * kPlaneLines;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(g.grp + base / kGroup + l * 16));
      }
    }
  }
  const uint32_t i0 = 2u * (blockIdx.x * kPairThreads + threadIdx.x);
  if (i0 >= n_fluid) return;
  if (i0 + 1u < n_fluid)
    step_pair_pull<T>(src, dst, g, links, k, i0, k.sr_seed);
  else
    step_node_pull<T, float, false>(src, dst, g, links, k, i0, k.sr_seed);
}

// Mass deviation of one node, sum_i d_i, to FP64 accuracy.  FP64 storage:
// the plain FP64 sum.  FP32 arithmetic: cascaded TwoSum in FP32 (the sum
// as if computed in twice the working precision, Ogita, Rump and Oishi's
// Sum2), then one conversion -- the FP64 units of this GPU are few, and nine
// conversions and eight FP64 additions per node would bound the pass.
__device__ __forceinline__ double node_mass(const double (&a)[9]) {
  double sm = 0.0;
#pragma unroll
  for (int i = 0; i < 9; i++) sm += a[i];
  return sm;
}
__device__ __forceinline__ double node_mass(const float (&a)[9]) {
  float s = a[0], e = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; i++) {
    float t;
    two_sum(s, a[i], s, t);
    e += t;
  }
  return static_cast<double>(s) + static_cast<double>(e);
}

// Residual pass 1: thread g of the fixed grid reduces nodes g, g + G,
// g + 2G, ... (G threads in all) into num, den, mass deviation, non-finite
// count: per-node terms in the storage's arithmetic type, sums in FP64
// (warp shuffles, then shared memory), block b's four sums to
// partials[b * 4 + {0..3}].  The node-to-thread map is fixed, so the result
// is bitwise reproducible.
template <typename T>
__global__ void __launch_bounds__(kResidualThreads)
residual_partials_compact(const T *__restrict__ cur, const T *__restrict__ prev,
                          const NodeMap map, int64_t n_fluid, int64_t plane, double ax, double ay,
                          double inv_scale, double *__restrict__ partials) {
  using C = typename Stor<T>::C;
  const C inv = static_cast<C>(inv_scale);
  double num = 0.0, den = 0.0, dm = 0.0, bad = 0.0;
  const int64_t G = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t node = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; node < n_fluid;
       node += G) {
    uint32_t s[9];
    map.slots(static_cast<uint32_t>(node), static_cast<uint32_t>(plane), s);
    C a[9], b[9];
    bool sat = false;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      a[i] = Stor<T>::ld(cur[s[i]], inv);
      b[i] = Stor<T>::ld(prev[s[i]], inv);
      if constexpr (kStochastic<T>)
        sat |= fabsf(Stor<T>::ld_raw(cur[s[i]])) >= Stor<T>::kMaxRaw ||
               fabsf(Stor<T>::ld_raw(prev[s[i]])) >= Stor<T>::kMaxRaw;
    }
    C n1, d1, m1;
    residual_terms<C>(a, b, static_cast<C>(ax), static_cast<C>(ay), n1, d1, m1);
    // a saturated 16-bit value (stochastic rounding saturates instead of
    // overflowing to infinity) counts as non-finite
    if (sat || !(isfinite(n1) && isfinite(d1) && isfinite(m1))) {
      bad += 1.0;
      continue;
    }
    num += static_cast<double>(n1);
    den += static_cast<double>(d1);
    dm += node_mass(a);
  }
  __shared__ double sh[kResidualThreads / 32][kPartialStride];
  num = warp_sum(num);
  den = warp_sum(den);
  dm = warp_sum(dm);
  bad = warp_sum(bad);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[w][0] = num;
    sh[w][1] = den;
    sh[w][2] = dm;
    sh[w][3] = bad;
  }
  __syncthreads();
  if (threadIdx.x < kPartialStride) {
    double t = 0.0;
    for (int i = 0; i < kResidualThreads / 32; i++) t += sh[i][threadIdx.x];
    partials[blockIdx.x * kPartialStride + threadIdx.x] = t;
  }
}

// The interval residual's pass 1 (same grid and order as
// residual_partials_compact): per node the velocity of cur (Eq. FluidMacr,
// in the storage's arithmetic type) against the snapshot, which it replaces.
template <typename T>
__global__ void __launch_bounds__(kResidualThreads)
residual_interval_compact(const T *__restrict__ cur, const NodeMap map, int64_t n_fluid,
                          int64_t plane, double ax, double ay, double inv_scale,
                          typename Stor<T>::C *__restrict__ snap, double *__restrict__ partials) {
  using C = typename Stor<T>::C;
  const C inv = static_cast<C>(inv_scale);
  double num = 0.0, den = 0.0, dm = 0.0, bad = 0.0;
  const int64_t G = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t node = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; node < n_fluid;
       node += G) {
    uint32_t s[9];
    map.slots(static_cast<uint32_t>(node), static_cast<uint32_t>(plane), s);
    C a[9];
    bool sat = false;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      a[i] = Stor<T>::ld(cur[s[i]], inv);
      if constexpr (kStochastic<T>) sat |= fabsf(Stor<T>::ld_raw(cur[s[i]])) >= Stor<T>::kMaxRaw;
    }
    const C r = C(1) + (((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])) + a[8]);
    const C jx = a[1] - a[3] + (a[5] - a[6]) + (a[8] - a[7]);
    const C jy = a[2] - a[4] + (a[5] + a[6]) - (a[7] + a[8]);
    const C ux = (jx + C(0.5) * r * static_cast<C>(ax)) / r;
    const C uy = (jy + C(0.5) * r * static_cast<C>(ay)) / r;
    const C px = snap[2 * node], py = snap[2 * node + 1];
    snap[2 * node] = ux;
    snap[2 * node + 1] = uy;
    if (sat || !(isfinite(ux) && isfinite(uy) && isfinite(r))) {
      bad += 1.0;
      continue;
    }
    const C dx = ux - px, dy = uy - py;
    num += static_cast<double>(dx * dx + dy * dy);
    den += static_cast<double>(ux * ux + uy * uy);
    dm += node_mass(a);
  }
  __shared__ double sh[kResidualThreads / 32][kPartialStride];
  num = warp_sum(num);
  den = warp_sum(den);
  dm = warp_sum(dm);
  bad = warp_sum(bad);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[w][0] = num;
    sh[w][1] = den;
    sh[w][2] = dm;
    sh[w][3] = bad;
  }
  __syncthreads();
  if (threadIdx.x < kPartialStride) {
    double t = 0.0;
    for (int i = 0; i < kResidualThreads / 32; i++) t += sh[i][threadIdx.x];
    partials[blockIdx.x * kPartialStride + threadIdx.x] = t;
  }
}

// Pass 2: one block of kFinalThreads sums the partials in a fixed order
// (thread t first adds blocks t, t + kFinalThreads, ...).
constexpr int kFinalThreads = 1024;
static_assert(kResidualBlocks % kFinalThreads == 0, "whole rounds of partials");
__global__ void __launch_bounds__(kFinalThreads)
residual_final(const double *__restrict__ partials, double *__restrict__ out) {
  __shared__ double sh[kFinalThreads / 32][kPartialStride];
  double v[kPartialStride];
  for (int c = 0; c < kPartialStride; c++) {
    double t = 0.0;
    for (int b = threadIdx.x; b < kResidualBlocks; b += kFinalThreads)
      t += partials[b * kPartialStride + c];
    v[c] = warp_sum(t);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int c = 0; c < kPartialStride; c++) sh[w][c] = v[c];
  __syncthreads();
  if (threadIdx.x < kPartialStride) {
    double s = 0.0;
    for (int i = 0; i < kFinalThreads / 32; i++) s += sh[i][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

template <typename T>
__global__ void fields_kernel(const T *__restrict__ f, const NodeMap map, int64_t plane, double ax,
                              double ay, double inv_scale, double *rho, double *ux, double *uy) {
  using C = typename Stor<T>::C;
  const int64_t n = static_cast<int64_t>(map.nx) * map.ny;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t y = p / map.nx, x = p - y * map.nx;
    const int64_t node = map.at(static_cast<int>(x), static_cast<int>(y));
    double r = 0.0, u = 0.0, v = 0.0;
    if (node >= 0) {
      uint32_t s[9];
      map.slots(static_cast<uint32_t>(node), static_cast<uint32_t>(plane), s);
      double a[9];
      for (int i = 0; i < 9; i++)
        a[i] = static_cast<double>(Stor<T>::ld(f[s[i]], static_cast<C>(inv_scale)));
      node_velocity(a, ax, ay, r, u, v);
    }
    if (rho) rho[p] = r;
    if (ux) ux[p] = u;
    if (uy) uy[p] = v;
  }
}

// Populations from macroscopic fields (a warm start): for every fluid node
// f_i = f_i^eq(rho, u - a/2) - 3 tau_s w_i rho (c_i c_i - I/3) : grad u,
// i.e. the equilibrium (Eq. LBEequi) at the velocity whose half-force
// corrected moment (Eq. FluidMacr) is u, plus the first-order
// Chapman-Enskog non-equilibrium part; grad u by central differences over
// fluid neighbours (one-sided next to a wall, 0 if both neighbours are
// solid).  Written as deviations into both lattices; solid nodes get 0.
template <typename T>
__global__ void set_fields_kernel(const double *__restrict__ rho, const double *__restrict__ ux,
                                  const double *__restrict__ uy, const NodeMap map, int64_t plane,
                                  int32_t px, int32_t py, double ax, double ay, double tau_s,
                                  double scale, T *f0, T *f1) {
  using C = typename Stor<T>::C;
  const int32_t nx = map.nx, ny = map.ny;
  const int64_t n = static_cast<int64_t>(nx) * ny;
  const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int y = static_cast<int>(p / nx), x = static_cast<int>(p - static_cast<int64_t>(y) * nx);
    const int64_t node = map.at(x, y);
    if (node < 0) continue;
    double dv[9];
    {
      auto fluid_at = [&](int xx, int yy, int64_t *q) {
        if (xx < 0 || xx >= nx) {
          if (!px) return false;
          xx = (xx + nx) % nx;
        }
        if (yy < 0 || yy >= ny) {
          if (!py) return false;
          yy = (yy + ny) % ny;
        }
        if (map.at(xx, yy) < 0) return false;
        *q = static_cast<int64_t>(yy) * nx + xx;
        return true;
      };
      // d/dx and d/dy of (ux, uy)
      double g[2][2];
      for (int axis = 0; axis < 2; axis++) {
        int64_t qp = 0, qm = 0;
        const bool hp = fluid_at(x + (axis == 0), y + (axis == 1), &qp);
        const bool hm = fluid_at(x - (axis == 0), y - (axis == 1), &qm);
        for (int comp = 0; comp < 2; comp++) {
          const double *u = comp == 0 ? ux : uy;
          double d = 0.0;
          if (hp && hm) d = 0.5 * (u[qp] - u[qm]);
          else if (hp) d = u[qp] - u[p];
          else if (hm) d = u[p] - u[qm];
          g[axis][comp] = d;  // d u_comp / d x_axis
        }
      }
      const double r = rho[p];
      const double vx = ux[p] - 0.5 * ax, vy = uy[p] - 0.5 * ay;
      const double vv = vx * vx + vy * vy;
      const double div = g[0][0] + g[1][1];
      for (int i = 0; i < 9; i++) {
        const double cu = cx[i] * vx + cy[i] * vy;
        const double feq = w[i] * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * vv);
        const double qg = cx[i] * cx[i] * g[0][0] + cx[i] * cy[i] * (g[0][1] + g[1][0]) +
                          cy[i] * cy[i] * g[1][1] - div / 3.0;
        dv[i] = feq - 3.0 * tau_s * w[i] * r * qg - w[i];
      }
    }
    uint32_t s[9];
    map.slots(static_cast<uint32_t>(node), static_cast<uint32_t>(plane), s);
    for (int i = 0; i < 9; i++) {
      const T v = Stor<T>::st(static_cast<C>(dv[i]), static_cast<C>(scale));
      f0[s[i]] = v;
      f1[s[i]] = v;
    }
  }
}

__constant__ double kWd[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

template <typename T>
__global__ void export_kernel(const T *__restrict__ f, const NodeMap map, int64_t plane,
                              double inv_scale, double *out) {
  using C = typename Stor<T>::C;
  const int64_t n = static_cast<int64_t>(map.nx) * map.ny;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < 9 * n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = p / n, q = p - i * n, y = q / map.nx, x = q - y * map.nx;
    // solid nodes carry no state (the compacted lattice has no slots for
    // them): they read as the rest state
    const int64_t node = map.at(static_cast<int>(x), static_cast<int>(y));
    double d = 0.0;
    if (node >= 0) {
      uint32_t s[9];
      map.slots(static_cast<uint32_t>(node), static_cast<uint32_t>(plane), s);
      d = static_cast<double>(Stor<T>::ld(f[s[i]], static_cast<C>(inv_scale)));
    }
    out[p] = kWd[i] + d;
  }
}

template <typename T>
__global__ void import_kernel(const double *__restrict__ in, const NodeMap map, int64_t plane,
                              double scale, T *f) {
  using C = typename Stor<T>::C;
  const int64_t n = static_cast<int64_t>(map.nx) * map.ny;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < 9 * n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = p / n, q = p - i * n, y = q / map.nx, x = q - y * map.nx;
    const int64_t node = map.at(static_cast<int>(x), static_cast<int>(y));
    if (node >= 0) {
      uint32_t s[9];
      map.slots(static_cast<uint32_t>(node), static_cast<uint32_t>(plane), s);
      f[s[i]] = Stor<T>::st(static_cast<C>(in[p] - kWd[i]), static_cast<C>(scale));
    }
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return static_cast<int>(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace

template <typename T, typename C>
int pull_resident_ctas() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  cudaError_t e;
  if constexpr (kStochastic<T>)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_kernel_pair<T>, kPairThreads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_kernel_pull<T, C, false>,
                                                      kPullThreads, 0);
  return e == cudaSuccess ? sms * per : 0;
}

template <typename T, typename C>
cudaError_t launch_step_pull(const T *src, T *dst, const PullGeom &g, int64_t n_fluid,
                             const LinkCoef<C> *links, const StepConst<C> &k, cudaStream_t s) {
  if (n_fluid <= 0) return cudaSuccess;
  if constexpr (kStochastic<T>) {
    const int64_t pairs = (n_fluid + 1) / 2;
    step_kernel_pair<T><<<static_cast<unsigned>((pairs + kPairThreads - 1) / kPairThreads),
                          kPairThreads, 0, s>>>(src, dst, g, static_cast<uint32_t>(n_fluid), links,
                                                k);
  } else {
    const int64_t blocks = (n_fluid + kPullThreads - 1) / kPullThreads;
    if constexpr (std::is_same<T, float>::value) {
      if (k.exact) {
        if (!g.links64 || !g.carry || !g.carry0) return cudaErrorInvalidValue;
        step_kernel_pull<T, C, true><<<static_cast<unsigned>(blocks), kPullThreads, 0, s>>>(
            src, dst, g, static_cast<uint32_t>(n_fluid), links, k);
        return cudaGetLastError();
      }
    }
    step_kernel_pull<T, C, false><<<static_cast<unsigned>(blocks), kPullThreads, 0, s>>>(
        src, dst, g, static_cast<uint32_t>(n_fluid), links, k);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_compact(const T *cur, const T *prev, const NodeMap &map,
                                    int64_t n_fluid, int64_t plane, double ax, double ay,
                                    double scale, double *partials, double *result, cudaStream_t s) {
  residual_partials_compact<T><<<kResidualBlocks, kResidualThreads, 0, s>>>(
      cur, prev, map, n_fluid, plane, ax, ay, 1.0 / scale, partials);
  residual_final<<<1, kFinalThreads, 0, s>>>(partials, result);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_interval(const T *cur, const NodeMap &map, int64_t n_fluid,
                                     int64_t plane, double ax, double ay, double scale, void *snap,
                                     double *partials, double *result, cudaStream_t s) {
  residual_interval_compact<T><<<kResidualBlocks, kResidualThreads, 0, s>>>(
      cur, map, n_fluid, plane, ax, ay, 1.0 / scale, static_cast<typename Stor<T>::C *>(snap),
      partials);
  residual_final<<<1, kFinalThreads, 0, s>>>(partials, result);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fields(const T *f, const NodeMap &map, int64_t plane, double ax, double ay,
                          double scale, double *rho, double *ux, double *uy, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(map.nx) * map.ny;
  fields_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(f, map, plane, ax, ay, 1.0 / scale, rho, ux, uy);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export_f(const T *f, const NodeMap &map, int64_t plane, double scale,
                            double *out, cudaStream_t s) {
  const int64_t n = 9 * static_cast<int64_t>(map.nx) * map.ny;
  export_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(f, map, plane, 1.0 / scale, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_set_fields(const double *rho, const double *ux, const double *uy,
                              const NodeMap &map, int64_t plane, int32_t px, int32_t py,
                              double ax, double ay, double tau_s, double scale, T *f0, T *f1,
                              cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(map.nx) * map.ny;
  set_fields_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(rho, ux, uy, map, plane, px, py, ax, ay,
                                                        tau_s, scale, f0, f1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_import_f(const double *in, const NodeMap &map, int64_t plane, double scale,
                            T *f, cudaStream_t s) {
  const int64_t n = 9 * static_cast<int64_t>(map.nx) * map.ny;
  import_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(in, map, plane, scale, f);
  return cudaGetLastError();
}

#define LBM_INSTANTIATE(T, C)                                                                      \
  template int pull_resident_ctas<T, C>();                                                         \
  template cudaError_t launch_step_pull<T, C>(const T *, T *, const PullGeom &, int64_t,          \
                                              const LinkCoef<C> *, const StepConst<C> &,           \
                                              cudaStream_t);                                       \
  template cudaError_t launch_residual_compact<T>(const T *, const T *, const NodeMap &, int64_t,  \
                                                  int64_t, double, double, double, double *,       \
                                                  double *, cudaStream_t);                         \
  template cudaError_t launch_residual_interval<T>(const T *, const NodeMap &, int64_t, int64_t,   \
                                                   double, double, double, void *, double *,       \
                                                   double *, cudaStream_t);                        \
  template cudaError_t launch_fields<T>(const T *, const NodeMap &, int64_t, double, double,       \
                                        double, double *, double *, double *, cudaStream_t);       \
  template cudaError_t launch_export_f<T>(const T *, const NodeMap &, int64_t, double, double *,   \
                                          cudaStream_t);                                           \
  template cudaError_t launch_import_f<T>(const double *, const NodeMap &, int64_t, double, T *,   \
                                          cudaStream_t);                                           \
  template cudaError_t launch_set_fields<T>(const double *, const double *, const double *,        \
                                            const NodeMap &, int64_t, int32_t, int32_t, double,    \
                                            double, double, double, T *, T *, cudaStream_t);

LBM_INSTANTIATE(double, double)
LBM_INSTANTIATE(float, float)
LBM_INSTANTIATE(__half, float)
LBM_INSTANTIATE(__nv_bfloat16, float)

}  // namespace lbm
