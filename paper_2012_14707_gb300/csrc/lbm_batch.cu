// Batched solver of liblbm.so (lbm_batch_*): many independent cases of
// different sizes, geometries and parameters advanced together.
//
// All cases live in one device arena (each case's compacted lattice in the
// pull layout of pull_slots: two lattices of its nine deviation planes over
// its fluid nodes plus its link tail, node words, group records, row
// starts, link coefficients and f_jb slots).  In the node arena every
// case starts on a multiple of kChunk nodes, so a CTA of the step launch
// (at most kChunk threads) runs nodes of one case only, found in a
// per-chunk case index: a time step is one launch over the whole node
// arena; a CTA looks up its case's constants in a descriptor table and runs
// the single-case kernel's per-node update (step_node_pull), so a case in a
// batch follows exactly the arithmetic of the case run alone.  Every K
// steps a batched reduction (one CTA per case, fixed order) computes each
// case's residual and retires converged cases on the device; retired
// cases' CTAs return immediately.  K steps plus the reduction are captured
// once in a CUDA graph that the host replays, reading back only the number
// of active cases.  The CTA width and the L2 prefetch are picked by timing
// the candidates on the batch itself (autotuner), cached per size class and
// precision.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

using namespace dev;

// One case in the arenas: its compacted lattice (see CompactCase) at these
// offsets.  Indices inside a case (pull slots, links) are the case's own.
template <typename C>
struct BatchCase {
  StepConst<C> k;    // plane = the case's padded fluid-node count
  int64_t f_off;     // element offset of the case's lattice (9 planes + link tail)
  int64_t node_off;  // offset of the case in the node-word arena (a multiple of kChunk)
  int64_t grp_off;   // offset of the case's group records
  int64_t row_off;   // offset of the case's rowstart
  int64_t idx_off;   // offset of the case's node map (nx * ny)
  int64_t link_off;  // offset of the case's links (coefficients, f_jb slots)
  int64_t n_fluid;
};

// The pull geometry of case bc inside the arenas.
template <typename C>
__host__ __device__ inline PullGeom case_geom(const BatchCase<C> &bc, const uint2 *node,
                                              const int2 *grp, const int32_t *rowstart,
                                              const uint32_t *jbslot,
                                              const LinkCoefDF *links64 = nullptr,
                                              float *carry = nullptr, float *carry0 = nullptr,
                                              const uint16_t *ldesc = nullptr) {
  PullGeom g;
  g.node = node + bc.node_off;
  g.grp = grp + bc.grp_off;
  g.rowstart = rowstart + bc.row_off;
  g.jbslot = jbslot ? jbslot + bc.link_off : nullptr;
  g.ldesc = ldesc ? ldesc + bc.link_off : nullptr;
  g.ny = bc.k.ny;
  g.periodic_y = bc.k.periodic_y;
  g.plane = static_cast<uint32_t>(bc.k.plane);
  g.n_fluid = static_cast<uint32_t>(bc.n_fluid);
  g.pf_dist = 0;
  g.links64 = links64 ? links64 + bc.link_off : nullptr;
  g.carry = carry ? carry + bc.link_off : nullptr;
  g.carry0 = carry0 ? carry0 + bc.node_off : nullptr;
  return g;
}


constexpr int kBatchResidualThreads = 256;
constexpr int kChunk = 256;  // node-arena alignment of every case (>= any CTA width)

// Registers bounded like the single-case kernel (the same resident threads
// per SM).  CTA b runs node-arena entries b * THREADS .. b * THREADS +
// THREADS - 1, all of case ccase[b * THREADS / kChunk] (the index is
// CTA-uniform, so the case's constants stay out of the per-thread
// registers).  Like the single-case kernel, each CTA first asks L2 for the
// node words and case index of the CTA pf_dist blocks ahead.  The step
// count of every active case is *counter + j (the graph replays K steps,
// j = 0 .. K-1, between advances of the counter), which seeds the random
// bits exactly as the case's own step count does when it runs alone.  FP32
// cases with moving walls (k.exact) are left to batch_exact_kernel.
template <typename T, typename C, int THREADS>
__global__ void __launch_bounds__(THREADS, PullOcc<T>::min_blocks * kPullThreads / THREADS)
batch_step_kernel(const T *__restrict__ src, T *__restrict__ dst,
                  const uint2 *__restrict__ node, const int2 *__restrict__ grp,
                  const int32_t *__restrict__ ccase, const int32_t *__restrict__ rowstart,
                  const uint32_t *__restrict__ jbslot, const LinkCoef<C> *__restrict__ links,
                  const BatchCase<C> *__restrict__ cases, const int32_t *__restrict__ active,
                  const int32_t *__restrict__ work, const uint32_t n_blocks,
                  const uint32_t pf_dist, const int64_t *__restrict__ counter, const uint32_t j,
                  const PullGeom *__restrict__ geoms) {
  static_assert(kChunk % THREADS == 0, "a CTA stays inside one chunk");
  constexpr uint32_t kPer = kChunk / THREADS;  // CTAs per chunk
  {
    // L2 prefetch for the CTA pf_dist blocks ahead: its node words, chunk
    // case index and, in the case's nine planes, its nodes' own slots
    constexpr uint32_t kNodeLines = THREADS * sizeof(uint2) / 128;
    constexpr uint32_t kPlaneLines = (THREADS * sizeof(T) + 127) / 128;
    constexpr uint32_t kPerLine = 128 / sizeof(T);
    const uint32_t b2 = blockIdx.x + pf_dist;
    const uint32_t t = threadIdx.x;
    if (pf_dist && t < kNodeLines + 9 * kPlaneLines + 1 && b2 < n_blocks) {
      const uint32_t chunk2 = static_cast<uint32_t>(work[b2 / kPer]);
      const uint32_t base2 = chunk2 * kChunk + (b2 % kPer) * THREADS;
      if (t < kNodeLines) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(node + base2 + t * 16));
      } else if (t == kNodeLines) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ccase + chunk2));
      } else {
        const BatchCase<C> &c2 = cases[ccase[chunk2]];
        const uint32_t q = (t - kNodeLines - 1) / kPlaneLines, l = (t - kNodeLines - 1) % kPlaneLines;
        const uint32_t i2 = base2 - static_cast<uint32_t>(c2.node_off) + l * kPerLine;
        if (i2 < static_cast<uint32_t>(c2.n_fluid))
          asm volatile("prefetch.global.L2 [%0];" ::"l"(src + c2.f_off + q * c2.k.plane + i2));
      }
    }
  }
  const int32_t chunk = work[blockIdx.x / kPer];
  const int c = ccase[chunk];
  if (!active[c]) return;
  const BatchCase<C> &bc = cases[c];
  const uint32_t i = static_cast<uint32_t>(chunk) * kChunk + (blockIdx.x % kPer) * THREADS +
                     threadIdx.x - static_cast<uint32_t>(bc.node_off);
  if (i >= static_cast<uint32_t>(bc.n_fluid)) return;
  // exact-mass cases run in batch_exact_kernel
  if (std::is_same<T, float>::value && bc.k.exact) return;
  // the case's geometry from the device table (a local copy would be
  // spilled at this kernel's register budget)
  const PullGeom &g = geoms[c];
  uint32_t seed = 0;
  if constexpr (kStochastic<T>) seed = step_seed(*counter + j);
  step_node_pull<T, C, false, THREADS / 32>(src + bc.f_off, dst + bc.f_off, g,
                                            links + bc.link_off, bc.k, i, seed);
}

// 16-bit batches: the paired step of the single-case kernel
// (step_pair_pull).  CTA b runs node-arena entries b * 2 THREADS ..
// (b + 1) * 2 THREADS - 1, two per thread, all of one case (2 THREADS
// divides kChunk); the step seed is the batch step kernel's.
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS, PairOcc::min_blocks * kPairThreads / THREADS)
batch_pair_kernel(const T *__restrict__ src, T *__restrict__ dst, const uint2 *__restrict__ node,
                  const int2 *__restrict__ grp, const int32_t *__restrict__ ccase,
                  const int32_t *__restrict__ rowstart, const uint32_t *__restrict__ jbslot,
                  const LinkCoef<float> *__restrict__ links,
                  const BatchCase<float> *__restrict__ cases, const int32_t *__restrict__ active,
                  const int32_t *__restrict__ work, const int64_t *__restrict__ counter,
                  const uint32_t j, const PullGeom *__restrict__ geoms) {
  static_assert(kChunk % (2 * THREADS) == 0, "a CTA stays inside one chunk");
  constexpr uint32_t kPer = kChunk / (2 * THREADS);  // CTAs per chunk
  const int32_t chunk = work[blockIdx.x / kPer];
  const int c = ccase[chunk];
  if (!active[c]) return;
  const BatchCase<float> &bc = cases[c];
  const uint32_t i0 = static_cast<uint32_t>(chunk) * kChunk + (blockIdx.x % kPer) * 2 * THREADS +
                      2 * threadIdx.x - static_cast<uint32_t>(bc.node_off);
  if (i0 >= static_cast<uint32_t>(bc.n_fluid)) return;
  const PullGeom &g = geoms[c];
  const uint32_t seed = step_seed(*counter + j);
  if (i0 + 1u < static_cast<uint32_t>(bc.n_fluid))
    step_pair_pull<T>(src + bc.f_off, dst + bc.f_off, g, links + bc.link_off, bc.k, i0, seed);
  else
    step_node_pull<T, float, false>(src + bc.f_off, dst + bc.f_off, g, links + bc.link_off, bc.k,
                                    i0, seed);
}

// The exact-mass cases of an FP32 batch (moving walls; see collide and
// link_epilogue_pull): one CTA of kChunk threads per node-arena chunk in
// `chunks` (the chunks of those cases); the same register budget per thread
// (64) as the single-case exact kernel.
__global__ void __launch_bounds__(kChunk, 4)
batch_exact_kernel(const float *__restrict__ src, float *__restrict__ dst,
                   const int32_t *__restrict__ ccase, const LinkCoef<float> *__restrict__ links,
                   const BatchCase<float> *__restrict__ cases, const int32_t *__restrict__ active,
                   const int32_t *__restrict__ chunks, const int64_t *__restrict__ counter,
                   const uint32_t j, const PullGeom *__restrict__ geoms) {
  const int32_t ch = chunks[blockIdx.x];
  const int c = ccase[ch];
  if (!active[c]) return;
  const BatchCase<float> &bc = cases[c];
  const uint32_t i = static_cast<uint32_t>(ch) * kChunk + threadIdx.x -
                     static_cast<uint32_t>(bc.node_off);
  if (i >= static_cast<uint32_t>(bc.n_fluid)) return;
  // the case's geometry and constants from device tables (not copied into
  // this thread's local memory to be passed to the out-of-line step)
  step_node_exact(src + bc.f_off, dst + bc.f_off, geoms[c], links + bc.link_off, bc.k, i,
                  step_seed(*counter + j));
}

// One CTA per case: residual of the case (FP64 sums in a fixed order); a
// case whose residual fell below tol, or whose state is no longer finite,
// is retired with the step count at which that happened (negative when
// unstable).  A case with residual_mode 1 takes the interval residual: its
// velocity against the snapshot of the previous check (snap, two values per
// node-arena entry), divided by the K steps since, and the snapshot is
// replaced.  init: only write the snapshots of those cases (the start of
// the first interval), retire nothing.
template <typename T, typename C>
__global__ void __launch_bounds__(kBatchResidualThreads)
batch_residual_kernel(const T *__restrict__ cur, const T *__restrict__ prev,
                      const uint2 *__restrict__ node, const int2 *__restrict__ grp,
                      const int32_t *__restrict__ rowstart,
                      const BatchCase<C> *__restrict__ cases,
                      int32_t *__restrict__ active, double tol, const int64_t *__restrict__ counter,
                      int64_t K, int64_t *__restrict__ steps_done, double *__restrict__ res_out,
                      int32_t *__restrict__ n_active, C *__restrict__ snap, const int init) {
  const int c = blockIdx.x;
  if (!active[c]) return;
  const BatchCase<C> &bc = cases[c];
  const StepConst<C> k = bc.k;
  const bool interval = k.residual_mode == 1 && snap;
  if (init && !interval) return;
  const T *a_base = cur + bc.f_off;
  const T *b_base = prev + bc.f_off;
  C *sn = interval ? snap + 2 * bc.node_off : nullptr;
  NodeMap map;
  map.pull = case_geom(bc, node, grp, rowstart, static_cast<const uint32_t *>(nullptr));
  double num = 0.0, den = 0.0, bad = 0.0;
  {
    for (int64_t i = threadIdx.x; i < bc.n_fluid; i += blockDim.x) {
      uint32_t s[9];
      map.slots(static_cast<uint32_t>(i), static_cast<uint32_t>(k.plane), s);
      C a[9], b[9];
      bool sat = false;
#pragma unroll
      for (int q = 0; q < 9; q++) {
        a[q] = Stor<T>::ld(a_base[s[q]], k.inv_sc);
        b[q] = interval ? C(0) : Stor<T>::ld(b_base[s[q]], k.inv_sc);
        if constexpr (kStochastic<T>)
          sat |= fabsf(Stor<T>::ld_raw(a_base[s[q]])) >= Stor<T>::kMaxRaw ||
                 (!interval && fabsf(Stor<T>::ld_raw(b_base[s[q]])) >= Stor<T>::kMaxRaw);
      }
      C n1, d1, m1;
      if (interval) {
        const C r = C(1) + (((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])) + a[8]);
        const C jx = a[1] - a[3] + (a[5] - a[6]) + (a[8] - a[7]);
        const C jy = a[2] - a[4] + (a[5] + a[6]) - (a[7] + a[8]);
        const C ux = (jx + C(0.5) * r * k.ax) / r, uy = (jy + C(0.5) * r * k.ay) / r;
        const C dx = ux - sn[2 * i], dy = uy - sn[2 * i + 1];
        sn[2 * i] = ux;
        sn[2 * i + 1] = uy;
        n1 = dx * dx + dy * dy;
        d1 = ux * ux + uy * uy;
        m1 = r - C(1);
      } else {
        residual_terms<C>(a, b, k.ax, k.ay, n1, d1, m1);
      }
      // a saturated 16-bit value counts as non-finite
      if (sat || !(isfinite(n1) && isfinite(d1) && isfinite(m1))) {
        bad += 1.0;
        continue;
      }
      num += static_cast<double>(n1);
      den += static_cast<double>(d1);
    }
  }
  if (init) return;
  __shared__ double sh[kBatchResidualThreads / 32][3];
  num = warp_sum(num);
  den = warp_sum(den);
  bad = warp_sum(bad);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[w][0] = num;
    sh[w][1] = den;
    sh[w][2] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < kBatchResidualThreads / 32; i++)
      for (int q = 0; q < 3; q++) s[q] += sh[i][q];
    const double res = (s[1] > 0.0 ? sqrt(s[0] / s[1]) : (s[0] > 0.0 ? INFINITY : 0.0)) /
                       (interval ? static_cast<double>(K) : 1.0);
    res_out[c] = res;
    const int64_t now = *counter + K;
    if (s[2] > 0.0 || isnan(res)) {
      active[c] = 0;
      steps_done[c] = -now;
      atomicSub(n_active, 1);
    } else if (res < tol) {
      active[c] = 0;
      steps_done[c] = now;
      atomicSub(n_active, 1);
    }
  }
}

__global__ void batch_advance(int64_t *counter, int64_t K) { *counter += K; }

template <typename T, typename C, int THREADS>
cudaError_t launch_batch_step(const T *src, T *dst, const uint2 *node, const int2 *grp,
                              const int32_t *ccase, const int32_t *rowstart,
                              const uint32_t *jbslot, const void *links, const void *cases,
                              const int32_t *active, const int32_t *work, int32_t n_work,
                              uint32_t pf_dist, const int64_t *counter, uint32_t j,
                              const PullGeom *geoms, const int32_t *exact_chunks,
                              int32_t n_exact_chunks, cudaStream_t s) {
  if constexpr (kStochastic<T>) {
    if constexpr (THREADS <= kChunk / 2) {
      if (n_work > 0)
        batch_pair_kernel<T, THREADS><<<static_cast<unsigned>(n_work) * (kChunk / (2 * THREADS)),
                                        THREADS, 0, s>>>(
            src, dst, node, grp, ccase, rowstart, jbslot,
            static_cast<const LinkCoef<float> *>(links),
            static_cast<const BatchCase<float> *>(cases), active, work, counter, j, geoms);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;  // 16-bit batches use widths 64 and 128
    }
  }
  const int64_t blocks = static_cast<int64_t>(n_work) * (kChunk / THREADS);
  if (blocks > 0)
    batch_step_kernel<T, C, THREADS><<<static_cast<unsigned>(blocks), THREADS, 0, s>>>(
        src, dst, node, grp, ccase, rowstart, jbslot, static_cast<const LinkCoef<C> *>(links),
        static_cast<const BatchCase<C> *>(cases), active, work, static_cast<uint32_t>(blocks),
        pf_dist, counter, j, geoms);
  if constexpr (std::is_same<T, float>::value) {
    if (n_exact_chunks > 0) {
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      batch_exact_kernel<<<static_cast<unsigned>(n_exact_chunks), kChunk, 0, s>>>(
          src, dst, ccase, static_cast<const LinkCoef<float> *>(links),
          static_cast<const BatchCase<float> *>(cases), active, exact_chunks, counter, j, geoms);
    }
  }
  return cudaGetLastError();
}

// CTAs of batch_step_kernel<T, C, THREADS> resident at once on the current device.
template <typename T, typename C, int THREADS>
int batch_resident_ctas() {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  cudaError_t e;
  if constexpr (kStochastic<T> && THREADS <= kChunk / 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_pair_kernel<T, THREADS>, THREADS,
                                                      0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_step_kernel<T, C, THREADS>,
                                                      THREADS, 0);
  return e == cudaSuccess ? sms * per : 0;
}

// Autotuner cache: CTA width and prefetch distance per (precision, size
// class = floor(log2 nodes)).
struct TuneChoice {
  int threads;
  uint32_t pf_dist;
};
std::mutex g_tune_mu;
std::map<std::pair<int, int>, TuneChoice> g_tune_cache;

}  // namespace
}  // namespace lbm

struct lbm_batch {
  int precision = LBM_FP32;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_cases = 0;
  std::vector<int32_t> nx, ny;
  std::vector<int64_t> f_off, node_off, grp_off, row_off, idx_off, plane, n_fluid;
  std::vector<double> ax, ay, scale, tau_s;
  std::vector<int32_t> px, py;
  void *f[2] = {nullptr, nullptr};
  uint2 *node = nullptr;
  int2 *grp = nullptr;
  int32_t *ccase = nullptr;  // per kChunk node-arena entries: their case
  int64_t arena_nodes = 0;   // node-arena entries (cases padded to kChunk)
  int32_t *rowstart = nullptr;
  uint32_t *jbslot = nullptr;
  uint16_t *ldesc = nullptr;  // per link: (x mod 64) << 4 | j (lbm::link_descriptors)
  int32_t *index = nullptr;
  void *links = nullptr;
  void *cases = nullptr;
  // FP32 cases with moving walls: FP64 link records and per-link carry
  // (the exact-mass variant), over the whole link arena; null if no case
  // needs them
  lbm::LinkCoefDF *links64 = nullptr;
  float *carry = nullptr;   // per link of the link arena, then per node-arena entry
  float *carry0 = nullptr;  // = carry + max(1, n_links_total)
  int64_t n_links_total = 0;
  int32_t *exact_chunks = nullptr;  // node-arena chunks of the active exact-mass cases
  int32_t n_exact_chunks = 0;
  lbm::PullGeom *geoms = nullptr;   // per case, its pull geometry inside the arenas
  // Work lists: the step kernels run only the node-arena chunks listed
  // (work: the other active cases'), so retired cases cost no CTAs.  Per
  // case its first chunk and chunk count; the lists are rebuilt (and the
  // graph captured again) each time the active cases halve.
  std::vector<int32_t> chunk_first, chunk_count;
  std::vector<char> case_exact;
  int32_t *work = nullptr;
  int32_t n_work = 0;
  int32_t n_listed = 0;  // active cases when the lists were last built
  void *snap = nullptr;  // interval-residual snapshots (2 values per node-arena entry), or null
  int threads = 0;
  uint32_t pf_dist = 0;  // L2 prefetch distance of the step kernel (CTAs), for `threads`
  int32_t *active = nullptr;
  int64_t *steps_done = nullptr;
  double *res = nullptr;
  int64_t *counter = nullptr;
  int32_t *n_active = nullptr;
  int32_t *h_n_active = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_K = 0;
  double graph_tol = 0.0;
  int cur = 0;
  int64_t steps = 0;
  int64_t total_nodes = 0, total_fluid = 0;
  int64_t arena_elems = 0;  // elements of one lattice arena (all cases' planes and link tails)
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

size_t elem_size_b(int precision) {
  return precision == LBM_FP64 ? 8 : (precision == LBM_FP32 ? 4 : 2);
}

template <typename F>
cudaError_t dispatch_b(int precision, F &&f) {
  switch (precision) {
    case LBM_FP64: return f(static_cast<double *>(nullptr), static_cast<double *>(nullptr));
    case LBM_FP32: return f(static_cast<float *>(nullptr), static_cast<float *>(nullptr));
    case LBM_BF16: return f(static_cast<__nv_bfloat16 *>(nullptr), static_cast<float *>(nullptr));
    default: return f(static_cast<__half *>(nullptr), static_cast<float *>(nullptr));
  }
}

lbm::NodeMap case_map(const lbm_batch_t *b, int c) {
  lbm::NodeMap m;
  m.index = b->index + b->idx_off[c];
  m.nx = b->nx[c];
  m.ny = b->ny[c];
  m.pull.node = b->node + b->node_off[c];
  m.pull.grp = b->grp + b->grp_off[c];
  m.pull.rowstart = b->rowstart + b->row_off[c];
  m.pull.ny = b->ny[c];
  m.pull.periodic_y = b->py[c];
  m.pull.plane = static_cast<uint32_t>(b->plane[c]);
  m.pull.n_fluid = static_cast<uint32_t>(b->n_fluid[c]);
  return m;
}

// One step launch; j = the step's position after the last advance of the
// device step counter (seeds the random bits).
cudaError_t step_once(lbm_batch_t *b, int threads, uint32_t pf_dist, int src, uint32_t j) {
  const int dst = 1 - src;
  return dispatch_b(b->precision, [&](auto tT, auto tC) {
    using T = std::remove_pointer_t<decltype(tT)>;
    using C = std::remove_pointer_t<decltype(tC)>;
    auto go = [&](auto kernel_threads) {
      constexpr int TH = decltype(kernel_threads)::value;
      return lbm::launch_batch_step<T, C, TH>(
          static_cast<const T *>(b->f[src]), static_cast<T *>(b->f[dst]), b->node, b->grp,
          b->ccase, b->rowstart, b->jbslot, b->links, b->cases, b->active, b->work, b->n_work,
          pf_dist, b->counter, j, b->geoms, b->exact_chunks, b->n_exact_chunks, b->stream);
    };
    if (threads == 64) return go(std::integral_constant<int, 64>());
    if (threads == 128) return go(std::integral_constant<int, 128>());
    return go(std::integral_constant<int, 256>());
  });
}

// Rebuild the work lists from the active flags (host copy; all cases when
// null) and upload them.
cudaError_t build_lists(lbm_batch_t *b, const int32_t *active_host) {
  std::vector<int32_t> w, x;
  int32_t n_act = 0;
  for (int c = 0; c < b->n_cases; c++) {
    if (active_host && !active_host[c]) continue;
    n_act++;
    std::vector<int32_t> &dst = b->case_exact[c] ? x : w;
    for (int32_t q = 0; q < b->chunk_count[c]; q++) dst.push_back(b->chunk_first[c] + q);
  }
  cudaError_t e = cudaSuccess;
  if (!w.empty())
    e = cudaMemcpyAsync(b->work, w.data(), w.size() * 4, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && !x.empty())
    e = cudaMemcpyAsync(b->exact_chunks, x.data(), x.size() * 4, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  b->n_work = static_cast<int32_t>(w.size());
  b->n_exact_chunks = static_cast<int32_t>(x.size());
  b->n_listed = n_act;
  // a captured graph holds the old lists' grid sizes
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return e;
}

// Snapshots of the interval residual from the current state (lattice 0,
// every active case with residual_mode 1): the start of an interval.
cudaError_t init_snapshots(lbm_batch_t *b) {
  if (!b->snap) return cudaSuccess;
  return dispatch_b(b->precision, [&](auto tT, auto tC) {
    using T = std::remove_pointer_t<decltype(tT)>;
    using C = std::remove_pointer_t<decltype(tC)>;
    lbm::batch_residual_kernel<T, C><<<b->n_cases, lbm::kBatchResidualThreads, 0, b->stream>>>(
        static_cast<const T *>(b->f[0]), static_cast<const T *>(b->f[1]), b->node, b->grp,
        b->rowstart, static_cast<const lbm::BatchCase<C> *>(b->cases), b->active, 0.0, b->counter,
        1, b->steps_done, b->res, b->n_active, static_cast<C *>(b->snap), 1);
    return cudaGetLastError();
  });
}

int bfail(lbm_batch_t *b, int code, const std::string &m) {
  if (b) b->err = m;
  return code;
}

void batch_release(lbm_batch_t *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void *p : {b->f[0], b->f[1], static_cast<void *>(b->node), static_cast<void *>(b->grp),
                  static_cast<void *>(b->jbslot), static_cast<void *>(b->ldesc), static_cast<void *>(b->rowstart), static_cast<void *>(b->index), b->links, b->cases, static_cast<void *>(b->ccase), static_cast<void *>(b->active),
                  static_cast<void *>(b->steps_done), static_cast<void *>(b->res),
                  static_cast<void *>(b->counter), static_cast<void *>(b->n_active),
                  static_cast<void *>(b->links64), static_cast<void *>(b->carry),
                  static_cast<void *>(b->exact_chunks), static_cast<void *>(b->geoms), b->snap,
                  static_cast<void *>(b->work)})
    if (p) cudaFree(p);
  if (b->h_n_active) cudaFreeHost(b->h_n_active);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

// CTAs of the step kernel resident at once for this precision and width.
int resident_ctas(int precision, int threads) {
  int r = 0;
  dispatch_b(precision, [&](auto tT, auto tC) {
    using T = std::remove_pointer_t<decltype(tT)>;
    using C = std::remove_pointer_t<decltype(tC)>;
    if (threads == 64) r = lbm::batch_resident_ctas<T, C, 64>();
    else if (threads == 128) r = lbm::batch_resident_ctas<T, C, 128>();
    else r = lbm::batch_resident_ctas<T, C, 256>();
    return cudaSuccess;
  });
  return r;
}

// Autotuner: times each candidate (CTA width; L2 prefetch off or half the
// resident CTAs ahead) for a few steps of the batch itself (from rest; the
// caller resets the state afterwards) and keeps the fastest, cached per
// (precision, size class).
lbm::TuneChoice autotune(lbm_batch_t *b) {
  const int size_class = static_cast<int>(std::log2(static_cast<double>(b->total_nodes) + 1.0));
  {
    std::lock_guard<std::mutex> lock(lbm::g_tune_mu);
    auto it = lbm::g_tune_cache.find({b->precision, size_class});
    if (it != lbm::g_tune_cache.end()) return it->second;
  }
  // CTA widths (threads); a 16-bit CTA runs two nodes per thread, so its
  // widths stop at half a chunk
  const bool pairs = b->precision == LBM_BF16 || b->precision == LBM_FP16;
  const std::vector<int> cand = pairs ? std::vector<int>{64, 128} : std::vector<int>{64, 128, 256};
  // every candidate timed over 12 steps (after 2 untimed ones), in two
  // passes over the list; a candidate's time is its faster pass
  std::vector<lbm::TuneChoice> opts;
  for (int th : cand) {
    const uint32_t half = static_cast<uint32_t>(resident_ctas(b->precision, th) / 2);
    opts.push_back(lbm::TuneChoice{th, 0u});
    opts.push_back(lbm::TuneChoice{th, half});
  }
  std::vector<float> t_ms(opts.size(), std::numeric_limits<float>::infinity());
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int pass = 0; pass < 2; pass++)
    for (size_t o = 0; o < opts.size(); o++) {
      const int th = opts[o].threads;
      const uint32_t pf = opts[o].pf_dist;
      for (int w = 0; w < 2; w++) step_once(b, th, pf, w & 1, static_cast<uint32_t>(w));
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < 12; r++) step_once(b, th, pf, r & 1, static_cast<uint32_t>(r));
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t_ms[o] = std::min(t_ms[o], ms);
    }
  lbm::TuneChoice best{128, 0};
  float best_ms = std::numeric_limits<float>::infinity();
  for (size_t o = 0; o < opts.size(); o++)
    if (t_ms[o] < best_ms) {
      best_ms = t_ms[o];
      best = opts[o];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(lbm::g_tune_mu);
  lbm::g_tune_cache[{b->precision, size_class}] = best;
  return best;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_case_t *cases, int32_t n_cases, int32_t precision, void *stream,
                     lbm_batch_t **out) {
  g_batch_error.clear();
  if (!out || !cases || n_cases < 1) {
    g_batch_error = "null argument or empty batch";
    return LBM_EINVAL;
  }
  *out = nullptr;
  if (precision < LBM_FP64 || precision > LBM_FP16) {
    g_batch_error = "precision must be LBM_FP64, LBM_FP32, LBM_BF16 or LBM_FP16";
    return LBM_EINVAL;
  }
  std::vector<lbm::HostCase> hc(static_cast<size_t>(n_cases));
  std::vector<lbm::CompactCase> cc(static_cast<size_t>(n_cases));
  int64_t nodes = 0, elems = 0, groups = 0, links = 0, rows = 0, dense = 0;
  for (int c = 0; c < n_cases; c++) {
    lbm_params_t p = cases[c].params;
    p.precision = precision;
    std::string msg;
    const lbm_case_t &cs = cases[c];
    int rc = lbm::build_host_case(&cs.dom, cs.solid, cs.n_links, cs.link_x, cs.link_y,
                                  cs.link_dir, cs.link_q, cs.link_ubx, cs.link_uby, cs.Kn, &p,
                                  &hc[c], &msg);
    if (rc != LBM_OK) {
      g_batch_error = "case " + std::to_string(c) + ": " + msg;
      return rc;
    }
    const std::string cerr = lbm::build_compact(hc[c], &cc[c]);
    if (!cerr.empty()) {
      g_batch_error = "case " + std::to_string(c) + ": " + cerr;
      return LBM_EINVAL;
    }
    nodes += (std::max<int64_t>(cc[c].n_fluid, 1) + lbm::kChunk - 1) / lbm::kChunk * lbm::kChunk;
    elems += 9 * cc[c].plane + (hc[c].n_links + 31) / 32 * 32;
    groups += static_cast<int64_t>(cc[c].grp.size());
    links += hc[c].n_links;
    rows += hc[c].ny + 1;
    dense += static_cast<int64_t>(hc[c].nx) * hc[c].ny;
  }
  if (elems >= (int64_t(1) << 40) || links >= (int64_t(1) << 31)) {
    g_batch_error = "batch too large";
    return LBM_EINVAL;
  }
  lbm_batch_t *b = new (std::nothrow) lbm_batch_t();
  if (!b) {
    g_batch_error = "host allocation failed";
    return LBM_ENOMEM;
  }
  b->precision = precision;
  b->n_cases = n_cases;
  b->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!b->stream) {  // graphs need a stream that can be captured
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  const size_t es = elem_size_b(precision);
  const size_t ces = precision == LBM_FP64 ? 8 : 4;
  std::vector<uint2> node(static_cast<size_t>(nodes), uint2{0u, 0u});
  std::vector<int2> grp(static_cast<size_t>(std::max<int64_t>(1, groups)), int2{0, 0});
  std::vector<int32_t> ccase(static_cast<size_t>(std::max<int64_t>(1, nodes / lbm::kChunk)), 0);
  std::vector<uint32_t> jbs(static_cast<size_t>(std::max<int64_t>(1, links)), 0u);
  std::vector<uint16_t> lds(static_cast<size_t>(std::max<int64_t>(1, links)), 0u);
  std::vector<int32_t> rowstart(static_cast<size_t>(rows), 0), index(static_cast<size_t>(dense), -1);
  std::vector<unsigned char> lhost(std::max<int64_t>(1, links) * 4 * ces, 0);
  std::vector<double> l64;  // FP64 link records (filled if some case runs the exact variant)
  bool any_exact = false;
  for (int c = 0; c < n_cases; c++) any_exact |= lbm::exact_mass(hc[c]);
  if (any_exact) l64.assign(static_cast<size_t>(std::max<int64_t>(1, links)) * 4, 0.0);
  std::vector<unsigned char> chost;
  std::vector<int32_t> xchunks;
  bool any_interval = false;
  for (int c = 0; c < n_cases; c++) any_interval |= hc[c].params.residual_mode == 1;
  int64_t noff = 0, foff = 0, goff = 0, loff = 0, roff = 0, ioff = 0;
  for (int c = 0; c < n_cases; c++) {
    const lbm::HostCase &h = hc[c];
    lbm::CompactCase &k = cc[c];
    b->nx.push_back(h.nx);
    b->ny.push_back(h.ny);
    b->f_off.push_back(foff);
    b->node_off.push_back(noff);
    b->grp_off.push_back(goff);
    b->row_off.push_back(roff);
    b->idx_off.push_back(ioff);
    b->plane.push_back(k.plane);
    b->n_fluid.push_back(h.n_fluid);
    b->ax.push_back(h.ax);
    b->ay.push_back(h.ay);
    b->scale.push_back(h.scale);
    b->tau_s.push_back(h.cp.tau_s);
    b->px.push_back(h.px);
    b->py.push_back(h.py);
    b->total_nodes += static_cast<int64_t>(h.nx) * h.ny;
    b->total_fluid += h.n_fluid;
    std::copy(k.node.begin(), k.node.end(), node.begin() + noff);
    std::copy(k.grp.begin(), k.grp.end(), grp.begin() + goff);
    // (at least one chunk: the case's node words, `plane` of them, fit)
    const int64_t padded =
        (std::max<int64_t>(k.n_fluid, 1) + lbm::kChunk - 1) / lbm::kChunk * lbm::kChunk;
    std::fill(ccase.begin() + noff / lbm::kChunk, ccase.begin() + (noff + padded) / lbm::kChunk, c);
    const std::vector<uint32_t> kj = lbm::link_jb_slots(k, h.ny, h.py, h.n_links);
    std::copy(kj.begin(), kj.end(), jbs.begin() + loff);
    const std::vector<uint16_t> kd = lbm::link_descriptors(k, h.n_links);
    std::copy(kd.begin(), kd.end(), lds.begin() + loff);
    std::copy(k.rowstart.begin(), k.rowstart.end(), rowstart.begin() + roff);
    std::copy(k.index.begin(), k.index.end(), index.begin() + ioff);
    b->chunk_first.push_back(static_cast<int32_t>(noff / lbm::kChunk));
    b->chunk_count.push_back(static_cast<int32_t>(padded / lbm::kChunk));
    b->case_exact.push_back(lbm::exact_mass(h) ? 1 : 0);
    if (lbm::exact_mass(h)) {
      std::copy(h.coef.begin(), h.coef.begin() + 4 * h.n_links, l64.begin() + 4 * loff);
      for (int64_t q = noff / lbm::kChunk; q < (noff + padded) / lbm::kChunk; q++)
        xchunks.push_back(static_cast<int32_t>(q));
    }
    for (int64_t q = 0; q < h.n_links; q++) {
      const double *cf = &h.coef[4 * q];
      if (ces == 8) {
        std::memcpy(&lhost[(loff + q) * 32], cf, 32);
      } else {
        float f4[4];
        for (int j = 0; j < 4; j++) f4[j] = static_cast<float>(cf[j]);
        std::memcpy(&lhost[(loff + q) * 16], f4, 16);
      }
    }
    // descriptor
    auto put = [&](auto tag) {
      using C = decltype(tag);
      lbm::BatchCase<C> d;
      d.k = lbm::make_step_const<C>(h.cp, h.nx, h.ny, 0, k.plane, h.n_fluid, h.px, h.py, h.ax,
                                    h.ay, h.params.diffuse_mode, h.scale);
      d.k.exact = lbm::exact_mass(h) ? 1 : 0;
      d.k.residual_mode = h.params.residual_mode;
      d.f_off = foff;
      d.node_off = noff;
      d.grp_off = goff;
      d.row_off = roff;
      d.idx_off = ioff;
      d.link_off = loff;
      d.n_fluid = h.n_fluid;
      const unsigned char *p = reinterpret_cast<const unsigned char *>(&d);
      chost.insert(chost.end(), p, p + sizeof(d));
    };
    if (precision == LBM_FP64)
      put(double());
    else
      put(float());
    noff += padded;
    foff += 9 * k.plane + (h.n_links + 31) / 32 * 32;
    goff += static_cast<int64_t>(k.grp.size());
    loff += h.n_links;
    roff += h.ny + 1;
    ioff += static_cast<int64_t>(h.nx) * h.ny;
  }
  hc.clear();
  cc.clear();
  b->arena_elems = elems;
  auto alloc = [&](void **p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)); };
  const size_t fbytes = static_cast<size_t>(elems) * es;
  if (e == cudaSuccess) e = alloc(&b->f[0], fbytes);
  if (e == cudaSuccess) e = alloc(&b->f[1], fbytes);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->node), node.size() * sizeof(uint2));
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->grp), grp.size() * sizeof(int2));
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->ccase), ccase.size() * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->jbslot), jbs.size() * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->ldesc), lds.size() * 2);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->rowstart), rowstart.size() * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->index), index.size() * 4);
  if (e == cudaSuccess) e = alloc(&b->links, lhost.size());
  b->n_links_total = links;
  if (any_exact) {
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->links64), l64.size() * 8);
    if (e == cudaSuccess)
      e = alloc(reinterpret_cast<void **>(&b->carry), (l64.size() / 4 + nodes) * 4);
    if (e == cudaSuccess) b->carry0 = b->carry + l64.size() / 4;
    if (e == cudaSuccess) e = cudaMemset(b->carry, 0, (l64.size() / 4 + nodes) * 4);
    if (e == cudaSuccess) {
      std::vector<lbm::LinkCoefDF> ldf(l64.size() / 4);
      for (size_t l = 0; l < ldf.size(); l++) ldf[l] = lbm::link_coef_df(&l64[4 * l]);
      e = cudaMemcpy(b->links64, ldf.data(), ldf.size() * sizeof(lbm::LinkCoefDF),
                     cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->exact_chunks), xchunks.size() * 4);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->exact_chunks, xchunks.data(), xchunks.size() * 4, cudaMemcpyHostToDevice);
    b->n_exact_chunks = static_cast<int32_t>(xchunks.size());
  }
  if (e == cudaSuccess) e = alloc(&b->cases, chost.size());
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->active), n_cases * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->steps_done), n_cases * 8);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->res), n_cases * 8);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->counter), 8);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->n_active), 4);
  if (e == cudaSuccess && any_interval)
    e = alloc(&b->snap, static_cast<size_t>(nodes) * 2 * (precision == LBM_FP64 ? 8 : 4));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&b->h_n_active), 4);
  auto up = [&](void *dst, const void *src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(b->node, node.data(), node.size() * sizeof(uint2));
  up(b->grp, grp.data(), grp.size() * sizeof(int2));
  up(b->ccase, ccase.data(), ccase.size() * 4);
  b->arena_nodes = nodes;
  if (e == cudaSuccess)
    e = alloc(reinterpret_cast<void **>(&b->work),
              static_cast<size_t>(std::max<int64_t>(1, nodes / lbm::kChunk)) * 4);
  if (e == cudaSuccess) e = build_lists(b, nullptr);
  up(b->jbslot, jbs.data(), jbs.size() * 4);
  up(b->ldesc, lds.data(), lds.size() * 2);
  if (e == cudaSuccess) {
    // every case's pull geometry inside the arenas (read by the step kernels)
    std::vector<lbm::PullGeom> gs(static_cast<size_t>(n_cases));
    for (int32_t c = 0; c < n_cases; c++) {
      if (precision == LBM_FP64)
        gs[c] = lbm::case_geom(reinterpret_cast<const lbm::BatchCase<double> *>(chost.data())[c],
                               b->node, b->grp, b->rowstart, b->jbslot, b->links64, b->carry,
                               b->carry0, b->ldesc);
      else
        gs[c] = lbm::case_geom(reinterpret_cast<const lbm::BatchCase<float> *>(chost.data())[c],
                               b->node, b->grp, b->rowstart, b->jbslot, b->links64, b->carry,
                               b->carry0, b->ldesc);
    }
    e = alloc(reinterpret_cast<void **>(&b->geoms), gs.size() * sizeof(lbm::PullGeom));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->geoms, gs.data(), gs.size() * sizeof(lbm::PullGeom), cudaMemcpyHostToDevice);
  }
  up(b->rowstart, rowstart.data(), rowstart.size() * 4);
  up(b->index, index.data(), index.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(b->links, lhost.data(), lhost.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->cases, chost.data(), chost.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    // autotune from rest, then reset the state to rest
    std::vector<int32_t> ones(n_cases, 1);
    e = cudaMemcpy(b->active, ones.data(), n_cases * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->f[0], 0, fbytes);
    if (e == cudaSuccess) e = cudaMemset(b->f[1], 0, fbytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
      const lbm::TuneChoice t = autotune(b);
      b->threads = t.threads;
      b->pf_dist = t.pf_dist;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = lbm_batch_reset(b) == LBM_OK ? cudaSuccess : cudaErrorUnknown;
  if (e != cudaSuccess) {
    g_batch_error = std::string("device setup: ") + cudaGetErrorString(e);
    const int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    batch_release(b);
    return code;
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_reset(lbm_batch_t *b) {
  if (!b) return LBM_EINVAL;
  const size_t fbytes = static_cast<size_t>(b->arena_elems) * elem_size_b(b->precision);
  std::vector<int32_t> ones(b->n_cases, 1);
  std::vector<int64_t> zeros(b->n_cases, 0);
  const int32_t n = b->n_cases;
  const int64_t zero = 0;
  cudaError_t e = cudaMemsetAsync(b->f[0], 0, fbytes, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->f[1], 0, fbytes, b->stream);
  if (e == cudaSuccess && b->carry)
    e = cudaMemsetAsync(b->carry, 0,
                        static_cast<size_t>(std::max<int64_t>(1, b->n_links_total) + b->arena_nodes) * 4,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->active, ones.data(), n * 4, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->steps_done, zeros.data(), n * 8, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->counter, &zero, 8, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->n_active, &n, 4, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = init_snapshots(b);
  if (e == cudaSuccess && b->n_listed != b->n_cases) e = build_lists(b, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("lbm_batch_reset: ") + cudaGetErrorString(e));
  b->cur = 0;
  b->steps = 0;
  return LBM_OK;
}

int lbm_batch_run_to(lbm_batch_t *b, double tol, int64_t max_steps, int32_t check_every,
                     int64_t *steps_per_case, double *residual_per_case, int64_t *steps_total) {
  if (!b) return LBM_EINVAL;
  if (check_every < 2 || (check_every & 1))
    return bfail(b, LBM_EINVAL, "check_every must be an even number >= 2");
  if (max_steps < 0) return bfail(b, LBM_EINVAL, "negative max_steps");
  if (b->cur != 0) return bfail(b, LBM_EINVAL, "batch state is mid-graph; call lbm_batch_reset");
  cudaError_t e = cudaSuccess;
  // K steps, the batched reduction and the counter advance as one graph,
  // captured for the current work lists
  auto capture = [&]() -> cudaError_t {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t ec = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    for (int s = 0; s < check_every && ec == cudaSuccess; s++)
      ec = step_once(b, b->threads, b->pf_dist, s & 1, static_cast<uint32_t>(s));
    if (ec == cudaSuccess)
      ec = dispatch_b(b->precision, [&](auto tT, auto tC) {
        using T = std::remove_pointer_t<decltype(tT)>;
        using C = std::remove_pointer_t<decltype(tC)>;
        lbm::batch_residual_kernel<T, C><<<b->n_cases, lbm::kBatchResidualThreads, 0, b->stream>>>(
            static_cast<const T *>(b->f[0]), static_cast<const T *>(b->f[1]), b->node, b->grp,
            b->rowstart, static_cast<const lbm::BatchCase<C> *>(b->cases), b->active, tol,
            b->counter, check_every, b->steps_done, b->res, b->n_active, static_cast<C *>(b->snap),
            0);
        return cudaGetLastError();
      });
    if (ec == cudaSuccess) {
      lbm::batch_advance<<<1, 1, 0, b->stream>>>(b->counter, check_every);
      ec = cudaGetLastError();
    }
    if (ec == cudaSuccess)
      ec = cudaMemcpyAsync(b->h_n_active, b->n_active, 4, cudaMemcpyDeviceToHost, b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (ec == cudaSuccess) ec = e2;
    if (ec == cudaSuccess) ec = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ec != cudaSuccess) {
      b->graph = nullptr;
      return ec;
    }
    b->graph_K = check_every;
    b->graph_tol = tol;
    return cudaSuccess;
  };
  if (!b->graph || b->graph_K != check_every || b->graph_tol != tol) {
    e = capture();
    if (e != cudaSuccess)
      return bfail(b, LBM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  int64_t done = 0;
  *b->h_n_active = b->n_cases;
  std::vector<int32_t> act(static_cast<size_t>(b->n_cases));
  while (done < max_steps) {
    e = cudaGraphLaunch(b->graph, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    done += check_every;
    b->steps += check_every;
    if (*b->h_n_active <= 0) break;
    // half of the listed cases retired: list only the active ones' chunks
    if (*b->h_n_active * 2 <= b->n_listed && done < max_steps) {
      e = cudaMemcpy(act.data(), b->active, act.size() * 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = build_lists(b, act.data());
      if (e == cudaSuccess) e = capture();
      if (e != cudaSuccess)
        return bfail(b, LBM_ECUDA, std::string("work lists: ") + cudaGetErrorString(e));
    }
  }
  if (steps_per_case)
    e = cudaMemcpy(steps_per_case, b->steps_done, b->n_cases * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && residual_per_case)
    e = cudaMemcpy(residual_per_case, b->res, b->n_cases * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, cudaGetErrorString(e));
  if (steps_total) *steps_total = b->steps;
  return LBM_OK;
}

int lbm_batch_fields(lbm_batch_t *b, int32_t c, double *rho, double *ux, double *uy) {
  if (!b) return LBM_EINVAL;
  if (c < 0 || c >= b->n_cases) return bfail(b, LBM_EINVAL, "case index out of range");
  const int64_t n = static_cast<int64_t>(b->nx[c]) * b->ny[c];
  double *d = nullptr;
  cudaError_t e = cudaMalloc(&d, 3 * n * sizeof(double));
  if (e != cudaSuccess) return bfail(b, LBM_ENOMEM, cudaGetErrorString(e));
  const int64_t plane = b->plane[c];
  e = dispatch_b(b->precision, [&](auto tT, auto tC) {
    using T = std::remove_pointer_t<decltype(tT)>;
    return lbm::launch_fields<T>(static_cast<const T *>(b->f[b->cur]) + b->f_off[c], case_map(b, c),
                                 plane, b->ax[c], b->ay[c], b->scale[c], d, d + n, d + 2 * n,
                                 b->stream);
  });
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess && rho) e = cudaMemcpy(rho, d, n * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ux) e = cudaMemcpy(ux, d + n, n * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && uy) e = cudaMemcpy(uy, d + 2 * n, n * 8, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_set_fields(lbm_batch_t *b, int32_t c, const double *rho, const double *ux,
                         const double *uy) {
  if (!b || !rho || !ux || !uy) return b ? bfail(b, LBM_EINVAL, "null field") : LBM_EINVAL;
  if (c < 0 || c >= b->n_cases) return bfail(b, LBM_EINVAL, "case index out of range");
  if (b->cur != 0) return bfail(b, LBM_EINVAL, "batch state is mid-graph; call lbm_batch_reset");
  const int64_t n = static_cast<int64_t>(b->nx[c]) * b->ny[c];
  double *d = nullptr;
  cudaError_t e = cudaMalloc(&d, 3 * n * sizeof(double));
  if (e != cudaSuccess) return bfail(b, LBM_ENOMEM, cudaGetErrorString(e));
  e = cudaMemcpy(d, rho, n * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + n, ux, n * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + 2 * n, uy, n * 8, cudaMemcpyHostToDevice);
  const int64_t plane = b->plane[c];
  if (e == cudaSuccess)
    e = dispatch_b(b->precision, [&](auto tT, auto tC) {
      using T = std::remove_pointer_t<decltype(tT)>;
      return lbm::launch_set_fields<T>(d, d + n, d + 2 * n, case_map(b, c), plane, b->px[c],
                                       b->py[c], b->ax[c], b->ay[c], b->tau_s[c], b->scale[c],
                                       static_cast<T *>(b->f[0]) + b->f_off[c],
                                       static_cast<T *>(b->f[1]) + b->f_off[c], b->stream);
    });
  if (e == cudaSuccess) e = init_snapshots(b);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(d);
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_info(const lbm_batch_t *b, int64_t *total_nodes, int64_t *total_fluid,
                   int32_t *cta_threads, int32_t *n_ctas) {
  if (!b) return LBM_EINVAL;
  if (total_nodes) *total_nodes = b->total_nodes;
  if (total_fluid) *total_fluid = b->total_fluid;
  if (cta_threads) *cta_threads = b->threads;
  const bool pairs = b->precision == LBM_BF16 || b->precision == LBM_FP16;
  if (n_ctas) *n_ctas = static_cast<int32_t>(b->arena_nodes / (b->threads * (pairs ? 2 : 1)));
  return LBM_OK;
}

int lbm_batch_set_launch(lbm_batch_t *b, int32_t cta_threads, int32_t l2_prefetch) {
  if (!b) return LBM_EINVAL;
  const bool pairs = b->precision == LBM_BF16 || b->precision == LBM_FP16;
  const bool ok_th = cta_threads == 64 || cta_threads == 128 || (!pairs && cta_threads == 256);
  if (!ok_th) return bfail(b, LBM_EINVAL, "cta_threads must be 64, 128 or (FP32 / FP64) 256");
  if (l2_prefetch != 0 && l2_prefetch != 1) return bfail(b, LBM_EINVAL, "l2_prefetch must be 0 or 1");
  if (b->cur != 0) return bfail(b, LBM_EINVAL, "batch state is mid-graph; call lbm_batch_reset");
  b->threads = cta_threads;
  b->pf_dist = l2_prefetch ? static_cast<uint32_t>(resident_ctas(b->precision, cta_threads) / 2) : 0u;
  if (b->graph) {  // the captured graph holds the old launch shape
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch_t *b) { batch_release(b); }

const char *lbm_batch_last_error(const lbm_batch_t *b) {
  return b ? b->err.c_str() : g_batch_error.c_str();
}

}  // extern "C"
