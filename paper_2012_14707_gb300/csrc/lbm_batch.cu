// Batched solver of liblbm.so (lbm_batch_*): many independent cases of
// different sizes, geometries and parameters advanced together.
//
// All cases live in one device arena (each case's compacted lattice: two
// lattices of its nine deviation planes over its fluid nodes, node words,
// neighbour indices, link bases and link coefficients) and share one tile
// list: a tile is a run of fluid nodes of one row of one case.  A time step is one
// launch over all tiles; a CTA looks up its case's constants in a
// descriptor table and runs the same per-node update as the single-case
// kernel (so a case in a batch follows exactly the arithmetic of the case
// run alone).  Every K steps a batched reduction (one CTA per case, fixed
// order) computes each case's residual and retires converged cases on the
// device; retired cases' tiles return immediately.  K steps plus the
// reduction are captured once in a CUDA graph that the host replays, reading
// back only the number of active cases.  The CTA width is picked by timing
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
// offsets; link bases already global (case link offset added).
template <typename C>
struct BatchCase {
  StepConst<C> k;    // plane = the case's padded fluid-node count
  int64_t f_off;     // element offset of the case's plane 0 in a lattice arena
  int64_t node_off;  // offset of the case in the node-word / link-base arenas
  int64_t row_off;   // offset of the case's rowstart
  int64_t idx_off;   // offset of the case's node map (nx * ny)
  int64_t n_fluid;
};

// A row tile of one case: rows y, compacted indices start .. start + count - 1.
struct Tile {
  int32_t c, y, start, count;
};

constexpr int kBatchResidualThreads = 256;

// Registers bounded like the single-case kernel (the same resident threads
// per SM).
template <typename T, typename C, int THREADS>
__global__ void __launch_bounds__(THREADS, StepOcc<T>::min_blocks * kStepThreads / THREADS)
batch_step_kernel(const T *__restrict__ src, T *__restrict__ dst,
                  const uint2 *__restrict__ node, const int32_t *__restrict__ lbase,
                  const int32_t *__restrict__ rowstart, const LinkCoef<C> *__restrict__ links,
                  const BatchCase<C> *__restrict__ cases, const Tile *__restrict__ tiles,
                  const int32_t *__restrict__ active) {
  const Tile t = tiles[blockIdx.x];
  if (!active[t.c] || static_cast<int>(threadIdx.x) >= t.count) return;
  const BatchCase<C> &bc = cases[t.c];
  const int64_t no = bc.node_off;
  step_node_compact<T, C>(src + bc.f_off, dst + bc.f_off, node + no, lbase + no,
                          rowstart + bc.row_off, links, bc.k,
                          static_cast<uint32_t>(t.start) + threadIdx.x, t.y);
}

// One CTA per case: residual of the case (FP64 sums in a fixed order); a
// case whose residual fell below tol, or whose state is no longer finite,
// is retired with the step count at which that happened (negative when
// unstable).
template <typename T, typename C>
__global__ void __launch_bounds__(kBatchResidualThreads)
batch_residual_kernel(const T *__restrict__ cur, const T *__restrict__ prev,
                      const BatchCase<C> *__restrict__ cases,
                      int32_t *__restrict__ active, double tol, const int64_t *__restrict__ counter,
                      int64_t K, int64_t *__restrict__ steps_done, double *__restrict__ res_out,
                      int32_t *__restrict__ n_active) {
  const int c = blockIdx.x;
  if (!active[c]) return;
  const BatchCase<C> &bc = cases[c];
  const StepConst<C> k = bc.k;
  const T *a_base = cur + bc.f_off;
  const T *b_base = prev + bc.f_off;
  double num = 0.0, den = 0.0, bad = 0.0;
  {
    for (int64_t node = threadIdx.x; node < bc.n_fluid; node += blockDim.x) {
      C a[9], b[9];
#pragma unroll
      for (int i = 0; i < 9; i++) {
        a[i] = Stor<T>::ld(a_base[i * k.plane + node], k.inv_sc);
        b[i] = Stor<T>::ld(b_base[i * k.plane + node], k.inv_sc);
      }
      C n1, d1, m1;
      residual_terms<C>(a, b, k.ax, k.ay, n1, d1, m1);
      if (!(isfinite(n1) && isfinite(d1) && isfinite(m1))) {
        bad += 1.0;
        continue;
      }
      num += static_cast<double>(n1);
      den += static_cast<double>(d1);
    }
  }
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
    const double res = s[1] > 0.0 ? sqrt(s[0] / s[1]) : (s[0] > 0.0 ? INFINITY : 0.0);
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
cudaError_t launch_batch_step(const T *src, T *dst, const uint2 *node, const int32_t *lbase,
                              const int32_t *rowstart,
                              const void *links, const void *cases, const Tile *tiles,
                              int n_tiles, const int32_t *active, cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  batch_step_kernel<T, C, THREADS><<<n_tiles, THREADS, 0, s>>>(
      src, dst, node, lbase, rowstart, static_cast<const LinkCoef<C> *>(links),
      static_cast<const BatchCase<C> *>(cases), tiles, active);
  return cudaGetLastError();
}

// Autotuner cache: CTA width per (precision, size class = floor(log2 nodes)).
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tune_cache;

}  // namespace
}  // namespace lbm

struct lbm_batch {
  int precision = LBM_FP32;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_cases = 0;
  std::vector<int32_t> nx, ny;
  std::vector<int64_t> f_off, node_off, idx_off, plane, n_fluid;
  std::vector<std::vector<int32_t>> rowstart_h;  // per case, for the tile lists
  std::vector<double> ax, ay, scale, tau_s;
  std::vector<int32_t> px, py;
  void *f[2] = {nullptr, nullptr};
  uint2 *node = nullptr;
  int32_t *lbase = nullptr, *rowstart = nullptr;
  int32_t *index = nullptr;
  void *links = nullptr;
  void *cases = nullptr;
  lbm::Tile *tiles = nullptr;
  int n_tiles = 0;
  int threads = 0;
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
  int64_t arena_nodes = 0;  // padded nodes of all cases (one plane each)
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
  return m;
}

// Row tiles of `threads` fluid nodes (the CTA width) over every case.
std::vector<lbm::Tile> make_tiles(const lbm_batch_t *b, int threads) {
  std::vector<lbm::Tile> t;
  for (int c = 0; c < b->n_cases; c++) {
    const std::vector<int32_t> &rs = b->rowstart_h[c];
    for (int y = 0; y < b->ny[c]; y++)
      for (int32_t i = rs[y]; i < rs[y + 1]; i += threads)
        t.push_back(lbm::Tile{c, y, i, std::min<int32_t>(threads, rs[y + 1] - i)});
  }
  return t;
}

cudaError_t step_once(lbm_batch_t *b, int threads, const lbm::Tile *tiles, int n_tiles, int src) {
  const int dst = 1 - src;
  return dispatch_b(b->precision, [&](auto tT, auto tC) {
    using T = std::remove_pointer_t<decltype(tT)>;
    using C = std::remove_pointer_t<decltype(tC)>;
    auto go = [&](auto kernel_threads) {
      constexpr int TH = decltype(kernel_threads)::value;
      return lbm::launch_batch_step<T, C, TH>(
          static_cast<const T *>(b->f[src]), static_cast<T *>(b->f[dst]), b->node, b->lbase,
          b->rowstart, b->links, b->cases, tiles, n_tiles, b->active, b->stream);
    };
    if (threads == 64) return go(std::integral_constant<int, 64>());
    if (threads == 128) return go(std::integral_constant<int, 128>());
    return go(std::integral_constant<int, 256>());
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
  for (void *p : {b->f[0], b->f[1], static_cast<void *>(b->node), static_cast<void *>(b->lbase),
                  static_cast<void *>(b->rowstart), static_cast<void *>(b->index), b->links, b->cases, static_cast<void *>(b->tiles), static_cast<void *>(b->active),
                  static_cast<void *>(b->steps_done), static_cast<void *>(b->res),
                  static_cast<void *>(b->counter), static_cast<void *>(b->n_active)})
    if (p) cudaFree(p);
  if (b->h_n_active) cudaFreeHost(b->h_n_active);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Autotuner: times each candidate CTA width for a few steps of the batch
// itself (from rest; the caller resets the state afterwards) and keeps the
// fastest, cached per (precision, size class).
int autotune(lbm_batch_t *b) {
  const int size_class = static_cast<int>(std::log2(static_cast<double>(b->total_nodes) + 1.0));
  {
    std::lock_guard<std::mutex> lock(lbm::g_tune_mu);
    auto it = lbm::g_tune_cache.find({b->precision, size_class});
    if (it != lbm::g_tune_cache.end()) return it->second;
  }
  const int cand[3] = {64, 128, 256};
  float best_ms = std::numeric_limits<float>::infinity();
  int best = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int th : cand) {
    std::vector<lbm::Tile> t = make_tiles(b, th);
    lbm::Tile *dt = nullptr;
    if (cudaMalloc(&dt, t.size() * sizeof(lbm::Tile)) != cudaSuccess) continue;
    cudaMemcpy(dt, t.data(), t.size() * sizeof(lbm::Tile), cudaMemcpyHostToDevice);
    for (int w = 0; w < 2; w++) step_once(b, th, dt, static_cast<int>(t.size()), w & 1);
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < 6; r++) step_once(b, th, dt, static_cast<int>(t.size()), r & 1);
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(dt);
    if (ms < best_ms) {
      best_ms = ms;
      best = th;
    }
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
  int64_t nodes = 0, links = 0, rows = 0, dense = 0;
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
    // the arena's push layout reads no group offsets, so a case whose node
    // words cannot hold them (more than 16383 solid rows in a row) is fine here
    (void)lbm::build_compact(hc[c], &cc[c]);
    nodes += cc[c].plane;
    links += hc[c].n_links;
    rows += hc[c].ny + 1;
    dense += static_cast<int64_t>(hc[c].nx) * hc[c].ny;
  }
  if (nodes * 9 >= (int64_t(1) << 40) || links >= (int64_t(1) << 31)) {
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
  std::vector<int32_t> lbase(static_cast<size_t>(nodes), 0), rowstart(static_cast<size_t>(rows), 0),
      index(static_cast<size_t>(dense), -1);
  std::vector<unsigned char> lhost(std::max<int64_t>(1, links) * 4 * ces, 0);
  std::vector<unsigned char> chost;
  int64_t noff = 0, loff = 0, roff = 0, ioff = 0;
  for (int c = 0; c < n_cases; c++) {
    const lbm::HostCase &h = hc[c];
    lbm::CompactCase &k = cc[c];
    b->nx.push_back(h.nx);
    b->ny.push_back(h.ny);
    b->f_off.push_back(9 * noff);
    b->node_off.push_back(noff);
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
    for (size_t q = 0; q < k.lbase.size(); q++)
      lbase[noff + q] = static_cast<int32_t>(k.lbase[q] + loff);
    std::copy(k.rowstart.begin(), k.rowstart.end(), rowstart.begin() + roff);
    std::copy(k.index.begin(), k.index.end(), index.begin() + ioff);
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
      d.f_off = 9 * noff;
      d.node_off = noff;
      d.row_off = roff;
      d.idx_off = ioff;
      d.n_fluid = h.n_fluid;
      const unsigned char *p = reinterpret_cast<const unsigned char *>(&d);
      chost.insert(chost.end(), p, p + sizeof(d));
    };
    if (precision == LBM_FP64)
      put(double());
    else
      put(float());
    b->rowstart_h.push_back(k.rowstart);
    noff += k.plane;
    loff += h.n_links;
    roff += h.ny + 1;
    ioff += static_cast<int64_t>(h.nx) * h.ny;
  }
  hc.clear();
  cc.clear();
  b->arena_nodes = nodes;
  auto alloc = [&](void **p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)); };
  const size_t fbytes = 9 * static_cast<size_t>(nodes) * es;
  if (e == cudaSuccess) e = alloc(&b->f[0], fbytes);
  if (e == cudaSuccess) e = alloc(&b->f[1], fbytes);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->node), node.size() * sizeof(uint2));
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->lbase), lbase.size() * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->rowstart), rowstart.size() * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->index), index.size() * 4);
  if (e == cudaSuccess) e = alloc(&b->links, lhost.size());
  if (e == cudaSuccess) e = alloc(&b->cases, chost.size());
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->active), n_cases * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->steps_done), n_cases * 8);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->res), n_cases * 8);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->counter), 8);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->n_active), 4);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&b->h_n_active), 4);
  auto up = [&](void *dst, const void *src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(b->node, node.data(), node.size() * sizeof(uint2));
  up(b->lbase, lbase.data(), lbase.size() * 4);
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
    if (e == cudaSuccess) b->threads = autotune(b);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    std::vector<lbm::Tile> t = make_tiles(b, b->threads);
    b->n_tiles = static_cast<int>(t.size());
    e = alloc(reinterpret_cast<void **>(&b->tiles), t.size() * sizeof(lbm::Tile));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->tiles, t.data(), t.size() * sizeof(lbm::Tile), cudaMemcpyHostToDevice);
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
  const size_t fbytes = 9 * static_cast<size_t>(b->arena_nodes) * elem_size_b(b->precision);
  std::vector<int32_t> ones(b->n_cases, 1);
  std::vector<int64_t> zeros(b->n_cases, 0);
  const int32_t n = b->n_cases;
  const int64_t zero = 0;
  cudaError_t e = cudaMemsetAsync(b->f[0], 0, fbytes, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->f[1], 0, fbytes, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->active, ones.data(), n * 4, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->steps_done, zeros.data(), n * 8, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->counter, &zero, 8, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->n_active, &n, 4, cudaMemcpyHostToDevice, b->stream);
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
  if (!b->graph || b->graph_K != check_every || b->graph_tol != tol) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    for (int s = 0; s < check_every && e == cudaSuccess; s++)
      e = step_once(b, b->threads, b->tiles, b->n_tiles, s & 1);
    if (e == cudaSuccess)
      e = dispatch_b(b->precision, [&](auto tT, auto tC) {
        using T = std::remove_pointer_t<decltype(tT)>;
        using C = std::remove_pointer_t<decltype(tC)>;
        lbm::batch_residual_kernel<T, C><<<b->n_cases, lbm::kBatchResidualThreads, 0, b->stream>>>(
            static_cast<const T *>(b->f[0]), static_cast<const T *>(b->f[1]),
            static_cast<const lbm::BatchCase<C> *>(b->cases), b->active, tol, b->counter,
            check_every, b->steps_done, b->res, b->n_active);
        return cudaGetLastError();
      });
    if (e == cudaSuccess) {
      lbm::batch_advance<<<1, 1, 0, b->stream>>>(b->counter, check_every);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_n_active, b->n_active, 4, cudaMemcpyDeviceToHost, b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bfail(b, LBM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    b->graph_K = check_every;
    b->graph_tol = tol;
  }
  int64_t done = 0;
  *b->h_n_active = b->n_cases;
  while (done < max_steps) {
    e = cudaGraphLaunch(b->graph, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    done += check_every;
    b->steps += check_every;
    if (*b->h_n_active <= 0) break;
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
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(d);
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_info(const lbm_batch_t *b, int64_t *total_nodes, int64_t *total_fluid,
                   int32_t *cta_threads, int32_t *n_tiles) {
  if (!b) return LBM_EINVAL;
  if (total_nodes) *total_nodes = b->total_nodes;
  if (total_fluid) *total_fluid = b->total_fluid;
  if (cta_threads) *cta_threads = b->threads;
  if (n_tiles) *n_tiles = b->n_tiles;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch_t *b) { batch_release(b); }

const char *lbm_batch_last_error(const lbm_batch_t *b) {
  return b ? b->err.c_str() : g_batch_error.c_str();
}

}  // extern "C"
