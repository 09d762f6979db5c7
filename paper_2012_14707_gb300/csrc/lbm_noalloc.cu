// lbm_residual_noalloc: the residual/mass reduction for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they want the convergence monitor: for example code that runs inside
// another framework whose memory pool owns the whole device, or a
// time-critical loop where an allocation would synchronise the device or
// fail under memory pressure.  This entry point takes the two population
// states and the solid mask as device arrays the caller already holds, and
// keeps its partial sums in a fixed, file-scope device array instead of
// allocated scratch.
//
// The scratch array, g_row_partials, holds kNoallocMaxRows rows x 5 doubles
// (640 KiB).  Every GPU that loads the library holds it until the process
// exits.  Host code cannot use the array's name as a device address (in
// host code it names a host-side stand-in), so every call looks the address
// up with cudaGetSymbolAddress, with the caller's device current.  The
// lookup allocates nothing; it is not cached, because the array's address
// belongs to the context that loaded the library's device code, and a
// cached one would be stale after cudaDeviceReset or under another context
// of the same device.
#include <cmath>
#include <cstdint>
#include <limits>
#include <string>

#include "lbm_internal.h"

namespace lbm {

const char *set_thread_error(const std::string &msg);  // lbm_api.cu

namespace {

constexpr int kNoallocMaxRows = 16384;
constexpr int kNoallocSlots = 5;  // num, den, sum(rho - 1), fluid count, non-finite count
constexpr int kRowThreads = 256;
constexpr int kFinalThreads = 1024;

// Row partials of the latest call, then (at the end) its 5 totals.
static __device__ __align__(256) double g_row_partials[(kNoallocMaxRows + 1) * kNoallocSlots];

__constant__ double kW[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Eq. FluidMacr from full populations; returns rho - 1 summed from the
// deviations f_i - w_i.
__device__ __forceinline__ double macro(const double *f, int64_t n, int64_t p, double ax, double ay,
                                        double &ux, double &uy) {
  double d[9];
  for (int i = 0; i < 9; i++) d[i] = f[i * n + p] - kW[i];
  double drho = 0.0;
  for (int i = 0; i < 9; i++) drho += d[i];
  const double jx = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
  const double jy = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
  const double rho = 1.0 + drho;
  ux = (jx + 0.5 * rho * ax) / rho;
  uy = (jy + 0.5 * rho * ay) / rho;
  return drho;
}

// One block per lattice row: its sums go to row slot blockIdx.x.  Every
// slot the final pass reads is written here first, so nothing needs
// clearing between calls.
__global__ void __launch_bounds__(kRowThreads)
noalloc_rows(const double *__restrict__ cur, const double *__restrict__ prev,
             const uint8_t *__restrict__ solid, int32_t nx, int32_t ny, double ax, double ay,
             double *__restrict__ rows) {
  const int64_t n = static_cast<int64_t>(nx) * ny;
  const int64_t y = blockIdx.x;
  double acc[kNoallocSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int32_t x = threadIdx.x; x < nx; x += blockDim.x) {
    const int64_t p = y * nx + x;
    if (solid[p]) continue;
    double u1, v1, u0, v0;
    const double drho = macro(cur, n, p, ax, ay, u1, v1);
    const double drho0 = macro(prev, n, p, ax, ay, u0, v0);
    acc[3] += 1.0;
    // a non-finite value in either state counts, as in lbm_residual
    if (!(isfinite(drho) && isfinite(u1) && isfinite(v1) && isfinite(drho0) && isfinite(u0) &&
          isfinite(v0))) {
      acc[4] += 1.0;
      continue;
    }
    acc[0] += (u1 - u0) * (u1 - u0) + (v1 - v0) * (v1 - v0);
    acc[1] += u1 * u1 + v1 * v1;
    acc[2] += drho;
  }
  __shared__ double sh[kRowThreads / 32][kNoallocSlots];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < kNoallocSlots; c++) {
    const double v = warp_sum(acc[c]);
    if (lane == 0) sh[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNoallocSlots) {
    double s = 0.0;
    for (int i = 0; i < kRowThreads / 32; i++) s += sh[i][threadIdx.x];
    rows[y * kNoallocSlots + threadIdx.x] = s;
  }
}

// Sums the ny row slots in a fixed order into slot kNoallocMaxRows.
__global__ void __launch_bounds__(kFinalThreads) noalloc_final(double *rows, int32_t ny) {
  double acc[kNoallocSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int32_t y = threadIdx.x; y < ny; y += blockDim.x)
    for (int c = 0; c < kNoallocSlots; c++) acc[c] += rows[y * kNoallocSlots + c];
  __shared__ double sh[kFinalThreads / 32][kNoallocSlots];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < kNoallocSlots; c++) {
    const double v = warp_sum(acc[c]);
    if (lane == 0) sh[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNoallocSlots) {
    double s = 0.0;
    for (int i = 0; i < kFinalThreads / 32; i++) s += sh[i][threadIdx.x];
    rows[static_cast<int64_t>(kNoallocMaxRows) * kNoallocSlots + threadIdx.x] = s;
  }
}

// Device address of g_row_partials in the context current on the calling
// thread (see the file comment: looked up on every call, never cached).
cudaError_t scratch_for_current_device(double **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_row_partials);
  if (e != cudaSuccess) return e;
  *out = static_cast<double *>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_residual_noalloc(const double *f_cur, const double *f_prev,
                                    const uint8_t *solid, int32_t nx, int32_t ny, double ax,
                                    double ay, void *stream, double *residual, double *mass) {
  using namespace lbm;
  if (!f_cur || !f_prev || !solid || !residual || !mass) {
    set_thread_error("lbm_residual_noalloc: null argument");
    return LBM_EINVAL;
  }
  if (nx < 1 || ny < 1) {
    set_thread_error("lbm_residual_noalloc: nx and ny must be >= 1");
    return LBM_EINVAL;
  }
  if (ny > kNoallocMaxRows) {
    set_thread_error("lbm_residual_noalloc: ny = " + std::to_string(ny) +
                     " exceeds the static scratch of " + std::to_string(kNoallocMaxRows) + " rows");
    return LBM_EINVAL;
  }
  if (!std::isfinite(ax) || !std::isfinite(ay)) {
    set_thread_error("lbm_residual_noalloc: non-finite force");
    return LBM_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *rows = nullptr;
  cudaError_t e = scratch_for_current_device(&rows);
  if (e == cudaSuccess) {
    noalloc_rows<<<ny, kRowThreads, 0, s>>>(f_cur, f_prev, solid, nx, ny, ax, ay, rows);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    noalloc_final<<<1, kFinalThreads, 0, s>>>(rows, ny);
    e = cudaGetLastError();
  }
  double tot[kNoallocSlots];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tot, rows + static_cast<int64_t>(kNoallocMaxRows) * kNoallocSlots,
                        sizeof tot, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_thread_error(std::string("lbm_residual_noalloc: ") + cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  const double num = tot[0], den = tot[1];
  if (std::isnan(num) || std::isnan(den))
    *residual = std::numeric_limits<double>::quiet_NaN();
  else
    *residual = den > 0.0 ? std::sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
  *mass = tot[3] + tot[2];
  if (tot[4] > 0.0) {
    set_thread_error("lbm_residual_noalloc: fluid nodes with non-finite density or velocity");
    return LBM_EUNSTABLE;
  }
  return LBM_OK;
}
