// Warm-start network of liblbm.so (lbm_net_*): a 4-level convolutional
// encoder-decoder that predicts (rho, u) of a steady state from (solid
// mask, signed distance, Kn), trained on the GPU by the kernels below.
// The paper has no network; this is the learned initial state of the
// solver, which then runs to the same residual as from rest.
//
// Layout: activations NHWC, weights [kh][kw][ci][co] (the layout of the
// FP64 reference in the tests).  Storage type A of activations and
// activation gradients: BF16 (training) or FP32 (gradient checks); every
// product is accumulated in FP32; master weights, weight gradients and Adam
// moments are FP32.
//
// Kernels:
//   conv_fwd<KS>    y = act(conv(x, w) + b), KS = 3 (zero padding) or 1;
//                   a CTA computes a 16x16 pixel tile x 16 output channels,
//                   staging an input tile (with halo) and the weights of a
//                   16-channel input slice in shared memory.
//   conv_bwd_data   the same kernel on weights flipped in space and
//                   transposed in channels (a conv3x3 is its own adjoint
//                   pattern), after masking the output gradient by the ReLU.
//   conv_bwd_weight dW[dy][dx][c][o] = sum_pixels x[p + d][c] gz[p][o]: a
//                   CTA reduces a pixel chunk for a 16x16 (c, o) tile and
//                   adds it into FP32 dW; db by a column sum.
//   pool / upsample / concat / MSE / Adam: elementwise or simple reductions.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace lbm {
namespace net {
namespace {

template <typename A>
__device__ __forceinline__ float to_f(A v);
template <>
__device__ __forceinline__ float to_f<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <typename A>
__device__ __forceinline__ A from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

constexpr int TP = 16;  // pixel tile edge
constexpr int TC = 16;  // channel tile (input slice and output block)

// y[n, i, j, o] = act(b[o] + sum x[n, i+dy-p, j+dx-p, c] w[dy][dx][c][o])
// over a channel range; `relu` applies max(., 0).  xs: channel stride of x
// (x may be a slice of a wider tensor: element (n,i,j,c) at
// ((n*H + i)*W + j)*xs + c).  Grid: (ceil(W/16)*ceil(H/16), ceil(Co/16), N).
template <typename A, int KS>
__global__ void __launch_bounds__(TP * TP)
conv_fwd(const A *__restrict__ x, int xs, const A *__restrict__ w, const float *__restrict__ b,
         A *__restrict__ y, int ys, int H, int W, int Ci, int Co, int relu) {
  constexpr int HALO = KS / 2;
  constexpr int T = TP + 2 * HALO;
  __shared__ float sx[T][T][TC + 1];  // +1: conflict-free strided reads
  __shared__ float sw[KS][KS][TC][TC];
  const int tiles_x = (W + TP - 1) / TP;
  const int ti = blockIdx.x / tiles_x, tj = blockIdx.x % tiles_x;
  const int o0 = blockIdx.y * TC;
  const int n = blockIdx.z;
  const int li = threadIdx.x / TP, lj = threadIdx.x % TP;
  const int i = ti * TP + li, j = tj * TP + lj;
  float acc[TC];
#pragma unroll
  for (int q = 0; q < TC; q++) acc[q] = 0.f;
  for (int c0 = 0; c0 < Ci; c0 += TC) {
    // input tile with halo
    for (int e = threadIdx.x; e < T * T * TC; e += TP * TP) {
      const int c = e % TC, p = e / TC, pj = p % T, pi = p / T;
      const int gi = ti * TP + pi - HALO, gj = tj * TP + pj - HALO;
      float v = 0.f;
      if (gi >= 0 && gi < H && gj >= 0 && gj < W && c0 + c < Ci)
        v = to_f<A>(x[((static_cast<int64_t>(n) * H + gi) * W + gj) * xs + c0 + c]);
      sx[pi][pj][c] = v;
    }
    for (int e = threadIdx.x; e < KS * KS * TC * TC; e += TP * TP) {
      const int o = e % TC, c = (e / TC) % TC, d = e / (TC * TC);
      float v = 0.f;
      if (c0 + c < Ci && o0 + o < Co) v = to_f<A>(w[(static_cast<int64_t>(d) * Ci + c0 + c) * Co + o0 + o]);
      sw[d / KS][d % KS][c][o] = v;
    }
    __syncthreads();
#pragma unroll
    for (int dy = 0; dy < KS; dy++)
#pragma unroll
      for (int dx = 0; dx < KS; dx++)
#pragma unroll 4
        for (int c = 0; c < TC; c++) {
          const float xv = sx[li + dy][lj + dx][c];
#pragma unroll
          for (int q = 0; q < TC; q++) acc[q] = fmaf(xv, sw[dy][dx][c][q], acc[q]);
        }
    __syncthreads();
  }
  if (i < H && j < W) {
    A *yp = y + ((static_cast<int64_t>(n) * H + i) * W + j) * ys;
#pragma unroll
    for (int q = 0; q < TC; q++) {
      if (o0 + q < Co) {
        float v = acc[q] + (b ? b[o0 + q] : 0.f);
        if (relu) v = fmaxf(v, 0.f);
        yp[o0 + q] = from_f<A>(v);
      }
    }
  }
}

// dW[dy][dx][c][o] += sum over a pixel chunk of x[p + d - HALO][c] gz[p][o];
// db[o] += sum gz[p][o] (blockIdx.y == 0 tiles only).  Grid:
// (ceil(Ci/16) * ceil(Co/16), chunks); 256 threads = 16 (c) x 16 (o).
template <typename A, int KS>
__global__ void __launch_bounds__(256)
conv_bwd_weight(const A *__restrict__ x, int xs, const A *__restrict__ gz, int N, int H, int W,
                int Ci, int Co, int pix_per_chunk, float *__restrict__ dw, float *__restrict__ db) {
  constexpr int HALO = KS / 2;
  const int tiles_o = (Co + TC - 1) / TC;
  const int c0 = (blockIdx.x / tiles_o) * TC, o0 = (blockIdx.x % tiles_o) * TC;
  const int c = threadIdx.x / TC, o = threadIdx.x % TC;
  const int64_t npix = static_cast<int64_t>(N) * H * W;
  const int64_t p0 = static_cast<int64_t>(blockIdx.y) * pix_per_chunk;
  const int64_t p1 = p0 + pix_per_chunk < npix ? p0 + pix_per_chunk : npix;
  __shared__ float sg[32][TC];
  __shared__ float sxv[32][KS * KS][TC];
  float acc[KS * KS];
#pragma unroll
  for (int d = 0; d < KS * KS; d++) acc[d] = 0.f;
  float bacc = 0.f;
  for (int64_t pb = p0; pb < p1; pb += 32) {
    // stage 32 pixels: gz[p][o0..] and x[p + d][c0..] for every offset d
    for (int e = threadIdx.x; e < 32 * TC; e += 256) {
      const int pp = e / TC, oo = e % TC;
      const int64_t p = pb + pp;
      sg[pp][oo] = (p < p1 && o0 + oo < Co) ? to_f<A>(gz[p * Co + o0 + oo]) : 0.f;
    }
    for (int e = threadIdx.x; e < 32 * KS * KS * TC; e += 256) {
      const int cc = e % TC, d = (e / TC) % (KS * KS), pp = e / (TC * KS * KS);
      const int64_t p = pb + pp;
      float v = 0.f;
      if (p < p1 && c0 + cc < Ci) {
        const int64_t n = p / (static_cast<int64_t>(H) * W);
        const int rem = static_cast<int>(p - n * H * W);
        const int i = rem / W + d / KS - HALO, j = rem % W + d % KS - HALO;
        if (i >= 0 && i < H && j >= 0 && j < W)
          v = to_f<A>(x[((n * H + i) * W + j) * xs + c0 + cc]);
      }
      sxv[pp][d][cc] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int pp = 0; pp < 32; pp++) {
      const float g = sg[pp][o];
#pragma unroll
      for (int d = 0; d < KS * KS; d++) acc[d] = fmaf(sxv[pp][d][c], g, acc[d]);
      bacc += g;
    }
    __syncthreads();
  }
  if (c0 + c < Ci && o0 + o < Co) {
#pragma unroll
    for (int d = 0; d < KS * KS; d++)
      atomicAdd(&dw[(static_cast<int64_t>(d) * Ci + c0 + c) * Co + o0 + o], acc[d]);
    if (c == 0 && c0 == 0 && db) atomicAdd(&db[o0 + o], bacc);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core convolution (BF16 storage): an implicit GEMM on tcgen05.
//   D[p][o] = sum_{d, c} X[p + d - HALO][c] * Wk[o][d][c]      (M = pixels,
//   N = output channels, K = taps x input channels)
// A CTA owns 128 pixels x NT output channels (NT <= 128, a multiple of 16);
// D lives in tensor memory (FP32, NT columns).  K runs tap by tap in chunks
// of up to 64 channels: the 128 threads gather one pixel row each of A (the
// shifted input, zero outside the image) and one row each of B (packed
// weights, K-major), store both in shared memory in the canonical K-major
// layout without swizzle (8-row x 16-byte core matrices, core matrices
// along K 128 B apart, 8-row groups 1024 B apart), and one thread issues
// the MMAs (M = 128, N = NT, K = 16 each) and commits them to an mbarrier.
// Two stages: the gather of chunk k + 1 overlaps the MMAs of chunk k.  Every
// wait is bounded; a wait that runs out sets *err and the CTA stops issuing.
// The epilogue reads D back with tcgen05.ld (warp w owns lanes 32w..32w+31 =
// pixels 32w..), adds the bias, applies ReLU and stores BF16.

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Waits for the phase with parity `phase` of *bar; false if it did not come
// within `limit` polls (test_wait: each poll returns at once, so the bound
// is a bound in time).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, int limit) {
  for (int it = 0; it < limit; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Shared-memory matrix descriptor (K-major, no swizzle): start address,
// leading byte offset (between core matrices along K), stride byte offset
// (between 8-row groups), all in 16-byte units; bit 46 = descriptor version
// of this architecture; layout type 0 = no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

constexpr int kTcM = 128;        // pixels per CTA (MMA M)
constexpr int kTcKC = 64;        // channels per K chunk
constexpr int kTcNMax = 128;     // output channels per CTA (MMA N)
constexpr int kTcStageBytes = kTcM * kTcKC * 2;  // one operand, one stage: 16 KB
constexpr int kTcSmem = 4 * kTcStageBytes + 1024;  // A and B, two stages, + alignment
constexpr int kTcWaitLimit = 1 << 24;

// Wk[o][d][c] (BF16, K-major, Co rows padded to Cop, Ci padded to Cip with
// zeros) from the FP32 parameters w[d][c][o].  flip: the adjoint
// convolution's weights (taps reversed, channels swapped): Wk[c][d][o] =
// w[KS2 - 1 - d][c][o], i.e. a layer with Ci and Co exchanged.
__global__ void pack_wk(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wk, int KS2,
                        int Ci, int Co, int flip, int Cop, int Cip) {
  // output layer: Ci' = flip ? Co : Ci, Co' = flip ? Ci : Co
  const int64_t n = static_cast<int64_t>(Cop) * KS2 * Cip;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c2 = static_cast<int>(e % Cip);
    const int d = static_cast<int>((e / Cip) % KS2);
    const int o2 = static_cast<int>(e / (static_cast<int64_t>(Cip) * KS2));
    float v = 0.f;
    if (!flip) {
      if (o2 < Co && c2 < Ci) v = w[(static_cast<int64_t>(d) * Ci + c2) * Co + o2];
    } else {
      // o2 = original input channel, c2 = original output channel
      if (o2 < Ci && c2 < Co) v = w[(static_cast<int64_t>(KS2 - 1 - d) * Ci + o2) * Co + c2];
    }
    wk[e] = __float2bfloat16_rn(v);
  }
}

template <int KS>
__global__ void __launch_bounds__(kTcM)
conv_fwd_tc(const __nv_bfloat16 *__restrict__ x, int xs, const __nv_bfloat16 *__restrict__ wk,
            int Cip, const float *__restrict__ b, __nv_bfloat16 *__restrict__ y, int ys, int N,
            int H, int W, int Ci, int Co, int NT, int relu, int vec, int *__restrict__ err) {
  constexpr int HALO = KS / 2;
  constexpr int KS2 = KS * KS;
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t npix = static_cast<int64_t>(N) * H * W;
  const int64_t p = static_cast<int64_t>(blockIdx.x) * kTcM + tid;  // this thread's pixel (A row)
  const int o0 = blockIdx.y * NT;
  int pn = 0, pi = 0, pj = 0;
  if (p < npix) {
    pn = static_cast<int>(p / (static_cast<int64_t>(H) * W));
    const int r = static_cast<int>(p - static_cast<int64_t>(pn) * H * W);
    pi = r / W;
    pj = r - pi * W;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTcNMax)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = umma_idesc_bf16(kTcM, NT);
  const int nck = (Cip + kTcKC - 1) / kTcKC;  // channel chunks per tap
  const int iters = KS2 * nck;
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  for (int it = 0; it < iters; it++) {
    const int st = it & 1;
    if (it >= 2) {  // the MMAs that read this stage two chunks ago are done
      const bool got = mbar_wait(&mbar[st], phase[st], kTcWaitLimit);
      if (__syncthreads_or(!got)) {  // one decision for the whole CTA
        ok = false;
        if (tid == 0) atomicExch(err, 1);
        break;
      }
      phase[st] ^= 1u;
    }
    const int d = it / nck, c0 = (it % nck) * kTcKC;
    const int kc = min(kTcKC, Cip - c0);  // multiple of 16
    unsigned char *sa = smem + st * 2 * kTcStageBytes;
    unsigned char *sb = sa + kTcStageBytes;
    // A row `tid`: input pixel (pi + dy - HALO, pj + dx - HALO), channels c0 .. c0 + kc
    {
      const int ii = pi + d / KS - HALO, jj = pj + d % KS - HALO;
      const bool in = p < npix && ii >= 0 && ii < H && jj >= 0 && jj < W;
      const __nv_bfloat16 *src = x + ((static_cast<int64_t>(pn) * H + ii) * W + jj) * xs;
      unsigned char *row = sa + (tid >> 3) * 1024 + (tid & 7) * 16;
      for (int q = 0; q < kc / 8; q++) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        const int c = c0 + q * 8;
        if (in && c < Ci) {
          if (vec) {
            v = *reinterpret_cast<const uint4 *>(src + c);
          } else {
            __nv_bfloat16 t8[8];
#pragma unroll
            for (int e = 0; e < 8; e++) t8[e] = (c + e < Ci) ? src[c + e] : __float2bfloat16_rn(0.f);
            v = *reinterpret_cast<const uint4 *>(t8);
          }
        }
        *reinterpret_cast<uint4 *>(row + q * 128) = v;
      }
    }
    // B row `tid` (< NT): output channel o0 + tid, tap d, channels c0 .. c0 + kc
    if (tid < NT) {
      const __nv_bfloat16 *src = wk + (static_cast<int64_t>(o0 + tid) * KS2 + d) * Cip + c0;
      unsigned char *row = sb + (tid >> 3) * 1024 + (tid & 7) * 16;
      for (int q = 0; q < kc / 8; q++)
        *reinterpret_cast<uint4 *>(row + q * 128) = *reinterpret_cast<const uint4 *>(src + q * 8);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = smem_addr(sa), b0 = smem_addr(sb);
      for (int k = 0; k < kc / 16; k++) {
        const uint64_t ad = umma_desc(a0 + k * 256, 128, 1024);
        const uint64_t bd = umma_desc(b0 + k * 256, 128, 1024);
        const uint32_t acc = (it > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_addr(&mbar[st]))
                   : "memory");
    }
  }
  // all MMAs done: the last commit covers every earlier MMA of the issuing thread
  if (ok && iters > 0) {
    const int st = (iters - 1) & 1;
    const bool got = mbar_wait(&mbar[st], phase[st], kTcWaitLimit);
    if (__syncthreads_or(!got)) {
      ok = false;
      if (tid == 0) atomicExch(err, 1);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // tcgen05.ld is warp-collective (.sync.aligned): every lane loads, in
  // converged code, also lanes past the last pixel; only the stores are
  // predicated.  `ok` is uniform over the CTA.
  if (ok) {
    __syncwarp();
    __nv_bfloat16 *yp = y + (p < npix ? p : 0) * ys;
    for (int c = 0; c < NT; c += 8) {
      uint32_t r[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7])
          : "r"(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (p < npix) {
#pragma unroll
        for (int e = 0; e < 8; e++) {
          const int o = o0 + c + e;
          if (o < Co) {
            float v = __uint_as_float(r[e]) + (b ? b[o] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            yp[o] = __float2bfloat16_rn(v);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTcNMax)
                 : "memory");
  }
  (void)lane;
}

// The same convolution with its operands copied asynchronously (cp.async,
// 16 bytes per copy, zero-filled outside the image) through a ring of
// kTcAsyncStages stages: the copies of the next kTcAsyncStages - 1 chunks
// are in flight while the tensor cores work on the current one, instead of
// each chunk's gather waiting out its own memory latency.  Needs 16-byte
// aligned channel rows (input channels and their stride multiples of 8).
constexpr int kTcAsyncStages = 3;
constexpr int kTcAsyncSmem = kTcAsyncStages * 2 * kTcStageBytes + 1024;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int KS>
__global__ void __launch_bounds__(kTcM)
conv_fwd_tc_async(const __nv_bfloat16 *__restrict__ x, int xs,
                  const __nv_bfloat16 *__restrict__ wk, int Cip, const float *__restrict__ b,
                  __nv_bfloat16 *__restrict__ y, int ys, int N, int H, int W, int Ci, int Co,
                  int NT, int relu, int *__restrict__ err) {
  constexpr int HALO = KS / 2;
  constexpr int KS2 = KS * KS;
  constexpr int S = kTcAsyncStages;
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ uint64_t mbar[S];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t npix = static_cast<int64_t>(N) * H * W;
  const int64_t p = static_cast<int64_t>(blockIdx.x) * kTcM + tid;  // this thread's pixel (A row)
  const int o0 = blockIdx.y * NT;
  int pn = 0, pi = 0, pj = 0;
  if (p < npix) {
    pn = static_cast<int>(p / (static_cast<int64_t>(H) * W));
    const int r = static_cast<int>(p - static_cast<int64_t>(pn) * H * W);
    pi = r / W;
    pj = r - pi * W;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTcNMax)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < S; s++) mbar_init(&mbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = umma_idesc_bf16(kTcM, NT);
  const int nck = (Cip + kTcKC - 1) / kTcKC;  // channel chunks per tap
  const int iters = KS2 * nck;
  // copies of chunk `it` into its stage: A row `tid` (input pixel shifted by
  // the tap, zero outside the image) and B row `tid` (< NT: output channel
  // o0 + tid of the packed weights)
  auto load = [&](int it) {
    const int st = it % S;
    const int d = it / nck, c0 = (it % nck) * kTcKC;
    const int kc = min(kTcKC, Cip - c0);
    const uint32_t sa = smem_addr(smem + st * 2 * kTcStageBytes);
    const uint32_t sb = sa + kTcStageBytes;
    const uint32_t row = (tid >> 3) * 1024 + (tid & 7) * 16;
    const int ii = pi + d / KS - HALO, jj = pj + d % KS - HALO;
    const bool in = p < npix && ii >= 0 && ii < H && jj >= 0 && jj < W;
    const __nv_bfloat16 *src =
        in ? x + ((static_cast<int64_t>(pn) * H + ii) * W + jj) * xs : x;
    for (int q = 0; q < kc / 8; q++) {
      const int c = c0 + q * 8;
      const bool v = in && c < Ci;
      cp_async16(sa + row + q * 128, v ? src + c : x, v ? 16u : 0u);
    }
    if (tid < NT) {
      const __nv_bfloat16 *ws = wk + (static_cast<int64_t>(o0 + tid) * KS2 + d) * Cip + c0;
      for (int q = 0; q < kc / 8; q++) cp_async16(sb + row + q * 128, ws + q * 8, 16u);
    }
  };
  for (int s = 0; s < S - 1; s++) {
    if (s < iters) load(s);
    cp_async_commit();
  }
  bool ok = true;
  for (int it = 0; it < iters; it++) {
    const int st = it % S;
    const int nxt = it + S - 1;
    if (nxt < iters) {
      // stage nxt % S was last read by the MMAs of chunk it - 1
      if (it >= 1) {
        const bool got = mbar_wait(&mbar[(it - 1) % S], ((it - 1) / S) & 1, kTcWaitLimit);
        if (__syncthreads_or(!got)) {  // one decision for the whole CTA
          ok = false;
          if (tid == 0) atomicExch(err, 1);
          break;
        }
      }
      load(nxt);
    }
    cp_async_commit();
    cp_async_wait<S - 1>();  // this thread's copies of chunk `it` have landed
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int c0 = (it % nck) * kTcKC;
      const int kc = min(kTcKC, Cip - c0);
      const uint32_t a0 = smem_addr(smem + st * 2 * kTcStageBytes), b0 = a0 + kTcStageBytes;
      for (int k = 0; k < kc / 16; k++) {
        const uint64_t ad = umma_desc(a0 + k * 256, 128, 1024);
        const uint64_t bd = umma_desc(b0 + k * 256, 128, 1024);
        const uint32_t acc = (it > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_addr(&mbar[st]))
                   : "memory");
    }
  }
  cp_async_wait<0>();  // no copy left in flight, whatever happened above
  // all MMAs done: the last commit covers every earlier MMA of the issuing thread
  if (ok && iters > 0) {
    const int last = iters - 1;
    const bool got = mbar_wait(&mbar[last % S], (last / S) & 1, kTcWaitLimit);
    if (__syncthreads_or(!got)) {
      ok = false;
      if (tid == 0) atomicExch(err, 1);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok) {
    __syncwarp();
    __nv_bfloat16 *yp = y + (p < npix ? p : 0) * ys;
    for (int c = 0; c < NT; c += 8) {
      uint32_t r[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7])
          : "r"(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (p < npix) {
#pragma unroll
        for (int e = 0; e < 8; e++) {
          const int o = o0 + c + e;
          if (o < Co) {
            float v = __uint_as_float(r[e]) + (b ? b[o] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            yp[o] = __float2bfloat16_rn(v);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTcNMax)
                 : "memory");
  }
}

// Weight gradient on the tensor cores:
//   dW[d][c][o] = sum_p X[p + d - HALO][c] gz[p][o]     db[o] = sum_p gz[p][o]
// as D[m][n] = sum_k A[m][k] B[n][k] with m = d * Ci + c (M = 128 per CTA),
// n = o (N = NT), k = pixel (K, split over blockIdx.z: kper pixels each).
// Chunks of 32 pixels are staged K-major: thread t gathers row t of A (tap
// and channel of m, 32 consecutive pixels shifted by the tap) and row t of
// B (channel o0 + t of gz); 8 pixels of one row are one 16-byte core-matrix
// row.  The partial D of the CTA is added into dW with atomics.
constexpr int kWgKC = 32;                             // pixels per K chunk
constexpr int kWgStage = kTcM * kWgKC * 2;            // one operand, one stage: 8 KB
constexpr int kWgSmem = 4 * kWgStage + 1024;

template <int KS>
__global__ void __launch_bounds__(kTcM)
conv_wgrad_tc(const __nv_bfloat16 *__restrict__ x, int xs, const __nv_bfloat16 *__restrict__ gz,
              int gs, int N, int H, int W, int Ci, int Co, int NT, int kper,
              float *__restrict__ dw, float *__restrict__ db, int *__restrict__ err) {
  constexpr int HALO = KS / 2;
  constexpr int KS2 = KS * KS;
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t npix = static_cast<int64_t>(N) * H * W;
  const int m0 = blockIdx.x * kTcM, o0 = blockIdx.y * NT;
  const int64_t pstart = static_cast<int64_t>(blockIdx.z) * kper;
  const int64_t pend = min(npix, pstart + kper);
  const int nch = pend > pstart ? static_cast<int>((pend - pstart + kWgKC - 1) / kWgKC) : 0;
  // this thread's A row: tap d and channel c of m = m0 + tid
  const int m = m0 + tid;
  const bool mrow = m < KS2 * Ci;
  const int d = mrow ? m / Ci : 0, c = mrow ? m - (m / Ci) * Ci : 0;
  const int sy = d / KS - HALO, sx = d % KS - HALO;
  const bool nrow = tid < NT && o0 + tid < Co;
  float bsum = 0.f;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTcNMax)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = umma_idesc_bf16(kTcM, NT);
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  for (int it = 0; it < nch; it++) {
    const int st = it & 1;
    if (it >= 2) {
      const bool got = mbar_wait(&mbar[st], phase[st], kTcWaitLimit);
      if (__syncthreads_or(!got)) {
        ok = false;
        if (tid == 0) atomicExch(err, 1);
        break;
      }
      phase[st] ^= 1u;
    }
    const int64_t p0 = pstart + static_cast<int64_t>(it) * kWgKC;
    unsigned char *sa = smem + st * 2 * kWgStage;
    unsigned char *sb = sa + kWgStage;
    // pixel p0 as (image, row, column); advanced one pixel at a time
    int pn = static_cast<int>(p0 / (static_cast<int64_t>(H) * W));
    int rem = static_cast<int>(p0 - static_cast<int64_t>(pn) * H * W);
    int pi = rem / W, pj = rem - (rem / W) * W;
    for (int k8 = 0; k8 < kWgKC / 8; k8++) {
      __align__(16) __nv_bfloat16 va[8], vb[8];
#pragma unroll
      for (int e = 0; e < 8; e++) {
        const int64_t p = p0 + k8 * 8 + e;
        float a = 0.f, bb = 0.f;
        if (p < pend) {
          const int ii = pi + sy, jj = pj + sx;
          if (mrow && ii >= 0 && ii < H && jj >= 0 && jj < W)
            a = __bfloat162float(x[((static_cast<int64_t>(pn) * H + ii) * W + jj) * xs + c]);
          if (nrow) {
            bb = __bfloat162float(gz[p * gs + o0 + tid]);
            bsum += bb;
          }
        }
        va[e] = __float2bfloat16_rn(a);
        vb[e] = __float2bfloat16_rn(bb);
        if (++pj == W) {
          pj = 0;
          if (++pi == H) {
            pi = 0;
            ++pn;
          }
        }
      }
      *reinterpret_cast<uint4 *>(sa + (tid >> 3) * 512 + k8 * 128 + (tid & 7) * 16) =
          *reinterpret_cast<const uint4 *>(va);
      if (tid < NT)
        *reinterpret_cast<uint4 *>(sb + (tid >> 3) * 512 + k8 * 128 + (tid & 7) * 16) =
            *reinterpret_cast<const uint4 *>(vb);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = smem_addr(sa), b0 = smem_addr(sb);
      for (int k = 0; k < kWgKC / 16; k++) {
        const uint64_t ad = umma_desc(a0 + k * 256, 128, 512);
        const uint64_t bd = umma_desc(b0 + k * 256, 128, 512);
        const uint32_t acc = (it > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_addr(&mbar[st]))
                   : "memory");
    }
  }
  if (ok && nch > 0) {
    const int st = (nch - 1) & 1;
    const bool got = mbar_wait(&mbar[st], phase[st], kTcWaitLimit);
    if (__syncthreads_or(!got)) {
      ok = false;
      if (tid == 0) atomicExch(err, 1);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok && nch > 0) {  // uniform: every lane takes part in the warp-collective loads
    __syncwarp();
    const int mr = m0 + warp * 32 + (tid & 31);  // the TMEM lane this thread reads = row of D
    for (int cc = 0; cc < NT; cc += 8) {
      uint32_t r[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7])
          : "r"(tmem + (static_cast<uint32_t>(warp * 32) << 16) + cc));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (mr < KS2 * Ci) {
#pragma unroll
        for (int e = 0; e < 8; e++) {
          const int o = o0 + cc + e;
          if (o < Co) atomicAdd(&dw[static_cast<int64_t>(mr) * Co + o], __uint_as_float(r[e]));
        }
      }
    }
  }
  if (ok && db && blockIdx.x == 0 && nrow) atomicAdd(&db[o0 + tid], bsum);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTcNMax)
                 : "memory");
  }
}

// wt[d'][o][c] = w[KS*KS-1-d'][c][o]: the weights of the adjoint convolution.
template <typename A>
__global__ void flip_weights(const float *__restrict__ w, A *__restrict__ wt, int KS2, int Ci, int Co) {
  const int64_t n = static_cast<int64_t>(KS2) * Ci * Co;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % Ci), o = static_cast<int>((e / Ci) % Co),
              d = static_cast<int>(e / (static_cast<int64_t>(Ci) * Co));
    wt[e] = from_f<A>(w[(static_cast<int64_t>(KS2 - 1 - d) * Ci + c) * Co + o]);
  }
}

template <typename A>
__global__ void to_storage(const float *__restrict__ s, A *__restrict__ d, int64_t n) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    d[e] = from_f<A>(s[e]);
}

template <typename A>
__global__ void to_float(const A *__restrict__ s, int ss, float *__restrict__ d, int C, int64_t npix) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < npix * C;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = e / C;
    d[e] = to_f<A>(s[p * ss + e % C]);
  }
}

// g[p][c] *= (h[p][c] > 0)  (ReLU backward; h is the layer output)
template <typename A>
__global__ void relu_mask(A *__restrict__ g, const A *__restrict__ h, int64_t n) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    if (!(to_f<A>(h[e]) > 0.f)) g[e] = from_f<A>(0.f);
}

// 2x2 average pooling, y has H/2 x W/2 pixels; x channel stride xs.
template <typename A>
__global__ void pool2_fwd(const A *__restrict__ x, int xs, A *__restrict__ y, int N, int H, int W,
                          int C) {
  const int h2 = H / 2, w2 = W / 2;
  const int64_t n_out = static_cast<int64_t>(N) * h2 * w2 * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n_out;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % C);
    const int64_t p = e / C;
    const int j = static_cast<int>(p % w2), i = static_cast<int>((p / w2) % h2);
    const int64_t n = p / (static_cast<int64_t>(w2) * h2);
    float s = 0.f;
    for (int a = 0; a < 2; a++)
      for (int bb = 0; bb < 2; bb++)
        s += to_f<A>(x[((n * H + 2 * i + a) * W + 2 * j + bb) * xs + c]);
    y[e] = from_f<A>(0.25f * s);
  }
}

// gx[.] (+)= gy / 4 spread over each 2x2 block; gx channel stride xs
template <typename A>
__global__ void pool2_bwd(const A *__restrict__ gy, A *__restrict__ gx, int xs, int N, int H, int W,
                          int C, int accumulate) {
  const int64_t n_in = static_cast<int64_t>(N) * H * W * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n_in;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % C);
    const int64_t p = e / C;
    const int j = static_cast<int>(p % W), i = static_cast<int>((p / W) % H);
    const int64_t n = p / (static_cast<int64_t>(W) * H);
    float v = 0.25f * to_f<A>(gy[((n * (H / 2) + i / 2) * (W / 2) + j / 2) * C + c]);
    A *dst = gx + p * xs + c;
    if (accumulate) v += to_f<A>(*dst);
    *dst = from_f<A>(v);
  }
}

// y (channel stride ys, first C channels) = nearest 2x upsampling of x
template <typename A>
__global__ void up2_fwd(const A *__restrict__ x, A *__restrict__ y, int ys, int N, int H, int W,
                        int C) {
  const int64_t n_out = static_cast<int64_t>(N) * H * W * C;  // H, W: output size
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n_out;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % C);
    const int64_t p = e / C;
    const int j = static_cast<int>(p % W), i = static_cast<int>((p / W) % H);
    const int64_t n = p / (static_cast<int64_t>(W) * H);
    y[p * ys + c] = x[((n * (H / 2) + i / 2) * (W / 2) + j / 2) * C + c];
  }
}

// gx (H/2 x W/2, C channels) = sum of gy over each 2x2 block; gy channel stride gs
template <typename A>
__global__ void up2_bwd(const A *__restrict__ gy, int gs, A *__restrict__ gx, int N, int H, int W,
                        int C) {
  const int h2 = H / 2, w2 = W / 2;
  const int64_t n_out = static_cast<int64_t>(N) * h2 * w2 * C;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n_out;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % C);
    const int64_t p = e / C;
    const int j = static_cast<int>(p % w2), i = static_cast<int>((p / w2) % h2);
    const int64_t n = p / (static_cast<int64_t>(w2) * h2);
    float s = 0.f;
    for (int a = 0; a < 2; a++)
      for (int bb = 0; bb < 2; bb++) s += to_f<A>(gy[((n * H + 2 * i + a) * W + 2 * j + bb) * gs + c]);
    gx[e] = from_f<A>(s);
  }
}

// copy C channels between tensors with channel strides (and offsets applied by the caller)
template <typename A>
__global__ void copy_channels(const A *__restrict__ s, int ss, A *__restrict__ d, int ds, int C,
                              int64_t npix, int accumulate) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < npix * C;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t p = e / C;
    const int c = static_cast<int>(e % C);
    float v = to_f<A>(s[p * ss + c]);
    if (accumulate) v += to_f<A>(d[p * ds + c]);
    d[p * ds + c] = from_f<A>(v);
  }
}

// MSE: loss partials and gy = 2 (y - t) / n
template <typename A>
__global__ void mse_kernel(const A *__restrict__ y, const float *__restrict__ t, A *__restrict__ gy,
                           int64_t n, double *__restrict__ loss) {
  double s = 0.0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float d = to_f<A>(y[e]) - t[e];
    s += static_cast<double>(d) * d;
    gy[e] = from_f<A>(2.f * d / static_cast<float>(n));
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

int grid1(int64_t n) {
  int64_t b = (n + 255) / 256;
  return static_cast<int>(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace
}  // namespace net
}  // namespace lbm

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

struct Layer {
  int ks, ci, co;
  int64_t w_off, b_off;  // offsets into the flat FP32 parameter vector
};

thread_local std::string g_net_error;

}  // namespace

struct lbm_net {
  int base = 32, levels = 4, c_in = 3, c_out = 3, precision = LBM_BF16;
  int max_batch = 1, H = 0, W = 0;
  cudaStream_t stream = nullptr;
  std::vector<Layer> layers;
  int64_t n_params = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  void *wq = nullptr;   // weights in the storage type
  void *wt = nullptr;   // flipped weights (largest layer), storage type
  void *wk = nullptr;   // packed K-major BF16 weights of the tensor-core path (largest layer)
  int *d_err = nullptr; // set by a tensor-core kernel whose bounded wait ran out
  // activations: per level encoder outputs (skip), decoder concat inputs,
  // temporaries; all storage type, sized for max_batch
  std::vector<void *> bufs;
  std::vector<int64_t> buf_elems;
  double *loss = nullptr;
  int64_t adam_t = 0;
  std::string err;
};

namespace {

size_t asize(int precision) { return precision == LBM_FP32 ? 4 : 2; }

// Buffer plan (index -> meaning), all NHWC with the channel counts below:
//   x_in                       input, c_in channels
//   e[l]a_out, e[l]b_out       encoder outputs per level (b is the skip)
//   pool[l]                    pooled input of level l (l >= 1)
//   cat[l]                     decoder input of level l: [up, skip]
//   d[l]a_out, d[l]b_out
//   y                          head output
// Gradients use a second set of the same shapes.
struct Plan {
  std::vector<int64_t> elems;  // per buffer, per sample
  int x_in, y;
  std::vector<int> ea, eb, pool, cat, da, db;
};

Plan make_plan(const lbm_net_t *n) {
  Plan p;
  auto add = [&](int64_t e) {
    p.elems.push_back(e);
    return static_cast<int>(p.elems.size()) - 1;
  };
  const int64_t HW = static_cast<int64_t>(n->H) * n->W;
  p.x_in = add(HW * n->c_in);
  for (int l = 0; l < n->levels; l++) {
    const int64_t hw = HW >> (2 * l);
    const int ch = n->base << l;
    p.pool.push_back(l > 0 ? add(hw * (n->base << (l - 1))) : -1);
    p.ea.push_back(add(hw * ch));
    p.eb.push_back(add(hw * ch));
  }
  p.cat.assign(n->levels, -1);
  p.da.assign(n->levels, -1);
  p.db.assign(n->levels, -1);
  for (int l = n->levels - 2; l >= 0; l--) {
    const int64_t hw = HW >> (2 * l);
    const int ch = n->base << l;
    p.cat[l] = add(hw * (ch * 2 + ch));
    p.da[l] = add(hw * ch);
    p.db[l] = add(hw * ch);
  }
  p.y = add(HW * n->c_out);
  return p;
}

bool tc_timed_out(lbm_net_t *n) {
  int v = 0;
  return cudaMemcpy(&v, n->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && v != 0;
}

int nfail(lbm_net_t *n, int code, const std::string &m) {
  if (n) n->err = m;
  else g_net_error = m;
  return code;
}

// Output-channel tile of the tensor-core convolution and the padded sizes
// of its packed weights.
void tc_shape(int Ci, int Co, int *NT, int *Cop, int *Cip) {
  *NT = std::min(lbm::net::kTcNMax, (Co + 15) / 16 * 16);
  *Cop = (Co + *NT - 1) / *NT * *NT;
  *Cip = (Ci + 15) / 16 * 16;
}

// y = act(conv(x, w) + b) with Ci inputs and Co outputs.  FP32 storage: the
// CUDA-core kernel on w (layout [tap][ci][co]).  BF16 storage: the tensor-core
// kernel on weights packed from the FP32 parameters wsrc of layer (lci, lco),
// flipped for the adjoint convolution of the backward pass.
template <typename A>
void launch_conv(lbm_net_t *n, const A *x, int xs, const A *w, const float *b, A *y, int ys,
                 int N, int H, int W, int Ci, int Co, int ks, int relu, const float *wsrc, int flip,
                 int lci, int lco) {
  using namespace lbm::net;
  if constexpr (std::is_same<A, __nv_bfloat16>::value) {
    (void)w;
    int NT, Cop, Cip;
    tc_shape(Ci, Co, &NT, &Cop, &Cip);
    __nv_bfloat16 *wk = static_cast<__nv_bfloat16 *>(n->wk);
    pack_wk<<<grid1(static_cast<int64_t>(Cop) * ks * ks * Cip), 256, 0, n->stream>>>(
        wsrc, wk, ks * ks, lci, lco, flip, Cop, Cip);
    const int64_t npix = static_cast<int64_t>(N) * H * W;
    dim3 grid(static_cast<unsigned>((npix + kTcM - 1) / kTcM), Cop / NT);
    const bool vec = xs % 8 == 0 && Ci % 8 == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0;
    if (vec && ks == 3)
      conv_fwd_tc_async<3><<<grid, kTcM, kTcAsyncSmem, n->stream>>>(
          x, xs, wk, Cip, b, y, ys, N, H, W, Ci, Co, NT, relu, n->d_err);
    else if (vec)
      conv_fwd_tc_async<1><<<grid, kTcM, kTcAsyncSmem, n->stream>>>(
          x, xs, wk, Cip, b, y, ys, N, H, W, Ci, Co, NT, relu, n->d_err);
    else if (ks == 3)
      conv_fwd_tc<3><<<grid, kTcM, kTcSmem, n->stream>>>(x, xs, wk, Cip, b, y, ys, N, H, W, Ci, Co,
                                                         NT, relu, vec, n->d_err);
    else
      conv_fwd_tc<1><<<grid, kTcM, kTcSmem, n->stream>>>(x, xs, wk, Cip, b, y, ys, N, H, W, Ci, Co,
                                                         NT, relu, vec, n->d_err);
  } else {
    (void)wsrc;
    (void)flip;
    (void)lci;
    (void)lco;
    dim3 grid(((W + TP - 1) / TP) * ((H + TP - 1) / TP), (Co + TC - 1) / TC, N);
    if (ks == 3)
      conv_fwd<A, 3><<<grid, TP * TP, 0, n->stream>>>(x, xs, w, b, y, ys, H, W, Ci, Co, relu);
    else
      conv_fwd<A, 1><<<grid, TP * TP, 0, n->stream>>>(x, xs, w, b, y, ys, H, W, Ci, Co, relu);
  }
}

template <typename A>
void launch_wgrad(const lbm_net_t *n, const A *x, int xs, const A *gz, int N, int H, int W, int Ci,
                  int Co, int ks, float *dw, float *db) {
  using namespace lbm::net;
  if constexpr (std::is_same<A, __nv_bfloat16>::value) {
    // tensor cores: M tiles over (tap, channel), N tiles over output
    // channels, the pixels split so that the grid fills the GPU a few times
    const int64_t npix = static_cast<int64_t>(N) * H * W;
    const int NT = std::min(kTcNMax, (Co + 15) / 16 * 16);
    const int mt = (ks * ks * Ci + kTcM - 1) / kTcM, nt = (Co + NT - 1) / NT;
    const int64_t want = std::max<int64_t>(1, 1824 / (mt * nt));
    int64_t kper = (npix + want - 1) / want;
    kper = std::max<int64_t>(kWgKC * 4, (kper + kWgKC - 1) / kWgKC * kWgKC);
    const unsigned ks_split = static_cast<unsigned>((npix + kper - 1) / kper);
    dim3 grid(mt, nt, ks_split);
    if (ks == 3)
      conv_wgrad_tc<3><<<grid, kTcM, kWgSmem, n->stream>>>(x, xs, gz, Co, N, H, W, Ci, Co, NT,
                                                           static_cast<int>(kper), dw, db, n->d_err);
    else
      conv_wgrad_tc<1><<<grid, kTcM, kWgSmem, n->stream>>>(x, xs, gz, Co, N, H, W, Ci, Co, NT,
                                                           static_cast<int>(kper), dw, db, n->d_err);
    return;
  }
  const int64_t npix = static_cast<int64_t>(N) * H * W;
  const int chunks = static_cast<int>(std::min<int64_t>(1024, (npix + 255) / 256));
  const int per = static_cast<int>((npix + chunks - 1) / chunks);
  dim3 grid(((Ci + TC - 1) / TC) * ((Co + TC - 1) / TC), chunks);
  if (ks == 3)
    conv_bwd_weight<A, 3><<<grid, 256, 0, n->stream>>>(x, xs, gz, N, H, W, Ci, Co, per, dw, db);
  else
    conv_bwd_weight<A, 1><<<grid, 256, 0, n->stream>>>(x, xs, gz, N, H, W, Ci, Co, per, dw, db);
}

// forward (and, if t != nullptr, loss + backward into n->grads)
template <typename A>
cudaError_t run(lbm_net_t *n, const float *x_in, int N, const float *t, float *y_out, double *loss) {
  using namespace lbm::net;
  Plan p = make_plan(n);
  const int L = n->levels;
  A *wq = static_cast<A *>(n->wq);
  auto buf = [&](int i) { return static_cast<A *>(n->bufs[i]); };
  auto gbuf = [&](int i) { return static_cast<A *>(n->bufs[p.elems.size() + i]); };
  const int64_t HW = static_cast<int64_t>(n->H) * n->W;
  cudaStream_t s = n->stream;
  to_storage<A><<<grid1(HW * N * n->c_in), 256, 0, s>>>(x_in, buf(p.x_in), HW * N * n->c_in);
  to_storage<A><<<grid1(n->n_params), 256, 0, s>>>(n->params, wq, n->n_params);
  int li = 0;
  auto W_of = [&](int k) { return wq + n->layers[k].w_off; };
  auto B_of = [&](int k) { return n->params + n->layers[k].b_off; };
  auto P_of = [&](int k) { return n->params + n->layers[k].w_off; };
  // encoder
  const A *h = buf(p.x_in);
  int hc = n->c_in;
  for (int l = 0; l < L; l++) {
    const int H = n->H >> l, Wd = n->W >> l, ch = n->base << l;
    if (l > 0) {
      pool2_fwd<A><<<grid1(static_cast<int64_t>(N) * H * Wd * hc), 256, 0, s>>>(h, hc, buf(p.pool[l]), N,
                                                                                  H * 2, Wd * 2, hc);
      h = buf(p.pool[l]);
    }
    launch_conv<A>(n, h, hc, W_of(li), B_of(li), buf(p.ea[l]), ch, N, H, Wd, hc, ch, 3, 1, P_of(li),
                   0, hc, ch);
    li++;
    launch_conv<A>(n, buf(p.ea[l]), ch, W_of(li), B_of(li), buf(p.eb[l]), ch, N, H, Wd, ch, ch, 3, 1,
                   P_of(li), 0, ch, ch);
    li++;
    h = buf(p.eb[l]);
    hc = ch;
  }
  // decoder
  for (int l = L - 2; l >= 0; l--) {
    const int H = n->H >> l, Wd = n->W >> l, ch = n->base << l;
    const int cu = hc, ct = hc + ch;
    A *cat = buf(p.cat[l]);
    up2_fwd<A><<<grid1(static_cast<int64_t>(N) * H * Wd * cu), 256, 0, s>>>(h, cat, ct, N, H, Wd, cu);
    copy_channels<A><<<grid1(static_cast<int64_t>(N) * H * Wd * ch), 256, 0, s>>>(
        buf(p.eb[l]), ch, cat + cu, ct, ch, static_cast<int64_t>(N) * H * Wd, 0);
    launch_conv<A>(n, cat, ct, W_of(li), B_of(li), buf(p.da[l]), ch, N, H, Wd, ct, ch, 3, 1, P_of(li),
                   0, ct, ch);
    li++;
    launch_conv<A>(n, buf(p.da[l]), ch, W_of(li), B_of(li), buf(p.db[l]), ch, N, H, Wd, ch, ch, 3, 1,
                   P_of(li), 0, ch, ch);
    li++;
    h = buf(p.db[l]);
    hc = ch;
  }
  const int head = li;
  launch_conv<A>(n, h, hc, W_of(head), B_of(head), buf(p.y), n->c_out, N, n->H, n->W, hc, n->c_out, 1,
                 0, P_of(head), 0, hc, n->c_out);
  if (y_out)
    to_float<A><<<grid1(HW * N * n->c_out), 256, 0, s>>>(buf(p.y), n->c_out, y_out, n->c_out, HW * N);
  if (!t) return cudaGetLastError();

  // loss and backward
  cudaMemsetAsync(n->loss, 0, sizeof(double), s);
  mse_kernel<A><<<grid1(HW * N * n->c_out), 256, 0, s>>>(buf(p.y), t, gbuf(p.y), HW * N * n->c_out,
                                                        n->loss);
  cudaMemsetAsync(n->grads, 0, n->n_params * sizeof(float), s);
  A *wt = static_cast<A *>(n->wt);
  auto conv_back = [&](int k, const A *x, int xs, A *gz, A *gx, int gxs, int H, int Wd, bool need_gx) {
    const Layer &ly = n->layers[k];
    launch_wgrad<A>(n, x, xs, gz, N, H, Wd, ly.ci, ly.co, ly.ks, n->grads + ly.w_off,
                    n->grads + ly.b_off);
    if (need_gx) {
      if constexpr (!std::is_same<A, __nv_bfloat16>::value)
        flip_weights<A><<<grid1(static_cast<int64_t>(ly.ks * ly.ks) * ly.ci * ly.co), 256, 0, s>>>(
            n->params + ly.w_off, wt, ly.ks * ly.ks, ly.ci, ly.co);
      launch_conv<A>(n, gz, ly.co, wt, nullptr, gx, gxs, N, H, Wd, ly.co, ly.ci, ly.ks, 0,
                     n->params + ly.w_off, 1, ly.ci, ly.co);
    }
  };
  // head
  {
    const Layer &ly = n->layers[head];
    (void)ly;
    conv_back(head, h, hc, gbuf(p.y), gbuf(p.db[0] >= 0 ? p.db[0] : p.eb[0]), hc, n->H, n->W, true);
  }
  // decoder backward (level 0 up to L-2)
  li = head;
  int gh_idx = p.db[0] >= 0 ? p.db[0] : p.eb[0];
  for (int l = 0; l <= L - 2; l++) {
    const int H = n->H >> l, Wd = n->W >> l, ch = n->base << l;
    const int cu = ch * 2, ct = cu + ch;
    const int kb = head - 1 - 2 * l, ka = kb - 1;
    // through d_l b
    relu_mask<A><<<grid1(static_cast<int64_t>(N) * H * Wd * ch), 256, 0, s>>>(
        gbuf(gh_idx), buf(p.db[l]), static_cast<int64_t>(N) * H * Wd * ch);
    conv_back(kb, buf(p.da[l]), ch, gbuf(gh_idx), gbuf(p.da[l]), ch, H, Wd, true);
    relu_mask<A><<<grid1(static_cast<int64_t>(N) * H * Wd * ch), 256, 0, s>>>(
        gbuf(p.da[l]), buf(p.da[l]), static_cast<int64_t>(N) * H * Wd * ch);
    conv_back(ka, buf(p.cat[l]), ct, gbuf(p.da[l]), gbuf(p.cat[l]), ct, H, Wd, true);
    // split the concat gradient: skip part into the encoder level-l output grad,
    // upsampled part into the grad of the level-(l+1) output
    copy_channels<A><<<grid1(static_cast<int64_t>(N) * H * Wd * ch), 256, 0, s>>>(
        gbuf(p.cat[l]) + cu, ct, gbuf(p.eb[l]), ch, ch, static_cast<int64_t>(N) * H * Wd, 0);
    const int up_idx = (l + 1 <= L - 2) ? p.db[l + 1] : p.eb[L - 1];
    up2_bwd<A><<<grid1(static_cast<int64_t>(N) * (H / 2) * (Wd / 2) * cu), 256, 0, s>>>(
        gbuf(p.cat[l]), ct, gbuf(up_idx), N, H, Wd, cu);
    gh_idx = up_idx;
  }
  // encoder backward (level L-1 down to 0); gbuf(eb[l]) for l < L-1 already
  // holds the skip gradient, to which the pooled-path gradient is added
  for (int l = L - 1; l >= 0; l--) {
    const int H = n->H >> l, Wd = n->W >> l, ch = n->base << l;
    const int ka = 2 * l, kb = 2 * l + 1;
    const int cin = l == 0 ? n->c_in : (n->base << (l - 1));
    relu_mask<A><<<grid1(static_cast<int64_t>(N) * H * Wd * ch), 256, 0, s>>>(
        gbuf(p.eb[l]), buf(p.eb[l]), static_cast<int64_t>(N) * H * Wd * ch);
    conv_back(kb, buf(p.ea[l]), ch, gbuf(p.eb[l]), gbuf(p.ea[l]), ch, H, Wd, true);
    relu_mask<A><<<grid1(static_cast<int64_t>(N) * H * Wd * ch), 256, 0, s>>>(
        gbuf(p.ea[l]), buf(p.ea[l]), static_cast<int64_t>(N) * H * Wd * ch);
    const A *xin = l == 0 ? buf(p.x_in) : buf(p.pool[l]);
    conv_back(ka, xin, cin, gbuf(p.ea[l]), l == 0 ? nullptr : gbuf(p.pool[l]), cin, H, Wd, l > 0);
    if (l > 0)
      pool2_bwd<A><<<grid1(static_cast<int64_t>(N) * H * 2 * Wd * 2 * cin), 256, 0, s>>>(
          gbuf(p.pool[l]), gbuf(p.eb[l - 1]), cin, N, H * 2, Wd * 2, cin, 1);
  }
  if (loss) {
    cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    *loss /= static_cast<double>(HW * N * n->c_out);
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int lbm_net_create(int32_t base, int32_t levels, int32_t c_in, int32_t c_out, int32_t precision,
                   int32_t max_batch, int32_t H, int32_t W, uint64_t seed, void *stream,
                   lbm_net_t **out) {
  g_net_error.clear();
  if (!out) return nfail(nullptr, LBM_EINVAL, "null argument");
  *out = nullptr;
  if (base < 1 || levels < 1 || levels > 8 || c_in < 1 || c_out < 1 || max_batch < 1 || H < 1 ||
      W < 1)
    return nfail(nullptr, LBM_EINVAL, "bad network shape");
  if (precision != LBM_FP32 && precision != LBM_BF16)
    return nfail(nullptr, LBM_EINVAL, "network precision must be LBM_FP32 or LBM_BF16");
  if ((H % (1 << (levels - 1))) || (W % (1 << (levels - 1))))
    return nfail(nullptr, LBM_EINVAL, "H and W must be divisible by 2^(levels-1)");
  lbm_net_t *n = new (std::nothrow) lbm_net_t();
  if (!n) return nfail(nullptr, LBM_ENOMEM, "host allocation failed");
  n->base = base;
  n->levels = levels;
  n->c_in = c_in;
  n->c_out = c_out;
  n->precision = precision;
  n->max_batch = max_batch;
  n->H = H;
  n->W = W;
  n->stream = static_cast<cudaStream_t>(stream);
  // layers in parameter order (the order of the FP64 reference)
  int64_t off = 0;
  int prev = c_in;
  int64_t max_w = 0;
  auto add = [&](int ks, int ci, int co) {
    Layer ly{ks, ci, co, off, off + static_cast<int64_t>(ks) * ks * ci * co};
    off = ly.b_off + co;
    max_w = std::max<int64_t>(max_w, static_cast<int64_t>(ks) * ks * ci * co);
    n->layers.push_back(ly);
  };
  for (int l = 0; l < levels; l++) {
    add(3, prev, base << l);
    add(3, base << l, base << l);
    prev = base << l;
  }
  for (int l = levels - 2; l >= 0; l--) {
    add(3, (base << (l + 1)) + (base << l), base << l);
    add(3, base << l, base << l);
  }
  add(1, base, c_out);
  n->n_params = off;
  Plan p = make_plan(n);
  const size_t as = asize(precision);
  cudaError_t e = cudaSuccess;
  for (float **ptr : {&n->params, &n->grads, &n->m, &n->v})
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(ptr), off * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&n->wq, off * as);
  if (e == cudaSuccess) e = cudaMalloc(&n->wt, max_w * as);
  {
    int64_t max_wk = 1;
    for (const Layer &ly : n->layers)
      for (int fl = 0; fl < 2; fl++) {
        int NT, Cop, Cip;
        tc_shape(fl ? ly.co : ly.ci, fl ? ly.ci : ly.co, &NT, &Cop, &Cip);
        max_wk = std::max<int64_t>(max_wk, static_cast<int64_t>(Cop) * ly.ks * ly.ks * Cip);
      }
    if (e == cudaSuccess) e = cudaMalloc(&n->wk, max_wk * 2);
  }
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&n->d_err), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->d_err, 0, sizeof(int));
  if (e == cudaSuccess) {
    e = cudaFuncSetAttribute(lbm::net::conv_fwd_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             lbm::net::kTcSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lbm::net::conv_fwd_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               lbm::net::kTcSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lbm::net::conv_fwd_tc_async<3>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::net::kTcAsyncSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lbm::net::conv_fwd_tc_async<1>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::net::kTcAsyncSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lbm::net::conv_wgrad_tc<3>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::net::kWgSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(lbm::net::conv_wgrad_tc<1>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, lbm::net::kWgSmem);
  }
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&n->loss), sizeof(double));
  for (int g = 0; g < 2 && e == cudaSuccess; g++)
    for (size_t i = 0; i < p.elems.size() && e == cudaSuccess; i++) {
      void *b = nullptr;
      e = cudaMalloc(&b, p.elems[i] * max_batch * as);
      n->bufs.push_back(b);
    }
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, off * sizeof(float));
  if (e == cudaSuccess) {
    // He-normal weights from a counter-based generator (splitmix64 + Box-Muller), zero biases
    std::vector<float> hp(off, 0.f);
    uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&]() {
      uint64_t z = (st += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return (static_cast<double>(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (const Layer &ly : n->layers) {
      const double sd = std::sqrt(2.0 / (ly.ks * ly.ks * ly.ci));
      for (int64_t q = ly.w_off; q < ly.b_off; q++) {
        const double u1 = next(), u2 = next();
        hp[q] = static_cast<float>(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
      }
    }
    e = cudaMemcpy(n->params, hp.data(), off * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    g_net_error = std::string("device setup: ") + cudaGetErrorString(e);
    lbm_net_destroy(n);
    return LBM_ECUDA;
  }
  *out = n;
  return LBM_OK;
}

int64_t lbm_net_num_params(const lbm_net_t *n) { return n ? n->n_params : -1; }

int lbm_net_set_params(lbm_net_t *n, const float *params, int64_t count) {
  if (!n || !params || count != n->n_params) return nfail(n, LBM_EINVAL, "parameter count mismatch");
  cudaError_t e = cudaMemcpy(n->params, params, count * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, count * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, count * sizeof(float));
  n->adam_t = 0;
  return e == cudaSuccess ? LBM_OK : nfail(n, LBM_ECUDA, cudaGetErrorString(e));
}

int lbm_net_get_params(const lbm_net_t *n, float *params, int64_t count) {
  if (!n || !params || count != n->n_params) return LBM_EINVAL;
  return cudaMemcpy(params, n->params, count * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
             ? LBM_OK
             : LBM_ECUDA;
}

int lbm_net_forward(lbm_net_t *n, const float *x, int32_t batch, float *y) {
  if (!n || !x || !y || batch < 1 || batch > n->max_batch) return nfail(n, LBM_EINVAL, "bad batch");
  cudaError_t e = n->precision == LBM_FP32
                      ? run<float>(n, x, batch, nullptr, y, nullptr)
                      : run<__nv_bfloat16>(n, x, batch, nullptr, y, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e == cudaSuccess && tc_timed_out(n))
    return nfail(n, LBM_ETIMEOUT, "a tensor-core convolution's bounded wait ran out");
  return e == cudaSuccess ? LBM_OK : nfail(n, LBM_ECUDA, cudaGetErrorString(e));
}

int lbm_net_gradients(lbm_net_t *n, const float *x, const float *t, int32_t batch, float *grads,
                      double *loss) {
  if (!n || !x || !t || batch < 1 || batch > n->max_batch) return nfail(n, LBM_EINVAL, "bad batch");
  double l = 0.0;
  cudaError_t e = n->precision == LBM_FP32 ? run<float>(n, x, batch, t, nullptr, &l)
                                           : run<__nv_bfloat16>(n, x, batch, t, nullptr, &l);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e == cudaSuccess && tc_timed_out(n))
    return nfail(n, LBM_ETIMEOUT, "a tensor-core convolution's bounded wait ran out");
  if (e == cudaSuccess && grads)
    e = cudaMemcpy(grads, n->grads, n->n_params * sizeof(float), cudaMemcpyDeviceToHost);
  if (loss) *loss = l;
  return e == cudaSuccess ? LBM_OK : nfail(n, LBM_ECUDA, cudaGetErrorString(e));
}

int lbm_net_train_step(lbm_net_t *n, const float *x, const float *t, int32_t batch, float lr,
                       double *loss) {
  int rc = lbm_net_gradients(n, x, t, batch, nullptr, loss);
  if (rc) return rc;
  n->adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, static_cast<float>(n->adam_t));
  const float c2 = 1.f - std::pow(b2, static_cast<float>(n->adam_t));
  lbm::net::adam_kernel<<<lbm::net::grid1(n->n_params), 256, 0, n->stream>>>(
      n->params, n->grads, n->m, n->v, n->n_params, lr, b1, b2, 1e-8f, c1, c2);
  cudaError_t e = cudaStreamSynchronize(n->stream);
  return e == cudaSuccess ? LBM_OK : nfail(n, LBM_ECUDA, cudaGetErrorString(e));
}

void lbm_net_destroy(lbm_net_t *n) {
  if (!n) return;
  cudaStreamSynchronize(n->stream);
  for (void *p : {static_cast<void *>(n->params), static_cast<void *>(n->grads),
                  static_cast<void *>(n->m), static_cast<void *>(n->v), n->wq, n->wt, n->wk,
                  static_cast<void *>(n->d_err), static_cast<void *>(n->loss)})
    if (p) cudaFree(p);
  for (void *b : n->bufs)
    if (b) cudaFree(b);
  delete n;
}

const char *lbm_net_last_error(const lbm_net_t *n) { return n ? n->err.c_str() : g_net_error.c_str(); }

}  // extern "C"
