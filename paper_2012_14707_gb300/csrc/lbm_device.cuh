// Device-side building blocks shared by the kernels of liblbm.so: storage
// conversion, the fused collide-stream-boundary update of one node, and the
// pieces of the FP64 reductions.
#pragma once

#include <cstdint>

#include "lbm_internal.h"

namespace lbm {
namespace dev {


// Storage of a deviation d as T and its arithmetic type C.  FP32, FP64 and
// BF16 (which keeps FP32's exponent range) store d itself; FP16 stores
// d * scale (a power of two), so loads and stores are exact apart from the
// rounding to T.  ld_raw / st_raw move the stored value itself (d * scale)
// for the step kernel, which works in storage units where the storage is
// scaled (kScaled): scaling by a power of two commutes with every rounding,
// so that is the same arithmetic without a multiplication per value.
template <typename T>
struct Stor {
  using C = T;
  static constexpr bool kScaled = false;
  static __device__ __forceinline__ C ld(T v, C) { return v; }
  static __device__ __forceinline__ T st(C v, C) { return v; }
  static __device__ __forceinline__ C ld_raw(T v) { return v; }
  static __device__ __forceinline__ T st_raw(C v) { return v; }
};
template <>
struct Stor<__half> {
  using C = float;
  static constexpr bool kScaled = true;
  static __device__ __forceinline__ float ld(__half v, float inv) { return __half2float(v) * inv; }
  static __device__ __forceinline__ __half st(float v, float sc) { return __float2half_rn(v * sc); }
  static __device__ __forceinline__ float ld_raw(__half v) { return __half2float(v); }
  static __device__ __forceinline__ __half st_raw(float v) { return __float2half_rn(v); }
};
template <>
struct Stor<__nv_bfloat16> {
  using C = float;
  // the scale of BF16 storage is always 1 (the library sets no other)
  static __device__ __forceinline__ float ld(__nv_bfloat16 v, float) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 st(float v, float) {
    return __float2bfloat16_rn(v);
  }
  static constexpr bool kScaled = false;
  static __device__ __forceinline__ float ld_raw(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 st_raw(float v) { return __float2bfloat16_rn(v); }
};


template <typename C>
__device__ __forceinline__ C recip(C v);
// FP32: the hardware approximation (within one unit in the last place; rho
// is near 1, and u enters f_eq far below the resolution of the stored
// deviations at that level).
template <>
__device__ __forceinline__ float recip<float>(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
template <>
__device__ __forceinline__ double recip<double>(double v) {
  return 1.0 / v;
}

// Post-collision state of one node: the nine values (arithmetic type and
// rounded to storage; in storage units where the storage is scaled) and
// the macroscopic quantities the links need.
template <typename T, typename C>
struct Collided {
  C o[9];
  T t[9];
  C drho, rho, ux, uy, uu;
};

// Eq. FluidMacr, Eq. MomentPost and f' = M^-1 m' for the deviations d of one
// node (in storage units, d * scale, where Stor<T>::kScaled); f'_1..f'_8
// rounded to storage, f'_0 closing the mass balance.  Every quantity that
// carries the storage scale S is computed as S times its unscaled value
// exactly (S is a power of two), so the stored results do not depend on
// the units.
template <typename T, typename C>
__device__ __forceinline__ void collide(const C (&d)[9], const StepConst<C> &k, Collided<T, C> &r) {
  constexpr bool kS = Stor<T>::kScaled;
  C(&o)[9] = r.o;
  T(&t)[9] = r.t;
  // Moments of the deviations (rows of M, Sec. 2).  M w = (1, -2, 1, 0, ...).
  const C a13 = d[1] + d[3], a24 = d[2] + d[4];
  const C d5p6 = d[5] + d[6], d7p8 = d[7] + d[8];
  const C d5m6 = d[5] - d[6], d8m7 = d[8] - d[7];
  const C s14 = a13 + a24, s58 = d5p6 + d7p8;
  const C drho_s = (d[0] + s14) + s58;
  const C e = C(2) * s58 + (C(-4) * d[0] - s14);
  const C eps = C(-2) * s14 + (C(4) * d[0] + s58);
  const C u13 = d[1] - d[3], t58 = d5m6 + d8m7;
  const C v24 = d[2] - d[4], w58 = d5p6 - d7p8;
  const C jx_s = u13 + t58, qx = C(-2) * u13 + t58;
  const C jy_s = v24 + w58, qy = C(-2) * v24 + w58;
  const C pxx = a13 - a24;
  const C pxy = d5m6 - d8m7;
  const C drho = kS ? drho_s * k.inv_sc : drho_s;
  const C jx = kS ? jx_s * k.inv_sc : jx_s, jy = kS ? jy_s * k.inv_sc : jy_s;

  // Eq. FluidMacr.
  const C rho = C(1) + drho;
  const C rax = rho * k.ax, ray = rho * k.ay;
  const C inv_rho = recip<C>(rho);
  const C ux = (jx + C(0.5) * rax) * inv_rho;
  const C uy = (jy + C(0.5) * ray) * inv_rho;
  const C uu = ux * ux + uy * uy;
  const C rux = rho * ux, ruy = rho * uy;

  // Eq. MomentPost, m' = m - S (m - m_eq) + (I - S/2) M Fbar, applied as
  // the change f' - f = M^-1 (m' - m): the collision moves f by little, and
  // adding that small change to the stored d_i rounds f'_i once (building
  // f' from the full moments costs several roundings of |f| instead; in
  // FP32 that bias adds up over thousands of steps).  M f_eq and M Fbar in
  // closed form; each row of m' - m is already scaled by its entry of
  // M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) (the
  // constants k.e2 .. k.y3 fold s and 1 - s/2 with that scale, and the
  // storage scale into the forcing weights).  Mass does not change;
  // momentum changes by rho a exactly, for any s_j, since
  // rho u = j + rho a / 2.
  const C ua6 = C(6) * (rux * k.ax + ruy * k.ay);
  const C w3 = kS ? k.w3c * rho * uu : C(3) * rho * uu;
  const C rho_s = kS ? rho * k.sc : rho;
  const C rux_s = kS ? rux * k.sc : rux, ruy_s = kS ? ruy * k.sc : ruy;
  const C e36 = k.e3 * ua6 - k.e2 * (e + C(2) * drho_s - w3);
  const C p36 = -k.p2 * (eps - drho_s + w3) - k.p3 * ua6;
  const C jx6 = rax * k.j6, jy6 = ray * k.j6;
  const C qx12 = -k.q2 * (qx + rux_s) - k.q3 * rax;
  const C qy12 = -k.q2 * (qy + ruy_s) - k.q3 * ray;
  const C xx4 = k.x3 * (rux * k.ax - ruy * k.ay) - k.x2 * (pxx - rho_s * (ux * ux - uy * uy));
  const C xy4 = k.y3 * (rux * k.ay + ruy * k.ax) - k.x2 * (pxy - rho_s * ux * uy);

  // f' - f = M^-1 (m' - m).
  const C axis = -e36 - C(2) * p36;
  const C diag = C(2) * e36 + p36;
  const C ax_x = jx6 - C(2) * qx12, ax_y = jy6 - C(2) * qy12;
  const C dg_x = jx6 + qx12, dg_y = jy6 + qy12;
  o[1] = d[1] + (axis + ax_x + xx4);
  o[2] = d[2] + (axis + ax_y - xx4);
  o[3] = d[3] + (axis - ax_x + xx4);
  o[4] = d[4] + (axis - ax_y - xx4);
  o[5] = d[5] + (diag + dg_x + dg_y + xy4);
  o[6] = d[6] + (diag - dg_x + dg_y - xy4);
  o[7] = d[7] + (diag - dg_x - dg_y + xy4);
  o[8] = d[8] + (diag + dg_x - dg_y - xy4);
  // The rest population closes the mass balance (M^-1 m' conserves sum f
  // only in exact arithmetic).  Round f'_1..f'_8 to storage first (a no-op
  // for FP32/FP64), then take their changes f'_i - f_i as stored: each is
  // the difference of two nearby values of the storage grid, exact (or
  // off by a unit of the small change), and so is their small sum.  So
  // f'_0 = f_0 - sum_{i>0} (f'_i - f_i) changes the stored mass by the one
  // rounding of f'_0 -- not by roundings of the sums of the full |f|.
  C dd[9];
#pragma unroll
  for (int i = 1; i < 9; i++) {
    if constexpr (kS) {
      t[i] = Stor<T>::st_raw(o[i]);
      o[i] = Stor<T>::ld_raw(t[i]);
    } else {
      t[i] = Stor<T>::st(o[i], k.sc);
      o[i] = Stor<T>::ld(t[i], k.inv_sc);
    }
    dd[i] = o[i] - d[i];
  }
  o[0] = d[0] - (((dd[1] + dd[2]) + (dd[3] + dd[4])) + ((dd[5] + dd[6]) + (dd[7] + dd[8])));
  if constexpr (kS)
    t[0] = Stor<T>::st_raw(o[0]);
  else
    t[0] = Stor<T>::st(o[0], k.sc);

  r.drho = drho;
  r.rho = rho;
  r.ux = ux;
  r.uy = uy;
  r.uu = uu;
}

// The unknown populations of a boundary node for the next step (bits of
// fl, its flag byte; li is its first link), Eq. EqNewBDSC in the folded
// form of LinkCoef, written to the link tail of dst (pull layout, see
// pull_slots): link k of the table has tail element 9 P + k.  Inputs: the
// node's post-collision state c and its pre-collision f_jb(x, t), gathered
// again from src at the slot the link's jbslot entry names (a cache hit;
// fewer live registers than keeping nine values through the collision).
// The link records and jbslot entries were prefetched before the
// collision.  Where the storage is scaled, every term is taken times the
// scale, so the stored value is the same.  Directions that no active lane
// of the warp needs are skipped warp-uniformly.
template <typename T, typename C>
__device__ __forceinline__ void link_epilogue_pull(const T *__restrict__ src, T *__restrict__ dst,
                                                   const PullGeom &g, const uint32_t fl,
                                                   const uint32_t li,
                                                   const LinkCoef<C> *__restrict__ links,
                                                   const Collided<T, C> &c_,
                                                   const StepConst<C> &k) {
  const unsigned wmask = __reduce_or_sync(__activemask(), fl);
  if (!wmask) return;
  constexpr bool kS = Stor<T>::kScaled;
  const C(&o)[9] = c_.o;
  const C ux = c_.ux, uy = c_.uy, uu = c_.uu;
  // in storage units (times the storage scale) where the storage is scaled
  const C drho = kS ? c_.drho * k.sc : c_.drho, rho = kS ? c_.rho * k.sc : c_.rho;
  const uint32_t tail = 9u * g.plane;
#pragma unroll
  for (int j = 1; j < 9; j++) {
    if (!(wmask & (1u << (j - 1)))) continue;
    if (fl & (1u << (j - 1))) {
      constexpr int opp_tab[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
      constexpr int cx_tab[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
      constexpr int cy_tab[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
      constexpr double w_tab[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                   1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
      const int jb = opp_tab[j];
      // link j is the node's k-th, k = links in lower directions
      const uint32_t lj = li + __popc(fl & ((1u << (j - 1)) - 1u));
      const LinkCoef<C> c = links[lj];
      const C r = c.k1 + c.k2 + c.k3;
      C c0, c2;
      if (k.diffuse_mode == 0) {
        c0 = c.alpha;
        c2 = (C(1) - r) * C(w_tab[j]);
      } else {
        c0 = c.alpha + (r - C(1)) * C(w_tab[j]);
        c2 = C(0);
      }
      const C cu = C(cx_tab[j]) * ux + C(cy_tab[j]) * uy;
      const C pj = C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu;
      const C djb = kS ? Stor<T>::ld_raw(src[g.jbslot[lj]])
                       : Stor<T>::ld(src[g.jbslot[lj]], k.inv_sc);
      const C v = c.k1 * djb + c.k2 * o[j] + c.k3 * o[jb] + (kS ? c0 * k.sc : c0) +
                  c.alpha * drho + c2 * (drho + rho * pj);
      dst[tail + lj] = kS ? Stor<T>::st_raw(v) : Stor<T>::st(v, k.sc);
    }
  }
}

// One time step for fluid node i of a lattice in the pull layout
// (pull_slots): gather f(x, t) (streaming, Sec. 2), collide (collide),
// store f'(x, t) in the node's own slots of dst, then the link epilogue.
// Used by the single-case and the batched step kernels alike.
template <typename T, typename C>
__device__ __forceinline__ void step_node_pull(const T *__restrict__ src, T *__restrict__ dst,
                                               const PullGeom &g,
                                               const LinkCoef<C> *__restrict__ links,
                                               const StepConst<C> &k, const uint32_t i) {
  const uint32_t P = g.plane;
  const uint2 nw = g.node[i];
  const int2 gr = g.grp[i / kGroup];
  C d[9];
  {
    uint32_t s[9];
    pull_slots(nw, gr, i, P, g.n_fluid, g.ny, g.periodic_y, g.rowstart, s);
#pragma unroll
    for (int q = 0; q < 9; q++)
      d[q] = Stor<T>::kScaled ? Stor<T>::ld_raw(src[s[q]]) : Stor<T>::ld(src[s[q]], k.inv_sc);
    // the link records are read after the collision: start fetching them now
    if (nw.x & 0xFFu) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(links + gr.y + node_loff(nw)));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(g.jbslot + gr.y + node_loff(nw)));
    }
  }
  Collided<T, C> c;
  collide<T, C>(d, k, c);
#pragma unroll
  for (int q = 0; q < 9; q++) dst[q * P + i] = c.t[q];
  // flag byte and first link (li) of the node
  link_epilogue_pull<T, C>(src, dst, g, nw.x & 0xFFu,
                           static_cast<uint32_t>(gr.y) + node_loff(nw), links, c, k);
}

// Eq. FluidMacr from deviations: returns rho - 1 (kept exact for the mass sum).
__device__ __forceinline__ double node_velocity(const double *d, double ax, double ay, double &rho,
                                                double &ux, double &uy) {
  double drho = 0.0, jx, jy;
  for (int i = 0; i < 9; i++) drho += d[i];
  jx = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
  jy = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
  rho = 1.0 + drho;
  ux = (jx + 0.5 * rho * ax) / rho;
  uy = (jy + 0.5 * rho * ay) / rho;
  return drho;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Residual terms of one node from its deviations now (a) and one step
// earlier (b), in arithmetic type C.  The per-population change a - b is
// exact in floating point (Sterbenz) for the small steps near steady state,
// so u^n - u^(n-1) is formed from it rather than by subtracting velocities:
//   u1 - u0 = (dj rho0 - j0 drho) / (rho0 rho1)   (the a/2 terms cancel).
template <typename C>
__device__ __forceinline__ void residual_terms(const C (&a)[9], const C (&b)[9], C ax, C ay,
                                               C &num, C &den, C &drho1) {
  C dd[9];
#pragma unroll
  for (int i = 0; i < 9; i++) dd[i] = a[i] - b[i];
  const C r0 = C(1) + (((b[0] + b[1]) + (b[2] + b[3])) + ((b[4] + b[5]) + (b[6] + b[7])) + b[8]);
  const C dr = ((dd[0] + dd[1]) + (dd[2] + dd[3])) + ((dd[4] + dd[5]) + (dd[6] + dd[7])) + dd[8];
  const C jx0 = b[1] - b[3] + (b[5] - b[6]) + (b[8] - b[7]);
  const C jy0 = b[2] - b[4] + (b[5] + b[6]) - (b[7] + b[8]);
  const C djx = dd[1] - dd[3] + (dd[5] - dd[6]) + (dd[8] - dd[7]);
  const C djy = dd[2] - dd[4] + (dd[5] + dd[6]) - (dd[7] + dd[8]);
  const C r1 = r0 + dr;
  const C inv = C(1) / (r0 * r1);
  const C dux = (djx * r0 - jx0 * dr) * inv;
  const C duy = (djy * r0 - jy0 * dr) * inv;
  const C ux1 = (jx0 + djx + C(0.5) * r1 * ax) / r1;
  const C uy1 = (jy0 + djy + C(0.5) * r1 * ay) / r1;
  num = dux * dux + duy * duy;
  den = ux1 * ux1 + uy1 * uy1;
  drho1 = r1 - C(1);
}

}  // namespace dev
}  // namespace lbm
