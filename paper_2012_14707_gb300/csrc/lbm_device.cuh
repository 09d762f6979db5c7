// Device-side building blocks shared by the kernels of liblbm.so: storage
// conversion, the fused collide-stream-boundary update of one node, and the
// pieces of the FP64 reductions.
#pragma once

#include <cstdint>
#include <type_traits>

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
  static constexpr float kMaxRaw = 65504.0f;  // largest finite FP16
  static __device__ __forceinline__ float ld(__half v, float inv) { return __half2float(v) * inv; }
  static __device__ __forceinline__ __half st(float v, float sc) { return __float2half_rn(v * sc); }
  static __device__ __forceinline__ float ld_raw(__half v) { return __half2float(v); }
  static __device__ __forceinline__ __half st_raw(float v) { return __float2half_rn(v); }
  // Two stored values by stochastic rounding (hi from a, lo from b), with
  // the random bits rb: the result is the nearest value below or above with
  // probabilities that make it exact on average.  Finite overflow saturates
  // (the residual pass counts saturated values as non-finite).
  static __device__ __forceinline__ uint32_t st_rs2(float a, float b, uint32_t rb) {
    uint32_t d;
    asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rb));
    return d;
  }
  static __device__ __forceinline__ __half bits(uint32_t h) {
    return __ushort_as_half(static_cast<unsigned short>(h));
  }
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
  static constexpr float kMaxRaw = 3.38953139e38f;  // largest finite BF16
  static __device__ __forceinline__ float ld_raw(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 st_raw(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ uint32_t st_rs2(float a, float b, uint32_t rb) {
    uint32_t d;
    asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rb));
    return d;
  }
  static __device__ __forceinline__ __nv_bfloat16 bits(uint32_t h) {
    return __ushort_as_bfloat16(static_cast<unsigned short>(h));
  }
};

// 16-bit storage rounds stochastically (Stor<T>::st_rs2): a deterministic
// rounding drops every change smaller than half a unit of the stored
// deviation, and near steady state those dropped changes are the same step
// after step, so the stored state drifts away from the exact one.
template <typename T>
constexpr bool kStochastic = std::is_same<T, __half>::value || std::is_same<T, __nv_bfloat16>::value;

// The 32-bit finaliser of MurmurHash3 (Appleby): a bijective mix in which
// every output bit depends on every input bit.  The random bits of the
// stochastic rounding are this hash of the node index and a per-step seed
// (counter-based: a step's roundings are a function of the node and the
// step count only, so runs are reproducible and a resumed run is the
// uninterrupted one).
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
// Seed of time step n (the same on the host and the device).
__host__ __device__ __forceinline__ uint32_t step_seed(int64_t n) {
  return fmix32(static_cast<uint32_t>(n) * 0x9E3779B9u + static_cast<uint32_t>(n >> 32) +
                0x7F4A7C15u);
}

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

// Two arithmetic lanes: the same quantity of two nodes (the paired 16-bit
// step), each operation one packed FP32x2 instruction of this GPU with the
// rounding of the scalar FP32 operation (a - b as fma(b, -1, a), exact).
struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ explicit F2(float2 a) : v(a) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  return F2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
template <>
__device__ __forceinline__ F2 recip<F2>(F2 v) {
  return F2(make_float2(recip<float>(v.v.x), recip<float>(v.v.y)));
}

// Post-collision state of one node: the nine values (arithmetic type and
// rounded to storage; in storage units where the storage is scaled) and
// the macroscopic quantities the links need.
template <typename T, typename C>
struct Collided {
  C o[9];
  T t[9];
  C drho, rho, ux, uy, uu;
  // the exact-mass variant (FP32 storage): rho - 1 and j in twice the
  // working precision (hi + lo), for the FP64 link values
  float dr_hi, dr_lo, jx_hi, jx_lo, jy_hi, jy_lo;
};

// Error-free sum of two FP32 values: s + e == a + b exactly (Knuth's
// TwoSum; no multiplication, so nothing is contracted into an FMA).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Sum of n FP32 values in twice the working precision (cascaded TwoSum,
// Ogita, Rump and Oishi's Sum2): s + e.
template <int N>
__device__ __forceinline__ void sum2(const float (&a)[N], float &s, float &e) {
  s = a[0];
  e = 0.0f;
#pragma unroll
  for (int i = 1; i < N; i++) {
    float t;
    two_sum(s, a[i], s, t);
    e += t;
  }
}

// a + b rounded to FP32 stochastically: the FP32 sum s (round to nearest)
// or its neighbour on the side of the exact remainder e = a + b - s
// (TwoSum, Knuth), taken with probability |e| / (spacing there), so the
// result is a + b on average.  u16: 16 random bits.
__device__ __forceinline__ float add_stochastic(float a, float b, uint32_t u16) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  if (e == 0.0f || s == 0.0f) return s;
  const int bits = __float_as_int(s);
  const float s2 = __int_as_float(((e > 0.0f) == (s > 0.0f)) ? bits + 1 : bits - 1);
  return static_cast<float>(u16) * 0x1p-16f * fabsf(s2 - s) < fabsf(e) ? s2 : s;
}

// x rounded to FP32 stochastically: the nearest FP32 value s or its
// neighbour on the side of the remainder e = x - s (exact in FP64), taken
// with probability |e| / (spacing there), so the result is x on average.
// u16: 16 random bits.
__device__ __forceinline__ float round_stochastic(double x, uint32_t u16) {
  const float s = __double2float_rn(x);
  const double e = x - static_cast<double>(s);
  if (e == 0.0 || s == 0.0f) return s;
  const int bits = __float_as_int(s);
  const float s2 = __int_as_float(((e > 0.0) == (s > 0.0f)) ? bits + 1 : bits - 1);
  return static_cast<double>(u16) * 0x1p-16 * fabs(static_cast<double>(s2) - s) < fabs(e) ? s2
                                                                                          : s;
}

// Double-FP32 values h + l with |l| <= ulp(h) / 2 (Dekker's double-length
// arithmetic, 1971): about 48 significant bits from FP32 operations alone.
// The exact-mass link values use them instead of FP64, which this GPU runs
// at a small fraction of its FP32 rate.  Products through FMA (the exact
// error of a*b is fma(a, b, -a*b)); every operation is written with the
// round-to-nearest intrinsics, so nothing is contracted or reordered.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_norm(float s, float e) {
  float h, l;
  two_sum(s, e, h, l);
  return DF{h, l};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return df_norm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  const float p = __fmul_rn(a.h, b);
  return df_norm(p, __fmaf_rn(a.l, b, __fmaf_rn(a.h, b, -p)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.h, -p);
  return df_norm(p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e)));
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const DF r = df_add(a, df_mul_f(b, -q1));  // a - q1 b
  return df_norm(q1, __fdiv_rn(r.h, b.h));
}

// The collision of Eq. MomentPost as the change ch_i = f'_i - f_i of each
// population, with the node's rho - 1, rho, u and |u|^2 (Eq. FluidMacr),
// for the deviations d of one node (C = float or double) or of two nodes at
// once (C = F2); S is the scalar type of the constants.  kS: d is in
// storage units (times the storage scale).  kGiven: rho, ux, uy are taken
// from given[0..2] instead of being formed here.
template <bool kS, bool kGiven, typename C, typename S>
__device__ __forceinline__ void collision_change(const C (&d)[9], const StepConst<S> &k,
                                                 C (&ch)[9], C &drho, C &rho, C &ux, C &uy,
                                                 C &uu, const C *given = nullptr) {
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
  drho = kS ? drho_s * k.inv_sc : drho_s;
  const C jx = kS ? jx_s * k.inv_sc : jx_s, jy = kS ? jy_s * k.inv_sc : jy_s;

  // Eq. FluidMacr.
  rho = kGiven ? given[0] : C(1) + drho;
  const C rax = rho * k.ax, ray = rho * k.ay;
  const C inv_rho = recip<C>(rho);
  ux = kGiven ? given[1] : (jx + C(0.5) * rax) * inv_rho;
  uy = kGiven ? given[2] : (jy + C(0.5) * ray) * inv_rho;
  uu = ux * ux + uy * uy;
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
  ch[0] = C(0);
  ch[1] = axis + ax_x + xx4;
  ch[2] = axis + ax_y - xx4;
  ch[3] = axis - ax_x + xx4;
  ch[4] = axis - ax_y - xx4;
  ch[5] = diag + dg_x + dg_y + xy4;
  ch[6] = diag - dg_x + dg_y - xy4;
  ch[7] = diag - dg_x - dg_y + xy4;
  ch[8] = diag + dg_x - dg_y - xy4;
}

// Eq. FluidMacr, Eq. MomentPost and f' = M^-1 m' for the deviations d of one
// node (in storage units, d * scale, where Stor<T>::kScaled); f'_1..f'_8
// rounded to storage, f'_0 closing the mass balance.  Every quantity that
// carries the storage scale S is computed as S times its unscaled value
// exactly (S is a power of two), so the stored results do not depend on
// the units.
//
// kExact (FP32 storage only): the stored mass must follow the FP64
// trajectory to ~1e-10 over thousands of steps.  A moving wall exchanges
// mass with the fluid at a rate set by the velocity next to it, so every
// rounding that leans the same way step after step shows up in the mass.
// Hence: rho - 1 and j are summed in twice the working precision (sum2),
// rho and u rounded once each (u by the correctly rounded division, no
// approximate reciprocal) for the equilibrium, and kept for the links'
// FP64 values; f'_1..f'_8 are rounded to FP32 stochastically
// (add_stochastic, random bits from rs); f'_0 closes the node's mass in
// twice the working precision plus the node's carry c0 (what FP32 storage
// dropped from its earlier values), is stored rounded to nearest, and the
// new remainder is kept in c0.  Only boundary nodes do FP64 arithmetic
// (this GPU has few FP64 units).
// 16-bit storage rounds f'_0..f'_8 stochastically with random bits from rs,
// the node's random word (fmix32 of the node index and the step seed).
template <typename T, typename C, bool kExact = false>
__device__ __forceinline__ void collide(const C (&d)[9], const StepConst<C> &k, Collided<T, C> &r,
                                        const uint32_t rs = 0, float *c0 = nullptr) {
  constexpr bool kS = Stor<T>::kScaled;
  static_assert(!kExact || std::is_same<T, float>::value, "the exact-mass variant is FP32 storage");
  C(&o)[9] = r.o;
  T(&t)[9] = r.t;
  C ch[9];
  if constexpr (kExact) {
    // rho - 1 and j in twice the working precision; rho and u rounded once
    // each (u by the correctly rounded division, no approximate reciprocal)
    sum2(d, r.dr_hi, r.dr_lo);
    const float jxs[6] = {d[1], -d[3], d[5], -d[6], -d[7], d[8]};
    const float jys[6] = {d[2], -d[4], d[5], d[6], -d[7], -d[8]};
    sum2(jxs, r.jx_hi, r.jx_lo);
    sum2(jys, r.jy_hi, r.jy_lo);
    const float rho = 1.0f + (r.dr_hi + r.dr_lo);
    const C given[3] = {rho, __fdiv_rn(r.jx_hi + (r.jx_lo + 0.5f * rho * k.ax), rho),
                        __fdiv_rn(r.jy_hi + (r.jy_lo + 0.5f * rho * k.ay), rho)};
    collision_change<kS, true>(d, k, ch, r.drho, r.rho, r.ux, r.uy, r.uu, given);
  } else {
    collision_change<kS, false>(d, k, ch, r.drho, r.rho, r.ux, r.uy, r.uu);
  }
  if constexpr (kExact) {
    const uint32_t w1 = fmix32(rs + 0x9E3779B9u), w2 = fmix32(rs + 0x3C6EF372u),
                   w3 = fmix32(rs + 0xDAA66D2Bu);
    const uint32_t u16[9] = {0u, rs & 0xFFFFu, rs >> 16, w1 & 0xFFFFu, w1 >> 16,
                             w2 & 0xFFFFu, w2 >> 16, w3 & 0xFFFFu, w3 >> 16};
#pragma unroll
    for (int i = 1; i < 9; i++) o[i] = add_stochastic(d[i], ch[i], u16[i]);
  } else {
#pragma unroll
    for (int i = 1; i < 9; i++) o[i] = d[i] + ch[i];
  }
  // The rest population closes the mass balance (M^-1 m' conserves sum f
  // only in exact arithmetic).  Round f'_1..f'_8 to storage first (a no-op
  // for FP32/FP64), then take their changes f'_i - f_i as stored: each is
  // the difference of two nearby values of the storage grid, exact (or
  // off by a unit of the small change), and so is their small sum.  So
  // f'_0 = f_0 - sum_{i>0} (f'_i - f_i) changes the stored mass by the one
  // rounding of f'_0 -- not by roundings of the sums of the full |f|.
  C dd[9];
  if constexpr (kStochastic<T>) {
    // four pairs by stochastic rounding (in storage units: o is already
    // scaled where the storage is), then the rest population
    const uint32_t w1 = fmix32(rs + 0x9E3779B9u), w2 = fmix32(rs + 0x3C6EF372u);
    const uint32_t rb[5] = {rs, w1, w2, rs ^ __funnelshift_l(w1, w1, 16),
                            w1 ^ __funnelshift_l(w2, w2, 16)};
#pragma unroll
    for (int p = 0; p < 4; p++) {
      const uint32_t h = Stor<T>::st_rs2(o[1 + 2 * p], o[2 + 2 * p], rb[p]);
      t[1 + 2 * p] = Stor<T>::bits(h >> 16);
      t[2 + 2 * p] = Stor<T>::bits(h & 0xFFFFu);
    }
#pragma unroll
    for (int i = 1; i < 9; i++) {
      o[i] = Stor<T>::ld_raw(t[i]);
      dd[i] = o[i] - d[i];
    }
    o[0] = d[0] - (((dd[1] + dd[2]) + (dd[3] + dd[4])) + ((dd[5] + dd[6]) + (dd[7] + dd[8])));
    t[0] = Stor<T>::bits(Stor<T>::st_rs2(o[0], C(0), rb[4]) >> 16);
  } else {
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
    if constexpr (kExact) {
      // f'_0 = f_0 - sum (f'_i - f_i) plus the carry, in twice the working
      // precision (the eight changes are exact FP32 values); stored rounded
      // to nearest, the remainder kept as the new carry
      const float ddv[8] = {dd[1], dd[2], dd[3], dd[4], dd[5], dd[6], dd[7], dd[8]};
      float sh, sl, vh, e1, e2;
      sum2(ddv, sh, sl);
      two_sum(d[0], -sh, vh, e1);
      two_sum(vh, (e1 - sl) + *c0, t[0], e2);
      *c0 = e2;
      o[0] = t[0];
    } else {
      o[0] = d[0] - (((dd[1] + dd[2]) + (dd[3] + dd[4])) + ((dd[5] + dd[6]) + (dd[7] + dd[8])));
      if constexpr (kS)
        t[0] = Stor<T>::st_raw(o[0]);
      else
        t[0] = Stor<T>::st(o[0], k.sc);
    }
  }

}

// Eq. EqNewBDSC for the links of the exact-mass variant (FP32 storage):
// each link value in double-FP32 arithmetic (DF) from the DF coefficients
// (g.links64) and the node's DF rho - 1, rho and u, plus the link's carry
// (what FP32 storage dropped from its earlier values); stored rounded to
// nearest, the new remainder kept as the carry.  The stored values then add
// up, step after step, to the exact ones, so the mass a moving wall
// exchanges with the fluid does not drift by a rounding that repeats.
// The links of a warp's nodes are consecutive in the link table; the warp
// spreads them over its lanes, one link per lane at a time, each reading its node's
// values from the warp's shared record.  node = the node's index i; lane
// i mod 32 of the warp runs node i, and the lanes of nodes below g.n_fluid
// (a prefix of the warp) take part -- named explicitly, since the lanes
// need not have reconverged after the collision's data-dependent branches.
constexpr int kExactMaxWarps = 8;  // CTAs of up to 256 threads

// D2Q9 velocities (two bits each: c + 1, direction j in bits 2j, 2j + 1)
// and opposite directions (four bits each: opp(j) in bits 4 (j - 1) ..
// 4 (j - 1) + 3), for the link epilogues that meet a direction as a value.
constexpr uint32_t kVelX2 = (1u << 0) | (2u << 2) | (1u << 4) | (0u << 6) | (1u << 8) |
                            (2u << 10) | (0u << 12) | (0u << 14) | (2u << 16);
constexpr uint32_t kVelY2 = (1u << 0) | (1u << 2) | (2u << 4) | (1u << 6) | (0u << 8) |
                            (2u << 10) | (2u << 12) | (0u << 14) | (0u << 16);
constexpr uint32_t kOpp2 = 0x65872143u;
__device__ __forceinline__ int vel_x2(int j) { return static_cast<int>((kVelX2 >> (2 * j)) & 3u) - 1; }
__device__ __forceinline__ int vel_y2(int j) { return static_cast<int>((kVelY2 >> (2 * j)) & 3u) - 1; }
__device__ __forceinline__ int opp2(int j) { return static_cast<int>((kOpp2 >> (4 * (j - 1))) & 15u); }
__device__ __forceinline__ void link_epilogue_exact(const float *__restrict__ src,
                                                    float *__restrict__ dst, const PullGeom &g,
                                                    const uint32_t fl, const uint32_t li,
                                                    const Collided<float, float> &c_,
                                                    const StepConst<float> &k,
                                                    const uint32_t node) {
  __shared__ float xs_o[kExactMaxWarps][8][33];   // f'_1 .. f'_8
  __shared__ float xs_n[kExactMaxWarps][10][33];  // drho, rho, ux, uy, |u|^2 (DF)
  __shared__ uint32_t xs_ex[kExactMaxWarps][32], xs_fl[kExactMaxWarps][32];
  const int lane = static_cast<int>(threadIdx.x & 31u), w = static_cast<int>(threadIdx.x >> 5);
  const uint32_t first = node - static_cast<uint32_t>(lane);
  const int nact = g.n_fluid - first >= 32u ? 32 : static_cast<int>(g.n_fluid - first);
  const unsigned am = nact == 32 ? 0xFFFFFFFFu : ((1u << nact) - 1u);
  __syncwarp(am);
  const uint32_t nl = static_cast<uint32_t>(__popc(fl));
  const unsigned anyl = __ballot_sync(am, nl != 0u);
  if (anyl == 0u) return;
  if (fl) {
    const DF drho2 = df_norm(c_.dr_hi, c_.dr_lo);
    const DF rho2 = df_add(DF{1.0f, 0.0f}, drho2);
    const DF half_rho{0.5f * rho2.h, 0.5f * rho2.l};
    const DF ux2 = df_div(df_add(df_norm(c_.jx_hi, c_.jx_lo), df_mul_f(half_rho, k.ax)), rho2);
    const DF uy2 = df_div(df_add(df_norm(c_.jy_hi, c_.jy_lo), df_mul_f(half_rho, k.ay)), rho2);
    const DF uu2 = df_add(df_mul(ux2, ux2), df_mul(uy2, uy2));
#pragma unroll
    for (int q = 1; q < 9; q++) xs_o[w][q - 1][lane] = c_.o[q];
    const float nv[10] = {drho2.h, drho2.l, rho2.h, rho2.l, ux2.h, ux2.l, uy2.h, uy2.l, uu2.h, uu2.l};
#pragma unroll
    for (int q = 0; q < 10; q++) xs_n[w][q][lane] = nv[q];
  }
  // exclusive prefix of the lanes' link counts: link t of the warp is
  // link base + t of the table
  uint32_t incl = nl;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(am, incl, off);
    if (lane >= off) incl += v;
  }
  const uint32_t excl = incl - nl, total = __shfl_sync(am, incl, nact - 1);
  const uint32_t base = __shfl_sync(am, li - excl, __ffs(static_cast<int>(anyl)) - 1);
  xs_ex[w][lane] = excl;
  xs_fl[w][lane] = fl;
  __syncwarp(am);
  const uint32_t tail = 9u * g.plane;
  constexpr float kW9h = static_cast<float>(1.0 / 9);
  constexpr float kW36h = static_cast<float>(1.0 / 36);
  const float kW9l = static_cast<float>(1.0 / 9 - static_cast<double>(kW9h));
  const float kW36l = static_cast<float>(1.0 / 36 - static_cast<double>(kW36h));
  // the nact lanes of the warp take the links in turn
  for (uint32_t t = static_cast<uint32_t>(lane); t < total; t += static_cast<uint32_t>(nact)) {
    // the node (lane s) holding link t: the last active lane whose prefix is <= t
    int s = 0;
#pragma unroll
    for (int st = 16; st >= 1; st >>= 1)
      if (s + st < nact && xs_ex[w][s + st] <= t) s += st;
    uint32_t m = xs_fl[w][s];
    for (uint32_t r = t - xs_ex[w][s]; r; r--) m &= m - 1u;
    const int j = __ffs(static_cast<int>(m));  // flag bit j - 1: direction j
    const int jb = opp2(j), cx = vel_x2(j), cy = vel_y2(j);
    const uint32_t lj = base + t;
    const LinkCoefDF c = g.links64[lj];
    const DF k1{c.hi[0], c.lo[0]}, k2{c.hi[1], c.lo[1]}, k3{c.hi[2], c.lo[2]},
        al{c.hi[3], c.lo[3]};
    const DF w2 = j < 5 ? DF{kW9h, kW9l} : DF{kW36h, kW36l};
    const DF drho2{xs_n[w][0][s], xs_n[w][1][s]}, rho2{xs_n[w][2][s], xs_n[w][3][s]};
    const DF ux2{xs_n[w][4][s], xs_n[w][5][s]}, uy2{xs_n[w][6][s], xs_n[w][7][s]};
    const DF uu2{xs_n[w][8][s], xs_n[w][9][s]};
    const DF r = df_add(df_add(k1, k2), k3);
    DF c0, c2;
    if (k.diffuse_mode == 0) {
      c0 = al;
      c2 = df_mul(df_add(DF{1.0f, 0.0f}, DF{-r.h, -r.l}), w2);
    } else {
      c0 = df_add(al, df_mul(df_add(r, DF{-1.0f, 0.0f}), w2));
      c2 = DF{0.0f, 0.0f};
    }
    // c_j . u: the components are -1, 0 or 1
    const DF cu = df_add(DF{cx * ux2.h, cx * ux2.l}, DF{cy * uy2.h, cy * uy2.l});
    const DF pj = df_add(df_add(df_mul_f(cu, 3.0f), df_mul_f(df_mul(cu, cu), 4.5f)),
                         df_mul_f(uu2, -1.5f));
    const float djb = src[g.jbslot[lj]];
    DF v = df_add(df_mul_f(k1, djb), df_mul_f(k2, xs_o[w][j - 1][s]));
    v = df_add(v, df_mul_f(k3, xs_o[w][jb - 1][s]));
    v = df_add(v, c0);
    v = df_add(v, df_mul(al, drho2));
    v = df_add(v, df_mul(c2, df_add(drho2, df_mul(rho2, pj))));
    v = df_add(v, DF{g.carry[lj], 0.0f});
    const float tv = __fadd_rn(v.h, v.l);
    g.carry[lj] = __fadd_rn(__fadd_rn(v.h, -tv), v.l);
    dst[tail + lj] = tv;
  }
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
//
// 16-bit storage rounds each value stochastically (random bits: fmix32 of
// the node's word rs and the direction).  The exact-mass variant (kExact,
// FP32 storage) runs link_epilogue_exact instead.
template <typename T, typename C, bool kExact = false>
__device__ __forceinline__ void link_epilogue_pull(const T *__restrict__ src, T *__restrict__ dst,
                                                   const PullGeom &g, const uint32_t fl,
                                                   const uint32_t li,
                                                   const LinkCoef<C> *__restrict__ links,
                                                   const Collided<T, C> &c_,
                                                   const StepConst<C> &k, const uint32_t rs = 0,
                                                   const uint32_t node = 0) {
  if constexpr (kExact) {
    link_epilogue_exact(src, dst, g, fl, li, c_, k, node);
    return;
  }
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
      if constexpr (kStochastic<T>)
        dst[tail + lj] =
            Stor<T>::bits(Stor<T>::st_rs2(v, C(0), fmix32(rs ^ (0x27D4EB2Fu * j))) >> 16);
      else
        dst[tail + lj] = kS ? Stor<T>::st_raw(v) : Stor<T>::st(v, k.sc);
    }
  }
}

// Eq. EqNewBDSC for the links of the one-node FP32 / FP64 step, spread
// over the warp as in pair_links_warp: the links of the warp's 32 nodes
// are consecutive in the table; each lane takes one link at a time and
// reads its node's values (f'_1..f'_8, drho, rho, u, |u|^2) from the
// warp's shared record.  The value is link_epilogue_pull's, rounded to
// storage the same way.  The lanes of nodes below g.n_fluid take part (a
// prefix of the warp: lane i mod 32 runs node i).  kWarps: warps per CTA.
template <typename T, typename C, int kWarps>
__device__ __forceinline__ void node_links_warp(const T *__restrict__ src, T *__restrict__ dst,
                                                const PullGeom &g, const uint32_t fl,
                                                const uint32_t li,
                                                const LinkCoef<C> *__restrict__ links,
                                                const Collided<T, C> &c_, const StepConst<C> &k,
                                                const uint32_t node) {
  static_assert(!Stor<T>::kScaled && !kStochastic<T>, "FP32 / FP64 storage");
  __shared__ C nw_v[kWarps][13][33];
  __shared__ uint32_t nw_ex[kWarps][32], nw_fl[kWarps][32];
  const int lane = static_cast<int>(threadIdx.x & 31u), w = static_cast<int>(threadIdx.x >> 5);
  const uint32_t first = node - static_cast<uint32_t>(lane);
  const int nact = g.n_fluid - first >= 32u ? 32 : static_cast<int>(g.n_fluid - first);
  const unsigned am = nact == 32 ? 0xFFFFFFFFu : ((1u << nact) - 1u);
  __syncwarp(am);
  const uint32_t nl = static_cast<uint32_t>(__popc(fl));
  const unsigned anyl = __ballot_sync(am, nl != 0u);
  if (anyl == 0u) return;
  if (fl) {
#pragma unroll
    for (int q = 1; q < 9; q++) nw_v[w][q - 1][lane] = c_.o[q];
    nw_v[w][8][lane] = c_.drho;
    nw_v[w][9][lane] = c_.rho;
    nw_v[w][10][lane] = c_.ux;
    nw_v[w][11][lane] = c_.uy;
    nw_v[w][12][lane] = c_.uu;
  }
  uint32_t incl = nl;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(am, incl, off);
    if (lane >= off) incl += v;
  }
  const uint32_t excl = incl - nl, total = __shfl_sync(am, incl, nact - 1);
  const uint32_t base = __shfl_sync(am, li - excl, __ffs(static_cast<int>(anyl)) - 1);
  nw_ex[w][lane] = excl;
  nw_fl[w][lane] = fl;
  __syncwarp(am);
  const uint32_t tail = 9u * g.plane;
  for (uint32_t t = static_cast<uint32_t>(lane); t < total; t += static_cast<uint32_t>(nact)) {
    int s = 0;
#pragma unroll
    for (int st = 16; st >= 1; st >>= 1)
      if (s + st < nact && nw_ex[w][s + st] <= t) s += st;
    uint32_t m = nw_fl[w][s];
    for (uint32_t r = t - nw_ex[w][s]; r; r--) m &= m - 1u;
    const int j = __ffs(static_cast<int>(m)), jb = opp2(j);
    const uint32_t lj = base + t;
    const LinkCoef<C> c = links[lj];
    const C wj = j < 5 ? C(1.0 / 9) : C(1.0 / 36);
    const C r = c.k1 + c.k2 + c.k3;
    C c0, c2;
    if (k.diffuse_mode == 0) {
      c0 = c.alpha;
      c2 = (C(1) - r) * wj;
    } else {
      c0 = c.alpha + (r - C(1)) * wj;
      c2 = C(0);
    }
    const C ux = nw_v[w][10][s], uy = nw_v[w][11][s], uu = nw_v[w][12][s];
    const C drho = nw_v[w][8][s], rho = nw_v[w][9][s];
    const C cu = C(vel_x2(j)) * ux + C(vel_y2(j)) * uy;
    const C pj = C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu;
    const C djb = Stor<T>::ld(src[g.jbslot[lj]], k.inv_sc);
    const C v = c.k1 * djb + c.k2 * nw_v[w][j - 1][s] + c.k3 * nw_v[w][jb - 1][s] + c0 +
                c.alpha * drho + c2 * (drho + rho * pj);
    dst[tail + lj] = Stor<T>::st(v, k.sc);
  }
}

// Random word of node i in the step whose seed is `seed` (16-bit storage
// and the exact-mass variant; 0 otherwise, unused).
template <typename T, bool kExact>
__device__ __forceinline__ uint32_t node_random(const uint32_t seed, const uint32_t i) {
  if constexpr (kStochastic<T> || kExact)
    return fmix32(i ^ seed);
  else
    return 0u;
}

// One time step for fluid node i of a lattice in the pull layout
// (pull_slots): gather f(x, t) (streaming, Sec. 2), collide (collide),
// store f'(x, t) in the node's own slots of dst, then the link epilogue.
// Used by the single-case and the batched step kernels alike; seed is the
// step's seed of random bits (step_seed of the case's step count).
template <typename T, typename C, bool kExact = false, int kWarps = 0>
__device__ __forceinline__ void step_node_pull(const T *__restrict__ src, T *__restrict__ dst,
                                               const PullGeom &g,
                                               const LinkCoef<C> *__restrict__ links,
                                               const StepConst<C> &k, const uint32_t i,
                                               const uint32_t seed) {
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
      if constexpr (kExact)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(g.links64 + gr.y + node_loff(nw)));
      else
        asm volatile("prefetch.global.L1 [%0];" ::"l"(links + gr.y + node_loff(nw)));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(g.jbslot + gr.y + node_loff(nw)));
    }
  }
  const uint32_t rs = node_random<T, kExact>(seed, i);
  Collided<T, C> c;
  if constexpr (kExact) {
    float c0 = g.carry0[i];
    collide<T, C, kExact>(d, k, c, rs, &c0);
    g.carry0[i] = c0;
  } else {
    collide<T, C, kExact>(d, k, c, rs);
  }
#pragma unroll
  for (int q = 0; q < 9; q++) dst[q * P + i] = c.t[q];
  // flag byte and first link (li) of the node
  if constexpr (!kExact && !kStochastic<T> && kWarps > 0)
    node_links_warp<T, C, kWarps>(src, dst, g, nw.x & 0xFFu,
                                  static_cast<uint32_t>(gr.y) + node_loff(nw), links, c, k, i);
  else
    link_epilogue_pull<T, C, kExact>(src, dst, g, nw.x & 0xFFu,
                                     static_cast<uint32_t>(gr.y) + node_loff(nw), links, c, k, rs,
                                     i);
}

// ---------------------------------------------------------------------------
// The paired step of 16-bit storage: one thread advances fluid nodes i0 and
// i0 + 1 (i0 even).  The 16-bit step spends its time issuing instructions,
// not waiting on memory, and a pair shares some of them: one 16-byte load
// brings both node words; the collision runs on
// both nodes at once in packed FP32x2 arithmetic (F2); each stochastic
// rounding (cvt.rs ...x2) yields the 32-bit word that holds both nodes'
// values of one population, which is their own slot pair q P + i0, q P +
// i0 + 1 -- one aligned store per population.  Random bits: fmix32 of the
// pair's first node index and the step seed (words derived by rotations).

// Unknown population j of node x (link lj of the table): Eq. EqNewBDSC in
// the folded form of LinkCoef, in the storage's units, from the node's
// post-collision values oj = f'_j, ojb = f'_jb, its pre-collision f_jb,
// drho, rho (storage units where scaled) and u.
template <typename T>
__device__ __forceinline__ float link_value(const LinkCoef<float> &c, const int j, const float djb,
                                            const float oj, const float ojb, const float drho,
                                            const float rho, const float ux, const float uy,
                                            const float uu, const StepConst<float> &k) {
  constexpr bool kS = Stor<T>::kScaled;
  constexpr int cx_tab[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int cy_tab[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  constexpr float w_tab[9] = {4.0f / 9, 1.0f / 9, 1.0f / 9, 1.0f / 9, 1.0f / 9,
                              1.0f / 36, 1.0f / 36, 1.0f / 36, 1.0f / 36};
  const float r = c.k1 + c.k2 + c.k3;
  float c0, c2;
  if (k.diffuse_mode == 0) {
    c0 = c.alpha;
    c2 = (1.0f - r) * w_tab[j];
  } else {
    c0 = c.alpha + (r - 1.0f) * w_tab[j];
    c2 = 0.0f;
  }
  const float cu = float(cx_tab[j]) * ux + float(cy_tab[j]) * uy;
  const float pj = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
  return c.k1 * djb + c.k2 * oj + c.k3 * ojb + (kS ? c0 * k.sc : c0) + c.alpha * drho +
         c2 * (drho + rho * pj);
}

// link_value for a direction j known only at run time (the same
// arithmetic; the velocity components and weight come from packed tables).
template <typename T>
__device__ __forceinline__ float link_value_rt(const LinkCoef<float> &c, const int j,
                                               const float djb, const float oj, const float ojb,
                                               const float drho, const float rho, const float ux,
                                               const float uy, const float uu,
                                               const StepConst<float> &k) {
  constexpr bool kS = Stor<T>::kScaled;
  const float w = j < 5 ? 1.0f / 9 : 1.0f / 36;
  const float r = c.k1 + c.k2 + c.k3;
  float c0, c2;
  if (k.diffuse_mode == 0) {
    c0 = c.alpha;
    c2 = (1.0f - r) * w;
  } else {
    c0 = c.alpha + (r - 1.0f) * w;
    c2 = 0.0f;
  }
  const float cu = float(vel_x2(j)) * ux + float(vel_y2(j)) * uy;
  const float pj = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
  return c.k1 * djb + c.k2 * oj + c.k3 * ojb + (kS ? c0 * k.sc : c0) + c.alpha * drho +
         c2 * (drho + rho * pj);
}

// Eq. EqNewBDSC for the links of the paired 16-bit step: the warp's 64
// nodes (lane l holds nodes 2 l and 2 l + 1 of the warp) have consecutive
// links in the table; the warp spreads them over its lanes, one link per
// lane at a time, each reading its node's values (f'_1..f'_8, drho, rho, u,
// |u|^2 in the step's units, and the node's random word) from the warp's
// shared record.  The warp's nodes are one 64-aligned block, so each link's
// entry of g.ldesc ((x mod 64) << 4 | j) names its node's column in the
// record and its direction.  Each link value is rounded stochastically with
// the random bits of its node and direction, as a node doing its own links
// would.  The lanes whose pair is complete take part (a prefix of the
// warp; a lone last node runs the one-node step instead).
constexpr int kPairMaxWarps = 4;  // CTAs of up to 128 threads
template <typename T>
__device__ __forceinline__ void pair_links_warp(const T *__restrict__ src, T *__restrict__ dst,
                                                const PullGeom &g,
                                                const LinkCoef<float> *__restrict__ links,
                                                const StepConst<float> &k, const uint32_t i0,
                                                const uint32_t fl0, const uint32_t fl1,
                                                const uint32_t li0, const uint32_t li1,
                                                const F2 (&o)[9], const F2 drho_s, const F2 rho_s,
                                                const F2 ux, const F2 uy, const F2 uu,
                                                const uint32_t h0, const uint32_t h1) {
  __shared__ float pw_v[kPairMaxWarps][13][65];
  __shared__ uint32_t pw_h[kPairMaxWarps][64];
  const int lane = static_cast<int>(threadIdx.x & 31u), w = static_cast<int>(threadIdx.x >> 5);
  const uint32_t first = i0 - 2u * static_cast<uint32_t>(lane);
  const uint32_t pairs = (g.n_fluid - first) / 2u;
  const int nact = pairs >= 32u ? 32 : static_cast<int>(pairs);
  const unsigned am = nact == 32 ? 0xFFFFFFFFu : ((1u << nact) - 1u);
  __syncwarp(am);
  const uint32_t nl = static_cast<uint32_t>(__popc(fl0)) + static_cast<uint32_t>(__popc(fl1));
  const unsigned anyl = __ballot_sync(am, nl != 0u);
  if (anyl == 0u) return;
  if (fl0) {
    const int n = 2 * lane;
#pragma unroll
    for (int q = 1; q < 9; q++) pw_v[w][q - 1][n] = o[q].v.x;
    pw_v[w][8][n] = drho_s.v.x;
    pw_v[w][9][n] = rho_s.v.x;
    pw_v[w][10][n] = ux.v.x;
    pw_v[w][11][n] = uy.v.x;
    pw_v[w][12][n] = uu.v.x;
    pw_h[w][n] = h0;
  }
  if (fl1) {
    const int n = 2 * lane + 1;
#pragma unroll
    for (int q = 1; q < 9; q++) pw_v[w][q - 1][n] = o[q].v.y;
    pw_v[w][8][n] = drho_s.v.y;
    pw_v[w][9][n] = rho_s.v.y;
    pw_v[w][10][n] = ux.v.y;
    pw_v[w][11][n] = uy.v.y;
    pw_v[w][12][n] = uu.v.y;
    pw_h[w][n] = h1;
  }
  // the warp's links are links base .. base + total - 1 of the table (its
  // first lane with links holds the first of them)
  const uint32_t total = __reduce_add_sync(am, nl);
  const uint32_t mine = fl0 ? li0 : li1;  // the lane's first link (where it has one)
  const uint32_t base = __shfl_sync(am, mine, __ffs(static_cast<int>(anyl)) - 1);
  __syncwarp(am);
  const uint32_t tail = 9u * g.plane;
  for (uint32_t t = static_cast<uint32_t>(lane); t < total; t += static_cast<uint32_t>(nact)) {
    const uint32_t lj = base + t;
    const uint32_t dsc = g.ldesc[lj];
    const int n = static_cast<int>(dsc >> 4), j = static_cast<int>(dsc & 15u), jb = opp2(j);
    const float v = link_value_rt<T>(links[lj], j, Stor<T>::ld_raw(src[g.jbslot[lj]]),
                                     pw_v[w][j - 1][n], pw_v[w][jb - 1][n], pw_v[w][8][n],
                                     pw_v[w][9][n], pw_v[w][10][n], pw_v[w][11][n],
                                     pw_v[w][12][n], k);
    dst[tail + lj] =
        Stor<T>::bits(Stor<T>::st_rs2(v, 0.0f, fmix32(pw_h[w][n] ^ (0x27D4EB2Fu * j))) >> 16);
  }
}

template <typename T>
__device__ __forceinline__ void step_pair_pull(const T *__restrict__ src, T *__restrict__ dst,
                                               const PullGeom &g,
                                               const LinkCoef<float> *__restrict__ links,
                                               const StepConst<float> &k, const uint32_t i0,
                                               const uint32_t seed) {
  static_assert(kStochastic<T>, "the paired step is the 16-bit storage step");
  const uint32_t P = g.plane;
  const uint4 nw2 = *reinterpret_cast<const uint4 *>(g.node + i0);
  const uint2 nw0 = make_uint2(nw2.x, nw2.y), nw1 = make_uint2(nw2.z, nw2.w);
  const int2 gr = g.grp[i0 / kGroup];  // i0 even: both nodes in one group
  const uint32_t m0 = nw0.x & kNodeMeta, m1 = nw1.x & kNodeMeta;
  const uint32_t fl0 = m0 & 0xFFu, fl1 = m1 & 0xFFu;
  const uint32_t li0 = static_cast<uint32_t>(gr.y) + node_loff(nw0);
  const uint32_t li1 = static_cast<uint32_t>(gr.y) + node_loff(nw1);
  F2 d[9];
  {
    uint32_t s0[9], s1[9];
    pull_slots(nw0, gr, i0, P, g.n_fluid, g.ny, g.periodic_y, g.rowstart, s0);
    pull_slots(nw1, gr, i0 + 1u, P, g.n_fluid, g.ny, g.periodic_y, g.rowstart, s1);
#pragma unroll
    for (int q = 0; q < 9; q++)
      d[q] = F2(make_float2(Stor<T>::ld_raw(src[s0[q]]), Stor<T>::ld_raw(src[s1[q]])));
    if (fl0) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(links + li0));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(g.jbslot + li0));
    }
    if (fl1) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(links + li1));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(g.jbslot + li1));
    }
  }
  constexpr bool kS = Stor<T>::kScaled;
  F2 ch[9], drho, rho, ux, uy, uu;
  collision_change<kS, false>(d, k, ch, drho, rho, ux, uy, uu);
  // random words of the pair
  const uint32_t h0 = fmix32(i0 ^ seed), h1 = fmix32(h0 + 0x9E3779B9u),
                 h2 = fmix32(h0 + 0x3C6EF372u);
  const uint32_t rb[9] = {h0,
                          h1,
                          h2,
                          h0 ^ __funnelshift_l(h1, h1, 8),
                          h1 ^ __funnelshift_l(h2, h2, 8),
                          h2 ^ __funnelshift_l(h0, h0, 8),
                          h0 ^ __funnelshift_l(h2, h2, 16),
                          h1 ^ __funnelshift_l(h0, h0, 16),
                          h2 ^ __funnelshift_l(h1, h1, 16)};
  F2 o[9];
  uint32_t t[9];
#pragma unroll
  for (int q = 1; q < 9; q++) {
    const F2 v = d[q] + ch[q];
    t[q] = Stor<T>::st_rs2(v.v.y, v.v.x, rb[q]);  // node i0 in the low half
    o[q] = F2(make_float2(Stor<T>::ld_raw(Stor<T>::bits(t[q] & 0xFFFFu)),
                          Stor<T>::ld_raw(Stor<T>::bits(t[q] >> 16))));
  }
  // the rest population closes each node's mass from the stored changes
  // (as in collide)
  {
    F2 dd[9];
#pragma unroll
    for (int q = 1; q < 9; q++) dd[q] = o[q] - d[q];
    o[0] = d[0] - (((dd[1] + dd[2]) + (dd[3] + dd[4])) + ((dd[5] + dd[6]) + (dd[7] + dd[8])));
    t[0] = Stor<T>::st_rs2(o[0].v.y, o[0].v.x, rb[0]);
  }
#pragma unroll
  for (int q = 0; q < 9; q++) *reinterpret_cast<uint32_t *>(dst + q * P + i0) = t[q];

  // boundary links of either node (Eq. EqNewBDSC is local to the node)
  const F2 drho_s = kS ? drho * k.sc : drho, rho_s = kS ? rho * k.sc : rho;
  pair_links_warp<T>(src, dst, g, links, k, i0, fl0, fl1, li0, li1, o, drho_s, rho_s, ux, uy, uu,
                     h0, h1);
}

// The exact-mass step of one node (FP32 storage) as a function of its own,
// not inlined: the single-case and the batched kernels then run bitwise the
// same compiled arithmetic (inlined into kernels with different register
// budgets, the compiler may fuse multiplies and adds differently).
static __device__ __noinline__ void step_node_exact(const float *__restrict__ src, float *__restrict__ dst,
                                             const PullGeom &g,
                                             const LinkCoef<float> *__restrict__ links,
                                             const StepConst<float> &k, const uint32_t i,
                                             const uint32_t seed) {
  step_node_pull<float, float, true>(src, dst, g, links, k, i, seed);
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
