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
// direction); the step runs one thread per fluid node from a list of the
// fluid nodes (index and flag word).  The collision works in moment space with the D3Q19 basis
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
#define LBM3_CX {0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 0, 0, 0, 0}
#define LBM3_CY {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1}
#define LBM3_CZ {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1}
#define LBM3_OPP {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15}

// component a (0 x, 1 y, 2 z) of c_q, and the opposite direction
__host__ __device__ constexpr int cvel3(int q, int a) {
  const int cx[Q] = LBM3_CX, cy[Q] = LBM3_CY, cz[Q] = LBM3_CZ;
  return a == 0 ? cx[q] : (a == 1 ? cy[q] : cz[q]);
}
__host__ __device__ constexpr int opp3(int q) {
  const int o[Q] = LBM3_OPP;
  return o[q];
}

// Moment basis of d'Humieres et al. (2002): row r evaluated at c_q.  Rows:
// rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww,
// p_xy, p_yz, p_xz, m_x, m_y, m_z.  Every entry is an integer.
__host__ __device__ constexpr int m3(int r, int q) {
  const int x = cvel3(q, 0), y = cvel3(q, 1), z = cvel3(q, 2), c2 = x * x + y * y + z * z;
  switch (r) {
    case 0: return 1;
    case 1: return 19 * c2 - 30;
    case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
    case 3: return x;
    case 4: return (5 * c2 - 9) * x;
    case 5: return y;
    case 6: return (5 * c2 - 9) * y;
    case 7: return z;
    case 8: return (5 * c2 - 9) * z;
    case 9: return 3 * x * x - c2;
    case 10: return (3 * c2 - 5) * (3 * x * x - c2);
    case 11: return y * y - z * z;
    case 12: return (3 * c2 - 5) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
  }
}

// the rows odd in c (j, q and the third-order m): m3(r, opp q) = -m3(r, q);
// the others are even
__host__ __device__ constexpr bool odd_row3(int r) { return (r >= 3 && r <= 8) || r >= 16; }

// one direction of each pair (q, opp q)
constexpr int kPairs3 = 9;
__host__ __device__ constexpr int rep3(int p) {
  const int t[kPairs3] = {1, 3, 5, 7, 8, 11, 12, 15, 16};
  return t[p];
}

constexpr int norm3(int r) {
  int s = 0;
  for (int q = 0; q < Q; q++) s += m3(r, q) * m3(r, q);
  return s;
}

// The basis is orthogonal, each row even or odd as odd_row3 says, and the
// representatives with their opposites cover directions 1..18 once.
constexpr bool basis3_ok() {
  for (int r = 0; r < Q; r++) {
    for (int s = 0; s < Q; s++) {
      int dot = 0;
      for (int q = 0; q < Q; q++) dot += m3(r, q) * m3(s, q);
      if (r != s && dot != 0) return false;
    }
    for (int q = 0; q < Q; q++)
      if (m3(r, opp3(q)) != (odd_row3(r) ? -m3(r, q) : m3(r, q))) return false;
  }
  int seen = 0;
  for (int p = 0; p < kPairs3; p++) seen |= (1 << rep3(p)) | (1 << opp3(rep3(p)));
  return seen == ((1 << Q) - 2);
}
static_assert(basis3_ok(), "D3Q19 moment basis");
static_assert(norm3(0) == 19 && norm3(1) == 2394 && norm3(2) == 252 && norm3(3) == 10 &&
                  norm3(4) == 40 && norm3(13) == 4 && norm3(16) == 8,
              "D3Q19 moment norms");

struct Lattice {
  int c[Q][3];
  int opp[Q];
  double w[Q];
  double M[Q][Q];  // moment basis, rows = moments
  double norm[Q];  // |M_k|^2
  Lattice() {
    for (int q = 0; q < Q; q++) {
      for (int a = 0; a < 3; a++) c[q][a] = cvel3(q, a);
      opp[q] = opp3(q);
      const int c2 = c[q][0] * c[q][0] + c[q][1] * c[q][1] + c[q][2] * c[q][2];
      w[q] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    for (int r = 0; r < Q; r++) {
      norm[r] = norm3(r);
      for (int q = 0; q < Q; q++) M[r][q] = m3(r, q);
    }
  }
};

const Lattice &lattice() {
  static const Lattice L;
  return L;
}

// Kernel constants of one case (passed by value): the relaxation rates
// s_k and forcing weights 1 - s_k/2 of the 19 moments, each divided by
// |M_k|^2 (the scale of M^-1 = M^T diag(1/|M_k|^2)).
template <typename C>
struct Const3 {
  C s_scaled[Q], f_scaled[Q];
  C ax, ay, az;
  int32_t nx, ny, nz, px, py, pz;
  int32_t diffuse_mode;
  int64_t plane;    // N
  int64_t n_links;  // the exact-mass variant: where the per-node carries start
  uint32_t sr_seed; // the exact-mass variant: random-bit seed of the step
};

// per link: k1, k2, k3, alpha of the folded form of Eq. EqNewBDSC (LinkCoef)
template <typename C>
struct Link3 {
  C k1, k2, k3, alpha;
};

// lattice weight of direction q
template <typename C>
__host__ __device__ constexpr C w3(int q) {
  return q == 0 ? C(1) / C(3) : (q < 7 ? C(1) / C(18) : C(1) / C(36));
}

// Coordinates of lattice node p (row-major x fastest; p < 2^31).
struct Coord3 {
  int x, y, z;
};
template <typename C>
__device__ __forceinline__ Coord3 coord3(const Const3<C> &k, int64_t p) {
  const unsigned u = static_cast<unsigned>(p), row = u / static_cast<unsigned>(k.nx);
  return Coord3{static_cast<int>(u - row * static_cast<unsigned>(k.nx)),
                static_cast<int>(row % static_cast<unsigned>(k.ny)),
                static_cast<int>(row / static_cast<unsigned>(k.ny))};
}

// Slot of f_q(x, t) for node p (pull layout): the neighbour x - c_q's own
// slot, or the node's tail element when x - c_q is solid.  A coordinate
// that leaves the lattice wraps (periodic axis); on a walled axis the link
// flag is set there, so the wrapped value is never used.
template <typename C>
__device__ __forceinline__ int64_t pull_slot3(const Const3<C> &k, int q, Coord3 c, uint32_t fl,
                                              uint32_t lbase, int64_t N) {
  if (fl & (1u << q)) return 19 * N + lbase + __popc(fl & ((1u << q) - 1u));
  int xs = c.x - cvel3(q, 0), ys = c.y - cvel3(q, 1), zs = c.z - cvel3(q, 2);
  xs += xs < 0 ? k.nx : (xs >= k.nx ? -k.nx : 0);
  ys += ys < 0 ? k.ny : (ys >= k.ny ? -k.ny : 0);
  zs += zs < 0 ? k.nz : (zs >= k.nz ? -k.nz : 0);
  return static_cast<int64_t>(q) * N + (static_cast<int64_t>(zs) * k.ny + ys) * k.nx + xs;
}

// acc + m x for a compile-time integer m (zero terms vanish, +-1 add)
template <typename C>
__device__ __forceinline__ C mac3(C acc, int m, C x) {
  return m == 0 ? acc : (m == 1 ? acc + x : (m == -1 ? acc - x : fma(C(m), x, acc)));
}

// Runtime forms of the velocity components and of the opposite direction
// (the link epilogue meets each direction as a value): two bits per
// direction hold c + 1.
constexpr uint64_t pack_c3(int a) {
  uint64_t t = 0;
  for (int q = 0; q < Q; q++) t |= static_cast<uint64_t>(cvel3(q, a) + 1) << (2 * q);
  return t;
}
constexpr uint64_t kPackX3 = pack_c3(0), kPackY3 = pack_c3(1), kPackZ3 = pack_c3(2);
__device__ __forceinline__ int cvel3_rt(int q, int a) {
  const uint64_t t = a == 0 ? kPackX3 : (a == 1 ? kPackY3 : kPackZ3);
  return static_cast<int>((t >> (2 * q)) & 3u) - 1;
}
__host__ __device__ constexpr int opp3_rt(int j) {
  return j <= 6 ? ((j - 1) ^ 1) + 1 : j + 3 - 2 * ((j - 7) & 3);
}
constexpr bool opp3_rt_ok() {
  for (int q = 1; q < Q; q++)
    if (opp3_rt(q) != opp3(q)) return false;
  return true;
}
static_assert(opp3_rt_ok(), "opposite directions");

// What the links of a boundary node read of it, one column per lane of a
// warp: f'_q (rows 0..17, q = 1..18), f_q (rows 18..35), drho, rho, u_x,
// u_y, u_z (rows 36..40); 33 columns so that a lane's rows fall in
// different banks.
constexpr int kLinkVals3 = 2 * (Q - 1) + 5;
template <typename C>
struct Warp3 {
  C v[kLinkVals3][33];
};

// Double-FP32 numbers (about 48 significant bits from FP32 operations) with
// the arithmetic operators, so that the exact-mass variant's moments
// (exact_moments3) read as the FP32 code does and mac3 serves them too.
// This GPU runs FP64 at a small fraction of its FP32 rate; the operations
// are those of lbm::dev::DF.  Its own namespace keeps its fma out of the
// ordinary lookup of float and double code (argument-dependent lookup finds
// it for D2).
namespace df {
struct D2 {
  float h, l;
  D2() = default;
  __host__ __device__ constexpr D2(float hi, float lo) : h(hi), l(lo) {}
  __host__ __device__ explicit constexpr D2(double x)
      : h(static_cast<float>(x)), l(static_cast<float>(x - static_cast<double>(static_cast<float>(x)))) {}
};
__device__ __forceinline__ lbm::dev::DF dv(D2 a) { return lbm::dev::DF{a.h, a.l}; }
__device__ __forceinline__ D2 d2(lbm::dev::DF a) { return D2(a.h, a.l); }
__device__ __forceinline__ D2 operator+(D2 a, D2 b) { return d2(lbm::dev::df_add(dv(a), dv(b))); }
__device__ __forceinline__ D2 operator-(D2 a, D2 b) {
  return d2(lbm::dev::df_add(dv(a), lbm::dev::DF{-b.h, -b.l}));
}
__device__ __forceinline__ D2 operator*(D2 a, D2 b) { return d2(lbm::dev::df_mul(dv(a), dv(b))); }
__device__ __forceinline__ D2 operator/(D2 a, D2 b) { return d2(lbm::dev::df_div(dv(a), dv(b))); }
__device__ __forceinline__ D2 &operator+=(D2 &a, D2 b) { return a = a + b; }
__device__ __forceinline__ D2 fma(D2 a, D2 b, D2 c) { return a * b + c; }
}  // namespace df
using df::D2;

// lattice weight of direction q in the arithmetic type A
template <typename A>
__device__ __forceinline__ A wq3(int q) {
  return w3<A>(q);
}
template <>
__device__ __forceinline__ D2 wq3<D2>(int q) {
  return D2(q == 0 ? 1.0 / 3.0 : (q < 7 ? 1.0 / 18.0 : 1.0 / 36.0));
}

template <typename A>
__device__ __forceinline__ void transform3(const A n0, const A F0, const A (&NS)[kPairs3],
                                           const A (&NA)[kPairs3], const A (&FS)[kPairs3],
                                           const A (&FA)[kPairs3], const Const3<A> &k,
                                           A (&ch)[Q]);

// The collision change f' - f of one node from its deviations d (Eq.
// FluidMacr, Eq. LBEequi, Eq. LBEforce, Eq. MomentPost through M^-1), in
// the arithmetic type A: ch[1..18] (f'_0 closes the mass instead), and the
// node's rho - 1, rho and u.  It runs on the pairs (q, opp q): d_q + d_opp
// carries the even moments and d_q - d_opp the odd ones, so each row of M
// touches at most ten values and, M being integer and known here at compile
// time, only its non-zero entries cost an instruction.
template <typename A>
__device__ __forceinline__ void collide3(const A (&d)[Q], const Const3<A> &k, A &drho, A &rho,
                                         A (&u)[3], A (&ch)[Q]) {
  // Eq. FluidMacr on the pair sums and differences
  A S[kPairs3], D[kPairs3];
  drho = d[0];
#pragma unroll
  for (int pp = 0; pp < kPairs3; pp++) {
    S[pp] = d[rep3(pp)] + d[opp3(rep3(pp))];
    D[pp] = d[rep3(pp)] - d[opp3(rep3(pp))];
    drho += S[pp];
  }
  A j[3] = {A(0), A(0), A(0)};
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int pp = 0; pp < kPairs3; pp++) j[a] = mac3(j[a], cvel3(rep3(pp), a), D[pp]);
  rho = A(1) + drho;
  u[0] = (j[0] + A(0.5) * rho * k.ax) / rho;
  u[1] = (j[1] + A(0.5) * rho * k.ay) / rho;
  u[2] = (j[2] + A(0.5) * rho * k.az) / rho;
  const A ux = u[0], uy = u[1], uz = u[2];
  const A uu = ux * ux + uy * uy + uz * uz, ua = ux * k.ax + uy * k.ay + uz * k.az;
  // d - d_eq (Eq. LBEequi) and Fbar (Eq. LBEforce), as pair sums (S) and
  // differences (A); the rest direction alone
  A NS[kPairs3], NA[kPairs3], FS[kPairs3], FA[kPairs3];
  const A n0 = d[0] - wq3<A>(0) * (drho - A(1.5) * rho * uu);
  const A F0 = A(-3) * wq3<A>(0) * rho * ua;
#pragma unroll
  for (int pp = 0; pp < kPairs3; pp++) {
    const int q = rep3(pp);
    const A cu = mac3(mac3(mac3(A(0), cvel3(q, 0), ux), cvel3(q, 1), uy), cvel3(q, 2), uz);
    const A ca = mac3(mac3(mac3(A(0), cvel3(q, 0), k.ax), cvel3(q, 1), k.ay), cvel3(q, 2), k.az);
    const A wr = wq3<A>(q) * rho;
    NS[pp] = S[pp] - A(2) * wq3<A>(q) * (drho + rho * (A(4.5) * cu * cu - A(1.5) * uu));
    NA[pp] = D[pp] - A(6) * wr * cu;
    FS[pp] = A(2) * wr * (A(9) * cu * ca - A(3) * ua);
    FA[pp] = A(6) * wr * ca;
  }
  transform3<A>(n0, F0, NS, NA, FS, FA, k, ch);
}

// The second half of the collision: from d - d_eq and Fbar as pair sums
// (NS, FS) and differences (NA, FA) plus the rest direction's (n0, F0), the
// change ch[q] = f'_q - f_q (ch[0] = 0).
template <typename A>
__device__ __forceinline__ void transform3(const A n0, const A F0, const A (&NS)[kPairs3],
                                           const A (&NA)[kPairs3], const A (&FS)[kPairs3],
                                           const A (&FA)[kPairs3], const Const3<A> &k,
                                           A (&ch)[Q]) {
  // m' - m = -s (m - m_eq) + (1 - s/2) M Fbar, scaled by 1/|M_k|^2
  A dm[Q];
#pragma unroll
  for (int r = 0; r < Q; r++) {
    A a = A(0), b = A(0);
    if (!odd_row3(r)) {
      a = mac3(a, m3(r, 0), n0);
      b = mac3(b, m3(r, 0), F0);
    }
#pragma unroll
    for (int pp = 0; pp < kPairs3; pp++) {
      a = mac3(a, m3(r, rep3(pp)), odd_row3(r) ? NA[pp] : NS[pp]);
      b = mac3(b, m3(r, rep3(pp)), odd_row3(r) ? FA[pp] : FS[pp]);
    }
    dm[r] = k.f_scaled[r] * b - k.s_scaled[r] * a;
  }
  // f' - f = M^T dm: even rows give the same change to q and opp q, odd
  // rows opposite ones
  ch[0] = A(0);
#pragma unroll
  for (int pp = 0; pp < kPairs3; pp++) {
    const int q = rep3(pp), qb = opp3(q);
    A ev = A(0), od = A(0);
#pragma unroll
    for (int r = 0; r < Q; r++) {
      if (odd_row3(r)) od = mac3(od, m3(r, q), dm[r]);
      else ev = mac3(ev, m3(r, q), dm[r]);
    }
    ch[q] = ev + od;
    ch[qb] = ev - od;
  }
}

// The exact-mass variant's first half of the collision (FP32 storage).  The
// pair sums and d_eq are ~100 times their difference d - d_eq, so the FP32
// rounding errors of the former become relative errors of ~1e-5 of the
// latter, and in a steady flow they repeat every step; so rho - 1, j, rho,
// u and d - d_eq are formed in double-FP32 (the pair sums exactly, by
// TwoSum) and d - d_eq is rounded once to FP32 for the transform.  Fbar,
// proportional to the body force and orders of magnitude smaller, stays in
// FP32.  rho - 1, rho and u are returned in double-FP32 for the links.
__device__ __forceinline__ float to_f(D2 x) { return __fadd_rn(x.h, x.l); }
__device__ __forceinline__ void exact_moments3(const float (&d)[Q], const Const3<D2> &kd, D2 &drho,
                                               D2 &rho, D2 (&u)[3], float &n0, float &F0,
                                               float (&NS)[kPairs3], float (&NA)[kPairs3],
                                               float (&FS)[kPairs3], float (&FA)[kPairs3]) {
  D2 S[kPairs3], Dd[kPairs3];
  drho = D2(d[0], 0.0f);
#pragma unroll
  for (int pp = 0; pp < kPairs3; pp++) {
    const int q = rep3(pp), qb = opp3(q);
    float h, l;
    lbm::dev::two_sum(d[q], d[qb], h, l);
    S[pp] = D2(h, l);
    lbm::dev::two_sum(d[q], -d[qb], h, l);
    Dd[pp] = D2(h, l);
    drho += S[pp];
  }
  D2 j[3] = {D2(0.0f, 0.0f), D2(0.0f, 0.0f), D2(0.0f, 0.0f)};
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int pp = 0; pp < kPairs3; pp++) j[a] = mac3(j[a], cvel3(rep3(pp), a), Dd[pp]);
  rho = D2(1.0f, 0.0f) + drho;
  const D2 acc[3] = {kd.ax, kd.ay, kd.az};
#pragma unroll
  for (int a = 0; a < 3; a++) u[a] = (j[a] + D2(0.5f, 0.0f) * rho * acc[a]) / rho;
  const D2 uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const float rf = rho.h, uaf = u[0].h * kd.ax.h + u[1].h * kd.ay.h + u[2].h * kd.az.h;
  n0 = to_f(D2(d[0], 0.0f) - wq3<D2>(0) * (drho - D2(1.5) * rho * uu));
  F0 = -3.0f * w3<float>(0) * rf * uaf;
  // one pair per iteration, not unrolled: the double-FP32 body is long, and
  // nine copies of it would overflow the instruction cache
#pragma unroll 1
  for (int pp = 0; pp < kPairs3; pp++) {
    const int q = rep3(pp);
    D2 cu(0.0f, 0.0f);
    float caf = 0.0f;
    const float ka[3] = {kd.ax.h, kd.ay.h, kd.az.h};
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const int c = cvel3_rt(q, a);
      if (c > 0) {
        cu = cu + u[a];
        caf += ka[a];
      } else if (c < 0) {
        cu = cu - u[a];
        caf -= ka[a];
      }
    }
    const D2 wq = wq3<D2>(q);
    NS[pp] = to_f(S[pp] - D2(2.0) * wq * (drho + rho * (D2(4.5) * cu * cu - D2(1.5) * uu)));
    NA[pp] = to_f(Dd[pp] - D2(6.0) * wq * rho * cu);
    const float wrf = w3<float>(q) * rf;
    FS[pp] = 2.0f * wrf * (9.0f * cu.h * caf - 3.0f * uaf);
    FA[pp] = 6.0f * wrf * caf;
  }
}

// The exact-mass variant's extra record per warp: rho - 1, rho, u_x, u_y,
// u_z of each boundary node in double-FP32 (pairs of rows).
struct Warp3X {
  float v[10][33];
};

// Gather, collide and store one fluid node (pull layout); a boundary node
// leaves what its links need in the warp's shared record.
//
// kExact (FP32 storage): the stored mass must follow the FP64 trajectory to
// ~1e-10 over thousands of steps where walls move, and a moving wall
// exchanges mass at a rate set by the populations next to it.  Any rounding
// that leans the same way step after step shifts that rate: the storage
// rounding of f' (round to nearest), and equally the FP32 arithmetic of the
// collision, whose rounding errors repeat every step once the flow is
// steady.  So d - d_eq is formed in double-FP32 (exact_moments3; kd: the
// body force as double-FP32 pairs) before the FP32 transform to f' - f,
// f'_1..f'_18 are rounded to FP32 stochastically, and f'_0 closes the
// node's mass in double-FP32 plus the node's carry c0 (what FP32 storage
// dropped from its earlier values); stored rounded to nearest, the new
// remainder is kept in c0.
template <typename C, bool kExact = false>
__device__ __forceinline__ void node3(const C *__restrict__ src, C *__restrict__ dst,
                                      const Const3<C> &k, const int64_t p, const uint32_t fl,
                                      const uint32_t lb, Warp3<C> &sh, const int lane,
                                      float *c0 = nullptr, const uint32_t rs = 0u,
                                      Warp3X *shx = nullptr, const Const3<D2> *kd = nullptr) {
  const int64_t N = k.plane;
  const Coord3 c = coord3(k, p);
  C d[Q];
  {
    // x - c_q from the wrapped coordinates, or the node's tail element
    // where x - c_q is solid (a select, so interior and boundary nodes run
    // the same instructions; on a walled axis the wrapped value is unused)
    const int xw[3] = {c.x + 1 < k.nx ? c.x + 1 : 0, c.x, c.x > 0 ? c.x - 1 : k.nx - 1};
    const int yw[3] = {c.y + 1 < k.ny ? c.y + 1 : 0, c.y, c.y > 0 ? c.y - 1 : k.ny - 1};
    const int zw[3] = {c.z + 1 < k.nz ? c.z + 1 : 0, c.z, c.z > 0 ? c.z - 1 : k.nz - 1};
    const int64_t sx = k.nx, sxy = static_cast<int64_t>(k.nx) * k.ny;
    const int64_t tail = 19 * N + lb;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int64_t nb = q * N + zw[cvel3(q, 2) + 1] * sxy + yw[cvel3(q, 1) + 1] * sx +
                         xw[cvel3(q, 0) + 1];
      const int64_t tq = tail + __popc(fl & ((1u << q) - 1u));
      d[q] = src[(fl >> q) & 1u ? tq : nb];
    }
  }
  C o[Q];
  if constexpr (kExact) {
    static_assert(std::is_same<C, float>::value, "the exact-mass variant is FP32 storage");
    D2 drx, rhx, ux3[3];
    float n0, F0, NS[kPairs3], NA[kPairs3], FS[kPairs3], FA[kPairs3], ch[Q];
    exact_moments3(d, *kd, drx, rhx, ux3, n0, F0, NS, NA, FS, FA);
    transform3<float>(n0, F0, NS, NA, FS, FA, k, ch);
    // f'_q = f_q + ch_q rounded to FP32 stochastically (16 random bits
    // each: the halves of the node's nine random words)
    uint32_t rw[kPairs3];
    rw[0] = lbm::dev::fmix32(rs);
#pragma unroll
    for (int pp = 1; pp < kPairs3; pp++) rw[pp] = lbm::dev::fmix32(rw[0] + 0x9E3779B9u * pp);
#pragma unroll
    for (int pp = 0; pp < kPairs3; pp++) {
      const int q = rep3(pp), qb = opp3(q);
      o[q] = lbm::dev::add_stochastic(d[q], ch[q], rw[pp] & 0xFFFFu);
      o[qb] = lbm::dev::add_stochastic(d[qb], ch[qb], rw[(pp + 4) % kPairs3] >> 16);
    }
    // f'_0 = f_0 - sum (f'_q - f_q) plus the carry, in double-FP32 (each
    // change is the exact difference of two FP32 values); stored rounded to
    // nearest, the remainder kept
    D2 sum(0.0f, 0.0f);
#pragma unroll
    for (int q = 1; q < Q; q++) {
      float h, l;
      lbm::dev::two_sum(o[q], -d[q], h, l);
      sum += D2(h, l);
    }
    const D2 v0 = (D2(d[0], 0.0f) - sum) + D2(*c0, 0.0f);
    float e0;
    lbm::dev::two_sum(v0.h, v0.l, o[0], e0);
    *c0 = e0;
#pragma unroll
    for (int q = 0; q < Q; q++) dst[q * N + p] = o[q];
    if (fl) {
#pragma unroll
      for (int q = 1; q < Q; q++) {
        sh.v[q - 1][lane] = o[q];
        sh.v[Q - 2 + q][lane] = d[q];
      }
      // rho - 1, rho and u as pairs of FP32 values for the links
      const D2 nv[5] = {drx, rhx, ux3[0], ux3[1], ux3[2]};
#pragma unroll
      for (int i = 0; i < 5; i++) {
        shx->v[2 * i][lane] = nv[i].h;
        shx->v[2 * i + 1][lane] = nv[i].l;
      }
    }
  } else {
    C drho, rho, u[3], ch[Q];
    collide3<C>(d, k, drho, rho, u, ch);
    // f'_0 closes the mass from the stored changes
    C sum = C(0);
#pragma unroll
    for (int pp = 0; pp < kPairs3; pp++) {
      const int q = rep3(pp), qb = opp3(q);
      o[q] = d[q] + ch[q];
      o[qb] = d[qb] + ch[qb];
      sum += (o[q] - d[q]) + (o[qb] - d[qb]);
    }
    o[0] = d[0] - sum;
#pragma unroll
    for (int q = 0; q < Q; q++) dst[q * N + p] = o[q];
    if (fl) {
#pragma unroll
      for (int q = 1; q < Q; q++) {
        sh.v[q - 1][lane] = o[q];
        sh.v[Q - 2 + q][lane] = d[q];
      }
      sh.v[36][lane] = drho;
      sh.v[37][lane] = rho;
      sh.v[38][lane] = u[0];
      sh.v[39][lane] = u[1];
      sh.v[40][lane] = u[2];
    }
  }
}

// One lattice step of every fluid node, then Eq. EqNewBDSC for every
// boundary link of the step's nodes into the lattice's tail.  The links of
// a warp's 32 nodes are consecutive in the link table (sorted by node); the
// warp spreads them over its lanes, one link per lane, each reading its
// node's values from the warp's shared record -- the links of a node
// cluster would otherwise run direction by direction on few lanes.
// kExact: 80 registers and 6 CTAs per SM (issue-bound; 4 and 5 CTAs per SM
// measured 2 to 4 % slower).
template <typename C, bool kExact = false>
__global__ void __launch_bounds__(kThreads3, kExact ? 6 : (sizeof(C) == 4 ? 8 : 2))
step3_kernel(const C *__restrict__ src, C *__restrict__ dst, const uint32_t *__restrict__ flags,
             const uint32_t *__restrict__ lbase, const Link3<C> *__restrict__ links,
             const uint2 *__restrict__ fluid, const __grid_constant__ Const3<C> k, int64_t n_fluid,
             const lbm::LinkCoefDF *__restrict__ links_df = nullptr, float *carry = nullptr,
             const __grid_constant__ Const3<D2> kd = Const3<D2>()) {
  constexpr int kW = kThreads3 / 32;
  __shared__ Warp3<C> sh[kW];
  __shared__ Warp3X shx[kExact ? kW : 1];
  __shared__ uint32_t sh_ex[kW][32], sh_fl[kW][32];
  // thread t of the launch runs the t-th fluid node (node order), so no
  // lane idles on a solid node
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int lane = static_cast<int>(threadIdx.x & 31u), w = static_cast<int>(threadIdx.x >> 5);
  // the fluid-node list holds each node's index and flag word together
  const uint2 pf = t0 < n_fluid ? fluid[t0] : make_uint2(0u, kSolid3);
  const int64_t p = pf.x;
  const uint32_t fl = pf.y;
  const bool live = fl != kSolid3;
  const uint32_t lb = live && fl ? lbase[p] : 0u;
  // the exact-mass variant's carries: one per link, then one per fluid node
  float *carry0 = kExact ? carry + k.n_links : nullptr;
  if (live) {
    if constexpr (kExact)
      node3<C, true>(src, dst, k, p, fl, lb, sh[w], lane, carry0 + t0,
                     static_cast<uint32_t>(t0) ^ k.sr_seed, &shx[w], &kd);
    else
      node3<C, false>(src, dst, k, p, fl, lb, sh[w], lane);
  }
  const uint32_t nl = live ? static_cast<uint32_t>(__popc(fl)) : 0u;
  const unsigned any = __ballot_sync(0xFFFFFFFFu, nl != 0u);
  if (any == 0u) return;
  // exclusive prefix of the lanes' link counts; link t of the warp is link
  // base + t of the table
  uint32_t incl = nl;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl += v;
  }
  const uint32_t excl = incl - nl, total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  const uint32_t base = __shfl_sync(0xFFFFFFFFu, lb - excl, __ffs(static_cast<int>(any)) - 1);
  sh_ex[w][lane] = excl;
  sh_fl[w][lane] = live ? fl : 0u;
  __syncwarp();
  const Warp3<C> &ws = sh[w];
  for (uint32_t t = static_cast<uint32_t>(lane); t < total; t += 32u) {
    // the node (lane s) holding link t: the last lane whose prefix is <= t
    int s = 0;
#pragma unroll
    for (int st = 16; st >= 1; st >>= 1)
      if (sh_ex[w][s + st] <= t) s += st;
    uint32_t m = sh_fl[w][s];
    for (uint32_t r = t - sh_ex[w][s]; r; r--) m &= m - 1u;
    const int j = __ffs(static_cast<int>(m)) - 1, jb = opp3_rt(j);
    const C oj = ws.v[j - 1][s], ojb = ws.v[jb - 1][s], djb = ws.v[Q - 2 + jb][s];
    if constexpr (kExact) {
      // Eq. EqNewBDSC in double-FP32 from the pairs of the FP64
      // coefficients and the node's double-FP32 rho - 1, rho, u, plus the
      // link's carry; stored rounded to nearest, the remainder kept
      using lbm::dev::DF;
      using lbm::dev::df_add;
      using lbm::dev::df_mul;
      using lbm::dev::df_mul_f;
      const Warp3X &wx = shx[w];
      const lbm::LinkCoefDF c = links_df[base + t];
      const DF k1{c.hi[0], c.lo[0]}, k2{c.hi[1], c.lo[1]}, k3{c.hi[2], c.lo[2]},
          al{c.hi[3], c.lo[3]};
      const double wd = j < 7 ? 1.0 / 18 : 1.0 / 36;
      const DF w2{static_cast<float>(wd), static_cast<float>(wd - static_cast<float>(wd))};
      const DF drho2{wx.v[0][s], wx.v[1][s]}, rho2{wx.v[2][s], wx.v[3][s]};
      const DF u2[3] = {{wx.v[4][s], wx.v[5][s]}, {wx.v[6][s], wx.v[7][s]}, {wx.v[8][s], wx.v[9][s]}};
      const DF uu2 = df_add(df_add(df_mul(u2[0], u2[0]), df_mul(u2[1], u2[1])), df_mul(u2[2], u2[2]));
      const DF r = df_add(df_add(k1, k2), k3);
      DF c0, c2;
      if (k.diffuse_mode == 0) {
        c0 = al;
        c2 = df_mul(df_add(DF{1.0f, 0.0f}, DF{-r.h, -r.l}), w2);
      } else {
        c0 = df_add(al, df_mul(df_add(r, DF{-1.0f, 0.0f}), w2));
        c2 = DF{0.0f, 0.0f};
      }
      DF cu{0.0f, 0.0f};
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const float ca = static_cast<float>(cvel3_rt(j, a));
        cu = df_add(cu, DF{ca * u2[a].h, ca * u2[a].l});
      }
      const DF pj = df_add(df_add(df_mul_f(cu, 3.0f), df_mul_f(df_mul(cu, cu), 4.5f)),
                           df_mul_f(uu2, -1.5f));
      DF v = df_add(df_mul_f(k1, djb), df_mul_f(k2, oj));
      v = df_add(v, df_mul_f(k3, ojb));
      v = df_add(v, c0);
      v = df_add(v, df_mul(al, drho2));
      v = df_add(v, df_mul(c2, df_add(drho2, df_mul(rho2, pj))));
      v = df_add(v, DF{carry[base + t], 0.0f});
      const float tv = __fadd_rn(v.h, v.l);
      carry[base + t] = __fadd_rn(__fadd_rn(v.h, -tv), v.l);
      dst[19 * k.plane + base + t] = tv;
    } else {
      const Link3<C> cl = links[base + t];
      const C drho = ws.v[36][s], rho = ws.v[37][s], ux = ws.v[38][s], uy = ws.v[39][s],
              uz = ws.v[40][s];
      const C uu = ux * ux + uy * uy + uz * uz;
      const C wj = j < 7 ? C(1) / C(18) : C(1) / C(36);
      const C r = cl.k1 + cl.k2 + cl.k3;
      C c0, c2;
      if (k.diffuse_mode == 0) {
        c0 = cl.alpha;
        c2 = (C(1) - r) * wj;
      } else {
        c0 = cl.alpha + (r - C(1)) * wj;
        c2 = C(0);
      }
      const C cu = C(cvel3_rt(j, 0)) * ux + C(cvel3_rt(j, 1)) * uy + C(cvel3_rt(j, 2)) * uz;
      const C pj = C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu;
      dst[19 * k.plane + base + t] = cl.k1 * djb + cl.k2 * oj + cl.k3 * ojb + c0 +
                                     cl.alpha * drho + c2 * (drho + rho * pj);
    }
  }
}

// Residual pass (FP64 sums, fixed grid and order): num, den, mass
// deviation, non-finite count of the states in cur and prev.
template <typename C>
__global__ void __launch_bounds__(kResThreads3)
residual3_kernel(const C *__restrict__ cur, const C *__restrict__ prev,
                 const uint32_t *__restrict__ flags, const uint32_t *__restrict__ lbase,
                 const uint2 *__restrict__ fluid, const Const3<C> k, int64_t n_fluid,
                 double *__restrict__ partials) {
  // per node: rho and j of both states in the storage's arithmetic type,
  // the node's mass deviation summed in FP64; sums over nodes in FP64
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t G = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n_fluid;
       t += G) {
    const uint2 pf = fluid[t];
    const int64_t p = pf.x;
    const uint32_t fl = pf.y;
    const Coord3 c = coord3(k, p);
    C r1 = C(0), r0 = C(0), j1[3] = {C(0), C(0), C(0)}, j0[3] = {C(0), C(0), C(0)};
    double dm = 0.0;
    const uint32_t lb = fl ? lbase[p] : 0u;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const int64_t s = pull_slot3(k, q, c, fl, lb, k.plane);
      const C a = cur[s], b = prev[s];
      r1 += a;
      r0 += b;
      dm += static_cast<double>(a);
#pragma unroll
      for (int e = 0; e < 3; e++) {
        j1[e] = mac3(j1[e], cvel3(q, e), a);
        j0[e] = mac3(j0[e], cvel3(q, e), b);
      }
    }
    r1 += C(1);
    r0 += C(1);
    const C acc3[3] = {k.ax, k.ay, k.az};
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      const C u1 = (j1[e] + C(0.5) * r1 * acc3[e]) / r1, u0 = (j0[e] + C(0.5) * r0 * acc3[e]) / r0;
      const double du = static_cast<double>(u1) - static_cast<double>(u0);
      num += du * du;
      den += static_cast<double>(u1) * static_cast<double>(u1);
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
  for (int cc = 0; cc < 4; cc++) {
    const double v = lbm::dev::warp_sum(acc[cc]);
    if (lane == 0) sh[w][cc] = v;
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
                               const uint32_t *__restrict__ lbase, const Const3<C> k,
                               int64_t n_nodes, double *out) {
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_nodes;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t fl = flags[p];
    const Coord3 c = coord3(k, p);
    const uint32_t lb = fl != kSolid3 && fl ? lbase[p] : 0u;
#pragma unroll
    for (int q = 0; q < Q; q++) {
      double v = w3<double>(q);
      if (fl != kSolid3) v += static_cast<double>(f[pull_slot3(k, q, c, fl, lb, k.plane)]);
      out[q * n_nodes + p] = v;
    }
  }
}

// Eq. FluidMacr at every node (solid nodes 0): rho, ux, uy, uz arrays of
// nx*ny*nz doubles.
template <typename C>
__global__ void fields3_kernel(const C *__restrict__ f, const uint32_t *__restrict__ flags,
                               const uint32_t *__restrict__ lbase, const Const3<C> k,
                               int64_t n_nodes, double *__restrict__ out) {
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_nodes;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t fl = flags[p];
    double r = 0.0, u[3] = {0.0, 0.0, 0.0};
    if (fl != kSolid3) {
      const Coord3 c = coord3(k, p);
      double dr = 0.0, j[3] = {0.0, 0.0, 0.0};
      const uint32_t lb = fl ? lbase[p] : 0u;
#pragma unroll
      for (int q = 0; q < Q; q++) {
        const double v = static_cast<double>(f[pull_slot3(k, q, c, fl, lb, k.plane)]);
        dr += v;
#pragma unroll
        for (int e = 0; e < 3; e++) j[e] += cvel3(q, e) * v;
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
                               const uint32_t *__restrict__ lbase, const Const3<C> k,
                               int64_t n_nodes, C *f) {
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n_nodes;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t fl = flags[p];
    if (fl == kSolid3) continue;
    const Coord3 c = coord3(k, p);
    const uint32_t lb = fl ? lbase[p] : 0u;
#pragma unroll
    for (int q = 0; q < Q; q++)
      f[pull_slot3(k, q, c, fl, lb, k.plane)] = static_cast<C>(in[q * n_nodes + p] - w3<double>(q));
  }
}

// a case's constants in both arithmetic types (the one of its precision is set)
struct Const3Both {
  Const3<double> d;
  Const3<float> f;
  Const3<D2> x;  // the same as double-FP32 pairs (the exact-mass variant's body force)
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
  uint32_t *lbase = nullptr;
  uint2 *fluid = nullptr;  // the fluid nodes in node order: index, flag word
  // the exact-mass variant (FP32): link coefficients as FP32 pairs and the
  // carries (one per link, then one per fluid node)
  int exact = 0;
  int64_t dev_bytes = 0;  // device memory the handle holds
  lbm::LinkCoefDF *links_df = nullptr;
  float *carry = nullptr;
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
                  static_cast<void *>(h->fluid), static_cast<void *>(h->links_df),
                  static_cast<void *>(h->carry),
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
  if (p.mass_mode < -1 || p.mass_mode > 1)
    return fail3(nullptr, LBM_EINVAL, "mass_mode must be -1, 0 or 1");
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
  std::vector<uint32_t> lbase(static_cast<size_t>(n), 0);
  int64_t total = 0;
  for (int64_t pn = 0; pn < n; pn++) {
    lbase[pn] = static_cast<uint32_t>(total);
    if (flags[pn] != kSolid3) total += __builtin_popcount(flags[pn]);
  }
  if (total > static_cast<int64_t>(UINT32_MAX))
    return fail3(nullptr, LBM_EINVAL, "more than 2^32 - 1 boundary links");
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
  const size_t es = p.precision == LBM_FP64 ? 8 : 4;
  const size_t fbytes = (19 * static_cast<size_t>(h->plane) + (n_links + 63) / 64 * 64) * es;
  auto alloc = [&](void **ptr, size_t bytes) {
    h->dev_bytes += static_cast<int64_t>(std::max<size_t>(bytes, 16));
    return cudaMalloc(ptr, std::max<size_t>(bytes, 16));
  };
  if (e == cudaSuccess) e = alloc(&h->f[0], fbytes);
  if (e == cudaSuccess) e = alloc(&h->f[1], fbytes);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->flags), n * 4);
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->lbase), n * 4);
  if (e == cudaSuccess) e = alloc(&h->links, std::max<size_t>(1, n_links) * 4 * es);
  if (e == cudaSuccess)
    e = alloc(reinterpret_cast<void **>(&h->partials), kResBlocks3 * 4 * sizeof(double));
  if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->result), 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->f[0], 0, fbytes);
  if (e == cudaSuccess) e = cudaMemset(h->f[1], 0, fbytes);
  if (e == cudaSuccess) e = cudaMemcpy(h->flags, flags.data(), n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->lbase, lbase.data(), n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    std::vector<uint2> fluid;
    fluid.reserve(static_cast<size_t>(n_fluid));
    for (int64_t pn = 0; pn < n; pn++)
      if (flags[pn] != kSolid3) fluid.push_back(make_uint2(static_cast<uint32_t>(pn), flags[pn]));
    e = alloc(reinterpret_cast<void **>(&h->fluid), std::max<size_t>(1, fluid.size()) * 8);
    if (e == cudaSuccess && !fluid.empty())
      e = cudaMemcpy(h->fluid, fluid.data(), fluid.size() * 8, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = dispatch3(h->precision, [&](auto tag) {
      using C = std::remove_pointer_t<decltype(tag)>;
      std::vector<Link3<C>> lk(std::max<size_t>(1, n_links));
      for (size_t k = 0; k < n_links; k++) {
        const double *cf = &coef[8 * k];
        lk[slot[k]] = Link3<C>{static_cast<C>(cf[0]), static_cast<C>(cf[1]), static_cast<C>(cf[2]),
                               static_cast<C>(cf[3])};
      }
      // the case's constants in each arithmetic type (the FP32 exact-mass
      // variant forms its moments in double-FP32)
      auto fill = [&](auto &kc) {
        using A = std::remove_reference_t<decltype(kc.ax)>;
        for (int a = 0; a < Q; a++) {
          const double s = 1.0 / tau[a];
          kc.s_scaled[a] = static_cast<A>(s / L.norm[a]);
          kc.f_scaled[a] = static_cast<A>((1.0 - 0.5 * s) / L.norm[a]);
        }
        kc.ax = static_cast<A>(dom->ax);
        kc.ay = static_cast<A>(dom->ay);
        kc.az = static_cast<A>(dom->az);
        kc.nx = nx;
        kc.ny = ny;
        kc.nz = nz;
        kc.px = per[0];
        kc.py = per[1];
        kc.pz = per[2];
        kc.diffuse_mode = p.diffuse_mode;
        kc.plane = h->plane;
        kc.n_links = h->n_links;
        kc.sr_seed = 0u;
      };
      fill(h->kc.f);
      fill(h->kc.d);
      fill(h->kc.x);
      return cudaMemcpy(h->links, lk.data(), lk.size() * sizeof(Link3<C>), cudaMemcpyHostToDevice);
    });
  // the exact-mass variant (FP32): where mass_mode asks for it, or by
  // default where a wall moves or the lattice has no boundary links
  bool moving = false;
  for (size_t k = 0; k < 3 * n_links && !moving; k++) moving = link_ub[k] != 0.0;
  h->exact = p.precision == LBM_FP32 && p.mass_mode >= 0 &&
             (p.mass_mode > 0 || moving || n_links == 0);
  if (e == cudaSuccess && h->exact) {
    std::vector<lbm::LinkCoefDF> ldf(std::max<size_t>(1, n_links));
    for (size_t k = 0; k < n_links; k++) ldf[slot[k]] = lbm::link_coef_df(&coef[8 * k]);
    e = alloc(reinterpret_cast<void **>(&h->links_df), ldf.size() * sizeof(lbm::LinkCoefDF));
    if (e == cudaSuccess)
      e = cudaMemcpy(h->links_df, ldf.data(), ldf.size() * sizeof(lbm::LinkCoefDF),
                     cudaMemcpyHostToDevice);
    const size_t nc = std::max<size_t>(1, n_links) + static_cast<size_t>(n_fluid);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&h->carry), nc * 4);
    if (e == cudaSuccess) e = cudaMemset(h->carry, 0, nc * 4);
  }
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
      if (h->n_fluid == 0) return cudaSuccess;
      const unsigned blocks = static_cast<unsigned>((h->n_fluid + kThreads3 - 1) / kThreads3);
      if constexpr (std::is_same<C, float>::value) {
        if (h->exact) {
          Const3<C> kx = h->kc.get(tag);
          kx.sr_seed = lbm::dev::step_seed(h->steps);
          step3_kernel<C, true><<<blocks, kThreads3, 0, h->stream>>>(
              static_cast<const C *>(h->f[src]), static_cast<C *>(h->f[dst]), h->flags, h->lbase,
              static_cast<const Link3<C> *>(h->links), h->fluid, kx, h->n_fluid, h->links_df,
              h->carry, h->kc.x);
          return cudaGetLastError();
        }
      }
      step3_kernel<C><<<blocks, kThreads3, 0, h->stream>>>(
          static_cast<const C *>(h->f[src]), static_cast<C *>(h->f[dst]), h->flags, h->lbase,
          static_cast<const Link3<C> *>(h->links), h->fluid, h->kc.get(tag), h->n_fluid);
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
        h->lbase, h->fluid, h->kc.get(tag), h->n_fluid, h->partials);
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
      export3_kernel<C><<<grid_for3(h->n_nodes, 256), 256, 0, h->stream>>>(
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
      import3_kernel<C><<<grid_for3(h->n_nodes, 256), 256, 0, h->stream>>>(
          d, h->flags, h->lbase, h->kc.get(tag), h->n_nodes, static_cast<C *>(h->f[b]));
      return cudaGetLastError();
    });
  if (e == cudaSuccess && h->carry)  // a new state owes no carries
    e = cudaMemsetAsync(h->carry, 0, (std::max<int64_t>(1, h->n_links) + h->n_fluid) * 4,
                        h->stream);
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

int lbm3d_get_info(const lbm3d_t *h, lbm_info_t *info) {
  if (!h || !info) return LBM_EINVAL;
  *info = lbm_info_t{};
  info->n_nodes = h->n_nodes;
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
  info->pitch = h->nx;
  info->exact_mass = h->exact;
  return LBM_OK;
}

void lbm3d_destroy(lbm3d_t *h) { release3(h); }

const char *lbm3d_last_error(const lbm3d_t *h) { return h ? h->err.c_str() : g_err3.c_str(); }

}  // extern "C"
