// rlb_node.cuh -- per-node arithmetic of the relativistic lattice Boltzmann step
// (Li, Luo & Li, arXiv 1211.3286) on the D3Q19 lattice.
//
// Link order (shared by every kernel of the library):
//   0 rest; pairs p = 0..8 hold links a = 2p+1 (direction c_p) and a+1 (-c_p):
//   p0 +x, p1 +y, p2 +z, p3 (1,1,0), p4 (1,-1,0), p5 (1,0,1), p6 (1,0,-1),
//   p7 (0,1,1), p8 (0,1,-1).
//   Weights: w0 = 1/3, axis links 1/18, diagonal links 1/36; c_s^2 = 1/3.
//
// One node update, given the 19 f and 19 g pulled to the node:
//   moments (Eq. 10): N0 = sum f, T00 = sum g, M = sum c g, formed from the
//     pair sums s_p = g_a + g_abar and differences d_p = g_a - g_abar;
//   recovery (Eq. 10 inverted under P = e/3): with A = 4 T00^2 - 3 |M|^2,
//     sigma = (2 T00 + sqrt(A)) / 3  [equivalent to u = 3M/(2T00+sqrt A) and
//     sigma = 4 T00/(3 + u^2)], u = M / sigma, P = sigma - T00;
//   equilibria (Eqs. 7-9) split per pair into an even part (shared by a and
//     abar) and an odd part (opposite signs):
//     f^eq = w N0 [(1 - 1.5 u^2) + 4.5 (c.u)^2] +- 3 w N0 (c.u)
//     g^eq = w [(3P - 1.5 sigma u^2) + 4.5 sigma (c.u)^2] +- 3 w sigma (c.u)
//     g^eq_0 = sigma - 3P - 0.5 sigma u^2            (Eq. 8 with w0 = 1/3)
//     (N0 = n gamma is the f density, so n and gamma are not needed per step);
//   relaxation: f* = f - omega_f (f - f^eq)  (Eq. 5);
//     g* = g - omega_v (g - g^eq) for BGK (Eq. 6);  for MRT (Eqs. 30, 35) the
//     D3Q19 basis is orthogonal and every non-conserved moment except e, eps
//     and q relaxes with omega_v, so Lambda = M^-1 S M acts as
//       g* = g - omega_v (g - g^eq) - sum_{k in e,eps,q} (s_k - omega_v)
//                                       [M_k.(g - g^eq) / |M_k|^2] M_k,
//     a rank-5 correction.  The e and eps rows depend on |c|^2 only, so their
//     correction is one constant per link class (rest / axis / diagonal); the q
//     rows are odd and correct the odd part of each pair.
//     The class sums of g^eq needed for M_k.(g - g^eq) are closed forms:
//       sum_axis g^eq = P,  sum_diag g^eq = P + 0.5 sigma u^2,
//       q^eq_i = -(2/3) sigma u_i.
//
// Arithmetic variants in this file:
//   node_collide_fx (and the warp-role kernel built from its parts): FP64
//     populations; sums, recovery (fx_recover) and per-link work in 64-bit
//     block fixed point on the integer pipes, each output rounded once to FP64
//     -- the FP64 step with constant relaxation times;
//   node_collide_f64: the same update in FP64 arithmetic -- the fixed-eta/s
//     mode, whose relaxation times vary per node;
//   node_collide_f32s: FP32 population storage, exact sums, recovery by one FP64
//     Newton step on sigma's quadratic from an FP32 seed, FP32 per-link work;
//   node_collide_d2q9_f64: the D2Q9 model of Sec. V.A.
#pragma once
#include <cmath>
#include <cstdint>

namespace rlb {

// link directions
__host__ __device__ constexpr int link_cx(int a) {
  constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return t[a];
}
__host__ __device__ constexpr int link_cy(int a) {
  constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return t[a];
}
__host__ __device__ constexpr int link_cz(int a) {
  constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return t[a];
}

// Constants of one step, prepared on the host from the relaxation times.
struct StepConst {
  // f (Eq. 5)
  double omf, omf1;                 // omega_f, 1 - omega_f
  double fA_k, fD_k, f0_k;          // omega_f w          (axis, diag, rest)
  double fA_s, fD_s;                // 4.5 omega_f w      (even coefficient / N0)
  double fA_a, fD_a;                // 3 omega_f w        (odd coefficient / N0)
  // g (Eq. 6 / 35)
  double omv, omv1;                 // omega_v, 1 - omega_v
  double gA_k, gD_k;                // omega_v w
  double gA_s, gD_s;                // 4.5 omega_v w
  double gA_a, gD_a;                // 3 omega_v w
  double ce, cp, cq;                // (s_e - omega_v)/2394, (s_eps - omega_v)/252, (s_q - omega_v)/40
  // single-precision copies for the FP32-storage collide
  float omf_f, omf1_f, fA_k_f, fD_k_f, f0_k_f, fA_s_f, fD_s_f, fA_a_f, fD_a_f;
  float omv_f, omv1_f, gA_k_f, gD_k_f, gA_s_f, gD_s_f, gA_a_f, gD_a_f;
  float ce_f, cp_f, cq_f;
  // fixed-eta/s relaxation: eta_s > 0 derives tau_g (BGK) / tau_v (MRT) per node; tauf_local:
  // tau_f = tau_g; for MRT the ratios a_x = (tau_x - 1/2) / (tau_v - 1/2) of e, eps, q
  double eta_s;
  int tauf_local;
  double a_e, a_p, a_q;
  // 64-bit fixed-point copies for the integer-pipe FP64 collide: omega * 2^63 (even),
  // ce * 2^73, cp * 2^69, cq * 2^67 (|ce| < 2/2394, |cp| < 2/252, |cq| < 2/40 keep them
  // below 2^63)
  unsigned long long Om_f, Om_v;
  // shift-free relaxation (fx::relax_r): r = 2 for omega >= 1 with (omega - 1) 2^64, r = 1
  // for omega < 1 with omega 2^64 (both even)
  unsigned long long Om2_f, Om2_v;
  int r_f, r_v;
  long long CE, CP, CQ;
  // coefficient of the theta term of the C_7 correction (Eq. 38): 1 (Eq. A17) or 2 (as printed)
  double c7_theta;
};

// q = 19 (D3Q19: weights 1/3, 1/18, 1/36; MRT row norms e 2394, eps 252, q 40) or
// q = 9 (D2Q9: weights 4/9, 1/9, 1/36; norms e 36, eps 36, q 12).
inline StepConst make_step_const(double tau_f, double tau_v, double tau_e, double tau_eps, double tau_q,
                                 bool mrt, int q = 19) {
  StepConst k{};
  const bool d2 = q == 9;
  const double wA = d2 ? 1.0 / 9.0 : 1.0 / 18.0, wD = 1.0 / 36.0, w0 = d2 ? 4.0 / 9.0 : 1.0 / 3.0;
  k.omf = 1.0 / tau_f;
  k.omf1 = 1.0 - k.omf;
  k.fA_k = k.omf * wA;
  k.fD_k = k.omf * wD;
  k.f0_k = k.omf * w0;
  k.fA_s = 4.5 * k.omf * wA;
  k.fD_s = 4.5 * k.omf * wD;
  k.fA_a = 3.0 * k.omf * wA;
  k.fD_a = 3.0 * k.omf * wD;
  k.omv = 1.0 / tau_v;
  k.omv1 = 1.0 - k.omv;
  k.gA_k = k.omv * wA;
  k.gD_k = k.omv * wD;
  k.gA_s = 4.5 * k.omv * wA;
  k.gD_s = 4.5 * k.omv * wD;
  k.gA_a = 3.0 * k.omv * wA;
  k.gD_a = 3.0 * k.omv * wD;
  if (mrt) {
    const double tq = tau_q > 0 ? tau_q : tau_v;
    k.ce = (1.0 / tau_e - k.omv) / (d2 ? 36.0 : 2394.0);
    k.cp = (1.0 / tau_eps - k.omv) / (d2 ? 36.0 : 252.0);
    k.cq = (1.0 / tq - k.omv) / (d2 ? 12.0 : 40.0);
  }
  k.omf_f = (float)k.omf; k.omf1_f = (float)k.omf1;
  k.fA_k_f = (float)k.fA_k; k.fD_k_f = (float)k.fD_k; k.f0_k_f = (float)k.f0_k;
  k.fA_s_f = (float)k.fA_s; k.fD_s_f = (float)k.fD_s; k.fA_a_f = (float)k.fA_a; k.fD_a_f = (float)k.fD_a;
  k.omv_f = (float)k.omv; k.omv1_f = (float)k.omv1;
  // the FP32-storage collide applies these to sigma u^2 - 2P = -(3P - 1.5 sigma u^2) / 1.5
  k.gA_k_f = (float)(-1.5 * k.gA_k);
  k.gD_k_f = (float)(-1.5 * k.gD_k);
  k.gA_s_f = (float)k.gA_s; k.gD_s_f = (float)k.gD_s; k.gA_a_f = (float)k.gA_a; k.gD_a_f = (float)k.gD_a;
  k.ce_f = (float)k.ce; k.cp_f = (float)k.cp; k.cq_f = (float)k.cq;
  k.Om_f = (unsigned long long)std::ldexp(k.omf, 63) & ~1ull;
  k.Om_v = (unsigned long long)std::ldexp(k.omv, 63) & ~1ull;
  k.r_f = k.omf >= 1.0 ? 2 : 1;
  k.r_v = k.omv >= 1.0 ? 2 : 1;
  k.Om2_f = (unsigned long long)std::ldexp(k.r_f == 2 ? k.omf - 1.0 : k.omf, 64) & ~1ull;
  k.Om2_v = (unsigned long long)std::ldexp(k.r_v == 2 ? k.omv - 1.0 : k.omv, 64) & ~1ull;
  k.CE = std::llround(std::ldexp(k.ce, 73));
  k.CP = std::llround(std::ldexp(k.cp, 69));
  k.CQ = std::llround(std::ldexp(k.cq, 67));
  return k;
}

// Macroscopic state recovered at a node (FP64).
struct NodeMacro {
  double N0, T00, Mx, My, Mz;
  double sigma, P, ux, uy, uz, u2;
  bool bad;
};

// Moments and recovery from the 19 g (and 19 f) values of a node, as FP64.
// Pair sums / differences are returned for reuse by the MRT correction.
template <typename S>
__device__ __forceinline__ void node_moments(const S (&f)[19], const S (&g)[19], double (&sp)[9], double (&dp)[9],
                                             double& Sa, double& Sd, NodeMacro& m) {
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const double a = (double)g[2 * p + 1], b = (double)g[2 * p + 2];
    sp[p] = a + b;
    dp[p] = a - b;
  }
  Sa = (sp[0] + sp[1]) + sp[2];
  Sd = ((sp[3] + sp[4]) + (sp[5] + sp[6])) + (sp[7] + sp[8]);
  m.T00 = ((double)g[0] + Sa) + Sd;
  m.Mx = ((dp[0] + dp[3]) + (dp[4] + dp[5])) + dp[6];
  m.My = ((dp[1] + dp[3]) - (dp[4] - dp[7])) + dp[8];
  m.Mz = ((dp[2] + dp[5]) - (dp[6] - dp[7])) - dp[8];
  double n0 = (double)f[0];
  double fs[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) fs[p] = (double)f[2 * p + 1] + (double)f[2 * p + 2];
  m.N0 = n0 + ((((fs[0] + fs[1]) + (fs[2] + fs[3])) + ((fs[4] + fs[5]) + (fs[6] + fs[7]))) + fs[8]);
}

__device__ __forceinline__ void node_recover(NodeMacro& m) {
  const double MM = fma(m.Mx, m.Mx, fma(m.My, m.My, m.Mz * m.Mz));
  const double A = fma(4.0 * m.T00, m.T00, -3.0 * MM);
  const double sA = sqrt(A);
  m.sigma = fma(2.0, m.T00, sA) * (1.0 / 3.0);
  const double is = 1.0 / m.sigma;
  m.ux = m.Mx * is;
  m.uy = m.My * is;
  m.uz = m.Mz * is;
  m.P = m.sigma - m.T00;
  m.u2 = fma(m.ux, m.ux, fma(m.uy, m.uy, m.uz * m.uz));
  // every comparison is false for NaN, so the negated form also catches NaN
  m.bad = !(A >= 0.0) || !(m.T00 > 0.0) || !(m.P > 0.0) || !(m.u2 < 1.0);
}

// ---------------------------------------------------------------------------
// Recovery for the FP32-storage path with the FP64 pipe kept for arithmetic:
// GB300 retires 2 FP64 instructions per clock per SM, and conversions and
// compares use the same pipe, so they are done with integer operations here.
//
// sqrt and reciprocal: an FP32 hardware seed (about 2^-23) refined by two
// Newton steps in FP64 (each step squares the relative error), i.e. to the FP64
// rounding level.
__device__ __forceinline__ float d2f_trunc_bits(double x) {   // seed only: truncating narrow, normal range
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  const unsigned b = (hi & 0x80000000u) | ((unsigned)(e < 1 ? 1 : (e > 254 ? 254 : e)) << 23) |
                     ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(b);
}
// the same with the result scaled by 2^es (seed arithmetic away from the FP32 range limits)
__device__ __forceinline__ float d2f_trunc_bits_s(double x, int es) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896 + es;
  const unsigned b = (hi & 0x80000000u) | ((unsigned)(e < 1 ? 1 : (e > 254 ? 254 : e)) << 23) |
                     ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(b);
}
__device__ __forceinline__ double widen_seed_s(float rf, int es) {   // normal float x 2^es -> double
  const unsigned rb = __float_as_uint(rf);
  return __hiloint2double(
      (int)((rb & 0x80000000u) | ((((rb >> 23) & 0xffu) + 896u + (unsigned)es) << 20) | ((rb & 0x7fffffu) >> 3)),
      (int)(rb << 29));
}
__device__ __forceinline__ double widen_seed(float rf) {   // normal float -> double by moving bits
  const unsigned rb = __float_as_uint(rf);
  return __hiloint2double((int)((rb & 0x80000000u) | ((((rb >> 23) & 0xffu) + 896u) << 20) | ((rb & 0x7fffffu) >> 3)),
                          (int)(rb << 29));
}
__device__ __forceinline__ double sqrt_seeded(double A) {
  float rf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(d2f_trunc_bits(A)));
  const double y = widen_seed(rf);           // 1/sqrt(A) to ~2^-23
  const double h = 0.5 * y;
  double s = A * y;                          // sqrt(A) to ~2^-23
  s = fma(h, fma(-s, s, A), s);              // s += h (A - s^2): ~2^-46
  return fma(h, fma(-s, s, A), s);           // ~2^-69: FP64 rounding level
}
__device__ __forceinline__ double rcp_seeded(double x) {
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(d2f_trunc_bits(x)));
  const double y = widen_seed(rf);           // ~2^-23
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);            // cubic step: ~2^-69
}

// Round-to-nearest-even narrowing of a double to float by moving bits (the
// result for values inside the normal float range; smaller magnitudes flush to
// a signed zero, larger saturate to a signed infinity).
__device__ __forceinline__ float d2f_rn_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  unsigned mag = ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned tail = lo & 0x1fffffffu;
  mag += (tail > 0x10000000u) | ((tail == 0x10000000u) & (mag & 1u));
  mag = e < 1 ? 0u : (e > 254 ? 0x7f800000u : mag);
  return __uint_as_float(sign | mag);
}

// d2f_rn_bits(x * 2^es) for a normal or zero x: the power of two goes into the exponent
// of the narrowed value (a zero x, exponent field 0, still flushes to zero).
__device__ __forceinline__ float d2f_rn_bits_scaled(double x, int es) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const unsigned ex = (hi >> 20) & 0x7ffu;
  const int e = (int)ex + es - 896;
  unsigned mag = ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned tail = lo & 0x1fffffffu;
  mag += (tail > 0x10000000u) | ((tail == 0x10000000u) & (mag & 1u));
  mag = (ex == 0u || e < 1) ? 0u : (e > 254 ? 0x7f800000u : mag);
  return __uint_as_float(sign | mag);
}

// Integer sign / magnitude tests on the high word of a double.
__device__ __forceinline__ bool pos_finite_hi(double x) {   // x > 0, finite (hi word of a normal positive)
  const int hi = __double2hiint(x);
  return hi > 0 && hi < 0x7ff00000;
}

__device__ __forceinline__ void node_recover_fast(NodeMacro& m) {
  // the recovery is homogeneous of degree 1 in (T00, M) with u scale free: run it on
  // T00 and M divided by the power of two of T00 (exact multiplies), which keeps A
  // inside the range of the FP32 seeds at any scale, and scale sigma and P back
  int es = (int)(((unsigned)__double2hiint(m.T00) >> 20) & 0x7ffu) - 1023;
  es = es < -1000 ? -1000 : (es > 1000 ? 1000 : es);
  const double down = __hiloint2double((1023 - es) << 20, 0), up = __hiloint2double((1023 + es) << 20, 0);
  const double T = m.T00 * down, mx = m.Mx * down, my = m.My * down, mz = m.Mz * down;
  const double MM = fma(mx, mx, fma(my, my, mz * mz));
  const double A = fma(4.0 * T, T, -3.0 * MM);
  const double sA = sqrt_seeded(A);
  const double sg = fma(2.0, T, sA) * (1.0 / 3.0);
  const double is = rcp_seeded(sg);
  m.ux = mx * is;
  m.uy = my * is;
  m.uz = mz * is;
  const double P = sg - T;
  m.sigma = sg * up;
  m.P = P * up;
  m.u2 = fma(m.ux, m.ux, fma(m.uy, m.uy, m.uz * m.uz));
  // A > 0, T00 > 0, P > 0 (all finite) and u^2 < 1 (bit patterns of non-negative
  // doubles order like the values; NaN and Inf fail every test)
  m.bad = !(pos_finite_hi(A) && pos_finite_hi(m.T00) && pos_finite_hi(P) &&
            (unsigned)__double2hiint(m.u2) < 0x3ff00000u);
}

// c.u for the 9 pair directions
template <typename C>
__device__ __forceinline__ void pair_cu(C ux, C uy, C uz, C (&cu)[9]) {
  cu[0] = ux; cu[1] = uy; cu[2] = uz;
  cu[3] = ux + uy; cu[4] = ux - uy;
  cu[5] = ux + uz; cu[6] = ux - uz;
  cu[7] = uy + uz; cu[8] = uy - uz;
}

// FP64 node collide: moments, recovery, equilibria, BGK f, BGK / MRT g.
// f and g hold the pulled populations on entry and the post-collision ones on exit.
// x * 2^e for a normal double whose scaled value stays normal (exponent add on the
// bits); zero stays zero
__device__ __forceinline__ double scale_pow2(double x, int e) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const bool zero = ((hi & 0x7fffffff) | lo) == 0;
  return __hiloint2double(zero ? hi : hi + (e << 20), lo);
}

// ---------------------------------------------------------------------------
// Exact moment sums of FP64 populations on the integer pipe.
//
// Each of the 19 values of a distribution becomes a 64-bit fixed-point integer
// on the grid of its largest exponent E: its 53-bit significand shifted left by 5
// (headroom for 19 terms) and right by E - e.  Signed sums of these integers are
// exact; they equal the true sums except for bits below 2^(E-1080) (below 2^-57 of
// the largest value), and each is rounded once to FP64.  This takes the ~57 FP64
// additions of the moments (Eq. 10) off GB300's FP64 pipe (2 instructions per
// clock per SM) onto the integer pipe.
__device__ __forceinline__ int max_exp19_f64(const double (&p)[19]) {
  int E = ((unsigned)__double2hiint(p[0]) >> 20) & 0x7ff;
#pragma unroll
  for (int a = 1; a < 19; ++a) E = max(E, (int)(((unsigned)__double2hiint(p[a]) >> 20) & 0x7ffu));
  return E;
}
__device__ __forceinline__ long long fixed_from_f64(double x, int E) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7ffu);
  const unsigned mhi = ex ? ((hi & 0xfffffu) | 0x100000u) : (hi & 0xfffffu);
  const int sh = min(E - (ex ? ex : 1), 63);
  const unsigned long long v = ((((unsigned long long)mhi << 32) | lo) << 5) >> sh;
  return (hi >> 31) ? -(long long)v : (long long)v;
}
struct ExactSums64 {
  long long T00, Mx, My, Mz, Sa, Sd, qx, qy, qz;
};
template <bool QSEP>
__device__ __forceinline__ void exact_sums_g64(const double (&g)[19], int E, ExactSums64& S) {
  // integer sums are exact in any order: accumulate pair by pair as the values are formed
  constexpr int cx[9] = {1, 0, 0, 1, 1, 1, 1, 0, 0};
  constexpr int cy[9] = {0, 1, 0, 1, -1, 0, 0, 1, 1};
  constexpr int cz[9] = {0, 0, 1, 0, 0, 1, -1, 1, -1};
  S.Sa = 0; S.Sd = 0; S.Mx = 0; S.My = 0; S.Mz = 0; S.qx = 0; S.qy = 0; S.qz = 0;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const long long va = fixed_from_f64(g[2 * p + 1], E), vb = fixed_from_f64(g[2 * p + 2], E);
    const long long sp = va + vb, dp = va - vb;
    if (p < 3) S.Sa += sp; else S.Sd += sp;
    if (cx[p] == 1) S.Mx += dp;
    if (cy[p] == 1) S.My += dp; else if (cy[p] == -1) S.My -= dp;
    if (cz[p] == 1) S.Mz += dp; else if (cz[p] == -1) S.Mz -= dp;
    if (QSEP) {   // q_i = (5|c|^2 - 9) c_i: axis weight -4, diagonal +1
      const long long w = p < 3 ? -4 : 1;
      if (cx[p] == 1) S.qx += w * dp;
      if (cy[p] == 1) S.qy += w * dp; else if (cy[p] == -1) S.qy -= w * dp;
      if (cz[p] == 1) S.qz += w * dp; else if (cz[p] == -1) S.qz -= w * dp;
    }
  }
  S.T00 = fixed_from_f64(g[0], E) + S.Sa + S.Sd;
}
__device__ __forceinline__ long long exact_sum_f64(const double (&f)[19], int E) {
  long long s = 0;
#pragma unroll
  for (int a = 0; a < 19; ++a) s += fixed_from_f64(f[a], E);
  return s;
}
// K * 2^(E - 1080) as the nearest double (one rounding, exponent set by integer add)
__device__ __forceinline__ double fixed_to_f64(long long K, int E) {
  return scale_pow2(__ll2double_rn(K), E - 1080);
}

// Relaxation coefficients of the BGK f and g collisions for given omega_f, omega_v
// (D3Q19 weights), as make_step_const prepares them for constant taus.
__device__ __forceinline__ void set_bgk_coefficients(StepConst& k, double omf, double omv) {
  const double wA = 1.0 / 18.0, wD = 1.0 / 36.0, w0 = 1.0 / 3.0;
  k.omf = omf; k.omf1 = 1.0 - omf;
  k.fA_k = omf * wA; k.fD_k = omf * wD; k.f0_k = omf * w0;
  k.fA_s = 4.5 * omf * wA; k.fD_s = 4.5 * omf * wD; k.fA_a = 3.0 * omf * wA; k.fD_a = 3.0 * omf * wD;
  k.omv = omv; k.omv1 = 1.0 - omv;
  k.gA_k = omv * wA; k.gD_k = omv * wD;
  k.gA_s = 4.5 * omv * wA; k.gD_s = 4.5 * omv * wD; k.gA_a = 3.0 * omv * wA; k.gD_a = 3.0 * omv * wD;
}

// Per-node MRT rates of the fixed-eta/s mode: tau_x = 1/2 + a_x (tau_v - 1/2) for e, eps, q;
// q = 19 or 9 selects the row norms.
__device__ __forceinline__ void set_mrt_eta_coefficients(StepConst& k, double tau_v, int q) {
  const bool d2 = q == 9;
  const double h = tau_v - 0.5;
  k.ce = (1.0 / fma(k.a_e, h, 0.5) - k.omv) * (d2 ? 1.0 / 36.0 : 1.0 / 2394.0);
  k.cp = (1.0 / fma(k.a_p, h, 0.5) - k.omv) * (d2 ? 1.0 / 36.0 : 1.0 / 252.0);
  k.cq = (1.0 / fma(k.a_q, h, 0.5) - k.omv) * (d2 ? 1.0 / 12.0 : 1.0 / 40.0);
}

// tau_g from a fixed eta/s (Sec. II and III.B): eta = (tau - 1/2) c_s^2 (e + P) gamma,
// eta = (eta/s) s, s = n (4 - ln(n / n_eq)), n_eq = d_G T^3 / pi^2 (d_G = 16), T = P / n.
__device__ __forceinline__ double tau_eta_over_s(double eta_s, const NodeMacro& m) {
  const double inv_gamma = sqrt(1.0 - m.u2);
  const double n = m.N0 * inv_gamma;
  const double T = m.P / n;
  const double n_eq = (16.0 / (M_PI * M_PI)) * T * T * T;
  const double s = n * (4.0 - log(n / n_eq));
  return 0.5 + (eta_s * s) * inv_gamma / ((1.0 / 3.0) * 4.0 * m.P);   // (e + P) = 4 P
}

template <bool MRT, bool QSEP, bool ETA = false>
__device__ __forceinline__ bool node_collide_f64(double (&f)[19], double (&g)[19], const StepConst& kc) {
  NodeMacro m;
  const int Eg = max_exp19_f64(g), Ef = max_exp19_f64(f);
  ExactSums64 X;
  exact_sums_g64<QSEP>(g, Eg, X);
  m.T00 = fixed_to_f64(X.T00, Eg);
  m.Mx = fixed_to_f64(X.Mx, Eg);
  m.My = fixed_to_f64(X.My, Eg);
  m.Mz = fixed_to_f64(X.Mz, Eg);
  node_recover_fast(m);
  m.N0 = fixed_to_f64(exact_sum_f64(f, Ef), Ef);
  const double Sa = MRT ? fixed_to_f64(X.Sa, Eg) : 0.0;
  const double Sd = MRT ? fixed_to_f64(X.Sd, Eg) : 0.0;
  m.bad |= (Eg == 0x7ff) || (Ef == 0x7ff);
  StepConst k = kc;
  if (ETA) {
    const double tv = tau_eta_over_s(kc.eta_s, m);
    const double omv = 1.0 / tv;
    set_bgk_coefficients(k, kc.tauf_local ? omv : kc.omf, omv);
    if (MRT) set_mrt_eta_coefficients(k, tv, 19);
  }

  double cu[9];
  pair_cu<double>(m.ux, m.uy, m.uz, cu);

  // ---- f (Eq. 5 with Eq. 7)
  {
    const double kf = fma(-1.5 * m.N0, m.u2, m.N0);      // N0 (1 - 1.5 u^2)
    const double KA = k.fA_k * kf, KD = k.fD_k * kf;
    const double SA = k.fA_s * m.N0, SD = k.fD_s * m.N0;
    const double AA = k.fA_a * m.N0, AD = k.fD_a * m.N0;
    f[0] = fma(k.omf1, f[0], k.f0_k * kf);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const bool ax = p < 3;
      const double ev = fma(ax ? SA : SD, cu[p] * cu[p], ax ? KA : KD);
      const double od = (ax ? AA : AD) * cu[p];
      f[2 * p + 1] = fma(k.omf1, f[2 * p + 1], ev + od);
      f[2 * p + 2] = fma(k.omf1, f[2 * p + 2], ev - od);
    }
  }
  // ---- g (Eq. 6 or Eq. 35 with Eqs. 8-9)
  {
    const double su2 = m.sigma * m.u2;
    const double P3 = 3.0 * m.P;
    const double kg = fma(-1.5, su2, P3);                 // 3P - 1.5 sigma u^2
    const double geq0 = fma(-0.5, su2, m.sigma - P3);      // sigma - 3P - 0.5 sigma u^2
    double KA = k.gA_k * kg, KD = k.gD_k * kg;
    const double SA = k.gA_s * m.sigma, SD = k.gD_s * m.sigma;
    const double AA = k.gA_a * m.sigma, AD = k.gD_a * m.sigma;
    double g0n = fma(k.omv1, g[0], k.omv * geq0);
    double dq[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) dq[p] = 0.0;
    if (MRT) {
      // non-equilibrium class sums of g and the e / eps projections
      const double n0 = g[0] - geq0;
      const double nA = Sa - m.P;
      const double nD = fma(-0.5, su2, Sd - m.P);
      const double ne = fma(8.0, nD, fma(-11.0, nA, -30.0 * n0));
      const double np = fma(-4.0, nA, fma(12.0, n0, nD));
      const double ae = k.ce * ne, ap = k.cp * np;
      g0n = g0n + fma(30.0, ae, -12.0 * ap);
      KA = KA + fma(11.0, ae, 4.0 * ap);
      KD = KD - fma(8.0, ae, ap);
      if (QSEP) {
        // energy-flux rows q_i = (5|c|^2 - 9) c_i: axis weight -4, diagonal +1
        const double qeq = -2.0 / 3.0;
        const double qx = fixed_to_f64(X.qx, Eg);
        const double qy = fixed_to_f64(X.qy, Eg);
        const double qz = fixed_to_f64(X.qz, Eg);
        const double aqx = k.cq * fma(-qeq, m.Mx, qx);
        const double aqy = k.cq * fma(-qeq, m.My, qy);
        const double aqz = k.cq * fma(-qeq, m.Mz, qz);
        dq[0] = 4.0 * aqx; dq[1] = 4.0 * aqy; dq[2] = 4.0 * aqz;
        dq[3] = -(aqx + aqy); dq[4] = -(aqx - aqy);
        dq[5] = -(aqx + aqz); dq[6] = -(aqx - aqz);
        dq[7] = -(aqy + aqz); dq[8] = -(aqy - aqz);
      }
    }
    g[0] = g0n;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const bool ax = p < 3;
      const double ev = fma(ax ? SA : SD, cu[p] * cu[p], ax ? KA : KD);
      double od = (ax ? AA : AD) * cu[p];
      if (MRT && QSEP) od += dq[p];
      g[2 * p + 1] = fma(k.omv1, g[2 * p + 1], ev + od);
      g[2 * p + 2] = fma(k.omv1, g[2 * p + 2], ev - od);
    }
  }
  return m.bad;
}

// ----------------------------------------------------------------------------
// FP64 collide in 64-bit block fixed point (integer pipe).
//
// GB300 retires 2 FP64 instructions per clock per SM but 64 integer ones, so the
// per-link arithmetic of the FP64 step runs on integers.  The 19 values of one
// distribution at one node are put on the grid of their largest binary exponent
// E: x = X * 2^(E - 1079), |X| < 2^57 for the largest value.  Every value then
// keeps its bits down to 2^-56 of the node's largest population.  Sums (Eq. 10),
// equilibria (Eqs. 7-9), the BGK relaxation (Eqs. 5-6) and the MRT projection
// (Eq. 35) are integer adds and 64 x 64 -> high-64 products, each off by at most a
// few grid units.  The recovery (Eq. 10 inverted) runs on the same integers: its
// square root and reciprocal are FP32 seeds refined by fixed-point Newton steps, to
// about 2^-58 (FP64 rounding is 2^-53).  Each output is rounded once to FP64, the
// only FP64-pipe work (38 conversions per node).
//
// Output rounding to FP64 has two routes: integer bit assembly (ALU pipe; the FP64
// pipe only for negative or tiny values) or __ll2double_rn (FP64 pipe).  RLB_FX_OUT_F / RLB_FX_OUT_G pick the route for the
// f and g outputs, one bit per link pair and bit 9 for the rest link (set = FP64
// pipe), to balance the two pipes.
#ifndef RLB_FX_OUT_F
#define RLB_FX_OUT_F 0x3ff
#endif
#ifndef RLB_FX_OUT_G
#define RLB_FX_OUT_G 0x3ff
#endif

namespace fx {

constexpr unsigned long long kThird = 0x5555555555555556ull;       // ceil(2^64 / 3)
constexpr unsigned long long kSixth = 0x2AAAAAAAAAAAAAABull;       // ceil(2^64 / 6)
constexpr unsigned long long kTwoThirds = 0xAAAAAAAAAAAAAAABull;   // ceil(2^65 / 3)
constexpr unsigned long long kEighteenth = 0x0E38E38E38E38E39ull;  // ceil(2^64 / 18)
constexpr unsigned long long kSignBit = 0x8000000000000000ull;

// floor(a b / 2^64) for unsigned a, b without the low partial products: low by at most 2.
__device__ __forceinline__ unsigned long long mulhi(unsigned long long a, unsigned long long b) {
  const unsigned a0 = (unsigned)a, a1 = (unsigned)(a >> 32), b0 = (unsigned)b, b1 = (unsigned)(b >> 32);
  return (unsigned long long)a1 * b1 + ((unsigned long long)__umulhi(a1, b0) + __umulhi(a0, b1));
}
// y b / 2^64 for signed y (|y| < 2^63) and unsigned b: y + 2^63 is y with its top bit
// flipped, and the bias adds b / 2 to the product (bh = b >> 1).
__device__ __forceinline__ long long mulhi_su(long long y, unsigned long long b, unsigned long long bh) {
  return (long long)(mulhi((unsigned long long)y ^ kSignBit, b) - bh);
}
// v with the sign s (0 or 1)
__device__ __forceinline__ long long with_sign(unsigned long long v, unsigned s) {
  const unsigned long long m = 0ull - (unsigned long long)s;
  return (long long)((v ^ m) - m);
}

// a 2^-64 as a float (significand truncated to 24 bits) for a nonzero a, by moving bits
__device__ __forceinline__ float top_float(unsigned long long a) {
  const unsigned lz = (unsigned)__clzll((long long)a);
  const unsigned m = (unsigned)((a << lz) >> 40);
  return __uint_as_float(((126u - lz) << 23) | (m & 0x7fffffu));
}
// x 2^S as an integer for a positive normal float x with x 2^S < 2^64 (S >= 22)
template <int S>
__device__ __forceinline__ unsigned long long fixed_from_float(float x) {
  const unsigned b = __float_as_uint(x);
  return (unsigned long long)((b & 0x7fffffu) | 0x800000u) << ((b >> 23) - (150u - S));
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// |x| * 2^(Er - 1086), truncated, for a double x whose biased exponent is at most Er:
// the 53-bit significand top-aligned in 64 bits and shifted right by Er - exponent.
// Zero and subnormal inputs give 0 when Er >= 64.
__device__ __forceinline__ unsigned long long to_fixed_abs(double x, int Er) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned r = (unsigned)(Er - (int)((hi >> 20) & 0x7ffu));
  const unsigned th = __funnelshift_l(lo, hi, 11) | 0x80000000u;
  const unsigned tl = lo << 11;
  const unsigned vh = __funnelshift_rc(th, 0u, r);
  const unsigned vl = r < 32u ? __funnelshift_rc(tl, th, r) : __funnelshift_rc(th, 0u, r - 32u);
  return ((unsigned long long)vh << 32) | vl;
}
__device__ __forceinline__ long long to_fixed(double x, int Er) {
  return with_sign(to_fixed_abs(x, Er), (unsigned)__double2hiint(x) >> 31);
}

// K * 2^(E - 1079) rounded to the nearest double (ties away from zero) by integer
// bit assembly; K = 0 gives +0.  Needs E >= 57 so that the result is normal.
__device__ __forceinline__ double from_fixed_int(long long K, int E) {
  const unsigned long long s = (unsigned long long)(K >> 63);
  const unsigned long long a = ((unsigned long long)K ^ s) - s;
  const int lz = __clzll((long long)a);
  const unsigned long long n = a << (lz & 63);
  const unsigned long long m = (n >> 11) + ((n >> 10) & 1ull);
  const unsigned long long bits = m + ((unsigned long long)(unsigned)(E + 6 - lz) << 52) + (s << 63);
  return a ? __longlong_as_double((long long)bits) : 0.0;
}
// Fast form of to_fixed for a positive normal x whose biased exponent lies within
// [Er - 31, Er] (no sign, no long shift).
__device__ __forceinline__ long long to_fixed_pos(double x, int Er) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned r = (unsigned)(Er - (int)(hi >> 20));
  const unsigned th = __funnelshift_l(lo, hi, 11) | 0x80000000u;
  const unsigned tl = lo << 11;
  return (long long)(((unsigned long long)(th >> r) << 32) | __funnelshift_r(tl, th, r));
}

// The same through the FP64 pipe's int64 conversion (round to nearest even) of K | 1:
// setting the lowest bit keeps the converted value away from zero, so the exponent
// can be rebased without a zero test.  It moves K by at most one grid unit (2^-56 of
// the node's largest population, the grid's own resolution): an exact zero comes out
// as that one unit, and a tie in the rounding of a wide K rounds away from zero.
__device__ __forceinline__ double from_fixed_dp(long long K, int E) {
  const double d = __ll2double_rn(K | 1ll);
  return __hiloint2double(__double2hiint(d) + (int)((unsigned)(E - 1079) << 20), __double2loint(d));
}
// K * 2^(E - 1079) rounded to the nearest double (ties to even) by integer bit
// assembly for 2^32 <= K < 2^63, the range of a population near its node's largest;
// other K (negative, zero, tiny) take the FP64-pipe conversion.
__device__ __forceinline__ double from_fixed_pos(long long K, int E) {
  const unsigned hi = (unsigned)((unsigned long long)K >> 32), lo = (unsigned)K;
  if ((hi - 1u) >= 0x7fffffffu) return from_fixed_dp(K, E);
  const int lz = __clz(hi);                                   // 1..31
  const unsigned nh = __funnelshift_l(lo, hi, lz), nl = lo << lz;   // K << lz, bit 63 set
  const unsigned mh = nh >> 11, ml = __funnelshift_r(nl, nh, 11);
  const unsigned rb = nl & 0x7ffu;                             // bits below the 53-bit significand
  const unsigned up = (rb > 0x400u) | ((rb == 0x400u) & ml);  // round half to even
  const unsigned long long m = (((unsigned long long)mh << 32) | ml) + up;
  return __hiloint2double((int)((unsigned)(m >> 32) + ((unsigned)(E + 6 - lz) << 20)), (int)(unsigned)m);
}

template <int DP>
__device__ __forceinline__ double from_fixed(long long K, int E) {
  if constexpr (DP) return from_fixed_dp(K, E);
  else return from_fixed_pos(K, E);
}

// One relaxation X - omega (X - X^eq) + c with Om = omega 2^63: the biased product
// mulhi(2 (X - X^eq) + 2^63, Om) is omega (X - X^eq) + Om / 2, and c carries + Om / 2.
__device__ __forceinline__ long long relax(long long X, long long Xeq, unsigned long long Om, long long c) {
  const unsigned long long y = (unsigned long long)(X - Xeq) << 1;
  return X - (long long)mulhi(y ^ kSignBit, Om) + c;
}
// The same without the shift, from the base the sign of omega - 1 picks (R = 1: omega < 1,
// Om2 = omega 2^64, X - omega d; R = 2: omega >= 1, Om2 = (omega - 1) 2^64,
// X^eq - (omega - 1) d; d = X - X^eq): mulhi(d + 2^63, Om2) is w d + Om2 / 2, and c
// carries + Om2 / 2.  R = 0 is relax.
template <int R>
__device__ __forceinline__ long long relax_r(long long X, long long Xeq, unsigned long long Om, long long c) {
  if constexpr (R == 0) {
    return relax(X, Xeq, Om, c);
  } else {
    const unsigned long long y = (unsigned long long)(X - Xeq) ^ kSignBit;
    return (R == 2 ? Xeq : X) - (long long)mulhi(y, Om) + c;
  }
}
// Per-distribution equilibrium pieces on its grid (Eqs. 7-9 split per link pair):
//   axis pair i:   ev = KA + X_i,                          od = Z_i
//   diagonal i,j:  ev = KA/2 + (X_i + X_j)/2 +- Y_ij,       od = (Z_i +- Z_j)/2
// with X_i = D u_i^2 / 4, Y_ij = D u_i u_j / 4, Z_i = D u_i / 6 for the density D
// (sigma for g, N0 for f).
struct EqPieces {
  long long KA, Xx, Xy, Xz, Yxy, Yxz, Yyz, Zx, Zy, Zz;
};
struct UFix {
  unsigned long long ax, ay, az;       // |u_i| 2^63
  unsigned sx, sy, sz;                 // sign bits
  unsigned long long xx, yy, zz;       // u_i^2 2^62
  unsigned long long xy, xz, yz;       // |u_i u_j| 2^62
};
__device__ __forceinline__ void eq_pieces(unsigned long long D, const UFix& u, EqPieces& q) {
  q.Xx = (long long)mulhi(D, u.xx);
  q.Xy = (long long)mulhi(D, u.yy);
  q.Xz = (long long)mulhi(D, u.zz);
  q.Yxy = with_sign(mulhi(D, u.xy), u.sx ^ u.sy);
  q.Yxz = with_sign(mulhi(D, u.xz), u.sx ^ u.sz);
  q.Yyz = with_sign(mulhi(D, u.yz), u.sy ^ u.sz);
  const unsigned long long D3 = mulhi(D, kThird);
  q.Zx = with_sign(mulhi(D3, u.ax), u.sx);
  q.Zy = with_sign(mulhi(D3, u.ay), u.sy);
  q.Zz = with_sign(mulhi(D3, u.az), u.sz);
}

// Relax the 18 moving links of one distribution: class constants cA (axis) and cD
// (diagonal) hold Om / 2 plus any MRT class correction, dq the odd corrections.
// DP selects the rounding route per link pair: bit p set = FP64 pipe for pair p
// (0 = all integer, 0x1ff = all FP64 pipe).
template <int DP, bool ODD>
__device__ __forceinline__ void relax_links(const long long (&X)[19], const EqPieces& q, unsigned long long Om,
                                            long long cA, long long cD, const long long (&dq)[9], int E,
                                            double (&out)[19]) {
  const long long ev[9] = {q.KA + q.Xx, q.KA + q.Xy, q.KA + q.Xz,
                           (q.KA >> 1) + ((q.Xx + q.Xy) >> 1) + q.Yxy, (q.KA >> 1) + ((q.Xx + q.Xy) >> 1) - q.Yxy,
                           (q.KA >> 1) + ((q.Xx + q.Xz) >> 1) + q.Yxz, (q.KA >> 1) + ((q.Xx + q.Xz) >> 1) - q.Yxz,
                           (q.KA >> 1) + ((q.Xy + q.Xz) >> 1) + q.Yyz, (q.KA >> 1) + ((q.Xy + q.Xz) >> 1) - q.Yyz};
  const long long od[9] = {q.Zx, q.Zy, q.Zz,
                           (q.Zx + q.Zy) >> 1, (q.Zx - q.Zy) >> 1, (q.Zx + q.Zz) >> 1, (q.Zx - q.Zz) >> 1,
                           (q.Zy + q.Zz) >> 1, (q.Zy - q.Zz) >> 1};
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const long long c = p < 3 ? cA : cD;
    const long long d = ODD ? dq[p] : 0;
    const long long ya = relax(X[2 * p + 1], ev[p] + od[p], Om, c + d);
    const long long yb = relax(X[2 * p + 2], ev[p] - od[p], Om, c - d);
    // (DP >> p) & 1 is a constant once the loop is unrolled
    out[2 * p + 1] = ((DP >> p) & 1) ? from_fixed_dp(ya, E) : from_fixed_pos(ya, E);
    out[2 * p + 2] = ((DP >> p) & 1) ? from_fixed_dp(yb, E) : from_fixed_pos(yb, E);
  }
}


// relax_links writing each link straight to out[a * stride] (when st) as soon as it is
// rounded, so that the results do not all stay live until a final store loop.
template <int DP, bool ODD, int R = 0>
__device__ __forceinline__ void relax_links_store(const long long (&X)[19], const EqPieces& q, unsigned long long Om,
                                                  long long cA, long long cD, const long long (&dq)[9], int E,
                                                  double* __restrict__ out, unsigned long long stride, bool st) {
  const long long KD = q.KA >> 1;
  const long long ev[9] = {q.KA + q.Xx, q.KA + q.Xy, q.KA + q.Xz,
                           KD + ((q.Xx + q.Xy) >> 1) + q.Yxy, KD + ((q.Xx + q.Xy) >> 1) - q.Yxy,
                           KD + ((q.Xx + q.Xz) >> 1) + q.Yxz, KD + ((q.Xx + q.Xz) >> 1) - q.Yxz,
                           KD + ((q.Xy + q.Xz) >> 1) + q.Yyz, KD + ((q.Xy + q.Xz) >> 1) - q.Yyz};
  const long long od[9] = {q.Zx, q.Zy, q.Zz,
                           (q.Zx + q.Zy) >> 1, (q.Zx - q.Zy) >> 1, (q.Zx + q.Zz) >> 1, (q.Zx - q.Zz) >> 1,
                           (q.Zy + q.Zz) >> 1, (q.Zy - q.Zz) >> 1};
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const long long c = p < 3 ? cA : cD;
    const long long d = ODD ? dq[p] : 0;
    const long long ya = relax_r<R>(X[2 * p + 1], ev[p] + od[p], Om, c + d);
    const long long yb = relax_r<R>(X[2 * p + 2], ev[p] - od[p], Om, c - d);
    const double da = ((DP >> p) & 1) ? from_fixed_dp(ya, E) : from_fixed_pos(ya, E);
    const double db = ((DP >> p) & 1) ? from_fixed_dp(yb, E) : from_fixed_pos(yb, E);
    if (st) {
      out[(2 * p + 1) * stride] = da;
      out[(2 * p + 2) * stride] = db;
    }
  }
}
}  // namespace fx

using fx::EqPieces;
using fx::UFix;

// Velocity on the fixed grid: |u_i| 2^63 and sign bits, and the six products
// u_i^2 2^62, |u_i u_j| 2^62 the equilibria need.
__device__ __forceinline__ void ufix_products(UFix& u) {
  using fx::mulhi;
  u.xx = mulhi(u.ax, u.ax);
  u.yy = mulhi(u.ay, u.ay);
  u.zz = mulhi(u.az, u.az);
  u.xy = mulhi(u.ax, u.ay);
  u.xz = mulhi(u.ax, u.az);
  u.yz = mulhi(u.ay, u.az);
}

// Recovery (Eq. 10 inverted under P = e/3) in 64-bit fixed point from the exact sums
// T00 and M on a node's grid, without an FP64 instruction: with A/4 = T00^2 - (3/4)|M|^2
// and H = T00 + sqrt(A/4) = 3 sigma / 2, sigma = 2H/3 and u = 3M / (2H).  T00 is shifted
// left until its top bit is set and M with it (|M_i| < T00 in every physical state), so
// the square root and the reciprocal act on numbers in a fixed binary range: an FP32
// seed each, then two Newton steps on 64-bit products (sigma within a few grid units,
// u within 2^-58).  Returns sigma on the grid and |u_i| 2^63 with sign bits in u; sets
// bad for T00 <= 0 or |M| >= T00 (|u| >= 1).
__device__ __forceinline__ unsigned long long fx_recover(long long T00, long long Mx, long long My, long long Mz,
                                                         UFix& u, bool& bad) {
  using namespace fx;
  const unsigned long long amx = (unsigned long long)(Mx < 0 ? -Mx : Mx);
  const unsigned long long amy = (unsigned long long)(My < 0 ? -My : My);
  const unsigned long long amz = (unsigned long long)(Mz < 0 ? -Mz : Mz);
  const unsigned long long T = T00 > 0 ? (unsigned long long)T00 : 1ull;
  bool badr = (T00 <= 0) | (amx >= T) | (amy >= T) | (amz >= T);
  const int nsh = __clzll((long long)T);                       // >= 2: T00 < 2^62
  const unsigned long long Tn = T << nsh;
  const unsigned long long mxn = badr ? 0ull : amx << nsh, myn = badr ? 0ull : amy << nsh,
                           mzn = badr ? 0ull : amz << nsh;
  const unsigned long long t2 = mulhi(Tn, Tn);
  const unsigned long long m2q = (mulhi(mxn, mxn) >> 2) + (mulhi(myn, myn) >> 2) + (mulhi(mzn, mzn) >> 2);
  badr |= m2q >= (t2 >> 2);                                    // |M| >= T00: |u| >= 1
  const unsigned long long a = t2 - 3ull * (badr ? 0ull : m2q);  // (A/4) 2^(2 nsh - 64), in (2^60, 2^64)
  // rho = (a 2^-64)^(-1/2) in (1, 4) as Y = rho 2^61 (< 2^63 even for a seed of 4):
  // Y <- Y (3 - a Y^2) / 2
  unsigned long long Y = fixed_from_float<61>(rsqrt_approx(top_float(a)));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const unsigned long long q = mulhi(a, mulhi(Y, Y));          // a rho^2 2^58
    Y = mulhi(Y, (3ull << 62) - (q << 4)) << 1;
  }
  const unsigned long long Sq = mulhi(a, Y) << 3;              // sqrt(A/4) 2^nsh, in (2^62, 2^64)
  const unsigned long long h = (Tn >> 1) + (Sq >> 1);          // H 2^(nsh - 1), in (1.5 2^62, 2^64)
  // R = 2^126 / h: R <- R (2 - h R 2^-126)
  unsigned long long R = fixed_from_float<62>(rcp_approx(top_float(h)));
#pragma unroll
  for (int it = 0; it < 2; ++it) R = mulhi(R, (1ull << 63) - mulhi(h, R)) << 2;
  // |u_i| 2^63 = (3/4)(|M_i| 2^nsh / h) 2^63 = (3/2) mulhi(|M_i| 2^nsh, R)
  const unsigned long long ux = mulhi(mxn, R), uy = mulhi(myn, R), uz = mulhi(mzn, R);
  u.ax = ux + (ux >> 1);
  u.ay = uy + (uy >> 1);
  u.az = uz + (uz >> 1);
  u.sx = (unsigned)((unsigned long long)Mx >> 63);
  u.sy = (unsigned)((unsigned long long)My >> 63);
  u.sz = (unsigned)((unsigned long long)Mz >> 63);
  bad = badr;
  // sigma = 2H/3 = (4/3) h 2^(1 - nsh)
  return mulhi(h, kTwoThirds) >> (nsh - 1);
}

// g half of the integer-pipe FP64 collide: block exponent, fixed-point values, the
// conserved sums (Eq. 10, exact on the grid), the recovery (Eq. 10 inverted under
// P = e/3) on those exact sums, and u on the fixed grid.
struct GState {
  long long G[19];
  long long dp[3];            // pair differences of the axis pairs (energy-flux rows)
  long long Sa, Sd, T00, Mx, My, Mz, Pf;
  unsigned long long sig;     // sigma on the grid
  int Eg;
  bool bad;
};
__device__ __forceinline__ void fx_g_recover(const double (&g)[19], GState& s, UFix& u) {
  using namespace fx;
  unsigned mg = 0;
#pragma unroll
  for (int a = 0; a < 19; ++a) mg = max(mg, (unsigned)__double2hiint(g[a]) & 0x7ff00000u);
  s.Eg = (int)(mg >> 20);
#pragma unroll
  for (int a = 0; a < 19; ++a) s.G[a] = to_fixed(g[a], s.Eg + 7);
  long long sp[9], dp[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    sp[p] = s.G[2 * p + 1] + s.G[2 * p + 2];
    dp[p] = s.G[2 * p + 1] - s.G[2 * p + 2];
  }
  s.dp[0] = dp[0]; s.dp[1] = dp[1]; s.dp[2] = dp[2];
  s.Sa = sp[0] + sp[1] + sp[2];
  s.Sd = ((sp[3] + sp[4]) + (sp[5] + sp[6])) + (sp[7] + sp[8]);
  s.T00 = s.G[0] + s.Sa + s.Sd;
  s.Mx = dp[0] + dp[3] + dp[4] + dp[5] + dp[6];
  s.My = dp[1] + dp[3] - dp[4] + dp[7] + dp[8];
  s.Mz = dp[2] + dp[5] - dp[6] + dp[7] - dp[8];
  bool badr;
  s.sig = fx_recover(s.T00, s.Mx, s.My, s.Mz, u, badr);
  s.Pf = (long long)s.sig - s.T00;
  ufix_products(u);
  // non-physical: T00 <= 0, |M| >= T00 (A < 0 among them), P <= 0, u^2 >= 1, or a
  // block exponent outside the normal range the grid needs
  s.bad = (s.Eg < 64) | (s.Eg > 2046) | badr | (s.Pf <= 0) | (u.xx + u.yy + u.zz >= (1ull << 62));
}

// g relaxation: Eq. 6 (BGK) or Eq. 35 (MRT as BGK plus the e, eps, q projections)
// with the equilibria of Eqs. 8-9, written to g as FP64.
template <bool MRT, bool QSEP>
__device__ __forceinline__ void fx_g_relax(const GState& s, const UFix& u, const StepConst& k, double (&g)[19]) {
  using namespace fx;
  EqPieces q;
  eq_pieces(s.sig, u, q);
  const long long SX = q.Xx + q.Xy + q.Xz;                                     // sigma u^2 / 4
  q.KA = (long long)mulhi((unsigned long long)s.Pf, kSixth) - (long long)mulhi((unsigned long long)SX, kThird);
  const long long geq0 = (long long)s.sig - 3 * s.Pf - 2 * SX;                 // sigma - 3P - sigma u^2 / 2
  const unsigned long long Om = k.Om_v;
  long long c0 = (long long)(Om >> 1), cA = c0, cD = c0;
  long long dq[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (MRT) {
    // e and eps projections of g - g^eq from the class sums (sum_axis g^eq = P,
    // sum_diag g^eq = P + sigma u^2 / 2), taken at 1/8 scale against overflow
    const long long n0 = (s.G[0] - geq0) >> 3;
    const long long nA = (s.Sa - s.Pf) >> 3;
    const long long nD = (s.Sd - s.Pf - 2 * SX) >> 3;
    const long long ae = __mul64hi(8 * nD - 11 * nA - 30 * n0, k.CE) >> 6;      // ce (M_e . (g - g^eq))
    const long long ap = __mul64hi(nD - 4 * nA + 12 * n0, k.CP) >> 2;           // cp (M_eps . (g - g^eq))
    c0 += 30 * ae - 12 * ap;
    cA += 11 * ae + 4 * ap;
    cD -= 8 * ae + ap;
    if (QSEP) {
      // energy-flux rows q_i = (5|c|^2 - 9) c_i, q^eq_i = -(2/3) M_i
      const unsigned long long h23 = kTwoThirds >> 1;
      const long long vx = ((s.Mx - 5 * s.dp[0]) >> 2) + (mulhi_su(s.Mx, kTwoThirds, h23) >> 2);
      const long long vy = ((s.My - 5 * s.dp[1]) >> 2) + (mulhi_su(s.My, kTwoThirds, h23) >> 2);
      const long long vz = ((s.Mz - 5 * s.dp[2]) >> 2) + (mulhi_su(s.Mz, kTwoThirds, h23) >> 2);
      const long long aqx = __mul64hi(vx, k.CQ) >> 1, aqy = __mul64hi(vy, k.CQ) >> 1, aqz = __mul64hi(vz, k.CQ) >> 1;
      dq[0] = 4 * aqx; dq[1] = 4 * aqy; dq[2] = 4 * aqz;
      dq[3] = -(aqx + aqy); dq[4] = -(aqx - aqy);
      dq[5] = -(aqx + aqz); dq[6] = -(aqx - aqz);
      dq[7] = -(aqy + aqz); dq[8] = -(aqy - aqz);
    }
  }
  g[0] = from_fixed<(RLB_FX_OUT_G >> 9) & 1>(relax(s.G[0], geq0, Om, c0), s.Eg);
  relax_links<RLB_FX_OUT_G, MRT && QSEP>(s.G, q, Om, cA, cD, dq, s.Eg, g);
}

// f half: block exponent, fixed-point values and N0 (Eq. 10, exact on the grid).
struct FState {
  long long F[19];
  long long N0;
  int Ef;
};
__device__ __forceinline__ void fx_f_load(const double (&f)[19], FState& s) {
  using namespace fx;
  unsigned mf = 0;
#pragma unroll
  for (int a = 0; a < 19; ++a) mf = max(mf, (unsigned)__double2hiint(f[a]) & 0x7ff00000u);
  s.Ef = (int)(mf >> 20);
#pragma unroll
  for (int a = 0; a < 19; ++a) s.F[a] = to_fixed(f[a], s.Ef + 7);
  s.N0 = s.F[0];
#pragma unroll
  for (int a = 1; a < 19; ++a) s.N0 += s.F[a];
}
__device__ __forceinline__ bool fx_f_bad(const FState& s) { return (s.Ef < 64) | (s.Ef > 2046); }

// f relaxation: Eq. 5 with the equilibrium of Eq. 7, written to f as FP64.
__device__ __forceinline__ void fx_f_relax(const FState& s, const UFix& u, const StepConst& k, double (&f)[19]) {
  using namespace fx;
  EqPieces q;
  const unsigned long long n0u = (unsigned long long)s.N0;
  eq_pieces(n0u, u, q);
  const long long SX = q.Xx + q.Xy + q.Xz;                                     // N0 u^2 / 4
  q.KA = (long long)mulhi(n0u, kEighteenth) - (long long)mulhi((unsigned long long)SX, kThird);
  const long long feq0 = (long long)mulhi(n0u, kThird) - 2 * SX;               // N0/3 - N0 u^2 / 2
  const unsigned long long Om = k.Om_f;
  const long long c = (long long)(Om >> 1);
  const long long dq0[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  f[0] = from_fixed<(RLB_FX_OUT_F >> 9) & 1>(relax(s.F[0], feq0, Om, c), s.Ef);
  relax_links<RLB_FX_OUT_F, false>(s.F, q, Om, c, c, dq0, s.Ef, f);
}

// FP64 node collide on the integer pipe: moments, recovery (fixed point), equilibria, BGK f,
// BGK / MRT g.  Same contract as node_collide_f64 with constant relaxation times; each
// link agrees with it to a few units of 2^-56 of the node's largest population.
template <bool MRT, bool QSEP>
__device__ __forceinline__ bool node_collide_fx(double (&f)[19], double (&g)[19], const StepConst& k) {
  GState gs;
  FState fs;
  UFix u;
  fx_g_recover(g, gs, u);
  fx_f_load(f, fs);
  fx_g_relax<MRT, QSEP>(gs, u, k, g);
  fx_f_relax(fs, u, k, f);
  return gs.bad | fx_f_bad(fs);
}

// ----------------------------------------------------------------------------
// Exact moment sums of FP32 populations (FP32-storage variant).
//
// The five conserved sums N0, T00, M_x, M_y, M_z of 19 FP32 values are formed
// without rounding by error-free extraction (Rump, Ogita & Oishi, "Accurate
// floating-point summation, part I", SIAM J. Sci. Comput. 31 (2008), ExtractVector):
// with sigma a power of two at least 2^5 times every |p|, q = fl(fl(sigma + p) - sigma)
// keeps the leading bits of p on the grid of sigma, r = p - q is exact, and any
// signed sum of the 19 q is exact in FP32.  Three levels (sigma, 2^-19 sigma,
// 2^-38 sigma) capture every bit of the inputs when max|p| / min|p| < 2^33 (what
// is left is below 2^-56 max|p|).  Each sum is returned as three non-overlapping
// FP32 parts; widening them bit-exactly to FP64 and adding gives the correctly
// rounded FP64 value of the exact sum -- at least as accurate as FP64 summation,
// while running on the FP32 and integer pipes instead of GB300's FP64 pipe.
struct Sums3 {
  float T00[3], Mx[3], My[3], Mz[3], Sa[3], Sd[3];
};

__device__ __forceinline__ float pow2_bits(int e) {  // 2^(e - 127), e clamped to the normal range
  e = e < 1 ? 1 : (e > 254 ? 254 : e);
  return __uint_as_float((unsigned)e << 23);
}

// Largest biased exponent of |p| over the 19 values (255 if any is Inf or NaN).  On
// magnitudes the float order is the order of the bit patterns, so the max runs as a
// float max with |.| operands (max.NaN keeps a NaN, whose pattern has exponent 255)
// instead of masking each pattern and comparing integers.
#ifndef RLB_F32_FMNMX
#define RLB_F32_FMNMX 1
#endif
__device__ __forceinline__ float fmax_keep_nan(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ int max_exp19(const float (&p)[19]) {
  if (RLB_F32_FMNMX) {
    float m = fabsf(p[0]);
#pragma unroll
    for (int a = 1; a < 19; ++a) m = fmax_keep_nan(m, fabsf(p[a]));
    return (int)(__float_as_uint(m) >> 23);
  }
  unsigned m = __float_as_uint(p[0]) & 0x7fffffffu;
#pragma unroll
  for (int a = 1; a < 19; ++a) m = max(m, __float_as_uint(p[a]) & 0x7fffffffu);
  return (int)(m >> 23);
}

// Smallest biased exponent of |p| over the 19 values (0 if any is zero or subnormal;
// a NaN is passed over, max_exp19 reports it).
__device__ __forceinline__ int min_exp19(const float (&p)[19]) {
  if (RLB_F32_FMNMX) {
    float m = fabsf(p[0]);
#pragma unroll
    for (int a = 1; a < 19; ++a) m = fminf(m, fabsf(p[a]));
    return (int)(__float_as_uint(m) >> 23);
  }
  unsigned m = __float_as_uint(p[0]) & 0x7fffffffu;
#pragma unroll
  for (int a = 1; a < 19; ++a) m = min(m, __float_as_uint(p[a]) & 0x7fffffffu);
  return (int)(m >> 23);
}

// Widen an FP32 value to FP64 by moving its bits (exact; no FP64-pipe conversion).
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned ex = (b >> 23) & 0xffu;
  // zero and subnormal parts (below 2^-126) flush to a signed zero
  const unsigned hi = ex == 0u ? (b & 0x80000000u) : ((b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3));
  return __hiloint2double((int)hi, ex == 0u ? 0 : (int)(b << 29));
}

__device__ __forceinline__ double sum3_to_f64(const float (&v)[3]) {
  return (f2d_bits(v[0]) + f2d_bits(v[1])) + f2d_bits(v[2]);
}

// Exact level sums of g: T00, M, and the axis / diagonal class sums.  LV levels
// (3 in general; 2 suffice when every value lies within 2^13 of the largest, since
// the third level's parts are then all zero); parts of unused levels are 0.
template <int LV>
__device__ __forceinline__ void exact_sums_g(const float (&g)[19], int E, Sums3& S) {
  const float sg[3] = {pow2_bits(E + 6), pow2_bits(E - 13), pow2_bits(E - 32)};
  float r[19];
#pragma unroll
  for (int a = 0; a < 19; ++a) r[a] = g[a];
#pragma unroll
  for (int L = 0; L < 3; ++L) {
    if (L >= LV) {
      S.Sa[L] = S.Sd[L] = S.T00[L] = S.Mx[L] = S.My[L] = S.Mz[L] = 0.0f;
      continue;
    }
    float q[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) {
      const float t = sg[L] + r[a];
      q[a] = t - sg[L];
      r[a] = r[a] - q[a];
    }
    float d[9];
#pragma unroll
    for (int pp = 0; pp < 9; ++pp) d[pp] = q[2 * pp + 1] - q[2 * pp + 2];
    S.Sa[L] = ((q[1] + q[2]) + (q[3] + q[4])) + (q[5] + q[6]);
    S.Sd[L] = (((q[7] + q[8]) + (q[9] + q[10])) + ((q[11] + q[12]) + (q[13] + q[14]))) +
              ((q[15] + q[16]) + (q[17] + q[18]));
    S.T00[L] = (q[0] + S.Sa[L]) + S.Sd[L];
    S.Mx[L] = ((d[0] + d[3]) + (d[4] + d[5])) + d[6];
    S.My[L] = ((d[1] + d[3]) - (d[4] - d[7])) + d[8];
    S.Mz[L] = ((d[2] + d[5]) - (d[6] - d[7])) - d[8];
  }
}

template <int LV>
__device__ __forceinline__ void exact_sum_f(const float (&f)[19], int E, float (&N0)[3]) {
  const float sg[3] = {pow2_bits(E + 6), pow2_bits(E - 13), pow2_bits(E - 32)};
  float r[19];
#pragma unroll
  for (int a = 0; a < 19; ++a) r[a] = f[a];
#pragma unroll
  for (int L = 0; L < 3; ++L) {
    if (L >= LV) {
      N0[L] = 0.0f;
      continue;
    }
    float q[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) {
      const float t = sg[L] + r[a];
      q[a] = t - sg[L];
      r[a] = r[a] - q[a];
    }
    N0[L] = ((((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + (q[6] + q[7]))) +
             (((q[8] + q[9]) + (q[10] + q[11])) + ((q[12] + q[13]) + (q[14] + q[15])))) +
            ((q[16] + q[17]) + q[18]);
  }
}

// The three level sums of one extraction are integer multiples of their grids
// 2^-24 sigma_L (sigma_1 = 2^(E+6-127), sigma_2 = 2^-19 sigma_1, sigma_3 = 2^-38 sigma_1),
// so the exact sum is K * 2^(E-56-127) with K = k1 2^38 + k2 2^19 + k3, |K| < 2^63.
// The integers are read from the float bits (exact: each part is a multiple of its grid).
__device__ __forceinline__ long long level_int(float v, int eg) {
  const unsigned b = __float_as_uint(v);
  const int es = (int)((b >> 23) & 0xffu);
  const unsigned m = (b & 0x7fffffu) | 0x800000u;
  int sh = 23 - (es - eg);
  sh = sh < 0 ? 0 : (sh > 31 ? 31 : sh);
  const long long k = es == 0 ? 0 : (long long)(m >> sh);
  return (b >> 31) ? -k : k;
}
template <int LV = 3>
__device__ __forceinline__ long long levels_to_int(const float (&v)[3], int E) {
  const long long k12 = (level_int(v[0], E - 18) << 38) + (level_int(v[1], E - 37) << 19);
  return LV > 2 ? k12 + level_int(v[2], E - 56) : k12;
}

// Two-level fast path of the exact sums, read back as integers on the FP32 pipe.  The
// first level splits each value x into q1, a multiple of 2^(E - 145), and the remainder
// r1 = x - q1 (both exact, |r1| <= 2^(E - 145)); when every value's exponent is at least
// E - 13 its last bit is at least 2^(E - 163), so r1 already lies on the second level's
// grid and is its part (the second extraction would return it unchanged).  At
// level L (grid unit u_L = 2^(E - 145 - 19 (L - 1))) every extracted part q is k u_L
// with |k| <= 2^19, so a sum S of at most 8 parts is k u_L with |k| <= 2^22; then
// S + C, C = 1.5 2^23 u_L, is exact and lies in C's binade or at its upper edge, where
// the float bit patterns step by one per u_L: k = bits(S + C) - bits(C).  The sums are
// taken in groups of at most 8 parts and the group integers added.  Returns the same
// integers as levels_to_int<2> (unit 2^(E - 183)).  Needs 16 <= E <= 240 (normal C,
// sigma) and every value within 2^13 of the largest (the third level is empty).
#ifndef RLB_F32_GROUP_INT
#define RLB_F32_GROUP_INT 1
#endif
__device__ __forceinline__ int group_int(float S, float C) {
  return (int)(__float_as_uint(S + C) - __float_as_uint(C));
}
__device__ __forceinline__ void exact_ints_g2(const float (&g)[19], int E, long long& KT, long long& KX,
                                              long long& KY, long long& KZ, float& Sa, float& Sd) {
  const float sg = pow2_bits(E + 6);
  const float C[2] = {__uint_as_float(((unsigned)(E + 5) << 23) | 0x400000u),
                      __uint_as_float(((unsigned)(E - 14) << 23) | 0x400000u)};
  float r[19];
#pragma unroll
  for (int a = 0; a < 19; ++a) r[a] = g[a];
  int kT[2], kX[2], kY[2], kZ[2];
  Sa = 0.0f;
  Sd = 0.0f;
#pragma unroll
  for (int L = 0; L < 2; ++L) {
    float q[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) {
      if (L == 0) {
        const float t = sg + r[a];
        q[a] = t - sg;
        r[a] = r[a] - q[a];
      } else {
        q[a] = r[a];   // the second level's parts are the first level's remainders
      }
    }
    float sp[9], dp[9];
#pragma unroll
    for (int pp = 0; pp < 9; ++pp) {
      sp[pp] = q[2 * pp + 1] + q[2 * pp + 2];
      dp[pp] = q[2 * pp + 1] - q[2 * pp + 2];
    }
    const float sa = (sp[0] + sp[1]) + sp[2];
    const float sd1 = (sp[3] + sp[4]) + sp[5], sd2 = (sp[6] + sp[7]) + sp[8];
    Sa += sa;
    Sd += sd1 + sd2;
    kT[L] = group_int(q[0] + sa, C[L]) + group_int(sd1, C[L]) + group_int(sd2, C[L]);
    kX[L] = group_int((dp[0] + dp[3]) + dp[4], C[L]) + group_int(dp[5] + dp[6], C[L]);
    kY[L] = group_int((dp[1] + dp[3]) - dp[4], C[L]) + group_int(dp[7] + dp[8], C[L]);
    kZ[L] = group_int((dp[2] + dp[5]) - dp[6], C[L]) + group_int(dp[7] - dp[8], C[L]);
  }
  KT = (((long long)kT[0] << 19) + kT[1]) << 19;
  KX = (((long long)kX[0] << 19) + kX[1]) << 19;
  KY = (((long long)kY[0] << 19) + kY[1]) << 19;
  KZ = (((long long)kZ[0] << 19) + kZ[1]) << 19;
}
__device__ __forceinline__ long long exact_int_f2(const float (&f)[19], int E) {
  const float sg = pow2_bits(E + 6);
  const float C[2] = {__uint_as_float(((unsigned)(E + 5) << 23) | 0x400000u),
                      __uint_as_float(((unsigned)(E - 14) << 23) | 0x400000u)};
  float r[19];
#pragma unroll
  for (int a = 0; a < 19; ++a) r[a] = f[a];
  int k[2];
#pragma unroll
  for (int L = 0; L < 2; ++L) {
    float q[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) {
      if (L == 0) {
        const float t = sg + r[a];
        q[a] = t - sg;
        r[a] = r[a] - q[a];
      } else {
        q[a] = r[a];
      }
    }
    const float s1 = ((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + q[6]);
    const float s2 = ((q[7] + q[8]) + (q[9] + q[10])) + (q[11] + q[12]);
    const float s3 = ((q[13] + q[14]) + (q[15] + q[16])) + (q[17] + q[18]);
    k[L] = group_int(s1, C[L]) + group_int(s2, C[L]) + group_int(s3, C[L]);
  }
  return (((long long)k[0] << 19) + k[1]) << 19;
}

// FP32-storage node collide: the conserved sums exact (above) and delivered in
// FP64, the recovery (sqrt, reciprocal) in FP64; equilibria, MRT projection and
// relaxation in FP32 with one rounding on store.  Split into the g part (sums,
// recovery, g relaxation) and the f part (N0, f relaxation), which share only u.
struct G32 {
  float sg, P, su2, kg, geq0;   // sigma, P, sigma u^2, sigma u^2 - 2P (= -(3P - 1.5 sigma u^2) / 1.5),
                                // g^eq_0
  float Sa, Sd;                 // axis / diagonal class sums of g (MRT)
  float Mx, My, Mz;             // momentum (energy-flux rows)
  float ux, uy, uz;
  bool bad;
};
template <bool MRT, bool QSEP>
__device__ __forceinline__ void f32s_g_recover(const float (&g)[19], G32& s) {
  Sums3 S;
  const int Eg = max_exp19(g);
  // exact sums as integers K * 2^(E - 183), rounded once to FP64 by integer bit
  // assembly (fx::from_fixed_int with unit scale: no FP64-pipe conversion); the
  // recovery is homogeneous of degree 1 in (T00, M) (u is scale free), so it runs on
  // the unscaled K and scales after
  long long KT, KX, KY, KZ;
  const bool two = min_exp19(g) >= Eg - 13;   // two extraction levels are exact
  if (RLB_F32_GROUP_INT && two && Eg >= 16 && Eg <= 240) {
    float sa, sd;
    exact_ints_g2(g, Eg, KT, KX, KY, KZ, sa, sd);
    S.Sa[0] = sa; S.Sa[1] = 0.0f; S.Sa[2] = 0.0f;
    S.Sd[0] = sd; S.Sd[1] = 0.0f; S.Sd[2] = 0.0f;
  } else if (two) {
    exact_sums_g<2>(g, Eg, S);
    KT = levels_to_int<2>(S.T00, Eg);
    KX = levels_to_int<2>(S.Mx, Eg);
    KY = levels_to_int<2>(S.My, Eg);
    KZ = levels_to_int<2>(S.Mz, Eg);
  } else {
    exact_sums_g<3>(g, Eg, S);
    KT = levels_to_int<3>(S.T00, Eg);
    KX = levels_to_int<3>(S.Mx, Eg);
    KY = levels_to_int<3>(S.My, Eg);
    KZ = levels_to_int<3>(S.Mz, Eg);
  }
  const double Tu = fx::from_fixed_int(KT, 1079);
  const double Mxu = fx::from_fixed_int(KX, 1079);
  const double Myu = fx::from_fixed_int(KY, 1079);
  const double Mzu = fx::from_fixed_int(KZ, 1079);
  const int eg = Eg - 183;
  const double MM = fma(Mxu, Mxu, fma(Myu, Myu, Mzu * Mzu));
  // sigma is the larger root of 3 s^2 - 4 T00 s + |M|^2 = 0 (Eq. 10 inverted): an FP32
  // seed s0 from the closed form on values scaled by 2^-64, then one Newton step on the
  // quadratic in FP64, s0 - q(s0) / q'(s0), with q'(s0) = 6 s0 - 4 T00 taken in FP32
  // (relative error about 2^-42, far below the FP32 rounding of everything it feeds);
  // 1 / sigma from an FP32 seed and one Newton step
  const float tf = d2f_trunc_bits_s(Tu, -64), xf = d2f_trunc_bits_s(Mxu, -64);
  const float yf = d2f_trunc_bits_s(Myu, -64), zf = d2f_trunc_bits_s(Mzu, -64);
  const float Af = fmaf(4.0f * tf, tf, -3.0f * fmaf(xf, xf, fmaf(yf, yf, zf * zf)));
  float rA, r0;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(rA) : "f"(Af));
  const float s0f = fmaf(2.0f, tf, rA) * (1.0f / 3.0f);
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rA) : "f"(fmaf(6.0f, s0f, -4.0f * tf)));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(s0f));
  const double s0 = widen_seed_s(s0f, 64);
  const double T4 = scale_pow2(Tu, 2);
  const double q = fma(s0, fma(3.0, s0, -T4), MM);
  const double sgu = fma(-q, widen_seed_s(rA, -64), s0);
  const double y = widen_seed_s(r0, -64);
  const double is = fma(y, fma(-sgu, y, 1.0), y);
  const double Pu = sgu - Tu;
  // per-node equilibrium constants (they cancel, sigma ~ 4P): FP64, then one rounding;
  // at the root |M|^2 / sigma = 4 T00 - 3 sigma, so the constants are linear in sigma
  // and T00: sigma u^2 = 4 T00 - 3 sigma; sigma u^2 - 2P, the equilibria's
  // 3P - 1.5 sigma u^2 over -1.5 (the FP32 constants carry the factor); and
  // g^eq_0 = sigma - 3P - sigma u^2 / 2 = T00 - sigma / 2
  const double su2u = fma(-3.0, sgu, T4);
  s.su2 = d2f_rn_bits_scaled(su2u, eg);
  s.kg = d2f_rn_bits_scaled(fma(-2.0, Pu, su2u), eg);
  s.geq0 = d2f_rn_bits_scaled(fma(-0.5, sgu, Tu), eg);
  // u to FP32 by the FP64 pipe's conversion (round to nearest; the other narrowings
  // stay on the integer pipes, which carry more of this kernel's work)
  s.ux = __double2float_rn(Mxu * is);
  s.uy = __double2float_rn(Myu * is);
  s.uz = __double2float_rn(Mzu * is);
  s.sg = d2f_rn_bits_scaled(sgu, eg);
  s.P = d2f_rn_bits_scaled(Pu, eg);
  if (MRT) {
    // non-equilibrium class sums in FP32 (their rounding is far below the FP32 storage rounding)
    s.Sa = (S.Sa[0] + S.Sa[1]) + S.Sa[2];
    s.Sd = (S.Sd[0] + S.Sd[1]) + S.Sd[2];
  }
  if (QSEP) {
    s.Mx = d2f_rn_bits_scaled(Mxu, eg);
    s.My = d2f_rn_bits_scaled(Myu, eg);
    s.Mz = d2f_rn_bits_scaled(Mzu, eg);
  }
  const float u2 = fmaf(s.ux, s.ux, fmaf(s.uy, s.uy, s.uz * s.uz));
  // A > 0 (its FP32 seed value), T00 > 0, P > 0 (finite), u^2 < 1 (on the rounded velocity; NaN fails)
  s.bad = !(Af > 0.0f && pos_finite_hi(Tu) && pos_finite_hi(Pu) && u2 < 1.0f) || Eg == 255;
}

template <bool MRT, bool QSEP>
__device__ __forceinline__ void f32s_g_relax(float (&g)[19], const G32& s, const StepConst& k) {
  float cu[9];
  pair_cu<float>(s.ux, s.uy, s.uz, cu);
  float KA = k.gA_k_f * s.kg, KD = k.gD_k_f * s.kg;
  const float SA = k.gA_s_f * s.sg, SD = k.gD_s_f * s.sg;
  const float AA = k.gA_a_f * s.sg, AD = k.gD_a_f * s.sg;
  float g0n = fmaf(k.omv1_f, g[0], k.omv_f * s.geq0);
  float dq[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) dq[p] = 0.0f;
  if (MRT) {
    const float n0 = g[0] - s.geq0;
    const float nA = s.Sa - s.P;
    const float nD = fmaf(-0.5f, s.su2, s.Sd - s.P);
    const float ne = fmaf(8.0f, nD, fmaf(-11.0f, nA, -30.0f * n0));
    const float np = fmaf(-4.0f, nA, fmaf(12.0f, n0, nD));
    const float ae = k.ce_f * ne, ap = k.cp_f * np;
    g0n = g0n + fmaf(30.0f, ae, -12.0f * ap);
    KA = KA + fmaf(11.0f, ae, 4.0f * ap);
    KD = KD - fmaf(8.0f, ae, ap);
    if (QSEP) {
      const float qeq = -2.0f / 3.0f;
      const float d0 = g[1] - g[2], d1 = g[3] - g[4], d2 = g[5] - g[6], d3 = g[7] - g[8], d4 = g[9] - g[10];
      const float d5 = g[11] - g[12], d6 = g[13] - g[14], d7 = g[15] - g[16], d8 = g[17] - g[18];
      const float qx = fmaf(-4.0f, d0, ((d3 + d4) + d5) + d6);
      const float qy = fmaf(-4.0f, d1, ((d3 - d4) + d7) + d8);
      const float qz = fmaf(-4.0f, d2, ((d5 - d6) + d7) - d8);
      const float cq = k.cq_f;
      const float aqx = cq * fmaf(-qeq, s.Mx, qx);
      const float aqy = cq * fmaf(-qeq, s.My, qy);
      const float aqz = cq * fmaf(-qeq, s.Mz, qz);
      dq[0] = 4.0f * aqx; dq[1] = 4.0f * aqy; dq[2] = 4.0f * aqz;
      dq[3] = -(aqx + aqy); dq[4] = -(aqx - aqy);
      dq[5] = -(aqx + aqz); dq[6] = -(aqx - aqz);
      dq[7] = -(aqy + aqz); dq[8] = -(aqy - aqz);
    }
  }
  g[0] = g0n;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const bool ax = p < 3;
    const float ev = fmaf(ax ? SA : SD, cu[p] * cu[p], ax ? KA : KD);
    float od = (ax ? AA : AD) * cu[p];
    if (MRT && QSEP) od += dq[p];
    g[2 * p + 1] = fmaf(k.omv1_f, g[2 * p + 1], ev + od);
    g[2 * p + 2] = fmaf(k.omv1_f, g[2 * p + 2], ev - od);
  }
}

// f part: N0 (exact sum rounded to FP32 through FP64) and the flag of a non-finite f.
__device__ __forceinline__ float f32s_f_sum(const float (&f)[19], bool& bad) {
  float N0p[3];
  const int Ef = max_exp19(f);
  bad = Ef == 255;
  long long K;
  const bool two = min_exp19(f) >= Ef - 13;   // two extraction levels are exact
  if (RLB_F32_GROUP_INT && two && Ef >= 16 && Ef <= 240) {
    K = exact_int_f2(f, Ef);
  } else if (two) {
    exact_sum_f<2>(f, Ef, N0p);
    K = levels_to_int<2>(N0p, Ef);
  } else {
    exact_sum_f<3>(f, Ef, N0p);
    K = levels_to_int<3>(N0p, Ef);
  }
  return d2f_rn_bits_scaled(fx::from_fixed_int(K, 1079), Ef - 183);
}

__device__ __forceinline__ void f32s_f_relax(float (&f)[19], float N0, float ux, float uy, float uz,
                                             const StepConst& k) {
  const float u2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
  float cu[9];
  pair_cu<float>(ux, uy, uz, cu);
  const float kf = fmaf(-1.5f * N0, u2, N0);
  const float KA = k.fA_k_f * kf, KD = k.fD_k_f * kf;
  const float SA = k.fA_s_f * N0, SD = k.fD_s_f * N0;
  const float AA = k.fA_a_f * N0, AD = k.fD_a_f * N0;
  f[0] = fmaf(k.omf1_f, f[0], k.f0_k_f * kf);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const bool ax = p < 3;
    const float ev = fmaf(ax ? SA : SD, cu[p] * cu[p], ax ? KA : KD);
    const float od = (ax ? AA : AD) * cu[p];
    f[2 * p + 1] = fmaf(k.omf1_f, f[2 * p + 1], ev + od);
    f[2 * p + 2] = fmaf(k.omf1_f, f[2 * p + 2], ev - od);
  }
}

template <bool MRT, bool QSEP>
__device__ __forceinline__ bool node_collide_f32s(float (&f)[19], float (&g)[19], const StepConst& k) {
  G32 s;
  f32s_g_recover<MRT, QSEP>(g, s);
  bool fbad;
  const float N0 = f32s_f_sum(f, fbad);
  f32s_f_relax(f, N0, s.ux, s.uy, s.uz, k);
  f32s_g_relax<MRT, QSEP>(g, s, k);
  return s.bad | fbad;
}

// Equilibrium populations of given fields (Eqs. 7-9, P = e/3), FP64.
__device__ __forceinline__ void node_equilibrium(double e, double ux, double uy, double uz, double n,
                                                 double (&f)[19], double (&g)[19]) {
  const double u2 = fma(ux, ux, fma(uy, uy, uz * uz));
  const double g2 = 1.0 / (1.0 - u2);
  const double P = e * (1.0 / 3.0);
  const double sigma = (e + P) * g2;
  const double N0 = n * sqrt(g2);
  double cu[9];
  pair_cu<double>(ux, uy, uz, cu);
  const double wA = 1.0 / 18.0, wD = 1.0 / 36.0;
  const double kf = N0 * (1.0 - 1.5 * u2);
  const double kg = 3.0 * P - 1.5 * sigma * u2;
  f[0] = (1.0 / 3.0) * kf;
  g[0] = sigma - 3.0 * P - 0.5 * sigma * u2;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const double w = p < 3 ? wA : wD;
    const double c2 = 4.5 * cu[p] * cu[p];
    const double fe = w * (kf + N0 * c2), fo = w * 3.0 * N0 * cu[p];
    const double ge = w * (kg + sigma * c2), go = w * 3.0 * sigma * cu[p];
    f[2 * p + 1] = fe + fo;
    f[2 * p + 2] = fe - fo;
    g[2 * p + 1] = ge + go;
    g[2 * p + 2] = ge - go;
  }
}

// ---------------------------------------------------------------------------
// D2Q9 (the MRT model of Sec. V.A, Eqs. 30-35), FP64.  Link order: 0 rest;
// pairs p = 0..3 hold links 2p+1 (direction c_p) and 2p+2 (-c_p): p0 +x, p1 +y,
// p2 (1,1), p3 (1,-1).  Rest equilibrium Eq. 32: g^eq_0 = sigma - (8/3) P - (2/3)
// sigma u^2; moving links Eq. 33 (the Eq. 9 form with the D2Q9 weights).  Class
// sums of g^eq: axis (4/3) P + sigma u^2 / 3, diagonal P / 3 + sigma u^2 / 3.  MRT
// rows e = 3|c|^2 - 4 (-4, -1, 2), eps (4, -2, 1), q_i = (3|c|^2 - 5) c_i.
__host__ __device__ constexpr int d2_cx(int a) {
  constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
  return t[a];
}
__host__ __device__ constexpr int d2_cy(int a) {
  constexpr int t[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
  return t[a];
}

template <typename S>
__device__ __forceinline__ void node_moments_d2q9(const S (&f)[9], const S (&g)[9], double (&dp)[4], double& Sa,
                                                  double& Sd, NodeMacro& m) {
  double sp[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const double a = (double)g[2 * p + 1], b = (double)g[2 * p + 2];
    sp[p] = a + b;
    dp[p] = a - b;
  }
  Sa = sp[0] + sp[1];
  Sd = sp[2] + sp[3];
  m.T00 = ((double)g[0] + Sa) + Sd;
  m.Mx = (dp[0] + dp[2]) + dp[3];
  m.My = (dp[1] + dp[2]) - dp[3];
  m.Mz = 0.0;
  m.N0 = (double)f[0] + ((((double)f[1] + (double)f[2]) + ((double)f[3] + (double)f[4])) +
                         (((double)f[5] + (double)f[6]) + ((double)f[7] + (double)f[8])));
}

// D2Q9 relaxation coefficients for given omega_f, omega_v (weights 4/9, 1/9, 1/36).
__device__ __forceinline__ void set_bgk_coefficients_d2q9(StepConst& k, double omf, double omv) {
  const double wA = 1.0 / 9.0, wD = 1.0 / 36.0, w0 = 4.0 / 9.0;
  k.omf = omf; k.omf1 = 1.0 - omf;
  k.fA_k = omf * wA; k.fD_k = omf * wD; k.f0_k = omf * w0;
  k.fA_s = 4.5 * omf * wA; k.fD_s = 4.5 * omf * wD; k.fA_a = 3.0 * omf * wA; k.fD_a = 3.0 * omf * wD;
  k.omv = omv; k.omv1 = 1.0 - omv;
  k.gA_k = omv * wA; k.gD_k = omv * wD;
  k.gA_s = 4.5 * omv * wA; k.gD_s = 4.5 * omv * wD; k.gA_a = 3.0 * omv * wA; k.gD_a = 3.0 * omv * wD;
}

template <bool MRT, bool QSEP, bool ETA = false>
__device__ __forceinline__ bool node_collide_d2q9_f64(double (&f)[9], double (&g)[9], const StepConst& kc,
                                                      NodeMacro& m) {
  double dp[4], Sa, Sd;
  node_moments_d2q9<double>(f, g, dp, Sa, Sd, m);
  node_recover_fast(m);
  StepConst k = kc;
  if (ETA) {
    const double tv = tau_eta_over_s(kc.eta_s, m);
    const double omv = 1.0 / tv;
    set_bgk_coefficients_d2q9(k, kc.tauf_local ? omv : kc.omf, omv);
    if (MRT) set_mrt_eta_coefficients(k, tv, 9);
  }
  double cu[4];
  cu[0] = m.ux; cu[1] = m.uy; cu[2] = m.ux + m.uy; cu[3] = m.ux - m.uy;
  {
    const double kf = fma(-1.5 * m.N0, m.u2, m.N0);
    const double KA = k.fA_k * kf, KD = k.fD_k * kf;
    const double SA = k.fA_s * m.N0, SD = k.fD_s * m.N0;
    const double AA = k.fA_a * m.N0, AD = k.fD_a * m.N0;
    f[0] = fma(k.omf1, f[0], k.f0_k * kf);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const bool ax = p < 2;
      const double ev = fma(ax ? SA : SD, cu[p] * cu[p], ax ? KA : KD);
      const double od = (ax ? AA : AD) * cu[p];
      f[2 * p + 1] = fma(k.omf1, f[2 * p + 1], ev + od);
      f[2 * p + 2] = fma(k.omf1, f[2 * p + 2], ev - od);
    }
  }
  {
    const double su2 = m.sigma * m.u2;
    const double kg = fma(-1.5, su2, 3.0 * m.P);
    const double geq0 = fma(-2.0 / 3.0, su2, fma(-8.0 / 3.0, m.P, m.sigma));
    double KA = k.gA_k * kg, KD = k.gD_k * kg;
    const double SA = k.gA_s * m.sigma, SD = k.gD_s * m.sigma;
    const double AA = k.gA_a * m.sigma, AD = k.gD_a * m.sigma;
    double g0n = fma(k.omv1, g[0], k.omv * geq0);
    double dq[4] = {0.0, 0.0, 0.0, 0.0};
    if (MRT) {
      const double n0 = g[0] - geq0;
      const double nA = Sa - fma(1.0 / 3.0, su2, (4.0 / 3.0) * m.P);
      const double nD = Sd - (m.P + su2) * (1.0 / 3.0);
      const double ne = fma(2.0, nD, fma(-4.0, n0, -nA));
      const double np = fma(-2.0, nA, fma(4.0, n0, nD));
      const double ae = k.ce * ne, ap = k.cp * np;
      g0n = g0n + 4.0 * (ae - ap);
      KA = KA + fma(2.0, ap, ae);
      KD = KD - fma(2.0, ae, ap);
      if (QSEP) {
        const double aqx = k.cq * (fma(-2.0, dp[0], dp[2] + dp[3]) + m.Mx);
        const double aqy = k.cq * (fma(-2.0, dp[1], dp[2] - dp[3]) + m.My);
        dq[0] = 2.0 * aqx;
        dq[1] = 2.0 * aqy;
        dq[2] = -(aqx + aqy);
        dq[3] = -(aqx - aqy);
      }
    }
    g[0] = g0n;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const bool ax = p < 2;
      const double ev = fma(ax ? SA : SD, cu[p] * cu[p], ax ? KA : KD);
      double od = (ax ? AA : AD) * cu[p];
      if (MRT && QSEP) od += dq[p];
      g[2 * p + 1] = fma(k.omv1, g[2 * p + 1], ev + od);
      g[2 * p + 2] = fma(k.omv1, g[2 * p + 2], ev - od);
    }
  }
  return m.bad;
}

// D2Q9 equilibrium populations of given fields (Eqs. 7, 32, 33), FP64.
__device__ __forceinline__ void node_equilibrium_d2q9(double e, double ux, double uy, double n, double (&f)[9],
                                                      double (&g)[9]) {
  const double u2 = fma(ux, ux, uy * uy);
  const double g2 = 1.0 / (1.0 - u2);
  const double P = e * (1.0 / 3.0);
  const double sigma = (e + P) * g2;
  const double N0 = n * sqrt(g2);
  const double cu[4] = {ux, uy, ux + uy, ux - uy};
  const double kf = N0 * (1.0 - 1.5 * u2);
  const double kg = 3.0 * P - 1.5 * sigma * u2;
  f[0] = (4.0 / 9.0) * kf;
  g[0] = sigma - (8.0 / 3.0) * P - (2.0 / 3.0) * sigma * u2;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const double w = p < 2 ? 1.0 / 9.0 : 1.0 / 36.0;
    const double c2 = 4.5 * cu[p] * cu[p];
    const double fe = w * (kf + N0 * c2), fo = w * 3.0 * N0 * cu[p];
    const double ge = w * (kg + sigma * c2), go = w * 3.0 * sigma * cu[p];
    f[2 * p + 1] = fe + fo;
    f[2 * p + 2] = fe - fo;
    g[2 * p + 1] = ge + go;
    g[2 * p + 2] = ge - go;
  }
}

}  // namespace rlb
