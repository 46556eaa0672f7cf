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
#pragma once
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
};

inline StepConst make_step_const(double tau_f, double tau_v, double tau_e, double tau_eps, double tau_q,
                                 bool mrt) {
  StepConst k{};
  const double wA = 1.0 / 18.0, wD = 1.0 / 36.0, w0 = 1.0 / 3.0;
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
    k.ce = (1.0 / tau_e - k.omv) / 2394.0;
    k.cp = (1.0 / tau_eps - k.omv) / 252.0;
    k.cq = (1.0 / tq - k.omv) / 40.0;
  }
  k.omf_f = (float)k.omf; k.omf1_f = (float)k.omf1;
  k.fA_k_f = (float)k.fA_k; k.fD_k_f = (float)k.fD_k; k.f0_k_f = (float)k.f0_k;
  k.fA_s_f = (float)k.fA_s; k.fD_s_f = (float)k.fD_s; k.fA_a_f = (float)k.fA_a; k.fD_a_f = (float)k.fD_a;
  k.omv_f = (float)k.omv; k.omv1_f = (float)k.omv1;
  k.gA_k_f = (float)k.gA_k; k.gD_k_f = (float)k.gD_k;
  k.gA_s_f = (float)k.gA_s; k.gD_s_f = (float)k.gD_s; k.gA_a_f = (float)k.gA_a; k.gD_a_f = (float)k.gD_a;
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
template <bool MRT, bool QSEP>
__device__ __forceinline__ bool node_collide_f64(double (&f)[19], double (&g)[19], const StepConst& k) {
  double sp[9], dp[9], Sa, Sd;
  NodeMacro m;
  node_moments<double>(f, g, sp, dp, Sa, Sd, m);
  node_recover(m);

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
        const double qx = fma(-4.0, dp[0], ((dp[3] + dp[4]) + dp[5]) + dp[6]);
        const double qy = fma(-4.0, dp[1], ((dp[3] - dp[4]) + dp[7]) + dp[8]);
        const double qz = fma(-4.0, dp[2], ((dp[5] - dp[6]) + dp[7]) - dp[8]);
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

// FP32-storage node collide: loads widened to FP64 for the moment sums, the
// recovery (sqrt, reciprocal) in FP64; equilibria and relaxation in FP32.
template <bool MRT, bool QSEP>
__device__ __forceinline__ bool node_collide_f32s(float (&f)[19], float (&g)[19], const StepConst& k) {
  double sp[9], dp[9], Sa, Sd;
  NodeMacro m;
  node_moments<float>(f, g, sp, dp, Sa, Sd, m);
  node_recover(m);

  const float ux = (float)m.ux, uy = (float)m.uy, uz = (float)m.uz;
  const float u2 = (float)m.u2, N0 = (float)m.N0, sg = (float)m.sigma, P = (float)m.P;
  float cu[9];
  pair_cu<float>(ux, uy, uz, cu);
  {
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
  {
    const double su2d = m.sigma * m.u2;
    const float su2 = (float)su2d;
    const float P3 = 3.0f * P;
    const float kg = fmaf(-1.5f, su2, P3);
    const double geq0d = fma(-0.5, su2d, m.sigma - 3.0 * m.P);
    const float geq0 = (float)geq0d;
    float KA = k.gA_k_f * kg, KD = k.gD_k_f * kg;
    const float SA = k.gA_s_f * sg, SD = k.gD_s_f * sg;
    const float AA = k.gA_a_f * sg, AD = k.gD_a_f * sg;
    float g0n = fmaf(k.omv1_f, g[0], k.omv_f * geq0);
    float dq[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) dq[p] = 0.0f;
    if (MRT) {
      const double n0 = (double)g[0] - geq0d;
      const double nA = Sa - m.P;
      const double nD = fma(-0.5, su2d, Sd - m.P);
      const double ne = fma(8.0, nD, fma(-11.0, nA, -30.0 * n0));
      const double np = fma(-4.0, nA, fma(12.0, n0, nD));
      const float ae = (float)(k.ce * ne), ap = (float)(k.cp * np);
      g0n = g0n + fmaf(30.0f, ae, -12.0f * ap);
      KA = KA + fmaf(11.0f, ae, 4.0f * ap);
      KD = KD - fmaf(8.0f, ae, ap);
      if (QSEP) {
        const double qeq = -2.0 / 3.0;
        const double qx = fma(-4.0, dp[0], ((dp[3] + dp[4]) + dp[5]) + dp[6]);
        const double qy = fma(-4.0, dp[1], ((dp[3] - dp[4]) + dp[7]) + dp[8]);
        const double qz = fma(-4.0, dp[2], ((dp[5] - dp[6]) + dp[7]) - dp[8]);
        const float aqx = (float)(k.cq * fma(-qeq, m.Mx, qx));
        const float aqy = (float)(k.cq * fma(-qeq, m.My, qy));
        const float aqz = (float)(k.cq * fma(-qeq, m.Mz, qz));
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
  return m.bad;
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

}  // namespace rlb
