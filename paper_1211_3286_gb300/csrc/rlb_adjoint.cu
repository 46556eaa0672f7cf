// rlb_adjoint.cu -- reverse-mode (adjoint) kernels of the fused step and the
// checkpointed driver rlb_adjoint (include/rlb_adjoint.h).
//
// Per step the forward map is g^{t+1} = C(h; omega), h = S g^t, with S the pull
// stream and C the per-node g collide of rlb_node.cuh (FP64).  The adjoint of step
// t computes, per node, mu^t = C_h^T lambda^{t+1} and omega_bar += C_omega^T
// lambda^{t+1} (the forward intermediates are recomputed from h, then the chain is
// walked backwards by hand), where lambda^{t+1} = S^T mu^{t+1} is gathered at the node
// inside the same kernel: the adjoint of "node x pulls link a from src(x)" is "node y
// collects link a from every x with src(x) = y" -- one node for a periodic axis, and
// for a zero-gradient axis also the edge node's own clamped pull.  Small lattices run
// the reverse step with four threads per node in two warp roles (k_adj_step_ws), larger
// ones with one thread per node (k_adj_step).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rlb.h"
#include "../../include/rlb_adjoint.h"
#include "rlb_internal.h"
#include "rlb_node.cuh"

using namespace rlb;

namespace {

constexpr int kThreads = 128;

struct AGeo {
  int nx, ny, nz;
  int zgx, zgy, zgz;
  unsigned long long n;
};

__device__ __forceinline__ int pull_src(int i, int c, int n, int zg) {
  int s = i - c;
  if (s < 0) s = zg ? 0 : n - 1;
  if (s >= n) s = zg ? n - 1 : 0;
  return s;
}

// Nodes x of one axis whose pull with offset c lands on i (at most two).
__device__ __forceinline__ int preimages(int i, int c, int n, int zg, int (&x)[2]) {
  if (c == 0) { x[0] = i; return 1; }
  if (!zg) { int v = i + c; if (v < 0) v += n; if (v >= n) v -= n; x[0] = v; return 1; }
  int k = 0;
  if (i + c >= 0 && i + c < n) x[k++] = i + c;
  if ((c == 1 && i == 0) || (c == -1 && i == n - 1)) x[k++] = i;
  return k;
}

struct GFwd {
  double sp[9], dp[9], Sa, Sd, T00, Mx, My, Mz, MM, A, sA, sigma, is, ux, uy, uz, P, u2, su2, P3, kg, geq0;
  double n0, nA, nD, ne, np, cu[9];
};

__device__ __forceinline__ void gforward(const double (&h)[19], const StepConst& k, bool mrt, GFwd& F) {
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    F.sp[p] = h[2 * p + 1] + h[2 * p + 2];
    F.dp[p] = h[2 * p + 1] - h[2 * p + 2];
  }
  F.Sa = (F.sp[0] + F.sp[1]) + F.sp[2];
  F.Sd = ((F.sp[3] + F.sp[4]) + (F.sp[5] + F.sp[6])) + (F.sp[7] + F.sp[8]);
  F.T00 = (h[0] + F.Sa) + F.Sd;
  F.Mx = ((F.dp[0] + F.dp[3]) + (F.dp[4] + F.dp[5])) + F.dp[6];
  F.My = ((F.dp[1] + F.dp[3]) - (F.dp[4] - F.dp[7])) + F.dp[8];
  F.Mz = ((F.dp[2] + F.dp[5]) - (F.dp[6] - F.dp[7])) - F.dp[8];
  F.MM = fma(F.Mx, F.Mx, fma(F.My, F.My, F.Mz * F.Mz));
  F.A = fma(4.0 * F.T00, F.T00, -3.0 * F.MM);
  // sqrt and reciprocal: FP32 seeds refined by Newton steps to the FP64 rounding level
  // (a lone warp per SM issues these on its FP64 pipe, so the short forms matter)
  F.sA = sqrt_seeded(F.A);
  F.sigma = fma(2.0, F.T00, F.sA) * (1.0 / 3.0);
  F.is = rcp_seeded(F.sigma);
  F.ux = F.Mx * F.is;
  F.uy = F.My * F.is;
  F.uz = F.Mz * F.is;
  F.P = F.sigma - F.T00;
  F.u2 = fma(F.ux, F.ux, fma(F.uy, F.uy, F.uz * F.uz));
  F.su2 = F.sigma * F.u2;
  F.P3 = 3.0 * F.P;
  F.kg = fma(-1.5, F.su2, F.P3);
  F.geq0 = fma(-0.5, F.su2, F.sigma - F.P3);
  pair_cu<double>(F.ux, F.uy, F.uz, F.cu);
  if (mrt) {
    F.n0 = h[0] - F.geq0;
    F.nA = F.Sa - F.P;
    F.nD = fma(-0.5, F.su2, F.Sd - F.P);
    F.ne = fma(8.0, F.nD, fma(-11.0, F.nA, -30.0 * F.n0));
    F.np = fma(-4.0, F.nA, fma(12.0, F.n0, F.nD));
  }
}

// Reverse of the recovery + moments given cotangents of (sigma, P via Pb, u, T00):
// accumulates into hb.
__device__ __forceinline__ void recovery_moments_reverse(const GFwd& F, double sigmab, double Pb, double uxb,
                                                         double uyb, double uzb, double T00b, double Sab, double Sdb,
                                                         double h0b_extra, double (&hb)[19]) {
  // P = sigma - T00
  sigmab += Pb;
  T00b -= Pb;
  // u = M * is
  double Mxb = F.is * uxb, Myb = F.is * uyb, Mzb = F.is * uzb;
  const double isb = F.Mx * uxb + F.My * uyb + F.Mz * uzb;
  // is = 1 / sigma
  sigmab -= F.is * F.is * isb;
  // sigma = (2 T00 + sA) / 3
  T00b += (2.0 / 3.0) * sigmab;
  const double sAb = sigmab * (1.0 / 3.0);
  // sA = sqrt(A)
  const double Ab = sAb * 0.5 * rcp_seeded(F.sA);
  // A = 4 T00^2 - 3 MM
  T00b += 8.0 * F.T00 * Ab;
  const double MMb = -3.0 * Ab;
  Mxb += 2.0 * F.Mx * MMb;
  Myb += 2.0 * F.My * MMb;
  Mzb += 2.0 * F.Mz * MMb;
  // T00 = h0 + Sa + Sd ; Sa, Sd from pair sums ; M from pair differences
  Sab += T00b;
  Sdb += T00b;
  hb[0] += T00b + h0b_extra;
  double dpb[9];
  dpb[0] = Mxb; dpb[1] = Myb; dpb[2] = Mzb;
  dpb[3] = Mxb + Myb; dpb[4] = Mxb - Myb;
  dpb[5] = Mxb + Mzb; dpb[6] = Mxb - Mzb;
  dpb[7] = Myb + Mzb; dpb[8] = Myb - Mzb;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const double spb = p < 3 ? Sab : Sdb;
    hb[2 * p + 1] += spb + dpb[p];
    hb[2 * p + 2] += spb - dpb[p];
  }
}

// Vector-Jacobian product of the g collide: given h (pulled) and lo (cotangent of
// the post-collision g), returns hb = C_h^T lo and the omega cotangents.
template <bool MRT>
__device__ __forceinline__ void g_collide_vjp(const double (&h)[19], const double (&lo)[19], const StepConst& k,
                                              double (&hb)[19], double& wvb, double& web, double& wpb) {
  GFwd F;
  gforward(h, k, MRT, F);
  const double om = k.omv, om1 = k.omv1;
  const double wA = 1.0 / 18.0, wD = 1.0 / 36.0;
  double SAb = 0, SDb = 0, AAb = 0, ADb = 0, KAb = 0, KDb = 0, cub[9];
  const double SA = k.gA_s * F.sigma, SD = k.gD_s * F.sigma, AA = k.gA_a * F.sigma, AD = k.gD_a * F.sigma;
  wvb = 0;
  web = 0;
  wpb = 0;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const double la = lo[2 * p + 1], lb = lo[2 * p + 2];
    hb[2 * p + 1] = om1 * la;
    hb[2 * p + 2] = om1 * lb;
    wvb -= h[2 * p + 1] * la + h[2 * p + 2] * lb;
    const double evb = la + lb, odb = la - lb;
    const double c = F.cu[p];
    if (p < 3) {
      SAb += evb * c * c; KAb += evb; AAb += odb * c;
      cub[p] = evb * 2.0 * SA * c + odb * AA;
    } else {
      SDb += evb * c * c; KDb += evb; ADb += odb * c;
      cub[p] = evb * 2.0 * SD * c + odb * AD;
    }
  }
  // rest link: out0 = (1 - om) h0 + om geq0 (+ 30 ae - 12 ap)
  const double l0 = lo[0];
  hb[0] = om1 * l0;
  wvb += (F.geq0 - h[0]) * l0;
  double geq0b = om * l0;
  double aeb = 30.0 * l0, apb = -12.0 * l0;
  // K_A = om wA kg + 11 ae + 4 ap ; K_D = om wD kg - 8 ae - ap
  aeb += 11.0 * KAb - 8.0 * KDb;
  apb += 4.0 * KAb - KDb;
  const double kgb = om * (wA * KAb + wD * KDb);
  wvb += F.kg * (wA * KAb + wD * KDb);
  // S = 4.5 om w sigma, A = 3 om w sigma
  double sigmab = om * (4.5 * (wA * SAb + wD * SDb) + 3.0 * (wA * AAb + wD * ADb));
  wvb += F.sigma * (4.5 * (wA * SAb + wD * SDb) + 3.0 * (wA * AAb + wD * ADb));
  double Sab = 0, Sdb = 0, Pb = 0, su2b = 0, h0x = 0;
  if (MRT) {
    const double neb = k.ce * aeb, npb = k.cp * apb;
    const double ceb = F.ne * aeb, cpb = F.np * apb;
    web += ceb / 2394.0;
    wpb += cpb / 252.0;
    wvb -= ceb / 2394.0 + cpb / 252.0;
    const double n0b = -30.0 * neb + 12.0 * npb;
    const double nAb = -11.0 * neb - 4.0 * npb;
    const double nDb = 8.0 * neb + npb;
    h0x += n0b;
    geq0b -= n0b;
    Sab += nAb;
    Pb -= nAb;
    Sdb += nDb;
    Pb -= nDb;
    su2b -= 0.5 * nDb;
  }
  // geq0 = sigma - P3 - 0.5 su2 ; kg = P3 - 1.5 su2 ; P3 = 3 P ; su2 = sigma u2
  sigmab += geq0b;
  double P3b = -geq0b + kgb;
  su2b += -0.5 * geq0b - 1.5 * kgb;
  Pb += 3.0 * P3b;
  sigmab += F.u2 * su2b;
  const double u2b = F.sigma * su2b;
  // cu_p = c_p . u ; u2 = |u|^2
  double uxb = ((cub[0] + cub[3]) + (cub[4] + cub[5])) + cub[6];
  double uyb = ((cub[1] + cub[3]) - (cub[4] - cub[7])) + cub[8];
  double uzb = ((cub[2] + cub[5]) - (cub[6] - cub[7])) - cub[8];
  uxb += 2.0 * F.ux * u2b;
  uyb += 2.0 * F.uy * u2b;
  uzb += 2.0 * F.uz * u2b;
  recovery_moments_reverse(F, sigmab, Pb, uxb, uyb, uzb, 0.0, Sab, Sdb, h0x, hb);
}

// lambda_a at node (x, y, z) from the adjoint of the pull stream: the sum of mu_a over
// the nodes whose pull of link a lands on (x, y, z) (at most two per axis: the
// neighbour, and at a zero-gradient end the node itself).  Loads are unrolled and
// predicated; the order of the sum is fixed.
// The same on a quasi-1D lattice (ny = nz = 1), where every pull's y and z source and
// preimage is the node's own row: only the x preimages are summed, in the same order.
__device__ __forceinline__ double gather_link_tube(const double* __restrict__ mu_a, int x, int cx, const AGeo& geo) {
  int px[2];
  const int nxp = preimages(x, cx, geo.nx, geo.zgx, px);
  double acc = 0.0;
#pragma unroll
  for (int ix = 0; ix < 2; ++ix)
    if (ix < nxp) acc += mu_a[px[ix]];
  return acc;
}
template <bool TUBE>
__device__ __forceinline__ double gather_any(const double* __restrict__ mu_a, int x, int y, int z, int cx, int cy,
                                             int cz, const AGeo& geo);
__device__ __forceinline__ double gather_link(const double* __restrict__ mu_a, int x, int y, int z, int cx, int cy,
                                              int cz, const AGeo& geo) {
  int px[2], py[2], pz[2];
  const int nxp = preimages(x, cx, geo.nx, geo.zgx, px);
  const int nyp = preimages(y, cy, geo.ny, geo.zgy, py);
  const int nzp = preimages(z, cz, geo.nz, geo.zgz, pz);
  double acc = 0.0;
#pragma unroll
  for (int iz = 0; iz < 2; ++iz)
#pragma unroll
    for (int iy = 0; iy < 2; ++iy)
#pragma unroll
      for (int ix = 0; ix < 2; ++ix)
        if (iz < nzp && iy < nyp && ix < nxp)
          acc += mu_a[((unsigned long long)pz[iz] * geo.ny + py[iy]) * geo.nx + px[ix]];
  return acc;
}
template <bool TUBE>
__device__ __forceinline__ double gather_any(const double* __restrict__ mu_a, int x, int y, int z, int cx, int cy,
                                             int cz, const AGeo& geo) {
  if constexpr (TUBE) return gather_link_tube(mu_a, x, cx, geo);
  else return gather_link(mu_a, x, y, z, cx, cy, cz, geo);
}

// One reverse step at node (x, y, z) of a (ceil(nx / blockDim), ny, nz) grid: lambda^{t+1}
// at the node (read directly for the last step, FIRST, else gathered from the mu of the
// step after it), then mu = C_h^T lambda^{t+1} and the omega contributions.
// TUBE: ny = nz = 1 (only x-neighbours exchange populations).
template <bool MRT, bool FIRST, bool TUBE = false>
__global__ void __launch_bounds__(kThreads) k_adj_step(const double* __restrict__ g, const double* __restrict__ in,
                                                      double* __restrict__ mu, double* __restrict__ tb, AGeo geo,
                                                      StepConst k, int lanes) {
  // `lanes` nodes per block along x
  const int x = blockIdx.x * lanes + threadIdx.x;
  if ((int)threadIdx.x >= lanes || x >= geo.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const unsigned long long i = ((unsigned long long)z * geo.ny + y) * geo.nx + x;
  double h[19], lo[19], hb[19];
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    const int xs = pull_src(x, link_cx(a), geo.nx, geo.zgx);
    const int ys = TUBE ? 0 : pull_src(y, link_cy(a), geo.ny, geo.zgy);
    const int zs = TUBE ? 0 : pull_src(z, link_cz(a), geo.nz, geo.zgz);
    const unsigned long long s = ((unsigned long long)zs * geo.ny + ys) * geo.nx + xs;
    h[a] = g[(unsigned long long)a * geo.n + s];
    lo[a] = FIRST ? in[(unsigned long long)a * geo.n + i]
                  : gather_any<TUBE>(in + (unsigned long long)a * geo.n, x, y, z, link_cx(a), link_cy(a), link_cz(a),
                                     geo);
  }
  double wvb, web, wpb;
  g_collide_vjp<MRT>(h, lo, k, hb, wvb, web, wpb);
#pragma unroll
  for (int a = 0; a < 19; ++a) mu[(unsigned long long)a * geo.n + i] = hb[a];
  tb[i] += wvb;
  tb[geo.n + i] += web;
  tb[2 * geo.n + i] += wpb;
}

// ---- four threads per node (small lattices)
//
// On a lattice of a few thousand nodes one thread per node leaves each SM with a
// single warp whose reverse step is one long dependent chain.  The helpers below give
// each node four lanes of a warp: lane j takes link pairs j, j + 4 and j + 8 (the rest
// link is read by all four), the moments and the per-pair cotangents are summed over
// the four lanes with xor shuffles, and the short scalar chains (recovery forward and
// backward, MRT scalars) run in all four lanes.  The arithmetic is that of
// g_collide_vjp summed in another order.

// Direction of link pair p (link 2p + 1 moves along it, link 2p + 2 against it) for a
// pair index known only at run time, from bit masks over p: x is +1 for p in
// {0, 3, 4, 5, 6}; y is +1 for {1, 3, 7, 8} and -1 for 4; z is +1 for {2, 5, 7} and
// -1 for {6, 8}.
__device__ __forceinline__ void pair_dir(int p, int& cx, int& cy, int& cz) {
  cx = (0x079 >> p) & 1;
  cy = ((0x19a >> p) & 1) * (p == 4 ? -1 : 1);
  cz = ((0x1e4 >> p) & 1) * ((p == 6 || p == 8) ? -1 : 1);
}

// c * v for c in {-1, 0, 1}, without a multiply
__device__ __forceinline__ double sel(int c, double v) { return c == 0 ? 0.0 : (c > 0 ? v : -v); }

// sum over the four lanes of one node (lanes 4m .. 4m + 3), returned to all four
__device__ __forceinline__ double quad_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// The pulled g of lane j's three link pairs p = j, j + 4, j + 8 at node (x, y, z) (zeros
// for p > 8) and their directions.
template <bool TUBE>
__device__ __forceinline__ void quad_pull(const double* __restrict__ g, int x, int y, int z, int j, const AGeo& geo,
                                          double (&ha)[3], double (&hb)[3], int (&cd)[3][3]) {
  const unsigned long long n = geo.n;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int p = j + 4 * s;
    int cx = 0, cy = 0, cz = 0;
    if (p <= 8) pair_dir(p, cx, cy, cz);
    cd[s][0] = cx;
    cd[s][1] = cy;
    cd[s][2] = cz;
    ha[s] = hb[s] = 0.0;
    if (p <= 8) {
      const unsigned long long a1 = 2 * p + 1, a2 = 2 * p + 2;
      const unsigned long long s1 =
          TUBE ? (unsigned long long)pull_src(x, cx, geo.nx, geo.zgx)
               : ((unsigned long long)pull_src(z, cz, geo.nz, geo.zgz) * geo.ny + pull_src(y, cy, geo.ny, geo.zgy)) *
                         geo.nx + pull_src(x, cx, geo.nx, geo.zgx);
      const unsigned long long s2 =
          TUBE ? (unsigned long long)pull_src(x, -cx, geo.nx, geo.zgx)
               : ((unsigned long long)pull_src(z, -cz, geo.nz, geo.zgz) * geo.ny + pull_src(y, -cy, geo.ny, geo.zgy)) *
                         geo.nx + pull_src(x, -cx, geo.nx, geo.zgx);
      ha[s] = g[a1 * n + s1];
      hb[s] = g[a2 * n + s2];
    }
  }
}

// lambda of lane j's pairs at the node: read directly (FIRST, the last step) or
// gathered from the mu of the step after it.
template <bool FIRST, bool TUBE>
__device__ __forceinline__ void quad_lambda(const double* __restrict__ in, int x, int y, int z, int j,
                                            unsigned long long i, const AGeo& geo, const int (&cd)[3][3],
                                            double (&la)[3], double (&lb)[3]) {
  const unsigned long long n = geo.n;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int p = j + 4 * s;
    la[s] = lb[s] = 0.0;
    if (p <= 8) {
      const unsigned long long a1 = 2 * p + 1, a2 = 2 * p + 2;
      const int cx = cd[s][0], cy = cd[s][1], cz = cd[s][2];
      la[s] = FIRST ? in[a1 * n + i] : gather_any<TUBE>(in + a1 * n, x, y, z, cx, cy, cz, geo);
      lb[s] = FIRST ? in[a2 * n + i] : gather_any<TUBE>(in + a2 * n, x, y, z, -cx, -cy, -cz, geo);
    }
  }
}

// The forward intermediates of the g collide that a node's reverse step uses; none of
// them depends on lambda.  Per node: u, sigma, 1/sigma and its square, u^2, kg, g^eq_0
// minus the rest population, the MRT scalars scaled by the row norms (ne / 2394,
// np / 252), M, 1 / (6 sqrt(A)), 8 T00, 2 sigma and the odd weights 3 omega w sigma of
// the axis and diagonal classes (the pulled state, Eq. 10 and the recovery).  Per link
// pair p, with c = c_p . u and the class weight w: 4.5 w c^2, 3 w c and 2 (4.5 omega w
// sigma) c, the products that multiply the pair's cotangents.
struct QFwd {
  double ux, uy, uz, sigma, is, is2, u2, kg, dg0, ne, np, Mx, My, Mz, rsA6, T8, s2, AA, AD;
};
constexpr int kFwdFields = 19;
constexpr int kPairFields = 3;   // per link pair, stored at (3 p + f) n + i

// QFwd and the pair products of lane j's pairs from the rest link h0 and lane j's
// pulled pairs: moments summed over the node's four lanes, then the scalar chain in
// every lane.
template <bool MRT>
__device__ __forceinline__ void quad_forward(double h0, const double (&ha)[3], const double (&hb)[3],
                                             const int (&cd)[3][3], int j, const StepConst& k, QFwd& F,
                                             double (&pc)[3][kPairFields]) {
  double Sa = 0, Sd = 0, Mx = 0, My = 0, Mz = 0;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int p = j + 4 * s;
    const double sp = ha[s] + hb[s], dp = ha[s] - hb[s];
    if (p < 3) Sa += sp;
    else Sd += sp;   // zero for p > 8
    Mx += sel(cd[s][0], dp);
    My += sel(cd[s][1], dp);
    Mz += sel(cd[s][2], dp);
  }
  Sa = quad_sum(Sa);
  Sd = quad_sum(Sd);
  Mx = quad_sum(Mx);
  My = quad_sum(My);
  Mz = quad_sum(Mz);
  const double T00 = (h0 + Sa) + Sd;
  const double MM = fma(Mx, Mx, fma(My, My, Mz * Mz));
  const double A = fma(4.0 * T00, T00, -3.0 * MM);
  const double sA = sqrt_seeded(A);
  const double sigma = fma(2.0, T00, sA) * (1.0 / 3.0);
  const double is = rcp_seeded(sigma);
  const double ux = Mx * is, uy = My * is, uz = Mz * is;
  const double P = sigma - T00;
  const double u2 = fma(ux, ux, fma(uy, uy, uz * uz));
  const double su2 = sigma * u2, P3 = 3.0 * P;
  const double geq0 = fma(-0.5, su2, sigma - P3);
  F.kg = fma(-1.5, su2, P3);
  F.dg0 = geq0 - h0;
  F.ne = F.np = 0.0;
  if (MRT) {
    const double n0 = h0 - geq0, nA = Sa - P, nD = fma(-0.5, su2, Sd - P);
    F.ne = fma(8.0, nD, fma(-11.0, nA, -30.0 * n0)) * (1.0 / 2394.0);
    F.np = fma(-4.0, nA, fma(12.0, n0, nD)) * (1.0 / 252.0);
  }
  F.ux = ux;
  F.uy = uy;
  F.uz = uz;
  F.sigma = sigma;
  F.is = is;
  F.is2 = is * is;
  F.u2 = u2;
  F.Mx = Mx;
  F.My = My;
  F.Mz = Mz;
  F.rsA6 = rcp_seeded(sA) * (1.0 / 6.0);
  F.T8 = 8.0 * T00;
  F.s2 = 2.0 * sigma;
  F.AA = k.gA_a * sigma;
  F.AD = k.gD_a * sigma;
  const double SA2 = 2.0 * k.gA_s * sigma, SD2 = 2.0 * k.gD_s * sigma;
  const double wA = 1.0 / 18.0, wD = 1.0 / 36.0;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const bool ax = j + 4 * s < 3;
    const double c = (sel(cd[s][0], ux) + sel(cd[s][1], uy)) + sel(cd[s][2], uz);
    const double w = ax ? wA : wD;
    pc[s][0] = (4.5 * w * c) * c;
    pc[s][1] = (3.0 * w) * c;
    pc[s][2] = (ax ? SA2 : SD2) * c;
  }
}

// Stored QFwd of node i (field q at q * n + i) and the pair products (pair p, field f
// at (kFwdFields + 3 p + f) * n + i).
__device__ __forceinline__ void store_fwd(double* __restrict__ fw, unsigned long long i, unsigned long long n,
                                          const QFwd& F, bool node_fields, int j, const double (&pc)[3][kPairFields]) {
  if (node_fields) {
    const double v[kFwdFields] = {F.ux, F.uy, F.uz, F.sigma, F.is, F.is2, F.u2, F.kg, F.dg0, F.ne,
                                  F.np, F.Mx, F.My, F.Mz, F.rsA6, F.T8, F.s2, F.AA, F.AD};
#pragma unroll
    for (int q = 0; q < kFwdFields; ++q) fw[q * n + i] = v[q];
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int p = j + 4 * s;
    if (p > 8) continue;
#pragma unroll
    for (int f = 0; f < kPairFields; ++f) fw[(kFwdFields + kPairFields * p + f) * n + i] = pc[s][f];
  }
}
__device__ __forceinline__ void load_fwd(const double* __restrict__ fw, unsigned long long i, unsigned long long n,
                                         int j, QFwd& F, double (&pc)[3][kPairFields]) {
  double v[kFwdFields];
#pragma unroll
  for (int q = 0; q < kFwdFields; ++q) v[q] = fw[q * n + i];
  F.ux = v[0]; F.uy = v[1]; F.uz = v[2]; F.sigma = v[3]; F.is = v[4]; F.is2 = v[5]; F.u2 = v[6]; F.kg = v[7];
  F.dg0 = v[8]; F.ne = v[9]; F.np = v[10]; F.Mx = v[11]; F.My = v[12]; F.Mz = v[13]; F.rsA6 = v[14]; F.T8 = v[15];
  F.s2 = v[16]; F.AA = v[17]; F.AD = v[18];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int p = j + 4 * s;
#pragma unroll
    for (int f = 0; f < kPairFields; ++f) pc[s][f] = p <= 8 ? fw[(kFwdFields + kPairFields * p + f) * n + i] : 0.0;
  }
}

// The reverse of the collide at one node in lane j: per-pair cotangents, sums over the
// node's four lanes, the scalar chain backwards (MRT scalars, equilibria, recovery,
// moments), then the stores of mu for lane j's pairs and, in lane 0, the rest link and
// the omega contributions.  An FP64 instruction holds its sub-partition's FP64 unit for
// about 64 cycles whatever its active lanes, so the chain is written for few of them:
// the forward-only products come stored, the four class sums of the shear/bulk term are
// combined before the lane sums, and the relaxations fold into fused multiply-adds.
template <bool MRT>
__device__ __forceinline__ void quad_backward(const QFwd& F, const double (&pc)[3][kPairFields], double l0,
                                              const double (&ha)[3], const double (&hb)[3], const double (&la)[3],
                                              const double (&lb)[3], const int (&cd)[3][3], int j, bool valid,
                                              unsigned long long i, const StepConst& k, double* __restrict__ mu,
                                              double* __restrict__ tb, unsigned long long n) {
  const double om = k.omv, om1 = k.omv1;
  const double wA = 1.0 / 18.0, wD = 1.0 / 36.0;
  double sw = 0, KAb = 0, KDb = 0, wvb = 0, uxb = 0, uyb = 0, uzb = 0;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const bool ax = j + 4 * s < 3;   // only slot 0 holds axis pairs; pairs past 8 are zero
    wvb = fma(-ha[s], la[s], fma(-hb[s], lb[s], wvb));
    const double evb = la[s] + lb[s], odb = la[s] - lb[s];
    sw = fma(evb, pc[s][0], fma(odb, pc[s][1], sw));
    if (s == 0) {
      KAb += ax ? evb : 0.0;
      KDb += ax ? 0.0 : evb;
    } else {
      KDb += evb;
    }
    const double cub = fma(evb, pc[s][2], odb * (ax ? F.AA : F.AD));
    uxb += sel(cd[s][0], cub);
    uyb += sel(cd[s][1], cub);
    uzb += sel(cd[s][2], cub);
  }
  sw = quad_sum(sw);
  KAb = quad_sum(KAb);
  KDb = quad_sum(KDb);
  wvb = quad_sum(wvb);
  uxb = quad_sum(uxb);
  uyb = quad_sum(uyb);
  uzb = quad_sum(uzb);
  // rest link: out0 = (1 - om) h0 + om geq0 (+ 30 ae - 12 ap)
  wvb = fma(F.dg0, l0, wvb);
  double geq0b = om * l0;
  const double aeb = fma(11.0, KAb, fma(-8.0, KDb, 30.0 * l0));
  const double apb = fma(-12.0, l0, fma(4.0, KAb, -KDb));
  const double t = fma(wA, KAb, wD * KDb);
  const double kgb = om * t;
  wvb = fma(F.kg, t, wvb);
  double sigmab = om * sw;
  wvb = fma(F.sigma, sw, wvb);
  double Sab = 0, Sdb = 0, Pb = 0, su2b = 0, h0x = 0, web = 0, wpb = 0;
  if (MRT) {
    const double neb = k.ce * aeb, npb = k.cp * apb;
    web = F.ne * aeb;
    wpb = F.np * apb;
    wvb = (wvb - web) - wpb;
    const double n0b = fma(-30.0, neb, 12.0 * npb);
    const double nAb = fma(-11.0, neb, -4.0 * npb);
    const double nDb = fma(8.0, neb, npb);
    h0x = n0b;
    geq0b -= n0b;
    Sab = nAb;
    Sdb = nDb;
    Pb = -nAb - nDb;
    su2b = -0.5 * nDb;
  }
  // geq0 = sigma - P3 - 0.5 su2 ; kg = P3 - 1.5 su2 ; P3 = 3 P ; su2 = sigma u2
  sigmab += geq0b;
  su2b = fma(-0.5, geq0b, fma(-1.5, kgb, su2b));
  Pb = fma(3.0, kgb - geq0b, Pb);
  sigmab = fma(F.u2, su2b, sigmab);
  const double u2b2 = F.s2 * su2b;   // 2 d/du2
  uxb = fma(F.ux, u2b2, uxb);
  uyb = fma(F.uy, u2b2, uyb);
  uzb = fma(F.uz, u2b2, uzb);
  // P = sigma - T00 ; u = M / sigma ; sigma = (2 T00 + sqrt(A)) / 3 ; A = 4 T00^2 - 3 |M|^2
  sigmab += Pb;
  double T00b = -Pb;
  double Mxb = F.is * uxb, Myb = F.is * uyb, Mzb = F.is * uzb;
  sigmab = fma(-F.is2, fma(F.Mx, uxb, fma(F.My, uyb, F.Mz * uzb)), sigmab);
  T00b = fma(2.0 / 3.0, sigmab, T00b);
  const double Ab = sigmab * F.rsA6;
  T00b = fma(F.T8, Ab, T00b);
  const double MMb = -6.0 * Ab;
  Mxb = fma(F.Mx, MMb, Mxb);
  Myb = fma(F.My, MMb, Myb);
  Mzb = fma(F.Mz, MMb, Mzb);
  // T00 = h0 + Sa + Sd
  Sab += T00b;
  Sdb += T00b;
  if (!valid) return;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int p = j + 4 * s;
    if (p > 8) continue;
    const double spb = p < 3 ? Sab : Sdb;
    const double dpb = (sel(cd[s][0], Mxb) + sel(cd[s][1], Myb)) + sel(cd[s][2], Mzb);
    mu[(unsigned long long)(2 * p + 1) * n + i] = fma(om1, la[s], spb + dpb);
    mu[(unsigned long long)(2 * p + 2) * n + i] = fma(om1, lb[s], spb - dpb);
  }
  if (j == 0) {
    mu[i] = fma(om1, l0, T00b + h0x);
    tb[i] += wvb;
    tb[n + i] += web;
    tb[2 * n + i] += wpb;
  }
}

// ---- two warp roles (small lattices, the reverse sweep's chain)
//
// Nothing in QFwd or the pair products depends on lambda, only on the forward state,
// so the reverse step need not compute them on its own dependent chain.  k_adj_step_ws
// runs 8 nodes per 64-thread block: warp 0 walks the backward chain of step t from the
// values stored for step t (fw), and warp 1 computes and stores those of step t - 1
// (from g_prev, the state at step t - 1, into fw_prev) for the next launch.  The two
// warps run on different sub-partitions, so each has its own FP64 unit.  k_adj_fwd
// stores the values of one step on its own (the last step, where the sweep starts).
template <bool MRT, bool TUBE>
__global__ void __launch_bounds__(64) k_adj_fwd(const double* __restrict__ g, double* __restrict__ fw, AGeo geo,
                                                StepConst k) {
  const int j = threadIdx.x & 3;
  const int xg = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 2);
  const bool valid = xg < geo.nx;
  const int x = valid ? xg : geo.nx - 1;
  const int y = blockIdx.y, z = blockIdx.z;
  const unsigned long long i = ((unsigned long long)z * geo.ny + y) * geo.nx + x;
  double ha[3], hb[3], pc[3][kPairFields];
  int cd[3][3];
  const double h0 = g[i];
  quad_pull<TUBE>(g, x, y, z, j, geo, ha, hb, cd);
  QFwd F;
  quad_forward<MRT>(h0, ha, hb, cd, j, k, F, pc);
  if (valid) store_fwd(fw, i, geo.n, F, j == 0, j, pc);
}

template <bool MRT, bool FIRST, bool TUBE>
__global__ void __launch_bounds__(64) k_adj_step_ws(const double* __restrict__ g, const double* __restrict__ in,
                                                    double* __restrict__ mu, double* __restrict__ tb,
                                                    const double* __restrict__ fw, const double* __restrict__ g_prev,
                                                    double* __restrict__ fw_prev, AGeo geo, StepConst k) {
  const int lane = threadIdx.x & 31, j = lane & 3;
  const int xg = (int)(blockIdx.x * 8 + (lane >> 2));
  const bool valid = xg < geo.nx;
  const int x = valid ? xg : geo.nx - 1;
  const int y = blockIdx.y, z = blockIdx.z;
  const unsigned long long i = ((unsigned long long)z * geo.ny + y) * geo.nx + x;
  double ha[3], hb[3], pc[3][kPairFields];
  int cd[3][3];
  QFwd F;
  if (threadIdx.x >= 32) {
    // step t - 1's forward values (none before step 0)
    if (g_prev == nullptr) return;
    const double h0 = g_prev[i];
    quad_pull<TUBE>(g_prev, x, y, z, j, geo, ha, hb, cd);
    quad_forward<MRT>(h0, ha, hb, cd, j, k, F, pc);
    if (valid) store_fwd(fw_prev, i, geo.n, F, j == 0, j, pc);
    return;
  }
  const double l0 = in[i];
  double la[3], lb[3];
  quad_pull<TUBE>(g, x, y, z, j, geo, ha, hb, cd);
  quad_lambda<FIRST, TUBE>(in, x, y, z, j, i, geo, cd, la, lb);
  load_fwd(fw, i, geo.n, j, F, pc);
  quad_backward<MRT>(F, pc, l0, ha, hb, la, lb, cd, j, valid, i, k, mu, tb, geo.n);
}

// lambda^T = dJ/dg^T and the per-node misfit.
__global__ void __launch_bounds__(kThreads) k_adj_loss(const double* __restrict__ g, const double* __restrict__ tP,
                                                      const double* __restrict__ tux, const double* __restrict__ tuy,
                                                      const double* __restrict__ tuz, double wP, double wu,
                                                      double* __restrict__ lam, double* __restrict__ lossn,
                                                      unsigned long long n) {
  const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double h[19], hb[19];
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    h[a] = g[(unsigned long long)a * n + i];
    hb[a] = 0.0;
  }
  GFwd F;
  StepConst dummy{};
  gforward(h, dummy, false, F);
  const double rP = F.P - tP[i], rx = F.ux - tux[i], ry = F.uy - tuy[i], rz = F.uz - tuz[i];
  lossn[i] = wP * rP * rP + wu * (rx * rx + ry * ry + rz * rz);
  recovery_moments_reverse(F, 0.0, 2.0 * wP * rP, 2.0 * wu * rx, 2.0 * wu * ry, 2.0 * wu * rz, 0.0, 0.0, 0.0, 0.0,
                           hb);
#pragma unroll
  for (int a = 0; a < 19; ++a) lam[(unsigned long long)a * n + i] = hb[a];
}

// dJ/de0 of an equilibrium initial state: g^0 is linear in e0, so sum_a lambda_a g0_a / e0.
// dJ/de0 at node (x, y, z): lambda^0 = S^T mu^0 gathered at the node, contracted with
// dg^eq/de of the initial state (g^eq is homogeneous of degree 1 in e at fixed u).
__global__ void __launch_bounds__(kThreads) k_adj_e0(const double* __restrict__ g0, const double* __restrict__ mu,
                                                    double* __restrict__ de0, AGeo geo, int lanes) {
  const int x = blockIdx.x * lanes + threadIdx.x;
  if ((int)threadIdx.x >= lanes || x >= geo.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const unsigned long long i = ((unsigned long long)z * geo.ny + y) * geo.nx + x;
  double h[19];
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    h[a] = g0[(unsigned long long)a * geo.n + i];
    const double l = gather_link(mu + (unsigned long long)a * geo.n, x, y, z, link_cx(a), link_cy(a), link_cz(a), geo);
    acc = fma(l, h[a], acc);
  }
  GFwd F;
  StepConst dummy{};
  gforward(h, dummy, false, F);
  de0[i] = acc / (3.0 * F.P);
}

// Deterministic sums of `rows` arrays of length n (one block per row).
__global__ void __launch_bounds__(256) k_rowsum(const double* __restrict__ a, unsigned long long n,
                                                double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  const double* r = a + blockIdx.x * n;
  for (unsigned long long i = threadIdx.x; i < n; i += 256) acc += r[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

int afail(rlb_handle* h, int code, const std::string& m) {
  h->err = m;
  return code;
}

// Buffers and the captured CUDA graph of one (nsteps, checkpoint interval) shape,
// kept on the handle so repeated gradients replay instead of re-launching ~4 T
// kernels one by one.
struct AdjPlan {
  int nsteps = -1, K = 0, nseg = 0, start_cur = 0, threads = 128, lanes = 128;
  bool quad = false;                          // reverse steps with four threads per node
  double wP = 0.0, wu = 0.0;                  // misfit weights baked into the graph
  std::vector<void*> ckpt, seg, segb, owned;     // seg / segb: the recomputed states of alternate segments
  double *lam = nullptr, *mu = nullptr, *tb = nullptr, *lossn = nullptr, *sums = nullptr, *dde0 = nullptr;
  double* fw[2] = {nullptr, nullptr};         // QFwd of alternate reverse steps (two warp roles)
  double* tgt = nullptr;
  void* g0copy = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t cap2 = nullptr;                // recompute of segment s - 1 beside the reverse sweep of s
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // fork, ready[2], free[2]
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

void free_plan(void* p) {
  AdjPlan* a = (AdjPlan*)p;
  if (!a) return;
  if (a->exec) cudaGraphExecDestroy(a->exec);
  if (a->graph) cudaGraphDestroy(a->graph);
  if (a->cap) cudaStreamDestroy(a->cap);
  if (a->cap2) cudaStreamDestroy(a->cap2);
  for (cudaEvent_t e : a->ev)
    if (e) cudaEventDestroy(e);
  for (void* q : a->owned) cudaFree(q);
  delete a;
}

bool plan_alloc(AdjPlan* a, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  a->owned.push_back(*p);
  return true;
}

// One reverse step with the kernel variant for the lattice: two warp roles with four
// threads per node (quad; fw holds step t's QFwd, and step t - 1's goes from g_prev
// into fw_prev) or one thread per node; quasi-1D (ny = nz = 1) or general; BGK or MRT.
template <bool FIRST>
cudaError_t reverse_step(bool quad, bool tube, bool mrt, dim3 grid8, dim3 grid3, int th, cudaStream_t st,
                         const double* gt, const double* in, double* out, double* tb, const double* fw,
                         const double* g_prev, double* fw_prev, const AGeo& geo, const StepConst& k, int lanes) {
  if (quad) {
    if (tube) {
      if (mrt) k_adj_step_ws<true, FIRST, true><<<grid8, 64, 0, st>>>(gt, in, out, tb, fw, g_prev, fw_prev, geo, k);
      else k_adj_step_ws<false, FIRST, true><<<grid8, 64, 0, st>>>(gt, in, out, tb, fw, g_prev, fw_prev, geo, k);
    } else {
      if (mrt) k_adj_step_ws<true, FIRST, false><<<grid8, 64, 0, st>>>(gt, in, out, tb, fw, g_prev, fw_prev, geo, k);
      else k_adj_step_ws<false, FIRST, false><<<grid8, 64, 0, st>>>(gt, in, out, tb, fw, g_prev, fw_prev, geo, k);
    }
  } else if (tube) {
    if (mrt) k_adj_step<true, FIRST, true><<<grid3, th, 0, st>>>(gt, in, out, tb, geo, k, lanes);
    else k_adj_step<false, FIRST, true><<<grid3, th, 0, st>>>(gt, in, out, tb, geo, k, lanes);
  } else {
    if (mrt) k_adj_step<true, FIRST><<<grid3, th, 0, st>>>(gt, in, out, tb, geo, k, lanes);
    else k_adj_step<false, FIRST><<<grid3, th, 0, st>>>(gt, in, out, tb, geo, k, lanes);
  }
  return cudaGetLastError();
}

// Enqueue the whole gradient computation on stream st (captured into the plan's graph).
cudaError_t enqueue_adjoint(rlb_handle* h, AdjPlan* a, double wP, double wu, bool mrt) {
  const unsigned long long N = h->nodes;
  const size_t state_bytes = 38 * N * sizeof(double);
  const int T = a->nsteps, K = a->K, th = a->threads;
  const unsigned grid = (unsigned)((N + th - 1) / th);
  const int lanes = a->lanes;
  const dim3 grid3((unsigned)((h->cfg.nx + lanes - 1) / lanes), (unsigned)h->cfg.ny, (unsigned)h->cfg.nz);
  const dim3 grid8((unsigned)((h->cfg.nx + 7) / 8), (unsigned)h->cfg.ny, (unsigned)h->cfg.nz);
  double* mu_cur = nullptr;   // buffer holding the mu of the latest reverse step (lam / mu alternate)
  cudaStream_t st = a->cap;
  AGeo geo{h->cfg.nx, h->cfg.ny, h->cfg.nz, h->cfg.bc[0] == RLB_ZERO_GRADIENT, h->cfg.bc[1] == RLB_ZERO_GRADIENT,
           h->cfg.bc[2] == RLB_ZERO_GRADIENT, N};
  const bool tube = h->cfg.ny == 1 && h->cfg.nz == 1;
  const double* tP = a->tgt;
  cudaError_t e;
#define ENQ(call) do { e = (call); if (e != cudaSuccess) return e; } while (0)
  // forward with checkpoints
  ENQ(cudaMemcpyAsync(a->g0copy, h->lat[h->cur], state_bytes, cudaMemcpyDeviceToDevice, st));
  for (int t = 0; t < T; ++t) {
    if (t % K == 0) ENQ(cudaMemcpyAsync(a->ckpt[t / K], h->lat[h->cur], state_bytes, cudaMemcpyDeviceToDevice, st));
    ENQ(enqueue_steps(h, 1, st));
  }
  // misfit and lambda^T
  const double* gT = (const double*)h->lat[h->cur] + 19 * N;
  k_adj_loss<<<grid, th, 0, st>>>(gT, tP, tP + N, tP + 2 * N, tP + 3 * N, wP, wu, a->lam, a->lossn, N);
  ENQ(cudaGetLastError());
  ENQ(cudaMemsetAsync(a->tb, 0, 3 * N * sizeof(double), st));
  // reverse sweep, segment by segment.  Each segment is recomputed from its checkpoint
  // on the second stream into one of two state buffers (segment s into buffer s & 1),
  // so the recompute of segment s - 1 runs beside the reverse sweep of segment s; a
  // buffer is refilled only after the reverse sweep that read it.
  cudaStream_t cs = a->cap2;
  cudaEvent_t ev_fork = a->ev[0], ev_ready[2] = {a->ev[1], a->ev[2]}, ev_free[2] = {a->ev[3], a->ev[4]};
  ENQ(cudaEventRecord(ev_fork, st));
  ENQ(cudaStreamWaitEvent(cs, ev_fork, 0));
  void* saved[2] = {h->lat[0], h->lat[1]};
  const int saved_cur = h->cur;
  const std::vector<void*>* buf[2] = {&a->seg, &a->segb};
  auto recompute = [&](int s) -> cudaError_t {
    const std::vector<void*>& b = *buf[s & 1];
    const int t0 = s * K, t1 = std::min(T, t0 + K);
    cudaError_t r = cudaMemcpyAsync(b[0], a->ckpt[s], state_bytes, cudaMemcpyDeviceToDevice, cs);
    for (int j = 0; r == cudaSuccess && j + 1 < t1 - t0; ++j) {   // b[j] holds g^{t0 + j}
      h->lat[0] = b[j];
      h->lat[1] = b[j + 1];
      h->cur = 0;
      r = enqueue_steps(h, 1, cs);
    }
    h->lat[0] = saved[0];
    h->lat[1] = saved[1];
    h->cur = saved_cur;
    if (r == cudaSuccess) r = cudaEventRecord(ev_ready[s & 1], cs);
    return r;
  };
  ENQ(recompute(a->nseg - 1));
  for (int s = a->nseg - 1; s >= 0; --s) {
    if (s >= 1) {
      if (s + 1 <= a->nseg - 1) ENQ(cudaStreamWaitEvent(cs, ev_free[(s + 1) & 1], 0));
      ENQ(recompute(s - 1));
    }
    ENQ(cudaStreamWaitEvent(st, ev_ready[s & 1], 0));
    const std::vector<void*>& b = *buf[s & 1];
    const int t0 = s * K, t1 = std::min(T, t0 + K);
    if (a->quad && t1 == T) {   // the QFwd of the last step
      if (tube) {
        if (mrt) k_adj_fwd<true, true><<<grid8, 64, 0, st>>>((const double*)b[T - 1 - t0] + 19 * N, a->fw[(T - 1) & 1], geo, h->k);
        else k_adj_fwd<false, true><<<grid8, 64, 0, st>>>((const double*)b[T - 1 - t0] + 19 * N, a->fw[(T - 1) & 1], geo, h->k);
      } else {
        if (mrt) k_adj_fwd<true, false><<<grid8, 64, 0, st>>>((const double*)b[T - 1 - t0] + 19 * N, a->fw[(T - 1) & 1], geo, h->k);
        else k_adj_fwd<false, false><<<grid8, 64, 0, st>>>((const double*)b[T - 1 - t0] + 19 * N, a->fw[(T - 1) & 1], geo, h->k);
      }
      ENQ(cudaGetLastError());
    }
    for (int t = t1 - 1; t >= t0; --t) {
      const double* gt = (const double*)b[t - t0] + 19 * N;
      // the state at step t - 1: in this segment, else the top of the one below, whose
      // recompute must have finished
      const double* g_prev = nullptr;
      if (t > t0) {
        g_prev = (const double*)b[t - 1 - t0] + 19 * N;
      } else if (s >= 1) {
        ENQ(cudaStreamWaitEvent(st, ev_ready[(s - 1) & 1], 0));
        g_prev = (const double*)(*buf[(s - 1) & 1])[K - 1] + 19 * N;
      }
      const double* fw = a->fw[t & 1];
      double* fw_prev = a->fw[(t + 1) & 1];
      // the last step reads lambda^T; later ones gather from the mu of the step after
      double* out = mu_cur == a->mu ? a->lam : a->mu;
      if (t == T - 1) {
        out = a->mu;
        ENQ(reverse_step<true>(a->quad, tube, mrt, grid8, grid3, th, st, gt, a->lam, out, a->tb, fw, g_prev, fw_prev,
                               geo, h->k, lanes));
      } else {
        ENQ(reverse_step<false>(a->quad, tube, mrt, grid8, grid3, th, st, gt, mu_cur, out, a->tb, fw, g_prev, fw_prev,
                                geo, h->k, lanes));
      }
      mu_cur = out;
    }
    ENQ(cudaEventRecord(ev_free[s & 1], st));
  }
  // join the second stream back into the capture
  ENQ(cudaEventRecord(ev_fork, cs));
  ENQ(cudaStreamWaitEvent(st, ev_fork, 0));
  ENQ(cudaGetLastError());
  k_adj_e0<<<grid3, th, 0, st>>>((const double*)a->g0copy + 19 * N, mu_cur, a->dde0, geo, lanes);
  k_rowsum<<<3, 256, 0, st>>>(a->tb, N, a->sums);
  k_rowsum<<<1, 256, 0, st>>>(a->lossn, N, a->sums + 3);
  ENQ(cudaGetLastError());
#undef ENQ
  return cudaSuccess;
}

}  // namespace

extern "C" int rlb_adjoint(rlb_handle* h, int nsteps, int checkpoint_every, const double* target_P,
                           const double* target_ux, const double* target_uy, const double* target_uz, double w_P,
                           double w_u, int where, double* loss, double* dtau, double* de0) {
  if (!h) return RLB_EINVAL;
  if (nsteps < 1) return afail(h, RLB_EINVAL, "nsteps must be >= 1");
  if (!target_P || !target_ux || !target_uy || !target_uz || !loss || !dtau)
    return afail(h, RLB_EINVAL, "null argument");
  if (where != RLB_HOST && where != RLB_DEVICE) return afail(h, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  if (h->esize != 8) return afail(h, RLB_EINVAL, "rlb_adjoint needs an RLB_FP64 lattice");
  if (h->Q != 19) return afail(h, RLB_EINVAL, "rlb_adjoint supports RLB_D3Q19 lattices");
  if (h->cfg.eta_over_s > 0) return afail(h, RLB_EINVAL, "rlb_adjoint needs constant relaxation times");
  if (h->cfg.collision == RLB_MRT && h->cfg.tau_q > 0 && h->cfg.tau_q != h->cfg.tau_v)
    return afail(h, RLB_EINVAL, "rlb_adjoint needs tau_q tied to tau_v (tau_q <= 0)");
  const bool mrt = h->cfg.collision == RLB_MRT;
  const unsigned long long N = h->nodes;
  const size_t state_bytes = 38 * N * sizeof(double), gbytes = 19 * N * sizeof(double);
  const int K = checkpoint_every > 0 ? checkpoint_every : std::max(1, (int)std::ceil(std::sqrt((double)nsteps)));
  cudaStream_t st = h->stream;

#define ACUDA(call)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return afail(h, RLB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

  // ---- plan (buffers + graph) for this shape
  AdjPlan* a = (AdjPlan*)h->adj_plan;
  if (a && (a->nsteps != nsteps || a->K != std::min(K, nsteps))) {
    ACUDA(cudaStreamSynchronize(st));
    free_plan(a);
    h->adj_plan = nullptr;
    a = nullptr;
  }
  if (!a) {
    a = new AdjPlan();
    a->nsteps = nsteps;
    a->K = std::min(K, nsteps);
    a->nseg = (nsteps + a->K - 1) / a->K;
    a->threads = N <= 152ull * 128ull * 2ull ? 32 : 128;
    // one node per thread (blocks with fewer active lanes, spreading a small lattice
    // over more SMs, measured slower on GB300)
    a->lanes = a->threads;
    // below ~2 warps per SM the one-thread-per-node step is one thread's dependent
    // chain; four threads per node shorten it (the scalar chain is repeated, so on
    // larger lattices, where the FP64 pipe is the limit, one thread per node is kept).
    // 1600-node tube, 4000 steps: 109 -> 87 ms per gradient on GB300.
    a->quad = a->threads == 32;
    a->ckpt.assign(a->nseg, nullptr);
    a->seg.assign(a->K + 1, nullptr);
    a->segb.assign(a->K + 1, nullptr);
    bool ok = true;
    for (int s = 0; s < a->nseg && ok; ++s) ok = plan_alloc(a, &a->ckpt[s], state_bytes);
    for (int j = 0; j <= a->K && ok; ++j) ok = plan_alloc(a, &a->seg[j], state_bytes);
    for (int j = 0; j <= a->K && ok; ++j) ok = plan_alloc(a, &a->segb[j], state_bytes);
    for (int i = 0; i < 5 && ok; ++i) ok = cudaEventCreateWithFlags(&a->ev[i], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&a->cap2, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && plan_alloc(a, (void**)&a->lam, gbytes) && plan_alloc(a, (void**)&a->mu, gbytes) &&
         plan_alloc(a, (void**)&a->tb, 3 * N * sizeof(double)) && plan_alloc(a, (void**)&a->lossn, N * sizeof(double)) &&
         plan_alloc(a, (void**)&a->sums, 8 * sizeof(double)) && plan_alloc(a, (void**)&a->dde0, N * sizeof(double)) &&
         plan_alloc(a, (void**)&a->tgt, 4 * N * sizeof(double)) && plan_alloc(a, &a->g0copy, state_bytes);
    for (int i = 0; i < 2 && ok && a->quad; ++i)
      ok = plan_alloc(a, (void**)&a->fw[i], (kFwdFields + 9 * kPairFields) * N * sizeof(double));
    if (!ok || cudaStreamCreateWithFlags(&a->cap, cudaStreamNonBlocking) != cudaSuccess) {
      free_plan(a);
      return afail(h, RLB_ENOMEM, "cannot allocate adjoint checkpoints and buffers");
    }
    a->start_cur = h->cur;
    h->adj_plan = a;
    h->adj_free = free_plan;
  }
  // the graph's lattice pointers assume the state starts in lat[start_cur]
  if (h->cur != a->start_cur) {
    ACUDA(cudaMemcpyAsync(h->lat[a->start_cur], h->lat[h->cur], state_bytes, cudaMemcpyDeviceToDevice, st));
    h->cur = a->start_cur;
  }
  // targets into the plan's buffer (outside the graph)
  {
    const double* src[4] = {target_P, target_ux, target_uy, target_uz};
    for (int c = 0; c < 4; ++c)
      ACUDA(cudaMemcpyAsync(a->tgt + c * N, src[c], N * sizeof(double),
                            where == RLB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  }
  // capture once per plan (the misfit weights are kernel arguments: recapture if they change)
  if (!a->exec || a->wP != w_P || a->wu != w_u) {
    if (a->exec) { cudaGraphExecDestroy(a->exec); a->exec = nullptr; }
    if (a->graph) { cudaGraphDestroy(a->graph); a->graph = nullptr; }
    const long long steps0 = h->steps;
    ACUDA(cudaStreamBeginCapture(a->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = enqueue_adjoint(h, a, w_P, w_u, mrt);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(a->cap, &g);
    h->cur = a->start_cur;   // nothing ran yet
    h->steps = steps0;
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return afail(h, RLB_ECUDA, std::string("adjoint graph capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    a->graph = g;
    ACUDA(cudaGraphInstantiate(&a->exec, a->graph, 0));
    a->wP = w_P;
    a->wu = w_u;
  }
  ACUDA(cudaGraphLaunch(a->exec, st));
  double hs[4];
  ACUDA(cudaMemcpyAsync(hs, a->sums, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (de0)
    ACUDA(cudaMemcpyAsync(de0, a->dde0, N * sizeof(double),
                          where == RLB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
  ACUDA(cudaStreamSynchronize(st));
  h->cur = a->start_cur ^ (nsteps & 1);
  h->steps += nsteps;
  {
    unsigned long long bad = ~0ull;
    ACUDA(cudaMemcpy(&bad, h->d_bad, sizeof bad, cudaMemcpyDeviceToHost));
    if (bad != ~0ull) {
      const unsigned long long none = ~0ull;
      ACUDA(cudaMemcpy(h->d_bad, &none, sizeof none, cudaMemcpyHostToDevice));
      char buf[128];
      std::snprintf(buf, sizeof buf, "non-physical state at node %llu during the forward run", bad);
      return afail(h, RLB_ENONPHYS, buf);
    }
  }
  // omega = 1 / tau  =>  dJ/dtau = -omega^2 dJ/domega
  const double wv = 1.0 / h->cfg.tau_v;
  *loss = hs[3];
  dtau[0] = -wv * wv * hs[0];
  if (mrt) {
    const double we = 1.0 / h->cfg.tau_e, wp = 1.0 / h->cfg.tau_eps;
    dtau[1] = -we * we * hs[1];
    dtau[2] = -wp * wp * hs[2];
  } else {
    dtau[1] = 0.0;
    dtau[2] = 0.0;
  }
  return RLB_OK;
#undef ACUDA
}
