// rlb_lattice.cu -- the lattice handle of librlb: allocation, initial state,
// fused pull-stream + collide step kernels, field output, conserved totals and
// raw state I/O (the C ABI declared in include/rlb.h).
//
// Data layout in HBM: two lattices (read / write, swapped every step), each
// holding f[19][nz][ny][nx] followed by g[19][nz][ny][nx] in the storage
// precision (FP64, or FP32 for RLB_FP32_STORAGE).  Populations are pulled from
// x - e_a (x-adjacent threads read adjacent addresses, so every load is
// coalesced), collided in registers with the per-node arithmetic of rlb_node.cuh,
// and written to the node's own slots.
//   FP64 (k_step_ws): two threads per node -- g warps (sums, recovery, g update)
//     and f warps (f update) of the same nodes, u handed over in shared memory;
//   FP32 storage, and FP64 with per-node relaxation times (k_step): one thread
//     per node;
//   D2Q9 (k_step_d2q9): one thread per node, with k_macro_d2q9 first when the
//     C7 correction needs gradients of the macroscopic fields.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rlb.h"
#include "rlb_internal.h"
#include "rlb_io.cuh"
#include "rlb_node.cuh"

using namespace rlb;


namespace {

thread_local std::string g_create_error;

int fail(rlb_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(rlb_handle* h, cudaError_t e, const char* what) {
  return fail(h, RLB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RLB_CUDA(h, call)                               \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

constexpr int kBlockX = 128;
constexpr int kRedBlocks = 608;   // 4 x 152 SMs; fixed so the reduction order is fixed
constexpr int kRedThreads = 256;

struct Geo {
  int nx, ny, nz;
  int bcx, bcy, bcz;   // 1 = zero-gradient
  unsigned long long plane;   // nodes
};

__device__ __forceinline__ int src_minus(int i, int n, int zg) {  // source of a pull with c = +1
  return i > 0 ? i - 1 : (zg ? 0 : n - 1);
}
__device__ __forceinline__ int src_plus(int i, int n, int zg) {   // source of a pull with c = -1
  return i < n - 1 ? i + 1 : (zg ? n - 1 : 0);
}

// Read-only population load.  FP64 populations are streamed past L1 (each value is
// read once per step from its plane; L2 serves the neighbouring rows' reuse), which
// leaves L1 to the FP64 step's register spills.
#ifndef RLB_LD_NOALLOC
#define RLB_LD_NOALLOC 1
#endif
template <typename S>
__device__ __forceinline__ S ldg_nc(const S* p) { return __ldg(p); }
// L2 prefetch size of the population loads: 256 B, the row segment a warp reads
// (512^3 FP32 step 6.763 -> 6.740 ms, 256^3 FP64 step 1.859 -> 1.856 ms)
#ifndef RLB_LD_PF
#define RLB_LD_PF 256
#endif
#if RLB_LD_NOALLOC
template <>
__device__ __forceinline__ double ldg_nc<double>(const double* p) {
  double v;
  if (RLB_LD_PF == 256) asm("ld.global.nc.L1::no_allocate.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p));
  else if (RLB_LD_PF == 128) asm("ld.global.nc.L1::no_allocate.L2::128B.f64 %0, [%1];" : "=d"(v) : "l"(p));
  else asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
#endif
#if RLB_LD_PF
template <>
__device__ __forceinline__ float ldg_nc<float>(const float* p) {
  float v;
  if (RLB_LD_PF == 256) asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  else asm("ld.global.nc.L2::128B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
#endif

// Gather the 19 populations of one distribution arriving at node (x, y, z):
// link a comes from (x - cx, y - cy, z - cz).
template <typename S>
__device__ __forceinline__ void pull19(const S* __restrict__ base, unsigned long long plane, const int (&xs)[3],
                                       const unsigned (&row)[3][3], S (&v)[19]) {
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    const int cx = link_cx(a), cy = link_cy(a), cz = link_cz(a);
    const unsigned idx = row[1 - cz][1 - cy] + (unsigned)xs[1 - cx];
    v[a] = ldg_nc(base + (unsigned long long)a * plane + idx);
  }
}

// Resident 128-thread blocks per SM the FP64 step is compiled for (register cap
// 65536 / (128 x blocks)).
#ifndef RLB_F64_BLOCKS_PER_SM
#define RLB_F64_BLOCKS_PER_SM 3
#endif
// and the FP32-storage step (6: 80 registers, none spilled)
#ifndef RLB_F32_BLOCKS_PER_SM
#define RLB_F32_BLOCKS_PER_SM 6
#endif

template <typename S, bool MRT, bool QSEP, bool ETA = false>
__global__ void __launch_bounds__(kBlockX, sizeof(S) == 8 ? RLB_F64_BLOCKS_PER_SM : RLB_F32_BLOCKS_PER_SM) k_step(const S* __restrict__ src, S* __restrict__ dst, Geo geo,
                                                  StepConst k, unsigned long long* __restrict__ bad) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= geo.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  // source coordinates for offsets c = +1, 0, -1 (index 0, 1, 2 = 1 - c)
  const int xs[3] = {src_minus(x, geo.nx, geo.bcx), x, src_plus(x, geo.nx, geo.bcx)};
  const int ys[3] = {src_minus(y, geo.ny, geo.bcy), y, src_plus(y, geo.ny, geo.bcy)};
  const int zs[3] = {src_minus(z, geo.nz, geo.bcz), z, src_plus(z, geo.nz, geo.bcz)};
  unsigned row[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) row[i][j] = ((unsigned)zs[i] * (unsigned)geo.ny + (unsigned)ys[j]) * (unsigned)geo.nx;

  S f[19], g[19];
  pull19<S>(src, geo.plane, xs, row, f);
  pull19<S>(src + 19ull * geo.plane, geo.plane, xs, row, g);
  bool b;
  if constexpr (sizeof(S) == 8 && ETA) b = node_collide_f64<MRT, QSEP, true>(f, g, k);
  else if constexpr (sizeof(S) == 8) b = node_collide_fx<MRT, QSEP>(f, g, k);
  else b = node_collide_f32s<MRT, QSEP>(f, g, k);
  const unsigned node = row[1][1] + (unsigned)x;
  if (b) atomicMin(bad, (unsigned long long)node);
#pragma unroll
  for (int a = 0; a < 19; ++a) {
    dst[(unsigned long long)a * geo.plane + node] = f[a];
    dst[(19ull + a) * geo.plane + node] = g[a];
  }
}

// FP64 step with warp roles (the integer-pipe collide of rlb_node.cuh).  A block of
// 2 W warps serves 32 W nodes along x: warps [0, W) pull and relax g, warps [W, 2W)
// pull and relax f of the same nodes.  The g warps recover u (Eq. 10 inverted) and
// hand it to the f warps through shared memory across one barrier per warp pair.  Each
// thread holds one distribution of one node, so twice as many warps fit in the
// registers the single-role kernel needs; out-of-range threads (x >= nx) pull the
// clamped node nx - 1, pass the barrier and store that node's values again.
// Resident warps per SM the launch bounds ask of the large-lattice blocks (the
// register cap follows: 24 warps -> 80 registers, 40 B spilled; 32 warps -> 64
// registers, 184 B spilled with the shift-free relaxation, which keeps X^eq live past
// the product); small lattices keep 14 64-thread blocks.
#ifndef RLB_WS_WARPS_PER_SM
#define RLB_WS_WARPS_PER_SM 24
#endif
// Output rounding route of the f and g warps, one bit per link pair and bit 9 for
// the rest link: set = FP64-pipe conversion, clear = integer bit assembly with the
// FP64 pipe only for negative or tiny values (fx::from_fixed_pos).
#ifndef RLB_WS_OUT_F
#define RLB_WS_OUT_F 0x3ff
#endif
#ifndef RLB_WS_OUT_G
#define RLB_WS_OUT_G 0x3ff
#endif
// warps per role in the blocks of large lattices (4: 256-thread blocks serving 128
// nodes along x)
#ifndef RLB_WS_WARPS
#define RLB_WS_WARPS 4
#endif

template <int W, bool MRT, bool QSEP, int RV, int RF>
__global__ void __launch_bounds__(64 * W, W == 1 ? 14 : RLB_WS_WARPS_PER_SM / (2 * W))
    k_step_ws(const double* __restrict__ src, double* __restrict__ dst, Geo geo, StepConst k,
              unsigned long long* __restrict__ bad) {
  __shared__ unsigned long long s_ax[32 * W], s_ay[32 * W], s_az[32 * W];
  __shared__ unsigned s_sg[32 * W];
  const int warp = threadIdx.x >> 5;
  const bool is_g = warp < W;
  const int slot = (is_g ? warp : warp - W) * 32 + (threadIdx.x & 31);
  const int x0 = blockIdx.x * (32 * W) + slot;
  const bool valid = x0 < geo.nx;
  const int x = valid ? x0 : geo.nx - 1;
  const int y = blockIdx.y, z = blockIdx.z;
  const int xs[3] = {src_minus(x, geo.nx, geo.bcx), x, src_plus(x, geo.nx, geo.bcx)};
  const int ys[3] = {src_minus(y, geo.ny, geo.bcy), y, src_plus(y, geo.ny, geo.bcy)};
  const int zs[3] = {src_minus(z, geo.nz, geo.bcz), z, src_plus(z, geo.nz, geo.bcz)};
  unsigned row[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) row[i][j] = ((unsigned)zs[i] * (unsigned)geo.ny + (unsigned)ys[j]) * (unsigned)geo.nx;
  const unsigned long long plane0 = is_g ? 19ull * geo.plane : 0ull;
  double v[19];
  pull19<double>(src + plane0, geo.plane, xs, row, v);

  using namespace fx;
  // both roles: block exponent and fixed-point values.  When every value of every
  // lane of the warp is positive, finite and within 2^24 of its node's largest (the
  // normal case), the conversion skips the sign and the long-shift handling.
  int hmax = __double2hiint(v[0]), hmin = hmax;
#pragma unroll
  for (int a = 1; a < 19; ++a) {
    const int h = __double2hiint(v[a]);
    hmax = max(hmax, h);
    hmin = min(hmin, h);
  }
  const bool fast = __all_sync(0xffffffffu, hmin > 0 && hmax < 0x7ff00000 && hmin >= (((hmax >> 20) - 24) << 20));
  int E;
  long long X[19];
  if (fast) {
    E = hmax >> 20;
#pragma unroll
    for (int a = 0; a < 19; ++a) X[a] = to_fixed_pos(v[a], E + 7);
  } else {
    unsigned me = 0;
#pragma unroll
    for (int a = 0; a < 19; ++a) me = max(me, (unsigned)__double2hiint(v[a]) & 0x7ff00000u);
    E = (int)(me >> 20);
#pragma unroll
    for (int a = 0; a < 19; ++a) X[a] = to_fixed(v[a], E + 7);
  }

  UFix u;
  long long Sa = 0, Sd = 0, T00 = 0, Mx = 0, My = 0, Mz = 0, Pf = 0, dp0 = 0, dp1 = 0, dp2 = 0, N0 = 0;
  unsigned long long sig = 0;
  bool b = (E < 64) | (E > 2046);
  if (is_g) {
    // conserved sums (Eq. 10) and the recovery on them, in fixed point
    long long sp[9], dp[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      sp[p] = X[2 * p + 1] + X[2 * p + 2];
      dp[p] = X[2 * p + 1] - X[2 * p + 2];
    }
    dp0 = dp[0]; dp1 = dp[1]; dp2 = dp[2];
    Sa = sp[0] + sp[1] + sp[2];
    Sd = ((sp[3] + sp[4]) + (sp[5] + sp[6])) + (sp[7] + sp[8]);
    T00 = X[0] + Sa + Sd;
    Mx = dp[0] + dp[3] + dp[4] + dp[5] + dp[6];
    My = dp[1] + dp[3] - dp[4] + dp[7] + dp[8];
    Mz = dp[2] + dp[5] - dp[6] + dp[7] - dp[8];
    bool br;
    sig = fx_recover(T00, Mx, My, Mz, u, br);
    Pf = (long long)sig - T00;
    s_ax[slot] = u.ax;
    s_ay[slot] = u.ay;
    s_az[slot] = u.az;
    s_sg[slot] = u.sx | (u.sy << 1) | (u.sz << 2);
    ufix_products(u);
    b |= br | (Pf <= 0) | (u.xx + u.yy + u.zz >= (1ull << 62));
  } else {
    N0 = X[0];
#pragma unroll
    for (int a = 1; a < 19; ++a) N0 += X[a];
  }
  // g warp i hands u to f warp i only: one named barrier per warp pair (ids 1..W, 64
  // threads each), so a slow g warp holds back its own f warp, not the whole block
  asm volatile("bar.sync %0, 64;" ::"r"(1 + (is_g ? warp : warp - W)) : "memory");
  if (!is_g) {
    u.ax = s_ax[slot];
    u.ay = s_ay[slot];
    u.az = s_az[slot];
    const unsigned sg = s_sg[slot];
    u.sx = sg & 1u;
    u.sy = (sg >> 1) & 1u;
    u.sz = sg >> 2;
    ufix_products(u);
  }

  // equilibria (Eqs. 7-9) and the relaxation constants of this role
  EqPieces q;
  eq_pieces(is_g ? sig : (unsigned long long)N0, u, q);
  const long long SX = q.Xx + q.Xy + q.Xz;             // D u^2 / 4
  long long eq0;
  if (is_g) {
    q.KA = (long long)mulhi((unsigned long long)Pf, kSixth) - (long long)mulhi((unsigned long long)SX, kThird);
    eq0 = (long long)sig - 3 * Pf - 2 * SX;             // sigma - 3P - sigma u^2 / 2
  } else {
    q.KA = (long long)mulhi((unsigned long long)N0, kEighteenth) - (long long)mulhi((unsigned long long)SX, kThird);
    eq0 = (long long)mulhi((unsigned long long)N0, kThird) - 2 * SX;   // N0/3 - N0 u^2 / 2
  }
  // shift-free relaxation (fx::relax_r): RV / RF = 2 for omega >= 1, 1 below
  const unsigned long long Om = is_g ? k.Om2_v : k.Om2_f;
  long long c0 = (long long)(Om >> 1), cA = c0, cD = c0;
  long long dq[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (MRT && is_g) {
    // e and eps projections of g - g^eq from the class sums, at 1/8 scale
    const long long n0 = (X[0] - eq0) >> 3;
    const long long nA = (Sa - Pf) >> 3;
    const long long nD = (Sd - Pf - 2 * SX) >> 3;
    const long long ae = __mul64hi(8 * nD - 11 * nA - 30 * n0, k.CE) >> 6;
    const long long ap = __mul64hi(nD - 4 * nA + 12 * n0, k.CP) >> 2;
    c0 += 30 * ae - 12 * ap;
    cA += 11 * ae + 4 * ap;
    cD -= 8 * ae + ap;
    if (QSEP) {
      const unsigned long long h23 = kTwoThirds >> 1;
      const long long vx = ((Mx - 5 * dp0) >> 2) + (mulhi_su(Mx, kTwoThirds, h23) >> 2);
      const long long vy = ((My - 5 * dp1) >> 2) + (mulhi_su(My, kTwoThirds, h23) >> 2);
      const long long vz = ((Mz - 5 * dp2) >> 2) + (mulhi_su(Mz, kTwoThirds, h23) >> 2);
      const long long aqx = __mul64hi(vx, k.CQ) >> 1, aqy = __mul64hi(vy, k.CQ) >> 1, aqz = __mul64hi(vz, k.CQ) >> 1;
      dq[0] = 4 * aqx; dq[1] = 4 * aqy; dq[2] = 4 * aqz;
      dq[3] = -(aqx + aqy); dq[4] = -(aqx - aqy);
      dq[5] = -(aqx + aqz); dq[6] = -(aqx - aqz);
      dq[7] = -(aqy + aqz); dq[8] = -(aqy - aqz);
    }
  }
  const unsigned node = row[1][1] + (unsigned)x;
  if (valid && b) atomicMin(bad, (unsigned long long)node);
  // Lanes past the row repeat node nx - 1 and compute its values bit for bit, so every
  // lane stores: those lanes write the same bytes to node nx - 1 again, and no branch
  // guards the 19 stores (1.8164 -> 1.7977 ms per 256^3 step).
  double* out = dst + plane0 + node;
  if (is_g) {
    out[0] = from_fixed<(RLB_WS_OUT_G >> 9) & 1>(relax_r<RV>(X[0], eq0, Om, c0), E);
    relax_links_store<RLB_WS_OUT_G, MRT && QSEP, RV>(X, q, Om, cA, cD, dq, E, out, geo.plane, true);
  } else {
    out[0] = from_fixed<(RLB_WS_OUT_F >> 9) & 1>(relax_r<RF>(X[0], eq0, Om, c0), E);
    relax_links_store<RLB_WS_OUT_F, false, RF>(X, q, Om, cA, cD, dq, E, out, geo.plane, true);
  }
}

// FP64 step for small lattices with four lanes per node and distribution: a 64-thread
// block serves 8 nodes along x, warp 0 their g and warp 1 their f.  Lane j = 0, 1, 2 of
// a node holds axis pair j (links 2j + 1, 2j + 2) and the two diagonal pairs of one
// plane, (a, b) = (x, y), (y, z), (x, z): the pairs e_a + e_b and e_a - e_b (pairs 3-4,
// 7-8, 5-6), six links each; lane 3 holds the rest link.  The block exponent, the exact
// integer sums and the rest value are combined over the node's lanes with shuffles, the
// recovery and the equilibrium pieces run in every lane, and each lane relaxes and
// stores its own links: the arithmetic of k_step_ws, link for link, with a node's
// dependent chain about a third as long.  u goes to the f warp through shared memory
// across named barrier 1.  No separate tau_q (QSEP) in this form.
__device__ __forceinline__ long long quad_sum64(long long v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}
__device__ __forceinline__ long long sel3(int j, long long v0, long long v1, long long v2) {
  return j == 0 ? v0 : (j == 1 ? v1 : v2);
}

template <bool MRT, int RV, int RF>
__global__ void __launch_bounds__(64, 8) k_step_quad(const double* __restrict__ src, double* __restrict__ dst, Geo geo,
                                                     StepConst k, unsigned long long* __restrict__ bad) {
  using namespace fx;
  __shared__ unsigned long long s_ax[8], s_ay[8], s_az[8];
  __shared__ unsigned s_sg[8];
  const int lane = threadIdx.x & 31;
  const bool is_g = threadIdx.x < 32;
  const int m = lane >> 2, j = lane & 3;
  const int xv = blockIdx.x * 8 + m;
  const bool valid = xv < geo.nx;
  const int x = valid ? xv : geo.nx - 1;
  const int y = blockIdx.y, z = blockIdx.z;
  const int xm = src_minus(x, geo.nx, geo.bcx), xp = src_plus(x, geo.nx, geo.bcx);
  const int ym = src_minus(y, geo.ny, geo.bcy), yp = src_plus(y, geo.ny, geo.bcy);
  const int zm = src_minus(z, geo.nz, geo.bcz), zp = src_plus(z, geo.nz, geo.bcz);
  // this lane's axes: axis pair i = j; diagonal plane (a, b) = (x, y), (y, z), (x, z)
  const int ai = j < 3 ? j : 0, da = j == 1 ? 1 : 0, db = j == 0 ? 1 : 2;
  const int pd = j == 0 ? 3 : (j == 1 ? 7 : 5);   // first diagonal pair of the plane
  // slot sl: link and direction (slots 0-1 the axis pair, 2-3 pair pd, 4-5 pair pd + 1);
  // lane 3 reads the rest link in every slot
  int link[6], cxs[6], cys[6], czs[6];
#pragma unroll
  for (int sl = 0; sl < 6; ++sl) {
    int cx, cy, cz;
    if (sl < 2) {
      const int c = sl == 0 ? 1 : -1;
      cx = ai == 0 ? c : 0;
      cy = ai == 1 ? c : 0;
      cz = ai == 2 ? c : 0;
      link[sl] = 2 * ai + 1 + sl;
    } else {
      const int sa = (sl & 1) ? -1 : 1;              // +(e_a + e_b), -(e_a + e_b), +(e_a - e_b), -(e_a - e_b)
      const int sb = sl < 4 ? sa : -sa;
      cx = da == 0 ? sa : 0;                          // db is never x
      cy = (da == 1 ? sa : 0) + (db == 1 ? sb : 0);
      cz = db == 2 ? sb : 0;                          // da is never z
      link[sl] = 2 * pd + 1 + (sl - 2);
    }
    const bool rest = j == 3;
    link[sl] = rest ? 0 : link[sl];
    cxs[sl] = rest ? 0 : cx;
    cys[sl] = rest ? 0 : cy;
    czs[sl] = rest ? 0 : cz;
  }
  const unsigned long long plane0 = is_g ? 19ull * geo.plane : 0ull;
  double v[6];
#pragma unroll
  for (int sl = 0; sl < 6; ++sl) {
    const int sx = cxs[sl] > 0 ? xm : (cxs[sl] < 0 ? xp : x);
    const int sy = cys[sl] > 0 ? ym : (cys[sl] < 0 ? yp : y);
    const int sz = czs[sl] > 0 ? zm : (czs[sl] < 0 ? zp : z);
    const unsigned idx = ((unsigned)sz * (unsigned)geo.ny + (unsigned)sy) * (unsigned)geo.nx + (unsigned)sx;
    v[sl] = ldg_nc(src + plane0 + (unsigned long long)link[sl] * geo.plane + idx);
  }
  // block exponent over the node's 19 values (max over its four lanes)
  int hmax = __double2hiint(v[0]), hmin = hmax;
#pragma unroll
  for (int sl = 1; sl < 6; ++sl) {
    const int h = __double2hiint(v[sl]);
    hmax = max(hmax, h);
    hmin = min(hmin, h);
  }
  hmax = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, 1));
  hmax = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, 2));
  const bool fast = __all_sync(0xffffffffu, hmin > 0 && hmax < 0x7ff00000 && hmin >= (((hmax >> 20) - 24) << 20));
  int E;
  long long X[6];
  if (fast) {
    E = hmax >> 20;
#pragma unroll
    for (int sl = 0; sl < 6; ++sl) X[sl] = to_fixed_pos(v[sl], E + 7);
  } else {
    unsigned me = 0;
#pragma unroll
    for (int sl = 0; sl < 6; ++sl) me = max(me, (unsigned)__double2hiint(v[sl]) & 0x7ff00000u);
    me = max(me, (unsigned)__shfl_xor_sync(0xffffffffu, (int)me, 1));
    me = max(me, (unsigned)__shfl_xor_sync(0xffffffffu, (int)me, 2));
    E = (int)(me >> 20);
#pragma unroll
    for (int sl = 0; sl < 6; ++sl) X[sl] = to_fixed(v[sl], E + 7);
  }
  const int base = lane & ~3;
  const long long Xr = __shfl_sync(0xffffffffu, X[0], base + 3);   // the rest link's value
  const long long spa = X[0] + X[1], dpa = X[0] - X[1];
  const long long spp = X[2] + X[3], dpp = X[2] - X[3];
  const long long spm = X[4] + X[5], dpm = X[4] - X[5];
  const bool pairs = j < 3;
  UFix u;
  unsigned long long sig = 0;
  long long Pf = 0, Sa = 0, Sd = 0, N0 = 0;
  bool b = (E < 64) | (E > 2046);
  if (is_g) {
    Sa = quad_sum64(pairs ? spa : 0);
    Sd = quad_sum64(pairs ? spp + spm : 0);
    const long long T00 = Xr + Sa + Sd;
    // momentum: lane 0 adds dp(x) + pairs 3, 4 to M_x and 3 - 4 to M_y; lane 1 dp(y) +
    // pairs 7, 8 to M_y and 7 - 8 to M_z; lane 2 dp(z) and 5 - 6 to M_z, 5 + 6 to M_x
    const long long S2 = dpp + dpm, S3 = dpp - dpm;
    const long long Mx = quad_sum64(j == 0 ? dpa + S2 : (j == 2 ? S2 : 0));
    const long long My = quad_sum64(j == 0 ? S3 : (j == 1 ? dpa + S2 : 0));
    const long long Mz = quad_sum64(j == 1 ? S3 : (j == 2 ? dpa + S3 : 0));
    bool br;
    sig = fx_recover(T00, Mx, My, Mz, u, br);
    Pf = (long long)sig - T00;
    if (j == 0) {
      s_ax[m] = u.ax;
      s_ay[m] = u.ay;
      s_az[m] = u.az;
      s_sg[m] = u.sx | (u.sy << 1) | (u.sz << 2);
    }
    ufix_products(u);
    b |= br | (Pf <= 0) | (u.xx + u.yy + u.zz >= (1ull << 62));
  } else {
    N0 = Xr + quad_sum64(pairs ? (spa + spp) + spm : 0);
  }
  asm volatile("bar.sync 1, 64;" ::: "memory");
  if (!is_g) {
    u.ax = s_ax[m];
    u.ay = s_ay[m];
    u.az = s_az[m];
    const unsigned sg = s_sg[m];
    u.sx = sg & 1u;
    u.sy = (sg >> 1) & 1u;
    u.sz = sg >> 2;
    ufix_products(u);
  }
  EqPieces q;
  eq_pieces(is_g ? sig : (unsigned long long)N0, u, q);
  const long long SX = q.Xx + q.Xy + q.Xz;
  long long eq0;
  if (is_g) {
    q.KA = (long long)mulhi((unsigned long long)Pf, kSixth) - (long long)mulhi((unsigned long long)SX, kThird);
    eq0 = (long long)sig - 3 * Pf - 2 * SX;
  } else {
    q.KA = (long long)mulhi((unsigned long long)N0, kEighteenth) - (long long)mulhi((unsigned long long)SX, kThird);
    eq0 = (long long)mulhi((unsigned long long)N0, kThird) - 2 * SX;
  }
  const unsigned long long Om = is_g ? k.Om2_v : k.Om2_f;   // relax_r forms, as in k_step_ws
  const auto rlx = [is_g](long long X, long long Xeq, unsigned long long O, long long c) {
    return is_g ? relax_r<RV>(X, Xeq, O, c) : relax_r<RF>(X, Xeq, O, c);
  };
  long long c0 = (long long)(Om >> 1), cA = c0, cD = c0;
  if (MRT && is_g) {
    const long long n0 = (Xr - eq0) >> 3;
    const long long nA = (Sa - Pf) >> 3;
    const long long nD = (Sd - Pf - 2 * SX) >> 3;
    const long long ae = __mul64hi(8 * nD - 11 * nA - 30 * n0, k.CE) >> 6;
    const long long ap = __mul64hi(nD - 4 * nA + 12 * n0, k.CP) >> 2;
    c0 += 30 * ae - 12 * ap;
    cA += 11 * ae + 4 * ap;
    cD -= 8 * ae + ap;
  }
  const unsigned node = ((unsigned)z * (unsigned)geo.ny + (unsigned)y) * (unsigned)geo.nx + (unsigned)x;
  if (valid && b && j == 0) atomicMin(bad, (unsigned long long)node);
  double* out = dst + plane0 + node;
  if (pairs) {
    // axis pair: ev = KA + X_i, od = Z_i; diagonal pairs: ev = KA/2 + (X_a + X_b)/2 +- Y_ab,
    // od = (Z_a +- Z_b)/2 (the pieces of relax_links_store)
    const long long Xi = sel3(ai, q.Xx, q.Xy, q.Xz), Zi = sel3(ai, q.Zx, q.Zy, q.Zz);
    const long long Xa = sel3(da, q.Xx, q.Xy, q.Xz), Xb = sel3(db, q.Xx, q.Xy, q.Xz);
    const long long Za = sel3(da, q.Zx, q.Zy, q.Zz), Zb = sel3(db, q.Zx, q.Zy, q.Zz);
    const long long Yab = j == 0 ? q.Yxy : (j == 1 ? q.Yyz : q.Yxz);
    const long long evA = q.KA + Xi, odA = Zi;
    const long long evD = (q.KA >> 1) + ((Xa + Xb) >> 1);
    const long long evP = evD + Yab, odP = (Za + Zb) >> 1;
    const long long evM = evD - Yab, odM = (Za - Zb) >> 1;
    const long long y0 = rlx(X[0], evA + odA, Om, cA), y1 = rlx(X[1], evA - odA, Om, cA);
    const long long y2 = rlx(X[2], evP + odP, Om, cD), y3 = rlx(X[3], evP - odP, Om, cD);
    const long long y4 = rlx(X[4], evM + odM, Om, cD), y5 = rlx(X[5], evM - odM, Om, cD);
    {   // every lane stores (lanes past the row repeat node nx - 1 bit for bit)
      out[(unsigned long long)link[0] * geo.plane] = from_fixed_dp(y0, E);
      out[(unsigned long long)link[1] * geo.plane] = from_fixed_dp(y1, E);
      out[(unsigned long long)link[2] * geo.plane] = from_fixed_dp(y2, E);
      out[(unsigned long long)link[3] * geo.plane] = from_fixed_dp(y3, E);
      out[(unsigned long long)link[4] * geo.plane] = from_fixed_dp(y4, E);
      out[(unsigned long long)link[5] * geo.plane] = from_fixed_dp(y5, E);
    }
  } else {
    out[0] = from_fixed_dp(rlx(X[0], eq0, Om, c0), E);
  }
}

// D2Q9 pull of the 9 f and 9 g arriving at node (x, y).
__device__ __forceinline__ unsigned pull_d2q9(const double* __restrict__ src, const Geo& geo, int x, int y,
                                              double (&f)[9], double (&g)[9]) {
  const int xs[3] = {src_minus(x, geo.nx, geo.bcx), x, src_plus(x, geo.nx, geo.bcx)};
  const unsigned row[3] = {(unsigned)src_minus(y, geo.ny, geo.bcy) * (unsigned)geo.nx, (unsigned)y * (unsigned)geo.nx,
                           (unsigned)src_plus(y, geo.ny, geo.bcy) * (unsigned)geo.nx};
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const unsigned idx = row[1 - d2_cy(a)] + (unsigned)xs[1 - d2_cx(a)];
    f[a] = __ldg(src + (unsigned long long)a * geo.plane + idx);
    g[a] = __ldg(src + (9ull + a) * geo.plane + idx);
  }
  return row[1] + (unsigned)x;
}

// Fields of the pulled D2Q9 state for the C_7 gradients (Eq. 38): per node
// c_s^2 sigma - P, gamma, sigma u_x^2, sigma u_x, sigma u_y^2, sigma u_y.
constexpr int kMacroD2Q9 = 6;
__global__ void __launch_bounds__(kBlockX) k_macro_d2q9(const double* __restrict__ src, double* __restrict__ q,
                                                        Geo geo) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= geo.nx) return;
  double f[9], g[9], dp[4], Sa, Sd;
  const unsigned node = pull_d2q9(src, geo, x, blockIdx.y, f, g);
  NodeMacro m;
  node_moments_d2q9<double>(f, g, dp, Sa, Sd, m);
  node_recover_fast(m);
  const double sux = m.sigma * m.ux, suy = m.sigma * m.uy;
  q[node] = fma(1.0 / 3.0, m.sigma, -m.P);
  q[geo.plane + node] = 1.0 / sqrt(1.0 - m.u2);
  q[2 * geo.plane + node] = sux * m.ux;
  q[3 * geo.plane + node] = sux;
  q[4 * geo.plane + node] = suy * m.uy;
  q[5 * geo.plane + node] = suy;
}

// One axis of the C_7 term (Eq. 38 for a flow along that axis): neighbours im, ip
// of the node along the axis, u its velocity component, qa = q + 2 plane (x) or
// q + 4 plane (y) the sigma u^2 / sigma u fields of that component.
__device__ __forceinline__ double c7_axis(const double* __restrict__ q, const double* __restrict__ qa,
                                          unsigned long long P, unsigned im, unsigned ip, double u, double sigma,
                                          double gam, double theta, double kth) {
  const double d1 = 0.5 * (q[ip] - q[im]);              // d(c_s^2 sigma - P)
  const double d2 = 0.5 * (q[P + ip] - q[P + im]);      // d(gamma)
  const double d3 = 0.5 * (qa[ip] - qa[im]);            // d(sigma u^2)
  const double d4 = 0.5 * (qa[P + ip] - qa[P + im]);    // d(sigma u)
  return 2.0 * (u * d1 - (sigma * (1.0 / 3.0)) * (u / gam) * d2 - u * d3) + kth * (u * u * theta * d4);
}

// D2Q9 (FP64): node (x, y) pulls link a from (x - c_x, y - c_y).  With CORR the
// C_7 term of Eqs. 37-38, C_7 = E_x - E_y, is added to the m_7 = p_xx moment of the
// result.
template <bool MRT, bool QSEP, bool CORR, bool ETA = false>
__global__ void __launch_bounds__(kBlockX) k_step_d2q9(const double* __restrict__ src, double* __restrict__ dst,
                                                       Geo geo, StepConst k, unsigned long long* __restrict__ bad,
                                                       const double* __restrict__ q) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= geo.nx) return;
  const int y = blockIdx.y;
  double f[9], g[9];
  const unsigned node = pull_d2q9(src, geo, x, y, f, g);
  NodeMacro m;
  const bool b = node_collide_d2q9_f64<MRT, QSEP, ETA>(f, g, k, m);
  if (b) atomicMin(bad, (unsigned long long)node);
  if (CORR) {
    // neighbours: a zero-gradient end reuses the edge node, a periodic axis wraps
    const unsigned nx = (unsigned)geo.nx, rowy = (unsigned)y * nx;
    const unsigned xm = rowy + (unsigned)(x > 0 ? x - 1 : (geo.bcx ? 0 : geo.nx - 1));
    const unsigned xp = rowy + (unsigned)(x < geo.nx - 1 ? x + 1 : (geo.bcx ? geo.nx - 1 : 0));
    const unsigned ym = (unsigned)(y > 0 ? y - 1 : (geo.bcy ? 0 : geo.ny - 1)) * nx + (unsigned)x;
    const unsigned yp = (unsigned)(y < geo.ny - 1 ? y + 1 : (geo.bcy ? geo.ny - 1 : 0)) * nx + (unsigned)x;
    const unsigned long long P = geo.plane;
    const double gam = q[P + node];
    const double theta = 1.0 + 1.0 / fma(4.0 * gam, gam, -1.0);   // e / P = 3
    const double c7 = c7_axis(q, q + 2 * P, P, xm, xp, m.ux, m.sigma, gam, theta, k.c7_theta) -
                      c7_axis(q, q + 4 * P, P, ym, yp, m.uy, m.sigma, gam, theta, k.c7_theta);
    // m_7 = p_xx (row c_x^2 - c_y^2, norm 4): (1 - s_7/2) C_7 spread over the axis links
    const double dq = 0.25 * (1.0 - 0.5 * k.omv) * c7;
    g[1] += dq;
    g[2] += dq;
    g[3] -= dq;
    g[4] -= dq;
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    dst[(unsigned long long)a * geo.plane + node] = f[a];
    dst[(9ull + a) * geo.plane + node] = g[a];
  }
}

// Deterministic two-pass sum of (N0, T00, Mx, My, Mz) over all nodes.
template <typename S, int Q = 19>
__global__ void __launch_bounds__(kRedThreads) k_totals_part(const S* __restrict__ lat, unsigned long long nodes,
                                                             double* __restrict__ part) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (unsigned long long i = blockIdx.x * (unsigned long long)kRedThreads + threadIdx.x; i < nodes;
       i += (unsigned long long)kRedBlocks * kRedThreads) {
    NodeMacro m;
    stored_moments<S, Q>(lat, nodes, i, m);
    acc[0] += m.N0; acc[1] += m.T00; acc[2] += m.Mx; acc[3] += m.My; acc[4] += m.Mz;
  }
  __shared__ double sh[5][kRedThreads];
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) part[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kRedThreads) k_totals_final(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[5][kRedThreads];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < kRedBlocks; b += kRedThreads)
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[c] += part[b * 5 + c];
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

Geo make_geo(const rlb_handle* h) {
  Geo g;
  g.nx = h->cfg.nx; g.ny = h->cfg.ny; g.nz = h->cfg.nz;
  g.bcx = h->cfg.bc[0] == RLB_ZERO_GRADIENT;
  g.bcy = h->cfg.bc[1] == RLB_ZERO_GRADIENT;
  g.bcz = h->cfg.bc[2] == RLB_ZERO_GRADIENT;
  g.plane = h->nodes;
  return g;
}

bool qsep(const rlb_config& c) {
  if (c.eta_over_s > 0) return c.collision == RLB_MRT && c.tau_q > 0 && c.tau_q != 1.0;   // tau_q is a ratio
  return c.collision == RLB_MRT && c.tau_q > 0 && c.tau_q != c.tau_v;
}

// The FP64 steps for the relaxation forms of omega_v and omega_f (1: omega < 1, 2: omega >= 1).
template <int W, bool MRT, bool QSEP>
void launch_ws(int rv, int rf, dim3 grid, cudaStream_t st, const double* s, double* d, const Geo& geo,
               const StepConst& k, unsigned long long* bad) {
  if (rv == 2 && rf == 2) k_step_ws<W, MRT, QSEP, 2, 2><<<grid, 64 * W, 0, st>>>(s, d, geo, k, bad);
  else if (rv == 2) k_step_ws<W, MRT, QSEP, 2, 1><<<grid, 64 * W, 0, st>>>(s, d, geo, k, bad);
  else if (rf == 2) k_step_ws<W, MRT, QSEP, 1, 2><<<grid, 64 * W, 0, st>>>(s, d, geo, k, bad);
  else k_step_ws<W, MRT, QSEP, 1, 1><<<grid, 64 * W, 0, st>>>(s, d, geo, k, bad);
}
template <bool MRT>
void launch_quad(int rv, int rf, dim3 grid, cudaStream_t st, const double* s, double* d, const Geo& geo,
                 const StepConst& k, unsigned long long* bad) {
  if (rv == 2 && rf == 2) k_step_quad<MRT, 2, 2><<<grid, 64, 0, st>>>(s, d, geo, k, bad);
  else if (rv == 2) k_step_quad<MRT, 2, 1><<<grid, 64, 0, st>>>(s, d, geo, k, bad);
  else if (rf == 2) k_step_quad<MRT, 1, 2><<<grid, 64, 0, st>>>(s, d, geo, k, bad);
  else k_step_quad<MRT, 1, 1><<<grid, 64, 0, st>>>(s, d, geo, k, bad);
}

template <typename S>
cudaError_t launch_step(rlb_handle* h, const void* src, void* dst, cudaStream_t st) {
  const Geo geo = make_geo(h);
  if (h->Q == 9) {
    const int bx = h->nodes <= 152ull * 128ull * 2ull ? 32 : kBlockX;
    dim3 grid2((geo.nx + bx - 1) / bx, geo.ny, 1);
    const bool mrt2 = h->cfg.collision == RLB_MRT, q2 = qsep(h->cfg);
    const double* s2 = (const double*)src;
    double* d2 = (double*)dst;
    if (h->cfg.eta_over_s > 0) {
      if (!mrt2) k_step_d2q9<false, false, false, true><<<grid2, bx, 0, st>>>(s2, d2, geo, h->k, h->d_bad, nullptr);
      else if (!q2) k_step_d2q9<true, false, false, true><<<grid2, bx, 0, st>>>(s2, d2, geo, h->k, h->d_bad, nullptr);
      else k_step_d2q9<true, true, false, true><<<grid2, bx, 0, st>>>(s2, d2, geo, h->k, h->d_bad, nullptr);
    } else if (h->cfg.correction != RLB_CORR_NONE) {
      k_macro_d2q9<<<grid2, bx, 0, st>>>(s2, h->d_macro, geo);
      if (!q2) k_step_d2q9<true, false, true><<<grid2, bx, 0, st>>>(s2, d2, geo, h->k, h->d_bad, h->d_macro);
      else k_step_d2q9<true, true, true><<<grid2, bx, 0, st>>>(s2, d2, geo, h->k, h->d_bad, h->d_macro);
    } else if (!mrt2) {
      k_step_d2q9<false, false, false><<<grid2, bx, 0, st>>>(s2, d2, geo, h->k, h->d_bad, nullptr);
    } else if (!q2) {
      k_step_d2q9<true, false, false><<<grid2, bx, 0, st>>>(s2, d2, geo, h->k, h->d_bad, nullptr);
    } else {
      k_step_d2q9<true, true, false><<<grid2, bx, 0, st>>>(s2, d2, geo, h->k, h->d_bad, nullptr);
    }
    return cudaGetLastError();
  }
  // small lattices (a 1600-node tube) spread over more SMs with one warp per block:
  // the FP64 pipe of an SM serves 2 lanes per clock, so fewer warps per SM means
  // shorter steps when the lattice cannot fill the GPU anyway
  const int bx = h->nodes <= 152ull * 128ull * 2ull ? 32 : kBlockX;
  dim3 grid((geo.nx + bx - 1) / bx, geo.ny, geo.nz);
  const bool mrt = h->cfg.collision == RLB_MRT, q = qsep(h->cfg);
  const S* s = (const S*)src;
  S* d = (S*)dst;
  if constexpr (sizeof(S) == 8) {
    if (h->cfg.eta_over_s > 0) {
      if (!mrt) k_step<S, false, false, true><<<grid, bx, 0, st>>>(s, d, geo, h->k, h->d_bad);
      else if (!q) k_step<S, true, false, true><<<grid, bx, 0, st>>>(s, d, geo, h->k, h->d_bad);
      else k_step<S, true, true, true><<<grid, bx, 0, st>>>(s, d, geo, h->k, h->d_bad);
      return cudaGetLastError();
    }
  }
  if constexpr (sizeof(S) == 8) {
    // warp roles: 64-thread blocks (one g and one f warp) for small lattices
    const double* s8 = (const double*)src;
    double* d8 = (double*)dst;
    const int rv = h->k.r_v, rf = h->k.r_f;
    if (bx == 32 && !q) {
      // four lanes per node: 8 nodes per 64-thread block
      dim3 gq((geo.nx + 7) / 8, geo.ny, geo.nz);
      if (mrt) launch_quad<true>(rv, rf, gq, st, s8, d8, geo, h->k, h->d_bad);
      else launch_quad<false>(rv, rf, gq, st, s8, d8, geo, h->k, h->d_bad);
    } else if (bx == 32) {
      dim3 gw((geo.nx + 31) / 32, geo.ny, geo.nz);
      launch_ws<1, true, true>(rv, rf, gw, st, s8, d8, geo, h->k, h->d_bad);
    } else {
      constexpr int W = RLB_WS_WARPS;
      dim3 gw((geo.nx + 32 * W - 1) / (32 * W), geo.ny, geo.nz);
      if (!mrt) launch_ws<W, false, false>(rv, rf, gw, st, s8, d8, geo, h->k, h->d_bad);
      else if (!q) launch_ws<W, true, false>(rv, rf, gw, st, s8, d8, geo, h->k, h->d_bad);
      else launch_ws<W, true, true>(rv, rf, gw, st, s8, d8, geo, h->k, h->d_bad);
    }
    return cudaGetLastError();
  } else {
    if (!mrt) k_step<S, false, false><<<grid, bx, 0, st>>>(s, d, geo, h->k, h->d_bad);
    else if (!q) k_step<S, true, false><<<grid, bx, 0, st>>>(s, d, geo, h->k, h->d_bad);
    else k_step<S, true, true><<<grid, bx, 0, st>>>(s, d, geo, h->k, h->d_bad);
    return cudaGetLastError();
  }
}

int check_flag(rlb_handle* h) {
  RLB_CUDA(h, cudaStreamSynchronize(h->stream));
  unsigned long long bad = ULLONG_MAX;
  RLB_CUDA(h, cudaMemcpy(&bad, h->d_bad, sizeof(bad), cudaMemcpyDeviceToHost));
  if (bad != ULLONG_MAX) {
    const unsigned long long reset = ULLONG_MAX;
    RLB_CUDA(h, cudaMemcpy(h->d_bad, &reset, sizeof(reset), cudaMemcpyHostToDevice));
    char buf[160];
    std::snprintf(buf, sizeof buf, "non-physical state at node %llu (x=%llu, y=%llu, z=%llu)", bad,
                  bad % (unsigned long long)h->cfg.nx, (bad / h->cfg.nx) % (unsigned long long)h->cfg.ny,
                  bad / ((unsigned long long)h->cfg.nx * h->cfg.ny));
    return fail(h, RLB_ENONPHYS, buf);
  }
  return RLB_OK;
}

int ensure_stage(rlb_handle* h) {
  if (h->d_stage) return RLB_OK;
  cudaError_t e = cudaMalloc(&h->d_stage, 6 * h->nodes * sizeof(double));
  if (e != cudaSuccess) {
    h->d_stage = nullptr;
    return fail(h, RLB_ENOMEM, "cannot allocate field staging buffer");
  }
  return RLB_OK;
}


}  // namespace

// ----------------------------------------------------------------------------- internal helpers
namespace rlb {
void set_handleless_error(const std::string& msg) { g_create_error = msg; }

cudaError_t enqueue_steps(rlb_handle* h, int nsteps, cudaStream_t st) {
  for (int s = 0; s < nsteps; ++s) {
    const void* src = h->lat[h->cur];
    void* dst = h->lat[1 - h->cur];
    cudaError_t e = h->esize == 8 ? launch_step<double>(h, src, dst, st) : launch_step<float>(h, src, dst, st);
    if (e != cudaSuccess) return e;
    h->cur = 1 - h->cur;
    ++h->steps;
  }
  return cudaSuccess;
}

int validate_taus(double tau_f, double tau_v, double tau_e, double tau_eps, double tau_q, int collision,
                  std::string& why) {
  if (!(tau_f > 0.5) || !(tau_v > 0.5)) { why = "tau_f and tau_v must be > 0.5"; return RLB_EINVAL; }
  if (collision == RLB_MRT) {
    if (!(tau_e > 0.5) || !(tau_eps > 0.5)) { why = "tau_e and tau_eps must be > 0.5"; return RLB_EINVAL; }
    if (tau_q > 0 && !(tau_q > 0.5)) { why = "tau_q must be > 0.5 (or <= 0 for tau_v)"; return RLB_EINVAL; }
  }
  return RLB_OK;
}
}  // namespace rlb

// ----------------------------------------------------------------------------- C ABI
extern "C" int rlb_create(const rlb_config* cfg, rlb_handle** out) {
  if (!cfg || !out) return fail(nullptr, RLB_EINVAL, "null argument");
  if (cfg->nx <= 0 || cfg->ny <= 0 || cfg->nz <= 0) return fail(nullptr, RLB_EINVAL, "lattice extents must be > 0");
  if (cfg->lattice != RLB_D3Q19 && cfg->lattice != RLB_D2Q9)
    return fail(nullptr, RLB_EINVAL, "lattice must be RLB_D3Q19 or RLB_D2Q9");
  if (cfg->lattice == RLB_D2Q9 && (cfg->nz != 1 || cfg->precision != RLB_FP64))
    return fail(nullptr, RLB_EINVAL, "RLB_D2Q9 needs nz == 1 and RLB_FP64");
  if (cfg->correction != RLB_CORR_NONE && cfg->correction != RLB_CORR_C7 && cfg->correction != RLB_CORR_C7_PRINTED)
    return fail(nullptr, RLB_EINVAL, "unknown correction");
  if (cfg->correction != RLB_CORR_NONE && (cfg->lattice != RLB_D2Q9 || cfg->collision != RLB_MRT))
    return fail(nullptr, RLB_EINVAL, "RLB_CORR_C7 needs RLB_D2Q9 and RLB_MRT");
  if (cfg->eos != RLB_EOS_ULTRAREL) return fail(nullptr, RLB_EINVAL, "only RLB_EOS_ULTRAREL (P = e/3) is supported");
  if (cfg->collision != RLB_BGK && cfg->collision != RLB_MRT) return fail(nullptr, RLB_EINVAL, "unknown collision");
  if (cfg->precision != RLB_FP64 && cfg->precision != RLB_FP32_STORAGE)
    return fail(nullptr, RLB_EINVAL, "unknown precision");
  for (int a = 0; a < 3; ++a)
    if (cfg->bc[a] != RLB_PERIODIC && cfg->bc[a] != RLB_ZERO_GRADIENT)
      return fail(nullptr, RLB_EINVAL, "unknown boundary type");
  std::string why;
  const bool eta_mode = cfg->eta_over_s > 0;
  if (eta_mode && (cfg->precision != RLB_FP64 || cfg->correction != RLB_CORR_NONE))
    return fail(nullptr, RLB_EINVAL, "eta_over_s needs RLB_FP64 and no correction term");
  if (eta_mode && cfg->collision == RLB_MRT && (!(cfg->tau_e > 0) || !(cfg->tau_eps > 0)))
    return fail(nullptr, RLB_EINVAL, "eta_over_s with RLB_MRT reads tau_e, tau_eps (and tau_q > 0) as ratios > 0");
  if (!(cfg->eta_over_s >= 0)) return fail(nullptr, RLB_EINVAL, "eta_over_s must be >= 0");
  if (!eta_mode &&
      rlb::validate_taus(cfg->tau_f, cfg->tau_v, cfg->tau_e, cfg->tau_eps, cfg->tau_q, cfg->collision, why))
    return fail(nullptr, RLB_EINVAL, why);
  if (eta_mode && cfg->tau_f > 0 && !(cfg->tau_f > 0.5))
    return fail(nullptr, RLB_EINVAL, "tau_f must be > 0.5 (or <= 0 for tau_f = tau_g)");
  const unsigned long long nodes = (unsigned long long)cfg->nx * cfg->ny * cfg->nz;
  if (nodes >= (1ull << 32) || (unsigned long long)cfg->ny * cfg->nz > 65535ull * 65535ull || cfg->ny > 65535 ||
      cfg->nz > 65535)
    return fail(nullptr, RLB_EINVAL, "lattice too large (nodes must be < 2^32, ny and nz <= 65535)");

  rlb_handle* h = new rlb_handle();
  h->cfg = *cfg;
  h->stream = (cudaStream_t)cfg->stream;
  h->nodes = nodes;
  h->esize = cfg->precision == RLB_FP64 ? 8 : 4;
  h->Q = cfg->lattice == RLB_D2Q9 ? 9 : 19;
  h->k = make_step_const(eta_mode && cfg->tau_f <= 0 ? 1.0 : cfg->tau_f, eta_mode ? 1.0 : cfg->tau_v, cfg->tau_e,
                         cfg->tau_eps, cfg->tau_q, cfg->collision == RLB_MRT, h->Q);
  h->k.eta_s = cfg->eta_over_s;
  h->k.tauf_local = eta_mode && cfg->tau_f <= 0;
  h->k.a_e = cfg->tau_e;
  h->k.a_p = cfg->tau_eps;
  h->k.a_q = cfg->tau_q > 0 ? cfg->tau_q : 1.0;
  h->k.c7_theta = cfg->correction == RLB_CORR_C7_PRINTED ? 2.0 : 1.0;
  cudaGetDevice(&h->device);
  const size_t bytes = 2 * (size_t)h->Q * h->nodes * h->esize;
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&h->lat[i], bytes) != cudaSuccess) {
      cudaGetLastError();
      rlb_destroy(h);
      return fail(nullptr, RLB_ENOMEM, "cannot allocate the two lattices");
    }
  }
  if (cfg->correction != RLB_CORR_NONE &&
      cudaMalloc(&h->d_macro, kMacroD2Q9 * h->nodes * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    h->d_macro = nullptr;
    rlb_destroy(h);
    return fail(nullptr, RLB_ENOMEM, "cannot allocate the correction fields");
  }
  if (cudaMalloc(&h->d_bad, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&h->d_part, (kRedBlocks * 5 + 8) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rlb_destroy(h);
    return fail(nullptr, RLB_ENOMEM, "cannot allocate small device buffers");
  }
  const unsigned long long none = ULLONG_MAX;
  if (cudaMemcpy(h->d_bad, &none, sizeof none, cudaMemcpyHostToDevice) != cudaSuccess) {
    rlb_destroy(h);
    return fail(nullptr, RLB_ECUDA, "cannot initialise device flag");
  }
  *out = h;
  return RLB_OK;
}

extern "C" void rlb_destroy(rlb_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->adj_plan && h->adj_free) h->adj_free(h->adj_plan);
  for (int i = 0; i < 2; ++i)
    if (h->lat[i]) cudaFree(h->lat[i]);
  if (h->d_bad) cudaFree(h->d_bad);
  if (h->d_part) cudaFree(h->d_part);
  if (h->d_stage) cudaFree(h->d_stage);
  if (h->d_macro) cudaFree(h->d_macro);
  delete h;
}

extern "C" const char* rlb_last_error(const rlb_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

extern "C" int rlb_set_fields(rlb_handle* h, const double* e, const double* ux, const double* uy, const double* uz,
                              const double* n, int where) {
  if (!h || !e || !ux || !uy || !uz || !n) return fail(h, RLB_EINVAL, "null argument");
  if (where != RLB_HOST && where != RLB_DEVICE) return fail(h, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  const size_t N = h->nodes;
  const double *de = e, *dx = ux, *dy = uy, *dz = uz, *dn = n;
  if (where == RLB_HOST) {
    // host fields go to the staging buffer; k_init validates both kinds of input on
    // the device (first bad node by atomicMin)
    int rc = ensure_stage(h);
    if (rc) return rc;
    double* s = h->d_stage;
    const double* src[5] = {e, ux, uy, uz, n};
    for (int c = 0; c < 5; ++c)
      RLB_CUDA(h, cudaMemcpyAsync(s + c * N, src[c], N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    de = s; dx = s + N; dy = s + 2 * N; dz = s + 3 * N; dn = s + 4 * N;
  }
  // validate on the device and build the equilibrium state in the spare lattice
  const int spare = 1 - h->cur;
  const unsigned long long none = ULLONG_MAX;
  RLB_CUDA(h, cudaMemcpyAsync(h->d_bad, &none, sizeof none, cudaMemcpyHostToDevice, h->stream));
  if (h->Q == 9)
    k_init<double, 9><<<grid_for(N), 256, 0, h->stream>>>((double*)h->lat[spare], N, de, dx, dy, dz, dn, h->d_bad);
  else if (h->esize == 8)
    k_init<double><<<grid_for(N), 256, 0, h->stream>>>((double*)h->lat[spare], N, de, dx, dy, dz, dn, h->d_bad);
  else
    k_init<float><<<grid_for(N), 256, 0, h->stream>>>((float*)h->lat[spare], N, de, dx, dy, dz, dn, h->d_bad);
  RLB_CUDA(h, cudaGetLastError());
  RLB_CUDA(h, cudaStreamSynchronize(h->stream));
  unsigned long long bad = ULLONG_MAX;
  RLB_CUDA(h, cudaMemcpy(&bad, h->d_bad, sizeof bad, cudaMemcpyDeviceToHost));
  if (bad != ULLONG_MAX) {
    RLB_CUDA(h, cudaMemcpy(h->d_bad, &none, sizeof none, cudaMemcpyHostToDevice));
    char buf[128];
    std::snprintf(buf, sizeof buf, "invalid field at node %llu (need e > 0, n > 0, |u| < 1)", bad);
    return fail(h, RLB_EINVAL, buf);
  }
  h->cur = spare;
  h->steps = 0;
  return RLB_OK;
}

extern "C" int rlb_step(rlb_handle* h, int nsteps) {
  if (!h) return fail(h, RLB_EINVAL, "null handle");
  if (nsteps < 0) return fail(h, RLB_EINVAL, "nsteps must be >= 0");
  cudaError_t e = rlb::enqueue_steps(h, nsteps, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
  return RLB_OK;
}

extern "C" int rlb_check(rlb_handle* h) {
  if (!h) return fail(h, RLB_EINVAL, "null handle");
  return check_flag(h);
}

extern "C" int rlb_get_fields(rlb_handle* h, double* e, double* P, double* ux, double* uy, double* uz, double* n,
                              int where) {
  if (!h) return fail(h, RLB_EINVAL, "null handle");
  if (where != RLB_HOST && where != RLB_DEVICE) return fail(h, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  int rc = ensure_stage(h);
  if (rc) return rc;
  const size_t N = h->nodes;
  double* s = h->d_stage;
  double* dev[6] = {s, s + N, s + 2 * N, s + 3 * N, s + 4 * N, s + 5 * N};
  double* want[6] = {e, P, ux, uy, uz, n};
  if (where == RLB_DEVICE)
    for (int c = 0; c < 6; ++c)
      if (want[c]) dev[c] = want[c];
  if (h->Q == 9)
    k_fields<double, 9><<<grid_for(N), 256, 0, h->stream>>>((const double*)h->lat[h->cur], N, dev[0], dev[1], dev[2],
                                                             dev[3], dev[4], dev[5], h->d_bad);
  else if (h->esize == 8)
    k_fields<double><<<grid_for(N), 256, 0, h->stream>>>((const double*)h->lat[h->cur], N, dev[0], dev[1], dev[2],
                                                          dev[3], dev[4], dev[5], h->d_bad);
  else
    k_fields<float><<<grid_for(N), 256, 0, h->stream>>>((const float*)h->lat[h->cur], N, dev[0], dev[1], dev[2],
                                                         dev[3], dev[4], dev[5], h->d_bad);
  RLB_CUDA(h, cudaGetLastError());
  if (where == RLB_HOST)
    for (int c = 0; c < 6; ++c)
      if (want[c])
        RLB_CUDA(h, cudaMemcpyAsync(want[c], dev[c], N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return check_flag(h);
}

extern "C" int rlb_conserved_totals(rlb_handle* h, double out[5]) {
  if (!h || !out) return fail(h, RLB_EINVAL, "null argument");
  const size_t N = h->nodes;
  if (h->Q == 9)
    k_totals_part<double, 9><<<kRedBlocks, kRedThreads, 0, h->stream>>>((const double*)h->lat[h->cur], N, h->d_part);
  else if (h->esize == 8)
    k_totals_part<double><<<kRedBlocks, kRedThreads, 0, h->stream>>>((const double*)h->lat[h->cur], N, h->d_part);
  else
    k_totals_part<float><<<kRedBlocks, kRedThreads, 0, h->stream>>>((const float*)h->lat[h->cur], N, h->d_part);
  RLB_CUDA(h, cudaGetLastError());
  k_totals_final<<<1, kRedThreads, 0, h->stream>>>(h->d_part, h->d_part + kRedBlocks * 5);
  RLB_CUDA(h, cudaGetLastError());
  RLB_CUDA(h, cudaMemcpyAsync(out, h->d_part + kRedBlocks * 5, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
  RLB_CUDA(h, cudaStreamSynchronize(h->stream));
  return RLB_OK;
}

extern "C" size_t rlb_state_bytes(const rlb_handle* h) { return h ? 2 * (size_t)h->Q * h->nodes * h->esize : 0; }

extern "C" int rlb_save_state(rlb_handle* h, void* buf, int where) {
  if (!h || !buf) return fail(h, RLB_EINVAL, "null argument");
  if (where != RLB_HOST && where != RLB_DEVICE) return fail(h, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  RLB_CUDA(h, cudaMemcpyAsync(buf, h->lat[h->cur], rlb_state_bytes(h),
                              where == RLB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
  RLB_CUDA(h, cudaStreamSynchronize(h->stream));
  return RLB_OK;
}

extern "C" int rlb_load_state(rlb_handle* h, const void* buf, int where) {
  if (!h || !buf) return fail(h, RLB_EINVAL, "null argument");
  if (where != RLB_HOST && where != RLB_DEVICE) return fail(h, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  RLB_CUDA(h, cudaMemcpyAsync(h->lat[h->cur], buf, rlb_state_bytes(h),
                              where == RLB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
  RLB_CUDA(h, cudaStreamSynchronize(h->stream));
  h->steps = 0;
  return RLB_OK;
}

extern "C" long long rlb_steps_done(const rlb_handle* h) { return h ? h->steps : -1; }
