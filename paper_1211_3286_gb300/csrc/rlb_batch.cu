// rlb_batch.cu -- batched quasi-1D shock tubes (include/rlb_batch.h).
//
// Layout: the tubes are concatenated into one flat node list; two lattices
// (f[19][nodes] then g[19][nodes] each) in the storage precision.
//
// Execution: one persistent kernel.  Each CTA repeatedly takes the next tube
// from a longest-first work list (an atomic counter; longest-processing-time
// order keeps the tail short) and advances that tube by all nsteps with
// CTA-local barriers.  Tubes never exchange data, so no grid-wide barrier exists
// and no CTA waits on another.  Steps run in place in pairs on one lattice (the AA
// scheme, tube_step), which halves a tube's working set in L2 against reading one
// lattice and writing the other; an odd last step goes into the other lattice.
// Lattice accesses use ld.global.cg / st.global.cg (coherent at L2 for the CTA's
// own writes after __syncthreads).
//
// Launch shape (threads per CTA, CTAs per SM) is picked by rlb_batch_autotune,
// which times each candidate on a copy of the state.  rlb_batch_run replays
// [reset counter, persistent kernel] from a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/rlb.h"
#include "../../include/rlb_batch.h"
#include "rlb_internal.h"
#include "rlb_io.cuh"
#include "rlb_node.cuh"

using namespace rlb;

namespace {

struct TubeInfo {
  unsigned long long off;
  int L;
  int id;
};

// FP32 lattice loads with a 256-byte L2 prefetch size (1024-tube sweep: about +1 %)
#ifndef RLB_TUBES_PF
#define RLB_TUBES_PF 1
#endif
template <typename S>
__device__ __forceinline__ S ld_cg(const S* p) { return __ldcg(p); }
#if RLB_TUBES_PF
template <>
__device__ __forceinline__ float ld_cg<float>(const float* p) {
  float v;
  asm volatile("ld.global.cg.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
#endif
template <typename S>
__device__ __forceinline__ void st_cg(S* p, S v) { __stcg(p, v); }

// Links with c_x = +1 and c_x = -1 (the ones a zero-gradient end clamps).
__device__ __forceinline__ int xplus_index(int a) {   // a in {1, 7, 9, 11, 13} -> 0..4
  return a == 1 ? 0 : (a - 5) / 2;
}
__device__ __forceinline__ int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

template <typename S, bool MRT>
__device__ __forceinline__ bool tube_collide(S (&f)[19], S (&g)[19], const StepConst& k) {
  if constexpr (sizeof(S) == 8) return node_collide_fx<MRT, false>(f, g, k);
  else return node_collide_f32s<MRT, false>(f, g, k);
}

// One step of a tube.  mode 0: two lattices, node x pulls from src (x - c_x, clamped
// at the zero-gradient ends) and stores at x in dst.  Modes 1 and 2 are the in-place
// pair of the AA scheme on one lattice (src == dst), which halves a tube's working set:
//   layout N: slot a of node x holds F_a(x), the post-collision population;
//   layout S: slot abar of node x holds the value node x pulls for link a at the next
//     step, F_a(x - c_a) (clamped).
//   mode 1 (N -> S): node x pulls F_a(x - c_a) from slot a of x - c_a, collides, and
//     writes each F'_a(x) to slot abar of x + c_a (and, at an end where x - c_a falls
//     outside, to slot abar of x itself).  Every slot a node reads is written only by
//     that node; the clamped pulls at the ends come from edge copies in shared memory,
//     since the neighbour overwrites the edge node's own slot within the step.
//   mode 2 (S -> N): node x reads its own slots abar, collides, writes its own slots a
//     and refreshes the edge copies.
// One collide call site serves the three modes; the mode picks whole load and store
// blocks, and only the two end nodes take the clamping / edge-copy path.
template <typename S, bool MRT>
__device__ __forceinline__ void tube_step(int mode, const S* src, S* dst, const TubeInfo& ti,
                                          unsigned long long nodes, const StepConst& k, S (&edge)[2][2][5],
                                          unsigned long long* bad) {
  for (int x = threadIdx.x; x < ti.L; x += blockDim.x) {
    const unsigned long long x0 = ti.off + (unsigned long long)x;
    const bool end = x == 0 || x == ti.L - 1;
    S f[19], g[19];
    if (mode == 2) {
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        f[a] = ld_cg(src + (unsigned long long)opp(a) * nodes + x0);
        g[a] = ld_cg(src + (19ull + opp(a)) * nodes + x0);
      }
    } else if (!end) {
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        const unsigned long long i = x0 - (long long)link_cx(a);
        f[a] = ld_cg(src + (unsigned long long)a * nodes + i);
        g[a] = ld_cg(src + (19ull + a) * nodes + i);
      }
    } else {
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        const int cx = link_cx(a), xs = x - cx;
        const bool outside = cx != 0 && (xs < 0 || xs >= ti.L);
        if (mode == 1 && outside) {                    // clamped pull: edge copy
          const int side = cx == 1 ? 0 : 1, j = xplus_index(cx == 1 ? a : opp(a));
          f[a] = edge[side][0][j];
          g[a] = edge[side][1][j];
        } else {
          const unsigned long long i = ti.off + (unsigned long long)(outside ? x : xs);
          f[a] = ld_cg(src + (unsigned long long)a * nodes + i);
          g[a] = ld_cg(src + (19ull + a) * nodes + i);
        }
      }
    }
    if (tube_collide<S, MRT>(f, g, k)) atomicMin(bad, x0);
    if (mode == 1 && !end) {
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        const unsigned long long i = x0 + (long long)link_cx(a);
        st_cg(dst + (unsigned long long)opp(a) * nodes + i, f[a]);
        st_cg(dst + (19ull + opp(a)) * nodes + i, g[a]);
      }
    } else if (mode == 1) {
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        const int cx = link_cx(a), ab = opp(a), xt = x + cx, xs = x - cx;
        if (xt >= 0 && xt < ti.L) {
          const unsigned long long i = ti.off + (unsigned long long)xt;
          st_cg(dst + (unsigned long long)ab * nodes + i, f[a]);
          st_cg(dst + (19ull + ab) * nodes + i, g[a]);
        }
        if (cx != 0 && (xs < 0 || xs >= ti.L)) {
          st_cg(dst + (unsigned long long)ab * nodes + x0, f[a]);
          st_cg(dst + (19ull + ab) * nodes + x0, g[a]);
        }
      }
    } else {
#pragma unroll
      for (int a = 0; a < 19; ++a) {
        st_cg(dst + (unsigned long long)a * nodes + x0, f[a]);
        st_cg(dst + (19ull + a) * nodes + x0, g[a]);
      }
      if (mode == 2 && end) {
#pragma unroll
        for (int a = 0; a < 19; ++a) {
          const int cx = link_cx(a);
          if (cx == 1 && x == 0) {
            edge[0][0][xplus_index(a)] = f[a];
            edge[0][1][xplus_index(a)] = g[a];
          }
          if (cx == -1 && x == ti.L - 1) {
            edge[1][0][xplus_index(opp(a))] = f[a];
            edge[1][1][xplus_index(opp(a))] = g[a];
          }
        }
      }
    }
  }
}

// Persistent tube kernel: each CTA takes the next tube of the longest-first list and
// advances it by nsteps: in place pairs of steps on latA (AA scheme), and for an odd
// nsteps one last two-lattice step into latB.
// FP32 storage: RLB_TUBES_F32_THREADS threads x RLB_TUBES_F32_BLOCKS CTAs per SM set the
// register cap (320 x 2: 96 registers, none spilled, 20 warps per SM, 304 tubes in
// flight; 256 x 3 at 80 registers ran 3 % slower: more warps, but 456 tubes overflow
// L2); FP64 (the integer-pipe collide needs about 170 registers): up to 256 threads.
// The autotuner skips shapes the bound excludes.
#ifndef RLB_TUBES_F32_THREADS
#define RLB_TUBES_F32_THREADS 320
#endif
#ifndef RLB_TUBES_F32_BLOCKS
#define RLB_TUBES_F32_BLOCKS 2
#endif
template <typename S, bool MRT>
__global__ void __launch_bounds__(sizeof(S) == 8 ? 256 : RLB_TUBES_F32_THREADS, sizeof(S) == 8 ? 1 : RLB_TUBES_F32_BLOCKS) k_tubes(const TubeInfo* __restrict__ order, int ntubes, const StepConst* __restrict__ consts,
                        S* latA, S* latB, unsigned long long nodes, int nsteps, unsigned* __restrict__ counter,
                        unsigned long long* __restrict__ bad) {
  __shared__ int s_t;
  __shared__ S edge[2][2][5];   // [left/right end][f/g][link with c_x = +1 / its opposite]
  __shared__ StepConst s_k;     // the tube's constants, read from shared memory where used
  for (;;) {
    if (threadIdx.x == 0) s_t = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int t = s_t;
    __syncthreads();
    if (t >= ntubes) return;
    const TubeInfo ti = order[t];
    if (threadIdx.x == 0) s_k = consts[ti.id];
    const StepConst& k = s_k;
    // edge copies of layout N: the end nodes' own populations of the clamped links
    if (threadIdx.x < 20) {
      const int side = threadIdx.x / 10, d = (threadIdx.x / 5) & 1, j = threadIdx.x % 5;
      const int a = side == 0 ? (j == 0 ? 1 : 2 * j + 5) : (j == 0 ? 2 : 2 * j + 6);
      const unsigned long long x0 = ti.off + (unsigned long long)(side == 0 ? 0 : ti.L - 1);
      edge[side][d][j] = ld_cg(latA + (19ull * d + a) * nodes + x0);
    }
    __syncthreads();
    for (int s = 0; s < nsteps; ++s) {
      // pairs in place (modes 1, 2); an odd last step into the other lattice (mode 0)
      const int mode = (nsteps & 1) && s == nsteps - 1 ? 0 : 1 + (s & 1);
      tube_step<S, MRT>(mode, latA, mode == 0 ? latB : latA, ti, nodes, k, edge, bad);
      __syncthreads();
    }
  }
}

}  // namespace

struct rlb_batch {
  int ntubes = 0;
  int collision = RLB_MRT;
  int precision = RLB_FP64;
  size_t esize = 8;
  size_t nodes = 0;
  std::vector<int> lengths;
  std::vector<size_t> offsets;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;                 // private stream used for graph capture
  void* lat[2] = {nullptr, nullptr};
  int cur = 0;
  TubeInfo* d_order = nullptr;
  StepConst* d_consts = nullptr;
  unsigned* d_counter = nullptr;
  unsigned long long* d_bad = nullptr;
  double* d_stage = nullptr;
  int threads = 128, ctas_per_sm = 0;         // 0 = maximum occupancy
  int sms = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int g_steps = -1, g_cur = -1, g_threads = -1, g_ctas = -1;
  std::string err;
};

namespace {

thread_local std::string g_batch_create_error;

int bfail(rlb_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  else g_batch_create_error = m;
  return code;
}

#define BCUDA(b, call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return bfail(b, RLB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename S, bool MRT>
void* kernel_ptr() { return (void*)k_tubes<S, MRT>; }

void* tube_kernel(const rlb_batch* b) {
  if (b->esize == 8) return b->collision == RLB_MRT ? kernel_ptr<double, true>() : kernel_ptr<double, false>();
  return b->collision == RLB_MRT ? kernel_ptr<float, true>() : kernel_ptr<float, false>();
}

int grid_size(const rlb_batch* b, int threads, int ctas_per_sm) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tube_kernel(b), threads, 0) != cudaSuccess) {
    cudaGetLastError();
    occ = 0;
  }
  if (occ < 1) occ = 1;
  int per = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  int grid = per * b->sms;
  return std::max(1, std::min(grid, b->ntubes));
}

cudaError_t launch_tubes(rlb_batch* b, cudaStream_t s, void* A, void* B, int nsteps, int threads, int grid) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const unsigned long long N = b->nodes;
  if (b->esize == 8) {
    if (b->collision == RLB_MRT)
      k_tubes<double, true><<<grid, threads, 0, s>>>(b->d_order, b->ntubes, b->d_consts, (double*)A, (double*)B, N,
                                                     nsteps, b->d_counter, b->d_bad);
    else
      k_tubes<double, false><<<grid, threads, 0, s>>>(b->d_order, b->ntubes, b->d_consts, (double*)A, (double*)B, N,
                                                      nsteps, b->d_counter, b->d_bad);
  } else {
    if (b->collision == RLB_MRT)
      k_tubes<float, true><<<grid, threads, 0, s>>>(b->d_order, b->ntubes, b->d_consts, (float*)A, (float*)B, N,
                                                    nsteps, b->d_counter, b->d_bad);
    else
      k_tubes<float, false><<<grid, threads, 0, s>>>(b->d_order, b->ntubes, b->d_consts, (float*)A, (float*)B, N,
                                                     nsteps, b->d_counter, b->d_bad);
  }
  return cudaGetLastError();
}

int ensure_stage(rlb_batch* b) {
  if (b->d_stage) return RLB_OK;
  if (cudaMalloc(&b->d_stage, 6 * b->nodes * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    b->d_stage = nullptr;
    return bfail(b, RLB_ENOMEM, "cannot allocate field staging buffer");
  }
  return RLB_OK;
}

int read_flag(rlb_batch* b) {
  BCUDA(b, cudaStreamSynchronize(b->stream));
  unsigned long long bad = ULLONG_MAX;
  BCUDA(b, cudaMemcpy(&bad, b->d_bad, sizeof bad, cudaMemcpyDeviceToHost));
  if (bad != ULLONG_MAX) {
    const unsigned long long none = ULLONG_MAX;
    BCUDA(b, cudaMemcpy(b->d_bad, &none, sizeof none, cudaMemcpyHostToDevice));
    const size_t t = std::upper_bound(b->offsets.begin(), b->offsets.end(), (size_t)bad) - b->offsets.begin() - 1;
    char buf[160];
    std::snprintf(buf, sizeof buf, "non-physical state at node %llu (tube %zu, x=%llu)", bad, t,
                  bad - (unsigned long long)b->offsets[t]);
    return bfail(b, RLB_ENONPHYS, buf);
  }
  return RLB_OK;
}

void drop_graph(rlb_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->g_steps = -1;
}

}  // namespace

extern "C" int rlb_batch_create(const rlb_batch_desc* d, rlb_batch** out) {
  if (!d || !out || !d->lengths || !d->taus) return bfail(nullptr, RLB_EINVAL, "null argument");
  if (d->ntubes < 1) return bfail(nullptr, RLB_EINVAL, "ntubes must be >= 1");
  if (d->collision != RLB_MRT && d->collision != RLB_BGK) return bfail(nullptr, RLB_EINVAL, "unknown collision");
  if (d->precision != RLB_FP64 && d->precision != RLB_FP32_STORAGE)
    return bfail(nullptr, RLB_EINVAL, "unknown precision");
  unsigned long long total = 0;
  for (int t = 0; t < d->ntubes; ++t) {
    if (d->lengths[t] < 1) return bfail(nullptr, RLB_EINVAL, "tube lengths must be >= 1");
    total += (unsigned long long)d->lengths[t];
    const double tf = d->tau_f ? d->tau_f[t] : d->taus[3 * t];
    std::string why;
    if (validate_taus(tf, d->taus[3 * t], d->taus[3 * t + 1], d->taus[3 * t + 2], 0.0, d->collision, why)) {
      char buf[200];
      std::snprintf(buf, sizeof buf, "tube %d: %s", t, why.c_str());
      return bfail(nullptr, RLB_EINVAL, buf);
    }
  }
  if (total >= (1ull << 32)) return bfail(nullptr, RLB_EINVAL, "too many nodes (sum of lengths must be < 2^32)");

  rlb_batch* b = new rlb_batch();
  b->ntubes = d->ntubes;
  b->collision = d->collision;
  b->precision = d->precision;
  b->esize = d->precision == RLB_FP64 ? 8 : 4;
  b->nodes = total;
  b->stream = (cudaStream_t)d->stream;
  b->lengths.assign(d->lengths, d->lengths + d->ntubes);
  b->offsets.resize(d->ntubes + 1);
  b->offsets[0] = 0;
  for (int t = 0; t < d->ntubes; ++t) b->offsets[t + 1] = b->offsets[t] + d->lengths[t];
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);

  // longest-processing-time order
  std::vector<int> idx(d->ntubes);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return d->lengths[a] > d->lengths[c]; });
  std::vector<TubeInfo> order(d->ntubes);
  for (int i = 0; i < d->ntubes; ++i) order[i] = TubeInfo{b->offsets[idx[i]], d->lengths[idx[i]], idx[i]};
  std::vector<StepConst> consts(d->ntubes);
  for (int t = 0; t < d->ntubes; ++t) {
    const double tv = d->taus[3 * t], te = d->taus[3 * t + 1], tp = d->taus[3 * t + 2];
    consts[t] = make_step_const(d->tau_f ? d->tau_f[t] : tv, tv, te, tp, 0.0, d->collision == RLB_MRT);
  }
  const size_t bytes = 38 * b->nodes * b->esize;
  bool ok = cudaMalloc(&b->lat[0], bytes) == cudaSuccess && cudaMalloc(&b->lat[1], bytes) == cudaSuccess &&
            cudaMalloc(&b->d_order, sizeof(TubeInfo) * d->ntubes) == cudaSuccess &&
            cudaMalloc(&b->d_consts, sizeof(StepConst) * d->ntubes) == cudaSuccess &&
            cudaMalloc(&b->d_counter, sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&b->d_bad, sizeof(unsigned long long)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    rlb_batch_destroy(b);
    return bfail(nullptr, RLB_ENOMEM, "cannot allocate the batch lattices");
  }
  const unsigned long long none = ULLONG_MAX;
  if (cudaMemcpy(b->d_order, order.data(), sizeof(TubeInfo) * d->ntubes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_consts, consts.data(), sizeof(StepConst) * d->ntubes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_bad, &none, sizeof none, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    rlb_batch_destroy(b);
    return bfail(nullptr, RLB_ECUDA, "cannot initialise the batch");
  }
  *out = b;
  return RLB_OK;
}

extern "C" void rlb_batch_destroy(rlb_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int i = 0; i < 2; ++i)
    if (b->lat[i]) cudaFree(b->lat[i]);
  if (b->d_order) cudaFree(b->d_order);
  if (b->d_consts) cudaFree(b->d_consts);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->d_bad) cudaFree(b->d_bad);
  if (b->d_stage) cudaFree(b->d_stage);
  delete b;
}

extern "C" const char* rlb_batch_last_error(const rlb_batch* b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

extern "C" size_t rlb_batch_nodes(const rlb_batch* b) { return b ? b->nodes : 0; }

extern "C" size_t rlb_batch_offset(const rlb_batch* b, int tube) {
  if (!b || tube < 0 || tube > b->ntubes) return 0;
  return b->offsets[tube];
}

extern "C" int rlb_batch_set_fields(rlb_batch* b, const double* e, const double* ux, const double* uy,
                                    const double* uz, const double* n, int where) {
  if (!b || !e || !ux || !uy || !uz || !n) return bfail(b, RLB_EINVAL, "null argument");
  if (where != RLB_HOST && where != RLB_DEVICE) return bfail(b, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  const size_t N = b->nodes;
  const double *de = e, *dx = ux, *dy = uy, *dz = uz, *dn = n;
  if (where == RLB_HOST) {
    int rc = ensure_stage(b);
    if (rc) return rc;
    const double* src[5] = {e, ux, uy, uz, n};
    for (int c = 0; c < 5; ++c)
      BCUDA(b, cudaMemcpyAsync(b->d_stage + c * N, src[c], N * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    de = b->d_stage; dx = de + N; dy = de + 2 * N; dz = de + 3 * N; dn = de + 4 * N;
  }
  const int spare = 1 - b->cur;
  const unsigned long long none = ULLONG_MAX;
  BCUDA(b, cudaMemcpyAsync(b->d_bad, &none, sizeof none, cudaMemcpyHostToDevice, b->stream));
  if (b->esize == 8)
    k_init<double><<<grid_for(N), 256, 0, b->stream>>>((double*)b->lat[spare], N, de, dx, dy, dz, dn, b->d_bad);
  else
    k_init<float><<<grid_for(N), 256, 0, b->stream>>>((float*)b->lat[spare], N, de, dx, dy, dz, dn, b->d_bad);
  BCUDA(b, cudaGetLastError());
  BCUDA(b, cudaStreamSynchronize(b->stream));
  unsigned long long bad = ULLONG_MAX;
  BCUDA(b, cudaMemcpy(&bad, b->d_bad, sizeof bad, cudaMemcpyDeviceToHost));
  if (bad != ULLONG_MAX) {
    BCUDA(b, cudaMemcpy(b->d_bad, &none, sizeof none, cudaMemcpyHostToDevice));
    char buf[128];
    std::snprintf(buf, sizeof buf, "invalid field at node %llu (need e > 0, n > 0, |u| < 1)", bad);
    return bfail(b, RLB_EINVAL, buf);
  }
  b->cur = spare;
  return RLB_OK;
}

extern "C" int rlb_batch_autotune(rlb_batch* b, int trial_steps, int* chosen) {
  if (!b) return bfail(b, RLB_EINVAL, "null batch");
  if (trial_steps < 1) return bfail(b, RLB_EINVAL, "trial_steps must be >= 1");
  const size_t bytes = rlb_batch_state_bytes(b);
  void* tr[2] = {nullptr, nullptr};
  if (cudaMalloc(&tr[0], bytes) != cudaSuccess || cudaMalloc(&tr[1], bytes) != cudaSuccess) {
    cudaGetLastError();
    if (tr[0]) cudaFree(tr[0]);
    return bfail(b, RLB_ENOMEM, "cannot allocate autotuning buffers");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int cand_threads[] = {64, 96, 128, 160, 192, 224, 256, 288, 320, 352, 384, 448, 512};
  const int cand_ctas[] = {1, 2, 3, 4, 5, 6, 8, 12, 16};
  float best = 1e30f;
  int bt = b->threads, bc = b->ctas_per_sm;
  int rc = RLB_OK;
  cudaFuncAttributes fa{};
  const int max_threads =
      cudaFuncGetAttributes(&fa, tube_kernel(b)) == cudaSuccess ? fa.maxThreadsPerBlock : 256;
  cudaGetLastError();
  for (int th : cand_threads) {
    int occ = 0;
    // block sizes above the kernel's launch bound are not candidates
    if (th > max_threads ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tube_kernel(b), th, 0) != cudaSuccess) {
      cudaGetLastError();
      occ = 0;
    }
    for (int c : cand_ctas) {
      if (c > occ) continue;
      cudaError_t e = cudaMemcpyAsync(tr[0], b->lat[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) e = launch_tubes(b, b->stream, tr[0], tr[1], trial_steps, th, grid_size(b, th, c));
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        rc = bfail(b, RLB_ECUDA, std::string("autotune trial: ") + cudaGetErrorString(e));
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bt = th;
        bc = c;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tr[0]);
  cudaFree(tr[1]);
  if (rc) return rc;
  // trial runs may have flagged nodes of the copies; the real state is untouched
  const unsigned long long none = ULLONG_MAX;
  BCUDA(b, cudaMemcpy(b->d_bad, &none, sizeof none, cudaMemcpyHostToDevice));
  b->threads = bt;
  b->ctas_per_sm = bc;
  if (chosen) {
    chosen[0] = bt;
    chosen[1] = bc;
  }
  return RLB_OK;
}

extern "C" int rlb_batch_set_shape(rlb_batch* b, int threads, int ctas_per_sm) {
  if (!b) return bfail(b, RLB_EINVAL, "null batch");
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, tube_kernel(b)) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, RLB_ECUDA, "cannot query the tube kernel");
  }
  if (threads < 32 || threads % 32 != 0 || threads > fa.maxThreadsPerBlock)
    return bfail(b, RLB_EINVAL, "threads must be a multiple of 32 up to " + std::to_string(fa.maxThreadsPerBlock));
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tube_kernel(b), threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, RLB_ECUDA, "cannot query the occupancy of the tube kernel");
  }
  if (ctas_per_sm < 0 || ctas_per_sm > occ)
    return bfail(b, RLB_EINVAL, "ctas_per_sm must be 0 to " + std::to_string(occ) + " at " +
                                    std::to_string(threads) + " threads");
  b->threads = threads;
  b->ctas_per_sm = ctas_per_sm;
  return RLB_OK;
}

extern "C" int rlb_batch_run(rlb_batch* b, int nsteps) {
  if (!b) return bfail(b, RLB_EINVAL, "null batch");
  if (nsteps < 0) return bfail(b, RLB_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return RLB_OK;
  if (!b->exec || b->g_steps != nsteps || b->g_cur != b->cur || b->g_threads != b->threads ||
      b->g_ctas != b->ctas_per_sm) {
    drop_graph(b);
    const int grid = grid_size(b, b->threads, b->ctas_per_sm);
    BCUDA(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = launch_tubes(b, b->cap, b->lat[b->cur], b->lat[1 - b->cur], nsteps, b->threads, grid);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, RLB_ECUDA, std::string("graph capture: ") +
                                     cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    b->graph = g;
    BCUDA(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->g_steps = nsteps;
    b->g_cur = b->cur;
    b->g_threads = b->threads;
    b->g_ctas = b->ctas_per_sm;
  }
  BCUDA(b, cudaGraphLaunch(b->exec, b->stream));
  if (nsteps & 1) b->cur = 1 - b->cur;
  return RLB_OK;
}

extern "C" int rlb_batch_check(rlb_batch* b) {
  if (!b) return bfail(b, RLB_EINVAL, "null batch");
  return read_flag(b);
}

extern "C" int rlb_batch_get_fields(rlb_batch* b, double* e, double* P, double* ux, double* uy, double* uz,
                                    double* n, int where) {
  if (!b) return bfail(b, RLB_EINVAL, "null batch");
  if (where != RLB_HOST && where != RLB_DEVICE) return bfail(b, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  int rc = ensure_stage(b);
  if (rc) return rc;
  const size_t N = b->nodes;
  double* dev[6];
  double* want[6] = {e, P, ux, uy, uz, n};
  for (int c = 0; c < 6; ++c) dev[c] = (where == RLB_DEVICE && want[c]) ? want[c] : b->d_stage + c * N;
  if (b->esize == 8)
    k_fields<double><<<grid_for(N), 256, 0, b->stream>>>((const double*)b->lat[b->cur], N, dev[0], dev[1], dev[2],
                                                          dev[3], dev[4], dev[5], b->d_bad);
  else
    k_fields<float><<<grid_for(N), 256, 0, b->stream>>>((const float*)b->lat[b->cur], N, dev[0], dev[1], dev[2],
                                                         dev[3], dev[4], dev[5], b->d_bad);
  BCUDA(b, cudaGetLastError());
  if (where == RLB_HOST)
    for (int c = 0; c < 6; ++c)
      if (want[c]) BCUDA(b, cudaMemcpyAsync(want[c], dev[c], N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  return read_flag(b);
}

extern "C" size_t rlb_batch_state_bytes(const rlb_batch* b) { return b ? 38 * b->nodes * b->esize : 0; }

extern "C" int rlb_batch_save_state(rlb_batch* b, void* buf, int where) {
  if (!b || !buf) return bfail(b, RLB_EINVAL, "null argument");
  if (where != RLB_HOST && where != RLB_DEVICE) return bfail(b, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  BCUDA(b, cudaMemcpyAsync(buf, b->lat[b->cur], rlb_batch_state_bytes(b),
                           where == RLB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  return RLB_OK;
}

extern "C" int rlb_batch_load_state(rlb_batch* b, const void* buf, int where) {
  if (!b || !buf) return bfail(b, RLB_EINVAL, "null argument");
  if (where != RLB_HOST && where != RLB_DEVICE) return bfail(b, RLB_EINVAL, "where must be RLB_HOST or RLB_DEVICE");
  BCUDA(b, cudaMemcpyAsync(b->lat[b->cur], buf, rlb_batch_state_bytes(b),
                           where == RLB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  return RLB_OK;
}
