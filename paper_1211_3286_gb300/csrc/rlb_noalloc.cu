// rlb_noalloc.cu -- conserved totals of a raw state without any allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// totals: code that has handed all of the GPU's memory to a pool reserved at
// start-up (a framework's caching allocator, a fixed arena) and must not go
// around it; monitoring code that has to report the conserved sums of a run that
// just failed with out-of-memory; and latency-sensitive loops in which
// cudaMalloc / cudaFree would stall the stream by synchronising the device.
// rlb_conserved_totals_noalloc serves them: its only scratch is a file-scope
// device array of fixed size, so it calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// It takes D3Q19 states only (38 values per node): the kernel reads 19 f and 19
// g planes and cannot tell a D2Q9 state (18 values per node) from its size.
//
// The scratch array lives in every GPU that loads librlb until the process
// exits.  All calls share it and it keeps the previous call's contents; each
// call overwrites every partial it later reads, so nothing needs clearing, but
// two calls whose kernels overlap on the GPU (different streams, or different
// host threads on one stream ordering) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/rlb.h"
#include "rlb_internal.h"
#include "rlb_node.cuh"

using namespace rlb;

namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kNodesPerBlock = 65536ull;
constexpr int kMaxBlocks = RLB_NOALLOC_MAX_NODES / kNodesPerBlock;   // 4096 partial slots

// 4096 partials x 5 sums + 5 results, FP64: 160 KiB + 40 B.
static __device__ __align__(256) double s_scratch[kMaxBlocks * 5 + 5];

struct DevicePtr {
  double* ptr = nullptr;
  bool ready = false;
};
std::mutex g_mu;
DevicePtr g_dev[256];

template <typename S>
__global__ void __launch_bounds__(kThreads) k_part(const S* __restrict__ lat, unsigned long long nodes,
                                                  double* __restrict__ part) {
  // block b sums nodes [b * kNodesPerBlock, (b + 1) * kNodesPerBlock) in a fixed order
  const unsigned long long lo = blockIdx.x * kNodesPerBlock;
  const unsigned long long hi = lo + kNodesPerBlock < nodes ? lo + kNodesPerBlock : nodes;
  double acc[5] = {0, 0, 0, 0, 0};
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += kThreads) {
    S f[19], g[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) {
      f[a] = lat[(unsigned long long)a * nodes + i];
      g[a] = lat[(19ull + a) * nodes + i];
    }
    double sp[9], dp[9], Sa, Sd;
    NodeMacro m;
    node_moments<S>(f, g, sp, dp, Sa, Sd, m);
    acc[0] += m.N0; acc[1] += m.T00; acc[2] += m.Mx; acc[3] += m.My; acc[4] += m.Mz;
  }
  __shared__ double sh[5][kThreads];
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) part[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kThreads) k_final(const double* __restrict__ part, int nblocks,
                                                   double* __restrict__ out) {
  __shared__ double sh[5][kThreads];
  double acc[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[c] += part[b * 5 + c];
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

// Device address of s_scratch on the current device, looked up once per device.
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_handleless_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return RLB_ECUDA; }
  if (dev < 0 || dev >= 256) { set_handleless_error("device ordinal out of range"); return RLB_EINVAL; }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev[dev].ready) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, s_scratch);
    if (e != cudaSuccess) {
      set_handleless_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return RLB_ECUDA;
    }
    g_dev[dev].ptr = (double*)p;
    g_dev[dev].ready = true;
  }
  *out = g_dev[dev].ptr;
  return RLB_OK;
}

}  // namespace

extern "C" int rlb_conserved_totals_noalloc(const void* state, size_t nodes, int precision, double* out, int where,
                                            void* stream) {
  if (!state || !out) { set_handleless_error("null argument"); return RLB_EINVAL; }
  if (nodes == 0) { set_handleless_error("nodes must be > 0"); return RLB_EINVAL; }
  if (nodes > (size_t)RLB_NOALLOC_MAX_NODES) {
    set_handleless_error("nodes exceeds the static scratch limit RLB_NOALLOC_MAX_NODES (268435456)");
    return RLB_EINVAL;
  }
  if (precision != RLB_FP64 && precision != RLB_FP32_STORAGE) { set_handleless_error("unknown precision"); return RLB_EINVAL; }
  if (where != RLB_HOST && where != RLB_DEVICE) { set_handleless_error("where must be RLB_HOST or RLB_DEVICE"); return RLB_EINVAL; }
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int nblocks = (int)((nodes + kNodesPerBlock - 1) / kNodesPerBlock);
  if (precision == RLB_FP64)
    k_part<double><<<nblocks, kThreads, 0, s>>>((const double*)state, nodes, scratch);
  else
    k_part<float><<<nblocks, kThreads, 0, s>>>((const float*)state, nodes, scratch);
  double* dst = where == RLB_DEVICE ? out : scratch + kMaxBlocks * 5;
  k_final<<<1, kThreads, 0, s>>>(scratch, nblocks, dst);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_handleless_error(std::string("launch: ") + cudaGetErrorString(e)); return RLB_ECUDA; }
  if (where == RLB_HOST) {
    e = cudaMemcpyAsync(out, dst, 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { set_handleless_error(std::string("copy: ") + cudaGetErrorString(e)); return RLB_ECUDA; }
  }
  return RLB_OK;
}

