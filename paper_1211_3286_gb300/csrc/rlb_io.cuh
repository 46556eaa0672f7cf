// rlb_io.cuh -- kernels shared by the lattice and batch handles of librlb:
// equilibrium initial state from FP64 fields (Eqs. 7-9; Eqs. 32-33 for D2Q9) and
// field output from a stored state (Eq. 10 plus the closed-form recovery).  Both
// treat the state as a flat list of `nodes` nodes with layout f[Q][nodes] then
// g[Q][nodes], Q = 19 (D3Q19) or 9 (D2Q9, u_z = 0).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "rlb_node.cuh"

namespace {
using namespace rlb;

// f = f^eq, g = g^eq of the given FP64 fields; flags invalid input nodes.
template <typename S, int Q = 19>
__global__ void k_init(S* __restrict__ lat, unsigned long long nodes, const double* __restrict__ e,
                       const double* __restrict__ ux, const double* __restrict__ uy, const double* __restrict__ uz,
                       const double* __restrict__ n, unsigned long long* __restrict__ bad) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nodes;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const double ei = e[i], xi = ux[i], yi = uy[i], zi = uz[i], ni = n[i];
    const double u2 = xi * xi + yi * yi + zi * zi;
    if (!(ei > 0.0) || !(ni > 0.0) || !(u2 < 1.0) || !isfinite(ei) || !isfinite(ni) || (Q == 9 && zi != 0.0)) {
      atomicMin(bad, i);
      continue;
    }
    double f[Q], g[Q];
    if constexpr (Q == 19) node_equilibrium(ei, xi, yi, zi, ni, f, g);
    else node_equilibrium_d2q9(ei, xi, yi, ni, f, g);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      lat[(unsigned long long)a * nodes + i] = (S)f[a];
      lat[((unsigned long long)Q + a) * nodes + i] = (S)g[a];
    }
  }
}

// Moments of the stored populations of node i (Eq. 10), FP64.
template <typename S, int Q = 19>
__device__ __forceinline__ void stored_moments(const S* __restrict__ lat, unsigned long long nodes,
                                               unsigned long long i, NodeMacro& m) {
  S f[Q], g[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    f[a] = lat[(unsigned long long)a * nodes + i];
    g[a] = lat[((unsigned long long)Q + a) * nodes + i];
  }
  if constexpr (Q == 19) {
    double sp[9], dp[9], Sa, Sd;
    node_moments<S>(f, g, sp, dp, Sa, Sd, m);
  } else {
    double dp[4], Sa, Sd;
    node_moments_d2q9<S>(f, g, dp, Sa, Sd, m);
  }
}

template <typename S, int Q = 19>
__global__ void k_fields(const S* __restrict__ lat, unsigned long long nodes, double* __restrict__ e,
                         double* __restrict__ P, double* __restrict__ ux, double* __restrict__ uy,
                         double* __restrict__ uz, double* __restrict__ n, unsigned long long* __restrict__ bad) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nodes;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    NodeMacro m;
    stored_moments<S, Q>(lat, nodes, i, m);
    node_recover(m);
    if (m.bad) atomicMin(bad, i);
    e[i] = 3.0 * m.P;
    P[i] = m.P;
    ux[i] = m.ux;
    uy[i] = m.uy;
    uz[i] = m.uz;
    n[i] = m.N0 * sqrt(1.0 - m.u2);
  }
}


inline int grid_for(size_t nodes) {
  size_t b = (nodes + 255) / 256;
  return (int)(b < 152 * 32 ? (b ? b : 1) : 152 * 32);
}

}  // namespace
