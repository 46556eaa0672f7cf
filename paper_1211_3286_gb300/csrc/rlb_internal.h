// rlb_internal.h -- helpers shared by the translation units of librlb (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/rlb.h"
#include "rlb_node.cuh"

// The lattice handle (opaque in the ABI).  Two lattices of f[19][nodes] then
// g[19][nodes] in the storage precision; lat[cur] holds the current state.
struct rlb_handle {
  rlb_config cfg;
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t nodes = 0;
  size_t esize = 8;
  int Q = 19;                                      // links per distribution: 19 (D3Q19) or 9 (D2Q9)
  void* lat[2] = {nullptr, nullptr};
  int cur = 0;
  unsigned long long* d_bad = nullptr;   // smallest non-physical node index, ULLONG_MAX if none
  double* d_part = nullptr;              // reduction partials
  double* d_stage = nullptr;             // 6 x nodes FP64 staging for host field I/O
  double* d_macro = nullptr;             // 6 x nodes FP64 fields for the C_7 gradients (RLB_CORR_C7*)
  rlb::StepConst k{};
  long long steps = 0;
  std::string err;
  void* adj_plan = nullptr;                       // cached adjoint buffers and graph (rlb_adjoint)
  void (*adj_free)(void*) = nullptr;              // its destructor
};


namespace rlb {
// Checks the relaxation times of a problem statement (every tau > 0.5, tau_q <= 0
// meaning tau_v); returns RLB_OK or RLB_EINVAL with the reason in `why`.
int validate_taus(double tau_f, double tau_v, double tau_e, double tau_eps, double tau_q, int collision,
                  std::string& why);
// Records the message that rlb_last_error(NULL) returns (calls that take no handle).
void set_handleless_error(const std::string& msg);
// Enqueue `nsteps` fused steps of h on stream s (no validation); returns the launch status.
cudaError_t enqueue_steps(rlb_handle* h, int nsteps, cudaStream_t s);
}  // namespace rlb
