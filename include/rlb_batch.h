/*
 * rlb_batch.h -- batched quasi-1D shock tubes of librlb (the relaxation-time sweep
 * of the paper's discontinuity study, Sec. V.B and Figs. 2-5 of arXiv 1211.3286).
 *
 * A batch holds T independent D3Q19 tubes of lengths L_t (nx = L_t, ny = nz = 1,
 * zero-gradient ends, periodic transverse axes), each with its own relaxation
 * times.  Every tube advances by the same fused step as rlb_step (pull stream,
 * Eq. 10 moments, closed-form recovery under P = e/3, Eqs. 7-9 equilibria, BGK f
 * by Eq. 5, BGK g by Eq. 6 or MRT g by Eqs. 30-35).  rlb_batch_run advances all
 * tubes by nsteps in ONE persistent kernel launch replayed from a CUDA graph:
 * each CTA takes whole tubes from a longest-first work list and runs all the steps
 * of a tube with CTA-local barriers (tubes never exchange data).
 *
 * Node numbering: tube t occupies the global node range [offset_t, offset_t + L_t)
 * with offset_t = L_0 + ... + L_{t-1}; field arrays of the batch are these
 * concatenated tube profiles (FP64, x along the tube).
 * Status codes, RLB_HOST / RLB_DEVICE and precision constants are those of rlb.h.
 */
#ifndef RLB_BATCH_H
#define RLB_BATCH_H

#include <stddef.h>

#include "rlb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlb_batch rlb_batch;

/*
 * ntubes     number of tubes (>= 1).
 * lengths    host array of ntubes lengths (each >= 1).
 * taus       host array of ntubes x 3 doubles (tau_v, tau_e, tau_eps) per tube,
 *            each > 0.5; tau_q = tau_v (the Case C / D convention of Sec. V.B).
 * tau_f      host array of ntubes doubles, or NULL for tau_f = tau_v.
 * collision  RLB_MRT or RLB_BGK (BGK relaxes g with tau_v).
 * precision  RLB_FP64 or RLB_FP32_STORAGE.
 * stream     cudaStream_t for all work of the batch (NULL = legacy default).
 */
typedef struct rlb_batch_desc {
  int ntubes;
  const int* lengths;
  const double* taus;
  const double* tau_f;
  int collision;
  int precision;
  void* stream;
} rlb_batch_desc;

/* Allocate a batch on the current device (two lattices of 38 x sum(L) values).
 * RLB_EINVAL for bad counts, lengths or taus; RLB_ENOMEM if it does not fit. */
int rlb_batch_create(const rlb_batch_desc* d, rlb_batch** out);
void rlb_batch_destroy(rlb_batch* b);
const char* rlb_batch_last_error(const rlb_batch* b);

/* Total nodes sum(L_t) and the offset of tube t. */
size_t rlb_batch_nodes(const rlb_batch* b);
size_t rlb_batch_offset(const rlb_batch* b, int tube);

/* Equilibrium initial state from concatenated FP64 fields (as rlb_set_fields). */
int rlb_batch_set_fields(rlb_batch* b, const double* e, const double* ux, const double* uy, const double* uz,
                         const double* n, int where);

/* Time a few launch shapes of the persistent kernel (threads per CTA x CTAs per
 * SM) on trial_steps steps of a copy of the current state, keep the fastest for
 * later rlb_batch_run calls and report it in chosen[0] (threads per CTA) and
 * chosen[1] (CTAs per SM); chosen may be NULL.  The state is left unchanged.
 * Synchronises. */
int rlb_batch_autotune(rlb_batch* b, int trial_steps, int* chosen);

/* Set the launch shape of later rlb_batch_run calls without timing anything (a shape
 * rlb_batch_autotune chose earlier, say): threads per CTA, a multiple of 32 up to the
 * kernel's launch bound (320 for FP32 storage, 256 for FP64), and CTAs per SM, 1 up to
 * the occupancy limit at that block size (0 = that limit).  RLB_EINVAL (state
 * unchanged) for any other value.  Results do not depend on the shape: each tube is
 * advanced by one CTA and every node's arithmetic is the same. */
int rlb_batch_set_shape(rlb_batch* b, int threads, int ctas_per_sm);

/* Advance every tube by nsteps (>= 0) in one persistent launch from a CUDA graph
 * (captured on first use for a given nsteps).  Asynchronous on the batch stream. */
int rlb_batch_run(rlb_batch* b, int nsteps);

/* Wait and report a device-flagged non-physical node (RLB_ENONPHYS, global node
 * index in the message). */
int rlb_batch_check(rlb_batch* b);

/* Concatenated fields of the current state (any pointer may be NULL).  Synchronises. */
int rlb_batch_get_fields(rlb_batch* b, double* e, double* P, double* ux, double* uy, double* uz, double* n,
                         int where);

/* Raw state (f[19][nodes] then g[19][nodes] in the storage precision) in / out. */
size_t rlb_batch_state_bytes(const rlb_batch* b);
int rlb_batch_save_state(rlb_batch* b, void* buf, int where);
int rlb_batch_load_state(rlb_batch* b, const void* buf, int where);

#ifdef __cplusplus
}
#endif
#endif /* RLB_BATCH_H */
