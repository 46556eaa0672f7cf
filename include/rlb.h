/*
 * rlb.h -- C ABI of librlb, a GB300 (sm_103a) implementation of the relativistic
 * lattice Boltzmann (RLB) scheme analysed by Li, Luo & Li, "Lattice Boltzmann
 * method for relativistic hydrodynamics: issues on conservation law of particle
 * number and discontinuities" (arXiv 1211.3286).
 *
 * The library advances two D3Q19 distribution sets on one GPU:
 *   f_a  (particle number N^mu, BGK relaxation, Eq. 5, equilibrium Eq. 7),
 *   g_a  (energy-momentum T^{mu nu}, BGK Eq. 6 or MRT Eqs. 30-35, equilibria Eqs. 8-9),
 * with the macroscopic fields recovered per node from Eq. 10 under the
 * ultrarelativistic equation of state P = e/3 (closed form, no iteration):
 *   sigma = (2 T00 + sqrt(4 T00^2 - 3 |M|^2)) / 3,  u = M / sigma,  P = sigma - T00,
 *   e = 3 P,  gamma = 1 / sqrt(1 - u^2),  n = N0 / gamma,
 * where N0 = sum f, T00 = sum g, M = sum e_a g_a.
 *
 * Conventions shared by every call
 *   - All entry points are extern "C", return an int status (RLB_OK = 0 on
 *     success) unless stated, and never throw.  On failure the handle's
 *     rlb_last_error() string says why.
 *   - Lattices are x-fastest: field arrays hold nx*ny*nz values indexed
 *     (z*ny + y)*nx + x.  The quasi-1D tube is {nx = L, ny = 1, nz = 1}.
 *   - Pointers tagged RLB_HOST are ordinary host memory; RLB_DEVICE pointers are
 *     device memory of the handle's GPU (for example a torch tensor's data_ptr()).
 *     The library never keeps a caller's pointer past the call.
 *   - Calls that launch work are asynchronous on the configured stream unless
 *     they say they synchronise.  Device-side detection of a non-physical state
 *     (4 T00^2 - 3|M|^2 < 0, T00 <= 0, e <= 0, |u| >= 1 or NaN) is reported by
 *     the next synchronising call as RLB_ENONPHYS, with the first bad node index
 *     in rlb_last_error().
 *   - The library owns the device lattices it allocates in rlb_create and frees
 *     them in rlb_destroy.
 */
#ifndef RLB_H
#define RLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RLB_OK        0
#define RLB_EINVAL    1  /* invalid argument or non-physical input field */
#define RLB_ENOMEM    2  /* device or host allocation failed */
#define RLB_ECUDA     3  /* a CUDA runtime call failed */
#define RLB_ENONPHYS  4  /* the device flagged a non-physical node during stepping */
#define RLB_ETIMEOUT  5  /* reserved for a bounded device-side wait that gives up; no kernel of this
                             library waits on another CTA or device, so no call returns it */

/* lattice, equation of state, collision, boundary, precision, memory space */
#define RLB_D3Q19               19
#define RLB_D2Q9                 9   /* the MRT model of Sec. V.A (Eqs. 30-35): nz = 1, RLB_FP64 */
#define RLB_EOS_ULTRAREL         1   /* P = e / 3 */
#define RLB_BGK                  0   /* Eq. 6 for g */
#define RLB_MRT                  1   /* Eqs. 30-35 (D3Q19 moment basis) for g */
#define RLB_PERIODIC             0
#define RLB_ZERO_GRADIENT        1   /* "open" end: a pull from outside takes the edge node */
#define RLB_FP64                 0   /* populations stored in FP64; the step runs in 64-bit block fixed point
                                        (every value on the grid of its node's largest: 2^-56 of it; the
                                        recovery's root and reciprocal to ~2^-58), rounded once to FP64 per
                                        link; the output fields are recovered in FP64 */
#define RLB_FP32_STORAGE         1   /* populations stored in FP32; conservation sums exact, recovery
                                        in FP64 arithmetic (one Newton step on sigma's quadratic from
                                        an FP32 seed, ~2^-40), gamma in FP64; per-link work in FP32 */
#define RLB_CORR_NONE            0
#define RLB_CORR_C7              1   /* Eq. 37 with C_7 of Eq. 38 on the m_7 = p_xx moment; its theta term
                                        with the coefficient 1 of Eq. A17 */
#define RLB_CORR_C7_PRINTED      2   /* the same with Eq. 38's theta term as printed (coefficient 2) */
#define RLB_HOST                 0
#define RLB_DEVICE               1

/*
 * Problem statement of one lattice: the lattice with c = dx/dt = 1 (Sec. III.B),
 * the EOS, the relaxation times tau_f (Eq. 5), tau_v / tau_e / tau_eps / tau_q
 * (the MRT rates of Eq. 31 and Sec. V.B), the boundary type per axis and the
 * storage precision.
 *   tau_f    relaxation time of f (BGK).  Must be > 0.5.
 *   tau_v    shear time; also the single g time under RLB_BGK.  > 0.5.
 *   tau_e    bulk (energy moment) time, MRT only.  > 0.5.
 *   tau_eps  energy-square moment time, MRT only.  > 0.5.
 *   tau_q    energy-flux moment time, MRT only; <= 0 means tau_q = tau_v.
 *   stream   a cudaStream_t (NULL = legacy default stream) on which all work of
 *            this handle is enqueued.
 *   correction  RLB_CORR_C7 adds the error-correction term of Eqs. 37-38 to the
 *            D2Q9 MRT collision: m* = m - S (m - m^eq) + (1 - s_7/2) C_7 e_7 on the
 *            moment m_7 = sum (c_x^2 - c_y^2) g (m^eq_7 = sigma (u_x^2 - u_y^2), Eq. 34),
 *            with C_7 = E_x - E_y and, for each axis a,
 *            E_a = 2 [u_a da(c_s^2 sigma - P) - c_s^2 sigma u_a da(gamma)/gamma
 *                     - u_a da(sigma u_a^2)] + k u_a^2 theta da(sigma u_a),
 *            theta = 1 + 1/((e/P + 1) gamma^2 - 1).  E_a is Eq. 38 for a flow along
 *            axis a (the paper's z); its sign in C_7 follows that axis's place in
 *            m_7, so a tube along x (the printed sign) and a tube along y (the paper's
 *            4 x 800 geometry, the opposite sign) are the same problem relabelled.
 *            k = 1 (RLB_CORR_C7, the coefficient Eq. A17 gives) or 2
 *            (RLB_CORR_C7_PRINTED, Eq. 38 as printed).  Derivatives are central
 *            differences of the fields pulled at the neighbours (a zero-gradient end
 *            reuses the edge value).  Each step then runs two kernels (fields, then
 *            the corrected collide).
 *   eta_over_s  > 0 selects the paper's fixed-eta/s relaxation (Sec. II and III.B):
 *            per node and step, tau_g = 1/2 + eta / (c_s^2 (e + P) gamma) with
 *            eta = (eta/s) s, s = 4 n - n ln(n / n_eq), n_eq = 16 T^3 / pi^2 and
 *            T = P / n; tau_v is then unused and tau_f <= 0 means tau_f = tau_g
 *            (the Fig. 1 cases); n must be given in the same units as P.  With
 *            RLB_MRT, tau_v = tau_g per node and tau_e, tau_eps, tau_q are read as
 *            the ratios a_x = (tau_x - 1/2) / (tau_v - 1/2) (Cases A-D of Sec. V.B;
 *            tau_q <= 0 means 1).
 */
typedef struct rlb_config {
  int nx, ny, nz;
  int lattice;      /* RLB_D3Q19 | RLB_D2Q9 */
  int eos;          /* RLB_EOS_ULTRAREL */
  int collision;    /* RLB_BGK | RLB_MRT */
  double tau_f, tau_v, tau_e, tau_eps, tau_q;
  int bc[3];        /* per axis x, y, z: RLB_PERIODIC | RLB_ZERO_GRADIENT */
  int precision;    /* RLB_FP64 | RLB_FP32_STORAGE */
  void* stream;
  int correction;   /* RLB_CORR_NONE | RLB_CORR_C7 | RLB_CORR_C7_PRINTED (RLB_D2Q9 + RLB_MRT only) */
  double eta_over_s; /* > 0: per-node tau_g / tau_v from eta/s (RLB_FP64); 0: constant taus */
} rlb_config;

typedef struct rlb_handle rlb_handle;

/* Allocate a lattice on the current CUDA device.  Returns RLB_EINVAL for a
 * zero or negative extent, an unknown enum, any tau <= 0.5, or RLB_D2Q9 with
 * nz != 1 or FP32 storage; RLB_ENOMEM if the two lattices (2 x 2Q x nodes x 8 or 4
 * bytes, Q = 19 or 9 links) do not fit.  *out is set only on success.
 * RLB_D2Q9 runs the D2Q9 model of Sec. V.A: rest equilibrium Eq. 32, moving links
 * Eq. 33, MRT basis of Eqs. 30-35 with S of Eq. 31 (its field arrays have u_z = 0;
 * rlb_set_fields rejects u_z != 0). */
int rlb_create(const rlb_config* cfg, rlb_handle** out);

/* Free the handle and its device memory (synchronises its stream).  NULL is a no-op. */
void rlb_destroy(rlb_handle* h);

/* Message describing the last failure on h (or on a failed rlb_create when h is
 * NULL); never NULL. */
const char* rlb_last_error(const rlb_handle* h);

/* Set the state to equilibrium of the given fields: f = f^eq(n, u) (Eq. 7),
 * g = g^eq(e, P = e/3, u) (Eqs. 8-9).  e, ux, uy, uz, n each hold nx*ny*nz FP64
 * values in `where` memory; e > 0, n > 0 and |u| < 1 are required (RLB_EINVAL
 * otherwise, state unchanged).  Synchronises. */
int rlb_set_fields(rlb_handle* h, const double* e, const double* ux, const double* uy,
                   const double* uz, const double* n, int where);

/* Advance nsteps time steps (nsteps >= 0): each step pulls f and g from x - e_a
 * (periodic axes wrap, zero-gradient axes clamp), recovers the fields from
 * Eq. 10, and relaxes f by Eq. 5 and g by Eq. 6 (BGK) or Eq. 35 (MRT).
 * Asynchronous on the handle's stream. */
int rlb_step(rlb_handle* h, int nsteps);

/* Wait for the handle's stream and report a device-flagged non-physical node
 * (RLB_ENONPHYS) since the last check; clears the flag. */
int rlb_check(rlb_handle* h);

/* Macroscopic fields of the current state (Eq. 10 plus the recovery): e, P,
 * ux, uy, uz, n, each nx*ny*nz FP64 values in `where` memory.  Any pointer may be
 * NULL to skip that field.  Synchronises and reports RLB_ENONPHYS like rlb_check. */
int rlb_get_fields(rlb_handle* h, double* e, double* P, double* ux, double* uy, double* uz,
                   double* n, int where);

/* Lattice sums of the conserved densities of the current state, in FP64 with a
 * fixed (deterministic) reduction order: out[0] = sum N0, out[1] = sum T00,
 * out[2..4] = sum M_x, M_y, M_z (the quantities Eq. A8 leaves unchanged under
 * collision).  out is host memory.  Synchronises. */
int rlb_conserved_totals(rlb_handle* h, double out[5]);

/* Number of bytes of one raw state: 2 x Q x nodes x (8 for RLB_FP64, 4 for
 * RLB_FP32_STORAGE), Q = 19 (D3Q19) or 9 (D2Q9).  Layout: f[Q][nz][ny][nx]
 * followed by g[Q][nz][ny][nx], post-collision populations of the current time step. */
size_t rlb_state_bytes(const rlb_handle* h);

/* Copy the raw state out to / in from `where` memory of rlb_state_bytes(h)
 * bytes (checkpoint and resume).  Synchronise. */
int rlb_save_state(rlb_handle* h, void* buf, int where);
int rlb_load_state(rlb_handle* h, const void* buf, int where);

/* Number of time steps taken since the last rlb_set_fields / rlb_load_state. */
long long rlb_steps_done(const rlb_handle* h);

/*
 * Conserved totals of a raw state, for callers that must not allocate.
 *
 * The paper has no counterpart of this call; it exists for callers that cannot
 * allocate device memory when they need the totals: code that has handed the
 * GPU's memory to a pool reserved at start-up (a framework's caching allocator
 * or a fixed arena) and must not allocate around it, monitoring code that reports
 * the conserved sums of a run that has just failed with out-of-memory, and
 * latency-sensitive loops in which cudaMalloc / cudaFree would stall the work by
 * synchronising the device.  It computes what rlb_conserved_totals computes
 * (sum N0, sum T00, sum M_x, sum M_y, sum M_z in FP64, fixed reduction order;
 * the order differs from rlb_conserved_totals, so the two agree to round-off)
 * but takes the state itself rather than a handle and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   state      device pointer to a raw D3Q19 state in the rlb_save_state layout
 *              (f[19][nodes] then g[19][nodes]), FP64 or FP32 per `precision`.
 *              D3Q19 states only: a D2Q9 state (f[9] g[9], from an RLB_D2Q9
 *              handle) holds 18 values per node, and passing one makes the call
 *              read past the end of the caller's buffer.
 *   nodes      lattice nodes, 1 <= nodes <= RLB_NOALLOC_MAX_NODES; larger sizes
 *              return RLB_EINVAL with the limit in rlb_last_error(NULL).
 *   precision  RLB_FP64 or RLB_FP32_STORAGE.
 *   out        5 doubles in `where` memory (RLB_DEVICE: written by a kernel on
 *              `stream`, asynchronous; RLB_HOST: copied back, the call then
 *              synchronises `stream`).
 *   stream     cudaStream_t to run on (NULL = legacy default stream).
 * Scratch: a file-scope device array of 4096 x 5 + 5 doubles (160 KiB) that every
 * GPU loading librlb holds until the process exits.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents (each call overwrites
 * every slot it reads, so nothing needs clearing); calls whose kernels overlap
 * on the GPU race on it, so serialise them (one stream, or events).  Errors are
 * reported by the return code and rlb_last_error(NULL).
 */
#define RLB_NOALLOC_MAX_NODES 268435456
int rlb_conserved_totals_noalloc(const void* state, size_t nodes, int precision, double* out, int where,
                                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RLB_H */
