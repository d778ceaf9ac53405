/*
 * esplit -- entropy-split SBP-SAT residual of the Euler / compressible
 * Navier-Stokes equations on curved periodic simplex meshes, for one GB300
 * (sm_103a).  Plain C ABI: host or device pointers and sizes only.
 *
 * Method: Worku & Zingg, "Entropy-split multidimensional summation-by-parts
 * discretization of the Euler and compressible Navier-Stokes equations".
 * Equation numbers below are the paper's.
 *
 * Conventions shared by every call
 *   d      spatial dimension (1, 2 or 3), n_c = d + 2 components
 *   state  u: float64 conservative variables [rho, rho V_1..V_d, e],
 *          layout [n_e][n_c][n_p] (element-major, node fastest)
 *   all pointers named *_dev are device pointers owned by the caller;
 *   *_host pointers are host pointers owned by the caller; the library copies
 *   what it keeps.  Calls taking a stream enqueue work on that stream
 *   (cudaStream_t passed as void*, NULL = legacy default stream) and return
 *   before it finishes unless stated otherwise.
 *   Every call returns ESPLIT_OK (0) or a negative code; the message of the
 *   last failure is available from esplit_last_error().
 */
#ifndef ESPLIT_H
#define ESPLIT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ESPLIT_OK 0
#define ESPLIT_ERR_ARG (-1)          /* bad argument (null, size, range)             */
#define ESPLIT_ERR_CUDA (-2)         /* a CUDA call failed                            */
#define ESPLIT_ERR_MESH (-3)         /* mesh rejected (pairing not an involution,
                                        J <= 0, normals of paired nodes not opposite) */
#define ESPLIT_ERR_NONPHYSICAL (-4)  /* rho <= 0, p <= 0 or a non-finite value seen   */
#define ESPLIT_ERR_RRK_NO_ROOT (-5)  /* relaxation parameter not bracketed            */
#define ESPLIT_ERR_UNSUPPORTED (-6)  /* operator size / dimension not compiled in     */
#define ESPLIT_ERR_STATE (-7)        /* call order (e.g. residual before mesh upload) */

#define ESPLIT_FP64 0       /* everything in float64                               */
#define ESPLIT_FP32_BULK 1  /* entropy-split volume term: operator contractions as
                               compensated float32 dot products (Dot2) on the
                               variations inside each element, fluxes, entropy
                               variables and A~_i products in float64 (accuracy of
                               the float64 path to ~1e-12); facet terms, viscous
                               terms, entropy functionals and the relaxation root
                               solve in float64.  Hadamard forms: their two-point
                               fluxes in plain float32                              */
#define ESPLIT_FP32 2       /* entropy-split scheme, inviscid, lines and
                               triangles: fluxes, entropy
                               variables, A~_i products, two-point fluxes,
                               dissipation and operator contractions in float32,
                               evaluated as deviations from float64 reference
                               states (cancellation-free rearrangements of Eqs.
                               (5), (25), (48), (69)); float64 for the state
                               differences, the residual's accumulation, the
                               entropy-production sums, the metric operators (formed
                               in float64, rounded once) and the relaxation step.
                               Max-norm error <= 1e-5 relative per component.
                               Other schemes, the viscous terms and tetrahedra
                               (whose operator rows amplify float32 flux rounding
                               beyond that bound): as ESPLIT_FP32_BULK              */

#define ESPLIT_SCHEME_SPLIT 0     /* entropy split, Eq. (100)                       */
#define ESPLIT_SCHEME_HADAMARD 1  /* Sjogreen-Yee Hadamard form, Eq. (99)            */
#define ESPLIT_SCHEME_HYBRID 2    /* per-element choice (Thm. 4), flags below        */
#define ESPLIT_SCHEME_HADAMARD_IR 3 /* Hadamard form with the Ismail-Roe flux, the
                                     * Sec. 6 comparator (standard entropy), with
                                     * dissipation: the matrix form of Eq. (69) for
                                     * the standard entropy at the Ismail-Roe mean
                                     * state (not printed in the paper); viscous
                                     * terms: the BO SATs of Sec. 5 in the standard
                                     * entropy variables; RRK step or VJP ->
                                     * ESPLIT_ERR_UNSUPPORTED */

typedef struct esplit_ctx esplit_ctx;

typedef struct esplit_params {
  double gam;      /* ratio of specific heats (Sec. 2.2), default 1.4                */
  double beta;     /* split parameter (Sec. 6.4), alpha = -gam - beta (gam - 1)      */
  double R;        /* gas constant                                                   */
  double mu;       /* dynamic viscosity (constant)                                   */
  double Pr;       /* Prandtl number                                                 */
  int dissipation; /* 1: add the matrix interface dissipation of Eq. (69)            */
  int viscous;     /* 1: add Eqs. (83)-(85) with Baumann-Oden SATs, Eq. (96)         */
  int heat_flux;   /* 1: include the heat flux in the viscous flux                   */
  int scheme;      /* ESPLIT_SCHEME_*                                                */
  int precision;   /* ESPLIT_FP64, ESPLIT_FP32_BULK or ESPLIT_FP32                   */
} esplit_params;

typedef struct esplit_stepinfo {
  double g;            /* relaxation parameter gamma_n of Eq. (97)                  */
  double estimate;     /* dt sum_i b_i w_i^T H r_i                                  */
  double S_before;     /* 1^T H s(u_n)                                              */
  double S_after;      /* 1^T H s(u_{n+1})                                          */
  int iterations;      /* root-solve evaluations of f                               */
  int status;          /* ESPLIT_OK or the step's error code                        */
  double stage_rate[4]; /* e_i = sum_k w(U_i)^T H r_i of the four stages, Eq. (97)  */
} esplit_stepinfo;

/* Library version (major * 10000 + minor * 100 + patch). */
int esplit_version(void);

/* Test aid (no counterpart in the paper): y_dev[i] = f(x_dev[i]) for the
 * float64 elementary functions the kernels use, fn 0..3 = log, log1p, exp,
 * expm1 (the library's table-driven versions), fn 4..7 = the same functions
 * of the CUDA math library.  x_dev, y_dev: n float64 on the current device.
 * Asynchronous on `stream`; ESPLIT_ERR_ARG for fn outside 0..7. */
int esplit_math_eval(int fn, const double* x_dev, double* y_dev, size_t n, void* stream);

/* Measurement aid (no counterpart in the paper): arithmetic throughput of
 * CUDA device `device`; mode 0 is the peak that the float64 kernels'
 * roofline fractions are taken against (those kernels are bound by the
 * float64 pipe), modes 1-6 the evidence for how they spend it.
 *   mode 0: independent float64 FMA chains, 8 per thread, 2048 threads per SM;
 *   mode 1: independent chains of the float64 tensor-core MMA (mma.sync
 *           m8n8k4, 256 FMAs per warp instruction), 8 per warp;
 *   mode 2: both interleaved in every warp (4 MMA and 8 FMA chains);
 *   mode 3: float32 FMA chains (as mode 0);
 *   mode 4: float64 divide chains x <- a / (x + 1);
 *   mode 5: chains of the library's float64 log (x <- log x + 2.5);
 *   mode 6: chains of the library's float64 exp (x <- exp(-x));
 *   modes 7, 8: the same chains with the CUDA math library's log and exp;
 *   mode 9: chains of a float64 -> float32 -> float64 round trip and an FMA;
 *   mode 10: chains of the warp-level bf16 tensor-core MMA (mma.sync
 *           m16n8k16, float32 accumulation), 8 per warp.
 * The best of five timed launches after one warm-up, on the legacy default
 * stream.  *rate receives FLOP/s (2 per FMA) for modes 0-3 and 10 and
 * operations per second for modes 4-9, *ms (may be NULL) the launch time.
 * ESPLIT_ERR_ARG for another mode.  Synchronises the device's default
 * stream. */
int esplit_measure_fp64(int device, int mode, double* rate, double* ms);

/* Create a context on CUDA device `device` for dimension `dim` (1, 2 or 3;
 * 1: the inviscid problems of Secs. 7.1-7.2, no VJP).
 * The context owns every device copy it makes (operators, mesh, scratch).
 * Defaults: gam 1.4, beta 2.5, R 1, mu 0, Pr 0.71, split scheme, FP64,
 * no dissipation, no viscous terms, heat flux on. */
int esplit_create(esplit_ctx** out, int dim, int device);
void esplit_destroy(esplit_ctx* ctx);

/* Reference diagonal-E SBP operator (Def. 1; diagonal H and E, Sec. 2.1).
 *   H_ref        [n_p]               diagonal norm (quadrature weights), > 0
 *   Q_ref        [d][n_p][n_p]       Q_xi_j, row-major
 *   facet_nodes  [n_fac][n_f]        volume node of each facet slot; every
 *                                    facet node belongs to exactly one slot
 *   facet_w      [n_fac][n_f]        facet quadrature weights (unused by the
 *                                    residual; kept for diagnostics)
 *   ref_normals  [n_fac][d]          outward unit normals of reference facets
 * Host pointers, copied.  Supported (d, n_p): (1, 2..5) (Gauss-Lobatto-
 * Legendre, p = 1..4), (2, 7), (2, 12), (2, 18),
 * (2, 27) (triangles, p = 1..4) and (3, 12), (3, 25), (3, 58), (3, 78)
 * (tetrahedra, p = 1..4); others -> ESPLIT_ERR_UNSUPPORTED. */
int esplit_upload_operator(esplit_ctx* ctx, int n_p, int n_fac, int n_f, const double* H_ref,
                           const double* Q_ref, const int* facet_nodes, const double* facet_w,
                           const double* ref_normals);

/* Curved mesh (Sec. 2.1 conforming meshes): periodic, or with boundary facets.
 *   J      [n_e][n_p]               mapping Jacobian at the nodes, > 0
 *   Lambda [n_e][d][d][n_p]         Lambda_ij = J dxi_j/dx_i at the nodes
 *   nu     [n_e][n_fac][n_f][d]     scaled outward normal b n at facet slots
 *                                   (the diagonal of E_x_i, Eq. (2))
 *   pair   [n_e][n_fac][n_f][2]     (neighbour element, neighbour flat slot),
 *                                   or (-1, -1) for a boundary facet slot
 *   hmin   [n_e]                    smallest node distance (may be NULL)
 * Host pointers, copied.  Validation: pair restricted to the other slots is
 * an involution, nu of paired slots are opposite (relative 1e-10), boundary
 * slots have a nonzero nu, J > 0; else ESPLIT_ERR_MESH.  A mesh with
 * boundary slots needs their exterior states (esplit_set_boundary_states)
 * before a residual.  The per-element physical operators Q_x_i = 1/2 sum_j
 * (Lam_ij Q_xi_j - Q_xi_j^T Lam_ij) + 1/2 E_x_i are formed on the device
 * here. */
int esplit_upload_mesh(esplit_ctx* ctx, int n_e, const double* J, const double* Lambda,
                       const double* nu, const int* pair, const double* hmin);

/* Exterior states of the boundary facet slots (bounded domains, e.g. the
 * shock tubes of Secs. 7.1-7.2; the paper's analysis is periodic and it does
 * not print its boundary treatment).  A boundary slot takes the interface
 * terms of an interior one -- the EC SAT of Eq. (43) with the two-point flux
 * of the scheme and, when on, the dissipation of Eq. (69) -- with the
 * neighbour's state replaced by its exterior state u_b (weak imposition of
 * the boundary data through the interface coupling; a supersonic inflow
 * state, or the undisturbed outer state at an outflow).
 *   slots  [n_b]        flat slot indices element * n_slot + slot, each a
 *                       boundary slot of the mesh, each given once
 *   states [n_b][n_c]   conservative exterior states (rho > 0, p > 0)
 * n_b must equal the mesh's number of boundary slots.  Host pointers,
 * copied; ESPLIT_ERR_ARG otherwise.  Inviscid only: a residual with viscous
 * terms on such a mesh, and the reverse-mode calls, return
 * ESPLIT_ERR_UNSUPPORTED. */
int esplit_set_boundary_states(esplit_ctx* ctx, int n_b, const int* slots, const double* states);

/* Parameters (host struct, copied).  Changing beta re-forms the stored
 * split operators. */
int esplit_set_params(esplit_ctx* ctx, const esplit_params* params);
int esplit_get_params(esplit_ctx* ctx, esplit_params* params);

/* Hybrid flags for ESPLIT_SCHEME_HYBRID (Thm. 4): flags_host[n_e], 0 = entropy
 * split volume term, 1 = Hadamard volume term.  Host pointer, copied. */
int esplit_set_hybrid_flags(esplit_ctx* ctx, const unsigned char* flags_host, int n_e);

/* Semi-discrete residual du/dt of Eq. (100) (split), Eq. (99) (Hadamard) or
 * the hybrid, with the EC SATs of Eq. (43) and, per the parameters, the
 * dissipation of Eq. (69) and the viscous terms of Eqs. (83)-(85).
 *   u_dev    [n_e][n_c][n_p] float64, device, read only
 *   dudt_dev [n_e][n_c][n_p] float64, device, written
 * Asynchronous on `stream`.  A non-physical node (rho <= 0, p <= 0,
 * non-finite) sets the context status ESPLIT_ERR_NONPHYSICAL, read with
 * esplit_get_status(). */
int esplit_residual(esplit_ctx* ctx, const double* u_dev, double* dudt_dev, void* stream);

/* The residual of esplit_residual for callers that must not allocate device
 * memory while they run: for example a host application whose device memory
 * is owned by its own pool allocator, or a time-critical loop that cannot
 * absorb the device-wide synchronisation cudaMalloc and cudaFree can cause.
 * This call allocates nothing -- no cudaMalloc, cudaFree, library allocator or
 * CUDA event (kernel timing, when enabled on the context, skips its launches)
 * -- and does not use the context's facet scratch: the facet contributions go
 * to a 16 MiB scratch array (2^21 doubles) that the library holds in static
 * device memory on every GPU that loads it, until the process exits.  Meshes
 * needing more than that, n_e * n_c * n_slot > 2^21, are rejected with
 * ESPLIT_ERR_ARG and a message giving both numbers.  The first call on a
 * device looks up the array's device address (with that device current) and
 * keeps it for the life of the process; make that first call before any
 * stream capture.  The address belongs to the device's primary context (the
 * one the CUDA runtime and PyTorch use): calling from another driver context,
 * or after cudaDeviceReset, is not supported (start a new process).  Every
 * call on a device shares the one array and overwrites all of the part it
 * uses (nothing has to start at zero), so calls whose kernels overlap on the
 * GPU -- on different streams, or from different threads or contexts -- race
 * on it: serialise them.  With viscous terms on, their scratch is the
 * context's own, allocated by esplit_set_params or esplit_upload_mesh when the
 * terms were switched on, not by this call.  Arguments, layout and errors as
 * for esplit_residual.  The facet terms take the kernel order in which the
 * facet kernel runs before the volume kernels (esplit_residual runs the
 * volume kernels first for the inviscid split scheme), so the result equals
 * esplit_residual's to rounding: within the float64 parity tolerance, or the
 * stated bound of a float32 precision setting.  The paper has no counterpart
 * of this entry point; it is a deployment convenience. */
int esplit_residual_noalloc(esplit_ctx* ctx, const double* u_dev, double* dudt_dev, void* stream);

/* Hybrid scheme (Sec. 4.4, Thm. 4): flags for the hybrid scheme computed on
 * the device from the state u_dev ([n_e][n_c][n_p] float64).  The paper
 * leaves the choice of troubled elements open; this detector flags element k
 * when, over the nodes of k and the neighbours' facet nodes coincident with
 * the facet nodes of k, max p / min p > threshold or a pressure there is not
 * positive and finite, p = (gam-1)(e - (0.5 |m|^2)/rho) evaluated in that
 * order in round-to-nearest float64; then every face neighbour of a flagged
 * element is flagged as well.  The flags replace those of
 * esplit_set_hybrid_flags and are used by every later residual of the hybrid
 * scheme (an RRK step keeps them for all four stages: call this before each
 * step to re-detect).  threshold: finite, >= 1 (ESPLIT_ERR_ARG otherwise).
 * *n_flagged (may be NULL) receives the number of flagged elements.
 * Synchronises `stream`. */
int esplit_detect_hybrid(esplit_ctx* ctx, const double* u_dev, double threshold, int* n_flagged, void* stream);

/* Copies the current hybrid flags (uint8, 0 or 1, [n_e]) to flags_host, from
 * esplit_set_hybrid_flags or the last esplit_detect_hybrid.  ESPLIT_ERR_STATE
 * when neither has run since the mesh upload.  Synchronises. */
int esplit_get_hybrid_flags(esplit_ctx* ctx, unsigned char* flags_host);

/* Same with host buffers: copies u_host to the device, evaluates, copies the
 * residual back, and synchronises `stream` before returning. */
int esplit_residual_host(esplit_ctx* ctx, const double* u_host, double* dudt_host, void* stream);

/* 1^T H s(u) with Harten's entropy, Eq. (16), in float64 (synchronises). */
int esplit_entropy(esplit_ctx* ctx, const double* u_dev, double* S_total, void* stream);

/* sum_k w_k^T H_k dudt_k (the rate of Thm. 2), float64 (synchronises). */
int esplit_entropy_rate(esplit_ctx* ctx, const double* u_dev, const double* dudt_dev,
                        double* rate, void* stream);

/* One relaxation RK4 step, Sec. 6.1, Eqs. (97)-(98): classical RK4 stages,
 * relaxation parameter g by a bracketed Newton iteration on the device to
 * round-off, u <- u + g dt sum_i b_i r_i.  u_dev is updated in place (left
 * untouched on failure).  Synchronises `stream` at the end; g and the step
 * summary are returned through g_out / info (either may be NULL). */
int esplit_rrk_step(esplit_ctx* ctx, double* u_dev, double dt, double* g_out, esplit_stepinfo* info,
                    void* stream);

/* n_steps relaxation RK4 steps of Sec. 6.1 with the same dt, without a host
 * round trip between steps (no counterpart in the paper: a launch-latency
 * measure for small meshes).  Each step makes exactly the launches of
 * esplit_rrk_step, so u_dev ends bit-identical to n_steps calls of it; the
 * step is recorded once as a CUDA graph (the root solve as a device-side
 * while loop) for this u_dev pointer, dt and configuration, and re-recorded
 * when any of them changes, the first step of a new recording running the
 * ordinary way.  With profiling on, the steps run one by one.
 *   g_out: n_steps doubles (host, may be NULL), each step's g.
 *   info:  the summary of the last step run (host, may be NULL).
 *   n_done: the number of completed steps (host, may be NULL).
 * Hybrid flags and parameters stay as they are for the whole batch.  On a
 * failing step (ESPLIT_ERR_NONPHYSICAL, ESPLIT_ERR_RRK_NO_ROOT) u_dev holds the
 * state after the last completed step: the failing step and the rest of the
 * batch, which still run, leave it unchanged.  Synchronises `stream` once per
 * 1024 steps and at the end. */
int esplit_rrk_steps(esplit_ctx* ctx, double* u_dev, double dt, int n_steps, double* g_out,
                     esplit_stepinfo* info, int* n_done, void* stream);

/* Same step with a host state: copies u_host (pinned or pageable) to the
 * device, steps, copies the new state back, and synchronises `stream`. */
int esplit_rrk_step_host(esplit_ctx* ctx, double* u_host, double dt, double* g_out, esplit_stepinfo* info,
                         void* stream);

/* Reverse mode of the residual: grad_dev = (d dudt / d u)^T cot_dev, for the
 * entropy-split scheme (Eq. (100)) with the EC SATs, the interface
 * dissipation of Eq. (69) and, when on, the viscous BO terms of Eqs.
 * (83)-(85), (96); float64 whatever the precision setting.  Other schemes:
 * ESPLIT_ERR_UNSUPPORTED.  u_dev, cot_dev, grad_dev: [n_e][n_c][n_p]
 * float64 device buffers; grad_dev must not alias the others. */
int esplit_residual_vjp(esplit_ctx* ctx, const double* u_dev, const double* cot_dev,
                        double* grad_dev, void* stream);

/* Gradient of the total entropy 1^T H s(u) (Eq. (16)): grad_dev = H w(u),
 * w the entropy variables of Eq. (25).  [n_e][n_c][n_p] device buffers. */
int esplit_entropy_grad(esplit_ctx* ctx, const double* u_dev, double* grad_dev, void* stream);

/* Reverse of one relaxation RK4 step (Eqs. (97)-(98)) for gradients through
 * many steps with per-step checkpoints: recomputes the step from the
 * checkpoint u_dev (unchanged), then maps the cotangent ubar_next_dev of
 * u_{n+1} to the cotangent ubar_dev of u_n, including the dependence of the
 * relaxation parameter on the state through the implicit function theorem
 * (dg = -(f_u du + f_d dd + f_est dest)/f_g).  Entropy-split scheme (with or
 * without dissipation and viscous terms).  Scratch: 12 state-sized device arrays owned
 * by the context, allocated on the first call.  Synchronises `stream`; the
 * step's g is returned through g_out (may be NULL). */
int esplit_rrk_step_vjp(esplit_ctx* ctx, const double* u_dev, double dt, const double* ubar_next_dev,
                        double* ubar_dev, double* g_out, void* stream);

/* Sticky status of asynchronous work (synchronises the context's last
 * stream): ESPLIT_OK, ESPLIT_ERR_NONPHYSICAL, or ESPLIT_ERR_CUDA when a
 * kernel's bounded wait for its shared-memory staging (bulk copy) ran out --
 * its result was then computed from global memory; reading clears it. */
int esplit_get_status(esplit_ctx* ctx);

/* Message of the last failure on this context (static storage of ctx). */
const char* esplit_last_error(esplit_ctx* ctx);

/* Number of kernels this context has launched so far (for accounting). */
long long esplit_launch_count(esplit_ctx* ctx);

/* Kernel timing: when enabled, every kernel launch of the context is
 * bracketed by CUDA events on its own stream.  Groups:
 *   0 facet kernel (EC SAT + dissipation)   1 entropy-split volume kernel
 *   2 Hadamard volume kernel                3 entropy functionals + reductions
 *   4 relaxation root solve                 5 RK stage / update kernels
 *   6 viscous terms (three kernels)
 * esplit_profile_read synchronises, fills ms[g] (total milliseconds) and
 * count[g] (launches) for g < n_groups, and resets the accumulators. */
#define ESPLIT_PROFILE_GROUPS 7
int esplit_profile_enable(esplit_ctx* ctx, int on);
int esplit_profile_read(esplit_ctx* ctx, double* ms, long long* count, int n_groups);

#ifdef __cplusplus
}
#endif

#endif /* ESPLIT_H */
