// Library-internal declarations: the context and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/esplit.h"

namespace esplit {

constexpr int MAX_NP = 80;

// row length of the float32 path's staged operators: the smallest multiple of
// 4 (one 16-byte load) not below n_p whose number of 16-byte chunks is odd, so
// that 8 consecutive rows fall in 8 different bank groups
__host__ __device__ constexpr int npp_for(int np) {
  return ((np + 3) / 4 % 2 == 1) ? (np + 3) / 4 * 4 : (np + 3) / 4 * 4 + 4;
}
constexpr int MAX_SLOT = 64;

// Reference-operator tables every kernel reads (constant memory).
struct RefTables {
  int n_p, n_fac, n_f, n_slot;
  int slot_node[MAX_SLOT];  // volume node of facet slot
  int node_slot[MAX_NP];    // facet slot of volume node, -1 for interior nodes
  double H[MAX_NP];         // reference norm
};

// Device-resident state of the relaxation root solve (Eq. (97)).
struct RootState {
  double S0, Sabs, est;      // 1^T H s(u_n), 1^T H |s(u_n)|, dt sum b_i e_i
  double g, ga, gb, lo, hi, flo, fhi;  // ga, gb: next evaluation points (gb < 0: one point)
  double f_last, df_last, dS_last;
  double dg_last;             // previous Newton step (0: none yet)
  int phase, done, iters, status;
  unsigned int arrivals;      // blocks of the running evaluation pass that are done
};

struct Buffers {
  // operators
  double* Qref = nullptr;      // [d][n_p][n_p]
  // mesh
  double* J = nullptr;         // [n_e][n_p]
  double* nu = nullptr;        // [n_e][n_slot][d]
  int* pair = nullptr;         // [n_e][n_slot][2]
  double* Lam = nullptr;       // [n_e][d][d][n_p]
  int2* face_pairs = nullptr;  // [n_pairs] (k*n_slot+s, v*n_slot+s') with owner k
  // per-element split/derivative operators, transposed ([k][n][m]):
  //   k <  d: M_i^T, M_i = H^-1 (Q_x_i/(beta+1) + Q_x_i^T)
  //   k >= d: D_i^T, D_i = H^-1 Q_x_i
  double* ops64 = nullptr;     // [n_e][2d][n_p][n_p]
  float* ops32 = nullptr;      // same, float (nearest)
  float* ops32lo = nullptr;    // same, float remainder ops64 - ops32 (compensated FP32-bulk contractions)
  double* rows = nullptr;      // [n_e][2d][n_p] row sums of the ops64 matrices
  float* ihf = nullptr;        // [n_e][n_p] 1/(H_ref J), float32 (the float32 path's facet scaling)
  double* ihd = nullptr;       // [n_e][n_p] 1/(H_ref J) (the float64 facet kernels' scaling)
  double* nscale = nullptr;    // [n_e][n_slot][d + 1] |nu|, nu/|nu| of every facet slot
  // the D_i of ops32 again, as rows: [e][i][m][n] with n padded to
  // npp_for(n_p) (zeros), each element padded to opsD_stride floats (a
  // multiple of 4), so that a block's elements are one contiguous, aligned
  // range for a bulk copy into shared memory and a thread reads its row 4
  // entries at a time (float32 path, d <= 2)
  float* opsD32 = nullptr;     // [n_e][opsD_stride]
  // element lists for the hybrid scheme (capacity n_e each), the flags they
  // come from, and the detector's scratch (unwidened flags, block counts + total)
  int* list_split = nullptr;
  int* list_had = nullptr;
  unsigned char* hflags = nullptr;
  unsigned char* hflag0 = nullptr;
  int* hcount = nullptr;
  // scratch
  double* sat = nullptr;       // [n_e][n_c][n_slot] facet contributions
  double* fcache = nullptr;    // [d + 9][n_e n_slot] facet-node quantities (split volume -> facet kernel)
  double* partial = nullptr;   // block partial sums
  double* scal = nullptr;      // small device scalars
  RootState* root = nullptr;
  int* status = nullptr;       // sticky error flag
  // RRK work arrays [n_e][n_c][n_p]
  double* stage_u = nullptr;
  double* stage_r = nullptr;
  double* dacc = nullptr;
  double* node_cache = nullptr;  // [3][n_e n_p]: s, 1/rho, 1/p of u_n
  // viscous scratch: nodal F^V [n_e][d][n_c][n_p], facet jump terms
  // [n_e][n_c][n_slot] and lift vectors a_j [n_e][d][n_c][n_slot]
  double* fv = nullptr;
  double* vsat = nullptr;
  double* va = nullptr;
  double* wslot = nullptr;  // [n_e][n_c][n_slot]: entropy variables at the facet slots, written by
                            // the viscous split kernel for the flux-jump kernel's entropy production
  // viscous reverse-mode scratch: [n_e][d][n_c][n_p], [n_e][d][n_c][n_slot], [n_e][n_c][n_slot]
  double* vfb = nullptr;
  double* vfs = nullptr;
  double* vus = nullptr;
  double* vjp_work = nullptr;    // 12 state-sized arrays for the RRK step reverse
  // boundary facet slots (pair (-1, -1)) and their exterior states [n_b][n_c]
  int* bslot = nullptr;
  double* bstate = nullptr;
  double* host_u = nullptr;    // device copies for the host-buffer entry point
  double* host_r = nullptr;
};

}  // namespace esplit

namespace esplit {
struct ProfRec {
  int group;
  cudaEvent_t a, b;
};
}  // namespace esplit

// one relaxation RK4 step recorded as a CUDA graph (stages, reductions, the
// root solve as a device-side while loop, the update and the step record),
// valid for one state pointer, dt and configuration version
struct StepGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double* u = nullptr;
  double dt = 0.0;
  unsigned long long version = 0;
  long long kernels = 0;  // kernel launches per step outside the root loop
};

struct esplit_ctx {
  int dim = 2, device = 0, n_c = 4;
  int n_p = 0, n_fac = 0, n_f = 0, n_slot = 0;
  int n_e = 0, n_pairs = 0;
  int n_split = 0, n_had = 0;
  int n_bslot = 0;                 // boundary facet slots of the mesh
  int opsD_stride = 0;             // floats per element in b.opsD32
  bool have_bstate = false;        // their exterior states are set
  std::vector<int> bslots;         // flat slot indices (element * n_slot + slot), ascending
  bool have_op = false, have_mesh = false, ops_beta_valid = false;
  double ops_beta = 0.0;
  esplit_params prm{};
  esplit::RefTables ref{};
  esplit::Buffers b;
  size_t partial_cap = 0;
  std::vector<unsigned char> flags;
  std::string err;
  long long launches = 0;
  // set by the relaxation step around its first stage residual: the split
  // volume kernel then also writes the entropy of u_n (node cache + block
  // partials of H s, H |s| at ent_part) and reports its block count in ent_n
  double* ent_part = nullptr;
  int ent_n = 0;
  cudaStream_t last_stream = nullptr;
  // bumped by every change that alters what a step launches (operator, mesh,
  // parameters, hybrid flags); a recorded step graph of another version is stale
  unsigned long long version = 1;
  StepGraph sg;
  cudaStream_t cap_s = nullptr, cap_s2 = nullptr;  // capture streams (non-blocking)
  // side stream of the relaxation step on the float32 path: the float64
  // entropy of u_n runs there beside the stages (fork and join events)
  cudaStream_t side_s = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void* hist = nullptr;                            // StepRecord[HIST_CAP] + int counter
  bool prof = false;
  std::vector<esplit::ProfRec> recs;
  std::vector<cudaEvent_t> pool;
};

namespace esplit {

// Brackets one kernel launch with CUDA events on its stream when the
// context's profiling is enabled (groups listed in include/esplit.h).
enum ProfGroup { PG_FACE = 0, PG_SPLIT = 1, PG_HAD = 2, PG_ENTROPY = 3, PG_ROOT = 4, PG_STAGE = 5, PG_VISC = 6 };
// set by the calling thread around launches that must create no CUDA event
// (the no-allocation residual); other threads' launches on the same context
// keep their timing
extern thread_local bool t_no_events;
struct ProfScope {
  esplit_ctx* c;
  int g;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(esplit_ctx* c_, int g_, cudaStream_t s_);
  ~ProfScope();
};

// launchers (kernels.cu)
int launch_build_ops(esplit_ctx* c, cudaStream_t s);
int launch_residual(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* prod_partial,
                    int* n_partial);
int launch_entropy(esplit_ctx* c, const double* u, cudaStream_t s, int* n_partial, double* cache = nullptr,
                   double* part = nullptr);
struct ReduceRegions {
  int n;
  int off[6], cnt[6], width[6];
  double* out[6];
};
int launch_reduce_regions(esplit_ctx* c, const double* partial, const ReduceRegions& R, cudaStream_t s);
int launch_entropy_rate(esplit_ctx* c, const double* u, const double* r, cudaStream_t s, int* n_partial,
                        double* part = nullptr, int width = 2);
int launch_viscous_vjp(esplit_ctx* c, const double* u, const double* cot, double* grad, cudaStream_t s);
int launch_reduce(esplit_ctx* c, const double* partial, int n_partial, int width, double* out, cudaStream_t s);
int launch_axpy(esplit_ctx* c, const double* x, double a, const double* y, double* out, size_t n, cudaStream_t s);
int launch_stage(esplit_ctx* c, const double* un, const double* r, double a_dt, double b_dt, int first,
                 double* u_next, double* dacc, size_t n, cudaStream_t s);
int launch_root_start(esplit_ctx* c, double dt, cudaStream_t s);
constexpr int ROOT_CHECK_EVERY = 4;
constexpr int ROOT_EVALS_MAX = 40;
int launch_root_eval(esplit_ctx* c, const double* un, const double* d, cudaStream_t s);
int launch_root_eval_cond(esplit_ctx* c, const double* un, const double* d, cudaStream_t s,
                          cudaGraphConditionalHandle h);
// per-step summary written on the device by graph-launched step batches
struct StepRecord {
  double g, est, S0, S_after;
  double stage_rate[4];
  int iters, status;
};
int launch_step_record(esplit_ctx* c, StepRecord* hist, int* counter, int cap, cudaStream_t s);
int launch_root_apply(esplit_ctx* c, double* un, const double* d, size_t n, cudaStream_t s);
int set_ref_tables(const RefTables& t);
bool uses_f32_path(const esplit_ctx* c);  // the residual takes the float32 path (fp32.cu)
int set_ref_tables_vjp(const RefTables& t);  // the reverse-mode unit's copy (vjp.cu)
// float32 path of the inviscid split scheme (fp32.cu): its own copy of the
// reference tables, and the launcher (volume kernel, then facet kernel adding
// into r); -2 for an operator size not compiled in
int set_ref_tables_f32(const RefTables& t);
int launch_split_f32(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* prod, int* n_partial,
                     double* scratch);
int launch_residual_vjp(esplit_ctx* c, const double* u, const double* cot, double* grad, cudaStream_t s);
// static facet scratch of esplit_residual_noalloc: 2^21 doubles (16 MiB)
constexpr size_t NOALLOC_SCRATCH_DOUBLES = size_t(1) << 21;
constexpr int NOALLOC_MAX_DEVICES = 64;
int noalloc_scratch_ptr(int device, double** out);
int launch_wH(esplit_ctx* c, const double* u, double scale, double* out, cudaStream_t s);
int launch_rrk_vjp_dots(esplit_ctx* c, const double* u1, const double* d, const double* ubar1, cudaStream_t s,
                        int* n_partial);
int launch_rrk_vjp_combine(esplit_ctx* c, const double* un, const double* u1, const double* ubar1, double lam,
                           double g, double* ubar0, double* dbar, cudaStream_t s);
int launch_rrk_vjp_stage(esplit_ctx* c, const double* U, const double* r, const double* dbar,
                         const double* ubar_next, double c_d, double c_e, double c_u, double* rbar, double* extra,
                         cudaStream_t s);
int launch_residual_noalloc(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* scratch);
// boundary facets, float64 (kernels.cu): the SAT and dissipation with the
// exterior state, written to the facet scratch `out` before the volume
// kernels (add = 0) or added into the residual `out` after them (add = 1,
// with entropy-production block partials at prod when not null); returns
// the number of partials written
int launch_face_bc(esplit_ctx* c, const double* u, double* out, int add, double* prod, cudaStream_t s);
int launch_detect_hybrid(esplit_ctx* c, const double* u, double threshold, cudaStream_t s);
int launch_math_eval(int fn, const double* x, double* y, size_t n, cudaStream_t s);

}  // namespace esplit
