// C ABI of the library (declared in include/esplit.h): context, uploads,
// validation, and the host side of the residual, entropy functionals and
// relaxation RK4 step.  All arithmetic of the method runs in kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using esplit::RefTables;

namespace {

constexpr double kNuTol = 1e-10;

int fail(esplit_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(c, ESPLIT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dalloc(esplit_ctx* c, T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) return ESPLIT_OK;
  CK(cudaMalloc((void**)p, count * sizeof(T)));
  return ESPLIT_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

bool supported(int dim, int n_p) {
  if (dim == 1) return n_p >= 2 && n_p <= 5;
  if (dim == 2) return n_p == 7 || n_p == 12 || n_p == 18 || n_p == 27;
  if (dim == 3) return n_p == 12 || n_p == 25 || n_p == 58 || n_p == 78;
  return false;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int check_ready(esplit_ctx* c) {
  if (!c) return ESPLIT_ERR_ARG;
  if (!c->have_op || !c->have_mesh) return fail(c, ESPLIT_ERR_STATE, "operator and mesh must be uploaded first");
  return ESPLIT_OK;
}

// floats per element of the D_i rows the float32 path stages in shared memory:
// at least d n_p npp, a multiple of 4 (16 bytes, the bulk copy's unit), and
// among those the one that spreads a warp's 16-byte row reads (lanes =
// consecutive nodes, in consecutive elements; 8 lanes per shared-memory
// phase) over the most bank groups
int opsD_stride_for(int d, int np) {
  const int npp = esplit::npp_for(np);
  const int base = d * np * npp;
  int best = base, best_worst = 1 << 30;
  for (int s = base; s < base + 32; s += 4) {
    int worst = 0;
    for (int w0 = 0; w0 < np; ++w0) {  // node of the warp's first lane
      for (int ph = 0; ph < 4; ++ph) {
        int cnt[8] = {0};
        for (int l = 8 * ph; l < 8 * ph + 8; ++l) {
          const int e = (w0 + l) / np, m = (w0 + l) % np;
          worst = std::max(worst, ++cnt[((e * s) / 4 + m * (npp / 4)) % 8]);
        }
      }
    }
    if (worst < best_worst) {
      best_worst = worst;
      best = s;
    }
  }
  return best;
}

int ensure_partial(esplit_ctx* c) {
  size_t need = 8 * ((size_t)c->n_e * c->n_p / 256 + 1) + 4 * ((size_t)c->n_e + 64);
  if (c->partial_cap >= need) return ESPLIT_OK;
  int rc = dalloc(c, &c->b.partial, need);
  if (rc) return rc;
  c->partial_cap = need;
  return ESPLIT_OK;
}

int rebuild_ops(esplit_ctx* c, cudaStream_t s) {
  if (!c->have_op || !c->have_mesh) return ESPLIT_OK;
  if (esplit::launch_build_ops(c, s)) return fail(c, ESPLIT_ERR_CUDA, "build_ops launch failed");
  CK(cudaStreamSynchronize(s));
  c->ops_beta = c->prm.beta;
  c->ops_beta_valid = true;
  return ESPLIT_OK;
}

int read_status(esplit_ctx* c, cudaStream_t s, bool clear) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->b.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (clear && h) CK(cudaMemsetAsync(c->b.status, 0, sizeof(int), s));
  if (h & 4) return fail(c, ESPLIT_ERR_CUDA, "a kernel's wait for its shared-memory staging timed out");
  return h ? ESPLIT_ERR_NONPHYSICAL : ESPLIT_OK;
}

}  // namespace

namespace esplit {

thread_local bool t_no_events = false;

ProfScope::ProfScope(esplit_ctx* c_, int g_, cudaStream_t s_) : c(c_), g(g_), s(s_) {
  if (!c->prof || t_no_events) return;
  for (cudaEvent_t* ev : {&a, &b}) {
    if (!c->pool.empty()) {
      *ev = c->pool.back();
      c->pool.pop_back();
    } else if (cudaEventCreate(ev) != cudaSuccess) {
      *ev = nullptr;
    }
  }
  if (a) cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
  if (!a || !b) return;
  cudaEventRecord(b, s);
  c->recs.push_back(ProfRec{g, a, b});
}

}  // namespace esplit

extern "C" {

int esplit_version(void) { return 100; }

int esplit_math_eval(int fn, const double* x, double* y, size_t n, void* stream) {
  if (fn < 0 || fn > 7 || (n > 0 && (!x || !y))) return ESPLIT_ERR_ARG;
  return esplit::launch_math_eval(fn, x, y, n, (cudaStream_t)stream) ? ESPLIT_ERR_CUDA : ESPLIT_OK;
}

int esplit_create(esplit_ctx** out, int dim, int device) {
  if (!out) return ESPLIT_ERR_ARG;
  *out = nullptr;
  if (dim < 1 || dim > 3) return ESPLIT_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return ESPLIT_ERR_CUDA;
  if (device < 0 || device >= ndev) return ESPLIT_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return ESPLIT_ERR_CUDA;
  esplit_ctx* c = new esplit_ctx();
  c->dim = dim;
  c->n_c = dim + 2;
  c->device = device;
  c->prm.gam = 1.4;
  c->prm.beta = 2.5;
  c->prm.R = 1.0;
  c->prm.mu = 0.0;
  c->prm.Pr = 0.71;
  c->prm.dissipation = 0;
  c->prm.viscous = 0;
  c->prm.heat_flux = 1;
  c->prm.scheme = ESPLIT_SCHEME_SPLIT;
  c->prm.precision = ESPLIT_FP64;
  if (cudaMalloc((void**)&c->b.status, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&c->b.root, sizeof(esplit::RootState)) != cudaSuccess ||
      cudaMalloc((void**)&c->b.scal, 64 * sizeof(double)) != cudaSuccess) {
    esplit_destroy(c);
    return ESPLIT_ERR_CUDA;
  }
  cudaMemset(c->b.status, 0, sizeof(int));
  cudaMemset(c->b.scal, 0, 64 * sizeof(double));
  *out = c;
  return ESPLIT_OK;
}

void esplit_destroy(esplit_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  esplit::Buffers& b = c->b;
  void* ps[] = {b.Qref, b.J,       b.nu,      b.pair,   b.Lam,     b.face_pairs, b.ops64,   b.ops32,   b.ops32lo,
                b.list_split, b.list_had, b.hflags, b.hflag0, b.hcount, b.sat, b.fcache, b.rows, b.partial, b.scal, b.root, b.status, b.stage_u,
                b.stage_r, b.dacc, b.node_cache, b.vjp_work, b.host_u, b.host_r, b.fv, b.vsat, b.va, b.wslot, b.vfb, b.vfs, b.vus,
                b.bslot, b.bstate, b.ihf, b.opsD32, b.ihd, b.nscale};
  for (void* p : ps) dfree(p);
  if (c->sg.exec) cudaGraphExecDestroy(c->sg.exec);
  if (c->sg.graph) cudaGraphDestroy(c->sg.graph);
  if (c->cap_s) cudaStreamDestroy(c->cap_s);
  if (c->cap_s2) cudaStreamDestroy(c->cap_s2);
  if (c->side_s) cudaStreamDestroy(c->side_s);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  dfree(c->hist);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  delete c;
}

int esplit_upload_operator(esplit_ctx* c, int n_p, int n_fac, int n_f, const double* H_ref, const double* Q_ref,
                           const int* facet_nodes, const double* facet_w, const double* ref_normals) {
  if (!c) return ESPLIT_ERR_ARG;
  c->version++;
  if (!H_ref || !Q_ref || !facet_nodes) return fail(c, ESPLIT_ERR_ARG, "null operator array");
  if (n_p <= 0 || n_fac <= 0 || n_f <= 0) return fail(c, ESPLIT_ERR_ARG, "operator sizes must be positive");
  if (!supported(c->dim, n_p))
    return fail(c, ESPLIT_ERR_UNSUPPORTED, "operator size n_p=" + std::to_string(n_p) + " not compiled in");
  int n_slot = n_fac * n_f;
  if (n_slot > esplit::MAX_SLOT || n_p > esplit::MAX_NP) return fail(c, ESPLIT_ERR_UNSUPPORTED, "too many nodes");
  cudaSetDevice(c->device);
  RefTables t{};
  t.n_p = n_p;
  t.n_fac = n_fac;
  t.n_f = n_f;
  t.n_slot = n_slot;
  for (int m = 0; m < esplit::MAX_NP; ++m) t.node_slot[m] = -1;
  for (int s = 0; s < n_slot; ++s) {
    int m = facet_nodes[s];
    if (m < 0 || m >= n_p) return fail(c, ESPLIT_ERR_ARG, "facet node index out of range");
    if (t.node_slot[m] >= 0) return fail(c, ESPLIT_ERR_ARG, "a volume node belongs to two facet slots");
    t.node_slot[m] = s;
    t.slot_node[s] = m;
  }
  for (int m = 0; m < n_p; ++m) {
    if (!(H_ref[m] > 0.0)) return fail(c, ESPLIT_ERR_ARG, "H_ref must be positive");
    t.H[m] = H_ref[m];
  }
  (void)facet_w;
  (void)ref_normals;
  int rc = dalloc(c, &c->b.Qref, (size_t)c->dim * n_p * n_p);
  if (rc) return rc;
  CK(cudaMemcpy(c->b.Qref, Q_ref, sizeof(double) * c->dim * n_p * n_p, cudaMemcpyHostToDevice));
  if (esplit::set_ref_tables(t) || esplit::set_ref_tables_f32(t))
    return fail(c, ESPLIT_ERR_CUDA, "constant-table upload failed");
  c->ref = t;
  c->n_p = n_p;
  c->n_fac = n_fac;
  c->n_f = n_f;
  c->n_slot = n_slot;
  c->have_op = true;
  c->have_mesh = false;  // a new operator invalidates the mesh-derived data
  return ESPLIT_OK;
}

static int ensure_viscous(esplit_ctx* c);

// hybrid lists and flags, capacity n_e (allocated once per mesh)
static int ensure_hybrid(esplit_ctx* c) {
  if (c->b.hcount) return ESPLIT_OK;
  int rc;
  size_t n = (size_t)c->n_e;
  if ((rc = dalloc(c, &c->b.list_split, n))) return rc;
  if ((rc = dalloc(c, &c->b.list_had, n))) return rc;
  if ((rc = dalloc(c, &c->b.hflags, n))) return rc;
  if ((rc = dalloc(c, &c->b.hflag0, n))) return rc;
  if ((rc = dalloc(c, &c->b.hcount, (n + 1023) / 1024 + 1))) return rc;
  return ESPLIT_OK;
}

int esplit_upload_mesh(esplit_ctx* c, int n_e, const double* J, const double* Lambda, const double* nu,
                       const int* pair, const double* hmin) {
  if (!c) return ESPLIT_ERR_ARG;
  c->version++;
  if (!c->have_op) return fail(c, ESPLIT_ERR_STATE, "upload the operator before the mesh");
  if (n_e <= 0 || !J || !Lambda || !nu || !pair) return fail(c, ESPLIT_ERR_ARG, "bad mesh arguments");
  (void)hmin;
  cudaSetDevice(c->device);
  const int d = c->dim, NP = c->n_p, NS = c->n_slot;
  // --- host validation
  for (size_t i = 0; i < (size_t)n_e * NP; ++i)
    if (!(J[i] > 0.0)) return fail(c, ESPLIT_ERR_MESH, "J must be positive at every node");
  std::vector<int2> fpairs;
  std::vector<int> bslots;
  fpairs.reserve((size_t)n_e * NS / 2);
  for (int k = 0; k < n_e; ++k) {
    for (int s = 0; s < NS; ++s) {
      size_t a = (size_t)k * NS + s;
      int v = pair[2 * a], s2 = pair[2 * a + 1];
      if (v == -1 && s2 == -1) {  // boundary facet slot: exterior state from esplit_set_boundary_states
        bool ok = false;
        for (int i = 0; i < d; ++i) ok = ok || nu[a * d + i] != 0.0;
        if (!ok) return fail(c, ESPLIT_ERR_MESH, "boundary facet slot with a zero normal");
        bslots.push_back((int)a);
        continue;
      }
      if (v < 0 || v >= n_e || s2 < 0 || s2 >= NS) return fail(c, ESPLIT_ERR_MESH, "pair index out of range");
      size_t b2 = (size_t)v * NS + s2;
      if (pair[2 * b2] != k || pair[2 * b2 + 1] != s) return fail(c, ESPLIT_ERR_MESH, "pairing is not an involution");
      if (b2 == a) return fail(c, ESPLIT_ERR_MESH, "facet slot paired with itself");
      double sc = 0.0, df = 0.0;
      for (int i = 0; i < d; ++i) {
        sc = std::max(sc, std::fabs(nu[a * d + i]));
        df = std::max(df, std::fabs(nu[a * d + i] + nu[b2 * d + i]));
      }
      if (!(sc > 0.0) || df > kNuTol * sc) return fail(c, ESPLIT_ERR_MESH, "normals of paired slots are not opposite");
      if (a < b2) fpairs.push_back(make_int2((int)a, (int)b2));
    }
  }
  c->n_e = n_e;
  c->n_pairs = (int)fpairs.size();
  c->n_bslot = (int)bslots.size();
  c->bslots = bslots;
  c->have_bstate = false;
  int rc;
  if ((rc = dalloc(c, &c->b.J, (size_t)n_e * NP))) return rc;
  if ((rc = dalloc(c, &c->b.nu, (size_t)n_e * NS * d))) return rc;
  if ((rc = dalloc(c, &c->b.pair, (size_t)n_e * NS * 2))) return rc;
  if ((rc = dalloc(c, &c->b.Lam, (size_t)n_e * d * d * NP))) return rc;
  if ((rc = dalloc(c, &c->b.face_pairs, fpairs.size()))) return rc;
  if ((rc = dalloc(c, &c->b.ops64, (size_t)n_e * 2 * d * NP * NP))) return rc;
  if ((rc = dalloc(c, &c->b.ops32, (size_t)n_e * 2 * d * NP * NP))) return rc;
  if ((rc = dalloc(c, &c->b.ops32lo, (size_t)n_e * 2 * d * NP * NP))) return rc;
  if ((rc = dalloc(c, &c->b.rows, (size_t)n_e * 2 * d * NP))) return rc;
  if ((rc = dalloc(c, &c->b.sat, (size_t)n_e * c->n_c * NS))) return rc;
  if ((rc = dalloc(c, &c->b.fcache, (size_t)(d + 9) * n_e * NS))) return rc;
  if ((rc = dalloc(c, &c->b.ihf, (size_t)n_e * NP))) return rc;
  if ((rc = dalloc(c, &c->b.ihd, (size_t)n_e * NP))) return rc;
  if ((rc = dalloc(c, &c->b.nscale, (size_t)n_e * NS * (d + 1)))) return rc;
  if (d <= 2) {
    c->opsD_stride = opsD_stride_for(d, NP);
    if ((rc = dalloc(c, &c->b.opsD32, (size_t)n_e * c->opsD_stride))) return rc;
  } else {
    dalloc(c, &c->b.opsD32, 0);
    c->opsD_stride = 0;
  }
  c->partial_cap = 0;
  if ((rc = ensure_partial(c))) return rc;
  CK(cudaMemcpy(c->b.J, J, sizeof(double) * n_e * NP, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->b.nu, nu, sizeof(double) * n_e * NS * d, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->b.pair, pair, sizeof(int) * n_e * NS * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->b.Lam, Lambda, sizeof(double) * n_e * d * d * NP, cudaMemcpyHostToDevice));
  {
    std::vector<float> ih((size_t)n_e * NP);
    for (size_t i = 0; i < ih.size(); ++i) ih[i] = (float)(1.0 / (c->ref.H[i % NP] * J[i]));
    CK(cudaMemcpy(c->b.ihf, ih.data(), sizeof(float) * ih.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(c->b.face_pairs, fpairs.data(), sizeof(int2) * fpairs.size(), cudaMemcpyHostToDevice));
  dalloc(c, &c->b.bstate, 0);
  if ((rc = dalloc(c, &c->b.bslot, bslots.size()))) return rc;
  if (!bslots.empty())
    CK(cudaMemcpy(c->b.bslot, bslots.data(), sizeof(int) * bslots.size(), cudaMemcpyHostToDevice));
  // RRK / host-path scratch is (re)allocated lazily
  dalloc(c, &c->b.stage_u, 0);
  dalloc(c, &c->b.stage_r, 0);
  dalloc(c, &c->b.dacc, 0);
  dalloc(c, &c->b.node_cache, 0);
  dalloc(c, &c->b.vjp_work, 0);
  dalloc(c, &c->b.host_u, 0);
  dalloc(c, &c->b.host_r, 0);
  c->flags.assign(n_e, 0);
  dalloc(c, &c->b.list_split, 0);  // the hybrid scheme needs flags for the new mesh
  dalloc(c, &c->b.list_had, 0);
  dalloc(c, &c->b.hflags, 0);
  dalloc(c, &c->b.hflag0, 0);
  dalloc(c, &c->b.hcount, 0);
  dalloc(c, &c->b.fv, 0);
  dalloc(c, &c->b.vsat, 0);
  dalloc(c, &c->b.va, 0);
  dalloc(c, &c->b.wslot, 0);
  dalloc(c, &c->b.vfb, 0);
  dalloc(c, &c->b.vfs, 0);
  dalloc(c, &c->b.vus, 0);
  c->n_split = n_e;
  c->n_had = 0;
  c->have_mesh = true;
  if (c->prm.viscous && (rc = ensure_viscous(c))) return rc;
  return rebuild_ops(c, 0);
}

int esplit_set_params(esplit_ctx* c, const esplit_params* p) {
  if (!c || !p) return ESPLIT_ERR_ARG;
  c->version++;
  if (!(p->gam > 1.0)) return fail(c, ESPLIT_ERR_ARG, "gam must exceed 1");
  double alpha = -p->gam - p->beta * (p->gam - 1.0);
  if (!(alpha < -p->gam || alpha > 0.0)) return fail(c, ESPLIT_ERR_ARG, "beta must give alpha < -gam or alpha > 0");
  if (!(p->R > 0.0) || p->mu < 0.0 || !(p->Pr > 0.0)) return fail(c, ESPLIT_ERR_ARG, "R, Pr must be > 0, mu >= 0");
  if (p->scheme < 0 || p->scheme > 3) return fail(c, ESPLIT_ERR_ARG, "unknown scheme");
  if (p->precision != ESPLIT_FP64 && p->precision != ESPLIT_FP32_BULK && p->precision != ESPLIT_FP32)
    return fail(c, ESPLIT_ERR_ARG, "unknown precision");
  if (p->viscous && c->dim == 1) return fail(c, ESPLIT_ERR_UNSUPPORTED, "1D: inviscid only");
  cudaSetDevice(c->device);
  bool beta_changed = p->beta != c->prm.beta;
  c->prm = *p;
  if (p->viscous) {
    int rcv = ensure_viscous(c);
    if (rcv) return rcv;
  }
  if (beta_changed && c->have_mesh) return rebuild_ops(c, 0);
  return ESPLIT_OK;
}

int esplit_get_params(esplit_ctx* c, esplit_params* p) {
  if (!c || !p) return ESPLIT_ERR_ARG;
  *p = c->prm;
  return ESPLIT_OK;
}

int esplit_set_hybrid_flags(esplit_ctx* c, const unsigned char* flags, int n_e) {
  if (!c || !flags) return ESPLIT_ERR_ARG;
  c->version++;
  if (!c->have_mesh) return fail(c, ESPLIT_ERR_STATE, "upload the mesh before the hybrid flags");
  if (n_e != c->n_e) return fail(c, ESPLIT_ERR_ARG, "flags length must equal n_e");
  cudaSetDevice(c->device);
  std::vector<int> ls, lh;
  for (int e = 0; e < n_e; ++e) {
    if (flags[e] > 1) return fail(c, ESPLIT_ERR_ARG, "hybrid flags must be 0 or 1");
    (flags[e] ? lh : ls).push_back(e);
  }
  c->flags.assign(flags, flags + n_e);
  int rc;
  if ((rc = ensure_hybrid(c))) return rc;
  if (!ls.empty()) CK(cudaMemcpy(c->b.list_split, ls.data(), sizeof(int) * ls.size(), cudaMemcpyHostToDevice));
  if (!lh.empty()) CK(cudaMemcpy(c->b.list_had, lh.data(), sizeof(int) * lh.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->b.hflags, flags, n_e, cudaMemcpyHostToDevice));
  c->n_split = (int)ls.size();
  c->n_had = (int)lh.size();
  return ESPLIT_OK;
}

int esplit_set_boundary_states(esplit_ctx* c, int n_b, const int* slots, const double* states) {
  if (!c) return ESPLIT_ERR_ARG;
  c->version++;
  if (!c->have_mesh) return fail(c, ESPLIT_ERR_STATE, "upload the mesh first");
  if (n_b != c->n_bslot)
    return fail(c, ESPLIT_ERR_ARG, "n_b must equal the mesh's number of boundary facet slots (" +
                                       std::to_string(c->n_bslot) + ")");
  if (n_b == 0) return ESPLIT_OK;
  if (!slots || !states) return fail(c, ESPLIT_ERR_ARG, "null pointer");
  const int nc = c->n_c;
  std::vector<double> ordered((size_t)n_b * nc);
  std::vector<char> seen(n_b, 0);
  for (int i = 0; i < n_b; ++i) {
    auto it = std::lower_bound(c->bslots.begin(), c->bslots.end(), slots[i]);
    if (it == c->bslots.end() || *it != slots[i]) return fail(c, ESPLIT_ERR_ARG, "slot is not a boundary facet slot");
    const size_t pos = (size_t)(it - c->bslots.begin());
    if (seen[pos]) return fail(c, ESPLIT_ERR_ARG, "boundary facet slot given twice");
    seen[pos] = 1;
    const double* st = states + (size_t)i * nc;
    double ke = 0.0;
    for (int j = 0; j < c->dim; ++j) ke += 0.5 * st[1 + j] * st[1 + j] / st[0];
    const double p = (c->prm.gam - 1.0) * (st[nc - 1] - ke);
    if (!(st[0] > 0.0) || !(p > 0.0) || !std::isfinite(st[nc - 1]))
      return fail(c, ESPLIT_ERR_ARG, "exterior state not physical (rho, p must be positive and finite)");
    for (int q = 0; q < nc; ++q) ordered[pos * nc + q] = st[q];
  }
  cudaSetDevice(c->device);
  int rc;
  if (!c->b.bstate && (rc = dalloc(c, &c->b.bstate, ordered.size()))) return rc;
  CK(cudaMemcpy(c->b.bstate, ordered.data(), sizeof(double) * ordered.size(), cudaMemcpyHostToDevice));
  c->have_bstate = true;
  return ESPLIT_OK;
}

int esplit_detect_hybrid(esplit_ctx* c, const double* u, double threshold, int* n_flagged, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  c->version++;
  if (!u) return fail(c, ESPLIT_ERR_ARG, "null state pointer");
  if (!(threshold >= 1.0) || !std::isfinite(threshold)) return fail(c, ESPLIT_ERR_ARG, "threshold must be finite and >= 1");
  cudaSetDevice(c->device);
  if ((rc = ensure_hybrid(c))) return rc;
  cudaStream_t s = as_stream(stream);
  if (esplit::launch_detect_hybrid(c, u, threshold, s))
    return fail(c, ESPLIT_ERR_CUDA, std::string("detector launch: ") + cudaGetErrorString(cudaGetLastError()));
  int total = 0;
  CK(cudaMemcpyAsync(&total, c->b.hcount + (c->n_e + 1023) / 1024, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  c->n_had = total;
  c->n_split = c->n_e - total;
  c->last_stream = s;
  if (n_flagged) *n_flagged = total;
  return ESPLIT_OK;
}

int esplit_get_hybrid_flags(esplit_ctx* c, unsigned char* flags) {
  if (!c || !flags) return ESPLIT_ERR_ARG;
  if (!c->have_mesh) return fail(c, ESPLIT_ERR_STATE, "no mesh uploaded");
  if (!c->b.hflags) return fail(c, ESPLIT_ERR_STATE, "no hybrid flags set or detected");
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->last_stream));
  CK(cudaMemcpy(flags, c->b.hflags, c->n_e, cudaMemcpyDeviceToHost));
  return ESPLIT_OK;
}

static int boundary_ready(esplit_ctx* c) {
  if (c->n_bslot == 0) return ESPLIT_OK;
  if (!c->have_bstate) return fail(c, ESPLIT_ERR_STATE, "the mesh has boundary facets: esplit_set_boundary_states");
  if (c->prm.viscous) return fail(c, ESPLIT_ERR_UNSUPPORTED, "viscous terms on boundary facets are not built");
  return ESPLIT_OK;
}

static int residual_impl(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* prod, int* npart) {
  if (c->prm.scheme == ESPLIT_SCHEME_HYBRID && !c->b.list_split)
    return fail(c, ESPLIT_ERR_STATE, "hybrid scheme needs esplit_set_hybrid_flags");
  if (int brc = boundary_ready(c)) return brc;
  const bool visc = c->prm.viscous != 0;
  if (visc && !c->b.fv) return fail(c, ESPLIT_ERR_STATE, "viscous scratch missing");
  // the entropy production comes with the residual kernels' block partials:
  // the split kernel's (everything but the viscous flux jump) and the jump
  // kernel's; with viscous terms and Hadamard-form elements it is taken from
  // the complete residual after the viscous passes
  const bool fused = !visc || c->prm.scheme == ESPLIT_SCHEME_SPLIT;
  int rc = esplit::launch_residual(c, u, r, s, fused ? prod : nullptr, fused ? npart : nullptr);
  if (rc == -2) return fail(c, ESPLIT_ERR_UNSUPPORTED, "operator size not compiled in");
  if (rc) return fail(c, ESPLIT_ERR_CUDA, std::string("residual launch: ") + cudaGetErrorString(cudaGetLastError()));
  if (!fused && prod && esplit::launch_entropy_rate(c, u, r, s, npart, prod, 1))
    return fail(c, ESPLIT_ERR_CUDA, "entropy-production launch");
  c->last_stream = s;
  return ESPLIT_OK;
}

static int ensure_viscous(esplit_ctx* c) {
  if (!c->have_mesh || c->b.fv) return ESPLIT_OK;
  int rc;
  if ((rc = dalloc(c, &c->b.fv, (size_t)c->n_e * c->dim * c->n_c * c->n_p))) return rc;
  if ((rc = dalloc(c, &c->b.vsat, (size_t)c->n_e * c->n_c * c->n_slot))) return rc;
  if ((rc = dalloc(c, &c->b.va, (size_t)c->n_e * c->dim * c->n_c * c->n_slot))) return rc;
  if ((rc = dalloc(c, &c->b.wslot, (size_t)c->n_e * c->n_c * c->n_slot))) return rc;
  return ESPLIT_OK;
}

int esplit_residual(esplit_ctx* c, const double* u, double* r, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u || !r) return fail(c, ESPLIT_ERR_ARG, "null state pointer");
  if (u == r) return fail(c, ESPLIT_ERR_ARG, "u and dudt must not alias");
  cudaSetDevice(c->device);
  return residual_impl(c, u, r, as_stream(stream), nullptr, nullptr);
}

int esplit_residual_noalloc(esplit_ctx* c, const double* u, double* r, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u || !r) return fail(c, ESPLIT_ERR_ARG, "null state pointer");
  if (u == r) return fail(c, ESPLIT_ERR_ARG, "u and dudt must not alias");
  if (c->prm.scheme == ESPLIT_SCHEME_HYBRID && !c->b.list_split)
    return fail(c, ESPLIT_ERR_STATE, "hybrid scheme needs esplit_set_hybrid_flags");
  if (c->prm.viscous && !c->b.fv) return fail(c, ESPLIT_ERR_STATE, "viscous scratch missing");
  if ((rc = boundary_ready(c))) return rc;
  size_t need = (size_t)c->n_e * c->n_c * c->n_slot;
  if (need > esplit::NOALLOC_SCRATCH_DOUBLES)
    return fail(c, ESPLIT_ERR_ARG,
                "mesh too large for esplit_residual_noalloc: its facet scratch needs " + std::to_string(need) +
                    " doubles (n_e * n_c * n_slot), the static maximum is " +
                    std::to_string(esplit::NOALLOC_SCRATCH_DOUBLES));
  CK(cudaSetDevice(c->device));
  double* scratch = nullptr;
  if (esplit::noalloc_scratch_ptr(c->device, &scratch))
    return fail(c, ESPLIT_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
  rc = esplit::launch_residual_noalloc(c, u, r, as_stream(stream), scratch);
  if (rc == -2) return fail(c, ESPLIT_ERR_UNSUPPORTED, "operator size not compiled in");
  if (rc) return fail(c, ESPLIT_ERR_CUDA, std::string("residual launch: ") + cudaGetErrorString(cudaGetLastError()));
  c->last_stream = as_stream(stream);
  return ESPLIT_OK;
}

int esplit_residual_host(esplit_ctx* c, const double* u, double* r, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u || !r) return fail(c, ESPLIT_ERR_ARG, "null state pointer");
  cudaSetDevice(c->device);
  size_t n = (size_t)c->n_e * c->n_c * c->n_p;
  if (!c->b.host_u) {
    if ((rc = dalloc(c, &c->b.host_u, n))) return rc;
    if ((rc = dalloc(c, &c->b.host_r, n))) return rc;
  }
  cudaStream_t s = as_stream(stream);
  CK(cudaMemcpyAsync(c->b.host_u, u, n * sizeof(double), cudaMemcpyHostToDevice, s));
  if ((rc = residual_impl(c, c->b.host_u, c->b.host_r, s, nullptr, nullptr))) return rc;
  CK(cudaMemcpyAsync(r, c->b.host_r, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return ESPLIT_OK;
}

int esplit_entropy(esplit_ctx* c, const double* u, double* S_total, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u || !S_total) return fail(c, ESPLIT_ERR_ARG, "null pointer");
  cudaSetDevice(c->device);
  cudaStream_t s = as_stream(stream);
  int np = 0;
  if (esplit::launch_entropy(c, u, s, &np)) return fail(c, ESPLIT_ERR_CUDA, "entropy launch");
  if (esplit::launch_reduce(c, c->b.partial, np, 2, c->b.scal + 8, s)) return fail(c, ESPLIT_ERR_CUDA, "reduce");
  double h[2];
  CK(cudaMemcpyAsync(h, c->b.scal + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *S_total = h[0];
  return ESPLIT_OK;
}

int esplit_entropy_rate(esplit_ctx* c, const double* u, const double* r, double* rate, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u || !r || !rate) return fail(c, ESPLIT_ERR_ARG, "null pointer");
  cudaSetDevice(c->device);
  cudaStream_t s = as_stream(stream);
  int np = 0;
  if (esplit::launch_entropy_rate(c, u, r, s, &np)) return fail(c, ESPLIT_ERR_CUDA, "entropy-rate launch");
  if (esplit::launch_reduce(c, c->b.partial, np, 2, c->b.scal + 10, s)) return fail(c, ESPLIT_ERR_CUDA, "reduce");
  double h[2];
  CK(cudaMemcpyAsync(h, c->b.scal + 10, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *rate = h[0];
  return ESPLIT_OK;
}

// Preconditions of a relaxation step; allocates the stage buffers once.
static int rrk_prepare(esplit_ctx* c, const double* u, double dt) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u) return fail(c, ESPLIT_ERR_ARG, "null state pointer");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, ESPLIT_ERR_ARG, "dt must be positive and finite");
  if (c->prm.scheme == ESPLIT_SCHEME_HADAMARD_IR)
    return fail(c, ESPLIT_ERR_UNSUPPORTED, "the relaxation step uses Harten's entropy; the Ismail-Roe comparator "
                                           "conserves the standard one");
  cudaSetDevice(c->device);
  size_t n = (size_t)c->n_e * c->n_c * c->n_p;
  if (!c->b.stage_u) {
    if ((rc = dalloc(c, &c->b.stage_u, n))) return rc;
    if ((rc = dalloc(c, &c->b.stage_r, n))) return rc;
    if ((rc = dalloc(c, &c->b.dacc, n))) return rc;
    if ((rc = dalloc(c, &c->b.node_cache, 3 * (size_t)c->n_e * c->n_p))) return rc;
  }
  if (esplit::uses_f32_path(c) && !c->side_s) {
    CK(cudaStreamCreateWithFlags(&c->side_s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  return ESPLIT_OK;
}

// The four RK4 stages (Eq. (98) with the classical tableau), the entropy of
// u_n, the reduction of the stage entropy productions and the root-solve
// start, all enqueued on s.
static int rrk_enqueue_stages(esplit_ctx* c, const double* u, double dt, cudaStream_t s) {
  static const double A[4] = {0.0, 0.5, 0.5, 1.0};
  static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const size_t n = (size_t)c->n_e * c->n_c * c->n_p;
  int np = 0, rc;
  // block-partial regions: entropy of u_n (width 2) first, then the four stage
  // productions (width 1); reduced together after the stages
  esplit::ReduceRegions R{};
  const int ent_cap = (int)std::max<size_t>((size_t)c->n_e * c->n_p / 256 + 1, (size_t)c->n_e);
  int off = 2 * ent_cap;
  // stage 0: the split volume kernel computes the entropy of u_n on the way
  // (entropy-split scheme); otherwise the entropy kernel does.  On the
  // float32 path (whose kernels leave the float64 pipe mostly idle) it runs on
  // the side stream from the start of the step, joined before the reduction
  const bool side = esplit::uses_f32_path(c) && c->side_s;
  int ne_side = 0;
  if (side) {
    CK(cudaEventRecord(c->ev_fork, s));
    CK(cudaStreamWaitEvent(c->side_s, c->ev_fork, 0));
    if (esplit::launch_entropy(c, u, c->side_s, &ne_side, c->b.node_cache, c->b.partial))
      return fail(c, ESPLIT_ERR_CUDA, "entropy launch");
    CK(cudaEventRecord(c->ev_join, c->side_s));
  }
  c->ent_part = side ? nullptr : c->b.partial;
  c->ent_n = 0;
  for (int i = 0; i < 4; ++i) {
    const double* Ui = (i == 0) ? u : c->b.stage_u;
    rc = residual_impl(c, Ui, c->b.stage_r, s, c->b.partial + off, &np);
    if (i == 0) {
      c->ent_part = nullptr;
      if (rc) return rc;
      int ne = side ? ne_side : c->ent_n;
      if (ne == 0 && esplit::launch_entropy(c, u, s, &ne, c->b.node_cache, c->b.partial))
        return fail(c, ESPLIT_ERR_CUDA, "entropy launch");
      R.off[0] = 0;
      R.cnt[0] = ne;
      R.width[0] = 2;
      R.out[0] = c->b.scal;
    }
    if (rc) return rc;
    R.off[1 + i] = off;
    R.cnt[1 + i] = np;
    R.width[1 + i] = 1;
    R.out[1 + i] = c->b.scal + 2 + i;
    off += np;
    double a_next = (i < 3) ? A[i + 1] * dt : 0.0;
    if (esplit::launch_stage(c, u, c->b.stage_r, a_next, B[i] * dt, i == 0, (i < 3) ? c->b.stage_u : nullptr,
                             c->b.dacc, n, s))
      return fail(c, ESPLIT_ERR_CUDA, "stage launch");
  }
  R.n = 5;
  if (side) CK(cudaStreamWaitEvent(s, c->ev_join, 0));
  if (esplit::launch_reduce_regions(c, c->b.partial, R, s)) return fail(c, ESPLIT_ERR_CUDA, "reduce");
  if (esplit::launch_root_start(c, dt, s)) return fail(c, ESPLIT_ERR_CUDA, "root init");
  return ESPLIT_OK;
}

int esplit_rrk_step(esplit_ctx* c, double* u, double dt, double* g_out, esplit_stepinfo* info, void* stream) {
  int rc = rrk_prepare(c, u, dt);
  if (rc) return rc;
  cudaStream_t s = as_stream(stream);
  const size_t n = (size_t)c->n_e * c->n_c * c->n_p;
  if ((rc = rrk_enqueue_stages(c, u, dt, s))) return rc;
  esplit::RootState st{};
  // two evaluation passes and the (guarded) update go out without a host
  // round trip: the first pass usually ends the solve (Halley step at g = 1)
  for (int it = 0; it < 2; ++it)
    if (esplit::launch_root_eval(c, u, c->b.dacc, s))
      return fail(c, ESPLIT_ERR_CUDA, "root launch");
  if (esplit::launch_root_apply(c, u, c->b.dacc, n, s)) return fail(c, ESPLIT_ERR_CUDA, "apply launch");
  CK(cudaMemcpyAsync(&st, c->b.root, sizeof(st), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!st.done) {
    for (int it = 2; it < esplit::ROOT_EVALS_MAX; ++it) {
      if (esplit::launch_root_eval(c, u, c->b.dacc, s))
        return fail(c, ESPLIT_ERR_CUDA, "root launch");
      if ((it + 1) % esplit::ROOT_CHECK_EVERY == 0) {
        CK(cudaMemcpyAsync(&st, c->b.root, sizeof(st), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (st.done) break;
      }
    }
    if (esplit::launch_root_apply(c, u, c->b.dacc, n, s)) return fail(c, ESPLIT_ERR_CUDA, "apply launch");
  }
  double e_stage[4];
  CK(cudaMemcpyAsync(&st, c->b.root, sizeof(st), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(e_stage, c->b.scal + 2, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int phys = read_status(c, s, true);
  c->last_stream = s;
  int status = phys ? phys : st.status;
  if (g_out) *g_out = st.g;
  if (info) {
    info->g = st.g;
    info->estimate = st.est;
    info->S_before = st.S0;
    info->iterations = st.iters;
    info->status = status;
    // entropy change at the returned g (the last evaluation, carried to g to
    // first order when the final Newton correction was accepted without one)
    info->S_after = st.S0 + (st.phase == 3 ? st.dS_last : 0.0);
    for (int i = 0; i < 4; ++i) info->stage_rate[i] = e_stage[i];
  }
  if (status == ESPLIT_ERR_NONPHYSICAL) return fail(c, status, "non-physical state during the step");
  if (status == ESPLIT_ERR_RRK_NO_ROOT) return fail(c, status, "relaxation parameter could not be bracketed");
  return ESPLIT_OK;
}

namespace {
constexpr int HIST_CAP = 1024;  // step records per batch chunk (one host read each)

void drop_step_graph(esplit_ctx* c) {
  if (c->sg.exec) cudaGraphExecDestroy(c->sg.exec);
  if (c->sg.graph) cudaGraphDestroy(c->sg.graph);
  c->sg = StepGraph{};
}
}  // namespace

// Records one relaxation step for state u and dt as a CUDA graph: the stages,
// reductions and root start as captured from rrk_enqueue_stages, the root
// solve as a conditional while node whose body is one evaluation pass with its
// root update (the pass's last block clears the loop condition once the root
// is done), then
// the guarded update of u and the step record.  The launches are the ones
// esplit_rrk_step makes, in the same order, so the results are identical.
static int rrk_capture(esplit_ctx* c, double* u, double dt) {
  drop_step_graph(c);
  if (!c->cap_s) CK(cudaStreamCreateWithFlags(&c->cap_s, cudaStreamNonBlocking));
  if (!c->cap_s2) CK(cudaStreamCreateWithFlags(&c->cap_s2, cudaStreamNonBlocking));
  if (!c->hist) CK(cudaMalloc(&c->hist, HIST_CAP * sizeof(esplit::StepRecord) + 256));
  esplit::StepRecord* hist = static_cast<esplit::StepRecord*>(c->hist);
  int* counter = reinterpret_cast<int*>(hist + HIST_CAP);
  const size_t n = (size_t)c->n_e * c->n_c * c->n_p;
  cudaStream_t cs = c->cap_s;
  const long long l0 = c->launches;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  std::string why;
  int rc = rrk_enqueue_stages(c, u, dt, cs);
  if (rc) why = "stages";
  cudaGraphConditionalHandle h = 0;
  if (!rc) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphNode_t cn = nullptr;
    cudaGraphNodeParams prm = {};
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd);
    if (e == cudaSuccess && cst != cudaStreamCaptureStatusActive) e = cudaErrorStreamCaptureInvalidated;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, cg, 1u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      prm.type = cudaGraphNodeTypeConditional;
      prm.conditional.handle = h;
      prm.conditional.type = cudaGraphCondTypeWhile;
      prm.conditional.size = 1;
      e = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &prm);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(c->cap_s2, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      int r1 = esplit::launch_root_eval_cond(c, u, c->b.dacc, c->cap_s2, h);
      cudaGraph_t bg = nullptr;
      e = cudaStreamEndCapture(c->cap_s2, &bg);
      if (r1 && e == cudaSuccess) e = cudaErrorLaunchFailure;
    }
    if (e != cudaSuccess) {
      rc = ESPLIT_ERR_CUDA;
      why = std::string("root loop: ") + cudaGetErrorString(e);
    }
  }
  if (!rc && (esplit::launch_root_apply(c, u, c->b.dacc, n, cs) ||
              esplit::launch_step_record(c, hist, counter, HIST_CAP, cs))) {
    rc = ESPLIT_ERR_CUDA;
    why = "apply / record";
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (!rc && e != cudaSuccess) {
    rc = ESPLIT_ERR_CUDA;
    why = std::string("end capture: ") + cudaGetErrorString(e);
  }
  if (!rc) {
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
      rc = ESPLIT_ERR_CUDA;
      why = std::string("instantiate: ") + cudaGetErrorString(e);
    } else {
      c->sg.exec = x;
    }
  }
  if (rc) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    c->launches = l0;
    return fail(c, rc == ESPLIT_ERR_CUDA ? ESPLIT_ERR_CUDA : rc, "recording the step graph failed (" + why + ")");
  }
  c->sg.graph = g;
  c->sg.u = u;
  c->sg.dt = dt;
  c->sg.version = c->version;
  c->sg.kernels = c->launches - l0 - 2;  // the loop body's two launches are counted per pass
  c->launches = l0;
  return ESPLIT_OK;
}

static void fill_info(esplit_stepinfo* info, const esplit::StepRecord& r) {
  info->g = r.g;
  info->estimate = r.est;
  info->S_before = r.S0;
  info->S_after = r.S_after;
  info->iterations = r.iters;
  info->status = r.status;
  for (int i = 0; i < 4; ++i) info->stage_rate[i] = r.stage_rate[i];
}

int esplit_rrk_steps(esplit_ctx* c, double* u, double dt, int n_steps, double* g_out, esplit_stepinfo* info,
                     int* n_done, void* stream) {
  if (n_done) *n_done = 0;
  int rc = rrk_prepare(c, u, dt);
  if (rc) return rc;
  if (n_steps < 0) return fail(c, ESPLIT_ERR_ARG, "n_steps must be non-negative");
  cudaStream_t s = as_stream(stream);
  int done = 0;
  const bool fresh = c->sg.exec && c->sg.u == u && c->sg.dt == dt && c->sg.version == c->version;
  if (c->prof || !fresh) {
    // profiling brackets every launch with events, which a graph does not
    // take: steps one by one.  A new recording starts with one ordinary step,
    // which makes every lazy allocation and set-up before the capture.
    const int n_plain = c->prof ? n_steps : std::min(n_steps, 1);
    for (; done < n_plain; ++done) {
      esplit_stepinfo si{};
      rc = esplit_rrk_step(c, u, dt, nullptr, &si, stream);
      if (info) *info = si;
      if (rc) return rc;
      if (g_out) g_out[done] = si.g;
      if (n_done) *n_done = done + 1;
    }
    if (done == n_steps) return ESPLIT_OK;
    if ((rc = rrk_capture(c, u, dt))) return rc;
  }
  esplit::StepRecord* hist = static_cast<esplit::StepRecord*>(c->hist);
  int* counter = reinterpret_cast<int*>(hist + HIST_CAP);
  std::vector<esplit::StepRecord> h;
  while (done < n_steps) {
    const int chunk = std::min(HIST_CAP, n_steps - done);
    CK(cudaMemsetAsync(counter, 0, sizeof(int), s));
    for (int k = 0; k < chunk; ++k) CK(cudaGraphLaunch(c->sg.exec, s));
    h.resize(chunk);
    CK(cudaMemcpyAsync(h.data(), hist, chunk * sizeof(esplit::StepRecord), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    read_status(c, s, true);
    c->last_stream = s;
    for (int k = 0; k < chunk; ++k) {
      c->launches += c->sg.kernels + 2LL * h[k].iters;
      if (info) fill_info(info, h[k]);
      if (h[k].status == ESPLIT_ERR_NONPHYSICAL) return fail(c, h[k].status, "non-physical state during the step");
      if (h[k].status) return fail(c, h[k].status, "relaxation parameter could not be bracketed");
      if (g_out) g_out[done] = h[k].g;
      ++done;
      if (n_done) *n_done = done;
    }
  }
  return ESPLIT_OK;
}

int esplit_rrk_step_host(esplit_ctx* c, double* u_host, double dt, double* g_out, esplit_stepinfo* info,
                         void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u_host) return fail(c, ESPLIT_ERR_ARG, "null state pointer");
  cudaSetDevice(c->device);
  size_t n = (size_t)c->n_e * c->n_c * c->n_p;
  if (!c->b.host_u) {
    if ((rc = dalloc(c, &c->b.host_u, n))) return rc;
    if ((rc = dalloc(c, &c->b.host_r, n))) return rc;
  }
  cudaStream_t s = as_stream(stream);
  CK(cudaMemcpyAsync(c->b.host_u, u_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  rc = esplit_rrk_step(c, c->b.host_u, dt, g_out, info, stream);
  if (rc) return rc;
  CK(cudaMemcpyAsync(u_host, c->b.host_u, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return ESPLIT_OK;
}

// (d dudt/du)^T cot: inviscid split terms, then the viscous terms when on
static int vjp_impl(esplit_ctx* c, const double* u, const double* cot, double* grad, cudaStream_t s) {
  int rc = esplit::launch_residual_vjp(c, u, cot, grad, s);
  if (rc == -2) return fail(c, ESPLIT_ERR_UNSUPPORTED, "operator size not compiled in");
  if (rc) return fail(c, ESPLIT_ERR_CUDA, std::string("vjp launch: ") + cudaGetErrorString(cudaGetLastError()));
  if (c->prm.viscous) {
    if ((rc = ensure_viscous(c))) return rc;
    if (!c->b.vfb) {
      size_t per = (size_t)c->n_e * c->n_c;
      if ((rc = dalloc(c, &c->b.vfb, per * c->dim * c->n_p))) return rc;
      if ((rc = dalloc(c, &c->b.vfs, per * c->dim * c->n_slot))) return rc;
      if ((rc = dalloc(c, &c->b.vus, per * c->n_slot))) return rc;
    }
    rc = esplit::launch_viscous_vjp(c, u, cot, grad, s);
    if (rc == -2) return fail(c, ESPLIT_ERR_UNSUPPORTED, "operator size not compiled in");
    if (rc)
      return fail(c, ESPLIT_ERR_CUDA, std::string("viscous vjp launch: ") + cudaGetErrorString(cudaGetLastError()));
  }
  c->last_stream = s;
  return ESPLIT_OK;
}

int esplit_residual_vjp(esplit_ctx* c, const double* u, const double* cot, double* grad, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u || !cot || !grad) return fail(c, ESPLIT_ERR_ARG, "null pointer");
  if (grad == u || grad == cot) return fail(c, ESPLIT_ERR_ARG, "grad must not alias u or cot");
  if (c->prm.scheme != ESPLIT_SCHEME_SPLIT || c->dim == 1 || c->n_bslot > 0)
    return fail(c, ESPLIT_ERR_UNSUPPORTED,
                "the residual VJP is built for the entropy-split scheme in 2D and 3D on periodic meshes");
  cudaSetDevice(c->device);
  cudaStream_t s = as_stream(stream);
  return vjp_impl(c, u, cot, grad, s);
}

int esplit_entropy_grad(esplit_ctx* c, const double* u, double* grad, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u || !grad) return fail(c, ESPLIT_ERR_ARG, "null pointer");
  cudaSetDevice(c->device);
  if (esplit::launch_wH(c, u, 1.0, grad, as_stream(stream))) return fail(c, ESPLIT_ERR_CUDA, "entropy-grad launch");
  c->last_stream = as_stream(stream);
  return ESPLIT_OK;
}

int esplit_rrk_step_vjp(esplit_ctx* c, const double* u, double dt, const double* ubar1, double* ubar0,
                        double* g_out, void* stream) {
  int rc = check_ready(c);
  if (rc) return rc;
  if (!u || !ubar1 || !ubar0) return fail(c, ESPLIT_ERR_ARG, "null pointer");
  if (ubar0 == u || ubar0 == ubar1) return fail(c, ESPLIT_ERR_ARG, "ubar0 must not alias u or ubar1");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, ESPLIT_ERR_ARG, "dt must be positive and finite");
  if (c->prm.scheme != ESPLIT_SCHEME_SPLIT || c->dim == 1 || c->n_bslot > 0)
    return fail(c, ESPLIT_ERR_UNSUPPORTED,
                "the step reverse is built for the entropy-split scheme in 2D and 3D on periodic meshes");
  cudaSetDevice(c->device);
  cudaStream_t s = as_stream(stream);
  size_t n = (size_t)c->n_e * c->n_c * c->n_p;
  if (!c->b.vjp_work) {
    if ((rc = dalloc(c, &c->b.vjp_work, 12 * n))) return rc;
  }
  if (!c->b.node_cache) {
    if ((rc = dalloc(c, &c->b.node_cache, 3 * (size_t)c->n_e * c->n_p))) return rc;
  }
  double* W = c->b.vjp_work;
  double* Us[3] = {W, W + n, W + 2 * n};                  // U_2, U_3, U_4
  double* Rs[4] = {W + 3 * n, W + 4 * n, W + 5 * n, W + 6 * n};
  double* d = W + 7 * n;
  double* u1 = W + 8 * n;
  double* rbar = W + 9 * n;
  double* extra = W + 10 * n;
  double* Ubar = W + 11 * n;
  double* tmp = u1;  // u1 is consumed by the combine kernel before the stage loop
  static const double A[4] = {0.0, 0.5, 0.5, 1.0};
  static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  int np = 0;
  // ---- forward recompute from the checkpoint
  if (esplit::launch_entropy(c, u, s, &np, c->b.node_cache) || esplit::launch_reduce(c, c->b.partial, np, 2, c->b.scal, s))
    return fail(c, ESPLIT_ERR_CUDA, "entropy launch");
  for (int i = 0; i < 4; ++i) {
    const double* Ui = (i == 0) ? u : Us[i - 1];
    if ((rc = residual_impl(c, Ui, Rs[i], s, c->b.partial, &np))) return rc;
    if (esplit::launch_reduce(c, c->b.partial, np, 1, c->b.scal + 2 + i, s)) return fail(c, ESPLIT_ERR_CUDA, "reduce");
    if (esplit::launch_stage(c, u, Rs[i], (i < 3) ? A[i + 1] * dt : 0.0, B[i] * dt, i == 0, (i < 3) ? Us[i] : nullptr,
                             d, n, s))
      return fail(c, ESPLIT_ERR_CUDA, "stage launch");
  }
  if (esplit::launch_root_start(c, dt, s)) return fail(c, ESPLIT_ERR_CUDA, "root init");
  esplit::RootState st{};
  for (int it = 0; it < esplit::ROOT_EVALS_MAX; ++it) {
    if (esplit::launch_root_eval(c, u, d, s))
      return fail(c, ESPLIT_ERR_CUDA, "root launch");
    if ((it + 1) % esplit::ROOT_CHECK_EVERY == 0) {
      CK(cudaMemcpyAsync(&st, c->b.root, sizeof(st), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (st.done) break;
    }
  }
  CK(cudaMemcpyAsync(&st, c->b.root, sizeof(st), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int phys = read_status(c, s, true);
  if (phys) return fail(c, phys, "non-physical state during the step");
  if (st.status) return fail(c, st.status, "relaxation parameter could not be bracketed");
  const double g = st.g, est = st.est;
  if (esplit::launch_axpy(c, u, g, d, u1, n, s)) return fail(c, ESPLIT_ERR_CUDA, "axpy launch");
  // ---- reverse: implicit dependence of g, then the stages
  if (esplit::launch_rrk_vjp_dots(c, u1, d, ubar1, s, &np) ||
      esplit::launch_reduce(c, c->b.partial, np, 2, c->b.scal + 12, s))
    return fail(c, ESPLIT_ERR_CUDA, "dots launch");
  double h2[2];
  CK(cudaMemcpyAsync(h2, c->b.scal + 12, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double fg = h2[1] - est;
  if (!(fabs(fg) > 0.0)) return fail(c, ESPLIT_ERR_RRK_NO_ROOT, "f'(g) vanishes at the relaxation root");
  const double lam = -h2[0] / fg;
  double* dbar_keep = d;  // d was last read by the dots kernel: dbar reuses its storage
  if (esplit::launch_rrk_vjp_combine(c, u, u1, ubar1, lam, g, ubar0, dbar_keep, s))
    return fail(c, ESPLIT_ERR_CUDA, "combine launch");
  const double estbar = -lam * g;
  for (int i = 3; i >= 0; --i) {
    const double* Ui = (i == 0) ? u : Us[i - 1];
    double c_d = dt * B[i], c_e = dt * B[i] * estbar, c_u = (i < 3) ? A[i + 1] * dt : 0.0;
    if (esplit::launch_rrk_vjp_stage(c, Ui, Rs[i], dbar_keep, (i < 3) ? Ubar : nullptr, c_d, c_e, c_u, rbar, extra, s))
      return fail(c, ESPLIT_ERR_CUDA, "stage-reverse launch");
    if ((rc = vjp_impl(c, Ui, rbar, tmp, s))) return rc;
    if (esplit::launch_axpy(c, extra, 1.0, tmp, Ubar, n, s) || esplit::launch_axpy(c, ubar0, 1.0, Ubar, ubar0, n, s))
      return fail(c, ESPLIT_ERR_CUDA, "axpy launch");
  }
  CK(cudaStreamSynchronize(s));
  c->last_stream = s;
  if (g_out) *g_out = g;
  return ESPLIT_OK;
}

int esplit_get_status(esplit_ctx* c) {
  if (!c) return ESPLIT_ERR_ARG;
  cudaSetDevice(c->device);
  return read_status(c, c->last_stream, true);
}

const char* esplit_last_error(esplit_ctx* c) { return c ? c->err.c_str() : "null context"; }

long long esplit_launch_count(esplit_ctx* c) { return c ? c->launches : -1; }

int esplit_profile_enable(esplit_ctx* c, int on) {
  if (!c) return ESPLIT_ERR_ARG;
  c->prof = on != 0;
  return ESPLIT_OK;
}

int esplit_profile_read(esplit_ctx* c, double* ms, long long* count, int n_groups) {
  if (!c || n_groups < 0) return ESPLIT_ERR_ARG;
  cudaSetDevice(c->device);
  std::vector<double> acc(ESPLIT_PROFILE_GROUPS, 0.0);
  std::vector<long long> cnt(ESPLIT_PROFILE_GROUPS, 0);
  for (auto& r : c->recs) {
    float t = 0.f;
    CK(cudaEventSynchronize(r.b));
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    acc[r.group] += t;
    cnt[r.group] += 1;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  for (int g = 0; g < n_groups && g < ESPLIT_PROFILE_GROUPS; ++g) {
    if (ms) ms[g] = acc[g];
    if (count) count[g] = cnt[g];
  }
  return ESPLIT_OK;
}

}  // extern "C"
