// Float32 path of the entropy-split residual (precision ESPLIT_FP32): the
// inviscid split scheme of Eq. (100) with the EC SATs of Eq. (43) and the
// matrix dissipation of Eq. (69), with the fluxes, entropy variables, A~_i
// products, two-point fluxes, dissipation and operator contractions all
// evaluated in float32 on deviations (dev32.cuh).  Float64 is kept for the
// differences of the conservative states that the deviations start from, the
// accumulation of the residual and of the entropy production w^T H r, and
// everything outside the residual (the stored metric operators are formed in
// float64 and rounded once; entropy, relaxation root and update stay float64).
//
// Two kernels, one after the other on the stream:
//   face_f32_kernel: thread = coincident facet-node pair (k, m) ~ (v, n).
//     With G = nu . (F*(u_k, u_v) - F(u_k)) (sy_flux_dev32), the jump
//     df = nu . (F(u_v) - F(u_k)) and Dw = |nu|/2 X|L|SX^T (w_k - w_v):
//       H_k sat_k = -G - Dw            (= nu . F(u_k) - nu . F* - Dw)
//       H_v sat_v = G - df + Dw        (= nu . F* - nu . F(u_v) + Dw)
//     i.e. the SATs together with the facet part nu . f / H of the split
//     volume term (M_i = H^-1 E_i - beta/(beta+1) D_i), written to a float32
//     facet scratch (boundary slots: face_bc_f32_kernel).
//   split_volume_f32_kernel: thread = node, EB elements per block.  Variations
//     relative to the element's node 0, D_i = H^-1 Q_x_i applied to the
//     flux and entropy-variable variations (D_i 1 = 0 by the discrete metric
//     identity, so the node-0 values drop out; the float64 row sums of the
//     stored operators, ~eps |D_i|, are below float32 resolution):
//       r = -beta/(beta+1) sum_i D_i df_i - 1/(beta+1) sum_i A~_i(u) (D_i dw) + sat
//     stored to r (float64).
// The float64 <-> float32 conversions (state differences, stores) go through
// integer operations on the bit patterns (bits32.cuh), 1/(H J) through a
// float32 table: the float64 pipe does only the states' exponent checks.
// Entropy production (when requested): block partials of sum H w . r, per node
// in float32 with w the reference's W plus its variation, summed in float64.
#include <cuda_runtime.h>

#include "dev32.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "tma.cuh"

namespace esplit {

__constant__ RefTables c_ref32;

int set_ref_tables_f32(const RefTables& t) {
  return cudaMemcpyToSymbol(c_ref32, &t, sizeof(RefTables)) == cudaSuccess ? 0 : -1;
}

// s + a b with Kahan compensation: y = a b - c (one rounding), t = s + y,
// c = (t - s) - y (the part of y that t lost), s = t
__device__ __forceinline__ void kahan_fma(float a, float b, float& s, float& c) {
  const float y = __fmaf_rn(a, b, -c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// Dw = |nu|/2 X|L|SX^T (w_k - w_v) of Eq. (69) from the float32 pair averages
// and entropy-variable jump
template <int D>
__device__ __forceinline__ void diss32(const PairAvg<float, D>& a, const Phys<float>& c, const float* nuv,
                                       const float* mdw, float* Dw) {
  float b2 = 0.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) b2 += nuv[i] * nuv[i];
  const float b = sqrtf(b2);
  const float ib = 1.0f / b;
  float nh[D], o[D + 2];
#pragma unroll
  for (int i = 0; i < D; ++i) nh[i] = nuv[i] * ib;
  diss_apply<float, D>(a, c, nh, mdw, o);
#pragma unroll
  for (int q = 0; q < D + 2; ++q) Dw[q] = 0.5f * b * o[q];
}

// Variations of the element's nodes, one float4 per node and direction (the
// n_c <= 4 components of lines and triangles; unused lanes zero), rows padded
// to NPP with zeros and each element by one float4, so that the lanes of two
// elements in a warp read different bank groups.
template <int D, int NP, int EB>
struct SplitSmem32 {
  static constexpr int NPP = npp_for(NP);
  float4 df[EB][D * NPP + 1];  // flux variations: df[el][i * NPP + n]
  float4 dw[EB][NPP + 1];      // entropy-variable variations
  double u0[EB][D + 2];        // node-0 states
  uint64_t bar;                // completion barrier of the operators' bulk copy
};

__device__ __forceinline__ float4 f4(const float* v, int nc) {
  return make_float4(v[0], v[1], v[2], nc > 3 ? v[3] : 0.0f);
}

// acc += a f (four components), plain or Kahan-compensated
template <bool COMP>
__device__ __forceinline__ void fma4(float a, const float4& f, float4& acc, float4& cmp) {
  if constexpr (COMP) {
    kahan_fma(a, f.x, acc.x, cmp.x);
    kahan_fma(a, f.y, acc.y, cmp.y);
    kahan_fma(a, f.z, acc.z, cmp.z);
    kahan_fma(a, f.w, acc.w, cmp.w);
  } else {
    acc.x = fmaf(a, f.x, acc.x);
    acc.y = fmaf(a, f.y, acc.y);
    acc.z = fmaf(a, f.z, acc.z);
    acc.w = fmaf(a, f.w, acc.w);
  }
}

// acc = sum_i D_i df_i, g_i = D_i dw at node m of element el, from the
// element's D_i rows opr[(i NP + m) NPP + n] (shared memory, or global memory
// when SMEM is false): per 16-byte load of four row entries, eight 16-byte
// broadcast loads of the variations and 32 FMAs.  For operators above 20
// nodes the sums are Kahan-compensated: the rounding of partial sums much
// larger than the final, cancelling, result dominated the error there.
template <bool SMEM, int D, int NP, int EB>
__device__ __forceinline__ void contract32(const float* __restrict__ opr, const SplitSmem32<D, NP, EB>& sm, int el,
                                           int m, float4& acc, float4 (&g)[D]) {
  constexpr int NPP = SplitSmem32<D, NP, EB>::NPP;
  constexpr bool COMP = NP > 20;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 cacc = z, cg[D];
  acc = z;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    g[i] = z;
    cg[i] = z;
    const float4* row = reinterpret_cast<const float4*>(opr + (i * NP + m) * NPP);
#pragma unroll 1
    for (int nb = 0; nb < NPP / 4; ++nb) {
      const float4 a = SMEM ? row[nb] : __ldg(&row[nb]);
      const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int n = 4 * nb + t;
        fma4<COMP>(av[t], sm.df[el][i * NPP + n], acc, cacc);
        fma4<COMP>(av[t], sm.dw[el][n], g[i], cg[i]);
      }
    }
  }
  if constexpr (COMP) {
    acc.x = __fsub_rn(acc.x, cacc.x);
    acc.y = __fsub_rn(acc.y, cacc.y);
    acc.z = __fsub_rn(acc.z, cacc.z);
    acc.w = __fsub_rn(acc.w, cacc.w);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      g[i].x = __fsub_rn(g[i].x, cg[i].x);
      g[i].y = __fsub_rn(g[i].y, cg[i].y);
      g[i].z = __fsub_rn(g[i].z, cg[i].z);
      g[i].w = __fsub_rn(g[i].w, cg[i].w);
    }
  }
}

// STAGE: the block's operators (one contiguous range of opsD) are brought
// into shared memory by one bulk copy at the start, overlapping the pointwise
// phase; the contraction then reads them there.
template <int D, int NP, int EB, bool STAGE>
__global__ void __launch_bounds__(EB * NP, 4) split_volume_f32_kernel(
    const double* __restrict__ u, double* __restrict__ r, const float* __restrict__ opsD, int opsD_stride, const float* __restrict__ ihf, const float* __restrict__ satf,
    int n_e, Phys<float> c, int* __restrict__ status, double* __restrict__ prod) {
  constexpr int NC = D + 2;
  constexpr int NPP = SplitSmem32<D, NP, EB>::NPP;
  static_assert(NC <= 4, "one float4 per node and direction");
  __shared__ SplitSmem32<D, NP, EB> sm;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  const int NS = c_ref32.n_slot;
  const int el = threadIdx.x / NP;
  const int m = threadIdx.x - el * NP;
  const int e = blockIdx.x * EB + el;
  const bool active = (el < EB) && (e < n_e);
  float* ops_sm = reinterpret_cast<float*>(dyn_smem);
  if constexpr (STAGE) {
    if (threadIdx.x == 0) mbar_init(&sm.bar);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int e0 = blockIdx.x * EB;
      const uint32_t bytes = (uint32_t)(min(EB, n_e - e0) * opsD_stride) * 4u;
      mbar_expect_tx(&sm.bar, bytes);
      bulk_load(ops_sm, opsD + (size_t)e0 * opsD_stride, bytes, &sm.bar);
    }
  }
  double uu[NC];
  if (active) {
#pragma unroll
    for (int q = 0; q < NC; ++q) uu[q] = __ldg(&u[((size_t)e * NC + q) * NP + m]);
    if (m == 0) {
#pragma unroll
      for (int q = 0; q < NC; ++q) sm.u0[el][q] = uu[q];
    }
  }
  __syncthreads();
  Ref32<D> rf;
  Dev32<D> dv;
  float du[NC];
  if (active) {
    float u0f[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double u0 = sm.u0[el][q];
      u0f[q] = f32_round(u0);
      du[q] = f32_diff(uu[q], u0);
    }
    ref32_from_u<D>(u0f, c, rf);
    dev32<D>(rf, du, c, dv);
    if (!(dv.rho1 > 0.0f && dv.p1 > 0.0f && isfinite(dv.e1) && rf.rho > 0.0f && rf.p > 0.0f)) atomicOr(status, 1);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float F[NC];
      dflux32<D>(rf, du, dv, i, F);
      sm.df[el][i * NPP + m] = f4(F, NC);
    }
    sm.dw[el][m] = f4(dv.dW, NC);
    // zero rows for the padding nodes NP..NPP-1 (their operator entries are 0)
    for (int pz = m; pz < NPP - NP; pz += NP) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int i = 0; i < D; ++i) sm.df[el][i * NPP + NP + pz] = z;
      sm.dw[el][NP + pz] = z;
    }
  }
  __syncthreads();
  bool staged = false;
  if constexpr (STAGE) {
    staged = mbar_wait(&sm.bar, 0);
    if (!staged) {
      // report, wait (bounded) for the copy still in flight into this block's
      // shared memory, and contract from global memory instead
      atomicOr(status, 4);
      mbar_wait(&sm.bar, 0);
    }
  }
  double hw = 0.0;
  if (active) {
    float4 acc4, g4[D];
    if (staged)
      contract32<true, D, NP, EB>(ops_sm + (size_t)el * opsD_stride, sm, el, m, acc4, g4);
    else
      contract32<false, D, NP, EB>(opsD + (size_t)e * opsD_stride, sm, el, m, acc4, g4);
    float acc[NC], g[D][NC];
    {
      const float a4[4] = {acc4.x, acc4.y, acc4.z, acc4.w};
#pragma unroll
      for (int q = 0; q < NC; ++q) acc[q] = a4[q];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const float b4[4] = {g4[i].x, g4[i].y, g4[i].z, g4[i].w};
#pragma unroll
        for (int q = 0; q < NC; ++q) g[i][q] = b4[q];
      }
    }
    Node<float, D> nd;
    node32<D>(rf, dv, nd);
    const JvpPrep<float> jp = jvp_prep<float, D>(nd, c);
    float nonc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) nonc[q] = 0.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float dF[NC];
      dflux_dw<float, D>(nd, jp, c, i, g[i], dF);
#pragma unroll
      for (int q = 0; q < NC; ++q) nonc[q] += dF[q];
    }
    const float kf = c.beta * c.inv_bp1;
    const int sl = c_ref32.node_slot[m];
    float hwf = 0.0f;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const float rv = -kf * acc[q] - c.inv_bp1 * nonc[q];
      hwf = fmaf(nd.W[q], rv, hwf);
      // the facet terms (written by the facet kernel, which ran first)
      const float rt = sl >= 0 ? rv + __ldg(&satf[((size_t)e * NC + q) * NS + sl]) : rv;
      r[((size_t)e * NC + q) * NP + m] = widen_f32(rt);
    }
    // entropy production of the volume part, H w . r (the facet kernel adds
    // its part): per node in float32, summed in float64
    if (prod) hw = widen_f32(__fdiv_rn(hwf, __ldg(&ihf[(size_t)e * NP + m])));
  }
  if (prod) {
    double v[1] = {hw};
    block_sum<1>(v, prod + blockIdx.x);
  }
}

template <int D>
__global__ void __launch_bounds__(128) face_f32_kernel(float* __restrict__ satf, const double* __restrict__ u,
                                                       const int2* __restrict__ fp, int n_pairs,
                                                       const double* __restrict__ nu, const float* __restrict__ ihf,
                                                       Phys<float> c, int dissipation, int* __restrict__ status,
                                                       double* __restrict__ prod) {
  constexpr int NC = D + 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double hw = 0.0;
  if (t < n_pairs) {
    const int NP = c_ref32.n_p, NS = c_ref32.n_slot;
    const int2 pr = __ldg(&fp[t]);
    const int k = pr.x / NS, s = pr.x - k * NS;
    const int v = pr.y / NS, s2 = pr.y - v * NS;
    const int m = c_ref32.slot_node[s], n = c_ref32.slot_node[s2];
    float ukf[NC], du[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double a = __ldg(&u[((size_t)k * NC + q) * NP + m]);
      ukf[q] = f32_round(a);
      du[q] = f32_diff(__ldg(&u[((size_t)v * NC + q) * NP + n]), a);
    }
    Ref32<D> rk;
    Dev32<D> dv;
    ref32_from_u<D>(ukf, c, rk);
    dev32<D>(rk, du, c, dv);
    if (!(rk.rho > 0.0f && rk.p > 0.0f && dv.rho1 > 0.0f && dv.p1 > 0.0f && isfinite(dv.e1))) atomicOr(status, 1);
    float nuv[D];
#pragma unroll
    for (int i = 0; i < D; ++i) nuv[i] = f32_round(__ldg(&nu[((size_t)k * NS + s) * D + i]));
    float G[NC], df[NC], Dw[NC];
    PairAvg<float, D> a;
    sy_flux_dev32<D>(rk, dv, c, nuv, G, a);
    dflux32_dir<D>(rk, du, dv, nuv, df);
#pragma unroll
    for (int q = 0; q < NC; ++q) Dw[q] = 0.0f;
    if (dissipation) {
      float mdw[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) mdw[q] = -dv.dW[q];  // w_k - w_v
      diss32<D>(a, c, nuv, mdw, Dw);
    }
    const float ihk = __ldg(&ihf[(size_t)k * NP + m]);
    const float ihv = __ldg(&ihf[(size_t)v * NP + n]);
    float hwf = 0.0f;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const float gk = -G[q] - Dw[q];
      const float gv = G[q] - df[q] + Dw[q];
      satf[((size_t)k * NC + q) * NS + s] = gk * ihk;
      satf[((size_t)v * NC + q) * NS + s2] = gv * ihv;
      hwf = fmaf(rk.W[q], gk, fmaf(rk.W[q] + dv.dW[q], gv, hwf));
    }
    if (prod) hw = widen_f32(hwf);
  }
  if (prod) {
    double vv[1] = {hw};
    block_sum<1>(vv, prod + blockIdx.x);
  }
}

// boundary facet slots (pair (-1, -1)): the terms of face_f32_kernel for
// side k alone, the exterior state u_b in place of the neighbour's, into the
// facet scratch:  H_k sat_k = -G - Dw,  G = nu . (F*(u_k, u_b) - F(u_k)),
// Dw = |nu|/2 X|L|SX^T (w_k - w_b)
template <int D>
__global__ void __launch_bounds__(128) face_bc_f32_kernel(float* __restrict__ satf, const double* __restrict__ u,
                                                          const int* __restrict__ bslot,
                                                          const double* __restrict__ bstate, int n_b,
                                                          const double* __restrict__ nu,
                                                          const float* __restrict__ ihf, Phys<float> c,
                                                          int dissipation, int* __restrict__ status,
                                                          double* __restrict__ prod) {
  constexpr int NC = D + 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double hw = 0.0;
  if (t < n_b) {
    const int NP = c_ref32.n_p, NS = c_ref32.n_slot;
    const int a = __ldg(&bslot[t]);
    const int k = a / NS, s = a - k * NS;
    const int m = c_ref32.slot_node[s];
    float ukf[NC], du[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double x = __ldg(&u[((size_t)k * NC + q) * NP + m]);
      ukf[q] = f32_round(x);
      du[q] = f32_diff(__ldg(&bstate[(size_t)t * NC + q]), x);
    }
    Ref32<D> rk;
    Dev32<D> dv;
    ref32_from_u<D>(ukf, c, rk);
    dev32<D>(rk, du, c, dv);
    if (!(rk.rho > 0.0f && rk.p > 0.0f && dv.rho1 > 0.0f && dv.p1 > 0.0f && isfinite(dv.e1))) atomicOr(status, 1);
    float nuv[D];
#pragma unroll
    for (int i = 0; i < D; ++i) nuv[i] = f32_round(__ldg(&nu[((size_t)k * NS + s) * D + i]));
    float G[NC], Dw[NC];
    PairAvg<float, D> av;
    sy_flux_dev32<D>(rk, dv, c, nuv, G, av);
#pragma unroll
    for (int q = 0; q < NC; ++q) Dw[q] = 0.0f;
    if (dissipation) {
      float mdw[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) mdw[q] = -dv.dW[q];
      diss32<D>(av, c, nuv, mdw, Dw);
    }
    const float ihk = __ldg(&ihf[(size_t)k * NP + m]);
    float hwf = 0.0f;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const float gk = -G[q] - Dw[q];
      satf[((size_t)k * NC + q) * NS + s] = gk * ihk;
      hwf = fmaf(rk.W[q], gk, hwf);
    }
    if (prod) hw = widen_f32(hwf);
  }
  if (prod) {
    double vv[1] = {hw};
    block_sum<1>(vv, prod + blockIdx.x);
  }
}

template <int D, int NP>
static int split_f32_np(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* prod, int* n_partial,
                        float* satf) {
  constexpr int EB = (256 / NP) > 0 ? (256 / NP) : 1;
  const Phys<float> ph = make_phys<float>(c->prm.gam, c->prm.beta, c->prm.R, c->prm.mu, c->prm.Pr);
  int np_used = 0;
  {
    // facet terms first, into the float32 facet scratch the volume kernel adds
    const int bs = 128, nb = (c->n_pairs + bs - 1) / bs;
    ProfScope ps(c, PG_FACE, s);
    face_f32_kernel<D><<<nb, bs, 0, s>>>(satf, u, c->b.face_pairs, c->n_pairs, c->b.nu, c->b.ihf, ph,
                                         c->prm.dissipation, c->b.status, prod);
    c->launches++;
    if (prod) np_used += nb;
  }
  if (c->n_bslot > 0) {
    const int bs = 128, nb = (c->n_bslot + bs - 1) / bs;
    ProfScope ps(c, PG_FACE, s);
    face_bc_f32_kernel<D><<<nb, bs, 0, s>>>(satf, u, c->b.bslot, c->b.bstate, c->n_bslot, c->b.nu, c->b.ihf, ph,
                                            c->prm.dissipation, c->b.status, prod ? prod + np_used : nullptr);
    c->launches++;
    if (prod) np_used += nb;
  }
  {
    const int nb = (c->n_e + EB - 1) / EB;
    ProfScope ps(c, PG_SPLIT, s);
    constexpr bool STAGE = true;
    const size_t dyn = STAGE ? (size_t)EB * c->opsD_stride * sizeof(float) : 0;
    if (STAGE) {
      // static + dynamic shared memory above 48 KB needs the opt-in
      static size_t attr_set = 0;
      if (attr_set < dyn) {
        cudaFuncSetAttribute(split_volume_f32_kernel<D, NP, EB, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn);
        attr_set = dyn;
      }
    }
    split_volume_f32_kernel<D, NP, EB, STAGE><<<nb, EB * NP, dyn, s>>>(
        u, r, c->b.opsD32, c->opsD_stride, c->b.ihf, satf, c->n_e, ph, c->b.status,
        prod ? prod + np_used : nullptr);
    c->launches++;
    if (prod) np_used += nb;
  }
  if (n_partial) *n_partial = np_used;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_split_f32(esplit_ctx* c, const double* u, double* r, cudaStream_t s, double* prod, int* n_partial,
                     double* scratch) {
  // the float32 facet scratch [n_e][n_c][n_slot] lives in the first half of
  // the float64 facet scratch (the context's, or the static one of the
  // no-allocation entry point)
  float* satf = reinterpret_cast<float*>(scratch);
  if (c->dim == 1) {
    switch (c->n_p) {
      case 2: return split_f32_np<1, 2>(c, u, r, s, prod, n_partial, satf);
      case 3: return split_f32_np<1, 3>(c, u, r, s, prod, n_partial, satf);
      case 4: return split_f32_np<1, 4>(c, u, r, s, prod, n_partial, satf);
      case 5: return split_f32_np<1, 5>(c, u, r, s, prod, n_partial, satf);
    }
  } else if (c->dim == 2) {
    switch (c->n_p) {
      case 7: return split_f32_np<2, 7>(c, u, r, s, prod, n_partial, satf);
      case 12: return split_f32_np<2, 12>(c, u, r, s, prod, n_partial, satf);
      case 18: return split_f32_np<2, 18>(c, u, r, s, prod, n_partial, satf);
      case 27: return split_f32_np<2, 27>(c, u, r, s, prod, n_partial, satf);
    }
  }
  return -2;  // tetrahedra take the FP32-bulk kernels
}

}  // namespace esplit
