// Reverse mode of the residual (split scheme with EC SATs, matrix dissipation
// and the Baumann-Oden viscous terms) and of one relaxation RK4 step, in a
// translation unit of its own (compiled in parallel with kernels.cu).
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.h"
#include "phys.cuh"
#include "visc_flux.cuh"
#include "reduce.cuh"

namespace esplit {

// this unit's copy of the reference-operator tables (set_ref_tables fills it)
static __constant__ RefTables c_ref;

int set_ref_tables_vjp(const RefTables& t) {
  return cudaMemcpyToSymbol(c_ref, &t, sizeof(RefTables)) == cudaSuccess ? 0 : -1;
}

}  // namespace esplit

#include "vjp.cuh"
#include "visc_vjp.cuh"
#include "rrk_vjp.cuh"
