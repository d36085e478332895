// Region-adaptive L-infinity bounds (host planning; declarations).
#pragma once

#include "../../include/mgard_b300.h"
#include "quantize.cuh"

namespace mgb {

// Radius rho and width exponents k[r] for background tolerance `tol` and the
// boxes' tolerances (checks the boxes against the shape as passed).
mgard_status region_params(const Plan& p, int ndim, const int64_t* shape, double tol,
                           const mgard_region* rg, int n, int* rho, int32_t* k);
// Per-level dilated boxes in the plan's 4D view from rho and k.
mgard_status region_table(const Plan& p, int ndim, const int64_t* shape, int rho, const int32_t* k,
                          const mgard_region* rg, int n, RegionScale* out);

}  // namespace mgb
