// Internal declarations shared by the C-ABI translation units.
#pragma once
#include "../../include/mujica_pm.h"
#include "sort.cuh"

// scratch of the rank-order-matching sorts: all 2 * n^2 (n/2 + 1) real
// components of a half spectrum, keys of the plan's element size
inline size_t pm_sort_workspace_bytes(const pm_config &c) {
  const int64_t n = c.n;
  const int64_t ne = 2 * n * n * (n / 2 + 1);
  return pm::sortk::scratch_bytes(ne, c.precision == PM_PREC_F64 ? 8 : 4);
}

pm_status pm_validate_config(const pm_config *c);
