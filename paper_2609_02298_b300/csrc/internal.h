// Library-internal entry points shared between translation units (not exported
// in include/iblbm.h).
#pragma once

#include <stddef.h>

#include "iblbm.h"

// Batched stepping; use_graphs = 0 launches the kernels directly (for batches
// whose composition changes often, where a graph capture would not be reused).
int iblbm_internal_step_batch(iblbm_ctx** ctxs, int n, int nsteps, int use_graphs);

// Device bytes a lattice with one body of n markers (reach = largest marker
// distance from the centre) will hold once created.
size_t iblbm_internal_estimate_bytes(const iblbm_lattice_desc* d, int n, double reach, int kernel, int hist_cap);
