// Library-internal host functions shared between translation units (not
// part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/turbofft.h"

namespace tf {

// Intermediate bytes a two-pass exec of this plan needs (0 for one pass).
size_t plan_scratch_bytes(const turbofft_plan* plan);
// Device the plan was created on.
int plan_device(const turbofft_plan* plan);
// Record a failure message on the plan (turbofft_last_error).
void plan_set_error(turbofft_plan* plan, const char* msg);
// turbofft_exec with the two-pass intermediate at `scratch` (ignored for
// one-pass plans); allocates nothing.
turbofft_status exec_given_scratch(turbofft_plan* plan, const void* in, void* out, void* scratch,
                                   cudaStream_t stream);

}  // namespace tf
