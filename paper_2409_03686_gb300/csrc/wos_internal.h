// wos_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "wos.h"

namespace wos {

wos_status cuda_status(cudaError_t e);
int ctx_device(const wos_context *c);
int ctx_sm_count(const wos_context *c);
void count_launches(wos_context *c, int n);

}  // namespace wos
