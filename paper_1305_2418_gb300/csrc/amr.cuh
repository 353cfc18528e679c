// amr.cuh -- refined hierarchy (Sec. 3.1) entry points used by solver.cu.
#pragma once
#include "mgfr_internal.cuh"

void amr_free(mgfr_ctx* c);
