#include "amr.cuh"
void amr_free(mgfr_ctx*) {}
