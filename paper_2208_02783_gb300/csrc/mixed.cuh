// Mixed-precision solver entry (complex FP32 iteration inside FP64 refinement).
#pragma once

#include "engine.cuh"

namespace transec {

// Solve nitems (E, k, column) items: device item / result arrays, as run_plain.
int run_mixed(transec_ctx* ctx, int H, int nitems, const double* d_e, const int* d_ik,
              const long long* d_col, double* d_t, double* d_tm, int* d_it, int* d_st);

}  // namespace transec
