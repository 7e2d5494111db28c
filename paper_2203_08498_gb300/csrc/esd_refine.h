// Launchers of the FP64 refinement kernels (esd_refine.cu).
#pragma once

#include "esd_iter.h"

namespace esd {
// skip_done: leave a system whose refinement has stopped (a system of a pair) as it is
void launch_ref_residual(const IterCtx<double>& c, double* r64, const float* r32, RefineState* rs, State* st_in,
                         unsigned long long cond, cudaStream_t s, int skip_done = 0);
// the pair's refinement loop goes on (cond = 1) while either system has not stopped
void launch_pair_cond(const RefineState* rs1, const RefineState* rs2, unsigned long long cond, cudaStream_t s);
// a pair's inner loops: cond = 1 while both inner runs go on (st2 = NULL: while st1's does)
void launch_inner_cond(const State* st1, const State* st2, unsigned long long cond, cudaStream_t s);
void launch_ref_prep(int n, const double* r64, float* b32, float* x32, State* st_in, const RefineState* rs,
                     unsigned long long cond_in, cudaStream_t s);
void convert_d2f(long long cnt, const double* a, float* b, cudaStream_t s);
// FP32 slice-major copy (the layout IterCtx::wsm selects) of a column-major n x M block
void to_slice_major(int n, const int* rowpos, const double* X, size_t ld, int M, float* out, cudaStream_t s);
// b = a rounded to the nearest FP32 value (kept in FP64)
void round_to_f32(long long cnt, const double* a, double* b, cudaStream_t s);
}  // namespace esd
