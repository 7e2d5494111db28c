// FP64 instantiation of the iteration kernels, plus the FP64-only helpers (SpMV entry,
// preconditioner application, A W, the backward-Euler right-hand side, true residual).
#include "esd_iter.cuh"

namespace esd {

ESD_INSTANTIATE_ITER(double)

int pad_m(int m) {
  if (m <= 0) return 0;
  if (m <= 8) return 8;
  if (m <= 16) return 16;
  if (m <= 24) return 24;
  if (m <= 32) return 32;
  return 64;
}

void launch_spmv(const esd_matrix* A, const double* x, double* y, cudaStream_t s) {
  auto k = k_spmv<double>;
  ESD_LAUNCH(k, A->all.total(), s, A->A.view<double>(), A->all, x, y);
}

void launch_apply_ic(const esd_matrix* A, const double* r, double* z, double* work, cudaStream_t s) {
  const double* inv_d = A->inv_d.as<double>();
  auto kf = k_fwd_plain<double>;
  auto kb = k_bwd_plain<double>;
  for (const SliceSet& set : A->fwd_all_sets) ESD_LAUNCH(kf, set.total(), s, A->L.view<double>(), set, r, work, inv_d);
  for (const SliceSet& set : A->bwd_all_sets) ESD_LAUNCH(kb, set.total(), s, A->U.view<double>(), set, (const double*)work, z, inv_d);
}

void launch_spmm(const esd_matrix* A, const double* X, double* Y, size_t ld, int m, cudaStream_t s) {
  for (int j = 0; j < m; ++j) launch_spmv(A, X + (size_t)j * ld, Y + (size_t)j * ld, s);
}

__global__ void k_axpby(int n, const double* x, double a, const double* sv, double* b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    b[i] = fma(x[i], a, sv[i]);
}

void launch_axpby(int n, const double* x, double a, const double* sv, double* b, cudaStream_t s) {
  k_axpby<<<max_grid_blocks(), kBlock, 0, s>>>(n, x, a, sv, b);
  ESD_CUDA(cudaGetLastError());
}

void launch_true_residual(const IterCtx<double>& c, cudaStream_t s) {
  auto k = k_true_res<double>;
  ESD_LAUNCH(k, c.A->all.total(), s, c, c.A->all);
}

}  // namespace esd
