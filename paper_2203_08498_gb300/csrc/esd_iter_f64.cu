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

// Rayleigh-quotient pass of the power vector (Section 5.4): ||w||^2 and (w, A w).
__global__ void __launch_bounds__(kBlock, 4) k_power_rq(SellView<double> Av, SliceSet set, const double* w0,
                                                      const double* w1, PowerState* ps, double* partials,
                                                      int set_scale) {
  constexpr int R = 2;
  __shared__ double red[red_size<R>()];
  pdl_enter();
  const double* w = (ps->steps & 1) ? w1 : w0;
  double acc[R] = {0.0, 0.0};
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = Av.meta[s];
    const double awi = row_fma(Av, md, lane, w, 0.0);
    if (lane < md.w) {
      const double wi = w[md.z + lane];
      acc[0] = fma(wi, wi, acc[0]);
      acc[1] = fma(wi, awi, acc[1]);
    }
  }
  if (grid_sum_multi<R>(acc, red, partials, &ps->ticket)) {
    if (threadIdx.x == 0) {
      ps->ww = red[0];
      ps->wAw = red[1];
      if (set_scale) {  // a new start vector v_0 = w / ||w||
        const bool ok = red[0] > 0.0 && isfinite(red[0]);
        ps->scale = ok ? 1.0 / sqrt(red[0]) : 0.0;
        ps->failed = ok ? 0 : 1;
        ps->steps = 0;
      }
    }
  }
}

// unit = w / ||w|| with ||w||^2 from the preceding k_power_rq
__global__ void __launch_bounds__(kBlock) k_power_unit(int n, const double* w, const PowerState* ps, double* unit) {
  const double sc = 1.0 / sqrt(ps->ww);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) unit[i] = w[i] * sc;
}

void launch_power_rq(const esd_matrix* A, double* const pw[2], PowerState* ps, double* partials, int set_scale,
                     cudaStream_t s) {
  auto k = k_power_rq;
  ESD_LAUNCH(k, A->all.total(), s, A->A.view<double>(), A->all, (const double*)pw[0], (const double*)pw[1], ps,
             partials, set_scale);
}

void launch_power_unit(const esd_matrix* A, const double* w, const PowerState* ps, double* unit, cudaStream_t s) {
  k_power_unit<<<max_grid_blocks(), kBlock, 0, s>>>(A->n, w, ps, unit);
  ESD_CUDA(cudaGetLastError());
}

// Largest binary exponent of each column of AW or W (n x m, column-major, stride ld).
__global__ void k_aw_colexp(int n, const double* AW, size_t ld, int* cexp) {
  const int k = blockIdx.y;
  int e = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    e = max(e, dexp(AW[(size_t)k * ld + i]));
  e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
  if ((threadIdx.x & 31) == 0 && e > 0) atomicMax(&cexp[k], e);
}

// X 2^-e_k (X = AW or W) as double-float pairs in slice-major order; scale[k] = 2^e_k (1 for a
// zero or padding column)
__global__ void k_aw_df(int n, const int* rowpos, const double* AW, size_t ld, int m, int M, const int* cexp,
                        float2* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int pos = rowpos[i];
    const size_t base = (size_t)(pos >> 5) * M * kSlice + (pos & 31);
    for (int k = 0; k < m; ++k) {
      float h, l;
      df_split(AW[(size_t)k * ld + i], cexp[k], h, l);
      out[base + (size_t)k * kSlice] = make_float2(h, l);
    }
  }
}

__global__ void k_aw_scale(int M, const int* cexp, double* awscale) {
  for (int k = threadIdx.x; k < M; k += blockDim.x) awscale[k] = dpow2(cexp[k] > 0 ? cexp[k] : 1023);
}

void launch_df_pairs(const esd_matrix* A, const double* AW, size_t ld, int m, int M, float2* out, double* awscale,
                     int* cexp, cudaStream_t s) {
  ESD_CUDA(cudaMemsetAsync(cexp, 0, sizeof(int) * kMaxM, s));
  ESD_CUDA(cudaMemsetAsync(out, 0, sizeof(float2) * (size_t)A->nslices * kSlice * M, s));
  if (m > 0) {
    k_aw_colexp<<<dim3(std::min((A->n + 255) / 256, 2 * max_grid_blocks()), m), 256, 0, s>>>(A->n, AW, ld, cexp);
    ESD_CUDA(cudaGetLastError());
    k_aw_df<<<std::min((A->n + 255) / 256, 4 * max_grid_blocks()), 256, 0, s>>>(A->n, A->rowpos.as<int>(), AW, ld, m,
                                                                               M, cexp, out);
    ESD_CUDA(cudaGetLastError());
  }
  k_aw_scale<<<1, 64, 0, s>>>(M, cexp, awscale);
  ESD_CUDA(cudaGetLastError());
}

void launch_true_residual(const IterCtx<double>& c, cudaStream_t s) {
  auto k = k_true_res<double>;
  ESD_LAUNCH(k, c.A->all.total(), s, c, c.A->all);
}

}  // namespace esd
