// FP64 iterative refinement around FP32 inner PCG solves (the precision form): the FP64
// residual and the conversion of a refinement step's right-hand side to FP32. The inner
// solve is the FP32 instantiation of the iteration kernels; it adds its steps alpha p to
// the FP64 iterate directly (x += d in FP64 as it goes), so no rounding of an FP32 iterate
// separates x from the recursive residual.
//
// Two forms of the step. Restart: every inner solve is a fresh PCG run on A d = r.
// Resume (residual replacement, after van der Vorst & Ye, SIAM J. Sci. Comput. 22, 2000):
// the inner CG state (p, rho, iteration count, sampling schedule) carries over and only the
// residual is replaced by the FP64 one. An inner run stops right after its x, r update, so
// the start pass of the next run is the rest of that iteration on the replaced residual:
// z = M^-1 r, beta = (r, z) / rho, p = z + beta p. The steps together are one CG run whose
// residual is refreshed in FP64 whenever it has dropped by inner_tol.
#include "esd_iter.cuh"
#include "esd_refine.h"

namespace esd {

// r = b - A x in FP64, ||b||^2, ||r||^2 and, after a step, ||r - r_inner||^2 (the drift of
// the inner recursive residual r32 from the true one). The last block books the step that
// has just been applied (st_in != NULL: its inner iterations), decides whether the next
// resumed step must restart its direction (drift above half the residual, so the kept p no
// longer belongs to this residual, or a step that cut the true residual by less than 10%)
// and whether refinement goes on (stops when ||r|| <= tol ||b||, b = 0, or max_outer
// steps are done).
//
// skip_done (a system of a pair): a system whose refinement has already stopped is left as it is.
__global__ void __launch_bounds__(kBlock, 4) k_ref_residual(IterCtx<double> c, SliceSet set, double* r64,
                                                             const float* r32, RefineState* rs, State* st_in,
                                                             unsigned long long cond, int skip_done) {
  __shared__ double red[red_size<3>()];
  if (skip_done && rs->conv) return;
  double acc[3] = {0.0, 0.0, 0.0};
  const bool gap = st_in != nullptr;
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    const bool valid = lane < md.w;
    const int iv = md.z + lane;
    // A x in the difference form: its rounding error scales with |A x|, not |A| |x|, which
    // lowers the floor the refinement can reach on stiff problems
    const double ax = c.rowsum ? row_fma_diff(c.Av, md, lane, c.x, valid ? c.x[iv] : 0.0, valid ? c.rowsum[iv] : 0.0, 0.0)
                               : row_fma(c.Av, md, lane, c.x, 0.0);
    if (valid) {
      const int i = iv;
      const double bi = c.b[i];
      const double ri = bi - ax;
      r64[i] = ri;
      acc[0] = fma(bi, bi, acc[0]);
      acc[1] = fma(ri, ri, acc[1]);
      if (gap) {
        const double di = ri - (double)r32[i];
        acc[2] = fma(di, di, acc[2]);
      }
    }
  }
  if (grid_sum_multi<3>(acc, red, (double*)c.partials, &rs->ticket)) {
    if (threadIdx.x == 0) {
      if (st_in) {
        if (rs->outer == 0) rs->first_inner = st_in->iter;
        rs->inner_total = rs->keep ? st_in->iter : rs->inner_total + st_in->iter;
        rs->outer += 1;
        const double g2 = red[1] > 0.0 ? red[2] / red[1] : 0.0;
        rs->max_gap = fmax(rs->max_gap, sqrt(g2));
        // an inner breakdown ((p, P^T A p) or rho not positive in FP32) also restarts: the
        // step's x is the last good iterate, and p = z gives a clean direction again
        const bool broke = st_in->status == ESD_ERR_BREAKDOWN || st_in->status == ESD_ERR_INTERNAL;
        rs->fresh = rs->keep && (broke || g2 > 0.25 || red[1] > 0.81 * rs->rr);
        if (red[1] < 0.81 * rs->rr_best) {
          rs->rr_best = red[1];
          rs->stalled = 0;
        } else {
          rs->stalled += 1;
        }
        rs->restarts += rs->fresh;
        rs->breakdowns += broke;
      }
      const double bb = red[0], rr = red[1];
      if (!st_in) {
        rs->rr_best = rr;
        rs->stalled = 0;
      }
      rs->bb = bb;
      rs->rr = rr;
      rs->tol2bb = c.st->scal0 * bb;  // the outer tolerance^2 travels in the outer state's scal0
      bool stop = false;
      if (!(rr == rr) || !(bb == bb)) {
        rs->status = ESD_ERR_BREAKDOWN;
        rs->nonfinite = 1;
        stop = true;
      } else if (bb == 0.0 || rr <= rs->tol2bb) {
        stop = true;
      } else if (st_in && rs->keep && st_in->status == ESD_ERR_MAXIT) {
        // the iteration limit of a resumed run counts all its steps
        rs->status = ESD_ERR_MAXIT;
        stop = true;
      } else if (st_in && rs->stalled >= 4) {
        // four steps in a row without a 10% gain: the residual has reached the floor that
        // its own FP64 rounding allows
        rs->status = ESD_ERR_MAXIT;
        stop = true;
      } else if (rs->outer >= rs->max_outer) {
        rs->status = ESD_ERR_MAXIT;
        stop = true;
      }
      if (stop) {
        rs->conv = 1;
        if (st_in && st_in->defer_sample && st_in->pend_slot >= 0) {
          // no run follows: the last claimed slot keeps its earlier sample
          st_in->slot_iter[st_in->pend_slot] = st_in->pend_prev;
          st_in->pend_slot = -1;
        }
        if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
      }
    }
  }
}

// b32 = (float) r, x32 = 0; block 0 sets up the inner solve (fresh, or resumed) and opens
// its loop. The inner tolerance is inner_tol relative to ||r||, but never tighter than half
// of what the outer tolerance still asks for. A system of a pair whose refinement has stopped
// gets a stopped inner solve instead (the pair's inner kernels skip it).
__global__ void __launch_bounds__(kBlock, 4) k_ref_prep(int n, const double* r64, float* b32, float* x32,
                                                         State* st_in, const RefineState* rs,
                                                         unsigned long long cond_in) {
  if (rs->conv) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st_in->conv = 1;
    return;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    b32[i] = (float)r64[i];
    x32[i] = 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool first = rs->outer == 0;
    const bool resume = rs->keep && !first;
    if (!resume) {
      st_in->iter = 0;
      st_in->samp_m = first ? rs->samp_m : 0;
      st_in->h = 1;
      st_in->pend_slot = -1;
      st_in->rho = st_in->rho_acc = st_in->fu = 0.0;
      if (first)
        for (int k = 0; k < kMaxM; ++k) st_in->slot_iter[k] = 0;
    }
    st_in->defer_sample = rs->keep;
    st_in->fresh_dir = resume && rs->fresh;
    st_in->conv = 0;
    st_in->status = ESD_OK;
    st_in->zero_rhs = 0;
    st_in->guard = 0;
    st_in->maxit = rs->inner_maxit;
    st_in->lmax = rs->lmax;
    st_in->scal0 = fmax(rs->inner_tol2, 0.25 * rs->tol2bb / rs->rr);
    if (cond_in) cudaGraphSetConditional((cudaGraphConditionalHandle)cond_in, 1u);
  }
}

void launch_ref_residual(const IterCtx<double>& c, double* r64, const float* r32, RefineState* rs, State* st_in,
                         unsigned long long cond, cudaStream_t s, int skip_done) {
  const SliceSet& all = c.A->all;
  k_ref_residual<<<grid_for(k_ref_residual, all.total()), kBlock, 0, s>>>(c, all, r64, r32, rs, st_in, cond,
                                                                         skip_done);
  ESD_CUDA(cudaGetLastError());
}

// The loop of a pair of refinements goes on while either system has not stopped.
__global__ void k_pair_cond(const RefineState* rs1, const RefineState* rs2, unsigned long long cond) {
  cudaGraphSetConditional((cudaGraphConditionalHandle)cond, (rs1->conv && rs2->conv) ? 0u : 1u);
}

void launch_pair_cond(const RefineState* rs1, const RefineState* rs2, unsigned long long cond, cudaStream_t s) {
  k_pair_cond<<<1, 1, 0, s>>>(rs1, rs2, cond);
  ESD_CUDA(cudaGetLastError());
}

// The inner loops of a pair: the paired one runs while both inner runs go on (both = 1), a
// single one while its system's does (st2 = NULL).
__global__ void k_inner_cond(const State* st1, const State* st2, unsigned long long cond) {
  const bool go = !st1->conv && (st2 == nullptr || !st2->conv);
  cudaGraphSetConditional((cudaGraphConditionalHandle)cond, go ? 1u : 0u);
}

void launch_inner_cond(const State* st1, const State* st2, unsigned long long cond, cudaStream_t s) {
  k_inner_cond<<<1, 1, 0, s>>>(st1, st2, cond);
  ESD_CUDA(cudaGetLastError());
}

void launch_ref_prep(int n, const double* r64, float* b32, float* x32, State* st_in, const RefineState* rs,
                     unsigned long long cond_in, cudaStream_t s) {
  k_ref_prep<<<max_grid_blocks(), kBlock, 0, s>>>(n, r64, b32, x32, st_in, rs, cond_in);
  ESD_CUDA(cudaGetLastError());
}

__global__ void k_d2f(long long cnt, const double* a, float* b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// FP32 slice-major copy of a column-major n x M block: row i sits at lane (rowpos & 31) of
// slice (rowpos >> 5); the M columns of one slice are stored one after another.
__global__ void k_to_slice_major(int n, const int* rowpos, const double* X, size_t ld, int M, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int pos = rowpos[i];
    const size_t base = (size_t)(pos >> 5) * M * kSlice + (pos & 31);
    for (int k = 0; k < M; ++k) out[base + (size_t)k * kSlice] = (float)X[(size_t)k * ld + i];
  }
}

void to_slice_major(int n, const int* rowpos, const double* X, size_t ld, int M, float* out, cudaStream_t s) {
  if (n <= 0 || M <= 0) return;
  k_to_slice_major<<<max_grid_blocks(), kBlock, 0, s>>>(n, rowpos, X, ld, M, out);
  ESD_CUDA(cudaGetLastError());
}

__global__ void k_round_f32(long long cnt, const double* a, double* b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)(float)a[i];
}

void round_to_f32(long long cnt, const double* a, double* b, cudaStream_t s) {
  if (cnt <= 0) return;
  k_round_f32<<<max_grid_blocks(), kBlock, 0, s>>>(cnt, a, b);
  ESD_CUDA(cudaGetLastError());
}

void convert_d2f(long long cnt, const double* a, float* b, cudaStream_t s) {
  if (cnt <= 0) return;
  k_d2f<<<max_grid_blocks(), kBlock, 0, s>>>(cnt, a, b);
  ESD_CUDA(cudaGetLastError());
}

}  // namespace esd
