// Kernels of one PCG / deflated PCG / subspace-corrected PCG iteration and the launch
// sequences that form a solve. Instantiated for double (esd_iter_f64.cu) and float
// (esd_iter_f32.cu).
//
// Iteration i (plain IC(0) mode, 7-point stencil with 8 colours => 4 forward / 4 backward
// colour levels), one launch per line:
//   spmv_pq   q = A p, (p, q)                 [+ h = (AW)^T p, y = E^-1 h, deflation]
//   update    x += a p, r -= a q, ||r||^2, y = r/l_ii on forward level 0
//             [deflation: r -= a (q - AW y); SC: f = W^T r, u = E^-1 f]
//   fwd l     y_i = (r_i - sum_k l_ik y_k)/l_ii for the rows of level l, sum y_i^2
//             (rows without later neighbours store z_i = y_i/l_ii at once)
//   bwd l     z_i = (y_i - sum_j l_ji z_j)/l_ii, p_i = z_i [+ (W u)_i] + beta p_i
// rho = (r, M^-1 r) is accumulated as sum y_i^2 (= ||L^-1 r||^2) during the forward
// sweep, so beta is known before the backward sweep and p is updated in place by it.
// Scalars never leave the device: the last block of every reduction computes alpha, beta,
// the convergence test and the sampling decision, and ends the graph's while loop.
#pragma once

#include "esd_iter.h"

namespace esd {

enum { kModePlain = ESD_PLAIN, kModeDefl = ESD_DEFLATION, kModeSC = ESD_SUBSPACE_CORRECTION };

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }

// sum_k val[s,k,lane] * v[col[s,k,lane]] for the row of this lane in slice md
template <typename T>
__device__ __forceinline__ T row_dot(const SellView<T>& M, const int4& md, int lane, const T* __restrict__ v) {
  const int* cp = M.col + md.x + lane;
  const T* vp = M.val + md.x + lane;
  T acc = T(0);
#pragma unroll 4
  for (int k = 0; k < md.y; ++k) acc = fma(ld_stream(vp + k * kSlice), v[ld_stream(cp + k * kSlice)], acc);
  return acc;
}

__device__ __forceinline__ void end_loop(unsigned long long cond) {
  if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
}

// beta and rho after the forward sweep (first pass: p = z, no beta)
__device__ __forceinline__ bool finalize_rho(State* st, double rho_new, double* bhist,
                                             unsigned long long cond) {
  if (!(rho_new > 0.0)) {
    st->status = ESD_ERR_BREAKDOWN;
    st->conv = 1;
    end_loop(cond);
    return false;
  }
  const bool first = st->iter == 0;
  const double beta = first ? 0.0 : rho_new / st->rho;
  if (!first) bhist[st->iter - 1] = beta;
  st->beta = beta;
  st->rho = rho_new;
  return true;
}

// Sampling method A (Appendix A) at iteration i, called only while the solve goes on.
__device__ __forceinline__ void sampling_a(State* st) {
  const int i = st->iter, m = st->samp_m;
  if (i % st->h != 0) return;
  long long it = 0, q = i - 1;
  for (int l = 0; l <= st->lmax; ++l) {
    it += (l % 2 == 0) ? q : -q;
    q /= m;
  }
  const int slot = (int)(it % m);
  st->pend_slot = slot;
  st->slot_iter[slot] = i;
  if (i == st->h * m) st->h *= 2;
}

#define ESD_LOOP_SLICES(set)                                             \
  const int lane = lane_id();                                            \
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;           \
  const int nw = (gridDim.x * blockDim.x) >> 5;                          \
  for (int g = gw; g < (set).total(); g += nw)

// ------------------------------------------------------------------ plain kernels

template <typename T>
__global__ void __launch_bounds__(kBlock) k_spmv(SellView<T> A, SliceSet set, const T* __restrict__ x,
                                                 T* __restrict__ y) {
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = A.meta[s];
    const T acc = row_dot(A, md, lane, x);
    if (lane < md.w) y[md.z + lane] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_fwd_plain(SellView<T> L, SliceSet set, const T* __restrict__ r,
                                                      T* y, const T* __restrict__ inv_d) {
  ESD_LOOP_SLICES(set) {
    int rr;
    const int s = set.slice(g, &rr);
    const int4 md = L.meta[s];
    const T sum = row_dot(L, md, lane, y);
    if (lane < md.w) {
      const int i = md.z + lane;
      y[i] = (r[i] - sum) * inv_d[i];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_bwd_plain(SellView<T> U, SliceSet set, const T* __restrict__ y,
                                                      T* z, const T* __restrict__ inv_d) {
  ESD_LOOP_SLICES(set) {
    int rr;
    const int s = set.slice(g, &rr);
    const int4 md = U.meta[s];
    const T sum = row_dot(U, md, lane, z);
    if (lane < md.w) {
      const int i = md.z + lane;
      z[i] = (y[i] - sum) * inv_d[i];
    }
  }
}

// ------------------------------------------------------------------ solve kernels

// q = A p, pq = (p, q); deflation: h = (AW)^T p, y = E^-1 h, (p, P^T A p) = pq - h^T y.
// Last block: alpha = rho / (p, P^T A p).
template <typename T, int M>
__global__ void __launch_bounds__(kBlock) k_spmv_pq(IterCtx<T> c, SliceSet set) {
  constexpr int R = 1 + M;
  __shared__ T red[(kBlock / 32 + 1) * R];
  __shared__ double hy_s;
  State* st = c.st;
  // Independent of every reduction: a loop body that starts more than maxit + 2 times ends
  // the loop, so no failure of the scalar bookkeeping can keep the while node running.
  if (blockIdx.x == 0 && threadIdx.x == 0 && c.cond) {
    if (atomicAdd(&st->guard, 1) >= st->maxit + 2) {
      st->status = ESD_ERR_INTERNAL;
      st->conv = 1;
      end_loop(c.cond);
    }
  }
  if (st->conv) return;
  T acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = T(0);
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    const T qi = row_dot(c.Av, md, lane, c.p);
    if (lane < md.w) {
      const int i = md.z + lane;
      const T pi = c.p[i];
      c.q[i] = qi;
      acc[0] = fma(pi, qi, acc[0]);
#pragma unroll
      for (int k = 0; k < M; ++k) acc[1 + k] = fma(c.AW[k * c.ld + i], pi, acc[1 + k]);
    }
  }
  if (grid_sum_multi<R>(acc, red, (T*)c.partials, &st->ticket[kTkSpmv])) {
    if (M > 0) {
      if (threadIdx.x < 32) {
        double part = 0.0;
        for (int i = threadIdx.x; i < M; i += 32) {
          double y = 0.0;
          for (int k = 0; k < M; ++k) y += c.Einv[i * M + k] * (double)red[1 + k];
          st->y[i] = y;
          part += y * (double)red[1 + i];
        }
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (threadIdx.x == 0) hy_s = part;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double pq = (double)red[0];
      const double pap = pq - (M > 0 ? hy_s : 0.0);
      st->pq = pq;
      st->pap = pap;
      if (!(pap > 0.0) || !(st->rho > 0.0)) {
        st->status = ESD_ERR_BREAKDOWN;
        st->conv = 1;
        st->alpha = 0.0;
        end_loop(c.cond);
      } else {
        const double a = st->rho / pap;
        st->alpha = a;
        c.ahist[st->iter] = a;
      }
    }
  }
}

// x += alpha p; r -= alpha q (deflation: r -= alpha (q - AW y)); ||r||^2; the stored
// sample of the previous iteration; SC: f = W^T r; forward level 0 (y = r / l_ii).
// do_update = 0 runs the same epilogue on r0 (start of a solve).
template <typename T, int M, int MODE, int PRE>
__global__ void __launch_bounds__(kBlock) k_update(IterCtx<T> c, SliceSet set, int do_update,
                                                   int finalize) {
  constexpr int SCM = (MODE == kModeSC) ? M : 0;
  constexpr int DM = (MODE == kModeDefl) ? M : 0;
  constexpr int R = 2 + SCM;
  __shared__ T red[(kBlock / 32 + 1) * R];
  __shared__ double ys[DM > 0 ? DM : 1];
  __shared__ double fu_s;
  State* st = c.st;
  if (st->conv) return;
  const T alpha = (T)st->alpha;
  const int pend = do_update ? st->pend_slot : -1;
  if (DM > 0) {
    for (int k = threadIdx.x; k < DM; k += blockDim.x) ys[k] = st->y[k];
    __syncthreads();
  }
  T acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = T(0);
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    if (lane < md.w) {
      const int i = md.z + lane;
      T ri;
      if (do_update) {
        const T xi = c.x[i];
        if (pend >= 0) c.samples[(size_t)pend * c.ld + i] = xi;
        c.x[i] = fma(alpha, c.p[i], xi);
        T t = c.q[i];
#pragma unroll
        for (int k = 0; k < DM; ++k) t = fma(-c.AW[k * c.ld + i], (T)ys[k], t);
        ri = fma(-alpha, t, c.r[i]);
        c.r[i] = ri;
        acc[0] = fma(ri, ri, acc[0]);
      } else {
        ri = c.r[i];
      }
#pragma unroll
      for (int k = 0; k < SCM; ++k) acc[2 + k] = fma(c.W[k * c.ld + i], ri, acc[2 + k]);
      if (PRE == ESD_PRECOND_IC0) {
        const unsigned char f = c.sflags[s];
        if (f & 1) {
          const T d = c.inv_d[i];
          const T yv = ri * d;
          acc[1] = fma(yv, yv, acc[1]);
          c.Y[i] = (f & 2) ? yv * d : yv;
        }
      }
    }
  }
  if (grid_sum_multi<R>(acc, red, (T*)c.partials, &st->ticket[kTkUpdate])) {
    if (SCM > 0) {
      if (threadIdx.x < 32) {
        double part = 0.0;
        for (int i = threadIdx.x; i < SCM; i += 32) {
          double u = 0.0;
          for (int k = 0; k < SCM; ++k) u += c.Einv[i * SCM + k] * (double)red[2 + k];
          st->u[i] = u;
          part += u * (double)red[2 + i];
        }
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (threadIdx.x == 0) fu_s = part;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (do_update) {
        st->rr = (double)red[0];
        st->iter += 1;
        st->pend_slot = -1;
      }
      const double rr = st->rr;
      bool stop = false;
      if (!(rr == rr)) {
        st->status = ESD_ERR_BREAKDOWN;
        stop = true;
      } else if (st->zero_rhs || rr <= st->tol2bb) {
        stop = true;
      } else if (st->iter >= st->maxit) {
        st->status = ESD_ERR_MAXIT;
        stop = true;
      }
      if (!stop && do_update && st->samp_m > 0) sampling_a(st);
      st->fu = SCM > 0 ? fu_s : 0.0;
      if (PRE == ESD_PRECOND_IC0) st->rho_acc = (double)red[1];
      if (stop) {
        st->conv = 1;
        end_loop(c.cond);
      } else if (finalize) {
        // no forward level beyond 0 (or no preconditioner): rho is complete here
        const double rho_ic = (PRE == ESD_PRECOND_IC0) ? st->rho_acc : rr;
        finalize_rho(st, rho_ic + st->fu, c.bhist, c.cond);
      }
    }
  }
}

// One forward colour level: y_i = (r_i - sum_k l_ik y_k) / l_ii; rho += y_i^2.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fwd(IterCtx<T> c, SliceSet set, int last) {
  __shared__ T red[(kBlock / 32 + 1)];
  State* st = c.st;
  if (st->conv) return;
  T acc[1] = {T(0)};
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Lv.meta[s];
    const T sum = row_dot(c.Lv, md, lane, c.Y);
    if (lane < md.w) {
      const int i = md.z + lane;
      const T d = c.inv_d[i];
      const T yv = (c.r[i] - sum) * d;
      acc[0] = fma(yv, yv, acc[0]);
      c.Y[i] = ((set.bwd0 >> r) & 1u) ? yv * d : yv;
    }
  }
  if (grid_sum_multi<1>(acc, red, (T*)c.partials, &st->ticket[kTkSweep])) {
    if (threadIdx.x == 0) {
      st->rho_acc += (double)red[0];
      if (last) finalize_rho(st, st->rho_acc + st->fu, c.bhist, c.cond);
    }
  }
}

// One backward colour level: z_i = (y_i - sum_j l_ji z_j) / l_ii, then
// p_i = z_i [+ (W u)_i] + beta p_i. "elem" rows had z_i stored by the forward sweep and
// only take the direction update.
template <typename T, int SCM>
__global__ void __launch_bounds__(kBlock) k_bwd(IterCtx<T> c, SliceSet set, SliceSet elem) {
  __shared__ double us[SCM > 0 ? SCM : 1];
  State* st = c.st;
  if (st->conv) return;
  const T beta = (T)st->beta;
  const bool first = st->iter == 0;
  if (SCM > 0) {
    for (int k = threadIdx.x; k < SCM; k += blockDim.x) us[k] = st->u[k];
    __syncthreads();
  }
  const int nsweep = set.total();
  const int total = nsweep + elem.total();
  const int lane = lane_id();
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int g = gw; g < total; g += nw) {
    int r;
    const bool sweep = g < nsweep;
    const int s = sweep ? set.slice(g, &r) : elem.slice(g - nsweep, &r);
    const int4 md = sweep ? c.Uv.meta[s] : c.Av.meta[s];
    T zic = T(0);
    if (sweep) {
      const T sum = row_dot(c.Uv, md, lane, c.Y);
      if (lane < md.w) {
        const int i = md.z + lane;
        zic = (c.Y[i] - sum) * c.inv_d[i];
        c.Y[i] = zic;
      }
    } else if (lane < md.w) {
      zic = c.Y[md.z + lane];
    }
    if (lane < md.w) {
      const int i = md.z + lane;
      T z = zic;
#pragma unroll
      for (int k = 0; k < SCM; ++k) z = fma(c.W[k * c.ld + i], (T)us[k], z);
      c.p[i] = first ? z : fma(beta, c.p[i], z);
    }
  }
}

// No preconditioner: p = r [+ W u] + beta p.
template <typename T, int SCM>
__global__ void __launch_bounds__(kBlock) k_dir(IterCtx<T> c, SliceSet set) {
  __shared__ double us[SCM > 0 ? SCM : 1];
  State* st = c.st;
  if (st->conv) return;
  const T beta = (T)st->beta;
  const bool first = st->iter == 0;
  if (SCM > 0) {
    for (int k = threadIdx.x; k < SCM; k += blockDim.x) us[k] = st->u[k];
    __syncthreads();
  }
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    if (lane < md.w) {
      const int i = md.z + lane;
      T z = c.r[i];
#pragma unroll
      for (int k = 0; k < SCM; ++k) z = fma(c.W[k * c.ld + i], (T)us[k], z);
      c.p[i] = first ? z : fma(beta, c.p[i], z);
    }
  }
}

// r = b - A x, ||b||^2, ||r||^2 (start of a solve).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_residual0(IterCtx<T> c, SliceSet set) {
  __shared__ T red[(kBlock / 32 + 1) * 2];
  State* st = c.st;
  T acc[2] = {T(0), T(0)};
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    const T ax = row_dot(c.Av, md, lane, c.x);
    if (lane < md.w) {
      const int i = md.z + lane;
      const T bi = c.b[i];
      const T ri = bi - ax;
      c.r[i] = ri;
      acc[0] = fma(bi, bi, acc[0]);
      acc[1] = fma(ri, ri, acc[1]);
    }
  }
  if (grid_sum_multi<2>(acc, red, (T*)c.partials, &st->ticket[kTkAux])) {
    if (threadIdx.x == 0) {
      const double bb = (double)red[0];
      st->bb = bb;
      st->rr = (double)red[1];
      st->tol2bb = st->scal0 * bb;  // scal0 holds tol^2
      st->zero_rhs = (bb == 0.0);
    }
  }
}

// f = X^T v - Y^T w (Y optional), u = E^-1 f (stored in st->u).
template <typename T, int M>
__global__ void __launch_bounds__(kBlock) k_tallT(IterCtx<T> c, SliceSet set, const T* X, const T* v,
                                                  const T* Y2, const T* w) {
  __shared__ T red[(kBlock / 32 + 1) * M];
  State* st = c.st;
  T acc[M];
#pragma unroll
  for (int k = 0; k < M; ++k) acc[k] = T(0);
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    if (lane < md.w) {
      const int i = md.z + lane;
      const T vi = v[i];
#pragma unroll
      for (int k = 0; k < M; ++k) acc[k] = fma(X[k * c.ld + i], vi, acc[k]);
      if (Y2) {
        const T wi = w[i];
#pragma unroll
        for (int k = 0; k < M; ++k) acc[k] = fma(-Y2[k * c.ld + i], wi, acc[k]);
      }
    }
  }
  if (grid_sum_multi<M>(acc, red, (T*)c.partials, &st->ticket[kTkAux])) {
    if (threadIdx.x < 32) {
      for (int i = threadIdx.x; i < M; i += 32) {
        double u = 0.0;
        for (int k = 0; k < M; ++k) u += c.Einv[i * M + k] * (double)red[k];
        st->u[i] = u;
      }
    }
  }
}

// v += sign * Z u (u = st->u); optionally ||v||^2 into st->rr.
template <typename T, int M>
__global__ void __launch_bounds__(kBlock) k_tall_axpy(IterCtx<T> c, SliceSet set, const T* Z, T* v,
                                                      T sign, int norm) {
  __shared__ T red[(kBlock / 32 + 1)];
  __shared__ double us[M];
  State* st = c.st;
  for (int k = threadIdx.x; k < M; k += blockDim.x) us[k] = st->u[k];
  __syncthreads();
  T acc[1] = {T(0)};
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    if (lane < md.w) {
      const int i = md.z + lane;
      T t = T(0);
#pragma unroll
      for (int k = 0; k < M; ++k) t = fma(Z[k * c.ld + i], (T)us[k], t);
      const T vi = fma(sign, t, v[i]);
      v[i] = vi;
      acc[0] = fma(vi, vi, acc[0]);
    }
  }
  if (norm) {
    if (grid_sum_multi<1>(acc, red, (T*)c.partials, &st->ticket[kTkAux2])) {
      if (threadIdx.x == 0) st->rr = (double)red[0];
    }
  }
}

// The sample due at the last iteration (none is taken at the converging one), x = 0 for b = 0.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_finish(IterCtx<T> c, SliceSet set) {
  const State* st = c.st;
  const int pend = st->pend_slot;
  const bool zero = st->zero_rhs;
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    if (lane < md.w) {
      const int i = md.z + lane;
      if (pend >= 0 && c.samples) c.samples[(size_t)pend * c.ld + i] = c.x[i];
      if (zero) c.x[i] = T(0);
    }
  }
}

// ||b - A x||^2
template <typename T>
__global__ void __launch_bounds__(kBlock) k_true_res(IterCtx<T> c, SliceSet set) {
  __shared__ T red[(kBlock / 32 + 1)];
  State* st = c.st;
  T acc[1] = {T(0)};
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    const T ax = row_dot(c.Av, md, lane, c.x);
    if (lane < md.w) {
      const int i = md.z + lane;
      const T t = c.b[i] - ax;
      acc[0] = fma(t, t, acc[0]);
    }
  }
  if (grid_sum_multi<1>(acc, red, (T*)c.partials, &st->ticket[kTkAux])) {
    if (threadIdx.x == 0) st->true_rr = (double)red[0];
  }
}

// ------------------------------------------------------------------ launch sequences

#define ESD_DISPATCH_M(Mrt, ...)                                                      \
  switch (Mrt) {                                                                      \
    case 0: { constexpr int MM = 0; __VA_ARGS__; } break;                             \
    case 8: { constexpr int MM = 8; __VA_ARGS__; } break;                             \
    case 16: { constexpr int MM = 16; __VA_ARGS__; } break;                           \
    case 24: { constexpr int MM = 24; __VA_ARGS__; } break;                           \
    case 32: { constexpr int MM = 32; __VA_ARGS__; } break;                           \
    case 64: { constexpr int MM = 64; __VA_ARGS__; } break;                           \
    default: throw Error(ESD_ERR_INVALID, "unsupported padded column count");         \
  }

#define ESD_DISPATCH_MPOS(Mrt, ...)                                                   \
  switch (Mrt) {                                                                      \
    case 8: { constexpr int MM = 8; __VA_ARGS__; } break;                             \
    case 16: { constexpr int MM = 16; __VA_ARGS__; } break;                           \
    case 24: { constexpr int MM = 24; __VA_ARGS__; } break;                           \
    case 32: { constexpr int MM = 32; __VA_ARGS__; } break;                           \
    case 64: { constexpr int MM = 64; __VA_ARGS__; } break;                           \
    default: throw Error(ESD_ERR_INVALID, "unsupported padded column count");         \
  }

template <typename T>
static void launch_update(const IterCtx<T>& c, int do_update, int finalize, cudaStream_t s,
                          KernelMarks* marks = nullptr) {
  const SliceSet& all = c.A->all;
  const int G = grid_blocks(all.total());
  const int Mm = (c.mode == ESD_PLAIN) ? 0 : c.M;
  if (c.pre == ESD_PRECOND_IC0) {
    if (c.mode == ESD_PLAIN)
      k_update<T, 0, kModePlain, ESD_PRECOND_IC0><<<G, kBlock, 0, s>>>(c, all, do_update, finalize);
    else if (c.mode == ESD_DEFLATION)
      ESD_DISPATCH_MPOS(Mm, k_update<T, MM, kModeDefl, ESD_PRECOND_IC0><<<G, kBlock, 0, s>>>(c, all, do_update, finalize))
    else
      ESD_DISPATCH_MPOS(Mm, k_update<T, MM, kModeSC, ESD_PRECOND_IC0><<<G, kBlock, 0, s>>>(c, all, do_update, finalize))
  } else {
    if (c.mode == ESD_PLAIN)
      k_update<T, 0, kModePlain, ESD_PRECOND_NONE><<<G, kBlock, 0, s>>>(c, all, do_update, finalize);
    else if (c.mode == ESD_DEFLATION)
      ESD_DISPATCH_MPOS(Mm, k_update<T, MM, kModeDefl, ESD_PRECOND_NONE><<<G, kBlock, 0, s>>>(c, all, do_update, finalize))
    else
      ESD_DISPATCH_MPOS(Mm, k_update<T, MM, kModeSC, ESD_PRECOND_NONE><<<G, kBlock, 0, s>>>(c, all, do_update, finalize))
  }
  ESD_CUDA(cudaGetLastError());
  if (marks) marks->mark(s, "update");
}

// forward levels >= 1 then backward levels (with the direction update)
template <typename T>
static void launch_precond(const IterCtx<T>& c, cudaStream_t s, KernelMarks* marks = nullptr) {
  const esd_matrix* A = c.A;
  const int SCM = (c.mode == ESD_SUBSPACE_CORRECTION) ? c.M : 0;
  if (c.pre == ESD_PRECOND_NONE) {
    ESD_DISPATCH_M(SCM, k_dir<T, MM><<<grid_blocks(A->all.total()), kBlock, 0, s>>>(c, A->all));
    ESD_CUDA(cudaGetLastError());
    if (marks) marks->mark(s, "dir");
    return;
  }
  for (size_t l = 0; l < A->fwd_sets.size(); ++l) {
    const SliceSet& set = A->fwd_sets[l];
    k_fwd<T><<<grid_blocks(set.total()), kBlock, 0, s>>>(c, set, l + 1 == A->fwd_sets.size() ? 1 : 0);
    ESD_CUDA(cudaGetLastError());
    if (marks) marks->mark(s, ("fwd_" + std::to_string(l + 1)).c_str());
  }
  SliceSet none{};
  const size_t nb = std::max(A->bwd_sets.size(), A->bwd0_sets.size());
  for (size_t l = 0; l < nb; ++l) {
    const SliceSet& sw = l < A->bwd_sets.size() ? A->bwd_sets[l] : none;
    const SliceSet& el = l < A->bwd0_sets.size() ? A->bwd0_sets[l] : none;
    ESD_DISPATCH_M(SCM, k_bwd<T, MM><<<grid_blocks(sw.total() + el.total()), kBlock, 0, s>>>(c, sw, el));
    ESD_CUDA(cudaGetLastError());
    if (marks) marks->mark(s, ("bwd_" + std::to_string(l + 1)).c_str());
  }
}

template <typename T>
void launch_init(const IterCtx<T>& c, cudaStream_t s) {
  const SliceSet& all = c.A->all;
  const int G = grid_blocks(all.total());
  k_residual0<T><<<G, kBlock, 0, s>>>(c, all);
  ESD_CUDA(cudaGetLastError());
  if (c.mode == ESD_DEFLATION) {
    // r0 = P^T (b - A x0) = r - AW E^-1 W^T r
    ESD_DISPATCH_MPOS(c.M, k_tallT<T, MM><<<G, kBlock, 0, s>>>(c, all, c.W, c.r, (const T*)nullptr, (const T*)nullptr));
    ESD_CUDA(cudaGetLastError());
    ESD_DISPATCH_MPOS(c.M, k_tall_axpy<T, MM><<<G, kBlock, 0, s>>>(c, all, c.AW, c.r, T(-1), 1));
    ESD_CUDA(cudaGetLastError());
  }
  const bool fin = c.pre == ESD_PRECOND_NONE || c.A->fwd_sets.empty();
  launch_update<T>(c, 0, fin ? 1 : 0, s);
  launch_precond<T>(c, s);
}

template <typename T>
void launch_iteration(const IterCtx<T>& c, cudaStream_t s, KernelMarks* marks) {
  const SliceSet& all = c.A->all;
  const int G = grid_blocks(all.total());
  const int Mm = (c.mode == ESD_DEFLATION) ? c.M : 0;
  if (marks) marks->mark(s, "start");
  ESD_DISPATCH_M(Mm, k_spmv_pq<T, MM><<<G, kBlock, 0, s>>>(c, all));
  ESD_CUDA(cudaGetLastError());
  if (marks) marks->mark(s, "spmv_pq");
  const bool fin = c.pre == ESD_PRECOND_NONE || c.A->fwd_sets.empty();
  launch_update<T>(c, 1, fin ? 1 : 0, s, marks);
  launch_precond<T>(c, s, marks);
}

template <typename T>
void launch_finish(const IterCtx<T>& c, cudaStream_t s) {
  const SliceSet& all = c.A->all;
  const int G = grid_blocks(all.total());
  if (c.mode == ESD_DEFLATION) {
    // x = P x_i + W E^-1 W^T b = x_i + W E^-1 (W^T b - (AW)^T x_i)
    ESD_DISPATCH_MPOS(c.M, k_tallT<T, MM><<<G, kBlock, 0, s>>>(c, all, c.W, c.b, c.AW, c.x));
    ESD_CUDA(cudaGetLastError());
    ESD_DISPATCH_MPOS(c.M, k_tall_axpy<T, MM><<<G, kBlock, 0, s>>>(c, all, c.W, c.x, T(1), 0));
    ESD_CUDA(cudaGetLastError());
  }
  k_finish<T><<<G, kBlock, 0, s>>>(c, all);
  ESD_CUDA(cudaGetLastError());
}

#define ESD_INSTANTIATE_ITER(T)                                                        \
  template void launch_init<T>(const IterCtx<T>&, cudaStream_t);                      \
  template void launch_iteration<T>(const IterCtx<T>&, cudaStream_t, KernelMarks*);   \
  template void launch_finish<T>(const IterCtx<T>&, cudaStream_t);

}  // namespace esd
