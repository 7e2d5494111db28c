// Kernels of one PCG / deflated PCG / subspace-corrected PCG iteration and the launch
// sequences that form a solve. Instantiated for double (esd_iter_f64.cu) and float
// (esd_iter_f32.cu).
//
// Iteration i (IC(0), 7-point stencil with 8 colours => forward levels {0}{1,2,4}{3,5,6}{7},
// backward levels {7}{3,5,6}{1,2,4}{0}), one launch per line:
//   spmv_pq   q = A p, (p, q)                 [+ h = (AW)^T p, y = E^-1 h, deflation]
//   update    x += a p, r -= a q, ||r||^2, y = r/l_ii on forward level 0
//             [deflation: r -= a (q - AW y); SC: f = W^T r, u = E^-1 f]
//   fwd l     y_i = (r_i - sum_k l_ik y_k)/l_ii for the rows of level l, sum y_i^2
//             (rows without later neighbours store z_i = y_i/l_ii at once)
//   bwd l     z_i = (y_i - sum_j l_ji z_j)/l_ii, p_i = z_i [+ (W u)_i] + beta p_i
// rho = (r, M^-1 r) is accumulated as sum y_i^2 (= ||L^-1 r||^2) during the forward sweep,
// so beta is known before the backward sweep and p is updated in place by it. The
// strict factors are stored negated, so each substitution is one FMA chain started at r_i.
// Scalars never leave the device: the last block of a reduction computes alpha, beta, the
// convergence test and the sampling decision, and ends the graph's while loop. Every
// kernel is launched with programmatic stream serialisation: it waits for its predecessor
// at entry (griddepcontrol) and lets its successor be scheduled at once, which hides the
// launch and the tail of each grid behind its neighbour.
#pragma once

#include <mutex>
#include <unordered_map>
#include <utility>

#include "esd_iter.h"

namespace esd {

enum { kModePlain = ESD_PLAIN, kModeDefl = ESD_DEFLATION, kModeSC = ESD_SUBSPACE_CORRECTION };

// Resident blocks per SM requested from the compiler for the FP64 substitution kernels
// (3: up to 42 registers per thread; measured 3-4 % faster per iteration than 4 blocks at 32)
#ifndef ESD_SWEEP_MINB
#define ESD_SWEEP_MINB 3
#endif
// FP32 kernels move half the bytes per load, so they need more loads in flight per thread
#ifndef ESD_SWEEP_MINB_F32
#define ESD_SWEEP_MINB_F32 4
#endif
#ifndef ESD_ROW_UNROLL
#define ESD_ROW_UNROLL 4
#endif
// FP32 kernels read (value, column) as one 8-byte load per entry
#ifndef ESD_F32_INTERLEAVED
#define ESD_F32_INTERLEAVED 1
#endif
#ifndef ESD_ROW_UNROLL_F32
#define ESD_ROW_UNROLL_F32 4
#endif
// unroll of the FP64 row products of the substitution kernels (k_fwd, k_bwd): their rows
// hold 2 to 6 factor entries, and 2 beat 4 by another 1-2 % per iteration
#ifndef ESD_SWEEP_UNROLL
#define ESD_SWEEP_UNROLL 2
#endif
// resident blocks per SM of the FP64 SpMV without W terms (plain and SC modes)
#ifndef ESD_SPMV_MINB
#define ESD_SPMV_MINB 4
#endif
// resident blocks per SM of the FP64 deflated SpMV (double-float W terms)
#ifndef ESD_DF_MINB
#define ESD_DF_MINB 2
#endif
// resident blocks per SM of the SpMV that also multiplies the power vector
#ifndef ESD_POW_MINB
#define ESD_POW_MINB 2
#endif
#define ESD_PRAGMA(x) _Pragma(#x)
#define ESD_UNROLL(n) ESD_PRAGMA(unroll n)

template <typename T>
constexpr int sweep_minb() {
  return sizeof(T) == 4 ? ESD_SWEEP_MINB_F32 : ESD_SWEEP_MINB;
}

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }

// init + sum_k val[s,k,lane] * v[col[s,k,lane]] for the row of this lane in slice md; SWEEP
// selects the unroll of the substitution kernels for FP64
template <typename T, bool SWEEP = false>
__device__ __forceinline__ T row_fma(const SellView<T>& M, const int4& md, int lane, const T* __restrict__ v,
                                     T init) {
  const int* cp = M.col + md.x + lane;
  const T* vp = M.val + md.x + lane;
  T acc = init;
  if (sizeof(T) == 4 && ESD_F32_INTERLEAVED && M.ent) {
    const uint2* ep = M.ent + md.x + lane;
    ESD_UNROLL(ESD_ROW_UNROLL_F32)
    for (int k = 0; k < md.y; ++k) {
      const uint2 e = __ldcs(ep + k * kSlice);
      acc = fma((T)__uint_as_float(e.x), v[e.y], acc);
    }
  } else if (sizeof(T) == 4) {
    ESD_UNROLL(ESD_ROW_UNROLL_F32)
    for (int k = 0; k < md.y; ++k) acc = fma(ld_stream(vp + k * kSlice), v[ld_stream(cp + k * kSlice)], acc);
  } else if (SWEEP) {
    ESD_UNROLL(ESD_SWEEP_UNROLL)
    for (int k = 0; k < md.y; ++k) acc = fma(ld_stream(vp + k * kSlice), v[ld_stream(cp + k * kSlice)], acc);
  } else {
    ESD_UNROLL(ESD_ROW_UNROLL)
    for (int k = 0; k < md.y; ++k) acc = fma(ld_stream(vp + k * kSlice), v[ld_stream(cp + k * kSlice)], acc);
  }
  return acc;
}

// Difference form of the same row product: s_i v_i + sum_j a_ij (v_j - v_i), s = A 1. For
// a smooth v the differences are exact (or nearly) and nothing cancels, so in FP32 the
// result keeps its relative accuracy where the plain sum loses up to cond(A) of it.
template <typename T>
__device__ __forceinline__ T row_fma_diff(const SellView<T>& M, const int4& md, int lane, const T* __restrict__ v,
                                          T vi, T si, T init) {
  const int* cp = M.col + md.x + lane;
  const T* vp = M.val + md.x + lane;
  T acc = fma(si, vi, init);
  if (ESD_F32_INTERLEAVED && M.ent) {
    const uint2* ep = M.ent + md.x + lane;
    ESD_UNROLL(ESD_ROW_UNROLL_F32)
    for (int k = 0; k < md.y; ++k) {
      const uint2 e = __ldcs(ep + k * kSlice);
      acc = fma((T)__uint_as_float(e.x), v[e.y] - vi, acc);
    }
  } else {
    ESD_UNROLL(ESD_ROW_UNROLL_F32)
    for (int k = 0; k < md.y; ++k) acc = fma(ld_stream(vp + k * kSlice), v[ld_stream(cp + k * kSlice)] - vi, acc);
  }
  return acc;
}

// Two FP64 row products with one read of the matrix row: au = A u, av = A v (the fused
// SpMV of the power method, Section 5.4). au takes the FMAs in the order row_fma does.
__device__ __forceinline__ void row_fma2(const SellView<double>& M, const int4& md, int lane,
                                         const double* __restrict__ u, const double* __restrict__ v, double& au,
                                         double& av) {
  const int* cp = M.col + md.x + lane;
  const double* vp = M.val + md.x + lane;
  double a = 0.0, b = 0.0;
  ESD_UNROLL(ESD_ROW_UNROLL)
  for (int k = 0; k < md.y; ++k) {
    const double val = ld_stream(vp + k * kSlice);
    const int j = ld_stream(cp + k * kSlice);
    a = fma(val, u[j], a);
    b = fma(val, v[j], b);
  }
  au = a;
  av = b;
}

// Index of W / AW entry (row i = lane l of slice s, column k) in the layout of this context:
// column-major with stride ld, or slice-major (the M columns of a 32-row slice contiguous,
// so a warp streams one block instead of M columns far apart).
template <int M, typename T>
__device__ __forceinline__ size_t wix(const IterCtx<T>& c, int k, int i, int s, int lane) {
  return c.wsm ? ((size_t)s * M + k) * kSlice + lane : (size_t)k * c.ld + i;
}

// ------------------------------------------------------------------ double-float W terms
// GB300 issues 2 FP64 FMAs per clock per SM and 128 FP32 ones, and its FP64 pipe also carries
// the FP64 <-> FP32 conversions. The deflation terms (2m FMAs per row) therefore run on the
// FP32 pipe in double-float arithmetic: a value is an unevaluated sum hi + lo of two floats
// (about 48 significant bits), sums use Knuth's error-free two-sum and products Dekker's
// splitting via FMA (TAOCP vol. 2, 4.2.2; Dekker, Numer. Math. 18, 1971). Doubles are split
// with integer operations only, relative to a power-of-two reference, so every float stays
// far inside its exponent range; parts more than 2^-100 below the reference are dropped,
// which is below FP64's own rounding of the same sums.

__device__ __forceinline__ int dexp(double v) {  // biased binary exponent of a double
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}

// 2^(e - 1023) as a double (e in 1 .. 2046)
__device__ __forceinline__ double dpow2(int e) { return __longlong_as_double((long long)e << 52); }

// v 2^(1023 - eref) = hi + lo (truncated to 24 + 24 bits); eref >= dexp(v).
__device__ __forceinline__ void df_split(double v, int eref, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const int d = e - eref;  // exponent of the scaled value, <= 0
  if (e == 0 || d < -100) {
    hi = 0.f;
    lo = 0.f;
    return;
  }
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long m = b & 0xfffffffffffffull;  // 52 fraction bits
  hi = __uint_as_float(sgn | ((unsigned)(d + 127) << 23) | (unsigned)(m >> 29));
  const unsigned r = (unsigned)(m & 0x1fffffffu);  // the 29 bits below hi, unit 2^(d - 52)
  const int t = 31 - __clz(r | 1u);                 // position of the leading bit of r
  const int fe = t + d + 75;                        // biased float exponent of lo
  if (r == 0 || fe < 1) {
    lo = 0.f;
    return;
  }
  const unsigned mn = (t >= 23) ? (r >> (t - 23)) : (r << (23 - t));
  lo = __uint_as_float(sgn | ((unsigned)fe << 23) | (mn & 0x7fffffu));
}

// (sh, sl) += (ah + al)(bh + bl), the product's al*bl term (2^-48 relative) left out
__device__ __forceinline__ void df_fma(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float ph = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -ph);  // exact error of ph
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  const float s = __fadd_rn(sh, ph);  // two-sum of sh and ph
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
  const float t = __fadd_rn(sl, __fadd_rn(err, pe));
  sh = __fadd_rn(s, t);  // renormalise: |sl| <= ulp(sh)
  sl = __fsub_rn(t, __fsub_rn(sh, s));
}

// 2^k as a float for k in -126 .. 0, else 0
__device__ __forceinline__ float fpow2_neg(int k) { return k < -126 ? 0.f : __uint_as_float((unsigned)(127 + k) << 23); }

// f 2^(eunit - 1023) as a double, widened with integer operations (exact) when the result is
// a normal double; zeros stay zero, other cases take the FP64 multiply
__device__ __forceinline__ double f2d_pow2(float f, int eunit) {
  const unsigned u = __float_as_uint(f);
  const int fe = (int)((u >> 23) & 0xffu);
  const int de = fe - 127 + eunit;
  if ((u & 0x7fffffffu) == 0u) return 0.0;
  if (fe == 0 || fe == 255 || de <= 0 || de >= 2047 || eunit < 1 || eunit > 2046) return (double)f * dpow2(eunit < 1 ? 1 : (eunit > 2046 ? 2046 : eunit));
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)de << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// Asynchronous 16-byte global -> shared copies (completion by wait_group, no polling).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

extern __shared__ __align__(16) unsigned char esd_dyn_smem[];

// Dynamic shared memory of the FP64 deflated SpMV: one slice block of AW (M x 32 float2) per warp.
template <int M>
__host__ __device__ constexpr int df_stage_bytes() {
  return M <= 32 ? (kBlock / 32) * M * kSlice * (int)sizeof(float2) : 0;
}

// (ah, al) += (bh, bl)
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  const float t = __fadd_rn(__fadd_rn(al, bl), err);
  ah = __fadd_rn(s, t);
  al = __fsub_rn(t, __fsub_rn(ah, s));
}

// Warp sums of P double-float values per lane, by the halving butterfly of warp_sum_multi:
// on return lane l holds (in h[0], l[0]) the total of value warp_sum_index<P>(l).
template <int P>
__device__ __forceinline__ void df_warp_sum_multi(float (&h)[P], float (&l)[P]) {
  static_assert((P & (P - 1)) == 0 && P <= 32, "P must be a power of two <= 32");
  const int lane = lane_id();
  int half = P / 2;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (half >= 1) {
      const bool upper = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < (P / 2 > 0 ? P / 2 : 1); ++k) {
        if (k < half) {
          const float sh = upper ? h[k] : h[k + half], sl = upper ? l[k] : l[k + half];
          float kh = upper ? h[k + half] : h[k], kl = upper ? l[k + half] : l[k];
          df_add(kh, kl, __shfl_xor_sync(0xffffffffu, sh, o), __shfl_xor_sync(0xffffffffu, sl, o));
          h[k] = kh;
          l[k] = kl;
        }
      }
      half >>= 1;
    } else {
      df_add(h[0], l[0], __shfl_xor_sync(0xffffffffu, h[0], o), __shfl_xor_sync(0xffffffffu, l[0], o));
    }
  }
}

// Warp totals of the double-float values [C0, M) in power-of-two chunks, converted to double
// times unit and written by one lane per value into red[warp * R + off + j].
template <int C0, int M, int R>
__device__ __forceinline__ void df_warp_sum_chunks(const float (&h)[M], const float (&l)[M], double unit, double* red,
                                                   int off, int lane, int warp) {
  if constexpr (C0 < M) {
    constexpr int C = pow2_floor(M - C0);
    float vh[C], vl[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      vh[k] = h[C0 + k];
      vl[k] = l[C0 + k];
    }
    df_warp_sum_multi<C>(vh, vl);
    const int idx = warp_sum_index<C>(lane);
    if ((lane & ((32 / C) - 1)) == 0) red[warp * R + off + C0 + idx] = ((double)vh[0] + (double)vl[0]) * unit;
    df_warp_sum_chunks<C0 + C, M, R>(h, l, unit, red, off, lane, warp);
  }
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
  const bool first = st->iter == 0 || st->fresh_dir;
  const double beta = first ? 0.0 : rho_new / st->rho;
  if (st->iter > 0) bhist[st->iter - 1] = beta;
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
  st->pend_prev = st->slot_iter[slot];
  st->slot_iter[slot] = i;
  if (i == st->h * m) st->h *= 2;
}

// Sampling method B (Section 4.2): the iterate whose relative residual first reaches
// tol^(s/(m+1)), s = 1..m, is kept; an iteration that reaches several new levels is kept
// once, in the next slot. Compared on squares, rel2 = ||r||^2/||b||^2 and scal0 = tol^2.
__device__ __forceinline__ void sampling_b(State* st, double rel2) {
  const int m = st->samp_m;
  int lev = st->sb_reached;
  while (lev < m && rel2 <= pow(st->scal0, (double)(lev + 1) / (double)(m + 1))) ++lev;
  if (lev > st->sb_reached) {
    const int slot = st->sb_used++;
    st->pend_slot = slot;
    st->slot_iter[slot] = st->iter;
    st->sb_reached = lev;
  }
}

#define ESD_LOOP_SLICES(set)                                             \
  const int lane = lane_id();                                            \
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;           \
  const int nw = (gridDim.x * blockDim.x) >> 5;                          \
  for (int g = gw; g < (set).total(); g += nw)

// ------------------------------------------------------------------ launch helpers

// Blocks of this kernel that fit on the whole GPU at once (one wave), cached per kernel.
inline int wave_blocks(const void* kernel) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kernel);
  if (it != cache.end()) return it->second;
  int per_sm = 0;
  ESD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0));
  const int w = std::max(1, std::min(per_sm, 4)) * (max_grid_blocks() / 4);
  cache[kernel] = w;
  return w;
}

template <typename... KArgs>
inline int grid_for(void (*kernel)(KArgs...), int slices) {
  const int need = (slices * kSlice + kBlock - 1) / kBlock;
  return std::max(1, std::min(need, wave_blocks((const void*)kernel)));
}

// Launch with programmatic stream serialisation on (see the file comment).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), int blocks, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ESD_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// Blocks of one wave for a kernel with dynamic shared memory (the limit raised once).
inline int wave_blocks_smem(const void* kernel, int smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kernel);
  if (it != cache.end()) return it->second;
  ESD_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  ESD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem));
  const int w = std::max(1, std::min(per_sm, 4)) * (max_grid_blocks() / 4);
  cache[kernel] = w;
  return w;
}

// launch_pdl with dynamic shared memory
template <typename... KArgs, typename... Args>
inline void launch_pdl_smem(void (*kernel)(KArgs...), int slices, int smem, cudaStream_t s, Args&&... args) {
  const int need = (slices * kSlice + kBlock - 1) / kBlock;
  const int blocks = std::max(1, std::min(need, wave_blocks_smem((const void*)kernel, smem)));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ESD_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}


// ------------------------------------------------------------------ plain kernels

template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_spmv(SellView<T> A, SliceSet set, const T* __restrict__ x,
                                                 T* __restrict__ y) {
  pdl_enter();
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = A.meta[s];
    const T acc = row_fma(A, md, lane, x, T(0));
    if (lane < md.w) y[md.z + lane] = acc;
  }
}

// y_i = (r_i - sum_k l_ik y_k) / l_ii with the negated factor entries
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_fwd_plain(SellView<T> L, SliceSet set, const T* __restrict__ r,
                                                      T* y, const T* __restrict__ inv_d) {
  pdl_enter();
  ESD_LOOP_SLICES(set) {
    int rr;
    const int s = set.slice(g, &rr);
    const int4 md = L.meta[s];
    const int i = md.z + lane;
    const bool valid = lane < md.w;
    const T acc = row_fma(L, md, lane, y, valid ? r[i] : T(0));
    if (valid) y[i] = acc * inv_d[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_bwd_plain(SellView<T> U, SliceSet set, const T* __restrict__ y,
                                                      T* z, const T* __restrict__ inv_d) {
  pdl_enter();
  ESD_LOOP_SLICES(set) {
    int rr;
    const int s = set.slice(g, &rr);
    const int4 md = U.meta[s];
    const int i = md.z + lane;
    const bool valid = lane < md.w;
    const T acc = row_fma(U, md, lane, z, valid ? y[i] : T(0));
    if (valid) z[i] = acc * inv_d[i];
  }
}

// ------------------------------------------------------------------ solve kernels

// q = A p, pq = (p, q); deflation: h = (AW)^T p, y = E^-1 h, (p, P^T A p) = pq - h^T y.
// Last block: alpha = rho / (p, P^T A p).
// blocks per SM the deflated kernels must fit: their M accumulators per thread; FP32 needs
// half the registers of FP64
template <typename T, int M>
constexpr int defl_minb() {
  return M == 0 ? (sizeof(T) == 8 ? ESD_SPMV_MINB : sweep_minb<T>()) : ((sizeof(T) == 4 ? M <= 32 : M <= 16) ? 2 : 1);
}

// q = A p and (p, q) [+ h = (AW)^T p, y = E^-1 h in deflation]; the last block sets alpha.
// POW (FP64, M = 0): the same matrix pass also forms w' = A v = scale * (A w) of the power
// vector, with ||w'||^2 (Algorithm PCG-con's (q v) = A (p v)).
template <typename T, int M, bool POW = false>
__global__ void __launch_bounds__(kBlock, POW ? ESD_POW_MINB
                                             : ((sizeof(T) == 8 && df_cols(M)) ? (M <= 16 ? ESD_DF_MINB : 1) : defl_minb<T, M>()))
    k_spmv_pq(IterCtx<T> c, SliceSet set) {
  static_assert(!POW || (M == 0 && sizeof(T) == 8), "the power method runs in the FP64 M = 0 product");
  constexpr int R = 1 + M + (POW ? 1 : 0);
  constexpr bool DF = sizeof(T) == 8 && df_cols(M);  // h = (AW)^T p in double-float
  __shared__ T red[red_size<R>()];
  __shared__ double hy_s;
  pdl_enter();
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
  const double* w_in = nullptr;
  double* w_out = nullptr;
  double w_scale = 0.0;
  if (POW) {
    const int k = c.pws->steps;
    w_in = c.pw[k & 1];
    w_out = c.pw[(k + 1) & 1];
    w_scale = c.pws->scale;
  }
  T acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = T(0);
  // double-float partial sums of h in units of 2^(et - 1023), et the largest exponent of p
  // this warp has met (0: none yet)
  float dh[DF ? M : 1], dl[DF ? M : 1];
  int et = 0;
#pragma unroll
  for (int k = 0; k < (DF ? M : 1); ++k) dh[k] = dl[k] = 0.f;
  constexpr bool STAGE = DF && df_stage_bytes<M>() > 0;  // AW slice blocks via cp.async
  float2* aw_s = reinterpret_cast<float2*>(esd_dyn_smem) + (size_t)(threadIdx.x >> 5) * M * kSlice;
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    if constexpr (STAGE) {
      // this slice's AW block (contiguous M x 256 bytes) lands in shared memory while the
      // matrix product below waits on its own loads
      __syncwarp();  // every lane is done with the previous block
      const char* src = reinterpret_cast<const char*>(c.AWdf + (size_t)s * M * kSlice);
      char* dst = reinterpret_cast<char*>(aw_s);
#pragma unroll
      for (int j = lane; j < M * kSlice * (int)sizeof(float2) / 16; j += 32) cp_async16(dst + 16 * j, src + 16 * j);
      cp_async_commit();
    }
    const int4 md = c.Av.meta[s];
    const int i = md.z + lane;
    const bool valid = lane < md.w;
    T qi;
    double wi = 0.0;
    float ph = 0.f, pl = 0.f;
    if constexpr (DF) {
      // one reference exponent per warp, so the warp can add its partial sums in double-float
      const double pv = valid ? (double)c.p[i] : 0.0;
      const int ew = (int)__reduce_max_sync(0xffffffffu, (unsigned)dexp(pv));
      if (ew > et) {  // a larger p: bring the partial sums to the new unit (exact)
        const float f = fpow2_neg(et - ew);
#pragma unroll
        for (int k = 0; k < M; ++k) {
          dh[k] = __fmul_rn(dh[k], f);
          dl[k] = __fmul_rn(dl[k], f);
        }
        et = ew;
      }
      df_split(pv, et, ph, pl);
    }
    if constexpr (POW) {
      row_fma2(c.Av, md, lane, c.p, w_in, qi, wi);
    } else if (sizeof(T) == 4 && c.rowsum) {
      const T pv = valid ? c.p[i] : T(0);
      qi = row_fma_diff(c.Av, md, lane, c.p, pv, valid ? c.rowsum[i] : T(0), T(0));
    } else {
      qi = row_fma(c.Av, md, lane, c.p, T(0));
    }
    if constexpr (STAGE) {
      cp_async_wait_all();  // this lane's copies
      __syncwarp();         // and the other lanes' copies, visible to the warp
    }
    if (valid) {
      const T pi = c.p[i];
      c.q[i] = qi;
      acc[0] = fma(pi, qi, acc[0]);
      if constexpr (DF) {
        const float2* ap = (STAGE ? aw_s : c.AWdf + (size_t)s * M * kSlice) + lane;
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const float2 a = ap[k * kSlice];
          df_fma(a.x, a.y, ph, pl, dh[k], dl[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < M; ++k) acc[1 + k] = fma(c.AW[wix<M>(c, k, i, s, lane)], pi, acc[1 + k]);
      }
      if constexpr (POW) {
        const double wv = wi * w_scale;  // A v with v = scale * w
        w_out[i] = wv;
        acc[R - 1] = fma(wv, wv, acc[R - 1]);
      }
    }
  }
  bool last;
  if constexpr (DF) {
    // warp totals: (p, q) in FP64, h in double-float converted once per warp
    const int w = threadIdx.x >> 5;
    double v = acc[0];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0) red[w * R] = v;
    df_warp_sum_chunks<0, M, R>(dh, dl, et > 0 ? dpow2(et) : 0.0, (double*)red, 1, lane_id(), w);
    last = grid_sum_from_warps<R>(red, (T*)c.partials, &st->ticket[kTkSpmv]);
  } else {
    last = grid_sum_multi<R>(acc, red, (T*)c.partials, &st->ticket[kTkSpmv]);
  }
  if (last) {
    if constexpr (POW) {
      if (threadIdx.x == 0) {
        const double ww = red[R - 1];
        PowerState* ps = c.pws;
        ps->steps += 1;
        if (ww > 0.0 && isfinite(ww)) {
          ps->scale = 1.0 / sqrt(ww);
        } else {
          ps->scale = 0.0;
          ps->failed = 1;
        }
      }
    }
    if (M > 0) {
      if (threadIdx.x < 32) {
        if constexpr (DF) {  // the double-float sums hold (AW 2^-e_k)^T p
          for (int k = threadIdx.x; k < M; k += 32) red[1 + k] *= c.awscale[k];
          __syncwarp();
        }
        double part = 0.0;
        for (int i = threadIdx.x; i < M; i += 32) {
          double y = 0.0;
          for (int k = 0; k < M; ++k) y += c.Einv[i * M + k] * (double)red[1 + k];
          st->y[i] = y;
          part += y * (double)red[1 + i];
        }
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (threadIdx.x == 0) hy_s = part;
        if constexpr (DF) {
          // y_k 2^e_k as double-float pairs for the update, relative to their largest exponent
          __syncwarp();
          int e = 0;
          for (int k = threadIdx.x; k < M; k += 32) e = max(e, dexp(st->y[k] * c.awscale[k]));
          e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
          if (e == 0) e = 1023;
          for (int k = threadIdx.x; k < M; k += 32) {
            float h, l;
            df_split(st->y[k] * c.awscale[k], e, h, l);
            st->ydf[k] = make_float2(h, l);
          }
          if (threadIdx.x == 0) st->ydf_exp = e;
        }
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
        if (M > 0 && c.x64)  // (AW)^T x_i of the FP64 iterate, for the final correction
          for (int k = 0; k < M; ++k) st->gacc[k] += a * (double)red[1 + k];
      }
    }
  }
}

// x += alpha p; r -= alpha q (deflation: r -= alpha (q - AW y)); ||r||^2; the stored
// sample of the previous iteration; SC: f = W^T r; forward level 0 (y = r / l_ii).
// do_update = 0 runs the same epilogue on r0 (start of a solve).
template <typename T, int M, int MODE, int PRE>
__global__ void __launch_bounds__(kBlock, M == 0 ? 4 : defl_minb<T, M>()) k_update(IterCtx<T> c, SliceSet set, int do_update,
                                                                  int finalize) {
  constexpr int SCM = (MODE == kModeSC) ? M : 0;
  constexpr int DM = (MODE == kModeDefl) ? M : 0;
  constexpr int R = 2 + SCM;
  constexpr bool DF = sizeof(T) == 8 && df_cols(DM);    // AW y in double-float
  constexpr bool DFS = sizeof(T) == 8 && df_cols(SCM);  // f = W^T r in double-float
  __shared__ T red[red_size<R>()];
  __shared__ T ys[DM > 0 ? DM : 1];  // y in the kernel's type: converted once per block
  __shared__ float2 ys2[DF ? DM : 1];
  __shared__ int yexp;
  __shared__ double fu_s;
  pdl_enter();
  State* st = c.st;
  if (st->conv) return;
  const T alpha = (T)st->alpha;
  const double alpha_d = st->alpha;
  const int pend = do_update ? st->pend_slot : -1;
  if (DM > 0) {
    if constexpr (DF) {
      for (int k = threadIdx.x; k < DM; k += blockDim.x) ys2[k] = st->ydf[k];
      if (threadIdx.x == 0) yexp = st->ydf_exp;
    } else {
      for (int k = threadIdx.x; k < DM; k += blockDim.x) ys[k] = (T)st->y[k];
    }
    __syncthreads();
  }
  T acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = T(0);
  // SC: double-float partial sums of f in units of 2^(et - 1023), et the largest exponent of r
  // this warp has met
  float fh[DFS ? SCM : 1], fl[DFS ? SCM : 1];
  int et = 0;
#pragma unroll
  for (int k = 0; k < (DFS ? SCM : 1); ++k) fh[k] = fl[k] = 0.f;
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    double rv = 0.0;  // this lane's r_i for the double-float f (0: no row)
    if (lane < md.w) {
      const int i = md.z + lane;
      T ri;
      if (do_update) {
        if (c.x64) {
          // refinement form: the iterate is kept in FP64, so its rounding does not drift
          // from the recursive residual
          const double xi = c.x64[i];
          if (pend >= 0) c.samples64[(size_t)pend * c.ld + i] = xi;
          c.x64[i] = fma(alpha_d, (double)c.p[i], xi);
        } else {
          const T xi = c.x[i];
          if (pend >= 0) {
            if (c.samples64) c.samples64[(size_t)pend * c.ld + i] = c.xbase[i] + (double)xi;
            else c.samples[(size_t)pend * c.ld + i] = xi;
          }
          c.x[i] = fma(alpha, c.p[i], xi);
        }
        T t = c.q[i];
        if constexpr (DF) {
          float th = 0.f, tl = 0.f;
          const float2* ap = c.AWdf + (size_t)s * DM * kSlice + lane;
#pragma unroll
          for (int k = 0; k < DM; ++k) {
            const float2 a = ap[k * kSlice];
            const float2 yk = ys2[k];
            df_fma(a.x, a.y, yk.x, yk.y, th, tl);
          }
          t -= f2d_pow2(th, yexp) + f2d_pow2(tl, yexp);
        } else {
#pragma unroll
          for (int k = 0; k < DM; ++k) t = fma(-c.AW[wix<DM>(c, k, i, s, lane)], ys[k], t);
        }
        ri = fma(-alpha, t, c.r[i]);
        c.r[i] = ri;
        acc[0] = fma(ri, ri, acc[0]);
      } else {
        ri = c.r[i];
      }
      if constexpr (DFS) {
        rv = ri;
      } else {
#pragma unroll
        for (int k = 0; k < SCM; ++k) acc[2 + k] = fma(c.W[wix<SCM>(c, k, i, s, lane)], ri, acc[2 + k]);
      }
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
    if constexpr (DFS) {
      const int ew = (int)__reduce_max_sync(0xffffffffu, (unsigned)dexp(rv));
      if (ew > et) {  // a larger r: bring the partial sums to the new unit (exact)
        const float f = fpow2_neg(et - ew);
#pragma unroll
        for (int k = 0; k < SCM; ++k) {
          fh[k] = __fmul_rn(fh[k], f);
          fl[k] = __fmul_rn(fl[k], f);
        }
        et = ew;
      }
      if (lane < md.w) {
        float rh, rl;
        df_split(rv, et, rh, rl);
        const float2* wp = c.Wdf + (size_t)s * SCM * kSlice + lane;
#pragma unroll
        for (int k = 0; k < SCM; ++k) {
          const float2 w = wp[k * kSlice];
          df_fma(w.x, w.y, rh, rl, fh[k], fl[k]);
        }
      }
    }
  }
  bool last;
  if constexpr (DFS) {
    // warp totals: ||r||^2 and the level-0 rho part in FP64, f in double-float converted once
    const int w = threadIdx.x >> 5;
    double v0 = acc[0], v1 = acc[1];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      v0 += __shfl_xor_sync(0xffffffffu, v0, o);
      v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if (lane_id() == 0) {
      red[w * R] = v0;
      red[w * R + 1] = v1;
    }
    df_warp_sum_chunks<0, SCM, R>(fh, fl, et > 0 ? dpow2(et) : 0.0, (double*)red, 2, lane_id(), w);
    last = grid_sum_from_warps<R>(red, (T*)c.partials, &st->ticket[kTkUpdate]);
  } else {
    last = grid_sum_multi<R>(acc, red, (T*)c.partials, &st->ticket[kTkUpdate]);
  }
  if (last) {
    if (SCM > 0) {
      if (threadIdx.x < 32) {
        if constexpr (DFS) {  // the double-float sums hold (W 2^-e_k)^T r
          for (int k = threadIdx.x; k < SCM; k += 32) red[2 + k] *= c.wscale[k];
          __syncwarp();
        }
        double part = 0.0;
        for (int i = threadIdx.x; i < SCM; i += 32) {
          double u = 0.0;
          for (int k = 0; k < SCM; ++k) u += c.Einv[i * SCM + k] * (double)red[2 + k];
          st->u[i] = u;
          part += u * (double)red[2 + i];
        }
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (threadIdx.x == 0) fu_s = part;
        if constexpr (DFS) {
          // u_k 2^e_k as double-float pairs for the backward sweep
          __syncwarp();
          int e = 0;
          for (int k = threadIdx.x; k < SCM; k += 32) e = max(e, dexp(st->u[k] * c.wscale[k]));
          e = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
          if (e == 0) e = 1023;
          for (int k = threadIdx.x; k < SCM; k += 32) {
            float h, l;
            df_split(st->u[k] * c.wscale[k], e, h, l);
            st->udf[k] = make_float2(h, l);
          }
          if (threadIdx.x == 0) st->udf_exp = e;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (do_update) {
        st->rr = (double)red[0];
        st->iter += 1;
        st->pend_slot = -1;
        st->fresh_dir = 0;
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
      // a run that will be resumed goes on sampling at its stop: the iterate is written by
      // the next run's first update, or the claim is undone if no run follows
      if ((!stop || st->defer_sample) && do_update && st->samp_m > 0) {
        if (st->samp_method == 1) sampling_b(st, st->bb > 0.0 ? rr / st->bb : 0.0);
        else sampling_a(st);
      }
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

// The plain-mode update (no W terms) with three slices of a warp in flight: the meta and
// flags of slice k+2, the vector entries of slice k+1, the arithmetic and stores of slice k.
// Same arithmetic as k_update<T, 0, kModePlain, PRE>. Each slice of the update is a short
// chain (meta, then five loads, then stores), so overlapping the chains of consecutive slices
// pays: 152 -> 122 us for the FP32 update at 256^3, 30 -> 26 us for FP64 at 128^3. (The same
// scheme in the SpMV and the substitutions, whose stages hold a row's matrix entries, halved
// their occupancy and measured slower.)
#ifndef ESD_UPDATE_PIPE
#define ESD_UPDATE_PIPE 1
#endif
#ifndef ESD_UPDATE_PIPE_MINB
#define ESD_UPDATE_PIPE_MINB 2
#endif
#ifndef ESD_UPDATE_PIPE_MINB_F32
#define ESD_UPDATE_PIPE_MINB_F32 3
#endif
template <typename T>
__host__ __device__ constexpr int update_pipe_minb() {
  return sizeof(T) == 4 ? ESD_UPDATE_PIPE_MINB_F32 : ESD_UPDATE_PIPE_MINB;
}

// The plain update's decision, taken by the last block with the grid totals rr = ||r||^2
// and ry = sum y_i^2 over forward level 0: the convergence test, the sampling step, and
// (finalize: no later forward launch) beta.
template <int PRE>
__device__ __forceinline__ void update_decide(State* st, double rr_new, double ry, int do_update, int finalize,
                                              double* bhist, unsigned long long cond) {
  if (do_update) {
    st->rr = rr_new;
    st->iter += 1;
    st->pend_slot = -1;
    st->fresh_dir = 0;
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
  if ((!stop || st->defer_sample) && do_update && st->samp_m > 0) {
    if (st->samp_method == 1) sampling_b(st, st->bb > 0.0 ? rr / st->bb : 0.0);
    else sampling_a(st);
  }
  st->fu = 0.0;
  if (PRE == ESD_PRECOND_IC0) st->rho_acc = ry;
  if (stop) {
    st->conv = 1;
    end_loop(cond);
  } else if (finalize) {
    const double rho_ic = (PRE == ESD_PRECOND_IC0) ? st->rho_acc : rr;
    finalize_rho(st, rho_ic, bhist, cond);
  }
}

template <typename T>
struct UpdStage {
  int4 md;
  int slice;
  int flags;
  double x;  // the iterate entry (FP64 iterate of the refinement form, or x in T)
  T p, q, r, d;
};

template <typename T, int PRE>
__device__ __forceinline__ void upd_meta(const IterCtx<T>& c, const SliceSet& set, int g, UpdStage<T>& u) {
  if (g < set.total()) {
    int r;
    u.slice = set.slice(g, &r);
    u.md = c.Av.meta[u.slice];
    u.flags = PRE == ESD_PRECOND_IC0 ? (int)c.sflags[u.slice] : 0;
  } else {
    u.md = make_int4(0, 0, 0, 0);
    u.slice = 0;
    u.flags = 0;
  }
}

template <typename T>
__device__ __forceinline__ void upd_load(const IterCtx<T>& c, int lane, int do_update, UpdStage<T>& u) {
  if (lane < u.md.w) {
    const int i = u.md.z + lane;
    if (do_update) {
      u.x = c.x64 ? c.x64[i] : (double)c.x[i];
      u.p = c.p[i];
      u.q = c.q[i];
    }
    u.r = c.r[i];
    if (u.flags & 1) u.d = c.inv_d[i];
  }
}

template <typename T, int PRE>
__global__ void __launch_bounds__(kBlock, update_pipe_minb<T>()) k_update_pipe(IterCtx<T> c, SliceSet set, int do_update,
                                                                            int finalize) {
  __shared__ T red[red_size<2>()];
  pdl_enter();
  State* st = c.st;
  if (st->conv) return;
  const T alpha = (T)st->alpha;
  const double alpha_d = st->alpha;
  const int pend = do_update ? st->pend_slot : -1;
  T acc[2] = {T(0), T(0)};
  const int lane = lane_id();
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int total = set.total();
  UpdStage<T> cur, nxt;
  upd_meta<T, PRE>(c, set, gw, cur);
  upd_load(c, lane, do_update, cur);
  upd_meta<T, PRE>(c, set, gw + nw, nxt);
  for (int g = gw; g < total; g += nw) {
    UpdStage<T> far;
    upd_meta<T, PRE>(c, set, g + 2 * nw, far);
    upd_load(c, lane, do_update, nxt);
    if (lane < cur.md.w) {
      const int i = cur.md.z + lane;
      T ri;
      if (do_update) {
        if (c.x64) {
          if (pend >= 0) c.samples64[(size_t)pend * c.ld + i] = cur.x;
          c.x64[i] = fma(alpha_d, (double)cur.p, cur.x);
        } else {
          const T xi = (T)cur.x;
          if (pend >= 0) {
            if (c.samples64) c.samples64[(size_t)pend * c.ld + i] = c.xbase[i] + (double)xi;
            else c.samples[(size_t)pend * c.ld + i] = xi;
          }
          c.x[i] = fma(alpha, cur.p, xi);
        }
        ri = fma(-alpha, cur.q, cur.r);
        c.r[i] = ri;
        acc[0] = fma(ri, ri, acc[0]);
      } else {
        ri = cur.r;
      }
      if (PRE == ESD_PRECOND_IC0 && (cur.flags & 1)) {
        const T yv = ri * cur.d;
        acc[1] = fma(yv, yv, acc[1]);
        c.Y[i] = (cur.flags & 2) ? yv * cur.d : yv;
      }
    }
    cur = nxt;
    nxt = far;
  }
  if (grid_sum_multi<2>(acc, red, (T*)c.partials, &st->ticket[kTkUpdate]) && threadIdx.x == 0)
    update_decide<PRE>(st, (double)red[0], (double)red[1], do_update, finalize, c.bhist, c.cond);
}

// One forward colour level: y_i = (r_i - sum_k l_ik y_k) / l_ii and sum y_i^2. A launch that
// is not the last stores its block totals in rho slot `slot`; the last launch adds its own
// sum, the slots of the nprev earlier launches (their grids in prevG) and the level-0 part of
// the update, then sets beta.
template <typename T>
__global__ void __launch_bounds__(kBlock, sweep_minb<T>())
    k_fwd(IterCtx<T> c, SliceSet set, int slot, int nprev, const int* __restrict__ prevG) {
  __shared__ T red[red_size<1>()];
  __shared__ double own_s;
  pdl_enter();
  State* st = c.st;
  if (st->conv) return;
  T acc[1] = {T(0)};
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Lv.meta[s];
    const int i = md.z + lane;
    const bool valid = lane < md.w;
    const T d = valid ? c.inv_d[i] : T(0);
    const T raw = row_fma<T, true>(c.Lv, md, lane, c.Y, valid ? c.r[i] : T(0));
    if (valid) {
      const T yv = raw * d;
      acc[0] = fma(yv, yv, acc[0]);
      c.Y[i] = ((set.bwd0 >> r) & 1u) ? yv * d : yv;
    }
  }
  T* slots = (T*)c.rho_part;
  if (slot >= 0) {
    block_sum_multi<1>(acc, red);
    if (threadIdx.x == 0) slots[(size_t)slot * c.rho_stride + blockIdx.x] = red[0];
    return;
  }
  if (grid_sum_multi<1>(acc, red, (T*)c.partials, &st->ticket[kTkSweep])) {
    if (threadIdx.x == 0) own_s = (double)red[0];
    T acc2[1] = {T(0)};
    for (int k = 0; k < nprev; ++k) {
      const int gk = prevG[k];
      for (int b = threadIdx.x; b < gk; b += blockDim.x) acc2[0] += __ldcg(&slots[(size_t)k * c.rho_stride + b]);
    }
    block_sum_multi<1>(acc2, red);
    if (threadIdx.x == 0) finalize_rho(st, own_s + (double)red[0] + st->rho_acc + st->fu, c.bhist, c.cond);
  }
}

// One backward colour level: z_i = (y_i - sum_j l_ji z_j) / l_ii, then
// p_i = z_i [+ (W u)_i] + beta p_i. "elem" rows had z_i stored by the forward sweep and
// only take the direction update.
template <typename T, int SCM>
__global__ void __launch_bounds__(kBlock, SCM == 0 ? sweep_minb<T>() : 1) k_bwd(IterCtx<T> c, SliceSet set, SliceSet elem) {
  constexpr bool DFS = sizeof(T) == 8 && df_cols(SCM);  // W u in double-float
  __shared__ T us[SCM > 0 ? SCM : 1];  // u in the kernel's type: converted once per block
  __shared__ float2 us2[DFS ? SCM : 1];
  __shared__ int uexp;
  pdl_enter();
  State* st = c.st;
  if (st->conv) return;
  const T beta = (T)st->beta;
  const bool first = st->iter == 0 || st->fresh_dir;
  if (SCM > 0) {
    if constexpr (DFS) {
      for (int k = threadIdx.x; k < SCM; k += blockDim.x) us2[k] = st->udf[k];
      if (threadIdx.x == 0) uexp = st->udf_exp;
    } else {
      for (int k = threadIdx.x; k < SCM; k += blockDim.x) us[k] = (T)st->u[k];
    }
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
    int4 md = c.Uv.meta[s];
    if (!sweep) md.y = 0;  // rows whose z_i the forward sweep stored: no substitution
    const int i = md.z + lane;
    const bool valid = lane < md.w;
    const T d = (valid && sweep) ? c.inv_d[i] : T(1);
    const T pold = (valid && !first) ? c.p[i] : T(0);
    const T raw = row_fma<T, true>(c.Uv, md, lane, c.Y, valid ? c.Y[i] : T(0));
    if (valid) {
      const T zic = sweep ? raw * d : raw;
      if (sweep) c.Y[i] = zic;
      T z = zic;
      if constexpr (DFS) {
        float th = 0.f, tl = 0.f;
        const float2* wp = c.Wdf + (size_t)s * SCM * kSlice + lane;
#pragma unroll
        for (int k = 0; k < SCM; ++k) {
          const float2 w = wp[k * kSlice];
          df_fma(w.x, w.y, us2[k].x, us2[k].y, th, tl);
        }
        z += f2d_pow2(th, uexp) + f2d_pow2(tl, uexp);
      } else {
#pragma unroll
        for (int k = 0; k < SCM; ++k) z = fma(c.W[wix<SCM>(c, k, i, s, lane)], us[k], z);
      }
      c.p[i] = first ? z : fma(beta, pold, z);
    }
  }
}

// No preconditioner: p = r [+ W u] + beta p.
template <typename T, int SCM>
__global__ void __launch_bounds__(kBlock, SCM == 0 ? 4 : 1) k_dir(IterCtx<T> c, SliceSet set) {
  constexpr bool DFS = sizeof(T) == 8 && df_cols(SCM);  // W u in double-float
  __shared__ T us[SCM > 0 ? SCM : 1];  // u in the kernel's type: converted once per block
  __shared__ float2 us2[DFS ? SCM : 1];
  __shared__ int uexp;
  pdl_enter();
  State* st = c.st;
  if (st->conv) return;
  const T beta = (T)st->beta;
  const bool first = st->iter == 0 || st->fresh_dir;
  if (SCM > 0) {
    if constexpr (DFS) {
      for (int k = threadIdx.x; k < SCM; k += blockDim.x) us2[k] = st->udf[k];
      if (threadIdx.x == 0) uexp = st->udf_exp;
    } else {
      for (int k = threadIdx.x; k < SCM; k += blockDim.x) us[k] = (T)st->u[k];
    }
    __syncthreads();
  }
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    if (lane < md.w) {
      const int i = md.z + lane;
      T z = c.r[i];
      if constexpr (DFS) {
        float th = 0.f, tl = 0.f;
        const float2* wp = c.Wdf + (size_t)s * SCM * kSlice + lane;
#pragma unroll
        for (int k = 0; k < SCM; ++k) {
          const float2 w = wp[k * kSlice];
          df_fma(w.x, w.y, us2[k].x, us2[k].y, th, tl);
        }
        z += f2d_pow2(th, uexp) + f2d_pow2(tl, uexp);
      } else {
#pragma unroll
        for (int k = 0; k < SCM; ++k) z = fma(c.W[wix<SCM>(c, k, i, s, lane)], us[k], z);
      }
      c.p[i] = first ? z : fma(beta, c.p[i], z);
    }
  }
}

// r = b - A x, ||b||^2, ||r||^2 (start of a solve).
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_residual0(IterCtx<T> c, SliceSet set) {
  __shared__ T red[red_size<2>()];
  pdl_enter();
  State* st = c.st;
  T acc[2] = {T(0), T(0)};
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    T ax = T(0);
    if (!c.x_zero) {
      if (sizeof(T) == 4 && c.rowsum) {
        const bool valid = lane < md.w;
        const int i = md.z + lane;
        ax = row_fma_diff(c.Av, md, lane, c.x, valid ? c.x[i] : T(0), valid ? c.rowsum[i] : T(0), T(0));
      } else {
        ax = row_fma(c.Av, md, lane, c.x, T(0));
      }
    }
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
      for (int k = 0; k < kMaxM; ++k) st->gacc[k] = 0.0;
    }
  }
}

// f = X^T v - Y^T w (Y optional), u = E^-1 f (stored in st->u).
template <typename T, int M>
__global__ void __launch_bounds__(kBlock) k_tallT(IterCtx<T> c, SliceSet set, const T* X, const T* v,
                                                  const T* Y2, const T* w, int sub_gacc) {
  __shared__ T red[red_size<M>()];
  pdl_enter();
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
      for (int k = 0; k < M; ++k) acc[k] = fma(X[wix<M>(c, k, i, s, lane)], vi, acc[k]);
      if (Y2) {
        const T wi = w[i];
#pragma unroll
        for (int k = 0; k < M; ++k) acc[k] = fma(-Y2[wix<M>(c, k, i, s, lane)], wi, acc[k]);
      }
    }
  }
  if (grid_sum_multi<M>(acc, red, (T*)c.partials, &st->ticket[kTkAux])) {
    if (threadIdx.x < 32) {
      for (int i = threadIdx.x; i < M; i += 32) {
        double u = 0.0;
        for (int k = 0; k < M; ++k) u += c.Einv[i * M + k] * ((double)red[k] - (sub_gacc ? st->gacc[k] : 0.0));
        st->u[i] = u;
      }
    }
  }
}

// v += sign * Z u (u = st->u); optionally ||v||^2 into st->rr.
template <typename T, int M>
__global__ void __launch_bounds__(kBlock) k_tall_axpy(IterCtx<T> c, SliceSet set, const T* Z, T* v,
                                                      T sign, int norm) {
  __shared__ T red[red_size<1>()];
  __shared__ T us[M];  // u in the kernel's type: converted once per block
  pdl_enter();
  State* st = c.st;
  for (int k = threadIdx.x; k < M; k += blockDim.x) us[k] = (T)st->u[k];
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
      for (int k = 0; k < M; ++k) t = fma(Z[wix<M>(c, k, i, s, lane)], us[k], t);
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

// x64 += Z u (u = st->u): the correction summed in T, added to the FP64 iterate.
template <typename T, int M>
__global__ void __launch_bounds__(kBlock) k_tall_axpy64(IterCtx<T> c, SliceSet set, const T* Z) {
  __shared__ T us[M];  // u in the kernel's type: converted once per block
  pdl_enter();
  State* st = c.st;
  for (int k = threadIdx.x; k < M; k += blockDim.x) us[k] = (T)st->u[k];
  __syncthreads();
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    if (lane < md.w) {
      const int i = md.z + lane;
      T t = T(0);
#pragma unroll
      for (int k = 0; k < M; ++k) t = fma(Z[wix<M>(c, k, i, s, lane)], us[k], t);
      c.x64[i] += (double)t;
    }
  }
}

// The sample due at the last iteration (none is taken at the converging one), x = 0 for b = 0.
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_finish(IterCtx<T> c, SliceSet set) {
  pdl_enter();
  const State* st = c.st;
  const int pend = st->defer_sample ? -1 : st->pend_slot;
  const bool zero = st->zero_rhs;
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    if (lane < md.w) {
      const int i = md.z + lane;
      if (pend >= 0 && c.samples64) c.samples64[(size_t)pend * c.ld + i] = c.xbase[i] + (double)c.x[i];
      else if (pend >= 0 && c.samples) c.samples[(size_t)pend * c.ld + i] = c.x[i];
      if (zero) c.x[i] = T(0);
    }
  }
}

// ||b - A x||^2
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_true_res(IterCtx<T> c, SliceSet set) {
  __shared__ T red[red_size<1>()];
  pdl_enter();
  State* st = c.st;
  T acc[1] = {T(0)};
  ESD_LOOP_SLICES(set) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = c.Av.meta[s];
    const int i = md.z + lane;
    const bool valid = lane < md.w;
    const T t = row_fma(c.Av, md, lane, c.x, valid ? -c.b[i] : T(0));  // A x - b
    if (valid) acc[0] = fma(t, t, acc[0]);
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

}  // namespace esd

#include "esd_stream.cuh"
#include "esd_stream_pair.cuh"

namespace esd {

#define ESD_DISPATCH_MPOS(Mrt, ...)                                                   \
  switch (Mrt) {                                                                      \
    case 8: { constexpr int MM = 8; __VA_ARGS__; } break;                             \
    case 16: { constexpr int MM = 16; __VA_ARGS__; } break;                           \
    case 24: { constexpr int MM = 24; __VA_ARGS__; } break;                           \
    case 32: { constexpr int MM = 32; __VA_ARGS__; } break;                           \
    case 64: { constexpr int MM = 64; __VA_ARGS__; } break;                           \
    default: throw Error(ESD_ERR_INVALID, "unsupported padded column count");         \
  }

// launch kernel K over `slices` slices with one wave at most
#define ESD_LAUNCH(K, slices, s, ...) launch_pdl(K, grid_for(K, (slices)), (s), __VA_ARGS__)

template <typename T, int M, int MODE, int PRE>
static void launch_update_k(const IterCtx<T>& c, int do_update, int finalize, cudaStream_t s) {
  auto k = k_update<T, M, MODE, PRE>;
  ESD_LAUNCH(k, c.A->all.total(), s, c, c.A->all, do_update, finalize);
}

template <typename T>
static void launch_update(const IterCtx<T>& c, int do_update, int finalize, cudaStream_t s,
                          KernelMarks* marks = nullptr) {
  const int Mm = (c.mode == ESD_PLAIN) ? 0 : c.M;
  const esd_matrix* P = c.P ? c.P : c.A;  // its forward level 0 rides on the update
  if (sizeof(T) == 4 && c.mode == ESD_PLAIN && c.x64 && P->upd_ok && stream_enabled()) {
    // FP32 plain update of the refinement form, vectors staged by bulk copies
    if constexpr (sizeof(T) == 4) {
      int K = 1;
      const bool ic = c.pre == ESD_PRECOND_IC0;
      const StreamPlan pl = ic ? stream_plan(P->upd_sets[0], P->upd_sets[1], 0, 0, 4, 1, &K)
                               : stream_plan(SliceSet{}, c.A->all, 0, 0, 4, 1, &K);
      if (ic) {
        auto k = k_update_stream<T, ESD_PRECOND_IC0>;
        launch_stream(k, stream_blocks(k, pl), pl, s, c, pl, do_update, finalize);
      } else {
        auto k = k_update_stream<T, ESD_PRECOND_NONE>;
        launch_stream(k, stream_blocks(k, pl), pl, s, c, pl, do_update, finalize);
      }
    }
  } else if (c.mode == ESD_PLAIN && ESD_UPDATE_PIPE) {
    if (c.pre == ESD_PRECOND_IC0) {
      auto k = k_update_pipe<T, ESD_PRECOND_IC0>;
      ESD_LAUNCH(k, c.A->all.total(), s, c, c.A->all, do_update, finalize);
    } else {
      auto k = k_update_pipe<T, ESD_PRECOND_NONE>;
      ESD_LAUNCH(k, c.A->all.total(), s, c, c.A->all, do_update, finalize);
    }
  } else if (c.pre == ESD_PRECOND_IC0) {
    if (c.mode == ESD_PLAIN) {
      launch_update_k<T, 0, kModePlain, ESD_PRECOND_IC0>(c, do_update, finalize, s);
    } else if (c.mode == ESD_DEFLATION) {
      ESD_DISPATCH_MPOS(Mm, (launch_update_k<T, MM, kModeDefl, ESD_PRECOND_IC0>(c, do_update, finalize, s)))
    } else {
      ESD_DISPATCH_MPOS(Mm, (launch_update_k<T, MM, kModeSC, ESD_PRECOND_IC0>(c, do_update, finalize, s)))
    }
  } else {
    if (c.mode == ESD_PLAIN) {
      launch_update_k<T, 0, kModePlain, ESD_PRECOND_NONE>(c, do_update, finalize, s);
    } else if (c.mode == ESD_DEFLATION) {
      ESD_DISPATCH_MPOS(Mm, (launch_update_k<T, MM, kModeDefl, ESD_PRECOND_NONE>(c, do_update, finalize, s)))
    } else {
      ESD_DISPATCH_MPOS(Mm, (launch_update_k<T, MM, kModeSC, ESD_PRECOND_NONE>(c, do_update, finalize, s)))
    }
  }
  if (marks) marks->mark(s, "update");
}

// The FP32 substitutions of P stream their factor entries through staged shared memory
// (k_fwd_stream, k_bwd_stream) when every factor row fits a stage.
template <typename T>
static bool stream_sweeps(const esd_matrix* P) {
  return sizeof(T) == 4 && stream_enabled() && P->L.wmax <= kStreamWmax && P->U.wmax <= kStreamWmax;
}

// The staged sweeps read the column-free copies of L and U when both parts have one.
static bool affine_sweeps(const esd_matrix* P) { return P->L.affine && P->U.affine; }

// Plan of a staged launch over `with_entries` (+ `vectors_only`) of a part whose widest slice
// has wmax entries, or awmax slots in its column-free copy (aff), with nv4 staged FP32 vectors.
inline StreamPlan staged_plan(const SliceSet& with_entries, const SliceSet& vectors_only, bool aff, int wmax,
                              int awmax, int nv4, int* K) {
  return aff ? stream_plan(with_entries, vectors_only, awmax, 4, nv4, 0, K, true, kHdrAffine)
             : stream_plan(with_entries, vectors_only, wmax, 8, nv4, 0, K);
}

// Plan and grid of forward launch l (the last forward launch reads the rho block totals of
// the earlier ones, so every launch of a sweep uses exactly this grid).
template <typename T>
static int fwd_grid(const esd_matrix* P, size_t l, StreamPlan* plan = nullptr, int* K_out = nullptr) {
  const SliceSet& set = P->fwd_sets[l];
  if constexpr (sizeof(T) == 4) {
    if (stream_sweeps<T>(P)) {
      int K = 1;
      const bool aff = affine_sweeps(P);
      const StreamPlan pl = staged_plan(set, SliceSet{}, aff, P->fwd_wmax[l], aff ? P->fwd_awmax[l] : 0, 2, &K);
      if (plan) *plan = pl;
      if (K_out) *K_out = K;
      int G = 0;
      ESD_DISPATCH_K(K, {
        G = aff ? stream_blocks(k_fwd_stream<T, KK, WW, true>, pl) : stream_blocks(k_fwd_stream<T, KK, WW, false>, pl);
      });
      return G;
    }
  }
  auto kf = k_fwd<T>;
  return grid_for(kf, set.total());
}

// forward levels >= 1 then backward levels (with the direction update)
template <typename T>
std::vector<int> fwd_grids(const esd_matrix* P) {
  std::vector<int> g;
  for (size_t l = 0; l < P->fwd_sets.size(); ++l) g.push_back(fwd_grid<T>(P, l));
  return g;
}

template <typename T>
static void launch_precond(const IterCtx<T>& c, cudaStream_t s, KernelMarks* marks = nullptr) {
  const esd_matrix* A = c.P ? c.P : c.A;  // the preconditioning matrix (same slices as c.A)
  const int SCM = (c.mode == ESD_SUBSPACE_CORRECTION) ? c.M : 0;
  if (c.pre == ESD_PRECOND_NONE) {
    ESD_DISPATCH_M(SCM, { auto k = k_dir<T, MM>; ESD_LAUNCH(k, A->all.total(), s, c, A->all); });
    if (marks) marks->mark(s, "dir");
    return;
  }
  const size_t nf = A->fwd_sets.size();
  const int* dG = sizeof(T) == 8 ? A->fwd_grid64.as<int>() : A->fwd_grid32.as<int>();
  const bool staged = stream_sweeps<T>(A);
  if (staged)
    ESD_CHECK(c.Lv.ent && c.Uv.ent, ESD_ERR_INTERNAL, "the staged sweeps need the FP32 (value, column) factor entries");
  auto kf = k_fwd<T>;
  for (size_t l = 0; l < nf; ++l) {
    const SliceSet& set = A->fwd_sets[l];
    StreamPlan pl{};
    int K = 1;
    const int G = fwd_grid<T>(A, l, &pl, &K);
    const bool last = l + 1 == nf;
    if constexpr (sizeof(T) == 4) {
      if (staged) {
        const int slot = last ? -1 : (int)l, nprev = last ? (int)l : 0;
        ESD_DISPATCH_K(K, {
          if (affine_sweeps(A)) launch_stream(k_fwd_stream<T, KK, WW, true>, G, pl, s, c, pl, slot, nprev, dG);
          else launch_stream(k_fwd_stream<T, KK, WW, false>, G, pl, s, c, pl, slot, nprev, dG);
        });
      }
    }
    if (!staged) launch_pdl(kf, G, s, c, set, last ? -1 : (int)l, last ? (int)l : 0, dG);
    if (marks) marks->mark(s, ("fwd_" + std::to_string(l + 1)).c_str());
  }
  SliceSet none{};
  const size_t nb = std::max(A->bwd_sets.size(), A->bwd0_sets.size());
  for (size_t l = 0; l < nb; ++l) {
    const SliceSet& sw = l < A->bwd_sets.size() ? A->bwd_sets[l] : none;
    const SliceSet& el = l < A->bwd0_sets.size() ? A->bwd0_sets[l] : none;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (staged && SCM == 0) {
        int K = 1;
        const bool aff = affine_sweeps(A);
        const bool has = l < A->bwd_sets.size();
        const StreamPlan pl = staged_plan(sw, el, aff, has ? A->bwd_wmax[l] : 0, has && aff ? A->bwd_awmax[l] : 0, 3, &K);
        ESD_DISPATCH_K(K, {
          if (aff) {
            auto k = k_bwd_stream<T, KK, WW, true>;
            launch_stream(k, stream_blocks(k, pl), pl, s, c, pl);
          } else {
            auto k = k_bwd_stream<T, KK, WW, false>;
            launch_stream(k, stream_blocks(k, pl), pl, s, c, pl);
          }
        });
        done = true;
      }
    }
    if (!done) ESD_DISPATCH_M(SCM, { auto k = k_bwd<T, MM>; ESD_LAUNCH(k, sw.total() + el.total(), s, c, sw, el); });
    if (marks) marks->mark(s, ("bwd_" + std::to_string(l + 1)).c_str());
  }
}

template <typename T>
void launch_init(const IterCtx<T>& c, cudaStream_t s) {
  const SliceSet& all = c.A->all;
  {
    auto k = k_residual0<T>;
    ESD_LAUNCH(k, all.total(), s, c, all);
  }
  if (c.mode == ESD_DEFLATION) {
    // r0 = P^T (b - A x0) = r - AW E^-1 W^T r
    ESD_DISPATCH_MPOS(c.M, {
      auto k = k_tallT<T, MM>;
      ESD_LAUNCH(k, all.total(), s, c, all, (const T*)c.W, (const T*)c.r, (const T*)nullptr, (const T*)nullptr, 0);
    });
    ESD_DISPATCH_MPOS(c.M, {
      auto k = k_tall_axpy<T, MM>;
      ESD_LAUNCH(k, all.total(), s, c, all, (const T*)c.AW, c.r, T(-1), 1);
    });
  }
  const bool fin = c.pre == ESD_PRECOND_NONE || (c.P ? c.P : c.A)->fwd_sets.empty();
  launch_update<T>(c, 0, fin ? 1 : 0, s);
  launch_precond<T>(c, s);
}

template <typename T>
void launch_iteration(const IterCtx<T>& c, cudaStream_t s, KernelMarks* marks) {
  const SliceSet& all = c.A->all;
  const int Mm = (c.mode == ESD_DEFLATION) ? c.M : 0;
  if (marks) marks->mark(s, "start");
  if (c.pws) {
    if constexpr (sizeof(T) == 8) {
      if (Mm != 0) throw Error(ESD_ERR_STATE, "the power method runs in plain or subspace-correction mode");
      auto k = k_spmv_pq<T, 0, true>;
      ESD_LAUNCH(k, all.total(), s, c, all);
    } else {
      throw Error(ESD_ERR_STATE, "the power method runs in FP64 solves");
    }
  } else if (sizeof(T) == 8 && df_cols(Mm)) {  // double-float deflation terms, AW staged in shared memory
    ESD_DISPATCH_MPOS(Mm, {
      auto k = k_spmv_pq<T, MM>;
      launch_pdl_smem(k, all.total(), df_stage_bytes<MM>(), s, c, all);
    });
  } else if (sizeof(T) == 4 && Mm == 0 && c.rowsum && c.Av.ent && c.A->A.wmax <= kStreamWmax &&
             stream_enabled()) {
    // FP32 plain product: the matrix stream staged by bulk copies
    if constexpr (sizeof(T) == 4) {
      int K = 1;
      const bool aff = c.A->A.affine;
      const StreamPlan pl = staged_plan(all, SliceSet{}, aff, c.A->A.wmax, c.A->A.awmax, 2, &K);
      ESD_DISPATCH_K(K, {
        if (aff) {
          auto k = k_spmv_pq_stream<T, KK, WW, true>;
          launch_stream(k, stream_blocks(k, pl), pl, s, c, pl);
        } else {
          auto k = k_spmv_pq_stream<T, KK, WW, false>;
          launch_stream(k, stream_blocks(k, pl), pl, s, c, pl);
        }
      });
    }
  } else {
    ESD_DISPATCH_M(Mm, { auto k = k_spmv_pq<T, MM>; ESD_LAUNCH(k, all.total(), s, c, all); });
  }
  if (marks) marks->mark(s, "spmv_pq");
  const bool fin = c.pre == ESD_PRECOND_NONE || (c.P ? c.P : c.A)->fwd_sets.empty();
  launch_update<T>(c, 1, fin ? 1 : 0, s, marks);
  launch_precond<T>(c, s, marks);
}

template <typename T>
void launch_finish(const IterCtx<T>& c, cudaStream_t s) {
  const SliceSet& all = c.A->all;
  if (c.mode == ESD_DEFLATION) {
    // x = P x_i + W E^-1 W^T b = x_i + W E^-1 (W^T b - (AW)^T x_i); with the FP64 iterate
    // (AW)^T x_i was accumulated along the iteration
    if (c.x64) {
      ESD_DISPATCH_MPOS(c.M, {
        auto k = k_tallT<T, MM>;
        ESD_LAUNCH(k, all.total(), s, c, all, (const T*)c.W, (const T*)c.b, (const T*)nullptr, (const T*)nullptr, 1);
      });
      ESD_DISPATCH_MPOS(c.M, {
        auto k = k_tall_axpy64<T, MM>;
        ESD_LAUNCH(k, all.total(), s, c, all, (const T*)c.W);
      });
    } else {
      ESD_DISPATCH_MPOS(c.M, {
        auto k = k_tallT<T, MM>;
        ESD_LAUNCH(k, all.total(), s, c, all, (const T*)c.W, (const T*)c.b, (const T*)c.AW, (const T*)c.x, 0);
      });
      ESD_DISPATCH_MPOS(c.M, {
        auto k = k_tall_axpy<T, MM>;
        ESD_LAUNCH(k, all.total(), s, c, all, (const T*)c.W, c.x, T(1), 0);
      });
    }
  }
  {
    auto k = k_finish<T>;
    ESD_LAUNCH(k, all.total(), s, c, all);
  }
}

#define ESD_INSTANTIATE_ITER(T)                                                        \
  template std::vector<int> fwd_grids<T>(const esd_matrix*);                          \
  template void launch_init<T>(const IterCtx<T>&, cudaStream_t);                      \
  template void launch_iteration<T>(const IterCtx<T>&, cudaStream_t, KernelMarks*);   \
  template void launch_finish<T>(const IterCtx<T>&, cudaStream_t);

}  // namespace esd
