// Shared definitions of the CUDA path: sliced-ELL matrix views, the device-resident solver
// state, the grid-wide deterministic reductions and the error plumbing.
//
// Matrix layout (HBM): rows are grouped by colour; each colour is cut into slices of 32
// consecutive rows. A slice stores its entries column-major (entry k of lane l at
// off + 32*k + l), so the 32 threads of a warp, one per row, read consecutive words.
// Rows shorter than the slice width are padded with (column n, value 0); every vector the
// kernels gather from carries a sentinel element n that is always 0, so padding adds an
// exact zero. The same slicing serves A, the strict lower factor L and its transpose U.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>

#include "esdcg.h"

namespace esd {

constexpr int kSlice = 32;      // rows per slice (one warp, one row per lane)
constexpr int kBlock = 512;     // threads per block of the streaming kernels
constexpr int kMaxM = 64;       // maximum number of columns of W
constexpr int kMaxRanges = 16;  // slice ranges one launch may cover
constexpr int kMaxColours = 2048;  // e.g. the 3N-2 wavefronts of natural-order IC(0) on N^3

// A set of slice ranges processed by one launch (the colours of one level).
struct SliceSet {
  int nr;                       // number of ranges
  int begin[kMaxRanges];        // first slice of each range
  int cum[kMaxRanges + 1];      // prefix sums of range lengths (cum[0] = 0)
  unsigned fwd0;                // bit r: rows of range r have no earlier neighbour
  unsigned bwd0;                // bit r: rows of range r have no later neighbour
  __host__ __device__ int total() const { return cum[nr]; }
  // slice index of the g-th slice of the set, and the range it belongs to
  __device__ __forceinline__ int slice(int g, int* range) const {
    int r = 0;
#pragma unroll 1
    while (r + 1 < nr && g >= cum[r + 1]) ++r;
    *range = r;
    return begin[r] + (g - cum[r]);
  }
};

// meta per slice: x = entry offset, y = width, z = first row, w = rows in the slice
template <typename T>
struct SellView {
  const int4* meta;
  const int* col;
  const T* val;
  const uint2* ent = nullptr;  // FP32 copy: (value bits, column) per entry, one 8-byte load
  // FP32 column-free copy (null when the part has none): metas, slot bases, values
  const int4* ameta = nullptr;
  const int* abase = nullptr;
  const float* aval = nullptr;
};

// Device-resident scalar state of one solve. All Krylov scalars stay here; the host reads
// it back once per solve.
struct State {
  double bb;        // ||b||^2
  double rr;        // ||r||^2 of the recursive (deflated) residual
  double tol2bb;    // tol^2 ||b||^2
  double rho;       // (r, z) of the current iteration
  double rho_prev;  // (r, z) of the previous iteration
  double rho_acc;   // running sum of y_i^2 over the forward levels
  double pq;        // (p, A p)
  double pap;       // (p, P^T A p) in deflation, = pq otherwise
  double alpha, beta;
  double fu;        // f^T E^{-1} f of the subspace correction
  double true_rr;   // ||b - A x||^2 recomputed after the solve
  double scal0, scal1;  // scratch for auxiliary kernels
  int iter;         // alpha steps taken
  int maxit;
  int conv;         // 1 once the loop must stop (converged, maxit or breakdown)
  int status;       // ESD_OK / ESD_ERR_MAXIT / ESD_ERR_BREAKDOWN
  int zero_rhs;
  int samp_m;       // sampling method A: number of slots in use (0 = off)
  int lmax;
  int h;            // the interval h of sampling method A
  int pend_slot;    // slot to receive x at the next update (-1 = none)
  int pend_prev;    // slot_iter[pend_slot] before it was claimed (a deferred sample's undo)
  int guard;        // loop bodies started; a second, reduction-free bound on the loop
  int paired;       // bodies of a pair's paired loop started (kept in the first system's state)
  int defer_sample; // resumed runs: a stopping run leaves its sample to the run that resumes
  int fresh_dir;    // the next direction update starts afresh (p = z) without resetting iter
  int samp_method;  // 0: sampling method A, 1: method B (relative residual levels)
  int sb_reached;   // method B: residual levels reached so far
  int sb_used;      // method B: slots filled so far
  int slot_iter[kMaxM];
  double y[kMaxM];  // deflation: E^{-1} (AW)^T p
  double u[kMaxM];  // subspace correction / projection: E^{-1} f
  double gacc[kMaxM];  // FP64-iterate deflation: (AW)^T x_i accumulated as sum alpha_k h_k
  float2 ydf[kMaxM];   // FP64 deflation: y_k c_k 2^(1023-ey) as double-float pairs (c_k: AW column scales)
  int ydf_exp;         // ey, a biased binary exponent
  float2 udf[kMaxM];   // FP64 subspace correction: u_k c_k 2^(1023-eu) as double-float pairs (c_k: W scales)
  int udf_exp;         // eu
  unsigned int ticket[8];
};

enum Ticket { kTkSpmv = 0, kTkUpdate = 1, kTkSweep = 2, kTkAux = 3, kTkAux2 = 4 };

// Power method of the condition estimate (Section 5.4). It lives across solves: each CG
// iteration multiplies the power vector by A in the same matrix pass as A p. The vector is
// kept unnormalised as w (the raw product) with its normalising factor: v = scale * w.
struct PowerState {
  double scale;  // 1 / ||w||_2 of the stored w
  double ww;     // ||w||^2 of the last Rayleigh-quotient pass
  double wAw;    // (w, A w) of the last Rayleigh-quotient pass
  int steps;     // products taken since the start vector; w lives in buffer steps & 1
  int failed;    // a norm was zero or not finite
  unsigned int ticket;
};

// Device state of the FP64 iterative refinement around FP32 inner solves.
struct RefineState {
  double bb;          // ||b||^2
  double rr;          // ||b - A x||^2 of the current FP64 iterate
  double tol2bb;      // tol^2 ||b||^2
  double inner_tol2;  // relative tolerance^2 of every inner solve
  int outer;          // refinement steps done
  int max_outer;
  int inner_total;    // inner iterations over all steps
  int inner_maxit;
  int samp_m;         // sampling in the first inner solve (0 = off)
  int lmax;
  int status;
  int conv;
  unsigned int ticket;
  int first_inner;    // iterations of the first inner solve (the sampled one)
  int keep;           // 1: every step resumes CG with the previous step's direction
  int fresh;          // the step about to start resumes with p = z (the gap was too large)
  int restarts;       // resumed steps that restarted the direction
  int breakdowns;     // inner runs that ended in a breakdown
  int nonfinite;      // the FP64 residual was not finite
  int stalled;        // consecutive steps that did not lower the best residual by 10%
  double rr_best;     // the lowest ||b - A x||^2 so far
  double max_gap;     // largest ||r_true - r_inner|| / ||r_true|| at a resumed step
};

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define ESD_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw ::esd::Error(ESD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define ESD_CHECK(cond, code, msg)                   \
  do {                                               \
    if (!(cond)) throw ::esd::Error((code), (msg));  \
  } while (0)

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Sum of P values held by each lane of a warp: a butterfly that halves the values a lane
// holds at each exchange, so 32 values cost 31 additions per lane instead of 5 x 32.
// On return v[0] of lane l holds the warp total of value index warp_sum_index<P>(l).
template <int P, typename T>
__device__ __forceinline__ void warp_sum_multi(T (&v)[P]) {
  static_assert((P & (P - 1)) == 0 && P <= 32, "P must be a power of two <= 32");
  const int lane = lane_id();
  int h = P / 2;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (h >= 1) {
      const bool upper = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < (P / 2 > 0 ? P / 2 : 1); ++k) {
        if (k < h) {
          T send = upper ? v[k] : v[k + h];
          T keep = upper ? v[k + h] : v[k];
          v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      h >>= 1;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
}

template <int P>
__device__ __forceinline__ int warp_sum_index(int lane) {
  int idx = 0, h = P / 2;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (h >= 1) {
      if (lane & o) idx += h;
      h >>= 1;
    }
  }
  return idx;
}

__host__ __device__ constexpr int pow2_floor(int x) {
  return x >= 32 ? 32 : (x >= 16 ? 16 : (x >= 8 ? 8 : (x >= 4 ? 4 : (x >= 2 ? 2 : 1))));
}

// Warp totals of in[C0 .. R) in exact power-of-two chunks (17 values = 16 + 1), written by
// one lane per value into red[warp * R + j].
template <int C0, int R, typename T>
__device__ __forceinline__ void warp_sum_chunks(const T (&in)[R], T* red, int lane, int warp) {
  if constexpr (C0 < R) {
    constexpr int C = pow2_floor(R - C0);
    T v[C];
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = in[C0 + k];
    warp_sum_multi<C>(v);
    const int idx = warp_sum_index<C>(lane);
    if ((lane & ((32 / C) - 1)) == 0) red[warp * R + C0 + idx] = v[0];
    warp_sum_chunks<C0 + C, R>(in, red, lane, warp);
  }
}

// Block-wide sum of R values per thread (R <= 64) with one block barrier: a butterfly per
// warp, then warp 0 adds the warp totals. On return red[0..R) holds the totals, visible to
// warp 0 (and to every thread when R > 32). red needs (blockDim/32 + 1) * R entries.
// Second stage of block_sum_multi: red[w * R + j] holds warp w's totals (written before a
// block barrier); warp 0 adds them into red[0..R).
template <int R, typename T>
__device__ __forceinline__ void block_combine_warps(T* red) {
  const int lane = lane_id(), warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (warp == 0) {
    for (int j = lane; j < R; j += 32) {
      T s = 0;
      for (int w = 0; w < nwarp; ++w) s += red[w * R + j];
      red[j] = s;
    }
    __syncwarp();
  }
  if (R > 32) __syncthreads();
}

template <int R, typename T>
__device__ __forceinline__ void block_sum_multi(const T (&in)[R], T* red) {
  const int lane = lane_id(), warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  warp_sum_chunks<0, R>(in, red, lane, warp);
  __syncthreads();
  if (warp == 0) {
    for (int j = lane; j < R; j += 32) {
      T s = 0;
      for (int w = 0; w < nwarp; ++w) s += red[w * R + j];
      red[j] = s;
    }
    __syncwarp();
  }
  if (R > 32) __syncthreads();
}

// Shared-memory entries block_sum_multi<R> needs for kBlock threads.
template <int R>
__host__ __device__ constexpr int red_size() {
  return (kBlock / 32 + 1) * R;
}

// Grid-wide deterministic sum: every block stores its R block totals into
// partials[j * gridDim.x + blockIdx.x]; the last block to arrive adds them up in a fixed
// order and returns true with the totals in red[0..R). No block ever waits for another.
template <int R, typename T>
__device__ __forceinline__ bool grid_sum_stage(T* red, T* partials, unsigned int* ticket);

template <int R, typename T>
__device__ __forceinline__ bool grid_sum_multi(const T (&in)[R], T* red, T* partials,
                                               unsigned int* ticket) {
  block_sum_multi<R>(in, red);
  return grid_sum_stage<R>(red, partials, ticket);
}

// grid_sum_multi from warp totals already in red[w * R + j] (see block_combine_warps)
template <int R, typename T>
__device__ __forceinline__ bool grid_sum_from_warps(T* red, T* partials, unsigned int* ticket) {
  __syncthreads();
  block_combine_warps<R>(red);
  return grid_sum_stage<R>(red, partials, ticket);
}

// Block totals in red[0..R) -> partials; the last block to arrive adds them up.
template <int R, typename T>
__device__ __forceinline__ bool grid_sum_stage(T* red, T* partials, unsigned int* ticket) {
  __shared__ bool s_last;
  const int G = gridDim.x;
  if (threadIdx.x < R) {
    partials[threadIdx.x * G + blockIdx.x] = red[threadIdx.x];
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == (unsigned)G - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  T acc[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    T s = 0;
    for (int b = threadIdx.x; b < G; b += blockDim.x) s += __ldcg(&partials[j * G + b]);
    acc[j] = s;
  }
  block_sum_multi<R>(acc, red);
  if (threadIdx.x == 0) *ticket = 0u;  // ready for the next launch
  return true;
}

// Programmatic dependent launch: wait for the grids this one depends on (their memory is
// visible afterwards), then let the grids that depend on this one be scheduled.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// u = Einv f for the small dense (padded) M x M inverse stored row-major; one warp.
__device__ __forceinline__ void small_matvec_warp(const double* Einv, int M, const double* f,
                                                  double* u) {
  for (int i = lane_id(); i < M; i += 32) {
    double s = 0.0;
    for (int k = 0; k < M; ++k) s += Einv[i * M + k] * f[k];
    u[i] = s;
  }
}

}  // namespace esd
