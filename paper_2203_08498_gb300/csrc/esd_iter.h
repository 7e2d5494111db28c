// Launchers of the Krylov-iteration kernels. One IterCtx describes the buffers of one
// precision (double for the FP64 solver, float for the FP32 inner solver of the refinement).
#pragma once

#include <string>
#include <vector>

#include "esd_internal.h"

namespace esd {

// FP64 deflation with double-float W terms for up to this many (padded) columns; beyond, the
// 2M float accumulators of the SpMV no longer fit in registers and the terms stay FP64
__host__ __device__ constexpr bool df_cols(int M) { return M > 0 && M <= 32; }

template <typename T>
struct IterCtx {
  const esd_matrix* A = nullptr;
  SellView<T> Av{}, Lv{}, Uv{};
  const T* inv_d = nullptr;
  const T* rowsum = nullptr;  // set: A v is formed as s_i v_i + sum_j a_ij (v_j - v_i)
  T* b = nullptr;   // right-hand side
  T* x = nullptr;   // iterate
  T* r = nullptr;   // residual (deflated residual in deflation mode)
  T* p = nullptr;   // search direction
  T* q = nullptr;   // A p
  T* Y = nullptr;   // forward then backward substitution values (y, then L^-T y)
  // the paired kernels of two FP32 systems: (p_1, p_2) and (y_1, y_2) side by side
  float2* p12 = nullptr;
  float2* Y12 = nullptr;
  const T* W = nullptr;   // n x M column-major, stride ld
  const T* AW = nullptr;  // n x M column-major, stride ld
  size_t ld = 0;          // vector stride in elements
  const double* Einv = nullptr;  // M x M row-major (zero-padded)
  int M = 0;              // padded number of W columns (0, 8, 16, 24, 32, 64)
  T* samples = nullptr;   // sample slots, stride ld
  double* samples64 = nullptr;   // refinement form: FP64 slots receive xbase + x instead
  double* x64 = nullptr;  // refinement form: the iterate is updated here in FP64 (x stays 0)
  const double* xbase = nullptr;  // refinement form: the FP64 iterate the inner x corrects
  double* ahist = nullptr;
  double* bhist = nullptr;
  void* partials = nullptr;
  void* rho_part = nullptr;     // block totals of the forward launches before the last one
  size_t rho_stride = 0;        // entries per forward launch in rho_part
  const esd_matrix* P = nullptr;  // matrix whose IC(0) factor and colour levels precondition (A)
  State* st = nullptr;
  const unsigned char* sflags = nullptr;
  unsigned long long cond = 0;  // graph conditional handle (0 = none)
  int mode = ESD_PLAIN;
  int pre = ESD_PRECOND_IC0;
  int x_zero = 0;  // the start vector is known to be zero (r0 = b without a product)
  int wsm = 0;     // W and AW slice-major: entry (row of slice s, lane l; column k) at (s M + k) 32 + l
  // FP64 deflation: AW as double-float pairs, slice-major ((s M + k) 32 + lane), column k
  // scaled by 2^-e_k so that its largest entry lies in [1/2, 1); awscale[k] = 2^e_k
  const float2* AWdf = nullptr;
  const double* awscale = nullptr;
  const float2* Wdf = nullptr;     // W in the same form (FP64 subspace correction)
  const double* wscale = nullptr;
  // power method (FP64 plain / SC solves): w in pw[steps & 1], the next product into the other
  double* pw[2] = {nullptr, nullptr};
  PowerState* pws = nullptr;
};

// Optional event marks between the kernels of a launch sequence (profiling): mark() records
// an event after each kernel, labelled with the kernel's name.
struct KernelMarks {
  std::vector<cudaEvent_t> ev;
  std::vector<std::string> names;
  void mark(cudaStream_t s, const char* name) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    ev.push_back(e);
    names.push_back(name);
  }
  ~KernelMarks() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

// Grid of each forward launch of P's substitution (k_fwd<T>), in launch order.
template <typename T> std::vector<int> fwd_grids(const esd_matrix* P);

// Solve pieces, each a short sequence of kernel launches on stream s.
template <typename T> void launch_init(const IterCtx<T>& c, cudaStream_t s);       // r0, z0, p0
template <typename T>
void launch_iteration(const IterCtx<T>& c, cudaStream_t s, KernelMarks* marks = nullptr);  // one PCG step
template <typename T> void launch_finish(const IterCtx<T>& c, cudaStream_t s);     // flush, correction
// ||b - A x||^2 into st->true_rr
void launch_true_residual(const IterCtx<double>& c, cudaStream_t s);
// Power vector: ww = ||w||^2 and wAw = (w, A w) of the stored w (in pw[steps & 1]); with
// set_scale also scale = 1/||w|| and steps = 0 (w is a new start vector).
void launch_power_rq(const esd_matrix* A, double* const pw[2], PowerState* pws, double* partials, int set_scale,
                     cudaStream_t s);
// X (n x m, column-major, AW or W) as double-float pairs, nslices x 32 x M float2 in
// slice-major order with column k scaled by 2^-e_k, and scale[k] = 2^e_k; cexp: kMaxM ints
void launch_df_pairs(const esd_matrix* A, const double* X, size_t ld, int m, int M, float2* out, double* scale,
                     int* cexp, cudaStream_t s);
// unit = w / ||w||, with ||w||^2 from the last launch_power_rq
void launch_power_unit(const esd_matrix* A, const double* w, const PowerState* pws, double* unit, cudaStream_t s);
// y = A X for an n x m block (column-major, stride ld), m columns
void launch_spmm(const esd_matrix* A, const double* X, double* Y, size_t ld, int m, cudaStream_t s);
// b = x * a + s_vec
void launch_axpby(int n, const double* x, double a, const double* sv, double* b, cudaStream_t s);
int pad_m(int m);  // the compiled column count >= m

// Two FP32 refinement-form systems with the same matrix, one PCG iteration of both per pass
// over the matrix (plain mode, IC(0)); cond ends the paired loop once either has stopped.
std::string pair_unsupported(const IterCtx<float>& c1, const IterCtx<float>& c2);  // "" when supported
void launch_iteration_pair(const IterCtx<float>& c1, const IterCtx<float>& c2, unsigned long long cond,
                           cudaStream_t s, KernelMarks* marks = nullptr);
// c1.p12 = (c1.p, c2.p) before the paired loop (pack = true), and back after it
void launch_pair_pack(const IterCtx<float>& c1, const IterCtx<float>& c2, bool pack, cudaStream_t s);

}  // namespace esd
