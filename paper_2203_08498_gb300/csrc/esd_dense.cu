// Auxiliary-matrix construction on the device (Section 4.2): error vectors, tall-skinny
// Gram products, the small dense factorisations (Cholesky, triangular inverse, cyclic
// Jacobi eigensolver) run by one warp, and the tall x small products that apply them.
#include <algorithm>
#include <cmath>

#include "esd_dense.h"

namespace esd {

constexpr int kTile = 32;  // rows per shared-memory tile of the Gram kernel

// Offsets (in doubles) of the small dense workspace: square kMaxM x kMaxM matrices.
constexpr int kSq = kMaxM * kMaxM;
enum WsSlot { kWsG = 0, kWsWork = 1, kWsV = 2, kWsVs = 3, kWsL = 4, kWsLi = 5, kWsG0 = 6, kWsS = 7,
              kWsT = 8, kWsVec = 9 };  // kWsVec: eigenvalues, then the column scaling
constexpr size_t kWsDoubles = (size_t)kWsVec * kSq + 4 * kMaxM;

// ------------------------------------------------------------------ tall-skinny kernels

// E_hat[:, j] = x - samples[:, slot_j]
__global__ void k_errors(int n, const double* x, const double* samples, size_t ld,
                         const int* slots, int m, double* E) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double xi = x[i];
    for (int j = 0; j < m; ++j) E[(size_t)j * ld + i] = xi - samples[(size_t)slots[j] * ld + i];
  }
}

// out = X^T Y (mx x my, row-major); with sym only the pairs j <= k are summed and mirrored.
template <int PT>
__global__ void __launch_bounds__(kBlock) k_gram(int n, const double* X, int mx, const double* Y, int my,
                                                 size_t ld, int sym, double* partials, double* out,
                                                 unsigned int* ticket) {
  extern __shared__ double tile[];  // kTile x (mx + my), column-major
  __shared__ bool s_last;
  const int npairs = sym ? mx * (mx + 1) / 2 : mx * my;
  const int cols = mx + my;
  int pj[PT], pk[PT];
  double acc[PT];
#pragma unroll
  for (int t = 0; t < PT; ++t) {
    acc[t] = 0.0;
    int p = threadIdx.x + t * blockDim.x;
    pj[t] = -1;
    pk[t] = -1;
    if (p < npairs) {
      if (sym) {
        int j = 0;
        while (p >= mx - j) { p -= mx - j; ++j; }
        pj[t] = j;
        pk[t] = j + p;
      } else {
        pj[t] = p / my;
        pk[t] = p % my;
      }
    }
  }
  for (long long row0 = (long long)blockIdx.x * kTile; row0 < n; row0 += (long long)gridDim.x * kTile) {
    for (int idx = threadIdx.x; idx < kTile * cols; idx += blockDim.x) {
      const int r = idx % kTile, c = idx / kTile;
      const long long row = row0 + r;
      double v = 0.0;
      if (row < n) v = c < mx ? X[(size_t)c * ld + row] : Y[(size_t)(c - mx) * ld + row];
      tile[c * kTile + r] = v;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < PT; ++t) {
      if (pj[t] >= 0) {
        const double* a = tile + pj[t] * kTile;
        const double* b = tile + (mx + pk[t]) * kTile;
        double s = acc[t];
#pragma unroll 8
        for (int r = 0; r < kTile; ++r) s = fma(a[r], b[r], s);
        acc[t] = s;
      }
    }
    __syncthreads();
  }
  const int G = gridDim.x;
#pragma unroll
  for (int t = 0; t < PT; ++t) {
    const int p = threadIdx.x + t * blockDim.x;
    if (p < npairs) partials[(size_t)p * G + blockIdx.x] = acc[t];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == (unsigned)G - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int t = 0; t < PT; ++t) {
    const int p = threadIdx.x + t * blockDim.x;
    if (p < npairs) {
      double s = 0.0;
      for (int b = 0; b < G; ++b) s += __ldcg(&partials[(size_t)p * G + b]);
      const int j = pj[t], k = pk[t];
      if (sym) {
        out[j * mx + k] = s;
        out[k * mx + j] = s;
      } else {
        out[j * my + k] = s;
      }
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// Y[:, 0:my] = X[:, 0:mx] S (S row-major mx x my); Y columns my..mpad-1 are zeroed.
template <int MX>
__global__ void __launch_bounds__(kBlock) k_tall_small(int n, const double* X, int mx, const double* S,
                                                       int my, int mpad, double* Y, size_t ld) {
  __shared__ double ss[kMaxM * kMaxM];
  for (int idx = threadIdx.x; idx < mx * my; idx += blockDim.x) ss[idx] = S[idx];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double xr[MX];
#pragma unroll
    for (int k = 0; k < MX; ++k) xr[k] = k < mx ? X[(size_t)k * ld + i] : 0.0;
    for (int j = 0; j < my; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < MX; ++k)
        if (k < mx) s = fma(xr[k], ss[k * my + j], s);
      Y[(size_t)j * ld + i] = s;
    }
    for (int j = my; j < mpad; ++j) Y[(size_t)j * ld + i] = 0.0;
  }
}

// ------------------------------------------------------------------ one-warp dense algebra
// Matrices live in global memory, row-major with leading dimension m; the warp keeps them
// consistent with __syncwarp between dependent steps.

__device__ double warp_sum(double v) {
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A = L L^T, L lower (written to L, upper part zeroed). false if a pivot is not positive.
__device__ bool warp_cholesky(const double* A, double* L, int m) {
  const int lane = lane_id();
  for (int idx = lane; idx < m * m; idx += 32) L[idx] = 0.0;
  __syncwarp();
  for (int j = 0; j < m; ++j) {
    double part = 0.0;
    for (int k = lane; k < j; k += 32) part += L[j * m + k] * L[j * m + k];
    const double d = A[j * m + j] - warp_sum(part);
    if (!(d > 0.0)) return false;
    const double ljj = sqrt(d);
    if (lane == 0) L[j * m + j] = ljj;
    __syncwarp();
    for (int i = j + 1 + lane; i < m; i += 32) {
      double t = A[i * m + j];
      for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = t / ljj;
    }
    __syncwarp();
  }
  return true;
}

// Li = L^{-1} for lower triangular L (column j by lane j mod 32).
__device__ void warp_tri_inv(const double* L, double* Li, int m) {
  const int lane = lane_id();
  for (int idx = lane; idx < m * m; idx += 32) Li[idx] = 0.0;
  __syncwarp();
  for (int j = lane; j < m; j += 32) {
    Li[j * m + j] = 1.0 / L[j * m + j];
    for (int i = j + 1; i < m; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += L[i * m + k] * Li[k * m + j];
      Li[i * m + j] = -s / L[i * m + i];
    }
  }
  __syncwarp();
}

// Cyclic Jacobi: A (symmetric, overwritten) -> eigenvalues on the diagonal, V = eigenvectors
// (columns). Rotation as in Golub & Van Loan, "symmetric Schur decomposition".
__device__ void warp_jacobi(double* A, double* V, int m) {
  const int lane = lane_id();
  for (int idx = lane; idx < m * m; idx += 32) V[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
  __syncwarp();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int idx = lane; idx < m * m; idx += 32) {
      const int i = idx / m, j = idx % m;
      if (i != j) off += A[idx] * A[idx]; else dia += A[idx] * A[idx];
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    // off-diagonal mass 1e-28 of the diagonal: far below what any use of the eigenvalues
    // needs, and reachable (1e-32 sat at the rounding floor and ran every sweep)
    if (off <= 1e-28 * dia || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[p * m + q];
        const double app = A[p * m + p], aqq = A[q * m + q];
        // negligible coupling: the rotation would change nothing at working precision
        if (fabs(apq) <= 1e-18 * sqrt(fabs(app * aqq)) || apq == 0.0) continue;
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = lane; k < m; k += 32) {  // A J
          const double akp = A[k * m + p], akq = A[k * m + q];
          A[k * m + p] = c * akp - s * akq;
          A[k * m + q] = s * akp + c * akq;
        }
        __syncwarp();
        for (int k = lane; k < m; k += 32) {  // J^T (A J)
          const double apk = A[p * m + k], aqk = A[q * m + k];
          A[p * m + k] = c * apk - s * aqk;
          A[q * m + k] = s * apk + c * aqk;
        }
        for (int k = lane; k < m; k += 32) {  // V J
          const double vkp = V[k * m + p], vkq = V[k * m + q];
          V[k * m + p] = c * vkp - s * vkq;
          V[k * m + q] = s * vkp + c * vkq;
        }
        __syncwarp();
      }
    }
  }
}

// Sorted eigen-decomposition: ev ascending, Vs columns in the same order.
__device__ void warp_eig_sorted(const double* G, double* work, double* V, double* ev, double* Vs, int m) {
  const int lane = lane_id();
  for (int idx = lane; idx < m * m; idx += 32) work[idx] = G[idx];
  __syncwarp();
  warp_jacobi(work, V, m);
  __shared__ int order[kMaxM];
  if (lane == 0) {
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 0; i < m; ++i)  // selection sort, m <= 64
      for (int j = i + 1; j < m; ++j)
        if (work[order[j] * m + order[j]] < work[order[i] * m + order[i]]) {
          int t = order[i];
          order[i] = order[j];
          order[j] = t;
        }
  }
  __syncwarp();
  for (int i = lane; i < m; i += 32) ev[i] = work[order[i] * m + order[i]];
  for (int idx = lane; idx < m * m; idx += 32) {
    const int k = idx / m, j = idx % m;
    Vs[k * m + j] = V[k * m + order[j]];
  }
  __syncwarp();
}

// Phase 1 of W: from G0 = Ehat^T Ehat decide the rank and the transform S with
// Q1 = Ehat S. Columns are scaled to unit norm (D = diag(G0)^-1/2) first.
//   rank mbar = #{eig(D G0 D) > tol max eig}
//   mbar = m: S = D R^-1, R^T R = D G0 D        (first CholeskyQR pass)
//   mbar < m: S = D V_k Lambda_k^-1/2            (SVQB on the kept directions)
__global__ void k_w_phase1(const double* G0, int m, double rank_tol, double* ws, double* S,
                           int* out_mbar) {
  extern __shared__ double eig_smem[];  // the Jacobi iterate and its rotations (2 m^2)
  double* G = ws + kWsG * kSq;
  double* work = eig_smem;
  double* V = eig_smem + m * m;
  double* Vs = ws + kWsVs * kSq;
  double* L = ws + kWsL * kSq;
  double* Li = ws + kWsLi * kSq;
  double* ev = ws + kWsVec * kSq;
  double* dsc = ev + kMaxM;
  const int lane = lane_id();
  for (int i = lane; i < m; i += 32) {
    const double g = G0[i * m + i];
    dsc[i] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
  }
  __syncwarp();
  for (int idx = lane; idx < m * m; idx += 32) G[idx] = G0[idx] * dsc[idx / m] * dsc[idx % m];
  __syncwarp();
  warp_eig_sorted(G, work, V, ev, Vs, m);
  const double emax = ev[m - 1];
  int mbar = 0;
  for (int i = 0; i < m; ++i) mbar += (emax > 0.0 && ev[i] > rank_tol * emax) ? 1 : 0;
  bool chol_ok = false;
  if (mbar == m) chol_ok = warp_cholesky(G, L, m);
  if (chol_ok) {
    warp_tri_inv(L, Li, m);
    // S = D L^-T :  S[k][j] = d_k Li[j][k]
    for (int idx = lane; idx < m * m; idx += 32) {
      const int k = idx / m, j = idx % m;
      S[k * m + j] = dsc[k] * Li[j * m + k];
    }
  } else {
    // kept directions are the last mbar eigenvectors (ascending order)
    const int first = m - mbar;
    for (int idx = lane; idx < m * mbar; idx += 32) {
      const int k = idx / mbar, j = idx % mbar;
      S[k * mbar + j] = dsc[k] * Vs[k * m + first + j] / sqrt(ev[first + j]);
    }
  }
  __syncwarp();
  if (lane == 0) *out_mbar = chol_ok ? m : mbar;
}

// S = R^-1 with R^T R = G (second CholeskyQR pass); status 0 ok, 1 failure.
__global__ void k_w_phase2(const double* G, int m, double* ws, double* S, int* status) {
  double* L = ws + kWsL * kSq;
  double* Li = ws + kWsLi * kSq;
  const int lane = lane_id();
  const bool ok = warp_cholesky(G, L, m);
  if (ok) {
    warp_tri_inv(L, Li, m);
    for (int idx = lane; idx < m * m; idx += 32) {
      const int k = idx / m, j = idx % m;
      S[k * m + j] = Li[j * m + k];
    }
  }
  __syncwarp();
  if (lane == 0) *status = ok ? 0 : 1;
}

// From E (m x m): symmetrise, Ritz values (ascending) and vectors, then either keep the
// basis (theta = inf: Einv from the Cholesky factor of E) or select the Ritz vectors with
// value < theta (T = those vectors, E = diag, Einv = diag 1/lambda). Einv is written
// zero-padded to pad_cols(mkeep) squared. status: 0 ok, 1 E not positive definite.
__global__ void k_w_phase3(double* E, int m, double theta, double* ws, double* ritz, double* T,
                           int* mkeep, double* Einv, int* status) {
  extern __shared__ double eig_smem[];  // the Jacobi iterate and its rotations (2 m^2)
  double* work = eig_smem;
  double* V = eig_smem + m * m;
  double* Vs = ws + kWsVs * kSq;
  double* L = ws + kWsL * kSq;
  double* Li = ws + kWsLi * kSq;
  const int lane = lane_id();
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx / m, j = idx % m;
    if (i < j) {
      const double s = 0.5 * (E[i * m + j] + E[j * m + i]);
      E[i * m + j] = s;
      E[j * m + i] = s;
    }
  }
  __syncwarp();
  warp_eig_sorted(E, work, V, ritz, Vs, m);
  for (int idx = lane; idx < kSq; idx += 32) Einv[idx] = 0.0;
  __syncwarp();
  if (isinf(theta)) {
    const bool ok = warp_cholesky(E, L, m);
    if (!ok) {
      if (lane == 0) *status = 1;
      return;
    }
    warp_tri_inv(L, Li, m);
    const int mp = pad_cols(m);
    for (int idx = lane; idx < m * m; idx += 32) {  // Einv = Li^T Li
      const int i = idx / m, j = idx % m;
      double s = 0.0;
      for (int k = (i > j ? i : j); k < m; ++k) s += Li[k * m + i] * Li[k * m + j];
      Einv[i * mp + j] = s;
    }
    if (lane == 0) { *mkeep = m; *status = 0; }
    return;
  }
  int keep = 0;
  for (int i = 0; i < m; ++i) keep += ritz[i] < theta ? 1 : 0;
  for (int idx = lane; idx < m * keep; idx += 32) {
    const int k = idx / keep, j = idx % keep;
    T[k * keep + j] = Vs[k * m + j];
  }
  bool pos = true;
  for (int j = 0; j < keep; ++j) pos = pos && ritz[j] > 0.0;
  __syncwarp();
  const int mp = pad_cols(keep);
  for (int idx = lane; idx < keep * keep; idx += 32) {
    const int i = idx / keep, j = idx % keep;
    E[idx] = (i == j) ? ritz[i] : 0.0;
    Einv[i * mp + j] = (i == j && ritz[i] > 0.0) ? 1.0 / ritz[i] : 0.0;
  }
  if (lane == 0) { *mkeep = keep; *status = pos ? 0 : 1; }
}

// ------------------------------------------------------------------ host driver

// Dynamic shared memory of the one-warp eigensolver (iterate and rotations, 2 m^2 doubles;
// 64 KB at m = 64, above the default 48 KB, so the kernels are allowed it first).
static size_t eig_smem_bytes(int m) {
  const int bytes = 2 * kMaxM * kMaxM * (int)sizeof(double);
  ESD_CUDA(cudaFuncSetAttribute(k_w_phase1, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  ESD_CUDA(cudaFuncSetAttribute(k_w_phase3, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return 2 * (size_t)m * m * sizeof(double);
}

static void gram(int n, const double* X, int mx, const double* Y, int my, size_t ld, bool sym,
                 DevBuf& partials, double* out, unsigned int* ticket, cudaStream_t s) {
  const int npairs = sym ? mx * (mx + 1) / 2 : mx * my;
  const int G = std::max(1, std::min(max_grid_blocks() / 4, (n + kTile - 1) / kTile));
  const size_t need = sizeof(double) * (size_t)npairs * G;
  if (partials.bytes() < need) partials.alloc(need);
  const size_t smem = sizeof(double) * kTile * (mx + my);
  const int pt = (npairs + kBlock - 1) / kBlock;
  if (pt <= 1)
    k_gram<1><<<G, kBlock, smem, s>>>(n, X, mx, Y, my, ld, sym, partials.as<double>(), out, ticket);
  else if (pt <= 2)
    k_gram<2><<<G, kBlock, smem, s>>>(n, X, mx, Y, my, ld, sym, partials.as<double>(), out, ticket);
  else if (pt <= 4)
    k_gram<4><<<G, kBlock, smem, s>>>(n, X, mx, Y, my, ld, sym, partials.as<double>(), out, ticket);
  else
    k_gram<8><<<G, kBlock, smem, s>>>(n, X, mx, Y, my, ld, sym, partials.as<double>(), out, ticket);
  ESD_CUDA(cudaGetLastError());
}

static void tall_small(int n, const double* X, int mx, const double* S, int my, int mpad, double* Y,
                       size_t ld, cudaStream_t s) {
  const int G = max_grid_blocks();
  const int p = pad_cols(mx);
  switch (p) {
    case 8: k_tall_small<8><<<G, kBlock, 0, s>>>(n, X, mx, S, my, mpad, Y, ld); break;
    case 16: k_tall_small<16><<<G, kBlock, 0, s>>>(n, X, mx, S, my, mpad, Y, ld); break;
    case 24: k_tall_small<24><<<G, kBlock, 0, s>>>(n, X, mx, S, my, mpad, Y, ld); break;
    case 32: k_tall_small<32><<<G, kBlock, 0, s>>>(n, X, mx, S, my, mpad, Y, ld); break;
    default: k_tall_small<64><<<G, kBlock, 0, s>>>(n, X, mx, S, my, mpad, Y, ld); break;
  }
  ESD_CUDA(cudaGetLastError());
}

void AuxBuild::ensure(int n_, size_t ld_) {
  n = n_;
  ld = ld_;
  if (!small.get()) {
    small.alloc(sizeof(double) * kWsDoubles);
    ints.alloc(sizeof(int) * (kMaxM + 8));
    tick.alloc(sizeof(unsigned int) * 2);
    ESD_CUDA(cudaMemset(tick.get(), 0, tick.bytes()));
  }
  const size_t panel = sizeof(double) * ld * kMaxM;
  if (work1.bytes() < panel) {
    work1.alloc(panel);
    work2.alloc(panel);
  }
}

// Build W (n x mkeep, padded to mpad with zero columns, stride ld) from the basis X
// (n x m, stride ld): the CholeskyQR2 / SVQB orthonormalisation when orth is set,
// then AW, E, the Ritz data and Einv. Returns the number of columns kept.
int build_aux(const esd_matrix* A, AuxBuild& b, const double* X, int m, bool orth, double rank_tol,
              double theta, double* W, double* AW, double* E, double* Einv, double* ritz,
              int* mbar_out, cudaStream_t s) {
  const int n = A->n;
  const size_t ld = b.ld;
  double* ws = b.small.as<double>();
  double* G0 = ws + kWsG0 * kSq;
  double* S = ws + kWsS * kSq;
  double* dT = ws + kWsT * kSq;  // Ritz vectors
  int* dints = b.ints.as<int>();
  unsigned int* tk = b.tick.as<unsigned int>();
  int h_ints[4];
  int mcols = m;
  const double* basis = X;
  if (orth) {
    gram(n, X, m, X, m, ld, true, b.partials, G0, tk, s);
    k_w_phase1<<<1, 32, eig_smem_bytes(m), s>>>(G0, m, rank_tol, ws, S, dints);
    ESD_CUDA(cudaGetLastError());
    ESD_CUDA(cudaMemcpyAsync(h_ints, dints, sizeof(int), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaStreamSynchronize(s));
    const int mbar = h_ints[0];
    if (mbar_out) *mbar_out = mbar;
    ESD_CHECK(mbar >= 1, ESD_ERR_RANK, "the sampled error vectors have rank 0");
    // Q1 = X S  (work2), then the second pass Q = Q1 R2^-1 into work1
    tall_small(n, X, m, S, mbar, mbar, b.work2.as<double>(), ld, s);
    gram(n, b.work2.as<double>(), mbar, b.work2.as<double>(), mbar, ld, true, b.partials, G0, tk, s);
    k_w_phase2<<<1, 32, 0, s>>>(G0, mbar, ws, S, dints + 1);
    ESD_CUDA(cudaGetLastError());
    ESD_CUDA(cudaMemcpyAsync(h_ints + 1, dints + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaStreamSynchronize(s));
    ESD_CHECK(h_ints[1] == 0, ESD_ERR_RANK, "second CholeskyQR pass failed (basis numerically dependent)");
    tall_small(n, b.work2.as<double>(), mbar, S, mbar, mbar, b.work1.as<double>(), ld, s);
    basis = b.work1.as<double>();
    mcols = mbar;
  } else if (mbar_out) {
    *mbar_out = m;
  }
  // AW = A W and E = W^T (A W) for the basis
  launch_spmm(A, basis, b.work2.as<double>(), ld, mcols, s);
  gram(n, basis, mcols, b.work2.as<double>(), mcols, ld, false, b.partials, E, tk, s);
  k_w_phase3<<<1, 32, eig_smem_bytes(mcols), s>>>(E, mcols, theta, ws, ritz, dT, dints + 2, Einv, dints + 3);
  ESD_CUDA(cudaGetLastError());
  ESD_CUDA(cudaMemcpyAsync(h_ints + 2, dints + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  ESD_CUDA(cudaStreamSynchronize(s));
  ESD_CHECK(h_ints[3] == 0, ESD_ERR_CHOL_E, "E = W^T A W is not numerically positive definite");
  const int mkeep = h_ints[2];
  ESD_CHECK(mkeep >= 1, ESD_ERR_RANK, "no Ritz value below theta");
  const int mpad = pad_cols(mkeep);
  if (std::isinf(theta)) {
    ESD_CUDA(cudaMemcpyAsync(W, basis, sizeof(double) * ld * mcols, cudaMemcpyDeviceToDevice, s));
    ESD_CUDA(cudaMemcpyAsync(AW, b.work2.as<double>(), sizeof(double) * ld * mcols, cudaMemcpyDeviceToDevice, s));
    if (mpad > mcols) {
      ESD_CUDA(cudaMemsetAsync(W + ld * mcols, 0, sizeof(double) * ld * (mpad - mcols), s));
      ESD_CUDA(cudaMemsetAsync(AW + ld * mcols, 0, sizeof(double) * ld * (mpad - mcols), s));
    }
  } else {
    // Ritz vectors: W = basis T, AW = (A basis) T
    tall_small(n, basis, mcols, dT, mkeep, mpad, W, ld, s);
    tall_small(n, b.work2.as<double>(), mcols, dT, mkeep, mpad, AW, ld, s);
  }
  return mkeep;
}

}  // namespace esd
