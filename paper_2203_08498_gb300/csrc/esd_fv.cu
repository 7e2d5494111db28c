// Cell-centred finite-volume diffusion on a structured grid, assembled on the device, and
// the chain rule of the adjoint gradient back to the per-cell log-coefficient theta.
//
// Operator (the workloads' discretisation): A = inv_dt I + K(theta) with k_c = exp(theta_c),
// an interior face between cells a < b (natural order) has the transmissibility
// T = 2 k_a k_b / (k_a + k_b) / h^2 (harmonic mean), K gets T on both diagonals and -T off
// the diagonal, and a Dirichlet face of cell c adds 2 k_c / h^2 to its diagonal.
//
// Gradient: with A x = b and A lambda = dL/dx, dL/da_ij = -lambda_i x_j. Summed over the
// four entries a face touches, dL/dT = -(lambda_a - lambda_b)(x_a - x_b); a Dirichlet face
// gives dL/dk_c += -lambda_c x_c 2/h^2; dT/dk_a = 2 k_b^2 / (k_a + k_b)^2 / h^2 and
// dk/dtheta = k. Each thread owns one cell and gathers its own faces: no atomics.
#include <cmath>

#include "esd_internal.h"

namespace esd {

struct FvDev {
  int dims, nx, ny, nz;
  double h2inv, inv_dt;
  int n;
};

// neighbour of cell c along axis a in direction dir (+1 / -1), or -1 outside the grid
__device__ __forceinline__ int fv_neighbour(const FvDev& g, int c, int a, int dir) {
  const int ix = c % g.nx;
  const int iy = (c / g.nx) % g.ny;
  const int iz = c / (g.nx * g.ny);
  if (a == 0) {
    const int t = ix + dir;
    return (t < 0 || t >= g.nx) ? -1 : c + dir;
  }
  if (a == 1) {
    const int t = iy + dir;
    return (t < 0 || t >= g.ny) ? -1 : c + dir * g.nx;
  }
  const int t = iz + dir;
  return (t < 0 || t >= g.nz) ? -1 : c + dir * g.nx * g.ny;
}

// T of the face between the lower cell (ka) and the upper cell (kb), in the operation order
// of the host assembly and without contraction, so both round alike
__device__ __forceinline__ double fv_face(double ka, double kb, double h2inv) {
  return __dmul_rn(__ddiv_rn(__dmul_rn(__dmul_rn(2.0, ka), kb), __dadd_rn(ka, kb)), h2inv);
}

__device__ __forceinline__ int fv_row(const int* cell_row, int c, int n, int* err) {
  const int i = cell_row[c];
  if (i < 0 || i >= n) {
    atomicOr(err, 1);
    return -1;
  }
  return i;
}

__device__ __forceinline__ void fv_put(const int* rp, const int* ci, double* val, int i, int j, double v, int* err) {
  int b = rp[i], e = rp[i + 1];
  while (b < e) {
    const int mid = (b + e) >> 1;
    const int cm = ci[mid];
    if (cm == j) {
      val[mid] = v;
      return;
    }
    if (cm < j) b = mid + 1; else e = mid;
  }
  atomicOr(err, 2);  // the pattern has no (i, j) entry
}

__global__ void k_fv_assemble(FvDev g, const double* theta, const int* cell_row, const int* rp, const int* ci,
                              double* val, int* err) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += gridDim.x * blockDim.x) {
    const int i = fv_row(cell_row, c, g.n, err);
    if (i < 0) continue;
    const double kc = exp(theta[c]);
    double diag = g.inv_dt;
    for (int a = 0; a < g.dims; ++a) {
      const int up = fv_neighbour(g, c, a, +1);
      const int dn = fv_neighbour(g, c, a, -1);
      double tp = 0.0, tm = 0.0;
      if (up >= 0) {
        const int j = fv_row(cell_row, up, g.n, err);
        tp = fv_face(kc, exp(theta[up]), g.h2inv);
        if (j >= 0) fv_put(rp, ci, val, i, j, -tp, err);
      }
      if (dn >= 0) {
        const int j = fv_row(cell_row, dn, g.n, err);
        tm = fv_face(exp(theta[dn]), kc, g.h2inv);
        if (j >= 0) fv_put(rp, ci, val, i, j, -tm, err);
      }
      diag = __dadd_rn(diag, __dadd_rn(tp, tm));
      const double tb = __dmul_rn(__dmul_rn(2.0, kc), g.h2inv);
      if (dn < 0) diag = __dadd_rn(diag, tb);
      if (up < 0) diag = __dadd_rn(diag, tb);
    }
    fv_put(rp, ci, val, i, i, diag, err);
  }
}

__global__ void k_fv_grad_theta(FvDev g, const double* theta, const int* cell_row, const double* lam,
                                const double* x, double* grad, int* err) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += gridDim.x * blockDim.x) {
    const int i = fv_row(cell_row, c, g.n, err);
    if (i < 0) continue;
    const double kc = exp(theta[c]);
    const double li = lam[i], xi = x[i];
    double gk = 0.0;
    for (int a = 0; a < g.dims; ++a) {
      for (int dir = -1; dir <= 1; dir += 2) {
        const int d = fv_neighbour(g, c, a, dir);
        if (d < 0) {
          gk -= li * xi * 2.0 * g.h2inv;  // Dirichlet face
          continue;
        }
        const int j = fv_row(cell_row, d, g.n, err);
        if (j < 0) continue;
        const double kd = exp(theta[d]);
        const double s = kc + kd;
        const double dT_dk = 2.0 * kd * kd / (s * s) * g.h2inv;
        gk -= (li - lam[j]) * (xi - x[j]) * dT_dk;
      }
    }
    grad[c] = kc * gk;
  }
}

static FvDev fv_dev(const esd_fv_grid* g, int n) {
  ESD_CHECK(g, ESD_ERR_INVALID, "NULL grid");
  ESD_CHECK(g->dims == 2 || g->dims == 3, ESD_ERR_INVALID, "dims must be 2 or 3");
  ESD_CHECK(g->nx >= 1 && g->ny >= 1 && (g->dims == 2 || g->nz >= 1), ESD_ERR_INVALID, "grid sizes must be >= 1");
  const long long cells = (long long)g->nx * g->ny * (g->dims == 3 ? g->nz : 1);
  ESD_CHECK(cells == n, ESD_ERR_INVALID, "grid cells != matrix size");
  ESD_CHECK(g->h > 0.0 && std::isfinite(g->h), ESD_ERR_INVALID, "h must be positive");
  ESD_CHECK(g->inv_dt >= 0.0 && std::isfinite(g->inv_dt), ESD_ERR_INVALID, "inv_dt must be >= 0");
  FvDev d;
  d.dims = g->dims;
  d.nx = g->nx;
  d.ny = g->ny;
  d.nz = g->dims == 3 ? g->nz : 1;
  d.h2inv = 1.0 / (g->h * g->h);
  d.inv_dt = g->inv_dt;
  d.n = n;
  return d;
}

// device copy of an input that may live on the host
template <typename T>
static const T* staged(const T* p, size_t count, DevBuf& tmp, cudaStream_t s) {
  if (is_device_ptr(p)) return p;
  tmp.alloc(sizeof(T) * count);
  copy_in(p, tmp.get(), sizeof(T) * count, s);
  return tmp.as<T>();
}

static void check_err(DevBuf& derr, cudaStream_t s) {
  int herr = 0;
  ESD_CUDA(cudaMemcpyAsync(&herr, derr.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  ESD_CUDA(cudaStreamSynchronize(s));
  ESD_CHECK(!(herr & 1), ESD_ERR_INVALID, "cell_row holds a row index outside 0..n-1");
  ESD_CHECK(!(herr & 2), ESD_ERR_INVALID, "the matrix pattern lacks an entry of the grid stencil");
}

}  // namespace esd

using namespace esd;

extern "C" int esd_fv_assemble(esd_matrix* A, const esd_fv_grid* g, const double* theta, const int32_t* cell_row) {
  try {
    ESD_CHECK(A && theta && cell_row, ESD_ERR_INVALID, "NULL argument");
    ESD_CHECK(!A->scaled, ESD_ERR_STATE, "the finite-volume assembly writes the unscaled operator");
    const FvDev d = fv_dev(g, A->n);
    cudaStream_t s = A->stream;
    DevBuf t0, t1, derr(sizeof(int)), vals(sizeof(double) * (size_t)A->nnz);
    const double* th = staged(theta, (size_t)A->n, t0, s);
    const int* cr = staged(cell_row, (size_t)A->n, t1, s);
    ESD_CUDA(cudaMemsetAsync(derr.get(), 0, sizeof(int), s));
    // assembled into a copy first: a failed check leaves A as it was
    ESD_CUDA(cudaMemcpyAsync(vals.get(), A->csr_val.get(), vals.bytes(), cudaMemcpyDeviceToDevice, s));
    k_fv_assemble<<<max_grid_blocks(), kBlock, 0, s>>>(d, th, cr, A->csr_rowptr.as<int>(), A->csr_colind.as<int>(),
                                                       vals.as<double>(), derr.as<int>());
    ESD_CUDA(cudaGetLastError());
    check_err(derr, s);
    ESD_CUDA(cudaMemcpyAsync(A->csr_val.get(), vals.get(), vals.bytes(), cudaMemcpyDeviceToDevice, s));
    matrix_values_changed(A);
    ESD_CUDA(cudaStreamSynchronize(s));
    return ESD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

extern "C" int esd_fv_grad_theta(esd_matrix* A, const esd_fv_grid* g, const double* theta, const int32_t* cell_row,
                                 const double* lambda, const double* x, double* grad_theta) {
  try {
    ESD_CHECK(A && theta && cell_row && lambda && x && grad_theta, ESD_ERR_INVALID, "NULL argument");
    ESD_CHECK(!A->scaled, ESD_ERR_STATE, "the theta gradient refers to the unscaled operator");
    const FvDev d = fv_dev(g, A->n);
    cudaStream_t s = A->stream;
    const size_t n = (size_t)A->n;
    DevBuf t0, t1, t2, t3, tg, derr(sizeof(int));
    const double* th = staged(theta, n, t0, s);
    const int* cr = staged(cell_row, n, t1, s);
    const double* lm = staged(lambda, n, t2, s);
    const double* xx = staged(x, n, t3, s);
    const bool dev_out = is_device_ptr(grad_theta);
    if (!dev_out) tg.alloc(sizeof(double) * n);
    double* gout = dev_out ? grad_theta : tg.as<double>();
    ESD_CUDA(cudaMemsetAsync(derr.get(), 0, sizeof(int), s));
    k_fv_grad_theta<<<max_grid_blocks(), kBlock, 0, s>>>(d, th, cr, lm, xx, gout, derr.as<int>());
    ESD_CUDA(cudaGetLastError());
    if (!dev_out) copy_out(gout, grad_theta, sizeof(double) * n, s);
    check_err(derr, s);
    return ESD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}
