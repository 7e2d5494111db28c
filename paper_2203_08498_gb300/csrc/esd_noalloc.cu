// Condition estimate that allocates nothing: the Lanczos tridiagonal matrix of a CG run is
// written into a file-scope device array instead of library-allocated scratch, so callers
// that must not allocate device memory can still use it.
#include <cmath>
#include <mutex>

#include "esd_internal.h"

namespace esd {

constexpr int kNoAllocMaxK = ESD_NOALLOC_MAX_K;

// d[0..k) then e2[0..k): diagonal and squared off-diagonal of T. Every GPU that loads the
// library holds this array (512 KB) until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxK];

// Device addresses of g_noalloc_scratch, one per device, looked up on the first call.
constexpr int kMaxDevices = 64;
static double* g_scratch_ptr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

__device__ static int sturm_count_tab(const double* d, const double* e2, int k, double x) {
  int cnt = 0;
  double q = 1.0;
  const double pivmin = 1e-300;
  for (int j = 0; j < k; ++j) {
    q = (j == 0) ? d[j] - x : d[j] - x - e2[j] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Extreme eigenvalues of the CG Lanczos matrix T (diag 1/a_j + b_{j-1}/a_{j-1}, off-diagonal
// sqrt(b_j)/a_j) by multisection on Sturm counts: T's diagonal and squared off-diagonal are
// tabulated first (d = scratch[0..k), e2 = scratch[stride..stride+k)), then every round the
// 256 threads count the eigenvalues below 256 points of the current bracket.
__global__ void k_lanczos_extremes_tab(const double* a, const double* b, int k, double* scratch, size_t stride,
                                       double* out) {
  __shared__ double lo_s, hi_s;
  __shared__ int cnt_s[256];
  double* d = scratch;
  double* e2 = scratch + stride;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double dj = 1.0 / a[j];
    double ej2 = 0.0;
    if (j > 0) {
      dj += b[j - 1] / a[j - 1];
      const double e = sqrt(b[j - 1]) / a[j - 1];
      ej2 = e * e;
    }
    d[j] = dj;
    e2[j] = ej2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double lo = 1e300, hi = -1e300;
    for (int j = 0; j < k; ++j) {
      double r = 0.0;
      if (j > 0) r += sqrt(e2[j]);
      if (j + 1 < k) r += sqrt(e2[j + 1]);
      lo = fmin(lo, d[j] - r);
      hi = fmax(hi, d[j] + r);
    }
    const double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
    lo_s = lo - pad;
    hi_s = hi + pad;
  }
  __syncthreads();
  const double glo = lo_s, ghi = hi_s;
  double res[2];
  for (int which = 0; which < 2; ++which) {
    double lo = glo, hi = ghi;
    const int target = which == 0 ? 1 : k;
    for (int round = 0; round < 12; ++round) {
      const double x = lo + (hi - lo) * (threadIdx.x + 1) / 257.0;
      cnt_s[threadIdx.x] = sturm_count_tab(d, e2, k, x);
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 256;
        for (int i = 0; i < 256; ++i)
          if (cnt_s[i] >= target) { t = i; break; }
        const double w = (hi - lo) / 257.0;
        lo_s = lo + w * t;
        hi_s = (t < 256) ? lo + w * (t + 1) : hi;
      }
      __syncthreads();
      lo = lo_s;
      hi = hi_s;
      __syncthreads();
      if (hi - lo <= 1e-15 * fmax(fabs(lo), fabs(hi))) break;
    }
    res[which] = 0.5 * (lo + hi);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = res[0];
    out[1] = res[1];
    out[2] = res[1] / res[0];
  }
}

void launch_lanczos_extremes(const double* a, const double* b, int k, double* scratch, size_t stride, double* out,
                             cudaStream_t s) {
  k_lanczos_extremes_tab<<<1, 256, 0, s>>>(a, b, k, scratch, stride, out);
  ESD_CUDA(cudaGetLastError());
}

}  // namespace esd

using namespace esd;

// True when p is device (or managed) memory that the given device can address as its own.
static bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

extern "C" int esd_lanczos_extremes_noalloc(const double* alpha, const double* beta, int32_t k, double* out,
                                            void* stream) {
  try {
    ESD_CHECK(alpha && out && (k == 1 || beta), ESD_ERR_INVALID, "NULL argument");
    ESD_CHECK(k >= 1 && k <= kNoAllocMaxK, ESD_ERR_INVALID,
              "k must be 1.." + std::to_string(kNoAllocMaxK) + " (size of the static scratch array)");
    int dev = 0;
    ESD_CUDA(cudaGetDevice(&dev));
    ESD_CHECK(dev >= 0 && dev < kMaxDevices, ESD_ERR_INVALID, "device ordinal out of range");
    // The kernel reads alpha and beta and writes out directly: each must be memory of the
    // current device (a host array would be read through a host address on the GPU).
    ESD_CHECK(on_device(alpha, dev), ESD_ERR_INVALID, "alpha is not device memory of the current device");
    ESD_CHECK(k == 1 || on_device(beta, dev), ESD_ERR_INVALID, "beta is not device memory of the current device");
    ESD_CHECK(on_device(out, dev), ESD_ERR_INVALID, "out is not device memory of the current device");
    double* scratch = nullptr;
    {
      std::lock_guard<std::mutex> lock(g_scratch_mutex);
      if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        ESD_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = static_cast<double*>(p);
      }
      scratch = g_scratch_ptr[dev];
    }
    launch_lanczos_extremes(alpha, beta, k, scratch, kNoAllocMaxK, out, (cudaStream_t)stream);
    return ESD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}
