// Device construction of the auxiliary matrix W, AW, E and E^-1 (Section 4.2).
#pragma once

#include "esd_iter.h"

namespace esd {

// Work buffers of the construction: two n x 64 panels and the small dense scratch.
struct AuxBuild {
  int n = 0;
  size_t ld = 0;
  DevBuf work1, work2;  // n x kMaxM panels
  DevBuf small;         // small dense matrices (see the offsets in esd_dense.cu)
  DevBuf ints;          // small integer results
  DevBuf tick;          // reduction ticket
  DevBuf partials;      // Gram partial sums
  void ensure(int n_, size_t ld_);
};

// Orthonormalise (orth) the n x m basis X, then W, AW = A W, E = W^T A W, Ritz values
// (ascending) and E^-1 (padded to pad_m(mkeep)); with finite theta W holds the Ritz vectors
// of value < theta. Returns mkeep; *mbar_out gets the rank found. Throws Error on failure.
int build_aux(const esd_matrix* A, AuxBuild& b, const double* X, int m, bool orth, double rank_tol,
              double theta, double* W, double* AW, double* E, double* Einv, double* ritz,
              int* mbar_out, cudaStream_t s);

// E_hat[:, j] = x - samples[:, slots[j]], j < m (stride ld).
__global__ void k_errors(int n, const double* x, const double* samples, size_t ld, const int* slots, int m,
                         double* E);

__host__ __device__ inline int pad_cols(int m) {
  return m <= 0 ? 0 : (m <= 8 ? 8 : (m <= 16 ? 16 : (m <= 24 ? 24 : (m <= 32 ? 32 : 64))));
}

}  // namespace esd
