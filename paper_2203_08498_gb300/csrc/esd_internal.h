// Host-side objects behind the C handles: device buffers, the sliced matrix with its IC(0)
// factor, and the solver with its captured CUDA graphs.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "esd_common.cuh"

namespace esd {

// Owning device allocation.
class DevBuf {
 public:
  DevBuf() = default;
  explicit DevBuf(size_t bytes) { alloc(bytes); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p_(o.p_), bytes_(o.bytes_) { o.p_ = nullptr; o.bytes_ = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p_ = o.p_; bytes_ = o.bytes_; o.p_ = nullptr; o.bytes_ = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t bytes);
  void release();
  template <typename T> T* as() const { return static_cast<T*>(p_); }
  void* get() const { return p_; }
  size_t bytes() const { return bytes_; }

 private:
  void* p_ = nullptr;
  size_t bytes_ = 0;
};

// Sliced-ELL storage of one matrix part (A, strict L or strict U), double and optional float.
struct Sell {
  DevBuf meta;   // int4 per slice
  DevBuf col;    // int per entry (padded)
  DevBuf val;    // double per entry
  DevBuf val32;  // float per entry (FP32 inner solves)
  DevBuf ent32;  // uint2 per entry: (float bits, column), so an FP32 entry is one 8-byte load
  long long entries = 0;
  int wmax = 0;  // widest slice (entries per row)
  // Column-free FP32 copy for the staged kernels, built when every slice fits: slot k of
  // slice s holds, in lane l, the entry of column abase[8 s + k] + l of row (first row + l),
  // value 0 where that row has no such entry. The slot bases of a slice increase, so a row's
  // entries keep their order. Pattern at creation, values with the other FP32 copies.
  DevBuf ameta;  // int4 per slice: {value offset, slots, first row, rows}
  DevBuf abase;  // int[kAffineSlots] per slice: the slot bases
  DevBuf aval;   // float per slot entry (slots x 32 per slice)
  bool affine = false;
  bool adiag = true;          // the diagonal has its slot (A's copy omits it: see its creation)
  int awmax = 0;              // most slots of a slice
  std::vector<int> aslots;    // slots per slice (host)
  template <typename T> SellView<T> view() const;
};

template <> inline SellView<double> Sell::view<double>() const {
  return {meta.as<int4>(), col.as<int>(), val.as<double>()};
}
template <> inline SellView<float> Sell::view<float>() const {
  SellView<float> v{meta.as<int4>(), col.as<int>(), val32.as<float>(), ent32.as<uint2>()};
  if (affine) {
    v.ameta = ameta.as<int4>();
    v.abase = abase.as<int>();
    v.aval = aval.as<float>();
  }
  return v;
}

// Scratch for the grid-wide reductions of one stream of launches.
struct Scratch {
  DevBuf partials;  // double, kMaxGridBlocks * kMaxRed
  DevBuf state;     // State
};

constexpr int kMaxRed = 2 * kMaxM + 8;
constexpr int kAffineSlots = 8;  // slots of a slice in the column-free copy, at most
// zero elements before and after the FP32 vectors the column-free products gather: a slot's
// column base + lane lies in [-31, n + 30] for every lane, also where the row has no entry
constexpr int kGuard = 32;

int grid_blocks(int work_slices);  // blocks for a launch over this many slices
int max_grid_blocks();

}  // namespace esd

struct esd_matrix {
  int n = 0;
  long long nnz = 0;
  int ncol = 0;
  std::vector<int> cp;             // colour pointer (host)
  cudaStream_t stream = nullptr;
  int nslices = 0;
  std::vector<int> colour_first_slice;
  std::vector<int> fwd_level, bwd_level;
  // launch groups
  esd::SliceSet all;                       // every slice
  std::vector<esd::SliceSet> fwd_sets;     // forward levels >= 1 (level 0 is fused in the update)
  std::vector<esd::SliceSet> bwd_sets;     // backward levels >= 1 (+ elementwise ranges)
  std::vector<esd::SliceSet> fwd_all_sets; // all forward levels incl. level 0 (factor, apply)
  std::vector<esd::SliceSet> bwd_all_sets; // all backward levels incl. level 0 (apply)
  std::vector<esd::SliceSet> bwd0_sets;    // colours without later neighbours
  std::vector<int> fwd_wmax, bwd_wmax;     // widest L (U) row of each fwd_sets (bwd_sets) launch
  std::vector<int> fwd_awmax, bwd_awmax;   // most slots of a slice of the column-free L (U) copy, per launch
  esd::SliceSet upd_sets[2];               // forward level-0 slices, the other slices
  bool upd_ok = false;                     // both fit kMaxRanges ranges
  esd::DevBuf fwd_grid64, fwd_grid32;      // int per forward launch: its grid (FP64 / FP32 kernel)
  esd::Sell A, L, U;  // L and U hold the strict factor entries negated (-l_ij)
  esd::DevBuf slice_flags;   // uint8 per slice: bit0 fwd level 0, bit1 bwd level 0
  esd::DevBuf rowpos;        // int per row: slice*32 + lane
  esd::DevBuf diagpos;       // int per row: CSR index of the diagonal entry
  esd::DevBuf umap;          // int per U entry: index of the L entry holding l_ji (-1 = pad)
  esd::DevBuf csr_rowptr, csr_colind, csr_val;  // the CSR as given (int, int, double)
  esd::DevBuf ldiag;         // double: l_ii
  esd::DevBuf inv_d;         // double: 1/l_ii (n+1, sentinel 0)
  esd::DevBuf inv_d32;       // float copy
  esd::DevBuf rowsum32;      // s = A 1 (compensated FP64 sum), stored in FP32 (difference-form SpMV)
  esd::DevBuf rowsum64;      // the same row sums in FP64 (difference-form refinement residual)
  esd::DevBuf err;           // int[4] validation / factor error words
  esd::DevBuf tmp;           // 3 x (n+1) doubles for host-pointer staging
  esd::Scratch scratch;
  bool factored = false;
  int factor_version = 0;
  int values_version = 0;  // bumped whenever the values of A change (same pattern)
  int a32_version = -1;    // values_version of val32 / rowsum32
  int fp32_version = -1;
  double shift = 0.0;
  bool scaled = false;       // ESD_MATRIX_DIAG_SCALE: the values held are D^-1/2 A D^-1/2
  esd::DevBuf dscale;        // double: d_i = 1/sqrt(a_ii) of the last values given (scaled only)
  size_t vec_stride() const { return ((size_t)n + 1 + 31) / 32 * 32; }  // doubles per vector
  void ensure_fp32();
};

namespace esd {
// Helpers shared by the translation units.
void copy_in(const void* src, void* dst_dev, size_t bytes, cudaStream_t s);   // device or host src
void copy_out(const void* src_dev, void* dst, size_t bytes, cudaStream_t s);  // device or host dst
bool is_device_ptr(const void* p);
// Extremes of the CG Lanczos matrix from a[k], b[k-1] (out: lmin, lmax, lmax/lmin); scratch
// holds 2 tables of stride >= k doubles (esd_noalloc.cu).
void launch_lanczos_extremes(const double* a, const double* b, int k, double* scratch, size_t stride, double* out,
                             cudaStream_t s);
// After csr_val changed on the device: refill the sliced-ELL values of A, drop the factor.
void matrix_values_changed(esd_matrix* A);
// Scaled matrices: dst = D^-1/2 src D^-1/2 for D = diag(src), and A->dscale = d. Checks the
// diagonal (positive, finite) before it writes anything; src may equal dst.
void scale_values(esd_matrix* A, const int* diagpos, const double* src, double* dst);
void set_last_error(const std::string& msg);

// Kernel launchers used across files (defined in esd_iter.cu).
void launch_spmv(const esd_matrix* A, const double* x, double* y, cudaStream_t s);
void launch_apply_ic(const esd_matrix* A, const double* r, double* z, double* work, cudaStream_t s);
}  // namespace esd
