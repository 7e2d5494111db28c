// Matrix set-up: CSR validation, colour levels, the sliced-ELL copies of A, L and U, and
// the IC(0) factorisation computed colour level by colour level on the device.
#include <algorithm>
#include <climits>
#include <cstring>
#include <numeric>

#include "esd_internal.h"
#include "esd_iter.h"

namespace esd {

// ------------------------------------------------------------------ buffers and errors

void DevBuf::alloc(size_t bytes) {
  release();
  if (bytes == 0) return;
  cudaError_t e = cudaMalloc(&p_, bytes);
  if (e != cudaSuccess) {
    p_ = nullptr;
    (void)cudaGetLastError();
    throw Error(ESD_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                   cudaGetErrorString(e));
  }
  bytes_ = bytes;
}

void DevBuf::release() {
  if (p_) cudaFree(p_);
  p_ = nullptr;
  bytes_ = 0;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void copy_in(const void* src, void* dst_dev, size_t bytes, cudaStream_t s) {
  if (bytes) ESD_CUDA(cudaMemcpyAsync(dst_dev, src, bytes, cudaMemcpyDefault, s));
}

void copy_out(const void* src_dev, void* dst, size_t bytes, cudaStream_t s) {
  if (bytes) ESD_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, s));
}

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

static int g_sms = 0;
static int sm_count() {
  if (g_sms == 0) {
    int dev = 0;
    ESD_CUDA(cudaGetDevice(&dev));
    ESD_CUDA(cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return g_sms;
}
int max_grid_blocks() { return sm_count() * 4; }
int grid_blocks(int work_slices) {
  int need = (work_slices * kSlice + kBlock - 1) / kBlock;
  return std::max(1, std::min(need, max_grid_blocks()));
}

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ int colour_of(int i, const int* cp, int ncol) {
  int lo = 0, hi = ncol;  // cp[lo] <= i < cp[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (cp[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int find_col(const int* ci, int b, int e, int key) {
  while (b < e) {
    int mid = (b + e) >> 1;
    int v = ci[mid];
    if (v == key) return mid;
    if (v < key) b = mid + 1; else e = mid;
  }
  return -1;
}

enum ValidBits { kBadRowptr = 1, kBadCol = 2, kUnsorted = 4, kNoDiag = 8, kSameColour = 16, kNotSym = 32 };

// Every index is checked before it is used, so malformed input sets error bits instead of
// reading out of bounds.
// One thread per row. The colour adjacency is collected per row, merged across the lanes of a
// warp, and written with one atomic per (warp, colour pair): one atomic per entry on a few
// words serialised the launch. Up to 64 colours a row keeps a bit mask of its neighbour
// colours; beyond, a list of its first kNbList distinct neighbour colours (further ones go
// straight to their atomic).
constexpr int kNbList = 8;
__global__ void k_validate(int n, long long nnz, const int* rp, const int* ci, const int* cp,
                           int ncol, int* diagpos, unsigned* adj, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < n;
  const bool wide = ncol > 64;
  unsigned long long mask = 0ull;  // neighbour colours (ncol <= 64)
  int nb[kNbList];                 // neighbour colours (ncol > 64)
  int nn = 0;
  int ci_row = -1;
  if (active) {
    int b = rp[i], e = rp[i + 1];
    unsigned bad = 0;
    if (b < 0 || e < b || (long long)e > nnz) { bad |= kBadRowptr; b = 0; e = 0; }
    ci_row = colour_of(i, cp, ncol);
    int dpos = -1, prev = -1;
    for (int k = b; k < e; ++k) {
      int j = ci[k];
      if (j < 0 || j >= n) { bad |= kBadCol; continue; }
      if (j <= prev) bad |= kUnsorted;
      prev = j;
      if (j == i) { dpos = k; continue; }
      int cj = colour_of(j, cp, ncol);
      if (cj == ci_row) bad |= kSameColour;
      if (!wide) {
        mask |= 1ull << cj;
      } else if (cj >= 0) {
        bool seen = false;
        for (int t = 0; t < nn; ++t) seen |= nb[t] == cj;
        if (!seen) {
          if (nn < kNbList) nb[nn++] = cj;
          else atomicOr(&adj[ci_row * ncol + cj], 1u);
        }
      }
      // structural symmetry: (j, i) must exist
      int jb = rp[j], je = rp[j + 1];
      if (jb < 0 || je < jb || (long long)je > nnz || find_col(ci, jb, je, i) < 0) bad |= kNotSym;
    }
    if (dpos < 0) bad |= kNoDiag;
    diagpos[i] = dpos < 0 ? b : dpos;
    if (bad) {
      atomicOr(&err[0], (int)bad);
      atomicMin(&err[1], i);
    }
  }
  if (wide) {  // (warp-uniform) one atomic per distinct (row colour, neighbour colour) of a list slot
#pragma unroll
    for (int t = 0; t < kNbList; ++t) {
      const int key = (ci_row >= 0 && t < nn) ? ci_row * ncol + nb[t] : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicOr(&adj[key], 1u);
    }
    return;
  }
  const unsigned peers = __match_any_sync(0xffffffffu, ci_row);
  const unsigned lo = __reduce_or_sync(peers, (unsigned)(mask & 0xffffffffull));
  const unsigned hi = __reduce_or_sync(peers, (unsigned)(mask >> 32));
  if (ci_row >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) {
    const unsigned long long all = ((unsigned long long)hi << 32) | lo;
    for (int cj = 0; cj < ncol; ++cj)
      if ((all >> cj) & 1ull) atomicOr(&adj[ci_row * ncol + cj], 1u);
  }
}

__global__ void k_rowpos(int n, const int* cp, const int* first_slice, int ncol, int* rowpos) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = colour_of(i, cp, ncol);
  int off = i - cp[c];
  rowpos[i] = (first_slice[c] + off / kSlice) * kSlice + off % kSlice;
}

__global__ void k_slice_widths(int nslices, const int2* rows, const int* rp, const int* diagpos,
                               int* wA, int* wL, int* wU) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int s = g >> 5, lane = g & 31;
  if (s >= nslices) return;
  int2 r = rows[s];
  int la = 0, ll = 0, lu = 0;
  if (lane < r.y) {
    int i = r.x + lane;
    la = rp[i + 1] - rp[i];
    ll = diagpos[i] - rp[i];
    lu = rp[i + 1] - diagpos[i] - 1;
  }
  la = __reduce_max_sync(0xffffffffu, la);
  ll = __reduce_max_sync(0xffffffffu, ll);
  lu = __reduce_max_sync(0xffffffffu, lu);
  if (lane == 0) { wA[s] = la; wL[s] = ll; wU[s] = lu; }
}

__global__ void k_fill(int nslices, int n, const int4* mA, const int4* mL, const int4* mU,
                       const int* rp, const int* ci, const double* va, const int* diagpos,
                       const int* rowpos, int* colA, double* valA, int* colL, double* valL,
                       int* colU, int* umap) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int s = g >> 5, lane = g & 31;
  if (s >= nslices) return;
  int4 a = mA[s], l = mL[s], u = mU[s];
  bool valid = lane < a.w;
  int i = a.z + lane;
  int b = valid ? rp[i] : 0, e = valid ? rp[i + 1] : 0, d = valid ? diagpos[i] : 0;
  for (int k = 0; k < a.y; ++k) {
    bool has = valid && b + k < e;
    colA[a.x + k * kSlice + lane] = has ? ci[b + k] : n;
    valA[a.x + k * kSlice + lane] = has ? va[b + k] : 0.0;
  }
  for (int k = 0; k < l.y; ++k) {
    bool has = valid && b + k < d;
    colL[l.x + k * kSlice + lane] = has ? ci[b + k] : n;
    valL[l.x + k * kSlice + lane] = has ? va[b + k] : 0.0;
  }
  for (int k = 0; k < u.y; ++k) {
    bool has = valid && d + 1 + k < e;
    int j = has ? ci[d + 1 + k] : n;
    int m = -1;
    if (has) {
      int q = find_col(ci, rp[j], rp[j + 1], i);  // (j, i) exists: checked in validation
      int apos = q - rp[j];                       // position among row j's lower entries
      int pj = rowpos[j];
      m = mL[pj >> 5].x + apos * kSlice + (pj & 31);
    }
    colU[u.x + k * kSlice + lane] = j;
    umap[u.x + k * kSlice + lane] = m;
  }
}

// Column-free copy, pattern: one warp per slice. The slot bases of a slice are the distinct
// values of (column - lane) over its present entries (column < n; without the diagonal when
// skip_diag), in increasing order; every lane's columns increase, so its entries fall into
// increasing slots. slots[s] = their number, or -1 when a slice needs more than kAffineSlots.
__global__ void k_affine_slots(int nslices, int n, const int4* meta, const int* col, int skip_diag, int* slots,
                               int* abase) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int4 md = meta[s];
  const int row = md.z + lane;
  int e = 0, cnt = 0;
  auto base_at = [&](int k) {
    while (true) {
      const int c = k < md.y ? col[md.x + k * kSlice + lane] : n;
      if (c >= n) return INT_MAX;
      if (!(skip_diag && c == row)) return c - lane;
      e = ++k;  // the diagonal has no slot: move past it
    }
  };
  int cand = base_at(0);
  while (true) {
    const int m = __reduce_min_sync(0xffffffffu, cand);
    if (m == INT_MAX) break;
    if (cnt == kAffineSlots) {
      cnt = -1;
      break;
    }
    if (lane == 0) abase[(size_t)s * kAffineSlots + cnt] = m;
    if (cand == m) cand = base_at(++e);
    ++cnt;
  }
  if (lane == 0) {
    slots[s] = cnt;
    for (int k = cnt < 0 ? 0 : cnt; k < kAffineSlots; ++k) abase[(size_t)s * kAffineSlots + k] = 0;
  }
}

// Column-free copy, values: every present entry to its slot (the slots of absent entries keep
// the zero they were allocated with).
__global__ void k_affine_values(int nslices, int n, const int4* meta, const int* col, const double* val,
                                int skip_diag, const int4* ameta, const int* abase, float* aval) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= nslices) return;
  const int4 md = meta[s], am = ameta[s];
  const int* b = abase + (size_t)s * kAffineSlots;
  const int row = md.z + lane;
  int k = 0;
  for (int e = 0; e < md.y; ++e) {
    const int c = col[md.x + e * kSlice + lane];
    if (c >= n || (skip_diag && c == row)) continue;
    while (k < am.y && b[k] + lane != c) ++k;
    if (k < am.y) aval[am.x + k * kSlice + lane] = (float)val[md.x + e * kSlice + lane];
  }
}

// One colour level of IC(0): every row i of the level computes, in column order,
//   l_ik = (a_ik - sum_{j<k} l_ij l_kj) / l_kk       (sum over the common pattern)
//   l_ii = sqrt(a_ii (1 + shift) - sum_k l_ik^2),
// reading rows k of earlier levels, which are final.
__global__ void k_ic0_level(SliceSet set, int n, const int4* mL, const int* colL, double* valL,
                            const int* rowpos, const int* rp, const int* diagpos,
                            const double* csr_val, double shift, double* ldiag, int* err) {
  const int lane = lane_id();
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int g = gw; g < set.total(); g += nw) {
    int r;
    const int s = set.slice(g, &r);
    const int4 md = mL[s];
    if (lane >= md.w) continue;
    const int i = md.z + lane;
    const int off = md.x;
    double sumsq = 0.0;
    for (int a = 0; a < md.y; ++a) {
      const int k = colL[off + a * kSlice + lane];
      if (k >= n) break;
      double sacc = csr_val[rp[i] + a];
      const int pk = rowpos[k];
      const int4 mk = mL[pk >> 5];
      const int lk = pk & 31;
      int ai = 0, bk = 0;
      while (ai < a && bk < mk.y) {
        const int ji = colL[off + ai * kSlice + lane];
        const int jk = colL[mk.x + bk * kSlice + lk];
        if (jk >= n) break;
        if (ji == jk) {
          sacc -= valL[off + ai * kSlice + lane] * valL[mk.x + bk * kSlice + lk];
          ++ai;
          ++bk;
        } else if (ji < jk) {
          ++ai;
        } else {
          ++bk;
        }
      }
      const double lik = sacc / ldiag[k];
      valL[off + a * kSlice + lane] = lik;
      sumsq += lik * lik;
    }
    double dpiv = csr_val[diagpos[i]] * (1.0 + shift) - sumsq;
    if (!(dpiv > 0.0)) {
      atomicOr(&err[2], 1);
      atomicMin(&err[3], i);
      dpiv = 1.0;
    }
    ldiag[i] = sqrt(dpiv);
  }
}

// U = L^T as the negated strict factor: U[e] = -l_ji (read before L is negated).
__global__ void k_ic0_upper(int n, const double* ldiag, double* inv_d, long long nU, const int* umap,
                            const double* valL, double* valU) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = t; i < n; i += stride) inv_d[i] = 1.0 / ldiag[i];
  if (t == 0) inv_d[n] = 0.0;
  for (long long e = t; e < nU; e += stride) {
    int m = umap[e];
    valU[e] = m >= 0 ? -valL[m] : 0.0;
  }
}

// L's strict entries are stored negated, so a substitution is one FMA chain from r_i.
__global__ void k_negate(long long cnt, double* v) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = t; i < cnt; i += stride) v[i] = -v[i];
}

__global__ void k_to_float(long long cnt, const double* a, float* b) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = t; i < cnt; i += stride) b[i] = (float)a[i];
}

// values of A only (the pattern and the slice layout are those of creation)
__global__ void k_fill_values(int nslices, const int4* mA, const int* rp, const double* va, double* valA) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int s = g >> 5, lane = g & 31;
  if (s >= nslices) return;
  const int4 a = mA[s];
  const bool valid = lane < a.w;
  const int i = a.z + lane;
  const int b = valid ? rp[i] : 0, e = valid ? rp[i + 1] : 0;
  for (int k = 0; k < a.y; ++k) valA[a.x + k * kSlice + lane] = (valid && b + k < e) ? va[b + k] : 0.0;
}

// s_i = sum_j a_ij of the stored entries (padding adds zeros), by compensated (Kahan)
// summation: the row sum of a diffusion matrix is a small difference of large entries, and
// its own rounding error must stay far below it. Stored in FP64 and FP32.
__global__ void k_rowsum(SellView<double> A, int nslices, double* s64, float* s32) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int sl = gw; sl < nslices; sl += nw) {
    const int4 md = A.meta[sl];
    if (lane >= md.w) continue;
    double sum = 0.0, comp = 0.0;
    for (int k = 0; k < md.y; ++k) {
      const double y = A.val[md.x + lane + k * kSlice] - comp;
      const double t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
    s64[md.z + lane] = sum;
    s32[md.z + lane] = (float)sum;
  }
}

// FP32 entry (value, column) pairs of a sliced-ELL array
__global__ void k_interleave(long long cnt, const int* col, const double* val, uint2* ent) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
    ent[e] = make_uint2(__float_as_uint((float)val[e]), (unsigned)col[e]);
}

static void interleave(Sell& M, cudaStream_t s) {
  if (M.ent32.bytes() < (size_t)M.entries * sizeof(uint2)) M.ent32.alloc((size_t)std::max(M.entries, 1LL) * sizeof(uint2));
  if (M.entries == 0) return;
  k_interleave<<<max_grid_blocks(), kBlock, 0, s>>>(M.entries, M.col.as<int>(), M.val.as<double>(), M.ent32.as<uint2>());
  ESD_CUDA(cudaGetLastError());
}

// Column-free FP32 copy of one part (pattern only; values come with the other FP32 copies):
// built when every slice fits kAffineSlots slots.
static void build_affine(Sell& part, int NS, int n, const std::vector<int2>& rows, cudaStream_t s,
                         bool skip_diag = false) {
  part.affine = false;
  part.awmax = 0;
  part.aslots.clear();
  if (NS == 0) return;
  DevBuf dslots(sizeof(int) * NS), dbase(sizeof(int) * (size_t)NS * kAffineSlots);
  k_affine_slots<<<(NS * 32 + 255) / 256, 256, 0, s>>>(NS, n, part.meta.as<int4>(), part.col.as<int>(),
                                                      skip_diag ? 1 : 0, dslots.as<int>(), dbase.as<int>());
  ESD_CUDA(cudaGetLastError());
  std::vector<int> slots(NS);
  ESD_CUDA(cudaMemcpyAsync(slots.data(), dslots.get(), dslots.bytes(), cudaMemcpyDeviceToHost, s));
  ESD_CUDA(cudaStreamSynchronize(s));
  if (*std::min_element(slots.begin(), slots.end()) < 0) return;
  std::vector<int4> am(NS);
  long long off = 0;
  for (int i = 0; i < NS; ++i) {
    am[i] = make_int4((int)off, slots[i], rows[i].x, rows[i].y);
    off += (long long)slots[i] * kSlice;
    if (off >= (long long)INT32_MAX) return;
  }
  part.ameta.alloc(sizeof(int4) * NS);
  ESD_CUDA(cudaMemcpyAsync(part.ameta.get(), am.data(), part.ameta.bytes(), cudaMemcpyHostToDevice, s));
  part.aval.alloc(sizeof(float) * std::max(off, 1LL));
  ESD_CUDA(cudaMemsetAsync(part.aval.get(), 0, part.aval.bytes(), s));
  part.abase = std::move(dbase);
  ESD_CUDA(cudaStreamSynchronize(s));  // am is a stack vector
  part.awmax = *std::max_element(slots.begin(), slots.end());
  part.aslots = std::move(slots);
  part.affine = true;
  part.adiag = !skip_diag;
}

static void affine_values(const Sell& part, int NS, int n, cudaStream_t s) {
  if (!part.affine || NS == 0) return;
  k_affine_values<<<(NS * 32 + 255) / 256, 256, 0, s>>>(NS, n, part.meta.as<int4>(), part.col.as<int>(),
                                                       part.val.as<double>(), part.adiag ? 0 : 1,
                                                       part.ameta.as<int4>(),
                                                       part.abase.as<int>(), part.aval.as<float>());
  ESD_CUDA(cudaGetLastError());
}

static void to_float(const DevBuf& src, DevBuf& dst, long long cnt, cudaStream_t s) {
  if (dst.bytes() < (size_t)cnt * sizeof(float)) dst.alloc((size_t)cnt * sizeof(float));
  if (cnt == 0) return;
  k_to_float<<<max_grid_blocks(), kBlock, 0, s>>>(cnt, src.as<double>(), dst.as<float>());
  ESD_CUDA(cudaGetLastError());
}

}  // namespace esd

using namespace esd;

// Symmetric Jacobi scaling of the test matrices (Sections 5.1, 5.4): d_i = 1/sqrt(a_ii).
__global__ void k_scale_diag(int n, const int* diagpos, const double* val, double* d, int* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = val[diagpos[i]];
    if (a > 0.0 && isfinite(a)) {
      d[i] = 1.0 / sqrt(a);
    } else {
      d[i] = 0.0;
      atomicMin(err, i);
    }
  }
}

// a^_ij = (a_ij d_i) d_j, one thread per row
__global__ void k_scale_vals(int n, const int* rowptr, const int* colind, const double* d, const double* src,
                             double* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double di = d[i];
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) dst[k] = (src[k] * di) * d[colind[k]];
  }
}

void esd::scale_values(esd_matrix* A, const int* diagpos, const double* src, double* dst) {
  cudaStream_t s = A->stream;
  const int n = A->n;
  DevBuf d(sizeof(double) * A->vec_stride()), err(sizeof(int));
  ESD_CUDA(cudaMemsetAsync(d.get(), 0, d.bytes(), s));
  const int first_ok = INT32_MAX;
  ESD_CUDA(cudaMemcpyAsync(err.get(), &first_ok, sizeof(int), cudaMemcpyHostToDevice, s));
  const int G = std::min((n + 255) / 256, 4 * max_grid_blocks());
  k_scale_diag<<<G, 256, 0, s>>>(n, diagpos, src, d.as<double>(), err.as<int>());
  ESD_CUDA(cudaGetLastError());
  int bad = 0;
  ESD_CUDA(cudaMemcpyAsync(&bad, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  ESD_CUDA(cudaStreamSynchronize(s));
  ESD_CHECK(bad == INT32_MAX, ESD_ERR_INVALID,
            "diagonal scaling needs a positive finite diagonal (first bad row " + std::to_string(bad) + ")");
  k_scale_vals<<<G, 256, 0, s>>>(n, A->csr_rowptr.as<int>(), A->csr_colind.as<int>(), d.as<double>(), src, dst);
  ESD_CUDA(cudaGetLastError());
  A->dscale = std::move(d);
}

void esd::matrix_values_changed(esd_matrix* A) {
  const int NS = A->nslices;
  k_fill_values<<<(NS * 32 + 255) / 256, 256, 0, A->stream>>>(NS, A->A.meta.as<int4>(), A->csr_rowptr.as<int>(),
                                                              A->csr_val.as<double>(), A->A.val.as<double>());
  ESD_CUDA(cudaGetLastError());
  A->values_version++;
  A->factored = false;
  A->factor_version++;
}

void esd_matrix::ensure_fp32() {
  if (a32_version != values_version || !A.val32.get()) {
    to_float(A.val, A.val32, A.entries, stream);
    interleave(A, stream);
    affine_values(A, nslices, n, stream);
    if (!rowsum32.get()) {
      rowsum32.alloc(sizeof(float) * vec_stride());
      rowsum64.alloc(sizeof(double) * vec_stride());
      ESD_CUDA(cudaMemsetAsync(rowsum32.get(), 0, rowsum32.bytes(), stream));
      ESD_CUDA(cudaMemsetAsync(rowsum64.get(), 0, rowsum64.bytes(), stream));
    }
    k_rowsum<<<max_grid_blocks(), kBlock, 0, stream>>>(A.view<double>(), nslices, rowsum64.as<double>(),
                                                       rowsum32.as<float>());
    ESD_CUDA(cudaGetLastError());
    a32_version = values_version;
  }
  if (fp32_version == factor_version) return;
  if (factored) {
    to_float(L.val, L.val32, L.entries, stream);
    to_float(U.val, U.val32, U.entries, stream);
    interleave(L, stream);
    interleave(U, stream);
    affine_values(L, nslices, n, stream);
    affine_values(U, nslices, n, stream);
    to_float(inv_d, inv_d32, (long long)vec_stride(), stream);
  }
  fp32_version = factor_version;
}

// ------------------------------------------------------------------ creation

static void build_level_sets(esd_matrix* M, const std::vector<unsigned>& adj) {
  const int C = M->ncol;
  M->fwd_level.assign(C, 0);
  M->bwd_level.assign(C, 0);
  for (int c = 0; c < C; ++c) {
    int lv = -1;
    for (int d = 0; d < c; ++d)
      if (adj[c * C + d] || adj[d * C + c]) lv = std::max(lv, M->fwd_level[d]);
    M->fwd_level[c] = lv + 1;
  }
  for (int c = C - 1; c >= 0; --c) {
    int lv = -1;
    for (int d = c + 1; d < C; ++d)
      if (adj[c * C + d] || adj[d * C + c]) lv = std::max(lv, M->bwd_level[d]);
    M->bwd_level[c] = lv + 1;
  }
  auto nsl = [&](int c) { return M->colour_first_slice[c + 1] - M->colour_first_slice[c]; };
  // Ranges: maximal runs of consecutive colours that share the same flags; a set holds at
  // most kMaxRanges ranges (further ranges open a new launch of the same level).
  struct Range { int c0, c1; unsigned f0, b0, elem; };
  auto make_sets = [&](const std::vector<Range>& rs) {
    std::vector<SliceSet> out;
    SliceSet cur{};
    auto flush = [&]() { if (cur.nr) { out.push_back(cur); cur = SliceSet{}; } };
    for (const Range& r : rs) {
      int len = 0;
      for (int c = r.c0; c <= r.c1; ++c) len += nsl(c);
      if (len == 0) continue;
      if (cur.nr == kMaxRanges) flush();
      cur.begin[cur.nr] = M->colour_first_slice[r.c0];
      cur.cum[cur.nr + 1] = cur.cum[cur.nr] + len;
      if (r.f0) cur.fwd0 |= 1u << cur.nr;
      if (r.b0) cur.bwd0 |= 1u << cur.nr;
      (void)r.elem;
      ++cur.nr;
    }
    flush();
    return out;
  };
  auto ranges_of = [&](const std::vector<int>& cols, bool elem) {
    std::vector<Range> rs;
    for (int c : cols) {
      unsigned f0 = M->fwd_level[c] == 0, b0 = M->bwd_level[c] == 0;
      if (!rs.empty() && rs.back().c1 == c - 1 && rs.back().f0 == f0 && rs.back().b0 == b0)
        rs.back().c1 = c;
      else
        rs.push_back({c, c, f0, b0, elem ? 1u : 0u});
    }
    return rs;
  };
  int maxf = *std::max_element(M->fwd_level.begin(), M->fwd_level.end());
  int maxb = *std::max_element(M->bwd_level.begin(), M->bwd_level.end());
  M->fwd_sets.clear();
  M->bwd_sets.clear();
  M->fwd_all_sets.clear();
  for (int lv = 0; lv <= maxf; ++lv) {
    std::vector<int> cols;
    for (int c = 0; c < C; ++c)
      if (M->fwd_level[c] == lv) cols.push_back(c);
    auto sets = make_sets(ranges_of(cols, false));
    for (auto& s : sets) {
      M->fwd_all_sets.push_back(s);
      if (lv >= 1) M->fwd_sets.push_back(s);
    }
  }
  M->bwd_all_sets.clear();
  M->bwd0_sets.clear();
  for (int lv = 0; lv <= maxb; ++lv) {
    std::vector<int> cols;
    for (int c = 0; c < C; ++c)
      if (M->bwd_level[c] == lv) cols.push_back(c);
    auto sets = make_sets(ranges_of(cols, false));
    for (auto& s : sets) {
      M->bwd_all_sets.push_back(s);
      if (lv >= 1) M->bwd_sets.push_back(s); else M->bwd0_sets.push_back(s);
    }
  }
  // the update's two classes of slices: forward level 0 (ranges split by the bwd0 flag) and
  // the rest; the staged FP32 update needs each within kMaxRanges ranges
  M->upd_sets[0] = SliceSet{};
  M->upd_sets[1] = SliceSet{};
  M->upd_ok = true;
  {
    int prev_key = -1;
    for (int c = 0; c < C; ++c) {
      if (nsl(c) == 0) continue;
      const int cls = M->fwd_level[c] == 0 ? 0 : 1;
      const unsigned b0 = (cls == 0 && M->bwd_level[c] == 0) ? 1u : 0u;
      const int key = cls * 2 + (int)b0;
      SliceSet& set = M->upd_sets[cls];
      const bool extend = key == prev_key && set.nr > 0 &&
                          set.begin[set.nr - 1] + (set.cum[set.nr] - set.cum[set.nr - 1]) == M->colour_first_slice[c];
      if (extend) {
        set.cum[set.nr] += nsl(c);
      } else if (set.nr == kMaxRanges) {
        M->upd_ok = false;
      } else {
        set.begin[set.nr] = M->colour_first_slice[c];
        set.cum[set.nr + 1] = set.cum[set.nr] + nsl(c);
        if (b0) set.bwd0 |= 1u << set.nr;
        ++set.nr;
      }
      prev_key = key;
    }
  }
  // the "all slices" set
  SliceSet all{};
  all.nr = 1;
  all.begin[0] = 0;
  all.cum[1] = M->nslices;
  M->all = all;
}

extern "C" {

const char* esd_last_error(void) { return g_last_error.c_str(); }

int esd_create_matrix(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                      const double* val, const int32_t* colour_ptr, int32_t ncolours,
                      uint32_t flags, void* stream, esd_matrix** out) {
  try {
    ESD_CHECK(out != nullptr, ESD_ERR_INVALID, "out is NULL");
    *out = nullptr;
    ESD_CHECK(n >= 1 && n < INT32_MAX - 64, ESD_ERR_INVALID, "n out of range");
    ESD_CHECK(nnz >= n && nnz < (int64_t)INT32_MAX, ESD_ERR_INVALID, "nnz out of range");
    ESD_CHECK(rowptr && colind && val && colour_ptr, ESD_ERR_INVALID, "NULL array");
    ESD_CHECK(ncolours >= 1 && ncolours <= kMaxColours, ESD_ERR_INVALID, "ncolours must be 1..2048");
    ESD_CHECK((flags & ~ESD_MATRIX_DIAG_SCALE) == 0, ESD_ERR_INVALID, "unknown flag");
    std::unique_ptr<esd_matrix> M(new esd_matrix());
    M->n = n;
    M->nnz = nnz;
    M->ncol = ncolours;
    M->stream = (cudaStream_t)stream;
    cudaStream_t s = M->stream;
    M->cp.assign(colour_ptr, colour_ptr + ncolours + 1);
    ESD_CHECK(M->cp[0] == 0 && M->cp[ncolours] == n, ESD_ERR_INVALID, "colour_ptr must span 0..n");
    for (int c = 0; c < ncolours; ++c)
      ESD_CHECK(M->cp[c + 1] >= M->cp[c], ESD_ERR_INVALID, "colour_ptr must be non-decreasing");

    // the CSR as given
    M->csr_rowptr.alloc(sizeof(int) * (n + 1));
    M->csr_colind.alloc(sizeof(int) * nnz);
    M->csr_val.alloc(sizeof(double) * nnz);
    copy_in(rowptr, M->csr_rowptr.get(), sizeof(int) * (n + 1), s);
    copy_in(colind, M->csr_colind.get(), sizeof(int) * nnz, s);
    copy_in(val, M->csr_val.get(), sizeof(double) * nnz, s);
    int ends[2];
    ESD_CUDA(cudaMemcpyAsync(&ends[0], M->csr_rowptr.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaMemcpyAsync(&ends[1], M->csr_rowptr.as<int>() + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaStreamSynchronize(s));
    ESD_CHECK(ends[0] == 0 && ends[1] == nnz, ESD_ERR_INVALID, "rowptr[0] must be 0 and rowptr[n] = nnz");

    // validation + colour adjacency
    DevBuf dcp(sizeof(int) * (ncolours + 1)), adj(sizeof(unsigned) * ncolours * ncolours),
        diagpos(sizeof(int) * n);
    M->err.alloc(sizeof(int) * 4);
    int err_init[4] = {0, INT32_MAX, 0, INT32_MAX};
    ESD_CUDA(cudaMemcpyAsync(dcp.get(), M->cp.data(), sizeof(int) * (ncolours + 1), cudaMemcpyHostToDevice, s));
    ESD_CUDA(cudaMemsetAsync(adj.get(), 0, adj.bytes(), s));
    ESD_CUDA(cudaMemcpyAsync(M->err.get(), err_init, sizeof(err_init), cudaMemcpyHostToDevice, s));
    k_validate<<<(n + 255) / 256, 256, 0, s>>>(n, nnz, M->csr_rowptr.as<int>(), M->csr_colind.as<int>(),
                                               dcp.as<int>(), ncolours, diagpos.as<int>(),
                                               adj.as<unsigned>(), M->err.as<int>());
    ESD_CUDA(cudaGetLastError());
    int herr[4];
    std::vector<unsigned> hadj(ncolours * ncolours);
    ESD_CUDA(cudaMemcpyAsync(herr, M->err.get(), sizeof(herr), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaMemcpyAsync(hadj.data(), adj.get(), adj.bytes(), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaStreamSynchronize(s));
    if (herr[0]) {
      std::string why;
      if (herr[0] & kBadRowptr) why += " decreasing rowptr;";
      if (herr[0] & kBadCol) why += " column index out of range;";
      if (herr[0] & kUnsorted) why += " columns not strictly increasing;";
      if (herr[0] & kNoDiag) why += " missing diagonal entry;";
      if (herr[0] & kSameColour) why += " two rows of one colour are coupled;";
      if (herr[0] & kNotSym) why += " pattern not structurally symmetric;";
      throw Error(ESD_ERR_INVALID, "invalid matrix (first bad row " + std::to_string(herr[1]) + "):" + why);
    }
    if (flags & ESD_MATRIX_DIAG_SCALE) {
      M->scaled = true;
      scale_values(M.get(), diagpos.as<int>(), M->csr_val.as<double>(), M->csr_val.as<double>());
    }

    // slices: 32-row slices inside each colour
    M->colour_first_slice.assign(ncolours + 1, 0);
    std::vector<int2> rows;
    for (int c = 0; c < ncolours; ++c) {
      M->colour_first_slice[c] = (int)rows.size();
      for (int r0 = M->cp[c]; r0 < M->cp[c + 1]; r0 += kSlice)
        rows.push_back(make_int2(r0, std::min(kSlice, M->cp[c + 1] - r0)));
    }
    M->colour_first_slice[ncolours] = (int)rows.size();
    M->nslices = (int)rows.size();
    ESD_CHECK(M->nslices < (1 << 24), ESD_ERR_INVALID, "more than 2^24 slices (n too large)");
    const int NS = M->nslices;
    DevBuf drows(sizeof(int2) * NS), wA(sizeof(int) * NS), wL(sizeof(int) * NS), wU(sizeof(int) * NS),
        dfirst(sizeof(int) * (ncolours + 1));
    ESD_CUDA(cudaMemcpyAsync(drows.get(), rows.data(), drows.bytes(), cudaMemcpyHostToDevice, s));
    ESD_CUDA(cudaMemcpyAsync(dfirst.get(), M->colour_first_slice.data(), dfirst.bytes(), cudaMemcpyHostToDevice, s));
    M->rowpos.alloc(sizeof(int) * n);
    k_rowpos<<<(n + 255) / 256, 256, 0, s>>>(n, dcp.as<int>(), dfirst.as<int>(), ncolours, M->rowpos.as<int>());
    k_slice_widths<<<(NS * 32 + 255) / 256, 256, 0, s>>>(NS, drows.as<int2>(), M->csr_rowptr.as<int>(),
                                                         diagpos.as<int>(), wA.as<int>(), wL.as<int>(),
                                                         wU.as<int>());
    ESD_CUDA(cudaGetLastError());
    std::vector<int> hwA(NS), hwL(NS), hwU(NS);
    ESD_CUDA(cudaMemcpyAsync(hwA.data(), wA.get(), wA.bytes(), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaMemcpyAsync(hwL.data(), wL.get(), wL.bytes(), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaMemcpyAsync(hwU.data(), wU.get(), wU.bytes(), cudaMemcpyDeviceToHost, s));
    ESD_CUDA(cudaStreamSynchronize(s));

    auto build_meta = [&](const std::vector<int>& w, Sell& part) {
      std::vector<int4> meta(NS);
      long long off = 0;
      for (int i = 0; i < NS; ++i) {
        meta[i] = make_int4((int)off, w[i], rows[i].x, rows[i].y);
        off += (long long)w[i] * kSlice;
        ESD_CHECK(off < (long long)INT32_MAX, ESD_ERR_INVALID, "matrix too large for 32-bit slice offsets");
      }
      part.entries = off;
      part.wmax = NS > 0 ? *std::max_element(w.begin(), w.end()) : 0;
      part.meta.alloc(sizeof(int4) * NS);
      ESD_CUDA(cudaMemcpyAsync(part.meta.get(), meta.data(), part.meta.bytes(), cudaMemcpyHostToDevice, s));
      part.col.alloc(sizeof(int) * std::max(off, 1LL));
      part.val.alloc(sizeof(double) * std::max(off, 1LL));
      ESD_CUDA(cudaStreamSynchronize(s));  // meta is a stack vector
    };
    build_meta(hwA, M->A);
    build_meta(hwL, M->L);
    build_meta(hwU, M->U);
    M->umap.alloc(sizeof(int) * std::max(M->U.entries, 1LL));
    k_fill<<<(NS * 32 + 255) / 256, 256, 0, s>>>(
        NS, n, M->A.meta.as<int4>(), M->L.meta.as<int4>(), M->U.meta.as<int4>(), M->csr_rowptr.as<int>(),
        M->csr_colind.as<int>(), M->csr_val.as<double>(), diagpos.as<int>(), M->rowpos.as<int>(),
        M->A.col.as<int>(), M->A.val.as<double>(), M->L.col.as<int>(), M->L.val.as<double>(),
        M->U.col.as<int>(), M->umap.as<int>());
    ESD_CUDA(cudaGetLastError());
    // A's copy serves the difference-form product, s_i p_i + sum_j a_ij (p_j - p_i), in which
    // the diagonal multiplies p_i - p_i = 0: it gets no slot
    build_affine(M->A, NS, n, rows, s, true);
    build_affine(M->L, NS, n, rows, s);
    build_affine(M->U, NS, n, rows, s);

    // slice flags and launch sets
    build_level_sets(M.get(), hadj);
    // widest factor row of every sweep launch (the staged FP32 sweeps size their stages by it)
    auto set_wmax = [](const SliceSet& set, const std::vector<int>& w) {
      int m = 0;
      for (int r = 0; r < set.nr; ++r)
        for (int g = set.cum[r]; g < set.cum[r + 1]; ++g) m = std::max(m, w[set.begin[r] + (g - set.cum[r])]);
      return m;
    };
    M->fwd_wmax.clear();
    for (const SliceSet& set : M->fwd_sets) M->fwd_wmax.push_back(set_wmax(set, hwL));
    M->bwd_wmax.clear();
    for (const SliceSet& set : M->bwd_sets) M->bwd_wmax.push_back(set_wmax(set, hwU));
    M->fwd_awmax.clear();
    M->bwd_awmax.clear();
    if (M->L.affine && M->U.affine) {
      for (const SliceSet& set : M->fwd_sets) M->fwd_awmax.push_back(set_wmax(set, M->L.aslots));
      for (const SliceSet& set : M->bwd_sets) M->bwd_awmax.push_back(set_wmax(set, M->U.aslots));
    }
    // grid of every forward launch (one table per kernel precision): the last forward launch
    // of an iteration adds the block totals the earlier ones left
    for (int prec = 0; prec < 2; ++prec) {
      std::vector<int> g = prec == 0 ? fwd_grids<double>(M.get()) : fwd_grids<float>(M.get());
      if (g.empty()) g.push_back(0);
      DevBuf& dst = prec == 0 ? M->fwd_grid64 : M->fwd_grid32;
      dst.alloc(sizeof(int) * g.size());
      ESD_CUDA(cudaMemcpyAsync(dst.get(), g.data(), sizeof(int) * g.size(), cudaMemcpyHostToDevice, s));
      ESD_CUDA(cudaStreamSynchronize(s));  // g is a local vector
    }
    std::vector<unsigned char> sflags(NS, 0);
    for (int c = 0; c < ncolours; ++c)
      for (int sl = M->colour_first_slice[c]; sl < M->colour_first_slice[c + 1]; ++sl)
        sflags[sl] = (M->fwd_level[c] == 0 ? 1 : 0) | (M->bwd_level[c] == 0 ? 2 : 0);
    M->slice_flags.alloc(NS);
    ESD_CUDA(cudaMemcpyAsync(M->slice_flags.get(), sflags.data(), NS, cudaMemcpyHostToDevice, s));

    M->ldiag.alloc(sizeof(double) * M->vec_stride());
    M->inv_d.alloc(sizeof(double) * M->vec_stride());
    ESD_CUDA(cudaMemsetAsync(M->inv_d.get(), 0, M->inv_d.bytes(), s));
    M->tmp.alloc(sizeof(double) * M->vec_stride() * 3);
    ESD_CUDA(cudaMemsetAsync(M->tmp.get(), 0, M->tmp.bytes(), s));
    M->scratch.partials.alloc(sizeof(double) * (size_t)max_grid_blocks() * kMaxRed);
    M->scratch.state.alloc(sizeof(State));
    ESD_CUDA(cudaMemsetAsync(M->scratch.state.get(), 0, sizeof(State), s));
    M->diagpos = std::move(diagpos);  // kept for the factorisation
    ESD_CUDA(cudaStreamSynchronize(s));
    *out = M.release();
    return ESD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return ESD_ERR_INVALID;
  }
}

int esd_matrix_destroy(esd_matrix* A) {
  delete A;
  return ESD_OK;
}

int esd_matrix_diag_scale(const esd_matrix* A, double* d) {
  try {
    ESD_CHECK(A && d, ESD_ERR_INVALID, "NULL argument");
    ESD_CHECK(A->scaled, ESD_ERR_STATE, "the matrix was created without ESD_MATRIX_DIAG_SCALE");
    copy_out(A->dscale.get(), d, sizeof(double) * A->n, A->stream);
    ESD_CUDA(cudaStreamSynchronize(A->stream));
    return ESD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

int esd_matrix_info(const esd_matrix* A, int32_t* n, int64_t* nnz, int32_t* ncolours,
                    int32_t* fwd_levels, int32_t* bwd_levels) {
  if (!A) { set_last_error("NULL matrix"); return ESD_ERR_INVALID; }
  if (n) *n = A->n;
  if (nnz) *nnz = A->nnz;
  if (ncolours) *ncolours = A->ncol;
  if (fwd_levels) *fwd_levels = 1 + *std::max_element(A->fwd_level.begin(), A->fwd_level.end());
  if (bwd_levels) *bwd_levels = 1 + *std::max_element(A->bwd_level.begin(), A->bwd_level.end());
  return ESD_OK;
}

int esd_matrix_layout(const esd_matrix* A, int32_t* column_free, int64_t* slot_entries, int32_t* slices) {
  if (!A) { set_last_error("NULL matrix"); return ESD_ERR_INVALID; }
  const Sell* parts[3] = {&A->A, &A->L, &A->U};
  for (int k = 0; k < 3; ++k) {
    if (column_free) column_free[k] = parts[k]->affine ? 1 : 0;
    if (slot_entries) {
      long long e = 0;
      if (parts[k]->affine)
        for (int w : parts[k]->aslots) e += (long long)w * kSlice;
      slot_entries[k] = e;
    }
  }
  if (slices) *slices = A->nslices;
  return ESD_OK;
}

int esd_matrix_set_values(esd_matrix* A, const double* val) {
  try {
    ESD_CHECK(A && val, ESD_ERR_INVALID, "NULL argument");
    if (A->scaled) {
      // the new values are scaled by their own diagonal; a bad diagonal leaves A unchanged
      DevBuf raw(sizeof(double) * (size_t)A->nnz);
      copy_in(val, raw.get(), sizeof(double) * A->nnz, A->stream);
      scale_values(A, A->diagpos.as<int>(), raw.as<double>(), A->csr_val.as<double>());
      matrix_values_changed(A);
      ESD_CUDA(cudaStreamSynchronize(A->stream));
      return ESD_OK;
    }
    copy_in(val, A->csr_val.get(), sizeof(double) * A->nnz, A->stream);
    matrix_values_changed(A);
    ESD_CUDA(cudaStreamSynchronize(A->stream));
    return ESD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

int esd_factor_ic0(esd_matrix* A, int32_t max_tries, double* shift_used) {
  try {
    ESD_CHECK(A != nullptr, ESD_ERR_INVALID, "NULL matrix");
    ESD_CHECK(max_tries >= 1, ESD_ERR_INVALID, "max_tries must be >= 1");
    cudaStream_t s = A->stream;
    const int* diagpos = A->diagpos.as<int>();
    double shift = 0.0;
    for (int t = 0; t < max_tries; ++t) {
      int err_init[4] = {0, INT32_MAX, 0, INT32_MAX};
      ESD_CUDA(cudaMemcpyAsync(A->err.get(), err_init, sizeof(err_init), cudaMemcpyHostToDevice, s));
      for (const SliceSet& set : A->fwd_all_sets) {
        k_ic0_level<<<grid_blocks(set.total()), kBlock, 0, s>>>(
            set, A->n, A->L.meta.as<int4>(), A->L.col.as<int>(), A->L.val.as<double>(), A->rowpos.as<int>(),
            A->csr_rowptr.as<int>(), diagpos, A->csr_val.as<double>(), shift, A->ldiag.as<double>(),
            A->err.as<int>());
        ESD_CUDA(cudaGetLastError());
      }
      int herr[4];
      ESD_CUDA(cudaMemcpyAsync(herr, A->err.get(), sizeof(herr), cudaMemcpyDeviceToHost, s));
      ESD_CUDA(cudaStreamSynchronize(s));
      if (herr[2] == 0) {
        k_ic0_upper<<<max_grid_blocks(), kBlock, 0, s>>>(A->n, A->ldiag.as<double>(), A->inv_d.as<double>(),
                                                         A->U.entries, A->umap.as<int>(),
                                                         A->L.val.as<double>(), A->U.val.as<double>());
        ESD_CUDA(cudaGetLastError());
        k_negate<<<max_grid_blocks(), kBlock, 0, s>>>(A->L.entries, A->L.val.as<double>());
        ESD_CUDA(cudaGetLastError());
        ESD_CUDA(cudaStreamSynchronize(s));
        A->factored = true;
        A->shift = shift;
        A->factor_version++;
        if (shift_used) *shift_used = shift;
        return ESD_OK;
      }
      shift = (shift == 0.0) ? 1e-3 : 2.0 * shift;
    }
    A->factored = false;
    throw Error(ESD_ERR_NOT_SPD, "IC(0) pivot not positive after " + std::to_string(max_tries) + " attempts");
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

int esd_matrix_spmv(esd_matrix* A, const double* x, double* y) {
  try {
    ESD_CHECK(A && x && y, ESD_ERR_INVALID, "NULL argument");
    cudaStream_t s = A->stream;
    double* tx = A->tmp.as<double>();
    double* ty = tx + A->vec_stride();
    copy_in(x, tx, sizeof(double) * A->n, s);
    launch_spmv(A, tx, ty, s);
    copy_out(ty, y, sizeof(double) * A->n, s);
    ESD_CUDA(cudaStreamSynchronize(s));
    return ESD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

int esd_matrix_apply_ic(esd_matrix* A, const double* r, double* z) {
  try {
    ESD_CHECK(A && r && z, ESD_ERR_INVALID, "NULL argument");
    ESD_CHECK(A->factored, ESD_ERR_STATE, "esd_factor_ic0 has not succeeded on this matrix");
    cudaStream_t s = A->stream;
    double* tr = A->tmp.as<double>();
    double* tz = tr + A->vec_stride();
    double* ty = tz + A->vec_stride();
    copy_in(r, tr, sizeof(double) * A->n, s);
    launch_apply_ic(A, tr, tz, ty, s);
    copy_out(tz, z, sizeof(double) * A->n, s);
    ESD_CUDA(cudaStreamSynchronize(s));
    return ESD_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

}  // extern "C"
