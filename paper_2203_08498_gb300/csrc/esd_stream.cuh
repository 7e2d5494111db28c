// Bulk-staged matrix streaming for the FP32 kernels of the refinement form's inner PCG: the
// sliced-ELL entries and the row vectors of a launch reach shared memory by cp.async.bulk
// (the TMA engine's 1-D copies), chunk by chunk through a ring of stages, while consumer warps
// form the row products from shared memory.
//
// Why: in the one-warp-per-slice kernels every slice waits on three dependent memory round
// trips (its meta, then its entries and vector elements, then the gathers), so the SpMV and
// the sweeps were latency-bound at 55-72 % of the copy bandwidth. Here one producer warp per
// block issues large contiguous copies (kilobytes per request) up to three chunks ahead, so
// the matrix stream never waits on the gathers, and a slice costs its consumer warp one
// round trip (the gathers of the vector, mostly L2 hits). Short rows (the first levels of a
// sweep hold 2 factor entries per row) give a warp K slices per chunk, so that enough
// gathers are in flight.
//
// Layout of one stage: the chunk's slice metas (16 bytes each), the row vectors (the chunk's
// rows, widened to 16-byte boundaries), then its entries exactly as they lie in global memory
// (slice after slice, 32 x width 8-byte entries each). The slices of a chunk are consecutive,
// and so are their rows, so every copy is one contiguous range: 16-byte aligned, a multiple of
// 16 bytes, as cp.async.bulk requires.
//
// Synchronisation: stage k has a "full" mbarrier (one producer arrival + the copies' byte
// count) and an "empty" one (one arrival per consumer warp). Use u of a stage completes phase
// u of both. Every wait is bounded (about a second of the global timer); a wait that runs out
// sets ESD_ERR_INTERNAL, stops the solve's loop, and leaves its loop; the producer then waits
// (bounded again) for the copies it issued before the block exits.
#pragma once

#include <cstdlib>

namespace esd {

constexpr int kStreamWarps = 16;                             // consumer warps per block
constexpr int kStreamThreads = (kStreamWarps + 1) * 32;      // + one producer warp
constexpr int kStreamMaxStages = 3;                          // chunks in flight per block, at most
constexpr int kStreamWmax = 8;                               // widest slice the staged kernels take
// Shapes of a staged launch: K slices per consumer warp per chunk, rows of at most W entries
// (the register arrays of a lane hold K W entries). Code 10 K + W. The column-free copy's
// 4-byte values leave registers for K = 2 with W up to 8, which the (value, column) pairs do
// not; its widths 6, 7 and 8 are exact, since a slot past a row's width still costs the
// issue slots of its predicated instructions.
constexpr int kShapes[6] = {42, 24, 26, 27, 28, 18};
constexpr int kStreamMaxK = 4;                               // slices per consumer warp per chunk, at most
constexpr int kStreamStageCap = 50 * 1024;                   // bytes of one stage, at most
constexpr int kStreamRingCap = 100 * 1024;                   // bytes of the stage ring (2 blocks per SM)
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // bound of every mbarrier wait

// Chunks of one slice set: range r of the set holds chunks [ccum[r], ccum[r+1]) of cs slices
// each (the last one of a range may be shorter); no chunk spans two ranges, so its slices,
// and their rows, are consecutive in memory.
struct ChunkMap {
  int nr;
  int ccum[kMaxRanges + 1];
  __host__ __device__ int total() const { return ccum[nr]; }
};

inline ChunkMap chunk_map(const SliceSet& set, int cs) {
  ChunkMap m{};
  m.nr = set.nr;
  m.ccum[0] = 0;
  for (int r = 0; r < set.nr; ++r) {
    const int len = set.cum[r + 1] - set.cum[r];
    m.ccum[r + 1] = m.ccum[r] + (len + cs - 1) / cs;
  }
  return m;
}

// Row-vector elements a stage holds per vector: the chunk's rows, widened at both ends to
// 16-byte boundaries.
__host__ __device__ constexpr int stream_vcap(int cs, int vec_bytes) { return cs * kSlice + 2 * (16 / vec_bytes); }

// The row vectors a staged kernel copies with every chunk, in stage order: element bytes (4
// or 8), the vectors copied with an evict-last L2 policy (other rows gather them; the rest
// evict-first), and those copied for part-1 chunks (part-0 chunks copy all).
template <int NV>
struct VecSet {
  const void* ptr[NV];
  int vb[NV];
  unsigned keep;
  unsigned part1;
};

// Matrix entries of a staged kernel: one or two arrays per entry (FP32: (value, column)
// pairs; the column-free copy: values, with kAffineSlots slot bases per slice in sbase),
// eb[a] bytes per entry; none for vector-only kernels.
struct EntSet {
  const void* ptr[2];
  int eb[2];
  int n;
  const int* sbase = nullptr;
};

// Bytes of one stage: the slice headers (hdr bytes each: the meta, and the slot bases of the
// column-free copy), row vectors (nv4 of 4-byte and nv8 of 8-byte elements), then the entries
// of cs slices of at most wmax entries per row (ebytes per entry over all arrays).
__host__ __device__ constexpr int stream_stage_bytes(int cs, int wmax, int ebytes, int nv4, int nv8, int hdr = 16) {
  return cs * hdr + nv4 * stream_vcap(cs, 4) * 4 + nv8 * stream_vcap(cs, 8) * 8 + cs * wmax * kSlice * ebytes;
}

// Slice header bytes of a stage: the meta, plus the slot bases of the column-free copy.
constexpr int kHdrPlain = 16;
constexpr int kHdrAffine = 16 + kAffineSlots * 4;

// The chunks of one staged launch: those of set 0 (matrix entries and row vectors staged),
// then those of set 1 (row vectors only). cs = slices per chunk (kStreamWarps x K), ns =
// stages in the ring, stage = bytes of one stage, ecap = entries per entry array in a stage.
struct StreamPlan {
  SliceSet set[2];
  ChunkMap cm[2];
  int cs, ns, stage, ecap, hdr;
  __host__ __device__ int total() const { return cm[0].total() + cm[1].total(); }
};

// Plan of a launch whose set-0 rows hold at most wmax entries (ebytes per entry; 0 for a
// vector-only kernel) and that stages nv4 4-byte and nv8 8-byte row vectors: its shape (the
// first of kShapes whose W holds wmax and whose stage fits kStreamStageCap bytes; K = 2, W = 8
// only for the column-free copy), and the stages that fit kStreamRingCap (3, else 2). aff: the
// entries are the column-free copy's (hdr = kHdrAffine). *shape_out = the shape's code.
inline StreamPlan stream_plan(const SliceSet& with_entries, const SliceSet& vectors_only, int wmax, int ebytes,
                              int nv4, int nv8, int* shape_out, bool aff = false, int hdr = kHdrPlain) {
  int K = 1, shape = 18;
  for (int sh : kShapes) {
    const int k = sh / 10, w = sh % 10;
    if (sh >= 26 && sh <= 28 && !aff) continue;
    if (std::max(wmax, 1) <= w && stream_stage_bytes(kStreamWarps * k, wmax, ebytes, nv4, nv8, hdr) <= kStreamStageCap) {
      K = k;
      shape = sh;
      break;
    }
  }
  StreamPlan pl{};
  pl.cs = kStreamWarps * K;
  pl.hdr = hdr;
  pl.stage = stream_stage_bytes(pl.cs, wmax, ebytes, nv4, nv8, hdr);
  pl.ns = 3 * pl.stage <= kStreamRingCap ? 3 : 2;
  pl.ecap = pl.cs * wmax * kSlice;
  pl.set[0] = with_entries;
  pl.set[1] = vectors_only;
  pl.cm[0] = chunk_map(with_entries, pl.cs);
  pl.cm[1] = chunk_map(vectors_only, pl.cs);
  *shape_out = shape;
  return pl;
}

// Part (0 or 1), range of the part's set, and slices [s0, s1) of chunk ch.
struct ChunkPos {
  int part, range, s0, s1;
};

__device__ __forceinline__ ChunkPos chunk_pos(const StreamPlan& pl, int ch) {
  ChunkPos cp;
  const int n0 = pl.cm[0].total();
  cp.part = ch < n0 ? 0 : 1;
  const SliceSet& set = pl.set[cp.part];
  const ChunkMap& cm = pl.cm[cp.part];
  const int c = ch - (cp.part ? n0 : 0);
  int r = 0;
#pragma unroll 1
  while (r + 1 < cm.nr && c >= cm.ccum[r + 1]) ++r;
  const int g0 = set.cum[r] + (c - cm.ccum[r]) * pl.cs;
  const int g1 = min(g0 + pl.cs, set.cum[r + 1]);
  cp.range = r;
  cp.s0 = set.begin[r] + (g0 - set.cum[r]);
  cp.s1 = cp.s0 + (g1 - g0);
  return cp;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the completion of the phase of parity `parity`; false after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}

// L2 policy for data read once per pass: evict first, so the gathered vectors stay in L2.
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// L2 policy for data that other rows will gather soon: keep it.
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// bytes (a multiple of 16) from global src to shared dst (both 16-byte aligned), completing
// on bar's transaction count
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                          unsigned long long pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}

// The solve's loop stops with ESD_ERR_INTERNAL (a staged wait ran out, or a slice did not fit
// the stage shape the launch was planned for).
__device__ __forceinline__ void stream_fail(State* st, unsigned long long cond) {
  st->status = ESD_ERR_INTERNAL;
  st->conv = 1;
  end_loop(cond);
}

// First element of the widened row range of a chunk whose first row is z0, for elements of
// vb bytes (16-byte aligned).
__host__ __device__ __forceinline__ int stream_row0(int z0, int vb) { return z0 & ~(16 / vb - 1); }

// Producer loop of one block: chunks blockIdx.x, blockIdx.x + G, ... into the stage ring.
// A stage receives the chunk's metas, its row vectors (vec[v][a0 .. a1): the chunk's rows
// widened to 16-byte boundaries; every vector holds a multiple of 32 elements, so the widened
// end stays inside it) and, for part-0 chunks, its entries. Returns false if a wait ran out;
// on return every copy it issued has landed (or a drain wait ran out, reported as well).
template <int NV>
__device__ __forceinline__ bool stream_produce(const StreamPlan& pl, const int4* meta, const EntSet& es,
                                               const VecSet<NV>& vs, unsigned long long* full,
                                               unsigned long long* empty) {
  const unsigned long long pol_first = l2_evict_first(), pol_last = l2_evict_last();
  const int G = gridDim.x, nch = pl.total(), ns = pl.ns;
  bool ok = true;
  int j = 0;
  for (int ch = blockIdx.x; ch < nch; ch += G, ++j) {
    const int k = j % ns, u = j / ns;
    if (u > 0 && !mbar_wait(&empty[k], (unsigned)(u - 1) & 1u)) {
      ok = false;
      break;
    }
    const ChunkPos cp = chunk_pos(pl, ch);
    const int4 m0 = meta[cp.s0], m1 = meta[cp.s1 - 1];
    const unsigned mbytes = (unsigned)(cp.s1 - cp.s0) * 16u;
    const unsigned nent = cp.part ? 0u : (unsigned)(m1.x + m1.y * kSlice - m0.x);
    const unsigned vmask = cp.part ? vs.part1 : ~0u;
    const int z1 = m1.z + m1.w;
    const unsigned bbytes = es.sbase ? (unsigned)(cp.s1 - cp.s0) * (kAffineSlots * 4u) : 0u;
    unsigned tx = mbytes + bbytes;
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if ((vmask >> v) & 1u) {
        const int q = 16 / vs.vb[v];
        tx += (unsigned)(((z1 + q - 1) & ~(q - 1)) - stream_row0(m0.z, vs.vb[v])) * vs.vb[v];
      }
    for (int a = 0; a < es.n; ++a) tx += nent * es.eb[a];
    unsigned char* st = esd_dyn_smem + (size_t)k * pl.stage;
    mbar_arrive_expect_tx(&full[k], tx);
    bulk_load(st, meta + cp.s0, mbytes, &full[k], pol_first);
    if (bbytes) bulk_load(st + pl.cs * 16, es.sbase + (size_t)cp.s0 * kAffineSlots, bbytes, &full[k], pol_first);
    unsigned char* dst = st + pl.cs * pl.hdr;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int vb = vs.vb[v], q = 16 / vb;
      if ((vmask >> v) & 1u) {
        const int a0 = stream_row0(m0.z, vb), a1 = (z1 + q - 1) & ~(q - 1);
        bulk_load(dst, (const unsigned char*)vs.ptr[v] + (size_t)a0 * vb, (unsigned)(a1 - a0) * vb, &full[k],
                  ((vs.keep >> v) & 1u) ? pol_last : pol_first);
      }
      dst += stream_vcap(pl.cs, vb) * vb;
    }
    if (nent)
      for (int a = 0; a < es.n; ++a) {
        bulk_load(dst, (const unsigned char*)es.ptr[a] + (size_t)m0.x * es.eb[a], nent * es.eb[a], &full[k],
                  pol_first);
        dst += (size_t)pl.ecap * es.eb[a];
      }
  }
  // drain: the last use of every stage this block issued
  for (int k = 0; k < ns && k < j; ++k) {
    const int ulast = (j - 1 - k) / ns;
    if (!mbar_wait(&full[k], (unsigned)ulast & 1u)) ok = false;
  }
  return ok;
}

// One stage as a consumer warp sees it: the chunk's metas, the row vectors (element i of
// the chunk's rows is vec<V>(v, i)) and the entry arrays (entry x of the chunk at
// ent<E>(a)[x - x0]).
template <int NV>
struct StageView {
  const unsigned char* base;
  const unsigned char* vptr[NV];
  const unsigned char* eptr[2];
  const int* sbase;  // slot bases of the column-free copy (kAffineSlots per slice)
  int a0[NV];
  int x0;
  __device__ __forceinline__ const int4* meta() const { return reinterpret_cast<const int4*>(base); }
  template <typename V>
  __device__ __forceinline__ V vec(int v, int i) const {
    return reinterpret_cast<const V*>(vptr[v])[i - a0[v]];
  }
  template <typename E>
  __device__ __forceinline__ const E* ent(int a) const {
    return reinterpret_cast<const E*>(eptr[a]);
  }
};

// mbarriers of a staged block, set up by thread 0 (visible after the next block barrier)
__device__ __forceinline__ void stream_init_barriers(unsigned long long* full, unsigned long long* empty) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < kStreamMaxStages; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kStreamWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

// Consumer loop of one warp: for each chunk of this block, wait for its stage, call
// f(chunk position, stage view), then release the stage. Every consumer warp takes part in
// every chunk (the empty barrier counts kStreamWarps arrivals). False if a wait ran out.
template <int NV, typename F>
__device__ __forceinline__ bool stream_consume(const StreamPlan& pl, const EntSet& es, const VecSet<NV>& vs,
                                               unsigned long long* full, unsigned long long* empty, F&& f) {
  const int G = gridDim.x, nch = pl.total(), ns = pl.ns;
  int j = 0;
  for (int ch = blockIdx.x; ch < nch; ch += G, ++j) {
    const int k = j % ns, u = j / ns;
    if (!mbar_wait(&full[k], (unsigned)u & 1u)) return false;
    StageView<NV> sv;
    sv.base = esd_dyn_smem + (size_t)k * pl.stage;
    const int4 m0 = sv.meta()[0];
    sv.sbase = reinterpret_cast<const int*>(sv.base + pl.cs * 16);
    const unsigned char* q = sv.base + pl.cs * pl.hdr;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sv.vptr[v] = q;
      sv.a0[v] = stream_row0(m0.z, vs.vb[v]);
      q += stream_vcap(pl.cs, vs.vb[v]) * vs.vb[v];
    }
    sv.eptr[0] = q;
    sv.eptr[1] = q + (size_t)pl.ecap * es.eb[0];
    sv.x0 = m0.x;
    f(chunk_pos(pl, ch), sv);
    __syncwarp();
    if (lane_id() == 0) mbar_arrive(&empty[k]);
  }
  return true;
}

// The K slices of one consumer warp in a chunk (warp, warp + kStreamWarps, ...): their metas
// (zero for slices past the chunk's end: no rows, no entries).
template <int K, int NV>
__device__ __forceinline__ void stream_slices(const StageView<NV>& sv, const ChunkPos& cp, int warp, int4 (&md)[K]) {
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const int ls = warp + t * kStreamWarps;
    md[t] = ls < cp.s1 - cp.s0 ? sv.meta()[ls] : make_int4(0, 0, 0, 0);
  }
}

// Row products of K slices of one lane from staged FP32 entries: acc[t] += sum_e val_e *
// (v[col_e] - vi[t]) (vi = 0 in the plain form), the entries of a row in stored order, as
// row_fma and row_fma_diff take them. AFF = false: (value, column) pairs; AFF = true: the
// column-free copy, column = slot base + lane (a slot where the row has no entry holds 0 and
// points into the vector or into the kGuard zeros around it). The K slices are the warp's, at local indices
// warp + t kStreamWarps. Every gather of the K rows is issued before the first FMA. A row
// wider than W (which the launch plan excludes) is reported through `bad`.
template <int K, int W, bool DIFF, bool AFF, int NV>
__device__ __forceinline__ void staged_rows(const StageView<NV>& sv, const int4 (&md)[K], int warp, int lane,
                                            const float* __restrict__ v, const float (&vi)[K], float (&acc)[K],
                                            bool& bad) {
  float val[K][W], vj[K][W];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    bad |= md[t].y > W;
    const int off = (md[t].x - sv.x0) + lane;
    const int* sb = sv.sbase + (warp + t * kStreamWarps) * kAffineSlots;
#pragma unroll
    for (int e = 0; e < W; ++e) {
      int col = 0;
      val[t][e] = 0.f;
      if (e < md[t].y) {
        if constexpr (AFF) {
          val[t][e] = sv.template ent<float>(0)[off + e * kSlice];
          col = sb[e] + lane;
        } else {
          const uint2 pr = sv.template ent<uint2>(0)[off + e * kSlice];
          val[t][e] = __uint_as_float(pr.x);
          col = (int)pr.y;
        }
      }
      vj[t][e] = e < md[t].y ? v[col] : 0.f;
    }
  }
#pragma unroll
  for (int t = 0; t < K; ++t)
#pragma unroll
    for (int e = 0; e < W; ++e)
      if (e < md[t].y) acc[t] = fmaf(val[t][e], DIFF ? vj[t][e] - vi[t] : vj[t][e], acc[t]);
}

// The staged entries of a sliced-ELL part: the column-free copy (AFF) or the (value, column)
// pairs, and the metas that go with them.
template <bool AFF>
__device__ __forceinline__ EntSet stream_entries(const SellView<float>& M) {
  if constexpr (AFF) return EntSet{{M.aval, nullptr}, {4, 0}, 1, M.abase};
  else return EntSet{{M.ent, nullptr}, {8, 0}, 1, nullptr};
}
template <bool AFF>
__device__ __forceinline__ const int4* stream_metas(const SellView<float>& M) {
  return AFF ? M.ameta : M.meta;
}

// Compensated (Kahan) accumulation of one thread's partial sum: sum += v, with the rounding
// error of each addition carried in c. A thread of a staged kernel adds up to a few hundred
// terms of a dot product; with compensation its partial sum is exact to about the last bit
// whatever their number.
__device__ __forceinline__ void kahan_add(float& sum, float& c, float v) {
  const float y = __fsub_rn(v, c);
  const float t = __fadd_rn(sum, y);
  c = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

// Common entry of the staged kernels: barriers, the dependency wait, and the stop flag of the
// solve (false: the block leaves at once, before any copy is issued).
__device__ __forceinline__ bool stream_enter(State* st, unsigned long long* full, unsigned long long* empty,
                                             int* s_stop, bool loop_start, unsigned long long cond) {
  stream_init_barriers(full, empty);
  pdl_enter();
  if (threadIdx.x == 0) {
    // the loop-body bound of k_spmv_pq (the staged product starts the body in its place)
    if (loop_start && blockIdx.x == 0 && cond && atomicAdd(&st->guard, 1) >= st->maxit + 2) stream_fail(st, cond);
    *s_stop = st->conv;
  }
  __syncthreads();
  return *s_stop == 0;
}

// q = A p (difference form, FP32 inner solves) and (p, q); the last block sets alpha.
// Entries are (value bits, column) pairs; the products are formed in the order of
// row_fma_diff, so q is bit-identical to k_spmv_pq<float, 0>'s. Staged vectors: s = A 1, p.
template <typename T, int K, int W, bool AFF>
__global__ void __launch_bounds__(kStreamThreads, 2) k_spmv_pq_stream(IterCtx<T> c, StreamPlan pl) {
  static_assert(sizeof(T) == 4, "the staged product reads the FP32 (value, column) entries");
  __shared__ unsigned long long full[kStreamMaxStages], empty[kStreamMaxStages];
  __shared__ float red[kStreamThreads / 32 + 1];
  __shared__ int s_stop;
  State* st = c.st;
  if (!stream_enter(st, full, empty, &s_stop, true, c.cond)) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const EntSet es = stream_entries<AFF>(c.Av);
  const VecSet<2> vs{{c.rowsum, c.p}, {4, 4}, 2u, 0u};
  float acc[1] = {0.f}, cmp[1] = {0.f};
  if (warp == kStreamWarps) {
    if (lane == 0 && !stream_produce(pl, stream_metas<AFF>(c.Av), es, vs, full, empty)) stream_fail(st, c.cond);
  } else {
    const float* __restrict__ p = c.p;
    bool bad = false;
    const bool ok = stream_consume(pl, es, vs, full, empty, [&](const ChunkPos& cp, const StageView<2>& sv) {
      int4 md[K];
      stream_slices<K>(sv, cp, warp, md);
      float pv[K], q[K];
#pragma unroll
      for (int t = 0; t < K; ++t) {
        const bool valid = lane < md[t].w;
        const int i = md[t].z + lane;
        pv[t] = valid ? sv.template vec<float>(1, i) : 0.f;
        q[t] = fmaf(valid ? sv.template vec<float>(0, i) : 0.f, pv[t], 0.f);
      }
      staged_rows<K, W, true, AFF>(sv, md, warp, lane, p, pv, q, bad);
#pragma unroll
      for (int t = 0; t < K; ++t)
        if (lane < md[t].w) {
          c.q[md[t].z + lane] = q[t];
          kahan_add(acc[0], cmp[0], __fmul_rn(pv[t], q[t]));
        }
    });
    if (!ok || bad) stream_fail(st, c.cond);
  }
  acc[0] = __fsub_rn(acc[0], cmp[0]);
  if (grid_sum_multi<1>(acc, red, (float*)c.partials, &st->ticket[kTkSpmv]) && threadIdx.x == 0) {
    const double pq = (double)red[0];
    st->pq = pq;
    st->pap = pq;
    if (!(pq > 0.0) || !(st->rho > 0.0)) {
      st->status = ESD_ERR_BREAKDOWN;
      st->conv = 1;
      st->alpha = 0.0;
      end_loop(c.cond);
    } else if (st->status != ESD_ERR_INTERNAL) {
      const double a = st->rho / pq;
      st->alpha = a;
      c.ahist[st->iter] = a;
    }
  }
}

// x += alpha p (the FP64 iterate of the refinement form), r -= alpha q, ||r||^2, the pending
// sample, and forward level 0 (y = r / l_ii, sum y^2): the plain FP32 update of k_update_pipe
// with its vectors staged. Part 0 holds the forward-level-0 rows (x, p, q, r, 1/l_ii staged),
// part 1 the others (x, p, q, r). do_update = 0 runs the level-0 epilogue on r alone.
template <typename T, int PRE>
__global__ void __launch_bounds__(kStreamThreads, 2)
    k_update_stream(IterCtx<T> c, StreamPlan pl, int do_update, int finalize) {
  static_assert(sizeof(T) == 4, "the staged update is the FP32 inner solver's");
  __shared__ unsigned long long full[kStreamMaxStages], empty[kStreamMaxStages];
  __shared__ float red[2 * (kStreamThreads / 32 + 1)];
  __shared__ int s_stop;
  State* st = c.st;
  if (!stream_enter(st, full, empty, &s_stop, false, c.cond)) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const float alpha = (float)st->alpha;
  const double alpha_d = st->alpha;
  const int pend = do_update ? st->pend_slot : -1;
  const EntSet es{{nullptr, nullptr}, {0, 0}, 0};
  const VecSet<5> vs{{c.x64, c.p, c.q, c.r, c.inv_d}, {8, 4, 4, 4, 4}, 0u, 15u};
  float acc[2] = {0.f, 0.f}, cmp[2] = {0.f, 0.f};
  if (warp == kStreamWarps) {
    if (lane == 0 && !stream_produce(pl, c.Av.meta, es, vs, full, empty)) stream_fail(st, c.cond);
  } else {
    const unsigned bwd0 = pl.set[0].bwd0;
    const bool ok = stream_consume(pl, es, vs, full, empty, [&](const ChunkPos& cp, const StageView<5>& sv) {
      const bool lev0 = PRE == ESD_PRECOND_IC0 && cp.part == 0;
      const bool to_z = lev0 && ((bwd0 >> cp.range) & 1u);
      for (int ls = warp; ls < cp.s1 - cp.s0; ls += kStreamWarps) {
        const int4 md = sv.meta()[ls];
        if (lane >= md.w) continue;
        const int i = md.z + lane;
        float ri = sv.template vec<float>(3, i);
        if (do_update) {
          const double xi = sv.template vec<double>(0, i);
          if (pend >= 0 && c.samples64) c.samples64[(size_t)pend * c.ld + i] = xi;
          c.x64[i] = fma(alpha_d, (double)sv.template vec<float>(1, i), xi);
          ri = fmaf(-alpha, sv.template vec<float>(2, i), ri);
          c.r[i] = ri;
          kahan_add(acc[0], cmp[0], __fmul_rn(ri, ri));
        }
        if (lev0) {
          const float d = sv.template vec<float>(4, i);
          const float yv = ri * d;
          kahan_add(acc[1], cmp[1], __fmul_rn(yv, yv));
          c.Y[i] = to_z ? yv * d : yv;
        }
      }
    });
    if (!ok) stream_fail(st, c.cond);
  }
  acc[0] = __fsub_rn(acc[0], cmp[0]);
  acc[1] = __fsub_rn(acc[1], cmp[1]);
  if (grid_sum_multi<2>(acc, red, (float*)c.partials, &st->ticket[kTkUpdate]) && threadIdx.x == 0 &&
      st->status != ESD_ERR_INTERNAL)
    update_decide<PRE>(st, (double)red[0], (double)red[1], do_update, finalize, c.bhist, c.cond);
}

// One forward colour level (as k_fwd<float>): y_i = (r_i - sum_k l_ik y_k) / l_ii and
// sum y_i^2; the same slot / last-launch protocol for rho. Staged vectors: r, 1/l_ii.
template <typename T, int K, int W, bool AFF>
__global__ void __launch_bounds__(kStreamThreads, 2)
    k_fwd_stream(IterCtx<T> c, StreamPlan pl, int slot, int nprev, const int* __restrict__ prevG) {
  static_assert(sizeof(T) == 4, "the staged sweep reads the FP32 (value, column) entries");
  __shared__ unsigned long long full[kStreamMaxStages], empty[kStreamMaxStages];
  __shared__ float red[kStreamThreads / 32 + 1];
  __shared__ double own_s;
  __shared__ int s_stop;
  State* st = c.st;
  if (!stream_enter(st, full, empty, &s_stop, false, c.cond)) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const EntSet es = stream_entries<AFF>(c.Lv);
  const VecSet<2> vs{{c.r, c.inv_d}, {4, 4}, 0u, 0u};
  float acc[1] = {0.f}, cmp[1] = {0.f};
  if (warp == kStreamWarps) {
    if (lane == 0 && !stream_produce(pl, stream_metas<AFF>(c.Lv), es, vs, full, empty)) stream_fail(st, c.cond);
  } else {
    float* Y = c.Y;
    const unsigned bwd0 = pl.set[0].bwd0;
    bool bad = false;
    const bool ok = stream_consume(pl, es, vs, full, empty, [&](const ChunkPos& cp, const StageView<2>& sv) {
      int4 md[K];
      stream_slices<K>(sv, cp, warp, md);
      float d[K], y[K];
      const float zero[K] = {};
#pragma unroll
      for (int t = 0; t < K; ++t) {
        const bool valid = lane < md[t].w;
        const int i = md[t].z + lane;
        d[t] = valid ? sv.template vec<float>(1, i) : 0.f;
        y[t] = valid ? sv.template vec<float>(0, i) : 0.f;
      }
      staged_rows<K, W, false, AFF>(sv, md, warp, lane, Y, zero, y, bad);
      const bool to_z = (bwd0 >> cp.range) & 1u;
#pragma unroll
      for (int t = 0; t < K; ++t)
        if (lane < md[t].w) {
          const float yv = y[t] * d[t];
          kahan_add(acc[0], cmp[0], __fmul_rn(yv, yv));
          Y[md[t].z + lane] = to_z ? yv * d[t] : yv;
        }
    });
    if (!ok || bad) stream_fail(st, c.cond);
  }
  acc[0] = __fsub_rn(acc[0], cmp[0]);
  float* slots = (float*)c.rho_part;
  if (slot >= 0) {
    block_sum_multi<1>(acc, red);
    if (threadIdx.x == 0) slots[(size_t)slot * c.rho_stride + blockIdx.x] = red[0];
    return;
  }
  if (grid_sum_multi<1>(acc, red, (float*)c.partials, &st->ticket[kTkSweep])) {
    if (threadIdx.x == 0) own_s = (double)red[0];
    float acc2[1] = {0.f};
    for (int k = 0; k < nprev; ++k) {
      const int gk = prevG[k];
      for (int b = threadIdx.x; b < gk; b += blockDim.x) acc2[0] += __ldcg(&slots[(size_t)k * c.rho_stride + b]);
    }
    block_sum_multi<1>(acc2, red);
    if (threadIdx.x == 0 && st->status != ESD_ERR_INTERNAL)
      finalize_rho(st, own_s + (double)red[0] + st->rho_acc + st->fu, c.bhist, c.cond);
  }
}

// One backward colour level without subspace-correction terms (as k_bwd<float, 0>):
// z_i = (y_i - sum_j l_ji z_j) / l_ii, p_i = z_i + beta p_i. Part-1 chunks hold the rows
// whose z_i the forward sweep stored: direction update only. Staged vectors: y, 1/l_ii, p
// (part 1: y, p).
template <typename T, int K, int W, bool AFF>
__global__ void __launch_bounds__(kStreamThreads, 2) k_bwd_stream(IterCtx<T> c, StreamPlan pl) {
  static_assert(sizeof(T) == 4, "the staged sweep reads the FP32 (value, column) entries");
  __shared__ unsigned long long full[kStreamMaxStages], empty[kStreamMaxStages];
  __shared__ int s_stop;
  State* st = c.st;
  if (!stream_enter(st, full, empty, &s_stop, false, c.cond)) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const float beta = (float)st->beta;
  const bool first = st->iter == 0 || st->fresh_dir;
  const EntSet es = stream_entries<AFF>(c.Uv);
  const VecSet<3> vs{{c.Y, c.inv_d, c.p}, {4, 4, 4}, 0u, 5u};
  if (warp == kStreamWarps) {
    if (lane == 0 && !stream_produce(pl, stream_metas<AFF>(c.Uv), es, vs, full, empty)) stream_fail(st, c.cond);
  } else {
    float* Y = c.Y;
    bool bad = false;
    const bool ok = stream_consume(pl, es, vs, full, empty, [&](const ChunkPos& cp, const StageView<3>& sv) {
      const bool sweep = cp.part == 0;
      int4 md[K];
      stream_slices<K>(sv, cp, warp, md);
      float d[K], z[K], pold[K];
      const float zero[K] = {};
#pragma unroll
      for (int t = 0; t < K; ++t) {
        if (!sweep) md[t].y = 0;  // rows whose z_i the forward sweep stored
        const bool valid = lane < md[t].w;
        const int i = md[t].z + lane;
        z[t] = valid ? sv.template vec<float>(0, i) : 0.f;
        d[t] = (valid && sweep) ? sv.template vec<float>(1, i) : 1.f;
        pold[t] = (valid && !first) ? sv.template vec<float>(2, i) : 0.f;
      }
      if (sweep) staged_rows<K, W, false, AFF>(sv, md, warp, lane, Y, zero, z, bad);
#pragma unroll
      for (int t = 0; t < K; ++t)
        if (lane < md[t].w) {
          const int i = md[t].z + lane;
          const float zi = sweep ? z[t] * d[t] : z[t];
          if (sweep) Y[i] = zi;
          c.p[i] = first ? zi : fmaf(beta, pold[t], zi);
        }
    });
    if (!ok || bad) stream_fail(st, c.cond);
  }
}

// Whether the staged kernels are used (ESD_STREAM=0 in the environment turns them off, for
// comparisons); read once per process.
inline bool stream_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("ESD_STREAM");
    return !(e && e[0] == '0');
  }();
  return on;
}

// Blocks of a staged launch: one wave (as many as fit with the plan's stage ring), never
// more blocks than chunks.
template <typename... KArgs>
inline int stream_blocks(void (*kernel)(KArgs...), const StreamPlan& pl) {
  static std::mutex mu;
  static std::unordered_map<const void*, std::unordered_map<int, int>> cache;  // kernel -> smem -> blocks per SM
  const int smem = pl.ns * pl.stage;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto& per = cache[(const void*)kernel];
    if (per.empty())  // the largest stage ring a plan may have, set once per kernel
      ESD_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamRingCap));
    auto it = per.find(smem);
    if (it != per.end()) {
      per_sm = it->second;
    } else {
      ESD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kStreamThreads, smem));
      per_sm = std::max(1, per_sm);
      per[smem] = per_sm;
    }
  }
  return std::max(1, std::min(pl.total(), per_sm * (max_grid_blocks() / 4)));
}

// Launch a staged kernel on `blocks` blocks with programmatic stream serialisation on.
template <typename... KArgs, typename... Args>
inline void launch_stream(void (*kernel)(KArgs...), int blocks, const StreamPlan& pl, cudaStream_t s,
                          Args&&... args) {
  ESD_CHECK(pl.ns >= 2 && pl.ns <= kStreamMaxStages && pl.ns * pl.stage <= kStreamRingCap, ESD_ERR_INTERNAL,
            "staged launch: stage ring out of range");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kStreamThreads);
  cfg.dynamicSmemBytes = pl.ns * pl.stage;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ESD_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// Dispatch on the shape of a plan (KK slices per consumer warp, rows of at most WW entries).
#define ESD_DISPATCH_K(Srt, ...)                                                   \
  switch (Srt) {                                                                   \
    case 42: { constexpr int KK = 4, WW = 2; __VA_ARGS__; } break;                 \
    case 24: { constexpr int KK = 2, WW = 4; __VA_ARGS__; } break;                 \
    case 26: { constexpr int KK = 2, WW = 6; __VA_ARGS__; } break;                 \
    case 27: { constexpr int KK = 2, WW = 7; __VA_ARGS__; } break;                 \
    case 28: { constexpr int KK = 2, WW = 8; __VA_ARGS__; } break;                 \
    case 18: { constexpr int KK = 1, WW = 8; __VA_ARGS__; } break;                 \
    default: throw Error(ESD_ERR_INTERNAL, "unsupported staged shape");            \
  }

}  // namespace esd
