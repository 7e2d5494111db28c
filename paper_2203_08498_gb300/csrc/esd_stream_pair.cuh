// Two systems with the same matrix in one pass: the staged FP32 inner kernels of the
// refinement form for a pair of right-hand sides (plain PCG with IC(0)). Each kernel streams
// the matrix part of a chunk once and forms the rows of both systems from it; the two CG
// recurrences keep their own scalars, states and vectors (each solver's), so each system
// follows the iteration it would follow alone, up to the rounding of its dot products.
//
// Why: a staged launch costs a fixed 9-13 us (a block's first stage, the chunks of the last
// wave, the last block's reduction) plus its bytes, and half of an iteration's bytes are the
// matrix. Two systems that need only the same earlier solution (the adjoint of system t and
// the forward solve of system t + 1 of a time-stepping sequence both need x_t) can share both.
//
// The vectors the products gather, p and y, are kept for the paired loop side by side, (p_1,
// p_2) and (y_1, y_2) in one float2 array each (IterCtx::p12, Y12), so that one 8-byte gather
// serves both systems: k_pair_pack forms p12 from the two solvers' p before the loop and
// k_pair_unpack gives each its p back after it; y lives only within an iteration.
//
// Each row's products are taken in the same order as in the single kernels, so q, y and z
// are those of the single kernels for the same p, r and y; the dot products' per-thread
// partial sums cover other rows (the pair launches take their own chunks of slices), so the
// two systems follow their single runs up to that rounding. The paired loop ends when either
// inner run stops (the rest of that loop body skips it); the other goes on with the single
// kernels, from the state the paired ones left.
#pragma once

namespace esd {

constexpr int kPairUpdateChunk = 2 * kStreamWarps;  // slices per chunk of the pair update
constexpr int kPairSlices = 2;  // slices per consumer warp and chunk of the paired products, at most

// Slices per chunk of a paired product launch: kStreamWarps per pass of the consumer warps,
// up to kPairSlices passes (ESD_PAIR_SLICES = 1, 2 or 4 overrides it), as many as keep two
// stages in the ring.
inline int pair_chunk(int wmax, int ebytes, int nv4, int nv8, int hdr) {
  int kmax = kPairSlices;
  if (const char* e = std::getenv("ESD_PAIR_SLICES")) {
    const int v = std::atoi(e);
    if (v == 1 || v == 2 || v == 4) kmax = v;
  }
  for (int k = kmax; k > 1; k /= 2)
    if (2 * stream_stage_bytes(k * kStreamWarps, wmax, ebytes, nv4, nv8, hdr) <= kStreamRingCap)
      return k * kStreamWarps;
  return kStreamWarps;
}

// Plan with a fixed chunk of cs slices (no shape choice); ok = false when its ring of two
// stages does not fit kStreamRingCap.
inline StreamPlan pair_plan(const SliceSet& with_entries, const SliceSet& vectors_only, int cs, int wmax, int ebytes,
                            int nv4, int nv8, int hdr, bool* ok) {
  StreamPlan pl{};
  pl.cs = cs;
  pl.hdr = hdr;
  pl.stage = stream_stage_bytes(cs, wmax, ebytes, nv4, nv8, hdr);
  pl.ns = 3 * pl.stage <= kStreamRingCap ? 3 : 2;
  pl.ecap = cs * wmax * kSlice;
  pl.set[0] = with_entries;
  pl.set[1] = vectors_only;
  pl.cm[0] = chunk_map(with_entries, cs);
  pl.cm[1] = chunk_map(vectors_only, cs);
  *ok = 2 * pl.stage <= kStreamRingCap;
  return pl;
}

// Row width of a pair launch: the smallest of 2, 4, 6, 7, 8 that holds wmax (0: none fits).
inline int pair_width(int wmax) {
  for (int w : {2, 4, 6, 7, 8})
    if (std::max(wmax, 1) <= w) return w;
  return 0;
}

#define ESD_DISPATCH_W(Wrt, ...)                                                   \
  switch (Wrt) {                                                                   \
    case 2: { constexpr int WW = 2; __VA_ARGS__; } break;                          \
    case 4: { constexpr int WW = 4; __VA_ARGS__; } break;                          \
    case 6: { constexpr int WW = 6; __VA_ARGS__; } break;                          \
    case 7: { constexpr int WW = 7; __VA_ARGS__; } break;                          \
    case 8: { constexpr int WW = 8; __VA_ARGS__; } break;                          \
    default: throw Error(ESD_ERR_INTERNAL, "unsupported pair width");              \
  }

// One row of the warp's slice for both systems: acc_s += sum_e val_e (v_s[col_e] - vi_s),
// the entries in stored order (as staged_rows); v12 holds (v_1, v_2) side by side, so one
// 8-byte gather serves both systems. Every gather is issued before the first FMA.
template <int W, bool DIFF, bool AFF, int NV>
__device__ __forceinline__ void staged_rows_pair(const StageView<NV>& sv, const int4& md, int ls, int lane,
                                                 const float2* __restrict__ v12, float vi1, float vi2,
                                                 float& acc1, float& acc2, bool& bad) {
  float val[W];
  float2 t[W];
  bad |= md.y > W;
  const int off = (md.x - sv.x0) + lane;
  const int* sb = sv.sbase + ls * kAffineSlots;
#pragma unroll
  for (int e = 0; e < W; ++e) {
    int col = 0;
    val[e] = 0.f;
    if (e < md.y) {
      if constexpr (AFF) {
        val[e] = sv.template ent<float>(0)[off + e * kSlice];
        col = sb[e] + lane;
      } else {
        const uint2 pr = sv.template ent<uint2>(0)[off + e * kSlice];
        val[e] = __uint_as_float(pr.x);
        col = (int)pr.y;
      }
    }
    t[e] = e < md.y ? v12[col] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int e = 0; e < W; ++e)
    if (e < md.y) {
      acc1 = fmaf(val[e], DIFF ? t[e].x - vi1 : t[e].x, acc1);
      acc2 = fmaf(val[e], DIFF ? t[e].y - vi2 : t[e].y, acc2);
    }
}

// Entry of a pair kernel: barriers, the dependency wait, which systems are still running
// (act, in shared memory), and the loop-body bound of k_spmv_pq for each (loop_start). Block 0
// ends the paired loop when either has stopped. False: neither runs.
__device__ __forceinline__ bool pair_enter(State* st1, State* st2, unsigned long long* full, unsigned long long* empty,
                                           int* s_act, bool loop_start, unsigned long long cond) {
  stream_init_barriers(full, empty);
  pdl_enter();
  if (threadIdx.x == 0) {
    State* sts[2] = {st1, st2};
    for (int k = 0; k < 2; ++k) {
      if (loop_start && blockIdx.x == 0 && !sts[k]->conv && atomicAdd(&sts[k]->guard, 1) >= sts[k]->maxit + 2) {
        sts[k]->status = ESD_ERR_INTERNAL;
        sts[k]->conv = 1;
      }
      s_act[k] = !sts[k]->conv;
    }
    if (loop_start && blockIdx.x == 0 && s_act[0] && s_act[1]) st1->paired += 1;
    if ((!s_act[0] || !s_act[1]) && blockIdx.x == 0) end_loop(cond);
  }
  __syncthreads();
  return s_act[0] || s_act[1];
}

// q_s = A p_s (difference form) and (p_s, q_s) for both systems; the last block sets each
// running system's alpha. Staged vectors: s = A 1, (p_1, p_2).
template <int W, bool AFF>
__global__ void __launch_bounds__(kStreamThreads, 2)
    k_spmv_pq_pair(IterCtx<float> c1, IterCtx<float> c2, StreamPlan pl, unsigned long long cond) {
  __shared__ unsigned long long full[kStreamMaxStages], empty[kStreamMaxStages];
  __shared__ float red[2 * (kStreamThreads / 32 + 1)];
  __shared__ int s_act[2];
  if (!pair_enter(c1.st, c2.st, full, empty, s_act, true, cond)) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const EntSet es = stream_entries<AFF>(c1.Av);
  const VecSet<2> vs{{c1.rowsum, c1.p12}, {4, 8}, 2u, 0u};
  const bool act1 = s_act[0], act2 = s_act[1];
  float acc[2] = {0.f, 0.f}, cmp[2] = {0.f, 0.f};
  if (warp == kStreamWarps) {
    if (lane == 0 && !stream_produce(pl, stream_metas<AFF>(c1.Av), es, vs, full, empty)) {
      stream_fail(c1.st, cond);
      stream_fail(c2.st, cond);
    }
  } else {
    bool bad = false;
    const bool ok = stream_consume(pl, es, vs, full, empty, [&](const ChunkPos& cp, const StageView<2>& sv) {
      for (int ls = warp; ls < cp.s1 - cp.s0; ls += kStreamWarps) {
        const int4 md = sv.meta()[ls];
        const bool valid = lane < md.w;
        const int i = md.z + lane;
        const float si = valid ? sv.template vec<float>(0, i) : 0.f;
        const float2 pp = valid ? sv.template vec<float2>(1, i) : make_float2(0.f, 0.f);
        const float p1 = pp.x, p2 = pp.y;
        float q1 = fmaf(si, p1, 0.f), q2 = fmaf(si, p2, 0.f);
        staged_rows_pair<W, true, AFF>(sv, md, ls, lane, c1.p12, p1, p2, q1, q2, bad);
        if (valid) {
          if (act1) {
            c1.q[i] = q1;
            kahan_add(acc[0], cmp[0], __fmul_rn(p1, q1));
          }
          if (act2) {
            c2.q[i] = q2;
            kahan_add(acc[1], cmp[1], __fmul_rn(p2, q2));
          }
        }
      }
    });
    if (!ok || bad) {
      stream_fail(c1.st, cond);
      stream_fail(c2.st, cond);
    }
  }
  acc[0] = __fsub_rn(acc[0], cmp[0]);
  acc[1] = __fsub_rn(acc[1], cmp[1]);
  if (grid_sum_multi<2>(acc, red, (float*)c1.partials, &c1.st->ticket[kTkSpmv]) && threadIdx.x == 0) {
    State* sts[2] = {c1.st, c2.st};
    double* ah[2] = {c1.ahist, c2.ahist};
    const bool act[2] = {act1, act2};
    for (int k = 0; k < 2; ++k) {
      State* st = sts[k];
      if (!act[k] || st->status == ESD_ERR_INTERNAL) continue;
      const double pq = (double)red[k];
      st->pq = pq;
      st->pap = pq;
      if (!(pq > 0.0) || !(st->rho > 0.0)) {
        st->status = ESD_ERR_BREAKDOWN;
        st->conv = 1;
        st->alpha = 0.0;
      } else {
        const double a = st->rho / pq;
        st->alpha = a;
        ah[k][st->iter] = a;
      }
    }
    if (c1.st->conv || c2.st->conv) end_loop(cond);
  }
}

// The plain update of both systems (as k_update_stream): x_s += alpha_s p_s in FP64,
// r_s -= alpha_s q_s, ||r_s||^2 and forward level 0. Part 0: forward-level-0 rows (1/l_ii
// staged), part 1 the others. Staged vectors: x_1, x_2, (p_1, p_2), q_1, r_1, q_2, r_2, 1/l_ii.
template <int PRE>
__global__ void __launch_bounds__(kStreamThreads, 2)
    k_update_pair(IterCtx<float> c1, IterCtx<float> c2, StreamPlan pl, int finalize, unsigned long long cond) {
  __shared__ unsigned long long full[kStreamMaxStages], empty[kStreamMaxStages];
  __shared__ float red[4 * (kStreamThreads / 32 + 1)];
  __shared__ int s_act[2];
  if (!pair_enter(c1.st, c2.st, full, empty, s_act, false, cond)) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const bool act1 = s_act[0], act2 = s_act[1];
  const float al1 = (float)c1.st->alpha, al2 = (float)c2.st->alpha;
  const double ad1 = c1.st->alpha, ad2 = c2.st->alpha;
  const EntSet es{{nullptr, nullptr}, {0, 0}, 0};
  const VecSet<8> vs{{c1.x64, c2.x64, c1.p12, c1.q, c1.r, c2.q, c2.r, c1.inv_d}, {8, 8, 8, 4, 4, 4, 4, 4}, 0u,
                     127u};
  float acc[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
  if (warp == kStreamWarps) {
    if (lane == 0 && !stream_produce(pl, c1.Av.meta, es, vs, full, empty)) {
      stream_fail(c1.st, cond);
      stream_fail(c2.st, cond);
    }
  } else {
    const unsigned bwd0 = pl.set[0].bwd0;
    const bool ok = stream_consume(pl, es, vs, full, empty, [&](const ChunkPos& cp, const StageView<8>& sv) {
      const bool lev0 = PRE == ESD_PRECOND_IC0 && cp.part == 0;
      const bool to_z = lev0 && ((bwd0 >> cp.range) & 1u);
      for (int ls = warp; ls < cp.s1 - cp.s0; ls += kStreamWarps) {
        const int4 md = sv.meta()[ls];
        if (lane >= md.w) continue;
        const int i = md.z + lane;
        const float d = lev0 ? sv.template vec<float>(7, i) : 0.f;
        const float2 pp = sv.template vec<float2>(2, i);
        float2 y = make_float2(0.f, 0.f);  // a stopped system's y is not used
        if (act1) {
          const double xi = sv.template vec<double>(0, i);
          c1.x64[i] = fma(ad1, (double)pp.x, xi);
          const float ri = fmaf(-al1, sv.template vec<float>(3, i), sv.template vec<float>(4, i));
          c1.r[i] = ri;
          kahan_add(acc[0], cmp[0], __fmul_rn(ri, ri));
          if (lev0) {
            const float yv = ri * d;
            kahan_add(acc[1], cmp[1], __fmul_rn(yv, yv));
            y.x = to_z ? yv * d : yv;
          }
        }
        if (act2) {
          const double xi = sv.template vec<double>(1, i);
          c2.x64[i] = fma(ad2, (double)pp.y, xi);
          const float ri = fmaf(-al2, sv.template vec<float>(5, i), sv.template vec<float>(6, i));
          c2.r[i] = ri;
          kahan_add(acc[2], cmp[2], __fmul_rn(ri, ri));
          if (lev0) {
            const float yv = ri * d;
            kahan_add(acc[3], cmp[3], __fmul_rn(yv, yv));
            y.y = to_z ? yv * d : yv;
          }
        }
        if (lev0) c1.Y12[i] = y;
      }
    });
    if (!ok) {
      stream_fail(c1.st, cond);
      stream_fail(c2.st, cond);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] = __fsub_rn(acc[k], cmp[k]);
  if (grid_sum_multi<4>(acc, red, (float*)c1.partials, &c1.st->ticket[kTkUpdate]) && threadIdx.x == 0) {
    if (act1 && c1.st->status != ESD_ERR_INTERNAL)
      update_decide<PRE>(c1.st, (double)red[0], (double)red[1], 1, finalize, c1.bhist, 0ull);
    if (act2 && c2.st->status != ESD_ERR_INTERNAL)
      update_decide<PRE>(c2.st, (double)red[2], (double)red[3], 1, finalize, c2.bhist, 0ull);
    if (c1.st->conv || c2.st->conv) end_loop(cond);
  }
}

// One forward colour level of both systems (as k_fwd_stream), each system's rho sums in its
// own slots; the last launch sets each running system's beta. Staged vectors: r_1, r_2, 1/l_ii.
// y goes to (y_1, y_2) side by side (a stopped system's half is not used).
// Grids of the forward launches before the last one of a sweep (whose slots it adds up).
constexpr int kPairMaxLevels = 16;
struct PairGrids {
  int g[kPairMaxLevels];
};

template <int W, bool AFF>
__global__ void __launch_bounds__(kStreamThreads, 2)
    k_fwd_pair(IterCtx<float> c1, IterCtx<float> c2, StreamPlan pl, int slot, int nprev, PairGrids prevG,
               unsigned long long cond) {
  __shared__ unsigned long long full[kStreamMaxStages], empty[kStreamMaxStages];
  __shared__ float red[2 * (kStreamThreads / 32 + 1)];
  __shared__ double own_s[2];
  __shared__ int s_act[2];
  if (!pair_enter(c1.st, c2.st, full, empty, s_act, false, cond)) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const bool act1 = s_act[0], act2 = s_act[1];
  const EntSet es = stream_entries<AFF>(c1.Lv);
  const VecSet<3> vs{{c1.r, c2.r, c1.inv_d}, {4, 4, 4}, 0u, 0u};
  float acc[2] = {0.f, 0.f}, cmp[2] = {0.f, 0.f};
  if (warp == kStreamWarps) {
    if (lane == 0 && !stream_produce(pl, stream_metas<AFF>(c1.Lv), es, vs, full, empty)) {
      stream_fail(c1.st, cond);
      stream_fail(c2.st, cond);
    }
  } else {
    const unsigned bwd0 = pl.set[0].bwd0;
    bool bad = false;
    const bool ok = stream_consume(pl, es, vs, full, empty, [&](const ChunkPos& cp, const StageView<3>& sv) {
      for (int ls = warp; ls < cp.s1 - cp.s0; ls += kStreamWarps) {
        const int4 md = sv.meta()[ls];
        const bool valid = lane < md.w;
        const int i = md.z + lane;
        const float d = valid ? sv.template vec<float>(2, i) : 0.f;
        float y1 = valid ? sv.template vec<float>(0, i) : 0.f;
        float y2 = valid ? sv.template vec<float>(1, i) : 0.f;
        staged_rows_pair<W, false, AFF>(sv, md, ls, lane, c1.Y12, 0.f, 0.f, y1, y2, bad);
        const bool to_z = (bwd0 >> cp.range) & 1u;
        if (valid) {
          const float yv1 = y1 * d, yv2 = y2 * d;
          if (act1) kahan_add(acc[0], cmp[0], __fmul_rn(yv1, yv1));
          if (act2) kahan_add(acc[1], cmp[1], __fmul_rn(yv2, yv2));
          c1.Y12[i] = to_z ? make_float2(yv1 * d, yv2 * d) : make_float2(yv1, yv2);
        }
      }
    });
    if (!ok || bad) {
      stream_fail(c1.st, cond);
      stream_fail(c2.st, cond);
    }
  }
  acc[0] = __fsub_rn(acc[0], cmp[0]);
  acc[1] = __fsub_rn(acc[1], cmp[1]);
  float* slots[2] = {(float*)c1.rho_part, (float*)c2.rho_part};
  if (slot >= 0) {
    block_sum_multi<2>(acc, red);
    if (threadIdx.x == 0) {
      slots[0][(size_t)slot * c1.rho_stride + blockIdx.x] = red[0];
      slots[1][(size_t)slot * c2.rho_stride + blockIdx.x] = red[1];
    }
    return;
  }
  if (grid_sum_multi<2>(acc, red, (float*)c1.partials, &c1.st->ticket[kTkSweep])) {
    if (threadIdx.x < 2) own_s[threadIdx.x] = (double)red[threadIdx.x];
    float acc2[2] = {0.f, 0.f};
    for (int k = 0; k < nprev; ++k) {
      const int gk = prevG.g[k];
      for (int b = threadIdx.x; b < gk; b += blockDim.x) {
        acc2[0] += __ldcg(&slots[0][(size_t)k * c1.rho_stride + b]);
        acc2[1] += __ldcg(&slots[1][(size_t)k * c2.rho_stride + b]);
      }
    }
    block_sum_multi<2>(acc2, red);
    if (threadIdx.x == 0) {
      State* sts[2] = {c1.st, c2.st};
      double* bh[2] = {c1.bhist, c2.bhist};
      const bool act[2] = {act1, act2};
      for (int k = 0; k < 2; ++k)
        if (act[k] && sts[k]->status != ESD_ERR_INTERNAL)
          finalize_rho(sts[k], own_s[k] + (double)red[k] + sts[k]->rho_acc + sts[k]->fu, bh[k], 0ull);
      if (c1.st->conv || c2.st->conv) end_loop(cond);
    }
  }
}

// One backward colour level of both systems (as k_bwd_stream): z_s, then p_s = z_s +
// beta_s p_s. Part-1 chunks: direction update only. Staged vectors: (y_1, y_2), 1/l_ii,
// (p_1, p_2) (part 1: (y_1, y_2), (p_1, p_2)). A stopped system's p is written back unchanged.
template <int W, bool AFF>
__global__ void __launch_bounds__(kStreamThreads, 2)
    k_bwd_pair(IterCtx<float> c1, IterCtx<float> c2, StreamPlan pl, unsigned long long cond) {
  __shared__ unsigned long long full[kStreamMaxStages], empty[kStreamMaxStages];
  __shared__ int s_act[2];
  if (!pair_enter(c1.st, c2.st, full, empty, s_act, false, cond)) return;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const bool act1 = s_act[0], act2 = s_act[1];
  const float be1 = (float)c1.st->beta, be2 = (float)c2.st->beta;
  const bool first1 = c1.st->iter == 0 || c1.st->fresh_dir, first2 = c2.st->iter == 0 || c2.st->fresh_dir;
  const EntSet es = stream_entries<AFF>(c1.Uv);
  const VecSet<3> vs{{c1.Y12, c1.inv_d, c1.p12}, {8, 4, 8}, 0u, 5u};
  if (warp == kStreamWarps) {
    if (lane == 0 && !stream_produce(pl, stream_metas<AFF>(c1.Uv), es, vs, full, empty)) {
      stream_fail(c1.st, cond);
      stream_fail(c2.st, cond);
    }
  } else {
    bool bad = false;
    const bool ok = stream_consume(pl, es, vs, full, empty, [&](const ChunkPos& cp, const StageView<3>& sv) {
      for (int ls = warp; ls < cp.s1 - cp.s0; ls += kStreamWarps) {
        const bool sweep = cp.part == 0;
        int4 md = sv.meta()[ls];
        if (!sweep) md.y = 0;  // rows whose z_i the forward sweep stored
        const bool valid = lane < md.w;
        const int i = md.z + lane;
        const float2 yy = valid ? sv.template vec<float2>(0, i) : make_float2(0.f, 0.f);
        float z1 = yy.x, z2 = yy.y;
        const float d = (valid && sweep) ? sv.template vec<float>(1, i) : 1.f;
        const float2 po = valid ? sv.template vec<float2>(2, i) : make_float2(0.f, 0.f);
        if (sweep) staged_rows_pair<W, false, AFF>(sv, md, ls, lane, c1.Y12, 0.f, 0.f, z1, z2, bad);
        if (valid) {
          const float zi1 = sweep ? z1 * d : z1, zi2 = sweep ? z2 * d : z2;
          if (sweep) c1.Y12[i] = make_float2(zi1, zi2);
          const float pn1 = act1 ? (first1 ? zi1 : fmaf(be1, po.x, zi1)) : po.x;
          const float pn2 = act2 ? (first2 ? zi2 : fmaf(be2, po.y, zi2)) : po.y;
          c1.p12[i] = make_float2(pn1, pn2);
        }
      }
    });
    if (!ok || bad) {
      stream_fail(c1.st, cond);
      stream_fail(c2.st, cond);
    }
  }
}

}  // namespace esd
