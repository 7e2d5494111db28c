// FP32 instantiation of the iteration kernels (inner solves of the iterative refinement).
#include "esd_iter.cuh"

namespace esd {
ESD_INSTANTIATE_ITER(float)

// ------------------------------------------------------------------ pairs of systems

// Why a pair of FP32 refinement-form contexts cannot run the paired kernels (empty: it can).
std::string pair_unsupported(const IterCtx<float>& c1, const IterCtx<float>& c2) {
  const esd_matrix* P = c1.P ? c1.P : c1.A;
  if (!stream_enabled()) return "the staged kernels are switched off (ESD_STREAM=0)";
  if (c1.A != c2.A || c1.P != c2.P) return "the two solvers must share the matrix and the preconditioning matrix";
  if (c1.mode != ESD_PLAIN || c2.mode != ESD_PLAIN) return "the pair solve runs plain PCG";
  if (c1.pre != ESD_PRECOND_IC0 || c2.pre != ESD_PRECOND_IC0) return "the pair solve runs with IC(0)";
  if (!c1.x64 || !c2.x64 || !c1.rowsum || !c1.Av.ent) return "the pair solve needs the refinement form";
  if (c1.A->A.wmax > kStreamWmax || !stream_sweeps<float>(P)) return "matrix rows wider than the staged kernels take";
  if (!P->upd_ok || P->fwd_sets.empty() || P->fwd_sets.size() > (size_t)kPairMaxLevels)
    return "colour levels the pair solve does not take";
  if (!c1.p12 || !c1.Y12) return "no side-by-side vectors for the pair";
  return "";
}

// One PCG iteration of both systems (the body of the paired loop; cond ends it). marks: an
// event after each launch (the names as launch_iteration's).
void launch_iteration_pair(const IterCtx<float>& c1, const IterCtx<float>& c2, unsigned long long cond,
                           cudaStream_t s, KernelMarks* marks) {
  const esd_matrix* A = c1.A;
  const esd_matrix* P = c1.P ? c1.P : c1.A;
  bool ok = true;
  if (marks) marks->mark(s, "start");
  {
    const bool aff = A->A.affine;
    const int w = pair_width(aff ? A->A.awmax : A->A.wmax);
    const int wmax = aff ? A->A.awmax : A->A.wmax, eb = aff ? 4 : 8, hdr = aff ? kHdrAffine : kHdrPlain;
    const StreamPlan pl = pair_plan(A->all, SliceSet{}, pair_chunk(wmax, eb, 1, 1, hdr), wmax, eb, 1, 1, hdr, &ok);
    ESD_CHECK(ok && w > 0, ESD_ERR_INTERNAL, "pair SpMV plan");
    ESD_DISPATCH_W(w, {
      if (aff) {
        auto k = k_spmv_pq_pair<WW, true>;
        launch_stream(k, stream_blocks(k, pl), pl, s, c1, c2, pl, cond);
      } else {
        auto k = k_spmv_pq_pair<WW, false>;
        launch_stream(k, stream_blocks(k, pl), pl, s, c1, c2, pl, cond);
      }
    });
    if (marks) marks->mark(s, "spmv_pq");
  }
  {
    const StreamPlan pl = pair_plan(P->upd_sets[0], P->upd_sets[1], kPairUpdateChunk, 0, 0, 5, 3, kHdrPlain, &ok);
    ESD_CHECK(ok, ESD_ERR_INTERNAL, "pair update plan");
    auto k = k_update_pair<ESD_PRECOND_IC0>;
    launch_stream(k, stream_blocks(k, pl), pl, s, c1, c2, pl, 0, cond);
    if (marks) marks->mark(s, "update");
  }
  const bool aff = affine_sweeps(P);
  const int eb = aff ? 4 : 8, hdr = aff ? kHdrAffine : kHdrPlain;
  PairGrids prev{};
  const size_t nf = P->fwd_sets.size();
  for (size_t l = 0; l < nf; ++l) {
    const int wmax = aff ? P->fwd_awmax[l] : P->fwd_wmax[l];
    const StreamPlan pl = pair_plan(P->fwd_sets[l], SliceSet{}, pair_chunk(wmax, eb, 3, 0, hdr), wmax, eb, 3, 0, hdr,
                                    &ok);
    ESD_CHECK(ok, ESD_ERR_INTERNAL, "pair forward plan");
    const bool last = l + 1 == nf;
    ESD_DISPATCH_W(pair_width(wmax), {
      auto k = aff ? k_fwd_pair<WW, true> : k_fwd_pair<WW, false>;
      const int G = stream_blocks(k, pl);
      prev.g[l] = G;
      launch_stream(k, G, pl, s, c1, c2, pl, last ? -1 : (int)l, last ? (int)l : 0, prev, cond);
    });
    if (marks) marks->mark(s, ("fwd_" + std::to_string(l + 1)).c_str());
  }
  SliceSet none{};
  const size_t nb = std::max(P->bwd_sets.size(), P->bwd0_sets.size());
  for (size_t l = 0; l < nb; ++l) {
    const SliceSet& sw = l < P->bwd_sets.size() ? P->bwd_sets[l] : none;
    const SliceSet& el = l < P->bwd0_sets.size() ? P->bwd0_sets[l] : none;
    const bool has = l < P->bwd_sets.size();
    const int wmax = has ? (aff ? P->bwd_awmax[l] : P->bwd_wmax[l]) : 0;
    const StreamPlan pl = pair_plan(sw, el, pair_chunk(wmax, eb, 1, 2, hdr), wmax, eb, 1, 2, hdr, &ok);
    ESD_CHECK(ok, ESD_ERR_INTERNAL, "pair backward plan");
    ESD_DISPATCH_W(pair_width(wmax), {
      auto k = aff ? k_bwd_pair<WW, true> : k_bwd_pair<WW, false>;
      launch_stream(k, stream_blocks(k, pl), pl, s, c1, c2, pl, cond);
    });
    if (marks) marks->mark(s, ("bwd_" + std::to_string(l + 1)).c_str());
  }
}

// (p_1, p_2) side by side from the two systems' p before the paired loop, and back after it.
__global__ void k_pair_pack(int n, const float* __restrict__ p1, const float* __restrict__ p2,
                            float2* __restrict__ p12) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p12[i] = make_float2(p1[i], p2[i]);
}

__global__ void k_pair_unpack(int n, const float2* __restrict__ p12, float* __restrict__ p1,
                              float* __restrict__ p2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 v = p12[i];
    p1[i] = v.x;
    p2[i] = v.y;
  }
}

void launch_pair_pack(const IterCtx<float>& c1, const IterCtx<float>& c2, bool pack, cudaStream_t s) {
  const int n = c1.A->n;
  const int G = std::min(max_grid_blocks(), (n + kBlock - 1) / kBlock);
  if (pack)
    k_pair_pack<<<G, kBlock, 0, s>>>(n, c1.p, c2.p, c1.p12);
  else
    k_pair_unpack<<<G, kBlock, 0, s>>>(n, c1.p12, c1.p, c2.p);
  ESD_CUDA(cudaGetLastError());
}

}  // namespace esd
