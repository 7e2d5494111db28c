// Solver runtime: device buffers, one CUDA graph per mode (the whole solve, with the PCG
// loop as a device-side conditional while node), the auxiliary-matrix construction, the
// Lanczos condition estimate and the C ABI of the solver.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <limits>
#include <memory>
#include <vector>

#include "esd_dense.h"
#include "esd_refine.h"

namespace esd {

// ------------------------------------------------------------------ small kernels

__global__ void k_pattern_grad(int n, const int* rp, const int* ci, const double* lam, const double* x,
                               double* grad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double li = lam[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) grad[k] = -li * x[ci[k]];
  }
}

// Add a conditional while node after the current dependencies of the capture on stream s
// (whatever graph s captures into) and return its body graph.
static cudaGraph_t add_while_node(cudaStream_t s, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  ESD_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t wnode;
  ESD_CUDA(cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &np));
  ESD_CUDA(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  return np.conditional.phGraph_out[0];
}

// b = 0 gives x = 0 (refinement form)
__global__ void k_ref_final(int n, double* x, const RefineState* rs) {
  if (rs->bb != 0.0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
}

}  // namespace esd

using namespace esd;

struct esd_solver {
  esd_matrix* A = nullptr;
  esd_matrix* P = nullptr;  // preconditioning matrix (its IC(0) factor and levels), nullptr = A
  const esd_matrix* PM() const { return P ? P : A; }
  esd_params prm{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;   // private capture streams
  cudaStream_t cap2 = nullptr;
  cudaStream_t cap3 = nullptr;
  int mode = ESD_PLAIN;
  size_t ld = 0;
  DevBuf vb, vx, vr, vp, vq, vY, samples;
  DevBuf W, AW, E, Einv, ritz, ahist, bhist, state, partials, rho_part, ext, lz;
  DevBuf AWdf, awscale, awexp;  // AW as double-float pairs for the FP64 deflated iteration
  DevBuf Wdf, wscale;           // W likewise, for the FP64 subspace correction
  State* hst = nullptr;  // pinned host copy
  // FP32-inner / FP64-refinement form
  bool fp32 = false;
  DevBuf b32, x32, r32, p32, q32, Y32, W32, AW32, r64, state_in, rstate;
  State* hst_in = nullptr;      // pinned copy of the inner state
  RefineState* hrs = nullptr;   // pinned copy of the refinement state
  int last_outer = 0;
  int m = 0, M = 0;      // columns of W, padded count
  int mbar = 0;
  bool have_W = false;
  int w_version = 0;
  int w_values_version = -1;  // the matrix values W's AW and E were formed for
  // power method of the condition estimate: two vectors (stride ld) and its device state
  DevBuf pw_v, pw_state;
  bool pw_on = false;
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  int exec_version[3] = {-1, -1, -1};
  bool exec_pw[3] = {false, false, false};
  // the graph of a pair solve with another solver (esd_solve_pair), kept while neither
  // solver's graphs are dropped (epoch: bumped whenever they are, as buffers may have moved)
  unsigned long long uid = 0;
  int epoch = 0;
  cudaGraphExec_t pair_exec = nullptr;
  unsigned long long pair_uid = 0;
  int pair_epoch_self = -1, pair_epoch_other = -1;
  int last_iters = 0, last_status = 0, last_sample_m = 0, last_maxit = 0;
  double last_relres = 0.0, last_true = 0.0;
  AuxBuild aux;

  ~esd_solver() {
    for (auto& e : exec)
      if (e) cudaGraphExecDestroy(e);
    if (pair_exec) cudaGraphExecDestroy(pair_exec);
    if (cap) cudaStreamDestroy(cap);
    if (cap2) cudaStreamDestroy(cap2);
    if (cap3) cudaStreamDestroy(cap3);
    if (hst) cudaFreeHost(hst);
    if (hst_in) cudaFreeHost(hst_in);
    if (hrs) cudaFreeHost(hrs);
  }

  // (p_1, p_2) and (y_1, y_2) side by side for the paired kernels of the pairs this solver
  // leads, with kGuard zero pairs on each side (as p32 and Y32); allocated at its first pair
  DevBuf pair_p12, pair_Y12;
  void ensure_pair_vectors() {
    if (pair_p12.get()) return;
    const size_t bytes = sizeof(float2) * (ld + 2 * kGuard);
    for (DevBuf* b : {&pair_p12, &pair_Y12}) {
      b->alloc(bytes);
      ESD_CUDA(cudaMemsetAsync(b->get(), 0, bytes, stream));
    }
  }
  // this solver's plain FP32 context as a system of the pair that `lead` leads
  IterCtx<float> pair_ctx32(const esd_solver* lead) const {
    IterCtx<float> c = ctx32(ESD_PLAIN);
    c.p12 = lead->pair_p12.as<float2>() ? lead->pair_p12.as<float2>() + kGuard : nullptr;
    c.Y12 = lead->pair_Y12.as<float2>() ? lead->pair_Y12.as<float2>() + kGuard : nullptr;
    return c;
  }

  IterCtx<float> ctx32(int md) const {
    IterCtx<float> c;
    c.A = A;
    c.P = PM();
    c.Av = A->A.view<float>();
    c.Lv = PM()->L.view<float>();
    c.Uv = PM()->U.view<float>();
    c.inv_d = PM()->inv_d32.as<float>();
    c.rowsum = A->rowsum32.as<float>();
    c.b = b32.as<float>();
    c.x = x32.as<float>();
    c.r = r32.as<float>();
    c.p = p32.as<float>() + kGuard;
    c.q = q32.as<float>();
    c.Y = Y32.as<float>() + kGuard;
    c.ld = ld;
    c.mode = md;
    c.pre = prm.precond;
    if (md != ESD_PLAIN) {
      c.W = W32.as<float>();
      c.AW = AW32.as<float>();
      c.Einv = Einv.as<double>();
      c.M = M;
      c.wsm = 1;  // W32 / AW32 are slice-major
    }
    c.samples = nullptr;
    c.samples64 = samples.get() ? samples.as<double>() : nullptr;  // FP64 full iterates
    c.xbase = vx.as<double>();
    c.x64 = vx.as<double>();  // the inner iteration updates the FP64 iterate directly
    c.ahist = ahist.as<double>();
    c.bhist = bhist.as<double>();
    c.partials = partials.get();
    c.rho_part = rho_part.get();
    c.rho_stride = (size_t)max_grid_blocks();
    c.st = state_in.as<State>();
    c.sflags = PM()->slice_flags.as<unsigned char>();
    return c;
  }

  IterCtx<double> ctx(int md) const {
    IterCtx<double> c;
    c.A = A;
    c.P = PM();
    c.Av = A->A.view<double>();
    c.Lv = PM()->L.view<double>();
    c.Uv = PM()->U.view<double>();
    c.inv_d = PM()->inv_d.as<double>();
    c.b = vb.as<double>();
    c.x = vx.as<double>();
    c.r = vr.as<double>();
    c.p = vp.as<double>();
    c.q = vq.as<double>();
    c.Y = vY.as<double>();
    c.ld = ld;
    c.mode = md;
    c.pre = prm.precond;
    if (md != ESD_PLAIN) {
      c.W = W.as<double>();
      c.AW = AW.as<double>();
      c.Einv = Einv.as<double>();
      c.M = M;
      c.AWdf = AWdf.as<float2>();
      c.awscale = awscale.as<double>();
      c.Wdf = Wdf.as<float2>();
      c.wscale = wscale.as<double>();
      ESD_CHECK(!df_cols(M) || (c.AWdf && c.Wdf), ESD_ERR_INTERNAL, "the double-float copies of AW and W are missing");
    }
    c.samples = samples.get() ? samples.as<double>() : nullptr;
    c.ahist = ahist.as<double>();
    c.bhist = bhist.as<double>();
    c.partials = partials.get();
    c.rho_part = rho_part.get();
    c.rho_stride = (size_t)max_grid_blocks();
    c.st = state.as<State>();
    c.sflags = PM()->slice_flags.as<unsigned char>();
    if (pw_on) {
      c.pw[0] = pw_v.as<double>();
      c.pw[1] = pw_v.as<double>() + ld;
      c.pws = pw_state.as<PowerState>();
    }
    return c;
  }

  void build_graph(int md) {
    if (exec[md] && exec_version[md] == w_version && exec_pw[md] == pw_on) return;
    if (exec[md]) {
      cudaGraphExecDestroy(exec[md]);
      exec[md] = nullptr;
    }
    cudaGraph_t g;
    ESD_CUDA(cudaGraphCreate(&g, 0));
    try {
      if (fp32) capture_refine(g, md); else capture_fp64(g, md);
    } catch (...) {
      cudaGraphDestroy(g);
      throw;
    }
    cudaGraphExec_t e;
    cudaError_t err = cudaGraphInstantiate(&e, g, 0);
    cudaGraphDestroy(g);
    ESD_CUDA(err);
    exec[md] = e;
    exec_version[md] = w_version;
    exec_pw[md] = pw_on;
  }

  // r0, z0, p0 -> while (not stopped) { PCG iteration } -> correction, true residual
  void capture_fp64(cudaGraph_t g, int md) {
    cudaGraphConditionalHandle h;
    ESD_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    IterCtx<double> c = ctx(md);
    c.cond = (unsigned long long)h;
    ESD_CUDA(cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      launch_init<double>(c, cap);
      cudaGraph_t body = add_while_node(cap, h);
      ESD_CUDA(cudaStreamBeginCaptureToGraph(cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      try {
        launch_iteration<double>(c, cap2);
      } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(cap2, &dummy);
        throw;
      }
      ESD_CUDA(cudaStreamEndCapture(cap2, &body));
      launch_finish<double>(c, cap);
      launch_true_residual(c, cap);
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(cap, &dummy);
      throw;
    }
    ESD_CUDA(cudaStreamEndCapture(cap, &g));
  }

  // FP64 residual -> while (not converged) { b32 = r; FP32 PCG (its own while loop);
  // x += d; FP64 residual } -> x = 0 when b = 0
  void capture_refine(cudaGraph_t g, int md) {
    cudaGraphConditionalHandle h_out, h_in;
    ESD_CUDA(cudaGraphConditionalHandleCreate(&h_out, g, 1, cudaGraphCondAssignDefault));
    IterCtx<double> c64 = ctx(ESD_PLAIN);
    c64.rowsum = A->rowsum64.as<double>();  // difference-form FP64 residual
    IterCtx<float> c32 = ctx32(md);
    c32.x_zero = 1;  // every inner solve starts from d = 0
    RefineState* rs = rstate.as<RefineState>();
    const int n = A->n;
    ESD_CUDA(cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      launch_ref_residual(c64, r64.as<double>(), r32.as<float>(), rs, nullptr, (unsigned long long)h_out, cap);
      cudaGraph_t body = add_while_node(cap, h_out);
      // the inner loop's handle belongs to the graph that holds the inner while node
      ESD_CUDA(cudaGraphConditionalHandleCreate(&h_in, body, 0, 0));
      c32.cond = (unsigned long long)h_in;
      ESD_CUDA(cudaStreamBeginCaptureToGraph(cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      try {
        launch_ref_prep(n, r64.as<double>(), b32.as<float>(), x32.as<float>(), state_in.as<State>(), rs,
                        (unsigned long long)h_in, cap2);
        launch_init<float>(c32, cap2);
        cudaGraph_t inner = add_while_node(cap2, h_in);
        ESD_CUDA(cudaStreamBeginCaptureToGraph(cap3, inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        try {
          launch_iteration<float>(c32, cap3);
        } catch (...) {
          cudaGraph_t dummy;
          cudaStreamEndCapture(cap3, &dummy);
          throw;
        }
        ESD_CUDA(cudaStreamEndCapture(cap3, &inner));
        launch_finish<float>(c32, cap2);
        launch_ref_residual(c64, r64.as<double>(), r32.as<float>(), rs, state_in.as<State>(),
                            (unsigned long long)h_out, cap2);
      } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(cap2, &dummy);
        throw;
      }
      ESD_CUDA(cudaStreamEndCapture(cap2, &body));
      k_ref_final<<<max_grid_blocks(), kBlock, 0, cap>>>(n, vx.as<double>(), rs);
      ESD_CUDA(cudaGetLastError());
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(cap, &dummy);
      throw;
    }
    ESD_CUDA(cudaStreamEndCapture(cap, &g));
  }

  // Buffers of the refinement form (FP32 inner vectors, FP64 residual, inner and outer state)
  // and the FP32 copies of the matrix; allocated once.
  void enable_fp32() {
    if (!b32.get()) {
      const size_t fbytes = sizeof(float) * ld, vbytes = sizeof(double) * ld;
      for (DevBuf* b : {&b32, &x32, &r32, &p32, &q32, &Y32}) {
        // p and Y, which the row products gather, carry kGuard zeros before and after
        const size_t bytes = (b == &p32 || b == &Y32) ? fbytes + 2 * kGuard * sizeof(float) : fbytes;
        b->alloc(bytes);
        ESD_CUDA(cudaMemsetAsync(b->get(), 0, bytes, stream));
      }
      r64.alloc(vbytes);
      ESD_CUDA(cudaMemsetAsync(r64.get(), 0, vbytes, stream));
      state_in.alloc(sizeof(State));
      ESD_CUDA(cudaMemsetAsync(state_in.get(), 0, sizeof(State), stream));
      rstate.alloc(sizeof(RefineState));
      ESD_CUDA(cudaMemsetAsync(rstate.get(), 0, sizeof(RefineState), stream));
      ESD_CUDA(cudaMallocHost(&hst_in, sizeof(State)));
      ESD_CUDA(cudaMallocHost(&hrs, sizeof(RefineState)));
      std::memset(hst_in, 0, sizeof(State));
      std::memset(hrs, 0, sizeof(RefineState));
    }
    fp32 = true;
    A->ensure_fp32();
  }

  // AW and W as double-float pairs for the FP64 iteration (up to 32 padded columns); the
  // refinement form reads its FP32 copies instead and needs none
  void refresh_df() {
    if (fp32 || !have_W || !df_cols(M)) return;
    const size_t need = sizeof(float2) * (size_t)A->nslices * kSlice * M;
    if (AWdf.bytes() < need) {
      AWdf.alloc(need);
      Wdf.alloc(need);
    }
    if (!awscale.get()) {
      awscale.alloc(sizeof(double) * kMaxM);
      wscale.alloc(sizeof(double) * kMaxM);
      awexp.alloc(sizeof(int) * kMaxM);
    }
    launch_df_pairs(A, AW.as<double>(), ld, m, M, AWdf.as<float2>(), awscale.as<double>(), awexp.as<int>(), stream);
    launch_df_pairs(A, W.as<double>(), ld, m, M, Wdf.as<float2>(), wscale.as<double>(), awexp.as<int>(), stream);
    ESD_CUDA(cudaStreamSynchronize(stream));
  }

  void drop_graphs() {
    for (int md = 0; md < 3; ++md) {
      if (exec[md]) cudaGraphExecDestroy(exec[md]);
      exec[md] = nullptr;
      exec_version[md] = -1;
    }
    if (pair_exec) cudaGraphExecDestroy(pair_exec);
    pair_exec = nullptr;
    ++epoch;
  }

  // The refinement loop of this solver's system and `o`'s, run together: FP64 residuals ->
  // while (either has not stopped) { both inner runs prepared (a stopped one stays stopped)
  // and started; while (both inner runs go on) { one PCG iteration of both, sharing the
  // passes over the matrix }; while (the one left goes on) { its single iteration }; both
  // corrected, FP64 residuals } -> x = 0 where b = 0.
  void capture_refine_pair(cudaGraph_t g, esd_solver* o) {
    esd_solver* sv[2] = {this, o};
    cudaGraphConditionalHandle h_out, h_in, h_one[2];
    ESD_CUDA(cudaGraphConditionalHandleCreate(&h_out, g, 1, cudaGraphCondAssignDefault));
    IterCtx<double> c64[2];
    IterCtx<float> c32[2];
    RefineState* rs[2];
    State* st[2];
    for (int k = 0; k < 2; ++k) {
      c64[k] = sv[k]->ctx(ESD_PLAIN);
      c64[k].rowsum = A->rowsum64.as<double>();
      c32[k] = sv[k]->pair_ctx32(this);
      c32[k].x_zero = 1;
      c32[k].cond = 0;  // the paired loop is ended by the pair kernels
      rs[k] = sv[k]->rstate.as<RefineState>();
      st[k] = sv[k]->state_in.as<State>();
    }
    const int n = A->n;
    auto inner_loop = [&](cudaGraphConditionalHandle h, auto&& body_fn) {
      cudaGraph_t inner = add_while_node(cap2, h);
      ESD_CUDA(cudaStreamBeginCaptureToGraph(cap3, inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      try {
        body_fn();
      } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(cap3, &dummy);
        throw;
      }
      ESD_CUDA(cudaStreamEndCapture(cap3, &inner));
    };
    ESD_CUDA(cudaStreamBeginCaptureToGraph(cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      for (int k = 0; k < 2; ++k)
        launch_ref_residual(c64[k], sv[k]->r64.as<double>(), sv[k]->r32.as<float>(), rs[k], nullptr, 0ull, cap, 1);
      launch_pair_cond(rs[0], rs[1], (unsigned long long)h_out, cap);
      cudaGraph_t body = add_while_node(cap, h_out);
      ESD_CUDA(cudaGraphConditionalHandleCreate(&h_in, body, 0, 0));
      for (int k = 0; k < 2; ++k) ESD_CUDA(cudaGraphConditionalHandleCreate(&h_one[k], body, 0, 0));
      ESD_CUDA(cudaStreamBeginCaptureToGraph(cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      try {
        for (int k = 0; k < 2; ++k)
          launch_ref_prep(n, sv[k]->r64.as<double>(), sv[k]->b32.as<float>(), sv[k]->x32.as<float>(), st[k], rs[k],
                          0ull, cap2);
        for (int k = 0; k < 2; ++k) launch_init<float>(c32[k], cap2);
        launch_pair_pack(c32[0], c32[1], true, cap2);
        launch_inner_cond(st[0], st[1], (unsigned long long)h_in, cap2);
        inner_loop(h_in, [&] { launch_iteration_pair(c32[0], c32[1], (unsigned long long)h_in, cap3); });
        launch_pair_pack(c32[0], c32[1], false, cap2);
        for (int k = 0; k < 2; ++k) {
          IterCtx<float> c1 = c32[k];
          c1.cond = (unsigned long long)h_one[k];
          launch_inner_cond(st[k], nullptr, c1.cond, cap2);
          inner_loop(h_one[k], [&] { launch_iteration<float>(c1, cap3); });
        }
        for (int k = 0; k < 2; ++k) launch_finish<float>(c32[k], cap2);
        for (int k = 0; k < 2; ++k)
          launch_ref_residual(c64[k], sv[k]->r64.as<double>(), sv[k]->r32.as<float>(), rs[k], st[k], 0ull, cap2, 1);
        launch_pair_cond(rs[0], rs[1], (unsigned long long)h_out, cap2);
      } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(cap2, &dummy);
        throw;
      }
      ESD_CUDA(cudaStreamEndCapture(cap2, &body));
      for (int k = 0; k < 2; ++k) {
        k_ref_final<<<max_grid_blocks(), kBlock, 0, cap>>>(n, sv[k]->vx.as<double>(), rs[k]);
        ESD_CUDA(cudaGetLastError());
      }
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(cap, &dummy);
      throw;
    }
    ESD_CUDA(cudaStreamEndCapture(cap, &g));
  }

  void build_pair_graph(esd_solver* o) {
    if (pair_exec && pair_uid == o->uid && pair_epoch_self == epoch && pair_epoch_other == o->epoch) return;
    if (pair_exec) {
      cudaGraphExecDestroy(pair_exec);
      pair_exec = nullptr;
    }
    cudaGraph_t g;
    ESD_CUDA(cudaGraphCreate(&g, 0));
    try {
      capture_refine_pair(g, o);
    } catch (...) {
      cudaGraphDestroy(g);
      throw;
    }
    cudaGraphExec_t e;
    cudaError_t err = cudaGraphInstantiate(&e, g, 0);
    cudaGraphDestroy(g);
    ESD_CUDA(err);
    pair_exec = e;
    pair_uid = o->uid;
    pair_epoch_self = epoch;
    pair_epoch_other = o->epoch;
  }

  // FP32 slice-major copies of W and AW for the inner solves (padding lanes and columns 0)
  void refresh_w32() {
    if (!fp32 || !have_W) return;
    const size_t entries = (size_t)A->nslices * kSlice * kMaxM;
    if (!W32.get()) {
      W32.alloc(sizeof(float) * entries);
      AW32.alloc(sizeof(float) * entries);
    }
    ESD_CUDA(cudaMemsetAsync(W32.get(), 0, W32.bytes(), stream));
    ESD_CUDA(cudaMemsetAsync(AW32.get(), 0, AW32.bytes(), stream));
    to_slice_major(A->n, A->rowpos.as<int>(), W.as<double>(), ld, M, W32.as<float>(), stream);
    to_slice_major(A->n, A->rowpos.as<int>(), AW.as<double>(), ld, M, AW32.as<float>(), stream);
  }
};

static int smallest_lmax(int m, int maxit) {
  if (m < 2) return 0;
  int l = 0;
  long long p = 1;
  while (p <= maxit) {
    p *= m;
    ++l;
  }
  return l;
}

#define ESD_API_BEGIN try {
#define ESD_API_END                  \
  }                                  \
  catch (const Error& e) {           \
    set_last_error(e.what());        \
    return e.code;                   \
  }                                  \
  catch (const std::exception& e) {  \
    set_last_error(e.what());        \
    return ESD_ERR_INVALID;          \
  }

// The refinement form of esd_solve (b and x already copied into vb / vx).
// The outer and refinement states of a refinement-form solve, set on the host and copied to
// the device on stream s.
static void refine_init(esd_solver* S, double tol, int32_t maxit, int32_t sample_m, cudaStream_t s) {
  State* h = S->hst;
  std::memset(h, 0, sizeof(State));
  h->scal0 = tol * tol;
  ESD_CUDA(cudaMemcpyAsync(S->state.get(), h, sizeof(State), cudaMemcpyHostToDevice, s));
  RefineState* hr = S->hrs;
  std::memset(hr, 0, sizeof(RefineState));
  hr->max_outer = S->prm.max_outer;
  hr->inner_maxit = maxit;
  hr->samp_m = sample_m;
  hr->lmax = S->prm.lmax > 0 ? S->prm.lmax : smallest_lmax(sample_m, maxit);
  hr->inner_tol2 = S->prm.inner_tol * S->prm.inner_tol;
  hr->keep = S->prm.resume_direction ? 1 : 0;
  ESD_CUDA(cudaMemcpyAsync(S->rstate.get(), hr, sizeof(RefineState), cudaMemcpyHostToDevice, s));
}

// After the graph: x to the caller, the refinement and inner states back to the host.
static void refine_fetch(esd_solver* S, double* x, cudaStream_t s) {
  copy_out(S->vx.get(), x, sizeof(double) * S->A->n, s);
  ESD_CUDA(cudaMemcpyAsync(S->hrs, S->rstate.get(), sizeof(RefineState), cudaMemcpyDeviceToHost, s));
  ESD_CUDA(cudaMemcpyAsync(S->hst_in, S->state_in.get(), sizeof(State), cudaMemcpyDeviceToHost, s));
}

// The solve's outcome from the fetched states (after the stream has synchronised).
static int refine_result(esd_solver* S, int32_t maxit, int32_t sample_m, int32_t* iters, double* relres,
                         const char* which) {
  const RefineState* hr = S->hrs;
  // coefficients of the whole resumed run, or of the last restarted inner solve
  S->last_iters = hr->outer > 0 ? S->hst_in->iter : 0;
  S->last_status = hr->status;
  S->last_sample_m = sample_m;
  S->last_maxit = maxit;
  S->last_outer = hr->outer;
  S->last_relres = hr->bb > 0.0 ? std::sqrt(hr->rr / hr->bb) : 0.0;
  S->last_true = S->last_relres;
  // slot_iter of the sampled (first) inner solve stays in the inner state
  std::memcpy(S->hst->slot_iter, S->hst_in->slot_iter, sizeof(S->hst->slot_iter));
  if (iters) *iters = hr->inner_total;
  if (relres) *relres = S->last_relres;
  if (hr->status == ESD_ERR_MAXIT) {
    set_last_error(std::string(which) +
                   (hr->stalled >= 4 ? "refinement stalled: the FP64 residual stopped decreasing above the tolerance"
                                     : "refinement did not reach the tolerance within max_outer steps or maxit"));
    return ESD_ERR_MAXIT;
  }
  if (hr->status == ESD_ERR_BREAKDOWN) {
    set_last_error(std::string(which) + (hr->nonfinite ? "non-finite residual in the refinement"
                                                       : "inner CG breakdown in the refinement"));
    return ESD_ERR_BREAKDOWN;
  }
  return ESD_OK;
}

static int solve_refine(esd_solver* S, double* x, double tol, int32_t maxit, int32_t sample_m, int32_t* iters,
                        double* relres) {
  cudaStream_t s = S->stream;
  refine_init(S, tol, maxit, sample_m, s);
  ESD_CUDA(cudaGraphLaunch(S->exec[S->mode], s));
  refine_fetch(S, x, s);
  ESD_CUDA(cudaStreamSynchronize(s));
  return refine_result(S, maxit, sample_m, iters, relres, "");
}

extern "C" {

void esd_params_default(esd_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->precond = ESD_PRECOND_IC0;
  p->maxit_cap = 20000;
  p->sample_cap = 32;
  p->lmax = 0;
  p->rank_tol = 1e-12;
  p->precision = ESD_FP64;
  p->inner_tol = 0.1;
  p->max_outer = 60;
  p->resume_direction = 1;
  p->sampling = ESD_SAMPLING_A;
}

int esd_solver_create(esd_matrix* A, const esd_params* params, esd_solver** out) {
  ESD_API_BEGIN
  ESD_CHECK(A && out, ESD_ERR_INVALID, "NULL argument");
  *out = nullptr;
  esd_params p;
  if (params) p = *params; else esd_params_default(&p);
  ESD_CHECK(p.precond == ESD_PRECOND_NONE || p.precond == ESD_PRECOND_IC0, ESD_ERR_INVALID, "bad precond");
  ESD_CHECK(p.maxit_cap >= 1, ESD_ERR_INVALID, "maxit_cap must be >= 1");
  ESD_CHECK(p.sample_cap >= 0 && p.sample_cap <= kMaxM, ESD_ERR_INVALID, "sample_cap must be 0..64");
  ESD_CHECK(p.precision == ESD_FP64 || p.precision == ESD_FP32_REFINE, ESD_ERR_INVALID, "unknown precision");
  ESD_CHECK(p.sampling == ESD_SAMPLING_A || p.sampling == ESD_SAMPLING_B, ESD_ERR_INVALID, "unknown sampling method");
  ESD_CHECK(p.sampling == ESD_SAMPLING_A || p.precision == ESD_FP64, ESD_ERR_INVALID,
            "sampling method B is defined on the FP64 solve's relative residual (use method A with refinement)");
  ESD_CHECK(p.precision == ESD_FP64 || (p.inner_tol > 0.0 && p.inner_tol < 1.0 && p.max_outer >= 1),
            ESD_ERR_INVALID, "refinement needs 0 < inner_tol < 1 and max_outer >= 1");
  ESD_CHECK(p.precond == ESD_PRECOND_NONE || A->factored, ESD_ERR_STATE, "IC(0) preconditioner needs esd_factor_ic0");
  std::unique_ptr<esd_solver> S(new esd_solver());
  S->A = A;
  S->prm = p;
  S->stream = A->stream;
  static std::atomic<unsigned long long> next_uid{1};
  S->uid = next_uid++;
  S->ld = A->vec_stride();
  const size_t vbytes = sizeof(double) * S->ld;
  for (DevBuf* b : {&S->vb, &S->vx, &S->vr, &S->vp, &S->vq, &S->vY}) {
    b->alloc(vbytes);
    ESD_CUDA(cudaMemsetAsync(b->get(), 0, vbytes, S->stream));
  }
  if (p.sample_cap > 0) {
    S->samples.alloc(vbytes * p.sample_cap);
    ESD_CUDA(cudaMemsetAsync(S->samples.get(), 0, S->samples.bytes(), S->stream));
  }
  S->ahist.alloc(sizeof(double) * p.maxit_cap);
  S->bhist.alloc(sizeof(double) * p.maxit_cap);
  S->state.alloc(sizeof(State));
  ESD_CUDA(cudaMemsetAsync(S->state.get(), 0, sizeof(State), S->stream));
  S->partials.alloc(sizeof(double) * (size_t)max_grid_blocks() * kMaxRed);
  S->rho_part.alloc(sizeof(double) * (size_t)max_grid_blocks() * std::max<size_t>(1, A->fwd_sets.size()));
  S->E.alloc(sizeof(double) * kMaxM * kMaxM);
  S->Einv.alloc(sizeof(double) * kMaxM * kMaxM);
  S->ritz.alloc(sizeof(double) * kMaxM);
  S->ext.alloc(sizeof(double) * 4);
  ESD_CUDA(cudaMallocHost(&S->hst, sizeof(State)));
  std::memset(S->hst, 0, sizeof(State));
  ESD_CUDA(cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking));
  ESD_CUDA(cudaStreamCreateWithFlags(&S->cap2, cudaStreamNonBlocking));
  ESD_CUDA(cudaStreamCreateWithFlags(&S->cap3, cudaStreamNonBlocking));
  if (p.precision == ESD_FP32_REFINE) S->enable_fp32();
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  *out = S.release();
  return ESD_OK;
  ESD_API_END
}

int esd_solver_destroy(esd_solver* S) {
  if (S) {
    cudaStreamSynchronize(S->stream);
    delete S;
  }
  return ESD_OK;
}

int esd_set_mode(esd_solver* S, int32_t mode) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  ESD_CHECK(mode == ESD_PLAIN || mode == ESD_DEFLATION || mode == ESD_SUBSPACE_CORRECTION, ESD_ERR_INVALID,
            "unknown mode");
  ESD_CHECK(mode == ESD_PLAIN || S->have_W, ESD_ERR_STATE, "deflation / subspace correction need W");
  S->mode = mode;
  return ESD_OK;
  ESD_API_END
}

int esd_solve(esd_solver* S, const double* b, double* x, double tol, int32_t maxit, int32_t sample_m,
              int32_t* iters, double* relres) {
  ESD_API_BEGIN
  ESD_CHECK(S && b && x, ESD_ERR_INVALID, "NULL argument");
  ESD_CHECK(tol > 0.0 && std::isfinite(tol), ESD_ERR_INVALID, "tol must be positive");
  ESD_CHECK(maxit >= 1 && maxit <= S->prm.maxit_cap, ESD_ERR_INVALID, "maxit must be 1..maxit_cap");
  ESD_CHECK(sample_m >= 0 && sample_m <= S->prm.sample_cap, ESD_ERR_INVALID, "sample_m must be 0..sample_cap");
  ESD_CHECK(sample_m == 0 || S->mode != ESD_DEFLATION, ESD_ERR_STATE,
            "sampling is defined on plain / subspace-correction iterates, not in deflation mode");
  ESD_CHECK(sample_m != 1 || S->prm.sampling == ESD_SAMPLING_B, ESD_ERR_INVALID, "sampling method A needs m >= 2");
  ESD_CHECK(S->prm.precond == ESD_PRECOND_NONE || S->PM()->factored, ESD_ERR_STATE,
            "the IC(0) factor is missing or stale (the matrix values changed): call esd_factor_ic0");
  ESD_CHECK(S->mode == ESD_PLAIN || S->w_values_version == S->A->values_version, ESD_ERR_STATE,
            "the matrix values changed after W was built: call esd_refresh_W");
  ESD_CHECK(!S->pw_on || S->mode != ESD_DEFLATION, ESD_ERR_STATE,
            "the power method runs in plain or subspace-correction solves (esd_power_start(S, NULL) stops it)");
  cudaStream_t s = S->stream;
  const int n = S->A->n;
  if (S->fp32) {
    S->A->ensure_fp32();
    if (S->P) S->P->ensure_fp32();
  }
  S->build_graph(S->mode);
  copy_in(b, S->vb.get(), sizeof(double) * n, s);
  copy_in(x, S->vx.get(), sizeof(double) * n, s);
  if (S->fp32) return solve_refine(S, x, tol, maxit, sample_m, iters, relres);
  State* h = S->hst;
  std::memset(h, 0, sizeof(State));
  h->scal0 = tol * tol;
  h->maxit = maxit;
  h->samp_m = sample_m;
  h->lmax = S->prm.lmax > 0 ? S->prm.lmax : smallest_lmax(sample_m, maxit);
  h->h = 1;
  h->pend_slot = -1;
  h->samp_method = S->prm.sampling;
  ESD_CUDA(cudaMemcpyAsync(S->state.get(), h, sizeof(State), cudaMemcpyHostToDevice, s));
  ESD_CUDA(cudaGraphLaunch(S->exec[S->mode], s));
  copy_out(S->vx.get(), x, sizeof(double) * n, s);
  ESD_CUDA(cudaMemcpyAsync(h, S->state.get(), sizeof(State), cudaMemcpyDeviceToHost, s));
  ESD_CUDA(cudaStreamSynchronize(s));
  S->last_iters = h->iter;
  S->last_status = h->status;
  S->last_sample_m = sample_m;
  S->last_maxit = maxit;
  S->last_relres = h->bb > 0.0 ? std::sqrt(h->rr / h->bb) : 0.0;
  S->last_true = h->bb > 0.0 ? std::sqrt(h->true_rr / h->bb) : 0.0;
  if (iters) *iters = h->iter;
  if (relres) *relres = S->last_relres;
  if (h->status == ESD_ERR_MAXIT) {
    set_last_error("tolerance not reached within maxit iterations");
    return ESD_ERR_MAXIT;
  }
  if (h->status == ESD_ERR_INTERNAL) {
    set_last_error("internal loop guard stopped the solve");
    return ESD_ERR_INTERNAL;
  }
  if (h->status == ESD_ERR_BREAKDOWN) {
    set_last_error("CG breakdown: (p, Ap) or (r, z) not positive");
    return ESD_ERR_BREAKDOWN;
  }
  return ESD_OK;
  ESD_API_END
}

}  // extern "C"

// What esd_solve_pair and esd_profile_pair_iterations ask of a pair (throws when it fails);
// the FP32 copies of the matrix and its factor are brought up to date.
static void check_pair(esd_solver* S1, esd_solver* S2) {
  ESD_CHECK(S1 != S2, ESD_ERR_INVALID, "a pair needs two solvers");
  ESD_CHECK(S1->A == S2->A && S1->P == S2->P, ESD_ERR_INVALID,
            "the two solvers must share the matrix and the preconditioning matrix");
  ESD_CHECK(S1->fp32 && S2->fp32, ESD_ERR_STATE, "the pair solve runs in the refinement form (ESD_FP32_REFINE)");
  ESD_CHECK(S1->mode == ESD_PLAIN && S2->mode == ESD_PLAIN, ESD_ERR_STATE, "the pair solve runs plain PCG");
  ESD_CHECK(S1->prm.precond == ESD_PRECOND_IC0 && S2->prm.precond == ESD_PRECOND_IC0, ESD_ERR_STATE,
            "the pair solve runs with IC(0)");
  ESD_CHECK(S1->PM()->factored, ESD_ERR_STATE,
            "the IC(0) factor is missing or stale (the matrix values changed): call esd_factor_ic0");
  ESD_CHECK(!S1->pw_on && !S2->pw_on, ESD_ERR_STATE, "the power method runs in FP64 solves");
  S1->A->ensure_fp32();
  if (S1->P) S1->P->ensure_fp32();
  S1->ensure_pair_vectors();
  const std::string why = pair_unsupported(S1->pair_ctx32(S1), S2->pair_ctx32(S1));
  ESD_CHECK(why.empty(), ESD_ERR_STATE, "pair solve: " + why);
}

extern "C" {

int esd_solve_pair(esd_solver* S1, esd_solver* S2, const double* b1, double* x1, const double* b2, double* x2,
                   double tol, int32_t maxit, int32_t* iters1, double* relres1, int32_t* iters2, double* relres2,
                   int32_t* paired) {
  ESD_API_BEGIN
  ESD_CHECK(S1 && S2 && b1 && x1 && b2 && x2, ESD_ERR_INVALID, "NULL argument");
  ESD_CHECK(tol > 0.0 && std::isfinite(tol), ESD_ERR_INVALID, "tol must be positive");
  ESD_CHECK(maxit >= 1 && maxit <= S1->prm.maxit_cap && maxit <= S2->prm.maxit_cap, ESD_ERR_INVALID,
            "maxit must be 1..maxit_cap of both solvers");
  check_pair(S1, S2);
  cudaStream_t s = S1->stream;  // one matrix, one stream
  S1->build_pair_graph(S2);
  const int n = S1->A->n;
  copy_in(b1, S1->vb.get(), sizeof(double) * n, s);
  copy_in(x1, S1->vx.get(), sizeof(double) * n, s);
  copy_in(b2, S2->vb.get(), sizeof(double) * n, s);
  copy_in(x2, S2->vx.get(), sizeof(double) * n, s);
  refine_init(S1, tol, maxit, 0, s);
  refine_init(S2, tol, maxit, 0, s);
  ESD_CUDA(cudaMemsetAsync(&S1->state_in.as<State>()->paired, 0, sizeof(int), s));
  ESD_CUDA(cudaGraphLaunch(S1->pair_exec, s));
  refine_fetch(S1, x1, s);
  refine_fetch(S2, x2, s);
  ESD_CUDA(cudaStreamSynchronize(s));
  if (paired) *paired = S1->hst_in->paired;
  const int r1 = refine_result(S1, maxit, 0, iters1, relres1, "system 1: ");
  const std::string e1 = esd_last_error();
  const int r2 = refine_result(S2, maxit, 0, iters2, relres2, "system 2: ");
  if (r1 != ESD_OK) {
    set_last_error(e1);
    return r1;
  }
  return r2;
  ESD_API_END
}

int esd_true_relres(esd_solver* S, double* relres) {
  if (!S || !relres) { set_last_error("NULL argument"); return ESD_ERR_INVALID; }
  *relres = S->last_true;
  return ESD_OK;
}

static void install_W(esd_solver* S, const double* X, int m, bool orth, double theta) {
  const size_t ld = S->ld;
  S->aux.ensure(S->A->n, ld);
  const int mpad_max = kMaxM;
  if (!S->W.get()) {
    S->W.alloc(sizeof(double) * ld * mpad_max);
    S->AW.alloc(sizeof(double) * ld * mpad_max);
  }
  int mbar = 0;
  const int mkeep = build_aux(S->A, S->aux, X, m, orth, S->prm.rank_tol, theta, S->W.as<double>(),
                              S->AW.as<double>(), S->E.as<double>(), S->Einv.as<double>(),
                              S->ritz.as<double>(), &mbar, S->stream);
  if (S->fp32) {
    // The inner solves see W rounded to FP32. AW, E and E^-1 are formed again (in FP64) for
    // exactly that W, so that the FP64 coarse solve and the FP32 projection describe the
    // same subspace; otherwise E^-1 is off by eps32 * cond(E) for the FP32 W.
    round_to_f32((long long)ld * mkeep, S->W.as<double>(), S->aux.work1.as<double>(), S->stream);
    int unused = 0;
    build_aux(S->A, S->aux, S->aux.work1.as<double>(), mkeep, false, S->prm.rank_tol,
              std::numeric_limits<double>::infinity(), S->W.as<double>(), S->AW.as<double>(),
              S->E.as<double>(), S->Einv.as<double>(), S->ritz.as<double>(), &unused, S->stream);
  }
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  S->m = mkeep;
  S->M = pad_cols(mkeep);
  S->mbar = mbar;
  S->have_W = true;
  S->w_version++;
  S->w_values_version = S->A->values_version;
  S->refresh_df();
  S->refresh_w32();
  ESD_CUDA(cudaStreamSynchronize(S->stream));
}

int esd_sample_and_build_W(esd_solver* S, double theta, int32_t* m_kept) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  ESD_CHECK(S->last_sample_m > 0, ESD_ERR_STATE, "the last solve did not sample iterates");
  ESD_CHECK(!(theta <= 0.0), ESD_ERR_INVALID, "theta must be positive (or +inf)");
  std::vector<int> slots;
  for (int k = 0; k < S->last_sample_m; ++k)
    if (S->hst->slot_iter[k] > 0) slots.push_back(k);
  ESD_CHECK(!slots.empty(), ESD_ERR_RANK, "no iterate was sampled (the solve stopped too early)");
  const int m = (int)slots.size();
  S->aux.ensure(S->A->n, S->ld);
  DevBuf dslots(sizeof(int) * m);
  ESD_CUDA(cudaMemcpyAsync(dslots.get(), slots.data(), sizeof(int) * m, cudaMemcpyHostToDevice, S->stream));
  // (the refinement form stores FP64 iterates too: its FP64 base plus the inner iterate)
  k_errors<<<max_grid_blocks(), kBlock, 0, S->stream>>>(S->A->n, S->vx.as<double>(), S->samples.as<double>(),
                                                        S->ld, dslots.as<int>(), m, S->aux.work1.as<double>());
  ESD_CUDA(cudaGetLastError());
  install_W(S, S->aux.work1.as<double>(), m, true, theta);
  if (m_kept) *m_kept = S->m;
  return ESD_OK;
  ESD_API_END
}

int esd_set_W(esd_solver* S, const double* W, int32_t m) {
  ESD_API_BEGIN
  ESD_CHECK(S && W, ESD_ERR_INVALID, "NULL argument");
  ESD_CHECK(m >= 1 && m <= kMaxM, ESD_ERR_INVALID, "m must be 1..64");
  S->aux.ensure(S->A->n, S->ld);
  const int n = S->A->n;
  for (int j = 0; j < m; ++j)
    copy_in(W + (size_t)j * n, S->aux.work1.as<double>() + (size_t)j * S->ld, sizeof(double) * n, S->stream);
  install_W(S, S->aux.work1.as<double>(), m, false, std::numeric_limits<double>::infinity());
  return ESD_OK;
  ESD_API_END
}

int esd_solver_set_precond_matrix(esd_solver* S, esd_matrix* P) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  if (P) {
    ESD_CHECK(P->n == S->A->n && P->cp == S->A->cp, ESD_ERR_INVALID,
              "the preconditioning matrix needs the rows and colours of A (same n and colour_ptr)");
    ESD_CHECK(P->factored, ESD_ERR_STATE, "the preconditioning matrix has no IC(0) factor (esd_factor_ic0)");
  }
  const esd_matrix* PM = P ? P : S->A;
  const size_t need = sizeof(double) * (size_t)max_grid_blocks() * std::max<size_t>(1, PM->fwd_sets.size());
  if (S->rho_part.bytes() < need) S->rho_part.alloc(need);
  S->P = (P == S->A) ? nullptr : P;
  if (S->fp32 && S->P) S->P->ensure_fp32();
  S->drop_graphs();
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  return ESD_OK;
  ESD_API_END
}

int esd_set_precision(esd_solver* S, int32_t precision, double inner_tol) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  ESD_CHECK(precision == ESD_FP64 || precision == ESD_FP32_REFINE, ESD_ERR_INVALID, "unknown precision");
  if (precision == ESD_FP64) {
    if (S->fp32) S->drop_graphs();
    S->fp32 = false;
    S->prm.precision = ESD_FP64;
    S->refresh_df();  // the double-float copies of AW and W the FP64 iteration reads
    return ESD_OK;
  }
  ESD_CHECK(inner_tol > 0.0 && inner_tol < 1.0, ESD_ERR_INVALID, "refinement needs 0 < inner_tol < 1");
  ESD_CHECK(S->prm.sampling == ESD_SAMPLING_A, ESD_ERR_INVALID,
            "sampling method B is defined on the FP64 solve's relative residual");
  ESD_CHECK(!S->pw_on, ESD_ERR_STATE, "the power method runs in FP64 solves (esd_power_start(S, NULL) stops it)");
  const bool was_fp32 = S->fp32;
  S->prm.precision = ESD_FP32_REFINE;
  S->prm.inner_tol = inner_tol;
  if (was_fp32) return ESD_OK;
  S->drop_graphs();
  S->enable_fp32();
  if (S->have_W) {
    // the inner solves need W rounded to FP32 with AW, E, E^-1 formed for it (as esd_set_W)
    S->aux.ensure(S->A->n, S->ld);
    ESD_CUDA(cudaMemcpyAsync(S->aux.work1.get(), S->W.get(), sizeof(double) * S->ld * S->m, cudaMemcpyDeviceToDevice,
                             S->stream));
    const int mbar = S->mbar;
    install_W(S, S->aux.work1.as<double>(), S->m, false, std::numeric_limits<double>::infinity());
    S->mbar = mbar;
  }
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  return ESD_OK;
  ESD_API_END
}

int esd_refresh_W(esd_solver* S) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  ESD_CHECK(S->have_W, ESD_ERR_STATE, "no W");
  S->aux.ensure(S->A->n, S->ld);
  ESD_CUDA(cudaMemcpyAsync(S->aux.work1.get(), S->W.get(), sizeof(double) * S->ld * S->m, cudaMemcpyDeviceToDevice,
                           S->stream));
  const int mbar = S->mbar;
  install_W(S, S->aux.work1.as<double>(), S->m, false, std::numeric_limits<double>::infinity());
  S->mbar = mbar;
  return ESD_OK;
  ESD_API_END
}

int esd_get_W(esd_solver* S, double* W, double* AW, double* E, int32_t* m) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  ESD_CHECK(S->have_W, ESD_ERR_STATE, "no W");
  const int n = S->A->n;
  for (int j = 0; j < S->m; ++j) {
    if (W) copy_out(S->W.as<double>() + (size_t)j * S->ld, W + (size_t)j * n, sizeof(double) * n, S->stream);
    if (AW) copy_out(S->AW.as<double>() + (size_t)j * S->ld, AW + (size_t)j * n, sizeof(double) * n, S->stream);
  }
  if (E) copy_out(S->E.get(), E, sizeof(double) * S->m * S->m, S->stream);
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  if (m) *m = S->m;
  return ESD_OK;
  ESD_API_END
}

int esd_ritz_values(esd_solver* S, double* out, int32_t cap, int32_t* count) {
  ESD_API_BEGIN
  ESD_CHECK(S && out, ESD_ERR_INVALID, "NULL argument");
  ESD_CHECK(S->have_W, ESD_ERR_STATE, "no W");
  const int k = std::min<int>(cap, S->m);
  ESD_CUDA(cudaMemcpyAsync(out, S->ritz.get(), sizeof(double) * k, cudaMemcpyDeviceToHost, S->stream));
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  if (count) *count = S->m;
  return ESD_OK;
  ESD_API_END
}

int esd_power_start(esd_solver* S, const double* v0) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  if (!v0) {
    S->pw_on = false;
    return ESD_OK;
  }
  ESD_CHECK(!S->fp32, ESD_ERR_STATE, "the power method runs in FP64 solves");
  cudaStream_t s = S->stream;
  const size_t ld = S->ld;
  if (!S->pw_v.get()) {
    S->pw_v.alloc(sizeof(double) * 2 * ld);
    ESD_CUDA(cudaMemsetAsync(S->pw_v.get(), 0, S->pw_v.bytes(), s));  // sentinels (index n) stay 0
    S->pw_state.alloc(sizeof(PowerState));
  }
  S->pw_on = false;
  ESD_CUDA(cudaMemsetAsync(S->pw_state.get(), 0, sizeof(PowerState), s));
  copy_in(v0, S->pw_v.get(), sizeof(double) * S->A->n, s);
  double* const pw[2] = {S->pw_v.as<double>(), S->pw_v.as<double>() + ld};
  launch_power_rq(S->A, pw, S->pw_state.as<PowerState>(), S->partials.as<double>(), 1, s);
  PowerState h;
  ESD_CUDA(cudaMemcpyAsync(&h, S->pw_state.get(), sizeof(PowerState), cudaMemcpyDeviceToHost, s));
  ESD_CUDA(cudaStreamSynchronize(s));
  ESD_CHECK(!h.failed, ESD_ERR_INVALID, "the start vector is zero or not finite");
  S->pw_on = true;
  return ESD_OK;
  ESD_API_END
}

int esd_power_estimate(esd_solver* S, double* lmax, int32_t* steps, double* v) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  ESD_CHECK(S->pw_on, ESD_ERR_STATE, "the power method was not started (esd_power_start)");
  cudaStream_t s = S->stream;
  const size_t ld = S->ld;
  double* const pw[2] = {S->pw_v.as<double>(), S->pw_v.as<double>() + ld};
  PowerState* ps = S->pw_state.as<PowerState>();
  launch_power_rq(S->A, pw, ps, S->partials.as<double>(), 0, s);
  PowerState h;
  ESD_CUDA(cudaMemcpyAsync(&h, ps, sizeof(PowerState), cudaMemcpyDeviceToHost, s));
  ESD_CUDA(cudaStreamSynchronize(s));
  ESD_CHECK(!h.failed && h.ww > 0.0 && std::isfinite(h.ww), ESD_ERR_BREAKDOWN,
            "the power vector vanished or overflowed");
  if (lmax) *lmax = h.wAw / h.ww;
  if (steps) *steps = h.steps;
  if (v) {
    // the buffer the next product writes is free until then
    double* unit = pw[(h.steps + 1) & 1];
    launch_power_unit(S->A, pw[h.steps & 1], ps, unit, s);
    copy_out(unit, v, sizeof(double) * S->A->n, s);
    ESD_CUDA(cudaStreamSynchronize(s));
  }
  return ESD_OK;
  ESD_API_END
}

int esd_paper_cond_estimate(esd_solver* S, double* lmax, double* lmin, double* kappa) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  ESD_CHECK(S->have_W, ESD_ERR_STATE, "no W: the smallest Ritz value needs the sampled basis");
  double lx = 0.0;
  const int rc = esd_power_estimate(S, &lx, nullptr, nullptr);
  if (rc != ESD_OK) return rc;
  double r0 = 0.0;
  ESD_CUDA(cudaMemcpyAsync(&r0, S->ritz.get(), sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  ESD_CHECK(r0 > 0.0, ESD_ERR_CHOL_E, "the smallest Ritz value is not positive");
  if (lmax) *lmax = lx;
  if (lmin) *lmin = r0;
  if (kappa) *kappa = lx / r0;
  return ESD_OK;
  ESD_API_END
}

int esd_estimate_cond(esd_solver* S, double* lmin, double* lmax, double* kappa, double* ritz_min) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  ESD_CHECK(S->last_iters >= 1, ESD_ERR_STATE, "the last solve took no CG step");
  if (S->lz.bytes() < sizeof(double) * 2 * (size_t)S->prm.maxit_cap) S->lz.alloc(sizeof(double) * 2 * S->prm.maxit_cap);
  launch_lanczos_extremes(S->ahist.as<double>(), S->bhist.as<double>(), S->last_iters, S->lz.as<double>(),
                          (size_t)S->prm.maxit_cap, S->ext.as<double>(), S->stream);
  double h[2];
  ESD_CUDA(cudaMemcpyAsync(h, S->ext.get(), sizeof(h), cudaMemcpyDeviceToHost, S->stream));
  double r0 = std::numeric_limits<double>::quiet_NaN();
  if (S->have_W) ESD_CUDA(cudaMemcpyAsync(&r0, S->ritz.get(), sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  if (lmin) *lmin = h[0];
  if (lmax) *lmax = h[1];
  if (kappa) *kappa = h[1] / h[0];
  if (ritz_min) *ritz_min = r0;
  return ESD_OK;
  ESD_API_END
}

int esd_get_history(esd_solver* S, double* alpha, double* beta, int32_t cap, int32_t* count) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  const int k = std::min<int>(cap, S->last_iters);
  if (alpha && k > 0)
    ESD_CUDA(cudaMemcpyAsync(alpha, S->ahist.get(), sizeof(double) * k, cudaMemcpyDeviceToHost, S->stream));
  if (beta && k > 1)
    ESD_CUDA(cudaMemcpyAsync(beta, S->bhist.get(), sizeof(double) * (k - 1), cudaMemcpyDeviceToHost, S->stream));
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  if (count) *count = S->last_iters;
  return ESD_OK;
  ESD_API_END
}

int esd_get_samples(esd_solver* S, double* samples, int32_t* slot_iter, int32_t cap, int32_t* m) {
  ESD_API_BEGIN
  ESD_CHECK(S, ESD_ERR_INVALID, "NULL solver");
  const int k = std::min<int>(cap, S->last_sample_m);
  const int n = S->A->n;
  for (int j = 0; j < k; ++j) {
    if (slot_iter) slot_iter[j] = S->hst->slot_iter[j];
    if (samples)
      copy_out(S->samples.as<double>() + (size_t)j * S->ld, samples + (size_t)j * n, sizeof(double) * n, S->stream);
  }
  ESD_CUDA(cudaStreamSynchronize(S->stream));
  if (m) *m = S->last_sample_m;
  return ESD_OK;
  ESD_API_END
}

int esd_backward_euler_rhs(esd_solver* S, const double* x_prev, const double* s, double inv_dt, double* b) {
  ESD_API_BEGIN
  ESD_CHECK(S && x_prev && s && b, ESD_ERR_INVALID, "NULL argument");
  const int n = S->A->n;
  cudaStream_t st = S->stream;
  const bool dev = is_device_ptr(x_prev) && is_device_ptr(s) && is_device_ptr(b);
  if (dev) {
    launch_axpby(n, x_prev, inv_dt, s, b, st);
  } else {
    double* t0 = S->A->tmp.as<double>();
    double* t1 = t0 + S->ld;
    double* t2 = t1 + S->ld;
    copy_in(x_prev, t0, sizeof(double) * n, st);
    copy_in(s, t1, sizeof(double) * n, st);
    launch_axpby(n, t0, inv_dt, t1, t2, st);
    copy_out(t2, b, sizeof(double) * n, st);
    ESD_CUDA(cudaStreamSynchronize(st));
  }
  return ESD_OK;
  ESD_API_END
}

int esd_profile_iterations(esd_solver* S, const double* b, double* x, int32_t reps, double* ms, char* names,
                           int32_t cap, int32_t* count) {
  ESD_API_BEGIN
  ESD_CHECK(S && b && x && ms && count, ESD_ERR_INVALID, "NULL argument");
  ESD_CHECK(reps >= 1 && reps < S->prm.maxit_cap, ESD_ERR_INVALID, "reps must be 1..maxit_cap-1");
  cudaStream_t s = S->stream;
  const int n = S->A->n;
  copy_in(b, S->vb.get(), sizeof(double) * n, s);
  copy_in(x, S->vx.get(), sizeof(double) * n, s);
  State* h = S->hst;
  std::memset(h, 0, sizeof(State));
  h->scal0 = 0.0;  // tolerance 0: the iterations run for reps steps
  h->maxit = reps + 1;
  h->h = 1;
  h->pend_slot = -1;
  ESD_CUDA(cudaMemcpyAsync(S->state.get(), h, sizeof(State), cudaMemcpyHostToDevice, s));
  std::vector<std::unique_ptr<KernelMarks>> marks;
  if (S->fp32) {
    // the FP32 inner iteration on the system A d = b
    S->A->ensure_fp32();
    ESD_CUDA(cudaMemcpyAsync(S->state_in.get(), h, sizeof(State), cudaMemcpyHostToDevice, s));
    // r0 = b - A x0 from an FP32 copy of x0; the iterations then update the FP64 x
    convert_d2f(n, S->vb.as<double>(), S->b32.as<float>(), s);
    convert_d2f(n, S->vx.as<double>(), S->x32.as<float>(), s);
    IterCtx<float> c = S->ctx32(S->mode);
    launch_init<float>(c, s);
    for (int r = 0; r < reps; ++r) {
      marks.emplace_back(new KernelMarks());
      launch_iteration<float>(c, s, marks.back().get());
    }
  } else {
    IterCtx<double> c = S->ctx(S->mode);
    launch_init<double>(c, s);
    for (int r = 0; r < reps; ++r) {
      marks.emplace_back(new KernelMarks());
      launch_iteration<double>(c, s, marks.back().get());
    }
  }
  copy_out(S->vx.get(), x, sizeof(double) * n, s);
  ESD_CUDA(cudaStreamSynchronize(s));
  const int k = (int)marks[0]->ev.size() - 1;
  *count = k;
  for (int j = 0; j < std::min(k, (int)cap); ++j) {
    double tot = 0.0;
    for (auto& mk : marks) {
      float t = 0.f;
      ESD_CUDA(cudaEventElapsedTime(&t, mk->ev[j], mk->ev[j + 1]));
      tot += t;
    }
    ms[j] = tot / reps;
    if (names) {
      std::strncpy(names + 32 * j, marks[0]->names[j + 1].c_str(), 31);
      names[32 * j + 31] = 0;
    }
  }
  return ESD_OK;
  ESD_API_END
}

int esd_profile_pair_iterations(esd_solver* S1, esd_solver* S2, const double* b1, double* x1, const double* b2,
                                double* x2, int32_t reps, double* ms, char* names, int32_t cap, int32_t* count) {
  ESD_API_BEGIN
  ESD_CHECK(S1 && S2 && b1 && x1 && b2 && x2 && ms && count, ESD_ERR_INVALID, "NULL argument");
  ESD_CHECK(reps >= 1 && reps < S1->prm.maxit_cap && reps < S2->prm.maxit_cap, ESD_ERR_INVALID,
            "reps must be 1..maxit_cap-1 of both solvers");
  check_pair(S1, S2);
  cudaStream_t s = S1->stream;
  const int n = S1->A->n;
  esd_solver* sv[2] = {S1, S2};
  const double* bs[2] = {b1, b2};
  const double* xs[2] = {x1, x2};
  IterCtx<float> c[2];
  for (int k = 0; k < 2; ++k) {
    esd_solver* S = sv[k];
    copy_in(bs[k], S->vb.get(), sizeof(double) * n, s);
    copy_in(xs[k], S->vx.get(), sizeof(double) * n, s);
    State* h = S->hst;
    std::memset(h, 0, sizeof(State));
    h->scal0 = 0.0;  // tolerance 0: the iterations run for reps steps
    h->maxit = reps + 1;
    h->h = 1;
    h->pend_slot = -1;
    ESD_CUDA(cudaMemcpyAsync(S->state_in.get(), h, sizeof(State), cudaMemcpyHostToDevice, s));
    convert_d2f(n, S->vb.as<double>(), S->b32.as<float>(), s);
    convert_d2f(n, S->vx.as<double>(), S->x32.as<float>(), s);
    c[k] = S->pair_ctx32(S1);
    launch_init<float>(c[k], s);
  }
  launch_pair_pack(c[0], c[1], true, s);
  std::vector<std::unique_ptr<KernelMarks>> marks;
  for (int r = 0; r < reps; ++r) {
    marks.emplace_back(new KernelMarks());
    launch_iteration_pair(c[0], c[1], 0ull, s, marks.back().get());
  }
  copy_out(S1->vx.get(), x1, sizeof(double) * n, s);
  copy_out(S2->vx.get(), x2, sizeof(double) * n, s);
  ESD_CUDA(cudaStreamSynchronize(s));
  const int k = (int)marks[0]->ev.size() - 1;
  *count = k;
  for (int j = 0; j < std::min(k, (int)cap); ++j) {
    double tot = 0.0;
    for (auto& mk : marks) {
      float t = 0.f;
      ESD_CUDA(cudaEventElapsedTime(&t, mk->ev[j], mk->ev[j + 1]));
      tot += t;
    }
    ms[j] = tot / reps;
    if (names) {
      std::strncpy(names + 32 * j, marks[0]->names[j + 1].c_str(), 31);
      names[32 * j + 31] = 0;
    }
  }
  return ESD_OK;
  ESD_API_END
}

int esd_last_solve_info(esd_solver* S, int32_t* iters, int32_t* outer_steps, int32_t* first_inner,
                        int32_t* restarts, double* max_gap, double* true_relres, int32_t* status) {
  if (!S) { set_last_error("NULL solver"); return ESD_ERR_INVALID; }
  if (iters) *iters = S->fp32 ? S->hrs->inner_total : S->last_iters;
  if (outer_steps) *outer_steps = S->fp32 ? S->last_outer : 0;
  if (first_inner) *first_inner = S->fp32 ? S->hrs->first_inner : S->last_iters;
  if (restarts) *restarts = S->fp32 ? S->hrs->restarts : 0;
  if (max_gap) *max_gap = S->fp32 ? S->hrs->max_gap : 0.0;
  if (true_relres) *true_relres = S->last_true;
  if (status) *status = S->last_status;
  return ESD_OK;
}

int esd_pattern_grad(esd_matrix* A, const double* lambda, const double* x, double* grad) {
  ESD_API_BEGIN
  ESD_CHECK(A && lambda && x && grad, ESD_ERR_INVALID, "NULL argument");
  cudaStream_t s = A->stream;
  double* t0 = A->tmp.as<double>();
  double* t1 = t0 + A->vec_stride();
  copy_in(lambda, t0, sizeof(double) * A->n, s);
  copy_in(x, t1, sizeof(double) * A->n, s);
  const bool dev = is_device_ptr(grad);
  DevBuf tmp;
  double* g = grad;
  if (!dev) {
    tmp.alloc(sizeof(double) * A->nnz);
    g = tmp.as<double>();
  }
  k_pattern_grad<<<max_grid_blocks(), kBlock, 0, s>>>(A->n, A->csr_rowptr.as<int>(), A->csr_colind.as<int>(), t0,
                                                      t1, g);
  ESD_CUDA(cudaGetLastError());
  if (!dev) copy_out(g, grad, sizeof(double) * A->nnz, s);
  ESD_CUDA(cudaStreamSynchronize(s));
  return ESD_OK;
  ESD_API_END
}

}  // extern "C"
