// CryptoInvSqrt as a CUDA graph: the whole launch sequence of one configuration
// (input level, batch, scale and InvSqrt parameters fixed) is captured once and
// replayed with a single launch, removing the per-kernel launch overhead that
// dominates small batches.  Capture needs every lazily built table (level
// constants, switching keys, bootstrapping diagonals) to exist already, so the
// graph is built after one ordinary run of the same configuration; the
// intermediates are allocated and freed inside the graph (stream-ordered memory
// nodes), the result is copied into a buffer the graph object owns.
#include "internal.cuh"
#include "profiler.cuh"

struct hedap_graph {
  hedap::Ctx* C = nullptr;
  std::unique_ptr<hedap::Ct> in, out;               // one (batched) CryptoInvSqrt
  std::vector<std::unique_ptr<hedap::Ct>> ins, outs;  // many single ciphertexts (hedap_invsqrt_mixed)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
  ~hedap_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

namespace {

using namespace hedap;

void copy_ct(Ctx& C, const Ct& src, Ct& dst) {
  HEDAP_CUDA(cudaMemcpy2DAsync(dst.part(0), dst.part_stride() * 8, src.part(0), src.part_stride() * 8,
                               (size_t)(src.level + 1) * C.N * 8, src.parts(), cudaMemcpyDeviceToDevice, C.stream));
}

template <class F>
hedap_status graph_guard(F&& f) {
  try {
    f();
    return HEDAP_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc& e) {
    set_last_error(e.what());
    return HEDAP_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return HEDAP_ERR_ARG;
  }
}

// Capture `work` (issued on the context's stream) into G's graph and instantiate it: the context's stream is
// swapped for a fresh capturing stream meanwhile; G->kernels counts the launches captured.  The caller holds
// the context's lock and has run the same work once already (every lazily built table exists).
template <class F>
void capture(Ctx& C, hedap_graph& G, F&& work) {
  HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  cudaStream_t cs, old = C.stream;
  HEDAP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const uint64_t k0 = prof_launches();
  C.stream = cs;
  cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  std::string failure;
  if (ce == cudaSuccess) {
    try {
      work();
    } catch (const std::exception& e) {
      failure = e.what();
    }
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(cs, &g);
    G.graph = g;
  }
  C.stream = old;
  cudaStreamDestroy(cs);
  if (!failure.empty()) throw Error(HEDAP_ERR_CUDA, "graph capture: " + failure);
  if (ce != cudaSuccess) throw Error(HEDAP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  G.kernels = prof_launches() - k0;
  HEDAP_CUDA(cudaGraphInstantiate(&G.exec, G.graph, 0));
}

}  // namespace

#define API extern "C" __attribute__((visibility("default")))

API hedap_status hedap_invsqrt_graph_create(hedap_ctx* ctx, const hedap_ct* example, const hedap_invsqrt_cfg* cfg,
                                            hedap_graph** out) {
  return graph_guard([&] {
    if (!ctx || !example || !cfg || !out) throw Error(HEDAP_ERR_ARG, "null argument");
    *out = nullptr;
    if (prof_enabled()) throw Error(HEDAP_ERR_ARG, "graph capture with profiling enabled");
    Ctx& C = ctx_of(ctx);
    std::lock_guard<std::mutex> lk(C.mu);
    const Ct& ex = ct_of(ctx, example);
    std::unique_ptr<hedap_graph> G(new hedap_graph);
    G->C = &C;
    G->in = ct_copy(C, ex, ex.level);
    {  // ordinary run: builds every table the sequence needs, fixes the output shape
      auto w = invsqrt(C, *G->in, *cfg);
      G->out = ct_alloc(C, w->level, w->batch);
      G->out->scale = w->scale;
    }
    capture(C, *G, [&] { copy_ct(C, *invsqrt(C, *G->in, *cfg), *G->out); });
    *out = G.release();
  });
}

API hedap_status hedap_graph_run(hedap_graph* g, const hedap_ct* in, hedap_ct** out) {
  return graph_guard([&] {
    if (!g || !g->in) throw Error(HEDAP_ERR_ARG, "not a graph of one (batched) ciphertext");
    Ctx& C = *g->C;
    std::lock_guard<std::mutex> lk(C.mu);
    if (in) {
      const Ct& a = ct_of(nullptr, in);
      if (a.owner != &C) throw Error(HEDAP_ERR_ARG, "graph input made by another context");
      if (a.level != g->in->level || a.batch != g->in->batch || a.scale != g->in->scale)
        throw Error(HEDAP_ERR_ARG, "graph input must match the captured level, batch and scale");
      copy_ct(C, a, *g->in);
    }
    HEDAP_CUDA(cudaGraphLaunch(g->exec, C.stream));
    if (out) {
      *out = nullptr;
      auto r = ct_alloc(C, g->out->level, g->out->batch);
      r->scale = g->out->scale;
      copy_ct(C, *g->out, *r);
      *out = new hedap_ct;
      (*out)->c = std::move(r);
    }
  });
}

// CryptoInvSqrt of many single ciphertexts at their own levels (hedap_invsqrt_mixed) as one graph
API hedap_status hedap_invsqrt_mixed_graph_create(hedap_ctx* ctx, const hedap_ct* const* examples,
                                                  const hedap_invsqrt_cfg* cfgs, size_t n, hedap_graph** out) {
  return graph_guard([&] {
    if (!ctx || !examples || !cfgs || !out || n == 0) throw Error(HEDAP_ERR_ARG, "bad argument");
    *out = nullptr;
    if (prof_enabled()) throw Error(HEDAP_ERR_ARG, "graph capture with profiling enabled");
    Ctx& C = ctx_of(ctx);
    std::lock_guard<std::mutex> lk(C.mu);
    std::unique_ptr<hedap_graph> G(new hedap_graph);
    G->C = &C;
    const std::vector<hedap_invsqrt_cfg> cv(cfgs, cfgs + n);
    std::vector<const Ct*> in;
    for (size_t i = 0; i < n; ++i) {
      const Ct& e = ct_of(ctx, examples[i]);
      G->ins.push_back(ct_copy(C, e, e.level));
      in.push_back(G->ins.back().get());
    }
    {  // ordinary run: builds every table the sequence needs, fixes the outputs' shapes
      auto w = invsqrt_mixed(C, in, cv);
      for (auto& r : w) {
        G->outs.push_back(ct_alloc(C, r->level, r->batch));
        G->outs.back()->scale = r->scale;
      }
    }
    capture(C, *G, [&] {
      auto r = invsqrt_mixed(C, in, cv);
      for (size_t i = 0; i < n; ++i) copy_ct(C, *r[i], *G->outs[i]);
    });
    *out = G.release();
  });
}

API hedap_status hedap_graph_run_many(hedap_graph* g, const hedap_ct* const* in, size_t n, hedap_ct** out) {
  return graph_guard([&] {
    if (!g || g->ins.empty()) throw Error(HEDAP_ERR_ARG, "not a graph of many ciphertexts");
    if (n != g->ins.size()) throw Error(HEDAP_ERR_ARG, "graph input count differs");
    Ctx& C = *g->C;
    std::lock_guard<std::mutex> lk(C.mu);
    if (in)
      for (size_t i = 0; i < n; ++i) {
        const Ct& a = ct_of(nullptr, in[i]);
        if (a.owner != &C) throw Error(HEDAP_ERR_ARG, "graph input made by another context");
        if (a.level != g->ins[i]->level || a.batch != 1 || a.scale != g->ins[i]->scale)
          throw Error(HEDAP_ERR_ARG, "graph input must match the captured level and scale");
      }
    if (in)
      for (size_t i = 0; i < n; ++i) copy_ct(C, ct_of(nullptr, in[i]), *g->ins[i]);
    HEDAP_CUDA(cudaGraphLaunch(g->exec, C.stream));
    if (out) {
      for (size_t i = 0; i < n; ++i) out[i] = nullptr;
      for (size_t i = 0; i < n; ++i) {
        auto r = ct_alloc(C, g->outs[i]->level, 1);
        r->scale = g->outs[i]->scale;
        copy_ct(C, *g->outs[i], *r);
        out[i] = new hedap_ct;
        out[i]->c = std::move(r);
      }
    }
  });
}

API hedap_status hedap_graph_kernels(const hedap_graph* g, uint64_t* n) {
  return graph_guard([&] {
    if (!g || !n) throw Error(HEDAP_ERR_ARG, "null argument");
    *n = g->kernels;
  });
}

API void hedap_graph_destroy(hedap_graph* g) {
  if (!g) return;
  {
    std::lock_guard<std::mutex> lk(g->C->mu);
    cudaStreamSynchronize(g->C->stream);
  }
  delete g;
}
