// extern "C" entry points declared in include/hedap.h.  Every call catches
// exceptions and turns them into a status code plus a thread-local message.
#include <cstring>

#include "internal.cuh"
#include "kernels.cuh"
#include "profiler.cuh"

namespace {
thread_local std::string g_last_error;

template <class F>
hedap_status guarded(F&& f) {
  try {
    f();
    return HEDAP_OK;
  } catch (const hedap::Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc& e) {
    g_last_error = e.what();
    return HEDAP_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return HEDAP_ERR_ARG;
  }
}
// Every entry point that takes a context runs under the context's lock, so
// calls from several host threads (a user thread beside a server's worker)
// see its lazily built keys and constants consistently.
template <class F>
hedap_status guarded_on(const hedap_ctx* ctx, F&& f) {
  if (!ctx) return guarded(std::forward<F>(f));
  if (ctx->magic != kCtxMagic || !ctx->c) {
    g_last_error = "not a live context handle";
    return HEDAP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(ctx->c->mu);
  return guarded(std::forward<F>(f));
}
void need(bool ok, const char* what) {
  if (!ok) throw hedap::Error(HEDAP_ERR_ARG, what);
}
hedap_ct* wrap(std::unique_ptr<hedap::Ct> c) {
  hedap_ct* h = new hedap_ct;
  h->c = std::move(c);
  return h;
}
}  // namespace

namespace hedap {
Ct& ct_of(const hedap_ctx* ctx, const hedap_ct* h) {
  if (!h) throw Error(HEDAP_ERR_ARG, "null ciphertext");
  if (h->magic != kCtMagic || !h->c) throw Error(HEDAP_ERR_ARG, "not a live ciphertext handle");
  if (ctx && h->c->owner != ctx->c) throw Error(HEDAP_ERR_ARG, "ciphertext made by another context");
  return *h->c;
}
Ctx& ctx_of(const hedap_ctx* ctx) {
  if (!ctx || ctx->magic != kCtxMagic || !ctx->c) throw Error(HEDAP_ERR_ARG, "not a live context handle");
  return *ctx->c;
}
void set_last_error(const std::string& m) { g_last_error = m; }
hedap_status run_on_ctx(const hedap_ctx* ctx, const std::function<void()>& f) { return guarded_on(ctx, f); }
}  // namespace hedap

#define API extern "C" __attribute__((visibility("default")))

API const char* hedap_status_str(hedap_status s) {
  switch (s) {
    case HEDAP_OK: return "ok";
    case HEDAP_ERR_ARG: return "invalid argument";
    case HEDAP_ERR_LEVEL: return "not enough levels";
    case HEDAP_ERR_SCALE: return "scale mismatch";
    case HEDAP_ERR_OOM: return "out of device memory";
    case HEDAP_ERR_CUDA: return "CUDA error";
    case HEDAP_ERR_TIMEOUT: return "device wait timed out";
    case HEDAP_ERR_RANGE: return "input out of range";
    case HEDAP_ERR_KEY: return "missing switching key";
    case HEDAP_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}
API const char* hedap_last_error(void) { return g_last_error.c_str(); }

API hedap_status hedap_ctx_create(const hedap_params* params, uint64_t seed, void* cuda_stream, hedap_ctx** out) {
  return guarded([&] {
    need(params && out, "null argument");
    *out = nullptr;
    hedap::Ctx* c = hedap::ctx_create(*params, seed, (cudaStream_t)cuda_stream);
    *out = new hedap_ctx(c);
  });
}
API void hedap_ctx_destroy(hedap_ctx* ctx) {
  if (!ctx || ctx->magic != kCtxMagic) return;  // not a live context handle: ignored
  cudaStream_t s = ctx->c->stream;
  delete ctx->c;
  cudaStreamSynchronize(s);
  delete ctx;
}
API hedap_status hedap_ctx_primes(const hedap_ctx* ctx, uint64_t* out, size_t cap) {
  return guarded_on(ctx, [&] {
    need(ctx && out, "null argument");
    need(cap >= ctx->c->primes.size(), "capacity too small");
    std::memcpy(out, ctx->c->primes.data(), ctx->c->primes.size() * 8);
  });
}
API hedap_status hedap_sync(hedap_ctx* ctx) {
  return guarded_on(ctx, [&] {
    need(ctx, "null argument");
    HEDAP_CUDA(cudaStreamSynchronize(ctx->c->stream));
  });
}
API hedap_status hedap_galois_element(const hedap_ctx* ctx, int64_t steps, int conjugate, uint64_t* out) {
  return guarded([&] {
    need(ctx && out, "null argument");
    *out = conjugate ? 2 * ctx->c->N - 1 : hedap::galois_for_rotation(*ctx->c, steps);
  });
}
API hedap_status hedap_gen_galois_key(hedap_ctx* ctx, uint64_t g) {
  return guarded_on(ctx, [&] {
    need(ctx, "null argument");
    hedap::gen_galois_key(*ctx->c, g);
  });
}
API hedap_status hedap_export_key(hedap_ctx* ctx, uint64_t g, uint32_t digit, uint64_t* b, uint64_t* a) {
  return guarded_on(ctx, [&] {
    need(ctx && b && a, "null argument");
    hedap::Ctx& C = *ctx->c;
    hedap::gen_galois_key(C, g);
    need((int)digit < C.dnum(C.L()), "digit out of range");
    const size_t part = (size_t)C.total_primes() * C.N;
    const uint64_t* base = C.keys.at(g).p + (size_t)digit * 2 * part;
    HEDAP_CUDA(cudaMemcpyAsync(b, base, part * 8, cudaMemcpyDeviceToHost, C.stream));
    HEDAP_CUDA(cudaMemcpyAsync(a, base + part, part * 8, cudaMemcpyDeviceToHost, C.stream));
    HEDAP_CUDA(cudaStreamSynchronize(C.stream));
    // the key as defined, without the conversion factors folded into its stored limbs
    const int T = C.total_primes();
    for (int t = 0; t < T; ++t) {
      const uint64_t u = C.key_unscale[(size_t)digit * T + t], pt = C.primes[t];
      if (u == 1) continue;
      for (size_t n = 0; n < C.N; ++n) {
        b[(size_t)t * C.N + n] = hedap::h_mulmod(b[(size_t)t * C.N + n], u, pt);
        a[(size_t)t * C.N + n] = hedap::h_mulmod(a[(size_t)t * C.N + n], u, pt);
      }
    }
  });
}
API hedap_status hedap_encrypt(hedap_ctx* ctx, const double* re, const double* im, size_t n_slots, int level,
                               uint64_t seed, hedap_ct** out) {
  return guarded_on(ctx, [&] {
    need(ctx && re && out, "null argument");
    *out = nullptr;
    std::vector<double> r(re, re + n_slots), i;
    if (im) i.assign(im, im + n_slots);
    *out = wrap(hedap::encrypt(*ctx->c, r, i, level, seed));
  });
}
API hedap_status hedap_decrypt(hedap_ctx* ctx, const hedap_ct* ct, double* re, double* im, size_t n_slots) {
  return guarded_on(ctx, [&] {
    need(ctx && ct && re, "null argument");
    need(n_slots == ctx->c->N / 2, "n_slots must equal N/2");
    std::vector<double> r, i;
    hedap::decrypt(*ctx->c, hedap::ct_of(ctx, ct), r, i);
    std::memcpy(re, r.data(), n_slots * 8);
    if (im) std::memcpy(im, i.data(), n_slots * 8);
  });
}
API hedap_status hedap_ct_import(hedap_ctx* ctx, const uint64_t* limbs, int level, double scale, int on_device,
                                 hedap_ct** out) {
  return guarded_on(ctx, [&] {
    need(ctx && limbs && out, "null argument");
    *out = nullptr;
    hedap::Ctx& C = *ctx->c;
    need(level >= 0 && level <= C.L(), "level out of range");
    need(scale > 0, "scale must be positive");
    const size_t per = (size_t)(level + 1) * C.N;
    auto c = hedap::ct_alloc(C, level);
    c->scale = scale;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    HEDAP_CUDA(cudaMemcpyAsync(c->part(0), limbs, per * 8, kind, C.stream));
    HEDAP_CUDA(cudaMemcpyAsync(c->part(1), limbs + per, per * 8, kind, C.stream));
    if (!on_device) {  // host words are checked on the device after the copy (residues below their primes)
      hedap::DevBuf flag(1, C.stream);
      HEDAP_CUDA(cudaMemsetAsync(flag.p, 0, 8, C.stream));
      hedap::k_check_residues(C, c->part(0), c->part_stride(), 2, level + 1, (unsigned int*)flag.p);
      uint64_t bad = 0;
      HEDAP_CUDA(cudaMemcpyAsync(&bad, flag.p, 8, cudaMemcpyDeviceToHost, C.stream));
      HEDAP_CUDA(cudaStreamSynchronize(C.stream));
      if (bad) throw hedap::Error(HEDAP_ERR_RANGE, "residue not below its prime");
    }
    *out = wrap(std::move(c));
  });
}
API hedap_status hedap_ct_export(hedap_ctx* ctx, const hedap_ct* ct, uint64_t* out, size_t cap, int on_device) {
  return guarded_on(ctx, [&] {
    need(ctx && ct && out, "null argument");
    hedap::Ctx& C = *ctx->c;
    const size_t per = (size_t)(hedap::ct_of(ctx, ct).level + 1) * C.N;
    need(cap >= 2 * per, "capacity too small");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    HEDAP_CUDA(cudaMemcpyAsync(out, hedap::ct_of(ctx, ct).part(0), per * 8, kind, C.stream));
    HEDAP_CUDA(cudaMemcpyAsync(out + per, hedap::ct_of(ctx, ct).part(1), per * 8, kind, C.stream));
    if (!on_device) HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  });
}
API hedap_status hedap_batch_import(hedap_ctx* ctx, const uint64_t* limbs, size_t n, int level, double scale,
                                    int on_device, hedap_ct** out) {
  return guarded_on(ctx, [&] {
    need(ctx && limbs && out, "null argument");
    *out = nullptr;
    hedap::Ctx& C = *ctx->c;
    need(n >= 1 && n <= (size_t)hedap::kMaxBatchCts, "batch size must lie in [1, 16]");
    need(level >= 0 && level <= C.L(), "level out of range");
    need(scale > 0, "scale must be positive");
    auto c = hedap::ct_alloc(C, level, (int)n);
    c->scale = scale;
    // cap = level + 1: the batch's parts are contiguous, [n][2][level+1][N] as the host holds them
    const size_t words = (size_t)n * 2 * (level + 1) * C.N;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    HEDAP_CUDA(cudaMemcpyAsync(c->part(0), limbs, words * 8, kind, C.stream));
    if (!on_device) {  // host words are checked on the device after the copy (residues below their primes)
      hedap::DevBuf flag(1, C.stream);
      HEDAP_CUDA(cudaMemsetAsync(flag.p, 0, 8, C.stream));
      hedap::k_check_residues(C, c->part(0), c->part_stride(), c->parts(), level + 1, (unsigned int*)flag.p);
      uint64_t bad = 0;
      HEDAP_CUDA(cudaMemcpyAsync(&bad, flag.p, 8, cudaMemcpyDeviceToHost, C.stream));
      HEDAP_CUDA(cudaStreamSynchronize(C.stream));
      if (bad) throw hedap::Error(HEDAP_ERR_RANGE, "residue not below its prime");
    }
    *out = wrap(std::move(c));
  });
}
API hedap_status hedap_batch_export(hedap_ctx* ctx, const hedap_ct* batch, uint64_t* out, size_t cap, int on_device) {
  return guarded_on(ctx, [&] {
    need(ctx && batch && out, "null argument");
    hedap::Ctx& C = *ctx->c;
    const hedap::Ct& b = hedap::ct_of(ctx, batch);
    const size_t per = (size_t)(b.level + 1) * C.N;
    need(cap >= (size_t)b.parts() * per, "capacity too small");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    // one copy: the parts are cap limbs apart on the device and level + 1 limbs apart in out
    HEDAP_CUDA(cudaMemcpy2DAsync(out, per * 8, b.part(0), b.part_stride() * 8, per * 8, (size_t)b.parts(), kind,
                                 C.stream));
    if (!on_device) HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  });
}
API hedap_status hedap_ct_info(const hedap_ct* ct, int* level, double* scale) {
  return guarded([&] {
    need(ct, "null argument");
    if (level) *level = hedap::ct_of(nullptr, ct).level;
    if (scale) *scale = hedap::ct_of(nullptr, ct).scale;
  });
}
API void hedap_ct_free(hedap_ct* ct) {
  if (ct && ct->magic == kCtMagic) delete ct;  // anything else is not a live handle: ignored
}

#define CT_OP(...)                                  \
  return guarded_on(ctx, [&] {                      \
    need(ctx && out, "null argument");             \
    *out = nullptr;                                 \
    *out = wrap(__VA_ARGS__);                       \
  })

API hedap_status hedap_add(hedap_ctx* ctx, const hedap_ct* a, const hedap_ct* b, hedap_ct** out) {
  CT_OP((need(a && b, "null ciphertext"), hedap::ev_add(*ctx->c, hedap::ct_of(ctx, a), hedap::ct_of(ctx, b), false)));
}
API hedap_status hedap_sub(hedap_ctx* ctx, const hedap_ct* a, const hedap_ct* b, hedap_ct** out) {
  CT_OP((need(a && b, "null ciphertext"), hedap::ev_add(*ctx->c, hedap::ct_of(ctx, a), hedap::ct_of(ctx, b), true)));
}
API hedap_status hedap_mul_relin(hedap_ctx* ctx, const hedap_ct* a, const hedap_ct* b, hedap_ct** out) {
  CT_OP((need(a && b, "null ciphertext"), hedap::ev_mul_relin(*ctx->c, hedap::ct_of(ctx, a), hedap::ct_of(ctx, b))));
}
API hedap_status hedap_mul(hedap_ctx* ctx, const hedap_ct* a, const hedap_ct* b, hedap_ct** out) {
  CT_OP((need(a && b, "null ciphertext"), hedap::ev_mul(*ctx->c, hedap::ct_of(ctx, a), hedap::ct_of(ctx, b))));
}
API hedap_status hedap_rescale(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::ev_rescale(*ctx->c, hedap::ct_of(ctx, a))));
}
API hedap_status hedap_rotate_hoisted(hedap_ctx* ctx, const hedap_ct* a, const int64_t* steps, size_t n,
                                      hedap_ct** out) {
  return guarded_on(ctx, [&] {
    need(ctx && a && steps && out && n > 0, "null argument");
    std::vector<uint64_t> gs;
    for (size_t i = 0; i < n; ++i) gs.push_back(hedap::galois_for_rotation(*ctx->c, steps[i]));
    auto r = hedap::ev_galois_hoisted(*ctx->c, hedap::ct_of(ctx, a), gs);
    for (size_t i = 0; i < n; ++i) out[i] = wrap(std::move(r[i]));
  });
}
API hedap_status hedap_rotate(hedap_ctx* ctx, const hedap_ct* a, int64_t steps, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::ev_galois(*ctx->c, hedap::ct_of(ctx, a), hedap::galois_for_rotation(*ctx->c, steps))));
}
API hedap_status hedap_conjugate(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::ev_galois(*ctx->c, hedap::ct_of(ctx, a), 2 * ctx->c->N - 1)));
}
API hedap_status hedap_mul_const(hedap_ctx* ctx, const hedap_ct* a, double c, double target_scale, hedap_ct** out) {
  CT_OP((need(a && target_scale > 0, "bad argument"), hedap::ev_mul_const(*ctx->c, hedap::ct_of(ctx, a), c, target_scale)));
}
API hedap_status hedap_add_const(hedap_ctx* ctx, const hedap_ct* a, double c, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::ev_add_const(*ctx->c, hedap::ct_of(ctx, a), c)));
}
API hedap_status hedap_mul_int(hedap_ctx* ctx, const hedap_ct* a, int64_t m, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::ev_mul_int(*ctx->c, hedap::ct_of(ctx, a), m)));
}
API hedap_status hedap_drop_level(hedap_ctx* ctx, const hedap_ct* a, int level, hedap_ct** out) {
  CT_OP((need(a && level >= 0 && level <= a->c->level, "bad level"), hedap::ev_drop(*ctx->c, hedap::ct_of(ctx, a), level)));
}
API hedap_status hedap_invsqrt(hedap_ctx* ctx, const hedap_ct* in, const hedap_invsqrt_cfg* cfg, hedap_ct** out) {
  CT_OP((need(in && cfg, "null argument"), hedap::invsqrt(*ctx->c, hedap::ct_of(ctx, in), *cfg)));
}
API hedap_status hedap_ntt(hedap_ctx* ctx, uint64_t* limbs, size_t n_limbs, uint32_t first_prime, int inverse,
                           int on_device) {
  return guarded_on(ctx, [&] {
    need(ctx && limbs, "null argument");
    hedap::Ctx& C = *ctx->c;
    need(first_prime + n_limbs <= (size_t)C.total_primes(), "prime index out of range");
    if (n_limbs == 0) return;
    const size_t words = n_limbs * C.N;
    hedap::DevBuf tmp;
    uint64_t* d = limbs;
    if (!on_device) {
      tmp = hedap::DevBuf(words, C.stream);
      HEDAP_CUDA(cudaMemcpyAsync(tmp.p, limbs, words * 8, cudaMemcpyHostToDevice, C.stream));
      d = tmp.p;
    }
    hedap::LimbSet S{d, 0, 1, 0, (int)n_limbs, INT_MAX, (int)first_prime, 0};
    if (inverse) hedap::ntt_inverse(C.tab, S, C.stream);
    else hedap::ntt_forward(C.tab, S, C.stream);
    if (!on_device) {
      HEDAP_CUDA(cudaMemcpyAsync(limbs, tmp.p, words * 8, cudaMemcpyDeviceToHost, C.stream));
      HEDAP_CUDA(cudaStreamSynchronize(C.stream));
    }
  });
}

API hedap_status hedap_profile_enable(int on) {
  return guarded([&] {
    if (on) hedap::prof_reset();
    hedap::prof_enable(on != 0);
  });
}
API hedap_status hedap_profile_read_slots(const char* cls, double* slots) {
  return guarded([&] {
    need(cls && slots, "null argument");
    const int c = hedap::prof_class_of(cls);
    need(c >= 0, "unknown kernel class");
    *slots = hedap::prof_read_slots(c);
  });
}
API hedap_status hedap_profile_read(const char* cls, uint64_t* scopes, double* ms, double* bytes) {
  return guarded([&] {
    need(cls != nullptr, "null argument");
    const int c = hedap::prof_class_of(cls);
    need(c >= 0, "unknown kernel class");
    hedap::prof_read(c, scopes, ms, bytes);
  });
}
API hedap_status hedap_launch_count(uint64_t* out) {
  return guarded([&] {
    need(out != nullptr, "null argument");
    *out = hedap::prof_launches();
  });
}

// ---------------------------------------------------------------- key-switching steps (test ABI)
API hedap_status hedap_modup(hedap_ctx* ctx, const uint64_t* in, int level, uint64_t* out) {
  return guarded_on(ctx, [&] {
    need(ctx && in && out, "null argument");
    hedap::Ctx& C = *ctx->c;
    need(level >= 0 && level <= C.L(), "level out of range");
    const size_t N = C.N, ext = (size_t)level + 1 + C.n_p, dn = (size_t)C.dnum(level);
    hedap::DevBuf x((level + 1) * N, C.stream), y(dn * ext * N, C.stream);
    HEDAP_CUDA(cudaMemcpyAsync(x.p, in, (level + 1) * N * 8, cudaMemcpyHostToDevice, C.stream));
    hedap::k_modup(C, x.p, y.p, 1, level, hedap::level_consts(C, level).modup.p);
    HEDAP_CUDA(cudaMemcpyAsync(out, y.p, dn * ext * N * 8, cudaMemcpyDeviceToHost, C.stream));
    HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  });
}
API hedap_status hedap_moddown(hedap_ctx* ctx, const uint64_t* in, int level, uint64_t* out) {
  return guarded_on(ctx, [&] {
    need(ctx && in && out, "null argument");
    hedap::Ctx& C = *ctx->c;
    need(level >= 0 && level <= C.L(), "level out of range");
    const size_t N = C.N, ext = (size_t)level + 1 + C.n_p, nl = (size_t)level + 1;
    hedap::DevBuf acc(2 * ext * N, C.stream), v(2 * nl * N, C.stream), o(2 * nl * N, C.stream);
    HEDAP_CUDA(cudaMemcpyAsync(acc.p, in, 2 * ext * N * 8, cudaMemcpyHostToDevice, C.stream));
    hedap::LimbSet qs{acc.p, ext * N, 2, 0, (int)nl, INT_MAX, 0, 0};
    hedap::ntt_forward(C.tab, qs, C.stream);  // Q limbs enter ModDown in the NTT domain
    hedap::k_moddown_spread(C, acc.p, v.p, 2, level);
    hedap::ntt_forward(C.tab, hedap::LimbSet{v.p, nl * N, 2, 0, (int)nl, INT_MAX, 0, 0}, C.stream);
    hedap::k_moddown_finish(C, acc.p, v.p, o.p, nl * N, 2, level, false, false);
    hedap::ntt_inverse(C.tab, hedap::LimbSet{o.p, nl * N, 2, 0, (int)nl, INT_MAX, 0, 0}, C.stream);
    HEDAP_CUDA(cudaMemcpyAsync(out, o.p, 2 * nl * N * 8, cudaMemcpyDeviceToHost, C.stream));
    HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  });
}
API hedap_status hedap_key_switch(hedap_ctx* ctx, const uint64_t* d, int level, uint64_t galois, uint64_t* out) {
  return guarded_on(ctx, [&] {
    need(ctx && d && out, "null argument");
    hedap::Ctx& C = *ctx->c;
    need(level >= 0 && level <= C.L(), "level out of range");
    const size_t N = C.N, nl = (size_t)level + 1;
    hedap::DevBuf x(nl * N, C.stream), o(2 * nl * N, C.stream);
    HEDAP_CUDA(cudaMemcpyAsync(x.p, d, nl * N * 8, cudaMemcpyHostToDevice, C.stream));
    hedap::key_switch(C, x.p, nl * N, 1, level, galois, o.p, nl * N, false, false);
    HEDAP_CUDA(cudaMemcpyAsync(out, o.p, 2 * nl * N * 8, cudaMemcpyDeviceToHost, C.stream));
    HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  });
}

// ---------------------------------------------------------------- bootstrapping
API hedap_status hedap_bootstrap_setup(hedap_ctx* ctx, const hedap_bts_params* p, int* level_after) {
  return guarded_on(ctx, [&] {
    need(ctx && p, "null argument");
    const int l = hedap::bts_setup(*ctx->c, (int)p->K, (int)p->double_angles, (int)p->mod_degree,
                                   (int)p->cts_levels, (int)p->stc_levels);
    if (level_after) *level_after = l;
  });
}
API hedap_status hedap_bootstrap_encapsulate(hedap_ctx* ctx, uint32_t h) {
  return guarded_on(ctx, [&] {
    need(ctx, "null argument");
    hedap::bts_encapsulate(*ctx->c, (int)h);
  });
}
API hedap_status hedap_encapsulation_switch(hedap_ctx* ctx, const hedap_ct* a, int to_sparse, hedap_ct** out) {
  CT_OP((need(a && ctx->c->enc_hw, "null ciphertext or no encapsulation"),
         hedap::ev_switch_key(*ctx->c, hedap::ct_of(ctx, a), to_sparse ? hedap::kKeyToSparse : hedap::kKeyToDense)));
}
API hedap_status hedap_bootstrap_slots(hedap_ctx* ctx, const hedap_ct* a, uint32_t log_slots, hedap_ct** out) {
  CT_OP((need(a && log_slots >= 1 && log_slots < 31, "bad argument"),
         hedap::bootstrap_core(*ctx->c, hedap::ct_of(ctx, a), (int)log_slots)));
}
API hedap_status hedap_bootstrap_scaled_slots(hedap_ctx* ctx, const hedap_ct* a, int64_t Y, uint32_t log_slots,
                                              hedap_ct** out) {
  CT_OP((need(a && Y >= 1 && log_slots >= 1 && log_slots < 31, "bad argument"),
         hedap::bootstrap_scaled(*ctx->c, hedap::ct_of(ctx, a), Y, (int)log_slots)));
}
API hedap_status hedap_sub_sum(hedap_ctx* ctx, const hedap_ct* a, uint32_t log_slots, hedap_ct** out) {
  CT_OP((need(a && log_slots < 31, "bad argument"), hedap::sub_sum(*ctx->c, hedap::ct_of(ctx, a), (size_t)1 << log_slots)));
}
API hedap_status hedap_bootstrap(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::bootstrap_core(*ctx->c, hedap::ct_of(ctx, a))));
}
API hedap_status hedap_bootstrap_scaled(hedap_ctx* ctx, const hedap_ct* a, int64_t Y, hedap_ct** out) {
  CT_OP((need(a && Y >= 1, "bad argument"), hedap::bootstrap_scaled(*ctx->c, hedap::ct_of(ctx, a), Y)));
}
API hedap_status hedap_mod_raise(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::mod_raise(*ctx->c, hedap::ct_of(ctx, a))));
}
API hedap_status hedap_mul_monomial(hedap_ctx* ctx, const hedap_ct* a, uint64_t e, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::mul_monomial(*ctx->c, hedap::ct_of(ctx, a), e)));
}
API hedap_status hedap_bts_linear_transform(hedap_ctx* ctx, const hedap_ct* a, int inverse, int group,
                                            double target_scale, hedap_ct** out) {
  CT_OP((need(a && target_scale > 0, "bad argument"),
         hedap::bts_linear_transform(*ctx->c, hedap::ct_of(ctx, a), inverse != 0, group, target_scale)));
}
API hedap_status hedap_eval_mod(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out) {
  CT_OP((need(a, "null ciphertext"), hedap::eval_mod(*ctx->c, hedap::ct_of(ctx, a))));
}
API hedap_status hedap_set_scale(hedap_ctx* ctx, hedap_ct* a, double scale) {
  return guarded_on(ctx, [&] {
    need(ctx && a && scale > 0, "bad argument");
    hedap::ct_of(ctx, a).scale = scale;
  });
}
API hedap_status hedap_encode(hedap_ctx* ctx, const double* re, const double* im, size_t n_slots, double scale,
                              int64_t* out) {
  return guarded_on(ctx, [&] {
    need(ctx && re && out, "null argument");
    need(n_slots == ctx->c->N / 2, "n_slots must equal N/2");
    std::vector<std::complex<double>> z(n_slots);
    for (size_t j = 0; j < n_slots; ++j) z[j] = {re[j], im ? im[j] : 0.0};
    std::vector<double> m = hedap::encode_slots(*ctx->c, z, scale);
    for (size_t k = 0; k < m.size(); ++k) {
      need(std::fabs(m[k]) < 9.2e18, "coefficient exceeds 63 bits");
      out[k] = (int64_t)m[k];
    }
  });
}
API hedap_status hedap_bts_diagonal(hedap_ctx* ctx, int inverse, int group, int64_t offset, double* re, double* im) {
  return guarded_on(ctx, [&] {
    need(ctx && re && im, "null argument");
    std::vector<std::complex<double>> d;
    need(hedap::bts_diagonal(*ctx->c, inverse != 0, group, (long)offset, d), "no such diagonal");
    for (size_t s = 0; s < d.size(); ++s) { re[s] = d[s].real(); im[s] = d[s].imag(); }
  });
}

// ---------------------------------------------------------------- batches
API hedap_status hedap_batch_pack(hedap_ctx* ctx, const hedap_ct* const* cts, size_t n, hedap_ct** out) {
  return guarded_on(ctx, [&] {
    need(ctx && cts && out && n >= 1 && n <= 16, "bad argument");
    *out = nullptr;
    std::vector<const hedap::Ct*> v;
    for (size_t i = 0; i < n; ++i) {
      need(cts[i] != nullptr, "null ciphertext");
      v.push_back(&hedap::ct_of(ctx, cts[i]));
    }
    *out = wrap(hedap::batch_pack(*ctx->c, v));
  });
}
API hedap_status hedap_batch_unpack(hedap_ctx* ctx, const hedap_ct* batch, size_t index, hedap_ct** out) {
  CT_OP((need(batch != nullptr, "null ciphertext"), hedap::batch_unpack(*ctx->c, hedap::ct_of(ctx, batch), (int)index)));
}
API hedap_status hedap_ct_batch_size(const hedap_ct* ct, int* n) {
  return guarded([&] {
    need(ct && n, "null argument");
    *n = hedap::ct_of(nullptr, ct).batch;
  });
}
// groups of inputs run as one batch: equal scale and configuration, and equal level (band = 0)
// or levels in the same band [k band, (k+1) band) dropped to the lowest level present there;
// up to 16 per group, in input order
static void invsqrt_grouped(hedap_ctx* ctx, const hedap_ct* const* in, const hedap_invsqrt_cfg* cfgs, size_t n,
                            int band, hedap_ct** out) {
  need(ctx && in && cfgs && out && band >= 0, "bad argument");
  for (size_t i = 0; i < n; ++i) out[i] = nullptr;
  hedap::Ctx& C = *ctx->c;
  auto key = [&](size_t i) { return band ? hedap::ct_of(ctx, in[i]).level / band : hedap::ct_of(ctx, in[i]).level; };
  std::vector<bool> done(n, false);
  try {
    for (size_t i = 0; i < n; ++i) need(in[i] != nullptr && hedap::ct_of(ctx, in[i]).batch == 1, "inputs must be single ciphertexts");
    for (size_t i = 0; i < n; ++i) {
      if (done[i]) continue;
      std::vector<size_t> g{i};
      for (size_t j = i + 1; j < n && g.size() < 16; ++j) {
        if (done[j]) continue;
        const hedap::Ct &a = hedap::ct_of(ctx, in[i]), &b = hedap::ct_of(ctx, in[j]);
        if (key(i) == key(j) && a.scale == b.scale && hedap::same_cfg(cfgs[i], cfgs[j]))
          g.push_back(j);
      }
      int lmin = INT_MAX;
      for (size_t j : g) lmin = std::min(lmin, hedap::ct_of(ctx, in[j]).level);
      std::vector<std::unique_ptr<hedap::Ct>> dropped;
      std::vector<const hedap::Ct*> v;
      for (size_t j : g) {
        const hedap::Ct& a = hedap::ct_of(ctx, in[j]);
        if (a.level == lmin) {
          v.push_back(&a);
        } else {
          dropped.push_back(hedap::ev_drop(C, a, lmin));
          v.push_back(dropped.back().get());
        }
      }
      auto res = g.size() > 1 ? hedap::invsqrt(C, *hedap::batch_pack(C, v), cfgs[i]) : hedap::invsqrt(C, *v[0], cfgs[i]);
      for (size_t k = 0; k < g.size(); ++k) {
        out[g[k]] = wrap(g.size() > 1 ? hedap::batch_unpack(C, *res, (int)k) : std::move(res));
        done[g[k]] = true;
      }
    }
  } catch (...) {
    for (size_t i = 0; i < n; ++i) {
      delete out[i];
      out[i] = nullptr;
    }
    throw;
  }
}
API hedap_status hedap_invsqrt_batch(hedap_ctx* ctx, const hedap_ct* const* in, const hedap_invsqrt_cfg* cfgs,
                                     size_t n, hedap_ct** out) {
  return guarded_on(ctx, [&] { invsqrt_grouped(ctx, in, cfgs, n, 0, out); });
}
API hedap_status hedap_invsqrt_many(hedap_ctx* ctx, const hedap_ct* const* in, const hedap_invsqrt_cfg* cfgs, size_t n,
                                    int level_band, hedap_ct** out) {
  return guarded_on(ctx, [&] { invsqrt_grouped(ctx, in, cfgs, n, level_band, out); });
}
API hedap_status hedap_invsqrt_mixed(hedap_ctx* ctx, const hedap_ct* const* in, const hedap_invsqrt_cfg* cfgs,
                                     size_t n, hedap_ct** out) {
  return guarded_on(ctx, [&] {
    need(ctx && in && cfgs && out, "null argument");
    for (size_t i = 0; i < n; ++i) out[i] = nullptr;
    std::vector<const hedap::Ct*> v;
    for (size_t i = 0; i < n; ++i) v.push_back(&hedap::ct_of(ctx, in[i]));
    auto r = hedap::invsqrt_mixed(*ctx->c, v, std::vector<hedap_invsqrt_cfg>(cfgs, cfgs + n));
    for (size_t i = 0; i < n; ++i) out[i] = wrap(std::move(r[i]));
  });
}
API hedap_status hedap_ntt_batch(hedap_ctx* ctx, uint64_t* limbs, size_t n_limbs, size_t n_polys, uint32_t first_prime,
                                 int inverse, int on_device) {
  return guarded_on(ctx, [&] {
    need(ctx && limbs, "null argument");
    hedap::Ctx& C = *ctx->c;
    need(first_prime + n_limbs <= (size_t)C.total_primes(), "prime index out of range");
    need(n_polys * n_limbs <= 65535, "too many limbs in one batch");
    if (n_limbs == 0 || n_polys == 0) return;
    const size_t words = n_polys * n_limbs * C.N;
    hedap::DevBuf tmp;
    uint64_t* d = limbs;
    if (!on_device) {
      tmp = hedap::DevBuf(words, C.stream);
      HEDAP_CUDA(cudaMemcpyAsync(tmp.p, limbs, words * 8, cudaMemcpyHostToDevice, C.stream));
      d = tmp.p;
    }
    hedap::LimbSet S{d, n_limbs * C.N, (int)n_polys, 0, (int)n_limbs, INT_MAX, (int)first_prime, 0};
    if (inverse) hedap::ntt_inverse(C.tab, S, C.stream);
    else hedap::ntt_forward(C.tab, S, C.stream);
    if (!on_device) {
      HEDAP_CUDA(cudaMemcpyAsync(limbs, tmp.p, words * 8, cudaMemcpyDeviceToHost, C.stream));
      HEDAP_CUDA(cudaStreamSynchronize(C.stream));
    }
  });
}

API hedap_status hedap_ntt_tune(hedap_ctx* ctx, int limbs, int reps, float* fwd_ms, float* inv_ms, int cap,
                                int* fwd_variant, int* inv_variant) {
  return guarded_on(ctx, [&] {
    need(ctx != nullptr && limbs > 0 && reps > 0, "bad argument");
    std::vector<float> f, i;
    hedap::ntt_tune(*ctx->c, limbs, reps, &f, &i);
    for (int k = 0; k < cap && k < (int)f.size(); ++k) {
      if (fwd_ms) fwd_ms[k] = f[k];
      if (inv_ms) inv_ms[k] = i[k];
    }
    if (fwd_variant) *fwd_variant = ctx->c->tab.ntt_fwd_variant;
    if (inv_variant) *inv_variant = ctx->c->tab.ntt_inv_variant;
  });
}
API hedap_status hedap_butterfly_rate(hedap_ctx* ctx, double* per_s) {
  return guarded_on(ctx, [&] {
    need(ctx && per_s, "null argument");
    *per_s = hedap::butterfly_rate(*ctx->c);
  });
}
API hedap_status hedap_ntt_get_variant(const hedap_ctx* ctx, int* fwd_variant, int* inv_variant) {
  return guarded_on(ctx, [&] {
    need(ctx && fwd_variant && inv_variant, "null argument");
    *fwd_variant = ctx->c->tab.ntt_fwd_variant;
    *inv_variant = ctx->c->tab.ntt_inv_variant;
  });
}
API hedap_status hedap_ntt_set_variant(hedap_ctx* ctx, int fwd_variant, int inv_variant) {
  return guarded_on(ctx, [&] {
    need(ctx && fwd_variant >= 0 && fwd_variant < hedap::kNttVariants && inv_variant >= 0 &&
             inv_variant < hedap::kNttVariants,
         "variant out of range");
    hedap::Tables& T = ctx->c->tab;
    T.ntt_fwd_variant = T.ntt_modup_variant = T.ntt_fin_variant = fwd_variant;
    T.ntt_inv_variant = inv_variant;
  });
}
API hedap_status hedap_ntt_set_role_variant(hedap_ctx* ctx, int role, int variant) {
  return guarded_on(ctx, [&] {
    need(ctx && variant >= 0 && variant < hedap::kNttVariants, "variant out of range");
    need(role >= 0 && role < HEDAP_NTT_ROLES, "unknown NTT role");
    hedap::ntt_role_variant(ctx->c->tab, role) = variant;
  });
}
API hedap_status hedap_ntt_get_role_variant(const hedap_ctx* ctx, int role, int* variant) {
  return guarded_on(ctx, [&] {
    need(ctx && variant, "null argument");
    need(role >= 0 && role < HEDAP_NTT_ROLES, "unknown NTT role");
    *variant = hedap::ntt_role_variant(ctx->c->tab, role);
  });
}

// ---------------------------------------------------------------- selector
API hedap_status hedap_select(hedap_ctx* ctx, const hedap_select_cfg* cfg, hedap_select_entry* D, size_t D_cap,
                              size_t* n_D, hedap_select_entry* R, size_t R_cap, size_t* n_R,
                              hedap_select_trace* trace, size_t trace_cap, size_t* n_trace) {
  return guarded_on(ctx, [&] {
    need(ctx && cfg, "null argument");
    std::vector<hedap_select_entry> d, r;
    std::vector<hedap_select_trace> t;
    hedap::select(*ctx->c, *cfg, d, r, t);
    if (n_D) *n_D = d.size();
    if (n_R) *n_R = r.size();
    if (n_trace) *n_trace = t.size();
    need(!D || D_cap >= d.size(), "D capacity too small");
    need(!R || R_cap >= r.size(), "R capacity too small");
    need(!trace || trace_cap >= t.size(), "trace capacity too small");
    if (D) std::copy(d.begin(), d.end(), D);
    if (R) std::copy(r.begin(), r.end(), R);
    if (trace) std::copy(t.begin(), t.end(), trace);
  });
}
API hedap_status hedap_getoptiter_rule(const double* M, size_t n, double delta, int* I, double* threshold) {
  return guarded([&] {
    need(M && I, "null argument");
    *I = hedap::getoptiter_rule(M, n, delta, threshold);
  });
}
API hedap_status hedap_select_level_rule(const hedap_select_entry* D, size_t n, double theta, double mre_target,
                                         hedap_select_entry* u1, hedap_select_entry* u2, hedap_select_entry* u3,
                                         int* has_u3) {
  return guarded([&] {
    need(D && u1 && u2 && u3 && n > 0, "bad argument");
    const int r = hedap::level_rule(D, n, theta, mre_target, u1, u2, u3);
    if (has_u3) *has_u3 = r == 1;
  });
}
