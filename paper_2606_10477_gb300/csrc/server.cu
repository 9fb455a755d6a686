// Serving: a continuous-batching request loop for encrypted statistical
// queries that each need the inverse square root of an encrypted variance
// (the statistical workloads of Sec. 5.3: Z-score normalisation and the
// Pearson correlation coefficient).
//
// One worker thread drives the context.  Submitted queries wait in a FIFO; at
// every scheduling iteration the worker admits the oldest waiting query and
// the later ones that can share its group (one kind, input level, input scale
// and InvSqrt configuration; up to max_batch) while the estimated device
// memory of the admitted queries stays within the budget, and makes them a
// new group.  Groups advance one
// step at a time, round-robin, so a group admitted while others are in flight
// starts at once and its steps interleave with theirs:
//   stats      x^2 (and y^2, x*y) of every ciphertext of the group, batched;
//              per query: their sums and the sum of x (and y) over its
//              ciphertexts; over the group: rotate-and-sum over all slots;
//              per query: means, variance (PCC: covariance, var_x * var_y)
//   prepare    CryptoInvSqrt's Pre-BTS / pre-normalisation on the group batch
//   chebyshev  the Chebyshev initial value (Alg. 1)
//   newton i   one Newton step, with lazy bootstrapping (Alg. 1)
//   finish     a bootstrap of InvSqrt's result when it has no level left for
//              the last product, then z = (x - mean) * InvSqrt(var) per ciphertext, or
//              r = cov * InvSqrt(var_x var_y)
// Each step is one batched launch sequence over the group, issued on the
// context's stream without waiting; a finished group records an event and its
// queries complete when the event does.  Batched operations equal single
// operations bit for bit and every decision (a bootstrap, a level drop) is a
// function of the group's common kind, level and configuration, so a query's
// result does not depend on which other queries share its group or the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>

#include "internal.cuh"

namespace {

using namespace hedap;
using Clock = std::chrono::steady_clock;
typedef std::unique_ptr<Ct> CtP;

struct Query {
  uint64_t id = 0;
  uint32_t kind = 0;
  std::vector<const Ct*> x, y;  // borrowed until the query completes
  uint64_t n_records = 0;
  hedap_invsqrt_cfg cfg{};
  int level = 0;
  double scale = 0;
  size_t bytes = 0;  // admission estimate
  Clock::time_point submitted;
  CtP mean_x, cov, var;
  std::vector<CtP> out;
  double latency_ms = 0;
  uint32_t group_size = 0;
  bool done = false;
  std::string error;
};

bool same_group(const Query& a, const Query& b) {
  return a.kind == b.kind && a.level == b.level && a.scale == b.scale && same_cfg(a.cfg, b.cfg);
}

struct Group {
  std::vector<Query*> q;
  int step = 0;  // 0 stats, 1 prepare, 2 chebyshev, 3 .. 2+iters newton, then finish
  std::unique_ptr<InvSqrtRun> run;
};

struct Pending {
  cudaEvent_t ev;
  std::vector<Query*> q;
};

// rotate-and-sum: every slot of the result holds the sum of all N/2 slots
CtP all_slots_sum(Ctx& C, CtP a) {
  for (size_t r = 1; r < C.N / 2; r <<= 1) a = ev_add(C, *a, *ev_galois(C, *a, galois_for_rotation(C, (i64)r)), false);
  return a;
}

CtP sum_into(Ctx& C, CtP acc, const Ct& v) { return acc ? ev_add(C, *acc, v, false) : ct_copy(C, v, v.level); }

// products a[i] * b[i], as batched multiplications of up to 16 pairs (the
// a's share one level and scale, and so do the b's)
std::vector<CtP> mul_many(Ctx& C, const std::vector<const Ct*>& a, const std::vector<const Ct*>& b) {
  constexpr size_t kChunk = 16;
  std::vector<CtP> out;
  for (size_t i = 0; i < a.size(); i += kChunk) {
    const size_t n = std::min(kChunk, a.size() - i);
    if (n == 1) {
      out.push_back(ev_mul(C, *a[i], *b[i]));
      continue;
    }
    std::vector<const Ct*> pa(a.begin() + (long)i, a.begin() + (long)(i + n));
    std::vector<const Ct*> pb(b.begin() + (long)i, b.begin() + (long)(i + n));
    CtP prod = ev_mul(C, *batch_pack(C, pa), *batch_pack(C, pb));
    for (size_t k = 0; k < n; ++k) out.push_back(batch_unpack(C, *prod, (int)k));
  }
  return out;
}

}  // namespace

struct hedap_server {
  hedap::Ctx* C = nullptr;
  hedap_server_cfg cfg{};
  std::mutex mu;  // guards everything below but groups and pending (the context has its own lock)
  std::condition_variable cv, done_cv;
  std::deque<Query*> waiting;
  std::map<uint64_t, std::unique_ptr<Query>> all;
  std::vector<std::unique_ptr<Group>> groups;  // worker-only
  std::deque<Pending> pending;                 // worker-only
  size_t admitted_bytes = 0;
  uint64_t next_id = 1;
  bool stop = false;
  bool paused = false;
  std::thread worker;
  std::vector<double> latencies;
  Clock::time_point first_submit, last_done;
  bool any = false;
  std::vector<hedap_select_entry> table;  // HE-DAP per-level choices (guarded by mu)

  size_t estimate_bytes(size_t n_out, int level) const;
  void loop();
  void step(Group& g);
  void retire(bool block);
  void fail(const std::vector<Query*>& qs, const std::string& why);
};

// Device memory a query holds while admitted (its inputs are the caller's):
// its outputs, eight working ciphertexts at the input level, and its share of
// the key-switching scratch of one batched operation at the top level (the
// ModUp digits and two accumulators), doubled for bootstrapping.
size_t hedap_server::estimate_bytes(size_t n_out, int level) const {
  const size_t ct = 2 * (size_t)(level + 1) * C->N * 8;
  const size_t top = (size_t)(C->L() + 1 + C->n_p) * C->N * 8;
  const size_t ks = (size_t)(C->dnum(C->L()) + 2) * top;
  return (n_out + 8) * ct + 2 * ks;
}

void hedap_server::fail(const std::vector<Query*>& qs, const std::string& why) {
  std::lock_guard<std::mutex> lk(mu);
  for (Query* q : qs) {
    q->error = why;
    q->done = true;
    q->out.clear();
    q->x.clear();
    q->y.clear();
    admitted_bytes -= q->bytes;
  }
  done_cv.notify_all();
}

void hedap_server::step(Group& g) {
  Ctx& Cx = *C;
  const int B = (int)g.q.size();
  const bool pcc = g.q[0]->kind == HEDAP_QUERY_PCC;
  if (g.step == 0) {
    // the second moments of every query's ciphertexts, batched across the group
    std::vector<const Ct*> fa, fb;
    for (Query* q : g.q)
      for (size_t k = 0; k < q->x.size(); ++k) {
        fa.push_back(q->x[k]);
        fb.push_back(q->x[k]);
        if (pcc) {
          fa.insert(fa.end(), {q->y[k], q->x[k]});
          fb.insert(fb.end(), {q->y[k], q->y[k]});
        }
      }
    std::vector<CtP> prod = mul_many(Cx, fa, fb);
    std::vector<CtP> s1, s2, t1, t2, sxy;
    size_t at = 0;
    for (Query* q : g.q) {
      CtP a, a2, b, b2, ab;
      for (size_t k = 0; k < q->x.size(); ++k) {
        a = sum_into(Cx, std::move(a), *q->x[k]);
        a2 = sum_into(Cx, std::move(a2), *prod[at++]);
        if (pcc) {
          b = sum_into(Cx, std::move(b), *q->y[k]);
          b2 = sum_into(Cx, std::move(b2), *prod[at++]);
          ab = sum_into(Cx, std::move(ab), *prod[at++]);
        }
      }
      s1.push_back(std::move(a));
      s2.push_back(std::move(a2));
      if (pcc) {
        t1.push_back(std::move(b));
        t2.push_back(std::move(b2));
        sxy.push_back(std::move(ab));
      }
    }
    prod.clear();
    // one batched rotate-and-sum per moment over the whole group
    auto reduce = [&](std::vector<CtP>& v) {
      if (v.empty()) return;
      if (B == 1) {
        v[0] = all_slots_sum(Cx, std::move(v[0]));
        return;
      }
      std::vector<const Ct*> ptr;
      for (auto& c : v) ptr.push_back(c.get());
      CtP packed = all_slots_sum(Cx, batch_pack(Cx, ptr));
      for (int k = 0; k < B; ++k) v[k] = batch_unpack(Cx, *packed, k);
    };
    reduce(s1);
    reduce(s2);
    reduce(t1);
    reduce(t2);
    reduce(sxy);
    for (int k = 0; k < B; ++k) {
      Query* q = g.q[k];
      const double invn = 1.0 / (double)q->n_records;
      // E[v] - E[u] E[w] from the slot sum of v and the means u, w
      auto central = [&](const Ct& sum_v, const Ct& mu, const Ct& mw) {
        CtP m2 = ev_mul(Cx, mu, mw);
        CtP ev = ev_mul_const(Cx, *ev_drop(Cx, sum_v, m2->level + 1), invn, m2->scale);
        return ev_add(Cx, *ev, *m2, true);
      };
      q->mean_x = ev_mul_const(Cx, *s1[k], invn, q->scale);
      CtP var_x = central(*s2[k], *q->mean_x, *q->mean_x);
      if (pcc) {
        CtP mean_y = ev_mul_const(Cx, *t1[k], invn, q->scale);
        CtP var_y = central(*t2[k], *mean_y, *mean_y);
        q->cov = central(*sxy[k], *q->mean_x, *mean_y);
        q->var = ev_mul(Cx, *var_x, *var_y);
      } else {
        q->var = std::move(var_x);
      }
    }
    g.step = 1;
    return;
  }
  if (g.step == 1) {
    std::vector<const Ct*> v;
    for (Query* q : g.q) v.push_back(q->var.get());
    CtP packed = B > 1 ? batch_pack(Cx, v) : nullptr;
    g.run.reset(new InvSqrtRun(Cx, packed ? *packed : *v[0], g.q[0]->cfg));
    for (Query* q : g.q) q->var.reset();
    g.step = 2;
    return;
  }
  if (g.step == 2) {
    g.run->chebyshev();
    g.step = 3;
    return;
  }
  const int iters = (int)g.q[0]->cfg.newton_iters;
  if (g.step < 3 + iters) {
    g.run->newton(g.step - 3);
    ++g.step;
    return;
  }
  // finish: the last product needs one level; InvSqrt's output lies in (0, 1/sqrt(lo)]
  CtP s = g.run->result();
  g.run.reset();
  if (s->level < 1) {
    if (!Cx.bts) throw Error(HEDAP_ERR_LEVEL, "server: InvSqrt left no level for the final product");
    i64 Y = 1;
    while ((double)Y < 1.0 / std::sqrt(g.q[0]->cfg.lo)) Y *= 2;
    s = bootstrap_scaled(Cx, *s, Y, (int)g.q[0]->cfg.log_slots);
  }
  std::vector<CtP> sk;
  for (int k = 0; k < B; ++k) sk.push_back(B > 1 ? batch_unpack(Cx, *s, k) : std::move(s));
  // the final products of the whole group, batched
  std::vector<CtP> diff;
  std::vector<const Ct*> fa, fb;
  for (int k = 0; k < B; ++k) {
    Query* q = g.q[k];
    if (pcc) {
      fa.push_back(q->cov.get());
      fb.push_back(sk[k].get());
    } else {
      for (const Ct* xc : q->x) {
        diff.push_back(ev_add(Cx, *xc, *q->mean_x, true));
        fa.push_back(diff.back().get());
        fb.push_back(sk[k].get());
      }
    }
  }
  std::vector<CtP> prod = mul_many(Cx, fa, fb);
  size_t at = 0;
  for (Query* q : g.q) {
    const size_t n_out = pcc ? 1 : q->x.size();
    for (size_t k = 0; k < n_out; ++k) q->out.push_back(std::move(prod[at++]));
    q->mean_x.reset();
    q->cov.reset();
  }
  g.step = -1;
}

// complete finished groups whose event has passed (FIFO: they share one stream)
void hedap_server::retire(bool block) {
  while (!pending.empty()) {
    Pending& p = pending.front();
    const cudaError_t e = block ? cudaEventSynchronize(p.ev) : cudaEventQuery(p.ev);
    if (e == cudaErrorNotReady) return;
    block = false;
    cudaEventDestroy(p.ev);
    std::vector<Query*> qs = std::move(p.q);
    pending.pop_front();
    if (e != cudaSuccess) {
      fail(qs, std::string("CUDA: ") + cudaGetErrorString(e));
      continue;
    }
    const auto t = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    for (Query* q : qs) {
      q->latency_ms = std::chrono::duration<double, std::milli>(t - q->submitted).count();
      q->done = true;
      q->x.clear();
      q->y.clear();
      latencies.push_back(q->latency_ms);
      admitted_bytes -= q->bytes;
    }
    last_done = t;
    done_cv.notify_all();
  }
}

void hedap_server::loop() {
  cudaSetDevice(C->device);
  size_t rr = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stop || (!waiting.empty() && !paused) || !groups.empty() || !pending.empty(); });
      if (stop && waiting.empty() && groups.empty() && pending.empty()) return;
      // the oldest waiting query, then the later ones that can share its group
      std::unique_ptr<Group> g(new Group);
      for (auto it = waiting.begin(); !paused && it != waiting.end() && g->q.size() < cfg.max_batch;) {
        Query* q = *it;
        if (!g->q.empty() && !same_group(*q, *g->q[0])) {
          ++it;
          continue;
        }
        if (admitted_bytes + q->bytes > cfg.hbm_budget_bytes) break;
        it = waiting.erase(it);
        admitted_bytes += q->bytes;
        g->q.push_back(q);
      }
      for (Query* q : g->q) q->group_size = (uint32_t)g->q.size();
      if (!g->q.empty()) groups.push_back(std::move(g));
    }
    if (!groups.empty()) {
      rr %= groups.size();
      Group& g = *groups[rr];
      try {
        std::lock_guard<std::mutex> lk(C->mu);
        step(g);
        if (g.step < 0) {
          Pending p;
          HEDAP_CUDA(cudaEventCreateWithFlags(&p.ev, cudaEventDisableTiming));
          HEDAP_CUDA(cudaEventRecord(p.ev, C->stream));
          p.q = g.q;
          pending.push_back(std::move(p));
        }
      } catch (const std::exception& e) {
        fail(g.q, e.what());
        g.step = -1;
      }
      if (g.step < 0)
        groups.erase(groups.begin() + (long)rr);
      else
        ++rr;
    }
    // with nothing to issue (waiting queries, if any, wait for memory), wait
    // for the oldest finished group on the GPU
    retire(groups.empty());
  }
}

#define API extern "C" __attribute__((visibility("default")))

namespace {
template <class F>
hedap_status srv_guard(F&& f) {
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
}  // namespace

API hedap_status hedap_server_create(hedap_ctx* ctx, const hedap_server_cfg* cfg, hedap_server** out) {
  return srv_guard([&] {
    if (!ctx || !cfg || !out) throw Error(HEDAP_ERR_ARG, "null argument");
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > 16) throw Error(HEDAP_ERR_ARG, "max_batch must lie in [1, 16]");
    Ctx& C = *ctx->c;
    {
      // the power-of-two rotation keys of rotate-and-sum stay resident from here on
      std::lock_guard<std::mutex> lk(C.mu);
      for (size_t r = 1; r < C.N / 2; r <<= 1) gen_galois_key(C, galois_for_rotation(C, (i64)r));
      HEDAP_CUDA(cudaStreamSynchronize(C.stream));
    }
    std::unique_ptr<hedap_server> s(new hedap_server);
    s->C = &C;
    s->cfg = *cfg;
    s->paused = cfg->start_paused != 0;
    hedap_server* p = s.get();
    s->worker = std::thread([p] { p->loop(); });
    *out = s.release();
  });
}

API hedap_status hedap_server_submit(hedap_server* s, const hedap_query* q, uint64_t* id) {
  return srv_guard([&] {
    if (!s || !q || !id || !q->x || q->n_ct == 0 || q->n_records == 0) throw Error(HEDAP_ERR_ARG, "bad query");
    if (q->kind != HEDAP_QUERY_ZSCORE && q->kind != HEDAP_QUERY_PCC) throw Error(HEDAP_ERR_ARG, "unknown query kind");
    const bool pcc = q->kind == HEDAP_QUERY_PCC;
    if (pcc && !q->y) throw Error(HEDAP_ERR_ARG, "a correlation query needs y");
    if (q->n_records > (uint64_t)q->n_ct * (s->C->N / 2)) throw Error(HEDAP_ERR_ARG, "more records than slots");
    std::unique_ptr<Query> Q(new Query);
    Q->kind = q->kind;
    Q->n_records = q->n_records;
    Q->cfg = q->invsqrt;
    for (uint32_t k = 0; k < q->n_ct; ++k) {
      for (int side = 0; side < (pcc ? 2 : 1); ++side) {
        const hedap_ct* c = side ? q->y[k] : q->x[k];
        if (!c || c->c->batch != 1) throw Error(HEDAP_ERR_ARG, "query inputs must be single ciphertexts");
        if (k + side > 0 && (c->c->level != Q->level || c->c->scale != Q->scale))
          throw Error(HEDAP_ERR_ARG, "query inputs must share one level and scale");
        Q->level = c->c->level;
        Q->scale = c->c->scale;
        (side ? Q->y : Q->x).push_back(c->c.get());
      }
    }
    if (Q->level < 4) throw Error(HEDAP_ERR_LEVEL, "query inputs need level >= 4");
    if (q->choice) {  // (degree, c, iters) from the HE-DAP table for the variance's level
      if (q->choice > 3) throw Error(HEDAP_ERR_ARG, "query choice must be 0, 1, 2 or 3");
      const int vlevel = Q->level - (pcc ? 3 : 2);
      std::lock_guard<std::mutex> lk(s->mu);
      const hedap_select_entry* best = nullptr;
      for (const hedap_select_entry& e : s->table)
        if (e.kind == q->choice && e.level <= vlevel && (!best || e.level > best->level)) best = &e;
      if (!best) throw Error(HEDAP_ERR_ARG, "no HE-DAP table entry of that kind at or below the variance's level");
      Q->cfg.degree = best->degree;
      Q->cfg.pre_bts = best->c;
      Q->cfg.newton_iters = best->iters;
      Q->cfg.bts_mask = s->C->bts ? (1ull << 63) : 0;
    }
    Q->bytes = s->estimate_bytes(pcc ? 1 : q->n_ct, Q->level);
    if (Q->bytes > s->cfg.hbm_budget_bytes) throw Error(HEDAP_ERR_OOM, "query exceeds the server's memory budget");
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->stop) throw Error(HEDAP_ERR_ARG, "server is stopping");
      Q->submitted = Clock::now();
      if (!s->any) {
        s->first_submit = Q->submitted;
        s->any = true;
      }
      Q->id = s->next_id++;
      *id = Q->id;
      s->waiting.push_back(Q.get());
      s->all[Q->id] = std::move(Q);
    }
    s->cv.notify_all();
  });
}

API hedap_status hedap_server_poll(hedap_server* s, uint64_t id, int wait, int* done, hedap_ct** out, size_t cap,
                                   size_t* n_out, double* latency_ms, uint32_t* group_size) {
  return srv_guard([&] {
    if (!s || !done) throw Error(HEDAP_ERR_ARG, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) throw Error(HEDAP_ERR_ARG, "unknown query id");
    Query* q = it->second.get();
    if (wait) s->done_cv.wait(lk, [&] { return q->done; });
    *done = q->done ? 1 : 0;
    if (!q->done) return;
    if (!q->error.empty()) {
      const std::string why = "query failed: " + q->error;
      s->all.erase(it);
      throw Error(HEDAP_ERR_ARG, why);
    }
    if (n_out) *n_out = q->out.size();
    if (latency_ms) *latency_ms = q->latency_ms;
    if (group_size) *group_size = q->group_size;
    if (out) {
      if (cap < q->out.size()) throw Error(HEDAP_ERR_ARG, "output capacity too small");
      for (size_t k = 0; k < q->out.size(); ++k) {
        out[k] = new hedap_ct;
        out[k]->c = std::move(q->out[k]);
      }
      s->all.erase(it);
    }
  });
}

API hedap_status hedap_server_stats(hedap_server* s, double* p50_ms, double* p99_ms, double* qps, uint64_t* completed) {
  return srv_guard([&] {
    if (!s) throw Error(HEDAP_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {  // linear interpolation between order statistics
      if (v.empty()) return 0.0;
      const double r = p * (double)(v.size() - 1);
      const size_t a = (size_t)r, b = std::min(a + 1, v.size() - 1);
      return v[a] + (v[b] - v[a]) * (r - (double)a);
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (completed) *completed = v.size();
    if (qps) {
      const double span =
          s->any && !v.empty() ? std::chrono::duration<double>(s->last_done - s->first_submit).count() : 0;
      *qps = span > 0 ? (double)v.size() / span : 0;
    }
  });
}

API hedap_status hedap_server_resume(hedap_server* s) {
  return srv_guard([&] {
    if (!s) throw Error(HEDAP_ERR_ARG, "null argument");
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->paused = false;
    }
    s->cv.notify_all();
  });
}

API hedap_status hedap_server_set_table(hedap_server* s, const hedap_select_entry* R, size_t n) {
  return srv_guard([&] {
    if (!s || (n && !R)) throw Error(HEDAP_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->table.assign(R, R + n);
  });
}

API hedap_status hedap_server_estimate(const hedap_server* s, uint32_t kind, uint32_t n_ct, int level,
                                       uint64_t* bytes) {
  return srv_guard([&] {
    if (!s || !bytes || level < 0 || level > s->C->L()) throw Error(HEDAP_ERR_ARG, "bad argument");
    if (kind != HEDAP_QUERY_ZSCORE && kind != HEDAP_QUERY_PCC) throw Error(HEDAP_ERR_ARG, "unknown query kind");
    *bytes = s->estimate_bytes(kind == HEDAP_QUERY_PCC ? 1 : n_ct, level);
  });
}

API void hedap_server_destroy(hedap_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->paused = false;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
}
