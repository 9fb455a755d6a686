// Serving: a continuous-batching request loop for encrypted statistical
// queries that each need the inverse square root of an encrypted variance
// (the statistical workloads of Sec. 5.3: Z-score normalisation and the
// Pearson correlation coefficient).
//
// One worker thread drives the context.  Submitted queries wait in a FIFO; the
// worker admits the oldest waiting query and the later ones that can share its
// group (one kind, input level, input scale and InvSqrt configuration; up to
// max_batch) while the estimated device memory of the admitted queries stays
// within the budget.  A group is a batch advanced one step at a time:
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
// Every group runs on a CUDA stream of its own (from the context's pool), so the
// work of groups in flight overlaps on the device.  A group's next step is issued
// once its previous one has finished on the device (an event per step): groups
// move at the device's pace, and a group admitted later can catch up with an
// earlier one that needs the same steps.  At every step boundary groups with the
// same signature at the same step are merged into one batch (up to max_batch):
// a group with a partner further ahead (by at most kCatchUp steps) is stepped
// first while the partner waits, and the two become one group when they meet.
// Batched operations equal single operations bit for bit and every decision (a
// bootstrap, a level drop) is a function of the group's common kind, level and
// configuration, so a query's result does not depend on which other queries share
// its group, on merging, or on the GPU.
//
// Host-side failure handling: hedap_server_cancel withdraws a query (waiting: at
// once; in flight: at its group's next step boundary, the group dropped when
// every query in it is withdrawn); hedap_server_inject makes the next admissions
// fail as an allocation failure would (their queries end with HEDAP_ERR_OOM and
// the server goes on); hedap_server_wait bounds the host's wait for a query
// (HEDAP_ERR_TIMEOUT).  None of them touches the GPU.
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
  bool cancelled = false;  // withdrawn (hedap_server_cancel); ends with HEDAP_ERR_CANCELLED
  std::string error;
  hedap_status error_code = HEDAP_OK;
};

bool same_group(const Query& a, const Query& b) {
  return a.kind == b.kind && a.level == b.level && a.scale == b.scale && same_cfg(a.cfg, b.cfg);
}

struct Group {
  std::vector<Query*> q;
  int step = 0;  // 0 stats, 1 prepare, 2 chebyshev, 3 .. 2+iters newton, then finish; -1 finished
  std::unique_ptr<InvSqrtRun> run;
  cudaStream_t st = nullptr;  // the group's stream (context pool)
  cudaEvent_t ev = nullptr;   // recorded after each issued step
  bool in_flight = false;     // a step was issued and its event has not been seen complete
  uint64_t seq = 0;           // admission order
};

// the steps a group of this configuration goes through before `finish`
int finish_step(const Query& q) { return 3 + (int)q.cfg.newton_iters; }

// a group's buffers now belong to stream s: their stream-ordered frees go there
void rehome(Ct* c, cudaStream_t s) {
  if (c) c->buf.s = s;
}

constexpr int kCatchUp = 3;  // steps a group waits at most for a later partner with its signature

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
  std::mutex mu;  // guards everything below but groups (worker-only; the context has its own lock)
  std::condition_variable cv, done_cv;
  std::deque<Query*> waiting;
  std::map<uint64_t, std::unique_ptr<Query>> all;
  std::vector<std::unique_ptr<Group>> groups;  // worker-only: admitted, in flight or finishing
  size_t admitted_bytes = 0;
  uint64_t next_id = 1, next_seq = 1;
  uint32_t inject_admission_oom = 0;  // fault injection: admissions still to fail
  bool stop = false;
  bool paused = false;
  std::thread worker;
  std::vector<double> latencies;
  Clock::time_point first_submit, last_done;
  bool any = false;
  std::vector<hedap_select_entry> table;  // HE-DAP per-level choices (guarded by mu)
  uint64_t merges = 0;                    // groups merged into others (guarded by mu)

  size_t estimate_bytes(size_t n_out, int level) const;
  void loop();
  void step(Group& g);
  void issue(Group& g);
  bool merge_ready();
  Group* pick();
  bool retire_finished();
  void end(Group& g, hedap_status code, const std::string& why);
  void fail(const std::vector<Query*>& qs, hedap_status code, const std::string& why);
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

void hedap_server::fail(const std::vector<Query*>& qs, hedap_status code, const std::string& why) {
  std::lock_guard<std::mutex> lk(mu);
  for (Query* q : qs) {
    if (q->done) continue;
    q->error = why;
    q->error_code = code;
    q->done = true;
    q->out.clear();
    q->mean_x.reset();
    q->cov.reset();
    q->var.reset();
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

// issue the group's next step on its own stream (the context's stream swapped in under the context's
// lock), followed by its event
void hedap_server::issue(Group& g) {
  Ctx& Cx = *C;
  std::lock_guard<std::mutex> lk(Cx.mu);
  Cx.stream = g.st;
  try {
    step(g);
    HEDAP_CUDA(cudaEventRecord(g.ev, g.st));
    g.in_flight = true;
  } catch (...) {
    Cx.stream = Cx.home;
    throw;
  }
  Cx.stream = Cx.home;
}

// merge groups that are idle on the device, share a signature and stand at the same step (after the
// statistics, before the finish); the older group absorbs the younger.  Returns whether any merged.
bool hedap_server::merge_ready() {
  bool merged = false;
  for (size_t a = 0; a < groups.size(); ++a) {
    Group& A = *groups[a];
    if (A.in_flight || A.step < 1 || A.step >= finish_step(*A.q[0])) continue;
    for (size_t b = a + 1; b < groups.size();) {
      Group& B = *groups[b];
      if (B.in_flight || B.step != A.step || !same_group(*A.q[0], *B.q[0]) ||
          A.q.size() + B.q.size() > cfg.max_batch) {
        ++b;
        continue;
      }
      Ctx& Cx = *C;
      std::lock_guard<std::mutex> lk(Cx.mu);
      // A's stream takes over B's state: it waits for B's work, copies, and B's old buffers are freed
      // on A's stream after the copies
      HEDAP_CUDA(cudaStreamWaitEvent(A.st, B.ev, 0));
      for (Query* q : B.q) {
        rehome(q->mean_x.get(), A.st);
        rehome(q->cov.get(), A.st);
        rehome(q->var.get(), A.st);
      }
      if (A.step >= 2) {  // InvSqrt's state: t, x, y of the two batches packed into one
        Cx.stream = A.st;
        try {
          InvSqrtRun& ra = *A.run;
          InvSqrtRun& rb = *B.run;
          for (std::unique_ptr<Ct>* f : {&ra.t, &ra.x, &ra.y}) {
            std::unique_ptr<Ct>& fb = f == &ra.t ? rb.t : f == &ra.x ? rb.x : rb.y;
            if (!*f) continue;
            rehome(f->get(), A.st);
            rehome(fb.get(), A.st);
            *f = batch_pack(Cx, {f->get(), fb.get()});
          }
        } catch (...) {
          Cx.stream = Cx.home;
          throw;
        }
        Cx.stream = Cx.home;
        B.run.reset();
      }
      A.q.insert(A.q.end(), B.q.begin(), B.q.end());
      HEDAP_CUDA(cudaEventDestroy(B.ev));
      Cx.streams.put(B.st);
      groups.erase(groups.begin() + (long)b);
      {
        std::lock_guard<std::mutex> lk2(mu);
        ++merges;
      }
      merged = true;
    }
  }
  return merged;
}

// the next group to step: idle on the device and not waiting for a partner to catch up (a partner:
// same signature, room for both in one batch, and either a few steps behind or at the same step with
// that step still running on the device -- `step` counts issued steps); the most behind first
Group* hedap_server::pick() {
  Group* best = nullptr;
  for (auto& gp : groups) {
    Group& g = *gp;
    if (g.in_flight || g.step < 0) continue;
    bool wait = false;
    if (g.step >= 1 && g.step < finish_step(*g.q[0]))
      for (auto& hp : groups) {
        const Group& h = *hp;
        if (&h == &g || h.step < 0 || !same_group(*g.q[0], *h.q[0]) || g.q.size() + h.q.size() > cfg.max_batch)
          continue;
        if ((h.step < g.step && g.step - h.step <= kCatchUp) || (h.step == g.step && h.in_flight)) {
          wait = true;
          break;
        }
      }
    if (wait) continue;
    if (!best || g.step < best->step || (g.step == best->step && g.seq < best->seq)) best = &g;
  }
  return best;
}

// a group leaves: its queries complete (code HEDAP_OK) or fail; its stream goes back to the pool
void hedap_server::end(Group& g, hedap_status code, const std::string& why) {
  const auto t = Clock::now();
  std::lock_guard<std::mutex> lk(mu);
  for (Query* q : g.q) {
    if (q->done) continue;
    q->group_size = (uint32_t)g.q.size();
    if (code != HEDAP_OK || q->cancelled) {
      q->error = code != HEDAP_OK ? why : "cancelled";
      q->error_code = code != HEDAP_OK ? code : HEDAP_ERR_CANCELLED;
      q->out.clear();
    } else {
      q->latency_ms = std::chrono::duration<double, std::milli>(t - q->submitted).count();
      latencies.push_back(q->latency_ms);
      for (auto& o : q->out) rehome(o.get(), C->home);  // the caller's buffers now: freed on its stream
      last_done = t;
    }
    q->mean_x.reset();
    q->cov.reset();
    q->var.reset();
    q->done = true;
    q->x.clear();
    q->y.clear();
    admitted_bytes -= q->bytes;
  }
  done_cv.notify_all();
}

// groups whose last issued step finished on the device: finished groups leave, the others become idle
bool hedap_server::retire_finished() {
  bool any_change = false;
  for (size_t i = 0; i < groups.size();) {
    Group& g = *groups[i];
    if (g.in_flight) {
      const cudaError_t e = cudaEventQuery(g.ev);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      g.in_flight = false;
      any_change = true;
      if (e != cudaSuccess) {
        g.step = -1;
        end(g, HEDAP_ERR_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
        cudaEventDestroy(g.ev);
        C->streams.put(g.st);
        groups.erase(groups.begin() + (long)i);
        continue;
      }
    }
    bool all_cancelled = true;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (Query* q : g.q) all_cancelled = all_cancelled && q->cancelled;
    }
    if (g.step < 0 || all_cancelled) {  // finished, or nobody wants the result any more
      {
        std::lock_guard<std::mutex> lk(C->mu);
        g.run.reset();  // freed on the group's stream, ordered after its work
      }
      end(g, HEDAP_OK, "");
      cudaEventDestroy(g.ev);
      C->streams.put(g.st);
      groups.erase(groups.begin() + (long)i);
      any_change = true;
      continue;
    }
    ++i;
  }
  return any_change;
}

void hedap_server::loop() {
  cudaSetDevice(C->device);
  for (;;) {
    std::vector<std::unique_ptr<Group>> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stop || (!waiting.empty() && !paused) || !groups.empty(); });
      if (stop && waiting.empty() && groups.empty()) return;
      // the oldest waiting query, then the later ones that can share its group
      const size_t admit = cfg.admit_max ? std::min(cfg.admit_max, cfg.max_batch) : cfg.max_batch;
      while (!paused && !waiting.empty()) {
        std::unique_ptr<Group> g(new Group);
        for (auto it = waiting.begin(); it != waiting.end() && g->q.size() < admit;) {
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
        if (g->q.empty()) break;
        g->seq = next_seq++;
        admitted.push_back(std::move(g));
      }
    }
    for (auto& g : admitted) {
      try {
        {
          std::lock_guard<std::mutex> lk(mu);
          if (inject_admission_oom > 0) {
            --inject_admission_oom;
            throw Error(HEDAP_ERR_OOM, "device allocation failed at admission (injected)");
          }
        }
        std::lock_guard<std::mutex> lk(C->mu);
        g->st = C->streams.get();
        HEDAP_CUDA(cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming));
        // the inputs were made on the context's stream: the group's stream starts after that work
        HEDAP_CUDA(cudaEventRecord(g->ev, C->home));
        HEDAP_CUDA(cudaStreamWaitEvent(g->st, g->ev, 0));
        groups.push_back(std::move(g));
      } catch (const Error& e) {
        fail(g->q, e.code, e.what());
        if (g->ev) cudaEventDestroy(g->ev);
        if (g->st) C->streams.put(g->st);
      }
    }
    bool progressed = retire_finished();
    progressed = merge_ready() || progressed;
    if (Group* g = pick()) {
      try {
        issue(*g);
      } catch (const Error& e) {
        g->step = -1;
        end(*g, e.code, e.what());
      } catch (const std::exception& e) {
        g->step = -1;
        end(*g, HEDAP_ERR_ARG, e.what());
      }
      progressed = true;
    }
    if (!progressed) {
      // nothing to issue until a step in flight finishes or a query arrives: poll again shortly (a step
      // takes milliseconds on the device; the worker must notice whichever group finishes first)
      std::unique_lock<std::mutex> lk(mu);
      cv.wait_for(lk, std::chrono::microseconds(50));
    }
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
    Ctx& C = ctx_of(ctx);
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
        const Ct& c = ct_of(nullptr, side ? q->y[k] : q->x[k]);
        if (c.owner != s->C) throw Error(HEDAP_ERR_ARG, "query input made by another context");
        if (c.batch != 1) throw Error(HEDAP_ERR_ARG, "query inputs must be single ciphertexts");
        if (k + side > 0 && (c.level != Q->level || c.scale != Q->scale))
          throw Error(HEDAP_ERR_ARG, "query inputs must share one level and scale");
        Q->level = c.level;
        Q->scale = c.scale;
        (side ? Q->y : Q->x).push_back(&c);
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
      const hedap_status code = q->error_code != HEDAP_OK ? q->error_code : HEDAP_ERR_ARG;
      s->all.erase(it);
      throw Error(code, why);
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

API hedap_status hedap_server_wait(hedap_server* s, uint64_t id, double timeout_ms) {
  return srv_guard([&] {
    if (!s || !(timeout_ms >= 0)) throw Error(HEDAP_ERR_ARG, "bad argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) throw Error(HEDAP_ERR_ARG, "unknown query id");
    Query* q = it->second.get();
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double, std::milli>(timeout_ms));
    if (!s->done_cv.wait_until(lk, until, [&] { return q->done; }))
      throw Error(HEDAP_ERR_TIMEOUT, "query not done within the timeout");
  });
}

API hedap_status hedap_server_cancel(hedap_server* s, uint64_t id) {
  return srv_guard([&] {
    if (!s) throw Error(HEDAP_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) throw Error(HEDAP_ERR_ARG, "unknown query id");
    Query* q = it->second.get();
    if (q->done) throw Error(HEDAP_ERR_ARG, "query already finished");
    q->cancelled = true;
    auto w = std::find(s->waiting.begin(), s->waiting.end(), q);
    if (w != s->waiting.end()) {  // not admitted yet: withdrawn at once
      s->waiting.erase(w);
      q->done = true;
      q->error = "cancelled";
      q->error_code = HEDAP_ERR_CANCELLED;
      q->x.clear();
      q->y.clear();
      s->done_cv.notify_all();
    }
  });
}

API hedap_status hedap_server_inject(hedap_server* s, uint32_t fault, uint32_t count) {
  return srv_guard([&] {
    if (!s) throw Error(HEDAP_ERR_ARG, "null argument");
    if (fault != HEDAP_FAULT_ADMISSION_OOM) throw Error(HEDAP_ERR_ARG, "unknown fault");
    std::lock_guard<std::mutex> lk(s->mu);
    s->inject_admission_oom = count;
  });
}

API hedap_status hedap_server_merges(hedap_server* s, uint64_t* merged) {
  return srv_guard([&] {
    if (!s || !merged) throw Error(HEDAP_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *merged = s->merges;
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
