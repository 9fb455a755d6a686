#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "profiler.cuh"

namespace hedap {

namespace {
std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_on{false};
std::mutex g_mu;
struct Rec {
  int cls;
  double bytes, slots;
  cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free;
double g_ms[PROF_N_CLASSES], g_bytes[PROF_N_CLASSES], g_slots[PROF_N_CLASSES];
uint64_t g_scopes[PROF_N_CLASSES];
const char* kNames[PROF_N_CLASSES] = {"ntt", "modup", "ksk_inner", "moddown", "tensor", "rescale", "automorph",
                                      "elementwise"};

cudaEvent_t get_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
void drain() {  // caller holds g_mu
  for (auto& r : g_recs) {
    cudaEventSynchronize(r.b);
    float ms = 0;
    cudaEventElapsedTime(&ms, r.a, r.b);
    g_ms[r.cls] += ms;
    g_bytes[r.cls] += r.bytes;
    g_slots[r.cls] += r.slots;
    g_scopes[r.cls] += 1;
    g_free.push_back(r.a);
    g_free.push_back(r.b);
  }
  g_recs.clear();
}
}  // namespace

void prof_count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
uint64_t prof_launches() { return g_launches.load(); }
void prof_enable(bool on) { g_on.store(on); }
bool prof_enabled() { return g_on.load(); }
void prof_reset() {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  memset(g_ms, 0, sizeof(g_ms));
  memset(g_bytes, 0, sizeof(g_bytes));
  memset(g_slots, 0, sizeof(g_slots));
  memset(g_scopes, 0, sizeof(g_scopes));
}
void prof_read(int cls, uint64_t* scopes, double* ms, double* bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  if (cls < 0 || cls >= PROF_N_CLASSES) return;
  if (scopes) *scopes = g_scopes[cls];
  if (ms) *ms = g_ms[cls];
  if (bytes) *bytes = g_bytes[cls];
}
double prof_read_slots(int cls) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  return cls >= 0 && cls < PROF_N_CLASSES ? g_slots[cls] : 0.0;
}
int prof_class_of(const char* name) {
  for (int i = 0; i < PROF_N_CLASSES; ++i)
    if (!strcmp(name, kNames[i])) return i;
  return -1;
}

ProfScope::ProfScope(int cls_, cudaStream_t st_, double bytes_) : cls(cls_), st(st_), bytes(bytes_) {
  if (!g_on.load()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  a = get_event();
  b = get_event();
  cudaEventRecord(a, st);
}
ProfScope::~ProfScope() {
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(b, st);
  g_recs.push_back(Rec{cls, bytes, slots, a, b});
  if (g_recs.size() > 8192) drain();
}

}  // namespace hedap
