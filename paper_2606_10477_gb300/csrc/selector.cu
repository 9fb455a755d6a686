// HE-DAP provisioning (Sec. 4.2): Alg. 2 (GetOptIter) and Alg. 3 (per-level
// choice of degree d, Pre-BTS flag c and Newton iterations i), run on this
// library with costs measured on the GPU.
//
// Readings where the paper is silent:
//  - MRE is the mean relative error over the N/2 slots against FP64 1/sqrt.
//  - T[i] times only the HE operations (CUDA events), not Dec or GetMRE; for
//    c = 1 it includes the Pre-BTS, and for both it includes the
//    pre-normalisation step.
//  - The exponent l and mantissa alpha of MRE_min come from the shortest
//    decimal representation that round-trips the double (so that 3e-8 has
//    floor(alpha) = 3 exactly); MRE_delta = (floor(alpha) + delta) 10^l.
//  - Alg. 3's argmins break ties by smaller t, then smaller d, then c = 0,
//    then smaller i.  A third choice u3 minimises t subject to an absolute MRE
//    target when one is given.
//  - l_BTS = 1 in this library (the scaling into [-1, 1] before BTS takes one
//    level); profiled levels run from l_BTS + 1 to the highest level a
//    bootstrapped ciphertext has (or the top level without bootstrapping).
#include <charconv>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "internal.cuh"

namespace hedap {

// floor(alpha) and l of v = alpha * 10^l, 1 <= alpha < 10, from the shortest round-trip decimal
static void decimal_split(double v, int* lead, int* ell) {
  char buf[64];
  auto r = std::to_chars(buf, buf + sizeof(buf), v, std::chars_format::scientific);
  *r.ptr = 0;
  *lead = buf[0] - '0';
  const char* e = std::strchr(buf, 'e');
  *ell = e ? std::atoi(e + 1) : 0;
}
// (lead + delta) * 10^ell: exactly the nearest double to the decimal when delta is an integer
static double threshold(int lead, int ell, double delta) {
  if (delta == std::floor(delta) && std::fabs(delta) < 1e6) {
    char buf[64];
    std::snprintf(buf, sizeof(buf), "%lde%d", (long)(lead + (long)delta), ell);
    return std::strtod(buf, nullptr);
  }
  return (lead + delta) * std::pow(10.0, ell);
}

// Alg. 2, last lines: smallest i with M[i] <= MRE_delta (0-based; -1 when M has no finite value)
int getoptiter_rule(const double* M, size_t n, double delta, double* thr_out) {
  double mmin = INFINITY;
  for (size_t i = 0; i < n; ++i)
    if (M[i] < mmin) mmin = M[i];
  if (!std::isfinite(mmin)) return -1;
  double thr = 0;
  if (mmin > 0) {
    int lead, ell;
    decimal_split(mmin, &lead, &ell);
    thr = threshold(lead, ell, delta);
  }
  if (thr_out) *thr_out = thr;
  for (size_t i = 0; i < n; ++i)
    if (M[i] <= thr) return (int)i;
  return -1;
}

static bool better(const hedap_select_entry& a, const hedap_select_entry& b) {
  if (a.ms != b.ms) return a.ms < b.ms;
  if (a.degree != b.degree) return a.degree < b.degree;
  if (a.c != b.c) return a.c < b.c;
  return a.iters < b.iters;
}

// Alg. 3, per level: u1 = fastest with m <= m_theta, u2 = fastest, u3 = fastest with m <= target
int level_rule(const hedap_select_entry* D, size_t n, double theta, double target, hedap_select_entry* u1,
               hedap_select_entry* u2, hedap_select_entry* u3) {
  if (n == 0) return -1;
  double mmin = INFINITY;
  for (size_t k = 0; k < n; ++k) mmin = std::min(mmin, D[k].mre);
  double mth = 0;
  if (mmin > 0 && std::isfinite(mmin)) {
    int lead, ell;
    decimal_split(mmin, &lead, &ell);
    mth = threshold(lead, ell, theta);
  }
  bool h1 = false, h2 = false, h3 = false;
  for (size_t k = 0; k < n; ++k) {
    const hedap_select_entry& e = D[k];
    if (e.mre <= mth && (!h1 || better(e, *u1))) { *u1 = e; h1 = true; }
    if (!h2 || better(e, *u2)) { *u2 = e; h2 = true; }
    if (target > 0 && e.mre <= target && (!h3 || better(e, *u3))) { *u3 = e; h3 = true; }
  }
  u1->kind = 1;
  u2->kind = 2;
  if (h3) u3->kind = 3;
  return h3 ? 1 : 0;
}

namespace {
struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    HEDAP_CUDA(cudaEventCreate(&a));
    HEDAP_CUDA(cudaEventCreate(&b));
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  void start() { HEDAP_CUDA(cudaEventRecord(a, s)); }
  float stop() {
    HEDAP_CUDA(cudaEventRecord(b, s));
    HEDAP_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    HEDAP_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
};
}  // namespace

// Alg. 2 for one (level, d, c): returns false when the configuration does not fit the chain
static bool get_opt_iter(Ctx& C, const Ct& ct, const std::vector<double>& vals, const hedap_select_cfg& sc,
                         uint32_t d, uint32_t c, std::vector<hedap_select_trace>& trace, hedap_select_entry* out) {
  hedap_invsqrt_cfg cfg{sc.A, sc.B_max, sc.B, d, 0, c, C.bts ? (1ull << 63) : 0ull};
  Timer tm(C.stream);
  double t_total = 0;
  std::unique_ptr<InvSqrtRun> run;
  try {
    tm.start();
    run.reset(new InvSqrtRun(C, ct, cfg));
    run->chebyshev();
    t_total += tm.stop();
  } catch (const Error& e) {
    if (e.code == HEDAP_ERR_LEVEL) return false;
    throw;
  }
  std::vector<double> M, T;
  std::vector<double> re, im;
  for (uint32_t i = 0; i < sc.i_max; ++i) {
    try {
      tm.start();
      run->newton((int)i);
      t_total += tm.stop();
    } catch (const Error& e) {
      if (e.code == HEDAP_ERR_LEVEL) break;
      throw;
    }
    auto y = run->result();
    decrypt(C, *y, re, im);
    double s = 0;
    for (size_t k = 0; k < vals.size(); ++k) {
      const double ref = 1.0 / std::sqrt(vals[k]);
      s += std::fabs(re[k] - ref) / ref;
    }
    const double mre = s / (double)vals.size();
    M.push_back(mre);
    T.push_back(t_total);
    trace.push_back(hedap_select_trace{ct.level, d, c, i + 1, mre, t_total});
  }
  const int I = getoptiter_rule(M.data(), M.size(), sc.delta, nullptr);
  if (I < 0) return false;
  *out = hedap_select_entry{ct.level, d, c, (uint32_t)I + 1, M[I], T[I], 0};
  return true;
}

// Alg. 3 over the profiled levels
void select(Ctx& C, const hedap_select_cfg& sc, std::vector<hedap_select_entry>& D,
            std::vector<hedap_select_entry>& R, std::vector<hedap_select_trace>& trace) {
  if (!(sc.A > 0) || !(sc.B_max > sc.A) || !(sc.B > 0) || sc.d_e_min < 1 || sc.d_e_max < sc.d_e_min ||
      sc.d_e_max > 12 || sc.i_max < 1 || sc.i_max > 62)
    throw Error(HEDAP_ERR_ARG, "select: invalid configuration");
  const int l_bts = 1;
  int l_after = C.L();
  if (C.bts) {  // the level a bootstrapped ciphertext has
    auto probe = ct_alloc(C, 0, 1);
    HEDAP_CUDA(cudaMemsetAsync(probe->buf.p, 0, probe->buf.words * 8, C.stream));
    probe->scale = (double)C.primes[0] / 4096.0;
    l_after = bootstrap_core(C, *probe)->level;
  }
  const int lmax = C.bts ? l_after : C.L();
  const int lo = std::max(l_bts + 1, sc.level_min > 0 ? sc.level_min : 0);
  const int hi = std::min(lmax, sc.level_max > 0 ? sc.level_max : lmax);
  const size_t n = C.N / 2;
  std::vector<double> vals(n), zero;
  for (size_t k = 0; k < n; ++k) vals[k] = sc.A + (sc.B_max - sc.A) * (double)k / (double)(n - 1);  // linspace
  for (int l = lo; l <= hi; ++l) {
    std::vector<hedap_select_entry> Dl;
    for (uint32_t de = sc.d_e_min; de <= sc.d_e_max; ++de) {
      const uint32_t d = (1u << de) - 2;
      auto ct = encrypt(C, vals, zero, l, sc.seed + (uint64_t)l * 64 + de);
      hedap_select_entry e;
      if (l >= l_bts + 3 && get_opt_iter(C, *ct, vals, sc, d, 0, trace, &e)) Dl.push_back(e);
      if (C.bts && l < l_after - 1 && get_opt_iter(C, *ct, vals, sc, d, 1, trace, &e)) Dl.push_back(e);
    }
    D.insert(D.end(), Dl.begin(), Dl.end());
    hedap_select_entry u1{}, u2{}, u3{};
    const int r = level_rule(Dl.data(), Dl.size(), sc.theta, sc.mre_target, &u1, &u2, &u3);
    if (r < 0) continue;
    R.push_back(u1);
    R.push_back(u2);
    if (r == 1) R.push_back(u3);
  }
}

}  // namespace hedap
