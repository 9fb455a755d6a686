// ============================================================================
// ORACLE -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously-correct CPU implementation of the RNS-CKKS
// arithmetic that CryptoInvSqrt (Alg. 1) runs on, and of CryptoInvSqrt itself
// (Chebyshev initial value, Sec. 2.3; Newton iteration, Sec. 2.2).  Modular
// arithmetic uses unsigned __int128 and the '%' operator; floating point is
// FP64.  Nothing is blocked, fused or reordered for speed.
//
// Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
// load this library.  It shares no code, header or table generator with the
// GPU library; the two meet only through seeded inputs and compared outputs.
//
// The paper cites CKKS (Sec. 2.1) but states none of its ring-level details.
// The conventions implemented here are the textbook ones, fixed as follows:
//  * primes: for each requested bit size b, candidates 2^b + k*2N + 1 and
//    2^b - k*2N + 1 for k = 1, 2, ... (above first), first prime not yet used;
//  * psi: the first x^((q-1)/2N), x = 2, 3, ..., whose N-th power is -1;
//  * NTT: out[j] = sum_i a_i psi^(i(2 br(j) + 1)) (bit-reversed evaluation
//    order), inverse includes N^-1;
//  * slots: z_j = m(zeta^(5^j)), zeta = exp(i pi / N) (CKKS canonical
//    embedding restricted to the 5^j orbit);
//  * rescale and ModDown round to nearest (centred remainders);
//  * key switching: hybrid, digits of alpha consecutive Q primes (Han-Ki 2020);
//  * bootstrapping's linear transforms: baby-step / giant-step sums (Halevi-
//    Shoup), the baby steps hoisted and kept over Q_l u P, one ModDown per giant
//    step (double hoisting, Bossuat, Mouchet, Troncoso-Pastoriza, Hubaux 2021);
//  * randomness: SplitMix64 (Steele, Lea, Flood 2014), one stream per object,
//    errors from the centred binomial distribution with eta = 21 (sigma ~ 3.24,
//    Alkim et al. 2016), ternary secrets dense or of fixed Hamming weight.
// ============================================================================
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;
typedef std::complex<double> cd;
typedef std::vector<u64> Limb;
typedef std::vector<Limb> Poly;  // [limb][coefficient]

static thread_local std::string g_err;

// Loops over independent RNS limbs may run on several host threads (OpenMP,
// when the compiler provides it); every limb is computed exactly as in the
// serial loop, so results do not depend on the thread count.
#define PER_LIMB _Pragma("omp parallel for schedule(dynamic)")

// ---------------------------------------------------------------- arithmetic
static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + (q - b); }
static u64 powmod(u64 a, u64 e, u64 q) {
  u64 r = 1 % q; a %= q;
  while (e) { if (e & 1) r = mulmod(r, a, q); a = mulmod(a, a, q); e >>= 1; }
  return r;
}
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }  // q prime
// signed integer -> residue
static u64 smod(i64 v, u64 q) {
  if (v >= 0) return (u64)v % q;
  u64 m = (u64)(-(v + 1)) % q;  // -(v+1) >= 0
  return submod(q - 1, m, q);   // v = -(m'+1)
}

// Exact residue of an integer-valued double.  |x| may exceed 2^63: write
// x = M * 2^e with M a 53-bit integer and reduce each factor.
static u64 double_to_mod(double x, u64 q) {
  bool neg = x < 0; double ax = std::fabs(x);
  u64 r;
  if (ax < 9.2e18) {
    r = (u64)ax % q;
  } else {
    int e; double m = std::frexp(ax, &e);  // ax = m * 2^e, m in [0.5,1)
    u64 M = (u64)std::ldexp(m, 53);        // exact
    r = mulmod(M % q, powmod(2, (u64)(e - 53), q), q);
  }
  return neg ? (r == 0 ? 0 : q - r) : r;
}
static double round_half_away(double x) { return std::round(x); }

// ---------------------------------------------------------------- primes
static bool is_prime(u64 n) {
  if (n < 2) return false;
  static const u64 sp[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 p : sp) { if (n % p == 0) return n == p; }
  u64 d = n - 1; int s = 0;
  while ((d & 1) == 0) { d >>= 1; ++s; }
  for (u64 a : sp) {  // deterministic for n < 2^64 (Jaeschke / Sorenson-Webster)
    u64 x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) { x = mulmod(x, x, n); if (x == n - 1) { comp = false; break; } }
    if (comp) return false;
  }
  return true;
}

static std::vector<u64> prime_chain(int log_n, const std::vector<int>& bits) {
  u64 two_n = 2ull << log_n;
  std::vector<u64> out;
  for (int b : bits) {
    if (b < log_n + 2 || b > 60) throw std::runtime_error("prime bit size out of range [log_n+2, 60]");
    u64 base = 1ull << b;
    for (u64 k = 1;; ++k) {
      u64 up = base + k * two_n + 1;
      if (is_prime(up) && std::find(out.begin(), out.end(), up) == out.end()) { out.push_back(up); break; }
      if (k * two_n < base) {
        u64 dn = base - k * two_n + 1;
        if (is_prime(dn) && std::find(out.begin(), out.end(), dn) == out.end()) { out.push_back(dn); break; }
      }
    }
  }
  return out;
}

static u64 find_psi(u64 q, int log_n) {
  u64 N = 1ull << log_n;
  for (u64 x = 2;; ++x) {
    u64 psi = powmod(x, (q - 1) / (2 * N), q);
    if (powmod(psi, N, q) == q - 1) return psi;
  }
}

static u64 bitrev(u64 x, int bits) {
  u64 r = 0;
  for (int i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

// ---------------------------------------------------------------- PRNG
// SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma, then the
// 64-bit finaliser.  A stream for (seed, tag) starts at
// mix64(seed) ^ mix64(tag ^ 0x5851F42D4C957F2D).
static u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
struct Stream {
  u64 s;
  Stream(u64 seed, u64 tag) : s(mix64(seed) ^ mix64(tag ^ 0x5851F42D4C957F2Dull)) {}
  u64 next() { s += 0x9E3779B97F4A7C15ull; return mix64(s); }
};
// object tags
static u64 tag_evk_a(u64 g, u64 j) { return (2ull << 56) | (g << 8) | j; }
static u64 tag_evk_e(u64 g, u64 j) { return (3ull << 56) | (g << 8) | j; }
static const u64 TAG_SK = 1, TAG_ENC_A = 4ull << 56, TAG_ENC_E = 5ull << 56, TAG_SK_SPARSE = 6ull << 56;

static u64 sample_uniform(Stream& st, u64 q) {
  int bits = 64 - __builtin_clzll(q);
  for (;;) { u64 x = st.next() >> (64 - bits); if (x < q) return x; }
}
// centred binomial, eta = 21: popcount of 21 low bits minus popcount of the next 21
static i64 sample_cbd(Stream& st) {
  u64 r = st.next();
  return (i64)__builtin_popcountll(r & 0x1FFFFFull) - (i64)__builtin_popcountll((r >> 21) & 0x1FFFFFull);
}
static std::vector<i64> sample_ternary(Stream& st, int log_n, int h) {
  size_t N = 1ull << log_n;
  std::vector<i64> s(N, 0);
  if (h == 0) {
    for (size_t i = 0; i < N; ++i) { u64 x; do { x = st.next() >> 62; } while (x >= 3); s[i] = (i64)x - 1; }
  } else {
    int cnt = 0;
    while (cnt < h) {
      u64 r = st.next(); u64 pos = r >> (64 - log_n);
      if (s[pos] == 0) { s[pos] = (r & 1) ? 1 : -1; ++cnt; }
    }
  }
  return s;
}

// ---------------------------------------------------------------- big integers (CRT)
struct Big {  // unsigned, little-endian 32-bit words
  std::vector<uint32_t> w;
  static Big from(u64 v) { Big b; b.w = {(uint32_t)v, (uint32_t)(v >> 32)}; b.trim(); return b; }
  void trim() { while (!w.empty() && w.back() == 0) w.pop_back(); }
};
static Big big_mul(const Big& a, u64 m) {
  Big r; u128 carry = 0;
  for (uint32_t x : a.w) { u128 t = (u128)x * m + carry; r.w.push_back((uint32_t)t); carry = t >> 32; }
  while (carry) { r.w.push_back((uint32_t)carry); carry >>= 32; }
  r.trim(); return r;
}
static Big big_add(const Big& a, const Big& b) {
  Big r; u64 c = 0; size_t n = std::max(a.w.size(), b.w.size());
  for (size_t i = 0; i < n; ++i) {
    u64 t = c + (i < a.w.size() ? a.w[i] : 0) + (i < b.w.size() ? b.w[i] : 0);
    r.w.push_back((uint32_t)t); c = t >> 32;
  }
  if (c) r.w.push_back((uint32_t)c);
  r.trim(); return r;
}
static int big_cmp(const Big& a, const Big& b) {
  if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
  for (size_t i = a.w.size(); i-- > 0;) if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}
static Big big_sub(const Big& a, const Big& b) {  // a >= b
  Big r; i64 br = 0;
  for (size_t i = 0; i < a.w.size(); ++i) {
    i64 t = (i64)a.w[i] - (i < b.w.size() ? (i64)b.w[i] : 0) - br;
    br = t < 0; if (t < 0) t += (1ll << 32);
    r.w.push_back((uint32_t)t);
  }
  r.trim(); return r;
}
static double big_to_double(const Big& a) {
  double r = 0;
  for (size_t i = a.w.size(); i-- > 0;) r = r * 4294967296.0 + (double)a.w[i];
  return r;
}

// ---------------------------------------------------------------- encoding
// Special FFT over the 5^j orbit (the CKKS decoding map), written as its
// radix-2 recursion: for a size-n problem with a root of order M = 4n,
//   z_j = E_j + w_j O_j,  z_{j+n/2} = E_j - w_j O_j,  w_j = exp(2 pi i 5^j / M),
// where E, O are the size-n/2 transforms of the even / odd inputs.
static std::vector<cd> special_fft(const std::vector<cd>& w, u64 M) {
  size_t n = w.size();
  if (n == 1) return w;
  std::vector<cd> ev(n / 2), od(n / 2);
  for (size_t k = 0; k < n / 2; ++k) { ev[k] = w[2 * k]; od[k] = w[2 * k + 1]; }
  std::vector<cd> E = special_fft(ev, M / 2), O = special_fft(od, M / 2), z(n);
  u64 g = 1;
  for (size_t j = 0; j < n / 2; ++j) {
    cd r = std::polar(1.0, 2.0 * M_PI * (double)g / (double)M);
    z[j] = E[j] + r * O[j];
    z[j + n / 2] = E[j] - r * O[j];
    g = (g * 5) % M;
  }
  return z;
}
static std::vector<cd> special_ifft(const std::vector<cd>& z, u64 M) {
  size_t n = z.size();
  if (n == 1) return z;
  std::vector<cd> E(n / 2), O(n / 2);
  u64 g = 1;
  for (size_t j = 0; j < n / 2; ++j) {
    cd r = std::polar(1.0, 2.0 * M_PI * (double)g / (double)M);
    E[j] = (z[j] + z[j + n / 2]) * 0.5;
    O[j] = (z[j] - z[j + n / 2]) * 0.5 / r;
    g = (g * 5) % M;
  }
  std::vector<cd> ev = special_ifft(E, M / 2), od = special_ifft(O, M / 2), w(n);
  for (size_t k = 0; k < n / 2; ++k) { w[2 * k] = ev[k]; w[2 * k + 1] = od[k]; }
  return w;
}

// ---------------------------------------------------------------- context
struct KeyDigit { Poly b, a; };  // NTT domain over all Q and P primes
struct Ctx {
  int log_n = 0; size_t N = 0; int n_q = 0, n_p = 0, alpha = 1; double scale = 0; int hw = 0; u64 seed = 0;
  std::vector<u64> q;                    // n_q + n_p primes (Q first, then P)
  std::vector<u64> psi;
  std::vector<Limb> psi_rev, ipsi_rev;  // per prime, psi^(br(i)) and psi^(-br(i))
  std::vector<u64> n_inv;
  std::vector<i64> s;                    // secret coefficients
  Poly s_ntt;                            // per prime
  std::map<u64, std::vector<KeyDigit>> keys;  // galois element (0 = relinearisation) -> digits
  // sparse-secret encapsulation of bootstrapping: ephemeral secret of weight enc_hw (0 = off);
  // key 2 switches from s to it, key 4 back (even ids are never Galois elements)
  int enc_hw = 0;
  std::vector<i64> s_sparse;
  Poly s_sparse_ntt;
  // bootstrapping: off unless configured; K bounds the ModRaise overflow |I| < K,
  // r double-angle steps, degree of the cosine interpolant, levels of CtS / StC
  bool bts_on = false;
  int bts_K = 28, bts_r = 4, bts_deg = 31, bts_cts = 3, bts_stc = 3;
  int L() const { return n_q - 1; }
};
struct Ct { Poly c[2]; int level = 0; double scale = 1; };

static void ntt_forward(const Ctx& C, Limb& a, int pi) {
  // Cooley-Tukey decimation in time with the psi twist merged into the twiddles
  u64 q = C.q[pi]; size_t N = C.N, t = N;
  for (size_t m = 1; m < N; m <<= 1) {
    t >>= 1;
    for (size_t i = 0; i < m; ++i) {
      u64 S = C.psi_rev[pi][m + i]; size_t j1 = 2 * i * t;
      for (size_t j = j1; j < j1 + t; ++j) {
        u64 U = a[j], V = mulmod(a[j + t], S, q);
        a[j] = addmod(U, V, q); a[j + t] = submod(U, V, q);
      }
    }
  }
}
static void ntt_inverse(const Ctx& C, Limb& a, int pi) {
  // Gentleman-Sande decimation in frequency, then multiplication by N^-1
  u64 q = C.q[pi]; size_t N = C.N, t = 1;
  for (size_t m = N >> 1; m >= 1; m >>= 1) {
    size_t j1 = 0;
    for (size_t i = 0; i < m; ++i) {
      u64 S = C.ipsi_rev[pi][m + i];
      for (size_t j = j1; j < j1 + t; ++j) {
        u64 U = a[j], V = a[j + t];
        a[j] = addmod(U, V, q); a[j + t] = mulmod(submod(U, V, q), S, q);
      }
      j1 += 2 * t;
    }
    t <<= 1;
  }
  for (size_t j = 0; j < N; ++j) a[j] = mulmod(a[j], C.n_inv[pi], q);
}

static Limb residues_of(const Ctx& C, const std::vector<i64>& v, int pi) {
  Limb r(C.N);
  for (size_t i = 0; i < C.N; ++i) r[i] = smod(v[i], C.q[pi]);
  return r;
}
// the evk digit j for a key switch from s' (NTT over all primes) to s_to
static KeyDigit make_key_digit(const Ctx& C, const Poly& sp, const Poly& s_to, u64 g, int j) {
  int total = C.n_q + C.n_p;
  KeyDigit kd; kd.a.assign(total, Limb(C.N)); kd.b.assign(total, Limb(C.N));
  Stream sa(C.seed, tag_evk_a(g, j));
  for (int t = 0; t < total; ++t) for (size_t i = 0; i < C.N; ++i) kd.a[t][i] = sample_uniform(sa, C.q[t]);
  Stream se(C.seed, tag_evk_e(g, j));
  std::vector<i64> e(C.N); for (size_t i = 0; i < C.N; ++i) e[i] = sample_cbd(se);
  int lo = j * C.alpha, hi = std::min(lo + C.alpha, C.n_q);
  PER_LIMB
  for (int t = 0; t < total; ++t) {
    u64 qt = C.q[t];
    Limb et = residues_of(C, e, t); ntt_forward(C, et, t);
    u64 Pmod = 1 % qt;
    for (int k = 0; k < C.n_p; ++k) Pmod = mulmod(Pmod, C.q[C.n_q + k] % qt, qt);
    bool in_digit = t >= lo && t < hi;
    for (size_t i = 0; i < C.N; ++i) {
      u64 v = submod(et[i], mulmod(kd.a[t][i], s_to[t][i], qt), qt);
      if (in_digit) v = addmod(v, mulmod(Pmod, sp[t][i], qt), qt);
      kd.b[t][i] = v;
    }
  }
  return kd;
}
static int n_digits(const Ctx& C, int level) { return (level + 1 + C.alpha - 1) / C.alpha; }

static u64 galois_of_rotation(const Ctx& C, i64 r) {
  u64 M = 2 * C.N, h = C.N / 2;
  i64 rr = ((r % (i64)h) + (i64)h) % (i64)h;
  return powmod(5, (u64)rr, M);
}
// coefficient-domain automorphism X -> X^g (g odd)
static Limb automorph_coeff(const Ctx& C, const Limb& a, u64 g, u64 q) {
  Limb r(C.N, 0); u64 M = 2 * C.N;
  for (size_t i = 0; i < C.N; ++i) {
    u64 e = (u64)(((u128)i * g) % M);
    if (e < C.N) r[e] = a[i]; else r[e - C.N] = a[i] == 0 ? 0 : q - a[i];
  }
  return r;
}

static void gen_key(Ctx& C, u64 g) {
  if (C.keys.count(g)) return;
  int total = C.n_q + C.n_p;
  Poly sp(total);
  PER_LIMB
  for (int t = 0; t < total; ++t) {
    if (g == 0) {  // relinearisation: s^2
      sp[t].resize(C.N);
      for (size_t i = 0; i < C.N; ++i) sp[t][i] = mulmod(C.s_ntt[t][i], C.s_ntt[t][i], C.q[t]);
    } else {       // s(X^g)
      Limb sc = residues_of(C, C.s, t);
      sp[t] = automorph_coeff(C, sc, g, C.q[t]);
      ntt_forward(C, sp[t], t);
    }
  }
  std::vector<KeyDigit> ds;
  for (int j = 0; j < n_digits(C, C.L()); ++j) ds.push_back(make_key_digit(C, sp, C.s_ntt, g, j));
  C.keys[g] = std::move(ds);
}
// Sparse-secret encapsulation (Bossuat, Troncoso-Pastoriza, Hubaux 2022): an
// ephemeral ternary secret with exactly h non-zero coefficients and the keys
// s -> s~ (id 2) and s~ -> s (id 4)
static void encapsulate(Ctx& C, int h) {
  if (h < 1 || (size_t)h > C.N) throw std::runtime_error("encapsulation weight out of range");
  int total = C.n_q + C.n_p;
  Stream st(C.seed, TAG_SK_SPARSE);
  std::vector<i64> v = sample_ternary(st, C.log_n, h);
  C.s_sparse = v;
  C.s_sparse_ntt.assign(total, Limb());
  for (int t = 0; t < total; ++t) { C.s_sparse_ntt[t] = residues_of(C, v, t); ntt_forward(C, C.s_sparse_ntt[t], t); }
  std::vector<KeyDigit> to_sparse, to_dense;
  for (int j = 0; j < n_digits(C, C.L()); ++j) {
    to_sparse.push_back(make_key_digit(C, C.s_ntt, C.s_sparse_ntt, 2, j));
    to_dense.push_back(make_key_digit(C, C.s_sparse_ntt, C.s_ntt, 4, j));
  }
  C.keys[2] = std::move(to_sparse);
  C.keys[4] = std::move(to_dense);
  C.enc_hw = h;
}

static Ctx* ctx_create(int log_n, const std::vector<int>& qb, const std::vector<int>& pb, int alpha,
                       double log_scale, int hw, u64 seed) {
  if (log_n < 3 || log_n > 17) throw std::runtime_error("log_n out of range");
  if (qb.empty() || pb.empty() || alpha < 1) throw std::runtime_error("bad prime counts");
  std::unique_ptr<Ctx> C(new Ctx);
  C->log_n = log_n; C->N = 1ull << log_n; C->n_q = (int)qb.size(); C->n_p = (int)pb.size();
  C->alpha = alpha; C->scale = std::pow(2.0, log_scale); C->hw = hw; C->seed = seed;
  std::vector<int> all = qb; all.insert(all.end(), pb.begin(), pb.end());
  C->q = prime_chain(log_n, all);
  int total = (int)C->q.size();
  C->psi.resize(total); C->psi_rev.resize(total); C->ipsi_rev.resize(total); C->n_inv.resize(total);
  PER_LIMB
  for (int t = 0; t < total; ++t) {
    u64 q = C->q[t], psi = find_psi(q, log_n), ipsi = invmod(psi, q);
    C->psi[t] = psi;
    C->psi_rev[t].resize(C->N); C->ipsi_rev[t].resize(C->N);
    for (size_t i = 0; i < C->N; ++i) {
      u64 e = bitrev(i, log_n);
      C->psi_rev[t][i] = powmod(psi, e, q);
      C->ipsi_rev[t][i] = powmod(ipsi, e, q);
    }
    C->n_inv[t] = invmod(C->N % q, q);
  }
  Stream ss(seed, TAG_SK);
  C->s = sample_ternary(ss, log_n, hw);
  C->s_ntt.resize(total);
  PER_LIMB
  for (int t = 0; t < total; ++t) { C->s_ntt[t] = residues_of(*C, C->s, t); ntt_forward(*C, C->s_ntt[t], t); }
  gen_key(*C, 0);
  return C.release();
}

// ---------------------------------------------------------------- encode / decode
// slots (n = N/2 complex values) -> integer coefficients round(scale * m_k)
static std::vector<double> encode_coeffs(const Ctx& C, const std::vector<cd>& z, double scale) {
  size_t n = C.N / 2;
  if (z.size() != n) throw std::runtime_error("only full-slot packing (N/2 slots) is supported");
  std::vector<cd> w = special_ifft(z, 2 * C.N);
  std::vector<double> m(C.N);
  for (size_t k = 0; k < n; ++k) {
    m[k] = round_half_away(w[k].real() * scale);
    m[k + n] = round_half_away(w[k].imag() * scale);
  }
  return m;
}
static Poly coeffs_to_ntt(const Ctx& C, const std::vector<double>& m, int level) {
  Poly p(level + 1, Limb(C.N));
  PER_LIMB
  for (int i = 0; i <= level; ++i) {
    for (size_t k = 0; k < C.N; ++k) p[i][k] = double_to_mod(m[k], C.q[i]);
    ntt_forward(C, p[i], i);
  }
  return p;
}
// exact CRT of coefficient-domain residues (limbs 0..level), centred, as doubles
static std::vector<double> crt_centred(const Ctx& C, const Poly& coef, int level) {
  int n = level + 1;
  Big Q = Big::from(1); for (int i = 0; i < n; ++i) Q = big_mul(Q, C.q[i]);
  std::vector<Big> qhat(n); std::vector<u64> qhat_inv(n);
  for (int i = 0; i < n; ++i) {
    Big h = Big::from(1); u64 hm = 1;
    for (int k = 0; k < n; ++k) if (k != i) { h = big_mul(h, C.q[k]); hm = mulmod(hm, C.q[k] % C.q[i], C.q[i]); }
    qhat[i] = h; qhat_inv[i] = invmod(hm, C.q[i]);
  }
  Big halfQ = big_mul(Q, 1);  // compare 2x against Q
  std::vector<double> out(C.N);
  for (size_t k = 0; k < C.N; ++k) {
    Big x;
    for (int i = 0; i < n; ++i) x = big_add(x, big_mul(qhat[i], mulmod(coef[i][k], qhat_inv[i], C.q[i])));
    while (big_cmp(x, Q) >= 0) x = big_sub(x, Q);
    Big x2 = big_mul(x, 2);
    if (big_cmp(x2, halfQ) > 0) out[k] = -big_to_double(big_sub(Q, x));
    else out[k] = big_to_double(x);
  }
  return out;
}
static std::vector<cd> decode_coeffs(const Ctx& C, const std::vector<double>& m, double scale) {
  size_t n = C.N / 2;
  std::vector<cd> w(n);
  for (size_t k = 0; k < n; ++k) w[k] = cd(m[k] / scale, m[k + n] / scale);
  return special_fft(w, 2 * C.N);
}

// ---------------------------------------------------------------- ciphertext ops
static Ct encrypt(const Ctx& C, const std::vector<cd>& z, int level, u64 seed) {
  if (level < 0 || level > C.L()) throw std::runtime_error("level out of range");
  std::vector<double> m = encode_coeffs(C, z, C.scale);
  Ct ct; ct.level = level; ct.scale = C.scale;
  ct.c[0].assign(level + 1, Limb(C.N)); ct.c[1].assign(level + 1, Limb(C.N));
  Stream sa(seed, TAG_ENC_A);
  for (int i = 0; i <= level; ++i) for (size_t k = 0; k < C.N; ++k) ct.c[1][i][k] = sample_uniform(sa, C.q[i]);
  Stream se(seed, TAG_ENC_E);
  std::vector<i64> e(C.N); for (size_t k = 0; k < C.N; ++k) e[k] = sample_cbd(se);
  PER_LIMB
  for (int i = 0; i <= level; ++i) {
    u64 q = C.q[i];
    Limb mi(C.N);
    for (size_t k = 0; k < C.N; ++k) mi[k] = addmod(double_to_mod(m[k], q), smod(e[k], q), q);
    ntt_forward(C, mi, i);
    for (size_t k = 0; k < C.N; ++k) ct.c[0][i][k] = submod(mi[k], mulmod(ct.c[1][i][k], C.s_ntt[i][k], q), q);
  }
  return ct;
}
// c0 + c1 s over the ciphertext's primes, centred (the secret s in NTT form over every prime)
static std::vector<double> decrypt_coeffs_under(const Ctx& C, const Ct& ct, const Poly& S) {
  Poly m(ct.level + 1, Limb(C.N));
  PER_LIMB
  for (int i = 0; i <= ct.level; ++i) {
    u64 q = C.q[i];
    for (size_t k = 0; k < C.N; ++k) m[i][k] = addmod(ct.c[0][i][k], mulmod(ct.c[1][i][k], S[i][k], q), q);
    ntt_inverse(C, m[i], i);
  }
  return crt_centred(C, m, ct.level);
}
static std::vector<double> decrypt_coeffs(const Ctx& C, const Ct& ct) { return decrypt_coeffs_under(C, ct, C.s_ntt); }
static std::vector<cd> decrypt(const Ctx& C, const Ct& ct) { return decode_coeffs(C, decrypt_coeffs(C, ct), ct.scale); }

static Ct drop_to(const Ct& a, int level) {
  if (level > a.level || level < 0) throw std::runtime_error("drop_to: bad level");
  Ct r = a; r.level = level;
  for (int c = 0; c < 2; ++c) r.c[c].resize(level + 1);
  return r;
}
static void check_scales(double a, double b) {
  if (std::fabs(a / b - 1.0) > 1e-12) throw std::runtime_error("scale mismatch");
}
static Ct add_sub(const Ctx& C, const Ct& a0, const Ct& b0, bool sub) {
  int l = std::min(a0.level, b0.level);
  Ct a = drop_to(a0, l), b = drop_to(b0, l);
  check_scales(a.scale, b.scale);
  for (int c = 0; c < 2; ++c) for (int i = 0; i <= l; ++i) for (size_t k = 0; k < C.N; ++k)
    a.c[c][i][k] = sub ? submod(a.c[c][i][k], b.c[c][i][k], C.q[i]) : addmod(a.c[c][i][k], b.c[c][i][k], C.q[i]);
  return a;
}
// rescale by the last prime q_l, rounding to nearest:
//   c'_i = (c_i - [c_l]_centred) * q_l^-1 mod q_i
static Poly rescale_poly(const Ctx& C, const Poly& p, int l) {
  u64 ql = C.q[l], h = ql >> 1;
  Limb last = p[l]; ntt_inverse(C, last, l);
  Poly out(l, Limb(C.N));
  PER_LIMB
  for (int i = 0; i < l; ++i) {
    u64 qi = C.q[i], inv = invmod(ql % qi, qi);
    Limb r(C.N);
    for (size_t k = 0; k < C.N; ++k) {
      u64 v = last[k];  // centred representative: v if v <= h else v - q_l
      r[k] = v <= h ? v % qi : submod(v % qi, ql % qi, qi);
    }
    ntt_forward(C, r, i);
    for (size_t k = 0; k < C.N; ++k) out[i][k] = mulmod(submod(p[i][k], r[k], qi), inv, qi);
  }
  return out;
}
static Ct rescale(const Ctx& C, const Ct& a) {
  if (a.level < 1) throw std::runtime_error("rescale: level exhausted");
  Ct r; r.level = a.level - 1; r.scale = a.scale / (double)C.q[a.level];
  for (int c = 0; c < 2; ++c) r.c[c] = rescale_poly(C, a.c[c], a.level);
  return r;
}

// ModUp of digit j at level l: coefficient-domain residues of the digit's primes ->
// residues on every prime of Q_l u P (fast basis conversion, no correction):
//   y_t = sum_{i in digit} [x_i * qhat_i^-1]_{q_i} * qhat_i  mod t
static Poly modup_coeff(const Ctx& C, const Poly& dcoef, int l, int j) {
  int lo = j * C.alpha, hi = std::min(lo + C.alpha, l + 1);
  std::vector<int> ext; for (int i = 0; i <= l; ++i) ext.push_back(i);
  for (int k = 0; k < C.n_p; ++k) ext.push_back(C.n_q + k);
  std::vector<u64> qhat_inv(hi - lo);
  for (int i = lo; i < hi; ++i) {
    u64 h = 1; for (int k = lo; k < hi; ++k) if (k != i) h = mulmod(h, C.q[k] % C.q[i], C.q[i]);
    qhat_inv[i - lo] = invmod(h, C.q[i]);
  }
  Poly out(ext.size(), Limb(C.N));
  PER_LIMB
  for (size_t e = 0; e < ext.size(); ++e) {
    int t = ext[e]; u64 qt = C.q[t];
    if (t >= lo && t < hi) { out[e] = dcoef[t]; continue; }
    std::vector<u64> qhat_t(hi - lo);
    for (int i = lo; i < hi; ++i) {
      u64 h = 1 % qt; for (int k = lo; k < hi; ++k) if (k != i) h = mulmod(h, C.q[k] % qt, qt);
      qhat_t[i - lo] = h;
    }
    for (size_t n = 0; n < C.N; ++n) {
      u64 acc = 0;
      for (int i = lo; i < hi; ++i) {
        u64 y = mulmod(dcoef[i][n], qhat_inv[i - lo], C.q[i]);
        acc = addmod(acc, mulmod(y % qt, qhat_t[i - lo], qt), qt);
      }
      out[e][n] = acc;
    }
  }
  return out;
}
// ModDown at level l: coefficient-domain residues over Q_l u P -> round(x / P) on Q_l:
//   c'_i = (c_i + [floor(P/2)]_{q_i} - BConv_{P->q_i}([c + floor(P/2)]_P)) * P^-1 mod q_i
static Poly moddown_coeff(const Ctx& C, const Poly& x, int l) {
  int K = C.n_p;
  std::vector<u64> phat_inv(K);
  for (int k = 0; k < K; ++k) {
    u64 pk = C.q[C.n_q + k], h = 1;
    for (int m = 0; m < K; ++m) if (m != k) h = mulmod(h, C.q[C.n_q + m] % pk, pk);
    phat_inv[k] = invmod(h, pk);
  }
  auto half_mod = [&](u64 m) {  // floor(P/2) = (P-1)/2 mod m, P odd
    u64 Pm = 1 % m; for (int k = 0; k < K; ++k) Pm = mulmod(Pm, C.q[C.n_q + k] % m, m);
    return mulmod(submod(Pm, 1 % m, m), invmod(2 % m, m), m);
  };
  std::vector<u64> half_p(K); for (int k = 0; k < K; ++k) half_p[k] = half_mod(C.q[C.n_q + k]);
  Poly out(l + 1, Limb(C.N));
  PER_LIMB
  for (int i = 0; i <= l; ++i) {
    u64 qi = C.q[i], hq = half_mod(qi);
    u64 Pm = 1 % qi; for (int k = 0; k < K; ++k) Pm = mulmod(Pm, C.q[C.n_q + k] % qi, qi);
    u64 Pinv = invmod(Pm, qi);
    std::vector<u64> phat_q(K);
    for (int k = 0; k < K; ++k) {
      u64 h = 1 % qi; for (int m = 0; m < K; ++m) if (m != k) h = mulmod(h, C.q[C.n_q + m] % qi, qi);
      phat_q[k] = h;
    }
    for (size_t n = 0; n < C.N; ++n) {
      u64 v = 0;
      for (int k = 0; k < K; ++k) {
        u64 pk = C.q[C.n_q + k];
        u64 r = addmod(x[l + 1 + k][n], half_p[k], pk);
        v = addmod(v, mulmod(mulmod(r, phat_inv[k], pk) % qi, phat_q[k], qi), qi);
      }
      out[i][n] = mulmod(submod(addmod(x[i][n], hq, qi), v, qi), Pinv, qi);
    }
  }
  return out;
}
// hybrid key switch of d (NTT domain, limbs 0..l) under key g -> (ks0, ks1), NTT domain
static void key_switch(const Ctx& C, const Poly& d, int l, u64 g, Poly& o0, Poly& o1) {
  auto it = C.keys.find(g);
  if (it == C.keys.end()) throw std::runtime_error("missing switching key");
  const std::vector<KeyDigit>& key = it->second;
  Poly dcoef = d;
  PER_LIMB
  for (int i = 0; i <= l; ++i) ntt_inverse(C, dcoef[i], i);
  std::vector<int> ext; for (int i = 0; i <= l; ++i) ext.push_back(i);
  for (int k = 0; k < C.n_p; ++k) ext.push_back(C.n_q + k);
  Poly acc0(ext.size(), Limb(C.N, 0)), acc1(ext.size(), Limb(C.N, 0));
  for (int j = 0; j < n_digits(C, l); ++j) {
    Poly y = modup_coeff(C, dcoef, l, j);
    PER_LIMB
    for (size_t e = 0; e < ext.size(); ++e) {
      int t = ext[e]; u64 qt = C.q[t];
      ntt_forward(C, y[e], t);
      for (size_t n = 0; n < C.N; ++n) {
        acc0[e][n] = addmod(acc0[e][n], mulmod(y[e][n], key[j].b[t][n], qt), qt);
        acc1[e][n] = addmod(acc1[e][n], mulmod(y[e][n], key[j].a[t][n], qt), qt);
      }
    }
  }
  PER_LIMB
  for (size_t e = 0; e < ext.size(); ++e) { ntt_inverse(C, acc0[e], ext[e]); ntt_inverse(C, acc1[e], ext[e]); }
  o0 = moddown_coeff(C, acc0, l); o1 = moddown_coeff(C, acc1, l);
  PER_LIMB
  for (int i = 0; i <= l; ++i) { ntt_forward(C, o0[i], i); ntt_forward(C, o1[i], i); }
}
// tensor product + relinearisation (no rescale); both inputs at the same level
static Ct mul_relin(const Ctx& C, const Ct& a0, const Ct& b0) {
  int l = std::min(a0.level, b0.level);
  Ct a = drop_to(a0, l), b = drop_to(b0, l);
  Poly d0(l + 1, Limb(C.N)), d1(l + 1, Limb(C.N)), d2(l + 1, Limb(C.N));
  PER_LIMB
  for (int i = 0; i <= l; ++i) {
    u64 q = C.q[i];
    for (size_t k = 0; k < C.N; ++k) {
      d0[i][k] = mulmod(a.c[0][i][k], b.c[0][i][k], q);
      d1[i][k] = addmod(mulmod(a.c[0][i][k], b.c[1][i][k], q), mulmod(a.c[1][i][k], b.c[0][i][k], q), q);
      d2[i][k] = mulmod(a.c[1][i][k], b.c[1][i][k], q);
    }
  }
  Poly k0, k1; key_switch(C, d2, l, 0, k0, k1);
  Ct r; r.level = l; r.scale = a.scale * b.scale;
  r.c[0] = d0; r.c[1] = d1;
  for (int i = 0; i <= l; ++i) for (size_t k = 0; k < C.N; ++k) {
    r.c[0][i][k] = addmod(r.c[0][i][k], k0[i][k], C.q[i]);
    r.c[1][i][k] = addmod(r.c[1][i][k], k1[i][k], C.q[i]);
  }
  return r;
}
static Ct mul(const Ctx& C, const Ct& a, const Ct& b) { return rescale(C, mul_relin(C, a, b)); }

// automorphism X -> X^g applied to both parts, then key switch back to s
static Ct apply_galois(Ctx& C, const Ct& a, u64 g) {
  gen_key(C, g);
  int l = a.level;
  Poly p0(l + 1), p1(l + 1);
  PER_LIMB
  for (int i = 0; i <= l; ++i) {
    Limb x0 = a.c[0][i], x1 = a.c[1][i];
    ntt_inverse(C, x0, i); ntt_inverse(C, x1, i);
    p0[i] = automorph_coeff(C, x0, g, C.q[i]); p1[i] = automorph_coeff(C, x1, g, C.q[i]);
    ntt_forward(C, p0[i], i); ntt_forward(C, p1[i], i);
  }
  Poly k0, k1; key_switch(C, p1, l, g, k0, k1);
  Ct r; r.level = l; r.scale = a.scale; r.c[0] = p0; r.c[1] = k1;
  for (int i = 0; i <= l; ++i) for (size_t k = 0; k < C.N; ++k) r.c[0][i][k] = addmod(p0[i][k], k0[i][k], C.q[i]);
  return r;
}
static Ct rotate(Ctx& C, const Ct& a, i64 steps) { return apply_galois(C, a, galois_of_rotation(C, steps)); }
// key switch of c1 under the key `id`: (c0 + ks0, ks1)
static Ct switch_key(const Ctx& C, const Ct& a, u64 id) {
  Poly k0, k1; key_switch(C, a.c[1], a.level, id, k0, k1);
  Ct r = a; r.c[1] = k1;
  for (int i = 0; i <= a.level; ++i) for (size_t k = 0; k < C.N; ++k) r.c[0][i][k] = addmod(a.c[0][i][k], k0[i][k], C.q[i]);
  return r;
}
// Several rotations of one ciphertext sharing the ModUp of its second part (hoisting): the
// extended digits of c1 are formed once in the coefficient domain; each rotation applies its
// automorphism to every extended limb, then takes the inner product with its key, ModDown, and
// adds the rotated c0.
static std::vector<Ct> rotate_hoisted(Ctx& C, const Ct& a, const std::vector<i64>& steps) {
  const int l = a.level;
  Poly x0 = a.c[0], x1 = a.c[1];
  PER_LIMB
  for (int i = 0; i <= l; ++i) { ntt_inverse(C, x0[i], i); ntt_inverse(C, x1[i], i); }
  std::vector<int> ext;
  for (int i = 0; i <= l; ++i) ext.push_back(i);
  for (int k = 0; k < C.n_p; ++k) ext.push_back(C.n_q + k);
  std::vector<Poly> ys;
  for (int j = 0; j < n_digits(C, l); ++j) ys.push_back(modup_coeff(C, x1, l, j));
  std::vector<Ct> out;
  for (i64 st : steps) {
    const u64 g = galois_of_rotation(C, st);
    gen_key(C, g);
    const std::vector<KeyDigit>& key = C.keys.find(g)->second;
    Poly acc0(ext.size(), Limb(C.N, 0)), acc1(ext.size(), Limb(C.N, 0));
    for (size_t j = 0; j < ys.size(); ++j) {
      PER_LIMB
      for (size_t e = 0; e < ext.size(); ++e) {
        const int t = ext[e];
        const u64 qt = C.q[t];
        Limb yg = automorph_coeff(C, ys[j][e], g, qt);
        ntt_forward(C, yg, t);
        for (size_t n = 0; n < C.N; ++n) {
          acc0[e][n] = addmod(acc0[e][n], mulmod(yg[n], key[j].b[t][n], qt), qt);
          acc1[e][n] = addmod(acc1[e][n], mulmod(yg[n], key[j].a[t][n], qt), qt);
        }
      }
    }
    PER_LIMB
    for (size_t e = 0; e < ext.size(); ++e) { ntt_inverse(C, acc0[e], ext[e]); ntt_inverse(C, acc1[e], ext[e]); }
    Poly o0 = moddown_coeff(C, acc0, l), o1 = moddown_coeff(C, acc1, l);
    Ct r; r.level = l; r.scale = a.scale;
    r.c[0] = Poly(l + 1); r.c[1] = Poly(l + 1);
    PER_LIMB
    for (int i = 0; i <= l; ++i) {
      Limb p0 = automorph_coeff(C, x0[i], g, C.q[i]);
      ntt_forward(C, p0, i);
      ntt_forward(C, o0[i], i);
      ntt_forward(C, o1[i], i);
      for (size_t k = 0; k < C.N; ++k) p0[k] = addmod(p0[k], o0[i][k], C.q[i]);
      r.c[0][i] = p0;
      r.c[1][i] = o1[i];
    }
    out.push_back(r);
  }
  return out;
}
static Ct conjugate(Ctx& C, const Ct& a) { return apply_galois(C, a, 2 * C.N - 1); }

// multiply by a real constant c encoded at plaintext scale sp, then rescale
static Ct mul_const_sp(const Ctx& C, const Ct& a, double c, double sp) {
  double v = round_half_away(c * sp);
  Ct r = a;
  for (int i = 0; i <= a.level; ++i) {
    u64 cm = double_to_mod(v, C.q[i]);
    for (int p = 0; p < 2; ++p) for (size_t k = 0; k < C.N; ++k) r.c[p][i][k] = mulmod(r.c[p][i][k], cm, C.q[i]);
  }
  r.scale = a.scale * sp;
  return rescale(C, r);
}
// multiply by c at plaintext scale target * q_l / scale, without the rescale: the product is
// labelled target * q_l, so that products at one level with one target add exactly
static Ct mul_const_raw(const Ctx& C, const Ct& a, double c, double target) {
  double sp = target * (double)C.q[a.level] / a.scale;
  double v = round_half_away(c * sp);
  Ct r = a;
  for (int i = 0; i <= a.level; ++i) {
    u64 cm = double_to_mod(v, C.q[i]);
    for (int p = 0; p < 2; ++p) for (size_t k = 0; k < C.N; ++k) r.c[p][i][k] = mulmod(r.c[p][i][k], cm, C.q[i]);
  }
  r.scale = target * (double)C.q[a.level];
  return r;
}
// multiply by c so that the result (one level lower) has exactly scale target
static Ct mul_const_to(const Ctx& C, const Ct& a, double c, double target) {
  double sp = target * (double)C.q[a.level] / a.scale;
  Ct r = mul_const_sp(C, a, c, sp);
  r.scale = target;
  return r;
}
static Ct add_const(const Ctx& C, const Ct& a, double c) {
  double v = round_half_away(c * a.scale);
  Ct r = a;
  for (int i = 0; i <= a.level; ++i) {
    u64 cm = double_to_mod(v, C.q[i]);
    for (size_t k = 0; k < C.N; ++k) r.c[0][i][k] = addmod(r.c[0][i][k], cm, C.q[i]);
  }
  return r;
}
static Ct mul_int(const Ctx& C, const Ct& a, i64 m) {
  Ct r = a;
  for (int i = 0; i <= a.level; ++i) {
    u64 mm = smod(m, C.q[i]);
    for (int p = 0; p < 2; ++p) for (size_t k = 0; k < C.N; ++k) r.c[p][i][k] = mulmod(r.c[p][i][k], mm, C.q[i]);
  }
  return r;
}

// ---------------------------------------------------------------- Chebyshev (Sec. 2.3)
// Interpolant of f at the d+1 Chebyshev nodes of the first kind on [lo, hi]:
//   c_j = (2 - [j=0]) / (d+1) * sum_k f(x_k) cos(j pi (k + 1/2) / (d+1)),
//   x_k = (lo+hi)/2 + (hi-lo)/2 cos(pi (k + 1/2) / (d+1)),  f(x) = 1/sqrt(x).
static std::vector<double> cheb_coeffs(double lo, double hi, int d) {
  int n = d + 1;
  std::vector<double> fx(n), c(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double x = 0.5 * (lo + hi) + 0.5 * (hi - lo) * std::cos(M_PI * (k + 0.5) / n);
    fx[k] = 1.0 / std::sqrt(x);
  }
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int k = 0; k < n; ++k) s += fx[k] * std::cos(M_PI * j * (k + 0.5) / n);
    c[j] = (j == 0 ? 1.0 : 2.0) / n * s;
  }
  return c;
}
// Clenshaw evaluation of sum_j c_j T_j(t)
static double clenshaw(const std::vector<double>& c, double t) {
  double b1 = 0, b2 = 0;
  for (size_t j = c.size(); j-- > 1;) { double b0 = 2 * t * b1 - b2 + c[j]; b2 = b1; b1 = b0; }
  return t * b1 - b2 + c[0];
}

// Homomorphic evaluation in the Chebyshev basis: baby steps T_1..T_k (k = 2^ceil(m/2),
// m = ceil(log2(d+1))), giant steps T_k, T_2k, ..., and the split
//   p = q * T_G + r,  q_0 = c_G, q_i = 2 c_{G+i},  r_i = c_i - c_{2G-i} (2G-i <= deg),
// which follows from 2 T_G T_{j-G} = T_j + T_{2G-j}.  Every partial result is
// produced at a prescribed (level, scale), so additions never need adjustment.
// Two plans.  Fewest products: every polynomial below the baby-step degree is a
// leaf (constant products of T_1..T_D summed, one level below its lowest T_j);
// this takes ceil(log2(d+1)) + 1 levels for most d.  Fewest levels: such a
// polynomial is a leaf only when that reaches the level asked of it, and is
// otherwise split too, at the largest power of two G <= D (a baby step), so that
// constants multiply lower-degree T_j's that have a level to spare; a degree-d
// evaluation then takes ceil(log2(d+1)) levels (the paper: degree 2^{d_e} - 2
// consumes d_e levels, Sec. 4.3) for a few more products.  run() takes the
// fewest-products plan when its output level is at least `need`, else the other.
struct ChebEval {
  Ctx& C;
  std::map<int, Ct> T;  // index -> T_index(t)
  int k = 1;
  std::vector<int> giants;
  explicit ChebEval(Ctx& c) : C(c) {}

  static int deg_of(const std::vector<double>& p) { return (int)p.size() - 1; }
  void split(const std::vector<double>& p, int G, std::vector<double>& qp, std::vector<double>& rp) const {
    int D = deg_of(p);
    qp.assign(D - G + 1, 0.0);
    qp[0] = p[G];
    for (int i = 1; i <= D - G; ++i) qp[i] = 2.0 * p[G + i];
    rp.assign(p.begin(), p.begin() + G);
    for (int i = 0; i < G; ++i) if (2 * G - i <= D) rp[i] -= p[2 * G - i];
  }
  int giant_for(int D) const {
    int G = 0;
    for (int g : giants) if (g <= D) G = g;
    return G;
  }
  // where p of degree D is split: the largest giant step <= D, or, below the baby-step degree, the
  // largest power of two <= D
  int split_for(int D) const {
    if (D >= k) return giant_for(D);
    int G = 1;
    while (2 * G <= D) G *= 2;
    return G;
  }
  // output level of p summed as a leaf: one below the lowest of T_1 .. T_D
  int leaf_level(int D) const {
    int lv = 1 << 30;
    for (int j = 1; j <= D; ++j) lv = std::min(lv, T.at(j).level - 1);
    return lv;
  }
  bool fewest_levels = false;  // the plan (see above)
  bool as_leaf(int D, int level) const {
    return D < k && (!fewest_levels || D < 2 || leaf_level(D) >= level);
  }
  // highest level at which p can be produced
  int best_level(const std::vector<double>& p) const {
    int D = deg_of(p);
    int leaf = D < k ? leaf_level(D) : -(1 << 30);
    if (D < k && (!fewest_levels || D < 2)) return leaf;
    int G = split_for(D);
    std::vector<double> qp, rp; split(p, G, qp, rp);
    int lq = deg_of(qp) == 0 ? (1 << 30) : best_level(qp);
    int lvl = std::min(std::min(lq, T.at(G).level) - 1, best_level(rp));
    return std::max(leaf, lvl);
  }
  // p at (level + 1, label scale * q_{level+1}) before its final rescale: a leaf is the sum of the
  // unrescaled products c_j T_j plus c_0; an inner node adds the relinearised (q T_G) to the
  // unrescaled remainder r
  Ct eval_raw(const std::vector<double>& p, int level, double scale) {
    int D = deg_of(p);
    const double raw = scale * (double)C.q[level + 1];
    if (as_leaf(D, level)) {
      Ct acc;
      for (int j = 1; j <= D; ++j) {
        const Ct& tj = T.at(j);
        Ct term = mul_const_raw(C, drop_to(tj, level + 1), p[j], scale);
        acc = (j == 1) ? term : add_sub(C, acc, term, false);
      }
      acc.scale = raw;
      return add_const(C, acc, p[0]);
    }
    int G = split_for(D);
    std::vector<double> qp, rp; split(p, G, qp, rp);
    const Ct& tg = T.at(G);
    Ct prod;
    if (deg_of(qp) == 0) {
      prod = mul_const_raw(C, drop_to(tg, level + 1), qp[0], scale);
    } else {
      double sq = scale * (double)C.q[level + 1] / tg.scale;
      Ct qv = eval(qp, level + 1, sq);
      prod = mul_relin(C, qv, drop_to(tg, level + 1));
    }
    prod.scale = raw;
    Ct rv = eval_raw(rp, level, scale);
    return add_sub(C, prod, rv, false);
  }
  Ct eval(const std::vector<double>& p, int level, double scale) {
    Ct r = rescale(C, eval_raw(p, level, scale));
    r.scale = scale;
    return r;
  }
  // T_a * T_b -> 2 T_a T_b - T_c  with T_c = T_{|a-b|} (or the constant 1 when a == b)
  Ct cheb_product(const Ct& ta, const Ct& tb, int c_index) {
    Ct diff;
    if (c_index == 0) diff = add_const(C, mul(C, ta, tb), -0.5);
    else {  // the product and 0.5 T_c subtracted before one rescale
      Ct pr = mul_relin(C, ta, tb);
      const double out = pr.scale / (double)C.q[pr.level];
      const Ct& tc = T.at(c_index);
      Ct half = mul_const_raw(C, drop_to(tc, pr.level), 0.5, out);
      diff = rescale(C, add_sub(C, pr, half, true));
      diff.scale = out;
    }
    return mul_int(C, diff, 2);
  }
  // need < 0: the fewest-levels plan; else the fewest-products plan if it ends at level >= need
  Ct run(const Ct& t, const std::vector<double>& coeffs, int need) { return run(t, coeffs, C.scale, need); }
  Ct run(const Ct& t, const std::vector<double>& coeffs, double target, int need) {
    int d = deg_of(coeffs);
    int m = 0; while ((1 << m) < d + 1) ++m;
    int lb = (m + 1) / 2; if (lb < 1) lb = 1;
    k = 1 << lb;
    T.clear(); T[1] = t;
    for (int j = 2; j <= k; ++j) {
      if (j % 2 == 0) T[j] = cheb_product(T.at(j / 2), T.at(j / 2), 0);
      else T[j] = cheb_product(T.at(j / 2), T.at(j / 2 + 1), 1);
    }
    giants.clear();
    for (int g = k; g < (1 << m); g *= 2) {
      giants.push_back(g);
      if (!T.count(g)) T[g] = cheb_product(T.at(g / 2), T.at(g / 2), 0);
    }
    fewest_levels = need < 0;
    int lvl = best_level(coeffs);
    if (!fewest_levels && lvl < need) {
      fewest_levels = true;
      lvl = best_level(coeffs);
    }
    if (lvl < 0) throw std::runtime_error("Chebyshev evaluation: level exhausted");
    return eval(coeffs, lvl, target);
  }
};


// ---------------------------------------------------------------- bootstrapping
// The paper uses BTS as a black box (Sec. 2.1): it needs level >= l_BTS, takes
// inputs in [-1, 1] and returns a ciphertext at l_afterBTS.  This is the
// textbook full-slot CKKS bootstrapping (Cheon et al. 2018 with the
// CoeffToSlot / EvalMod / SlotToCoeff structure of Chen-Chillotti-Song 2019 and
// the cosine + double-angle EvalMod of Bossuat et al. 2021):
//   ModRaise   level-0 coefficients (centred mod q_0) lifted to every prime:
//              plaintext t = m + q_0 I, |I| < K
//   CoeffToSlot slots <- V^-1 slots, V the decoding matrix z = V w, factored into
//              the radix-2 stages of the special FFT and grouped into bts_cts
//              sparse matrices, each applied as baby-step / giant-step sums of
//              diagonals times rotations; real and imaginary parts split by
//              conjugation
//   EvalMod    u = t / (q_0 K) -> sin(2 pi K u) = sin(2 pi m / q_0): Chebyshev
//              interpolant of cos(2 pi (K u - 1/4) / 2^r), then r double angles
//   SlotToCoeff slots <- V slots (bts_stc groups)
// Constant factors are carried by the scale labels: ModRaise labels t with
// scale 2 q_0 K; after EvalMod the label is multiplied by 2 pi s_in / q_0.
typedef std::map<long, std::vector<cd>> DiagMap;  // rotation offset (mod n) -> diagonal

static std::vector<cd> rot_vec(const std::vector<cd>& v, long k) {  // out[s] = v[s + k]
  long n = (long)v.size();
  std::vector<cd> r(n);
  for (long s = 0; s < n; ++s) r[s] = v[(((s + k) % n) + n) % n];
  return r;
}
// one radix-2 stage (sub-transform length len) of the decoding FFT over
// bit-reversed input, or its inverse, as diagonals
static DiagMap fft_stage(size_t n, size_t len, bool inverse) {
  size_t h = len / 2; u64 M = 4 * len;
  std::vector<cd> d0(n), dp(n), dm(n);
  for (size_t s = 0; s < n; ++s) {
    size_t j = s % len;
    size_t jj = j < h ? j : j - h;
    cd z = std::polar(1.0, 2.0 * M_PI * (double)powmod(5, jj, M) / (double)M);
    if (!inverse) {
      if (j < h) { d0[s] = 1.0; dp[s] = z; } else { d0[s] = -z; dm[s] = 1.0; }
    } else {
      if (j < h) { d0[s] = 0.5; dp[s] = 0.5; } else { d0[s] = -std::conj(z) * 0.5; dm[s] = std::conj(z) * 0.5; }
    }
  }
  DiagMap D;  // offsets +h and -h coincide modulo n when h = n/2: add
  D[0] = d0;
  D[(long)h] = dp;
  std::vector<cd>& m = D[(long)(n - h)];
  if (m.empty()) m = dm; else for (size_t s = 0; s < n; ++s) m[s] += dm[s];
  return D;
}
// (A B) v = sum_{a,b} (A_a o rot(B_b, a)) o rot(v, a + b)
static DiagMap diag_compose(const DiagMap& A, const DiagMap& B, size_t n) {
  DiagMap R;
  for (auto& a : A) for (auto& b : B) {
    long o = (long)((a.first + b.first) % (long)n);
    std::vector<cd> rb = rot_vec(b.second, a.first);
    std::vector<cd>& dst = R[o];
    if (dst.empty()) dst.assign(n, cd(0, 0));
    for (size_t s = 0; s < n; ++s) dst[s] += a.second[s] * rb[s];
  }
  return R;
}
// the bts_cts (inverse) or bts_stc (forward) grouped factors, in application order
static std::vector<DiagMap> fft_groups(size_t n, int groups, bool inverse) {
  int logn = 0; while ((1ull << logn) < n) ++logn;
  std::vector<int> sizes(groups, logn / groups);
  for (int g = 0; g < logn % groups; ++g) sizes[g] += 1;
  std::vector<size_t> lens;  // stage lengths in application order
  if (!inverse) for (int i = 1; i <= logn; ++i) lens.push_back(1ull << i);
  else for (int i = logn; i >= 1; --i) lens.push_back(1ull << i);
  std::vector<DiagMap> out; size_t pos = 0;
  for (int g = 0; g < groups; ++g) {
    DiagMap M = fft_stage(n, lens[pos++], inverse);
    for (int k = 1; k < sizes[g]; ++k) M = diag_compose(fft_stage(n, lens[pos++], inverse), M, n);
    out.push_back(M);
  }
  return out;
}
static Poly encode_at(const Ctx& C, const std::vector<cd>& z, double scale, int level) {
  return coeffs_to_ntt(C, encode_coeffs(C, z, scale), level);
}
// Baby steps of a linear transform kept in the extended basis Q_l u P (double hoisting, Bossuat,
// Mouchet, Troncoso-Pastoriza and Hubaux, Eurocrypt 2021): rotation g of a is represented, before
// its ModDown, as the pair (P sigma_g(c0) + ks0, ks1) over Q_l u P (NTT domain), ks the key-switch
// sums of sigma_g(c1) (the hoisted digits, as in rotate_hoisted).  P x vanishes mod every p_k.
// Giant steps then sum plaintext products of these pairs and divide by P once (ModDown).
static std::vector<int> ext_primes(const Ctx& C, int l) {
  std::vector<int> ext;
  for (int i = 0; i <= l; ++i) ext.push_back(i);
  for (int k = 0; k < C.n_p; ++k) ext.push_back(C.n_q + k);
  return ext;
}
static u64 P_mod(const Ctx& C, u64 m) {
  u64 r = 1 % m;
  for (int k = 0; k < C.n_p; ++k) r = mulmod(r, C.q[C.n_q + k] % m, m);
  return r;
}
typedef std::array<Poly, 2> PolyPair;
// a itself over Q_l u P: (P c0, P c1)
static PolyPair lift_qp(const Ctx& C, const Ct& a) {
  const int l = a.level;
  const std::vector<int> ext = ext_primes(C, l);
  PolyPair r;
  for (int p = 0; p < 2; ++p) {
    r[p].assign(ext.size(), Limb(C.N, 0));
    for (int i = 0; i <= l; ++i) {
      const u64 Pm = P_mod(C, C.q[i]);
      for (size_t n = 0; n < C.N; ++n) r[p][i][n] = mulmod(a.c[p][i][n], Pm, C.q[i]);
    }
  }
  return r;
}
static std::vector<PolyPair> rotate_hoisted_qp(Ctx& C, const Ct& a, const std::vector<i64>& steps) {
  const int l = a.level;
  Poly x1 = a.c[1];
  PER_LIMB
  for (int i = 0; i <= l; ++i) ntt_inverse(C, x1[i], i);
  const std::vector<int> ext = ext_primes(C, l);
  std::vector<Poly> ys;
  for (int j = 0; j < n_digits(C, l); ++j) ys.push_back(modup_coeff(C, x1, l, j));
  std::vector<PolyPair> out;
  for (i64 st : steps) {
    const u64 g = galois_of_rotation(C, st);
    gen_key(C, g);
    const std::vector<KeyDigit>& key = C.keys.find(g)->second;
    PolyPair acc;
    acc[0].assign(ext.size(), Limb(C.N, 0));
    acc[1].assign(ext.size(), Limb(C.N, 0));
    for (size_t j = 0; j < ys.size(); ++j) {
      PER_LIMB
      for (size_t e = 0; e < ext.size(); ++e) {
        const int t = ext[e];
        const u64 qt = C.q[t];
        Limb yg = automorph_coeff(C, ys[j][e], g, qt);
        ntt_forward(C, yg, t);
        for (size_t n = 0; n < C.N; ++n) {
          acc[0][e][n] = addmod(acc[0][e][n], mulmod(yg[n], key[j].b[t][n], qt), qt);
          acc[1][e][n] = addmod(acc[1][e][n], mulmod(yg[n], key[j].a[t][n], qt), qt);
        }
      }
    }
    PER_LIMB
    for (int i = 0; i <= l; ++i) {  // + P sigma_g(c0) on the Q limbs
      Limb x0 = a.c[0][i];
      ntt_inverse(C, x0, i);
      Limb p0 = automorph_coeff(C, x0, g, C.q[i]);
      ntt_forward(C, p0, i);
      const u64 Pm = P_mod(C, C.q[i]);
      for (size_t n = 0; n < C.N; ++n) acc[0][i][n] = addmod(acc[0][i][n], mulmod(p0[n], Pm, C.q[i]), C.q[i]);
    }
    out.push_back(acc);
  }
  return out;
}
// ModDown of a pair over Q_l u P (NTT domain) into a ciphertext at level l
static Ct moddown_pair(const Ctx& C, PolyPair x, int l, double scale) {
  const std::vector<int> ext = ext_primes(C, l);
  Ct r; r.level = l; r.scale = scale;
  for (int p = 0; p < 2; ++p) {
    PER_LIMB
    for (size_t e = 0; e < ext.size(); ++e) ntt_inverse(C, x[p][e], ext[e]);
    r.c[p] = moddown_coeff(C, x[p], l);
    PER_LIMB
    for (int i = 0; i <= l; ++i) ntt_forward(C, r.c[p][i], i);
  }
  return r;
}
static Ct mul_plain(const Ctx& C, const Ct& a, const Poly& pt) {
  Ct r = a;
  PER_LIMB
  for (int i = 0; i <= a.level; ++i)
    for (int p = 0; p < 2; ++p) for (size_t k = 0; k < C.N; ++k) r.c[p][i][k] = mulmod(a.c[p][i][k], pt[i][k], C.q[i]);
  return r;
}
// a vector of n slots repeated to fill the N/2 slots (sparse packing: slot j and slot j + n hold
// the same value exactly when the plaintext lies in the subring of polynomials in X^(N/2n))
static std::vector<cd> tiled(const Ctx& C, const std::vector<cd>& v) {
  std::vector<cd> out(C.N / 2);
  for (size_t s = 0; s < out.size(); ++s) out[s] = v[s % v.size()];
  return out;
}
// sum_o diag_o o rot(v, o) as sum_g rot( sum_b rot(diag_{k}, -G_g) o rot(v, b h0), G_g ),
// offsets o = k h0, k = k_min + g n1 + b; one rescale at the end, result scale = target
static Ct linear_transform(Ctx& C, const Ct& v, const DiagMap& M, double target, long n) {
  long h0 = 0, kmin = 0, kmax = 0;
  std::map<long, const std::vector<cd>*> byk;
  for (auto& e : M) { long o = e.first <= n / 2 ? e.first : e.first - n; if (o) h0 = h0 ? std::__gcd(h0, std::labs(o)) : std::labs(o); }
  if (!h0) h0 = 1;
  for (auto& e : M) {
    long o = e.first <= n / 2 ? e.first : e.first - n;
    long k = o / h0; byk[k] = &e.second; kmin = std::min(kmin, k); kmax = std::max(kmax, k);
  }
  // n1 baby steps: the power of two with n1^2 >= 4 span (a giant step's full key switch costs about four
  // hoisted baby-step rotations, so the split leans to baby steps), at most 16 per giant step
  long span = kmax - kmin + 1, n1 = 1;
  while (n1 * n1 < 4 * span) n1 <<= 1;
  n1 = std::min(n1, 16L);
  long giants = (span + n1 - 1) / n1;
  double sp = target * (double)C.q[v.level] / v.scale;
  const int l = v.level;
  const std::vector<int> ext = ext_primes(C, l);
  // baby steps: every rotation of v used by some giant step, hoisted and kept over Q_l u P
  std::vector<PolyPair> baby(n1);
  std::vector<bool> have(n1, false);
  {
    std::vector<long> need;
    std::vector<i64> steps;
    for (long b = 1; b < n1; ++b)
      for (long g = 0; g < giants; ++g)
        if (byk.count(kmin + g * n1 + b)) { need.push_back(b); steps.push_back(b * h0); break; }
    std::vector<PolyPair> rot = rotate_hoisted_qp(C, v, steps);
    for (size_t i = 0; i < need.size(); ++i) { baby[need[i]] = rot[i]; have[need[i]] = true; }
    for (long g = 0; g < giants; ++g)
      if (byk.count(kmin + g * n1)) { baby[0] = lift_qp(C, v); have[0] = true; break; }
  }
  Ct acc; bool acc_set = false;
  for (long g = 0; g < giants; ++g) {
    long G = h0 * (kmin + g * n1);
    // sum_b diag o baby_b over Q_l u P, then one ModDown
    PolyPair inner;
    inner[0].assign(ext.size(), Limb(C.N, 0));
    inner[1].assign(ext.size(), Limb(C.N, 0));
    bool inner_set = false;
    for (long b = 0; b < n1; ++b) {
      long k = kmin + g * n1 + b;
      auto it = byk.find(k);
      if (it == byk.end() || !have[b]) continue;
      const std::vector<double> m = encode_coeffs(C, tiled(C, rot_vec(*it->second, -G)), sp);
      PER_LIMB
      for (size_t e = 0; e < ext.size(); ++e) {
        const int t = ext[e];
        const u64 qt = C.q[t];
        Limb pt(C.N);
        for (size_t n = 0; n < C.N; ++n) pt[n] = double_to_mod(m[n], qt);
        ntt_forward(C, pt, t);
        for (int p = 0; p < 2; ++p)
          for (size_t n = 0; n < C.N; ++n) inner[p][e][n] = addmod(inner[p][e][n], mulmod(baby[b][p][e][n], pt[n], qt), qt);
      }
      inner_set = true;
    }
    if (!inner_set) continue;
    Ct in = moddown_pair(C, inner, l, v.scale * sp);
    long Gm = ((G % n) + n) % n;
    Ct r = Gm ? rotate(C, in, G) : in;
    acc = acc_set ? add_sub(C, acc, r, false) : r; acc_set = true;
  }
  Ct out = rescale(C, acc);
  out.scale = target;
  return out;
}
static Ct mod_raise(const Ctx& C, const Ct& a) {
  if (a.level != 0) throw std::runtime_error("mod_raise: input must be at level 0");
  Ct r; r.level = C.L(); r.scale = a.scale;
  u64 q0 = C.q[0], h = q0 >> 1;
  for (int p = 0; p < 2; ++p) {
    Limb x = a.c[p][0]; ntt_inverse(C, x, 0);
    r.c[p].assign(C.L() + 1, Limb(C.N));
    PER_LIMB
    for (int i = 0; i <= C.L(); ++i) {
      u64 qi = C.q[i];
      for (size_t k = 0; k < C.N; ++k) r.c[p][i][k] = x[k] <= h ? x[k] % qi : submod(x[k] % qi, q0 % qi, qi);
      ntt_forward(C, r.c[p][i], i);
    }
  }
  return r;
}
// multiplication by the monomial X^e (0 <= e < 2N): negacyclic shift of the coefficients
static Ct mul_monomial(const Ctx& C, const Ct& a, u64 e) {
  Ct r = a; u64 M = 2 * C.N;
  for (int p = 0; p < 2; ++p) {
    PER_LIMB
    for (int i = 0; i <= a.level; ++i) {
      Limb x = a.c[p][i]; ntt_inverse(C, x, i);
      Limb y(C.N, 0);
      for (size_t k = 0; k < C.N; ++k) {
        u64 t = (k + e) % M;
        if (t < C.N) y[t] = x[k]; else y[t - C.N] = x[k] ? C.q[i] - x[k] : 0;
      }
      ntt_forward(C, y, i);
      r.c[p][i] = y;
    }
  }
  return r;
}
// Chebyshev interpolant of an arbitrary function on [lo, hi] (same closed form as cheb_coeffs)
template <class F>
static std::vector<double> cheb_interp_fn(F f, double lo, double hi, int d) {
  int n = d + 1;
  std::vector<double> fx(n), c(n, 0.0);
  for (int k = 0; k < n; ++k) fx[k] = f(0.5 * (lo + hi) + 0.5 * (hi - lo) * std::cos(M_PI * (k + 0.5) / n));
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int k = 0; k < n; ++k) s += fx[k] * std::cos(M_PI * j * (k + 0.5) / n);
    c[j] = (j == 0 ? 1.0 : 2.0) / n * s;
  }
  return c;
}
static Ct eval_mod(Ctx& C, const Ct& u) {
  const double K = C.bts_K, R = std::ldexp(1.0, C.bts_r);
  std::vector<double> coeffs = cheb_interp_fn([&](double x) { return std::cos(2.0 * M_PI * (K * x - 0.25) / R); },
                                              -1.0, 1.0, C.bts_deg);
  ChebEval ev(C);
  Ct c = ev.run(u, coeffs, u.scale, -1);  // fewest levels: every level of the chain is a level of output
  for (int i = 0; i < C.bts_r; ++i) c = mul_int(C, add_const(C, mul(C, c, c), -0.5), 2);  // cos 2x = 2 cos^2 x - 1
  return c;
}
static int bts_levels(const Ctx& C) { return C.bts_cts + C.bts_r + C.bts_stc + [&] { int m = 0; while ((1 << m) < C.bts_deg + 1) ++m; return m; }(); }
// Sparse packing, n = 2^log_slots < N/2 slots: the plaintext is a polynomial in Y = X^(N/2n)
// and its slots repeat with period n.  After ModRaise the overflow q_0 I is a general
// polynomial; the sum of the automorphisms that fix the subring (the rotations by multiples of
// n: X -> X^(5^(n j)), 5^(n j) = 1 mod 4n) maps X^i to (N/2n) X^i when (N/2n) | i and to 0
// otherwise, so rotating by n, 2n, ..., N/4 and adding projects onto the subring times N/2n.
static Ct sub_sum(Ctx& C, const Ct& a, size_t n) {
  Ct t = a;
  for (size_t k = n; k < C.N / 2; k *= 2) t = add_sub(C, t, rotate(C, t, (i64)k), false);
  return t;
}
// Sparse slots pack the real and imaginary parts into 2n slots of one ciphertext (2n <= N/2): the
// last CoeffToSlot factor is multiplied on its output by the 2n-periodic mask (1 on the first n
// slots, -i on the next n), so that s + conj(s) carries 2 Re u on [0, n) and 2 Im u on [n, 2n);
// after one EvalMod the first SlotToCoeff factor reads slot m and slot m + n as the real and
// imaginary parts of its n-periodic input: each diagonal d_k goes to offsets k and k + n, with the
// factor 1 on the offset that lands in [0, n) and i on the other.
static cd mul_minus_i(cd z) { return cd(z.imag(), -z.real()); }
static cd mul_i(cd z) { return cd(-z.imag(), z.real()); }
static DiagMap pack_cts_last(const DiagMap& M, size_t n) {
  DiagMap R;
  for (auto& e : M) {
    std::vector<cd> d(2 * n);
    for (size_t j = 0; j < 2 * n; ++j) d[j] = j < n ? e.second[j] : mul_minus_i(e.second[j - n]);
    R[e.first] = d;
  }
  return R;
}
static DiagMap pack_stc_first(const DiagMap& M, size_t n) {
  DiagMap R;
  long P = (long)(2 * n);
  for (auto& e : M) {
    long k = e.first;
    for (size_t j = 0; j < 2 * n; ++j) {
      cd v = e.second[j % n];
      bool lo = ((long)j + k) % P < (long)n;  // offset k reads a slot of [0, n)
      for (int h = 0; h < 2; ++h) {
        long off = (((k + h * (long)n) % P) + P) % P;
        std::vector<cd>& d = R[off];
        if (d.empty()) d.assign(2 * n, cd(0, 0));
        d[j] += (lo == (h == 0)) ? v : mul_i(v);
      }
    }
  }
  return R;
}
// Full-slot (log_slots = 0) or sparse-slot bootstrapping.  The sparse one is the full one of
// the ring of dimension 2n (CoeffToSlot / SlotToCoeff on n slots, diagonals repeated over the
// N/2 slots) after the projection of sub_sum, whose factor N/2n rides on the scale label.
static Ct bootstrap_core(Ctx& C, const Ct& a, int log_slots = 0) {
  if (!C.bts_on) throw std::runtime_error("bootstrapping is not configured");
  if (a.level != 0) throw std::runtime_error("bootstrap: input must be at level 0");
  if (log_slots < 0 || (log_slots && ((1ull << log_slots) > C.N / 2 || log_slots < std::max(C.bts_cts, C.bts_stc))))
    throw std::runtime_error("bootstrap: log_slots out of range");
  const size_t n = log_slots ? (1ull << log_slots) : C.N / 2;
  const double s_in = a.scale, q0 = (double)C.q[0];
  // with encapsulation: to the sparse secret at level 0, ModRaise, back to s at the top level
  Ct t = C.enc_hw ? switch_key(C, mod_raise(C, switch_key(C, a, 2)), 4) : mod_raise(C, a);
  if (n < C.N / 2) t = sub_sum(C, t, n);
  t.scale = 2.0 * q0 * C.bts_K * (double)(C.N / 2 / n);
  if (n < C.N / 2) {  // packed real and imaginary parts, one EvalMod
    std::vector<DiagMap> F = fft_groups(n, C.bts_cts, true);
    for (size_t g = 0; g + 1 < F.size(); ++g) t = linear_transform(C, t, F[g], (double)C.q[t.level - 1], (long)n);
    t = linear_transform(C, t, pack_cts_last(F.back(), n), (double)C.q[t.level - 1], (long)(2 * n));
    Ct w = eval_mod(C, add_sub(C, t, conjugate(C, t), false));  // 2 Re | 2 Im
    w.scale = w.scale * 2.0 * M_PI * s_in / q0;
    std::vector<DiagMap> G = fft_groups(n, C.bts_stc, false);
    w = linear_transform(C, w, pack_stc_first(G[0], n), G.size() == 1 ? C.scale : (double)C.q[w.level - 1],
                         (long)(2 * n));
    for (size_t g = 1; g < G.size(); ++g)
      w = linear_transform(C, w, G[g], g + 1 == G.size() ? C.scale : (double)C.q[w.level - 1], (long)n);
    return w;
  }
  for (const DiagMap& M : fft_groups(n, C.bts_cts, true))
    t = linear_transform(C, t, M, (double)C.q[t.level - 1], (long)n);
  Ct cj = conjugate(C, t);
  Ct re = add_sub(C, t, cj, false);
  Ct im = mul_monomial(C, add_sub(C, t, cj, true), 3 * C.N / 2);  // times -i
  re = eval_mod(C, re);
  im = eval_mod(C, im);
  Ct w = add_sub(C, re, mul_monomial(C, im, C.N / 2), false);  // re + i im
  w.scale = w.scale * 2.0 * M_PI * s_in / q0;
  std::vector<DiagMap> G = fft_groups(n, C.bts_stc, false);
  for (size_t g = 0; g < G.size(); ++g)
    w = linear_transform(C, w, G[g], g + 1 == G.size() ? C.scale : (double)C.q[w.level - 1], (long)n);
  return w;
}
// values of y in [-Y, Y]: scale by 1/Y into [-1, 1] (one level, landing at level 0
// with scale q_0 / 2^12), bootstrap, multiply back by the integer Y
static Ct bootstrap_scaled(Ctx& C, const Ct& y, i64 Y, int log_slots = 0) {
  if (y.level < 1) throw std::runtime_error("bootstrap: input needs level >= 1");
  Ct a = mul_const_to(C, drop_to(y, 1), 1.0 / (double)Y, (double)C.q[0] / 4096.0);
  Ct b = bootstrap_core(C, a, log_slots);
  return Y == 1 ? b : mul_int(C, b, Y);
}

// ---------------------------------------------------------------- CryptoInvSqrt (Alg. 1)
// log_slots: 0 for N/2 slots, else the inputs are sparsely packed (2^log_slots values repeated)
// and every bootstrap inside uses the sparse-slot transform
struct InvSqrtCfg { double lo, hi, B; int degree, iters, pre_bts; u64 bts_mask; int log_slots; };

// One Newton step y <- 1.5 y - (0.5 a) y^3 (Sec. 2.2), in the operation order of
// Alg. 1's loop body; tmp_alpha is produced last, at the level of the relinearised
// tmp_beta and labelled with its scale, and tmp_alpha - tmp_beta is rescaled once.
static Ct newton_step(Ctx& C, const Ct& x, const Ct& y) {
  int ly = y.level;
  Ct yy = mul(C, y, y);                            // y^2
  Ct xy = mul(C, drop_to(x, std::min(x.level, ly)), y);  // (0.5 a) y
  Ct tb = mul_relin(C, xy, yy);                     // tmp_beta = (0.5 a) y^3, before its rescale
  const double out = tb.scale / (double)C.q[tb.level];
  Ct ta = mul_const_raw(C, drop_to(y, tb.level), 1.5, out);  // tmp_alpha = 1.5 y, labelled tb's scale
  Ct r = rescale(C, add_sub(C, ta, tb, true));        // tmp_alpha - tmp_beta, one rescale
  r.scale = out;
  return r;
}

// Bootstrapping placement (the paper's Pre-BTS indicator c, Sec. 4.1, and BTS
// during the Newton loop, Sec. 4.3): pre_bts bootstraps the input a/B first;
// bit j (< 63) of bts_mask bootstraps y before Newton step j (bit 0: right
// after the Chebyshev step, as in Alg. 1); bit 63 bootstraps lazily, before a
// step that would leave y below level 1 (fewer than 3 levels), so that later
// bootstraps stay possible whatever number of steps follows.  ct_x is not
// bootstrapped in Alg. 1 (a Newton output sits two levels below it); bit 62 (a
// variant) bootstraps it too whenever y is bootstrapped and x has fewer than 5
// levels, scaled by Yx, the power of two bounding x = 0.5 a/B.  Y, the power of two
// that bounds y = 1/sqrt(a/B), scales y into [-1, 1] around each BTS.
static Ct invsqrt(Ctx& C, const Ct& in, const InvSqrtCfg& cfg) {
  if (cfg.B <= 0 || !(cfg.lo > 0) || !(cfg.hi > cfg.lo) || cfg.degree < 1 || cfg.iters < 0)
    throw std::runtime_error("invsqrt: bad configuration");
  if ((cfg.pre_bts || cfg.bts_mask) && !C.bts_on) throw std::runtime_error("invsqrt: bootstrapping not configured");
  double lo = cfg.lo / cfg.B, hi = cfg.hi / cfg.B;
  i64 Y = 1; while ((double)Y < 1.0 / std::sqrt(lo)) Y *= 2;
  Ct a = in; double Bf = cfg.B;
  if (cfg.pre_bts) {  // a -> BTS(a / B): values in (0, 1]
    if (in.level < 1) throw std::runtime_error("invsqrt: level exhausted");
    a = bootstrap_core(C, mul_const_to(C, drop_to(in, 1), 1.0 / cfg.B, (double)C.q[0] / 4096.0), cfg.log_slots);
    Bf = 1.0;
  }
  // pre-normalisation (Sec. 2.3): a -> a/B, then the affine map onto [-1, 1]
  // for the Chebyshev basis, folded into one constant multiplication
  double alpha = 2.0 / (Bf * (hi - lo)), beta = -(hi + lo) / (hi - lo);
  if (a.level < 2) throw std::runtime_error("invsqrt: level exhausted");
  Ct t = add_const(C, mul_const_to(C, a, alpha, C.scale), beta);
  Ct x = mul_const_to(C, a, 0.5 / Bf, C.scale);  // ct_x = 0.5 * a/B
  std::vector<double> coeffs = cheb_coeffs(lo, hi, cfg.degree);
  // with bootstrapping in the configuration, the fewest-levels plan (a level saved is a bootstrap
  // saved or postponed); without, the fewest products while the Newton steps still fit
  ChebEval ev(C);
  Ct y = ev.run(t, coeffs, (cfg.pre_bts || cfg.bts_mask) ? -1 : 2 * cfg.iters);
  const bool lazy = (cfg.bts_mask >> 63) & 1, lazy_x = (cfg.bts_mask >> 62) & 1;
  i64 Yx = 1; while ((double)Yx < 0.5 * hi) Yx *= 2;
  for (int i = 0; i < cfg.iters; ++i) {
    bool force = i < 62 && ((cfg.bts_mask >> i) & 1);
    bool need = lazy && y.level < 3;  // the step would leave y below level 1
    if (force || need) {
      y = bootstrap_scaled(C, y, Y, cfg.log_slots);
      if (lazy_x && x.level < 5) x = bootstrap_scaled(C, x, Yx, cfg.log_slots);
    }
    if (std::min(y.level, x.level) < 2) throw std::runtime_error("invsqrt: level exhausted in Newton loop");
    y = newton_step(C, x, y);
  }
  if (cfg.iters == 0 && (cfg.bts_mask & 1)) y = bootstrap_scaled(C, y, Y, cfg.log_slots);
  if (cfg.B != 1.0) y.scale *= std::sqrt(cfg.B);  // y / sqrt(B): relabelled, no level used
  return y;
}

// FP64 model of the same algorithm (the plaintext floor): Clenshaw + Newton
static void plain_invsqrt(const double* a, size_t n, const InvSqrtCfg& cfg, double* out) {
  double lo = cfg.lo / cfg.B, hi = cfg.hi / cfg.B;
  std::vector<double> c = cheb_coeffs(lo, hi, cfg.degree);
  for (size_t s = 0; s < n; ++s) {
    double x = a[s] / cfg.B;
    double t = (2.0 * x - (hi + lo)) / (hi - lo);
    double y = clenshaw(c, t);
    for (int i = 0; i < cfg.iters; ++i) y = 0.5 * y * (3.0 - x * y * y);
    out[s] = y / std::sqrt(cfg.B);
  }
}

// ============================================================================ C API
#define API extern "C" __attribute__((visibility("default")))
#define GUARD(...) try { __VA_ARGS__ } catch (const std::exception& e) { g_err = e.what(); }

API const char* orc_last_error() { return g_err.c_str(); }

API void* orc_ctx_create(uint32_t log_n, uint32_t n_q, const uint32_t* q_bits, uint32_t n_p, const uint32_t* p_bits,
                         uint32_t alpha, double log_scale, uint32_t hw, uint64_t seed) {
  GUARD(
    std::vector<int> qb(q_bits, q_bits + n_q), pb(p_bits, p_bits + n_p);
    return ctx_create((int)log_n, qb, pb, (int)alpha, log_scale, (int)hw, seed);
  )
  return nullptr;
}
API void orc_ctx_destroy(void* c) { delete (Ctx*)c; }
API int orc_ctx_info(void* c, uint32_t* log_n, uint32_t* n_q, uint32_t* n_p, uint32_t* alpha, double* scale) {
  Ctx* C = (Ctx*)c; *log_n = C->log_n; *n_q = C->n_q; *n_p = C->n_p; *alpha = C->alpha; *scale = C->scale; return 0;
}
API int orc_ctx_primes(void* c, uint64_t* out) {
  Ctx* C = (Ctx*)c; for (size_t i = 0; i < C->q.size(); ++i) out[i] = C->q[i]; return 0;
}
API int orc_ctx_psi(void* c, uint64_t* out) {
  Ctx* C = (Ctx*)c; for (size_t i = 0; i < C->psi.size(); ++i) out[i] = C->psi[i]; return 0;
}
API int orc_export_secret(void* c, int64_t* out) {
  Ctx* C = (Ctx*)c; for (size_t i = 0; i < C->N; ++i) out[i] = C->s[i]; return 0;
}
API int orc_export_sparse_secret(void* c, int64_t* out) {
  GUARD(
    Ctx* C = (Ctx*)c;
    if (!C->enc_hw) throw std::runtime_error("no encapsulation");
    for (size_t i = 0; i < C->N; ++i) out[i] = C->s_sparse[i];
    return 0;
  )
  return -1;
}
API int orc_gen_galois_key(void* c, uint64_t g) { GUARD(gen_key(*(Ctx*)c, g); return 0;) return -1; }
API uint64_t orc_galois_of_rotation(void* c, int64_t r) { return galois_of_rotation(*(Ctx*)c, r); }
// key digit j for galois element g (0 = relinearisation), each part [n_q+n_p][N], NTT domain
API int orc_export_key(void* c, uint64_t g, uint32_t j, uint64_t* out_b, uint64_t* out_a) {
  GUARD(
    Ctx* C = (Ctx*)c; gen_key(*C, g);
    const KeyDigit& kd = C->keys.at(g).at(j);
    size_t total = C->q.size();
    for (size_t t = 0; t < total; ++t) {
      std::memcpy(out_b + t * C->N, kd.b[t].data(), C->N * 8);
      std::memcpy(out_a + t * C->N, kd.a[t].data(), C->N * 8);
    }
    return 0;
  )
  return -1;
}
// single-limb transforms by prime index
API int orc_ntt(void* c, uint64_t* a, uint32_t pi, int inverse) {
  Ctx* C = (Ctx*)c; Limb v(a, a + C->N);
  if (inverse) ntt_inverse(*C, v, (int)pi); else ntt_forward(*C, v, (int)pi);
  std::memcpy(a, v.data(), C->N * 8); return 0;
}
// coefficient-domain RNS steps (arrays are [limb][N])
API int orc_modup_coeff(void* c, const uint64_t* in, int level, int digit, uint64_t* out) {
  GUARD(
    Ctx* C = (Ctx*)c; Poly d(level + 1);
    for (int i = 0; i <= level; ++i) d[i].assign(in + (size_t)i * C->N, in + (size_t)(i + 1) * C->N);
    Poly y = modup_coeff(*C, d, level, digit);
    for (size_t e = 0; e < y.size(); ++e) std::memcpy(out + e * C->N, y[e].data(), C->N * 8);
    return 0;
  )
  return -1;
}
API int orc_moddown_coeff(void* c, const uint64_t* in, int level, uint64_t* out) {
  GUARD(
    Ctx* C = (Ctx*)c; Poly x(level + 1 + C->n_p);
    for (size_t i = 0; i < x.size(); ++i) x[i].assign(in + i * C->N, in + (i + 1) * C->N);
    Poly y = moddown_coeff(*C, x, level);
    for (int i = 0; i <= level; ++i) std::memcpy(out + (size_t)i * C->N, y[i].data(), C->N * 8);
    return 0;
  )
  return -1;
}
API int orc_rescale_ntt(void* c, const uint64_t* in, int level, uint64_t* out) {
  GUARD(
    Ctx* C = (Ctx*)c; Poly x(level + 1);
    for (int i = 0; i <= level; ++i) x[i].assign(in + (size_t)i * C->N, in + (size_t)(i + 1) * C->N);
    Poly y = rescale_poly(*C, x, level);
    for (int i = 0; i < level; ++i) std::memcpy(out + (size_t)i * C->N, y[i].data(), C->N * 8);
    return 0;
  )
  return -1;
}
// encode / decode (full-slot): coefficients as integer-valued doubles
API int orc_encode_coeffs(void* c, const double* re, const double* im, double scale, double* out) {
  GUARD(
    Ctx* C = (Ctx*)c; size_t n = C->N / 2; std::vector<cd> z(n);
    for (size_t j = 0; j < n; ++j) z[j] = cd(re[j], im ? im[j] : 0.0);
    std::vector<double> m = encode_coeffs(*C, z, scale);
    std::memcpy(out, m.data(), C->N * 8); return 0;
  )
  return -1;
}
API int orc_decode_coeffs(void* c, const double* m, double scale, double* re, double* im) {
  GUARD(
    Ctx* C = (Ctx*)c; std::vector<double> mv(m, m + C->N);
    std::vector<cd> z = decode_coeffs(*C, mv, scale);
    for (size_t j = 0; j < z.size(); ++j) { re[j] = z[j].real(); if (im) im[j] = z[j].imag(); }
    return 0;
  )
  return -1;
}
// ciphertext handles: limbs are [2][level+1][N], NTT domain
API void* orc_ct_import(void* c, const uint64_t* limbs, int level, double scale) {
  GUARD(
    Ctx* C = (Ctx*)c; if (level < 0 || level > C->L()) throw std::runtime_error("bad level");
    Ct* ct = new Ct; ct->level = level; ct->scale = scale;
    for (int p = 0; p < 2; ++p) {
      ct->c[p].resize(level + 1);
      for (int i = 0; i <= level; ++i) {
        const uint64_t* src = limbs + ((size_t)p * (level + 1) + i) * C->N;
        ct->c[p][i].assign(src, src + C->N);
        for (size_t k = 0; k < C->N; ++k) if (ct->c[p][i][k] >= C->q[i]) { delete ct; throw std::runtime_error("residue out of range"); }
      }
    }
    return ct;
  )
  return nullptr;
}
API int orc_ct_info(void* h, int* level, double* scale) { Ct* ct = (Ct*)h; *level = ct->level; *scale = ct->scale; return 0; }
API int orc_ct_export(void* c, void* h, uint64_t* out) {
  Ctx* C = (Ctx*)c; Ct* ct = (Ct*)h;
  for (int p = 0; p < 2; ++p) for (int i = 0; i <= ct->level; ++i)
    std::memcpy(out + ((size_t)p * (ct->level + 1) + i) * C->N, ct->c[p][i].data(), C->N * 8);
  return 0;
}
API void orc_ct_free(void* h) { delete (Ct*)h; }
API void* orc_encrypt(void* c, const double* re, const double* im, uint64_t n_slots, int level, uint64_t seed) {
  GUARD(
    Ctx* C = (Ctx*)c; std::vector<cd> z(n_slots);
    for (size_t j = 0; j < n_slots; ++j) z[j] = cd(re[j], im ? im[j] : 0.0);
    return new Ct(encrypt(*C, z, level, seed));
  )
  return nullptr;
}
API int orc_bts_encapsulate(void* c, int h) { GUARD(encapsulate(*(Ctx*)c, h); return 0;) return -1; }
// decryption under the ephemeral sparse secret (for checks of the switch to it)
API int orc_decrypt_sparse(void* c, void* h, double* re, double* im) {
  GUARD(
    const Ctx& C = *(Ctx*)c; const Ct& ct = *(Ct*)h;
    if (!C.enc_hw) throw std::runtime_error("no encapsulation");
    std::vector<cd> z = decode_coeffs(C, decrypt_coeffs_under(C, ct, C.s_sparse_ntt), ct.scale);
    for (size_t j = 0; j < z.size(); ++j) { re[j] = z[j].real(); if (im) im[j] = z[j].imag(); }
    return 0;
  )
  return -1;
}
API int orc_decrypt(void* c, void* h, double* re, double* im) {
  GUARD(
    std::vector<cd> z = decrypt(*(Ctx*)c, *(Ct*)h);
    for (size_t j = 0; j < z.size(); ++j) { re[j] = z[j].real(); if (im) im[j] = z[j].imag(); }
    return 0;
  )
  return -1;
}
API int orc_decrypt_coeffs(void* c, void* h, double* out) {
  GUARD(
    std::vector<double> m = decrypt_coeffs(*(Ctx*)c, *(Ct*)h);
    std::memcpy(out, m.data(), m.size() * 8); return 0;
  )
  return -1;
}
#define CT_OP(...) GUARD(return new Ct(__VA_ARGS__);) return nullptr;
API void* orc_add(void* c, void* a, void* b) { CT_OP(add_sub(*(Ctx*)c, *(Ct*)a, *(Ct*)b, false)) }
API void* orc_sub(void* c, void* a, void* b) { CT_OP(add_sub(*(Ctx*)c, *(Ct*)a, *(Ct*)b, true)) }
API void* orc_mul_relin(void* c, void* a, void* b) { CT_OP(mul_relin(*(Ctx*)c, *(Ct*)a, *(Ct*)b)) }
API void* orc_mul(void* c, void* a, void* b) { CT_OP(mul(*(Ctx*)c, *(Ct*)a, *(Ct*)b)) }
API void* orc_rescale(void* c, void* a) { CT_OP(rescale(*(Ctx*)c, *(Ct*)a)) }
API void* orc_rotate(void* c, void* a, int64_t steps) { CT_OP(rotate(*(Ctx*)c, *(Ct*)a, steps)) }
API void* orc_encapsulation_switch(void* c, void* a, int to_sparse) {
  CT_OP(((Ctx*)c)->enc_hw ? switch_key(*(Ctx*)c, *(Ct*)a, to_sparse ? 2 : 4)
                          : throw std::runtime_error("no encapsulation"))
}
API void* orc_conjugate(void* c, void* a) { CT_OP(conjugate(*(Ctx*)c, *(Ct*)a)) }
// hoisted rotations: out[i] receives the rotation by steps[i]; returns 0 or -1
API int orc_rotate_hoisted(void* c, void* a, const int64_t* steps, int n, void** out) {
  GUARD(
    std::vector<i64> st(steps, steps + n);
    std::vector<Ct> r = rotate_hoisted(*(Ctx*)c, *(Ct*)a, st);
    for (int i = 0; i < n; ++i) out[i] = new Ct(r[i]);
    return 0;
  )
  return -1;
}
API void* orc_mul_const(void* c, void* a, double v, double target_scale) { CT_OP(mul_const_to(*(Ctx*)c, *(Ct*)a, v, target_scale)) }
API void* orc_add_const(void* c, void* a, double v) { CT_OP(add_const(*(Ctx*)c, *(Ct*)a, v)) }
API void* orc_mul_int(void* c, void* a, int64_t m) { CT_OP(mul_int(*(Ctx*)c, *(Ct*)a, m)) }
API void* orc_drop(void* c, void* a, int level) { (void)c; CT_OP(drop_to(*(Ct*)a, level)) }
API void* orc_invsqrt(void* c, void* a, double lo, double hi, double B, uint32_t degree, uint32_t iters,
                      uint32_t pre_bts, uint64_t bts_mask, uint32_t log_slots) {
  InvSqrtCfg cfg{lo, hi, B, (int)degree, (int)iters, (int)pre_bts, bts_mask, (int)log_slots};
  CT_OP(invsqrt(*(Ctx*)c, *(Ct*)a, cfg))
}
// sum_j c_j T_j(t) for t in [-1, 1], output at the context scale; need < 0: the fewest-levels plan,
// else the fewest-products plan when it ends at level >= need
API void* orc_cheb_eval(void* c, void* t, const double* coeffs, uint32_t d, int need) {
  std::vector<double> cv(coeffs, coeffs + d + 1);
  ChebEval ev(*(Ctx*)c);
  CT_OP(ev.run(*(Ct*)t, cv, need))
}
API int orc_cheb_coeffs(double lo, double hi, uint32_t d, double* out) {
  std::vector<double> c = cheb_coeffs(lo, hi, (int)d);
  std::memcpy(out, c.data(), c.size() * 8); return 0;
}
API double orc_clenshaw(const double* c, uint32_t d, double t) {
  std::vector<double> cv(c, c + d + 1); return clenshaw(cv, t);
}
API int orc_plain_invsqrt(const double* a, uint64_t n, double lo, double hi, double B, uint32_t degree, uint32_t iters,
                          double* out) {
  InvSqrtCfg cfg{lo, hi, B, (int)degree, (int)iters, 0, 0};
  plain_invsqrt(a, n, cfg, out); return 0;
}
// raw PRNG / sampler access for pins
API uint64_t orc_splitmix_stream(uint64_t seed, uint64_t tag, uint64_t n, uint64_t* out) {
  Stream s(seed, tag); for (uint64_t i = 0; i < n; ++i) out[i] = s.next(); return n;
}

// hybrid key switch of an NTT-domain polynomial d (limbs 0..level) under the key for g
API int orc_key_switch(void* c, const uint64_t* d, int level, uint64_t g, uint64_t* out) {
  GUARD(
    Ctx* C = (Ctx*)c; gen_key(*C, g);
    Poly x(level + 1);
    for (int i = 0; i <= level; ++i) x[i].assign(d + (size_t)i * C->N, d + (size_t)(i + 1) * C->N);
    Poly o0, o1; key_switch(*C, x, level, g, o0, o1);
    for (int i = 0; i <= level; ++i) {
      std::memcpy(out + (size_t)i * C->N, o0[i].data(), C->N * 8);
      std::memcpy(out + (size_t)(level + 1 + i) * C->N, o1[i].data(), C->N * 8);
    }
    return 0;
  )
  return -1;
}

API int orc_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

API int orc_bts_setup(void* c, int K, int r, int deg, int cts, int stc) {
  GUARD(
    Ctx* C = (Ctx*)c;
    C->bts_K = K; C->bts_r = r; C->bts_deg = deg; C->bts_cts = cts; C->bts_stc = stc;
    if (C->L() - bts_levels(*C) < 1) throw std::runtime_error("prime chain too short for bootstrapping");
    C->bts_on = true;
    return C->L() - bts_levels(*C);
  )
  return -1;
}
API void* orc_bootstrap(void* c, void* a) { CT_OP(bootstrap_core(*(Ctx*)c, *(Ct*)a)) }
API void* orc_bootstrap_scaled(void* c, void* a, int64_t Y) { CT_OP(bootstrap_scaled(*(Ctx*)c, *(Ct*)a, Y)) }
API void* orc_mod_raise(void* c, void* a) { CT_OP(mod_raise(*(Ctx*)c, *(Ct*)a)) }
API void* orc_mul_monomial(void* c, void* a, uint64_t e) { CT_OP(mul_monomial(*(Ctx*)c, *(Ct*)a, e)) }
// diagonals of the grouped special-FFT factors: writes the offsets of group g into
// offsets[cap] and returns how many (diagonals themselves via orc_fft_group_diag)
API int orc_fft_group_offsets(void* c, int groups, int inverse, int g, int64_t* offsets, int cap) {
  GUARD(
    Ctx* C = (Ctx*)c; std::vector<DiagMap> G = fft_groups(C->N / 2, groups, inverse != 0);
    int k = 0; for (auto& e : G.at(g)) { if (k < cap) offsets[k] = e.first; ++k; }
    return k;
  )
  return -1;
}
API int orc_fft_group_diag(void* c, int groups, int inverse, int g, int64_t offset, double* re, double* im) {
  GUARD(
    Ctx* C = (Ctx*)c; std::vector<DiagMap> G = fft_groups(C->N / 2, groups, inverse != 0);
    const std::vector<cd>& d = G.at(g).at(offset);
    for (size_t s = 0; s < d.size(); ++s) { re[s] = d[s].real(); im[s] = d[s].imag(); }
    return 0;
  )
  return -1;
}
// the same for 2^log_slots slots (sparse packing); packed = 1 gives the packed form of the last
// CoeffToSlot group (inverse) or the first SlotToCoeff group, of period 2^(log_slots+1)
static DiagMap fft_group_ex(const Ctx& C, int groups, int inverse, int g, int log_slots, int packed) {
  size_t n = log_slots ? (size_t)1 << log_slots : C.N / 2;
  std::vector<DiagMap> G = fft_groups(n, groups, inverse != 0);
  if (!packed) return G.at(g);
  if (inverse) { if (g != groups - 1) throw std::runtime_error("packed: last CoeffToSlot group only"); return pack_cts_last(G.back(), n); }
  if (g != 0) throw std::runtime_error("packed: first SlotToCoeff group only");
  return pack_stc_first(G[0], n);
}
API int orc_fft_group_ex_offsets(void* c, int groups, int inverse, int g, int log_slots, int packed, int64_t* offsets,
                                 int cap) {
  GUARD(
    DiagMap M = fft_group_ex(*(Ctx*)c, groups, inverse, g, log_slots, packed);
    int k = 0; for (auto& e : M) { if (k < cap) offsets[k] = e.first; ++k; }
    return k;
  )
  return -1;
}
API int orc_fft_group_ex_diag(void* c, int groups, int inverse, int g, int log_slots, int packed, int64_t offset,
                              double* re, double* im, int cap) {
  GUARD(
    DiagMap M = fft_group_ex(*(Ctx*)c, groups, inverse, g, log_slots, packed);
    const std::vector<cd>& d = M.at(offset);
    if ((int)d.size() > cap) throw std::runtime_error("diagonal longer than the buffer");
    for (size_t s = 0; s < d.size(); ++s) { re[s] = d[s].real(); im[s] = d[s].imag(); }
    return (int)d.size();
  )
  return -1;
}
// single steps of bootstrapping, for tests
API void* orc_linear_transform_group(void* c, void* a, int groups, int inverse, int g, double target) {
  CT_OP(linear_transform(*(Ctx*)c, *(Ct*)a, fft_groups(((Ctx*)c)->N / 2, groups, inverse != 0).at(g), target,
                         (long)(((Ctx*)c)->N / 2)))
}
API void* orc_bootstrap_slots(void* c, void* a, int log_slots) { CT_OP(bootstrap_core(*(Ctx*)c, *(Ct*)a, log_slots)) }
API void* orc_bootstrap_scaled_slots(void* c, void* a, int64_t Y, int log_slots) {
  CT_OP(bootstrap_scaled(*(Ctx*)c, *(Ct*)a, Y, log_slots))
}
API void* orc_sub_sum(void* c, void* a, int log_slots) { CT_OP(sub_sum(*(Ctx*)c, *(Ct*)a, 1ull << log_slots)) }
API void* orc_eval_mod(void* c, void* a) { CT_OP(eval_mod(*(Ctx*)c, *(Ct*)a)) }
API void* orc_set_scale(void* c, void* a, double scale) { (void)c; Ct r = *(Ct*)a; r.scale = scale; return new Ct(r); }
