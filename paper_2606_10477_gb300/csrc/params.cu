// Host-side number theory, randomness and device buffers.
#include <cmath>

#include "internal.cuh"

namespace hedap {

typedef unsigned __int128 u128;

u64 h_mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }
u64 h_powmod(u64 a, u64 e, u64 q) {
  u64 acc = 1 % q, base = a % q;
  for (; e; e >>= 1) {
    if (e & 1) acc = h_mulmod(acc, base, q);
    base = h_mulmod(base, base, q);
  }
  return acc;
}
u64 h_invmod(u64 a, u64 q) { return h_powmod(a, q - 2, q); }

// Miller-Rabin with the first twelve prime bases: deterministic below 2^64.
bool h_is_prime(u64 n) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 b : bases)
    if (n % b == 0) return n == b;
  u64 d = n - 1;
  int r = 0;
  while (!(d & 1)) { d >>= 1; ++r; }
  for (u64 b : bases) {
    u64 x = h_powmod(b, d, n);
    if (x == 1 || x == n - 1) continue;
    int i = 1;
    for (; i < r; ++i) {
      x = h_mulmod(x, x, n);
      if (x == n - 1) break;
    }
    if (i == r) return false;
  }
  return true;
}

// Prime chain: for bit size b, the candidates 2^b + k*2N + 1 then 2^b - k*2N + 1
// for k = 1, 2, ..., the first prime not already taken.
std::vector<u64> h_prime_chain(int log_n, const std::vector<int>& bits) {
  const u64 step = 2ull << log_n;
  std::vector<u64> chosen;
  auto taken = [&](u64 v) {
    for (u64 c : chosen)
      if (c == v) return true;
    return false;
  };
  for (int b : bits) {
    if (b < 33 || b > 60) throw Error(HEDAP_ERR_ARG, "prime bit sizes must lie in [33, 60]");
    const u64 center = 1ull << b;
    u64 pick = 0;
    for (u64 k = 1; !pick; ++k) {
      u64 above = center + k * step + 1;
      if (h_is_prime(above) && !taken(above)) { pick = above; break; }
      if (k * step < center) {
        u64 below = center - k * step + 1;
        if (h_is_prime(below) && !taken(below)) pick = below;
      }
    }
    chosen.push_back(pick);
  }
  return chosen;
}

// psi: the first x^((q-1)/2N), x = 2, 3, ..., with psi^N = -1 (a primitive 2N-th root).
u64 h_find_psi(u64 q, int log_n) {
  const u64 n = 1ull << log_n, e = (q - 1) >> (log_n + 1);
  for (u64 x = 2;; ++x) {
    u64 c = h_powmod(x, e, q);
    if (h_powmod(c, n, q) == q - 1) return c;
  }
}

u64 h_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

PrimeDev h_prime_dev(u64 q) {
  PrimeDev p;
  p.q = q;
  p.b = 64 - __builtin_clzll(q);
  p.mu = (u64)(((u128)1 << (2 * p.b)) / q);
  p.pad = 0;
  return p;
}

uint32_t h_bitrev(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

u64 h_smod(i64 v, u64 q) {
  if (v >= 0) return (u64)v % q;
  u64 m = (u64)(-(v + 1)) % q;  // |v| - 1 reduced
  return q - 1 - m;
}

// An integer-valued double x equals M * 2^k with M < 2^53 an integer; reduce
// each factor (|x| may exceed 2^64).
u64 h_double_to_mod(double x, u64 q) {
  double ax = std::fabs(x);
  u64 r;
  if (ax < 1.8e19) {
    r = (u64)ax % q;
  } else {
    int ex;
    double fr = std::frexp(ax, &ex);
    u64 M = (u64)std::ldexp(fr, 53);
    r = h_mulmod(M % q, h_powmod(2, (u64)(ex - 53), q), q);
  }
  return (x < 0 && r) ? q - r : r;
}

// ------------------------------------------------------------------ SplitMix64
static inline u64 sm_mix(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
SplitMix::SplitMix(u64 seed, u64 tag) : state(sm_mix(seed) ^ sm_mix(tag ^ 0x5851F42D4C957F2Dull)) {}
u64 SplitMix::next() {
  state += 0x9E3779B97F4A7C15ull;
  return sm_mix(state);
}
// uniform residue: top bits of a draw, rejected while >= q
u64 draw_uniform(SplitMix& s, u64 q) {
  const int shift = __builtin_clzll(q);
  for (;;) {
    u64 v = s.next() >> shift;
    if (v < q) return v;
  }
}
// centred binomial distribution with eta = 21 from one draw
i64 draw_cbd21(SplitMix& s) {
  u64 r = s.next();
  const u64 m21 = (1ull << 21) - 1;
  return (i64)__builtin_popcountll(r & m21) - (i64)__builtin_popcountll((r >> 21) & m21);
}
// ternary secret: dense uniform over {-1,0,1} (hw = 0) or fixed Hamming weight hw
std::vector<i64> draw_ternary(SplitMix& s, int log_n, int hw) {
  const size_t n = (size_t)1 << log_n;
  std::vector<i64> v(n, 0);
  if (hw == 0) {
    for (size_t i = 0; i < n; ++i) {
      u64 t;
      do { t = s.next() >> 62; } while (t == 3);
      v[i] = (i64)t - 1;
    }
    return v;
  }
  for (int placed = 0; placed < hw;) {
    u64 r = s.next();
    size_t pos = (size_t)(r >> (64 - log_n));
    if (v[pos] != 0) continue;
    v[pos] = (r & 1) ? 1 : -1;
    ++placed;
  }
  return v;
}

// ------------------------------------------------------------------ device buffers
DevBuf::DevBuf(size_t n, cudaStream_t st) : words(n), s(st) {
  if (n) HEDAP_CUDA(cudaMallocAsync((void**)&p, n * sizeof(u64), st));
}
DevBuf::~DevBuf() {
  if (p) cudaFreeAsync(p, s);
}
DevBuf& DevBuf::operator=(DevBuf&& o) noexcept {
  if (this != &o) {
    if (p) cudaFreeAsync(p, s);
    p = o.p; words = o.words; s = o.s;
    o.p = nullptr; o.words = 0;
  }
  return *this;
}

// ------------------------------------------------------------------ stream pool
cudaStream_t StreamPool::get() {
  if (!idle.empty()) {
    cudaStream_t s = idle.back();
    idle.pop_back();
    return s;
  }
  cudaStream_t s = nullptr;
  HEDAP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  all.push_back(s);
  return s;
}
void StreamPool::put(cudaStream_t s) { idle.push_back(s); }
StreamPool::~StreamPool() {
  for (cudaStream_t s : all) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
}

}  // namespace hedap
