// Host orchestration of the CKKS operations of Sec. 2.1 over the device
// kernels: Add/Sub, Mul_C (tensor product + hybrid key switching), rescale,
// Mul_P by constants, Galois automorphisms (rotation, conjugation).
// Ciphertexts stay in the NTT domain; every temporary is stream-ordered on the
// context's stream.
#include <cmath>

#include "internal.cuh"
#include "kernels.cuh"

namespace hedap {

static LimbSet qset(u64* base, size_t part_stride, int n_parts, int first, int count, int prime_offset = 0) {
  return LimbSet{base, part_stride, n_parts, first, count, INT_MAX, prime_offset, 0};
}

std::unique_ptr<Ct> ct_alloc(Ctx& C, int level) {
  if (level < 0 || level > C.L()) throw Error(HEDAP_ERR_LEVEL, "level out of range");
  auto c = std::make_unique<Ct>();
  c->N = C.N;
  c->cap = level + 1;
  c->level = level;
  c->scale = C.scale;
  c->buf = DevBuf(2 * (size_t)(level + 1) * C.N, C.stream);
  return c;
}

std::unique_ptr<Ct> ct_copy(Ctx& C, const Ct& a, int level) {
  if (level > a.level) throw Error(HEDAP_ERR_LEVEL, "cannot raise the level by copying");
  auto c = ct_alloc(C, level);
  c->scale = a.scale;
  for (int p = 0; p < 2; ++p)
    HEDAP_CUDA(cudaMemcpyAsync(c->part(p), a.part(p), (size_t)(level + 1) * C.N * 8, cudaMemcpyDeviceToDevice,
                               C.stream));
  return c;
}
std::unique_ptr<Ct> ev_drop(Ctx& C, const Ct& a, int level) {
  if (level < 0) throw Error(HEDAP_ERR_LEVEL, "negative level");
  return ct_copy(C, a, level);
}

static void check_scales(double a, double b) {
  if (std::fabs(a / b - 1.0) > 1e-12) throw Error(HEDAP_ERR_SCALE, "operand scales differ");
}

std::unique_ptr<Ct> ev_add(Ctx& C, const Ct& a, const Ct& b, bool sub) {
  const int l = std::min(a.level, b.level);
  check_scales(a.scale, b.scale);
  auto o = ct_alloc(C, l);
  o->scale = a.scale;
  k_add_sub(C, a.part(0), a.part_stride(), b.part(0), b.part_stride(), o->part(0), o->part_stride(), l + 1, sub);
  return o;
}

// ------------------------------------------------------------------ level constants
const LevelConsts& level_consts(Ctx& C, int l) {
  auto it = C.lc.find(l);
  if (it != C.lc.end()) return *it->second;
  auto L = std::make_unique<LevelConsts>();
  const int a = C.alpha, dn = C.dnum(l), K = C.n_p, ext = l + 1 + K;
  const u64* q = C.primes.data();
  auto prime_of_ext = [&](int t) { return t <= l ? q[t] : q[C.n_q + (t - l - 1)]; };
  std::vector<u64> v(2 * (l + 1) + (size_t)dn * a * ext, 0);
  for (int j = 0; j < dn; ++j) {
    const int lo = j * a, hi = std::min(lo + a, l + 1);
    for (int i = lo; i < hi; ++i) {
      u64 h = 1;
      for (int m = lo; m < hi; ++m)
        if (m != i) h = h_mulmod(h, q[m] % q[i], q[i]);
      const u64 inv = h_invmod(h, q[i]);
      v[i] = inv;
      v[(l + 1) + i] = h_shoup(inv, q[i]);
      for (int t = 0; t < ext; ++t) {
        const u64 pt = prime_of_ext(t);
        u64 hm = 1 % pt;
        for (int m = lo; m < hi; ++m)
          if (m != i) hm = h_mulmod(hm, q[m] % pt, pt);
        v[2 * (l + 1) + ((size_t)j * a + (i - lo)) * ext + t] = hm;
      }
    }
  }
  L->modup = DevBuf(v.size(), C.stream);
  HEDAP_CUDA(cudaMemcpyAsync(L->modup.p, v.data(), v.size() * 8, cudaMemcpyHostToDevice, C.stream));
  HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  if (l >= 1) {
    const u64 ql = q[l];
    for (int i = 0; i < l; ++i) {
      L->rescale.ql_mod[i] = ql % q[i];
      L->rescale.inv[i] = h_invmod(ql % q[i], q[i]);
      L->rescale.inv_sh[i] = h_shoup(L->rescale.inv[i], q[i]);
    }
  }
  auto& ref = *L;
  C.lc[l] = std::move(L);
  return ref;
}

// ------------------------------------------------------------------ key switching
// Hybrid key switching (Han-Ki 2020) of d (NTT domain, limbs 0..l) with the key
// for `galois`: iNTT, ModUp of every digit to Q_l u P, NTT, inner product with
// the key digits, iNTT of the P limbs, ModDown (rounded division by P), NTT.
void key_switch(Ctx& C, const u64* d_ntt, int l, u64 galois, u64* out0, u64* out1, bool acc0, bool acc1) {
  auto it = C.keys.find(galois);
  if (it == C.keys.end()) {
    gen_galois_key(C, galois);
    it = C.keys.find(galois);
  }
  const size_t N = C.N;
  const int K = C.n_p, ext = l + 1 + K, dn = C.dnum(l);
  const LevelConsts& LC = level_consts(C, l);
  DevBuf dc((size_t)(l + 1) * N, C.stream);
  HEDAP_CUDA(cudaMemcpyAsync(dc.p, d_ntt, (size_t)(l + 1) * N * 8, cudaMemcpyDeviceToDevice, C.stream));
  ntt_inverse(C.tab, qset(dc.p, 0, 1, 0, l + 1), C.stream);
  DevBuf y((size_t)dn * ext * N, C.stream);
  k_modup(C, dc.p, y.p, l, LC.modup.p);
  ntt_forward(C.tab, LimbSet{y.p, (size_t)ext * N, dn, 0, ext, l + 1, 0, C.n_q}, C.stream);
  DevBuf acc(2 * (size_t)ext * N, C.stream);
  k_ksk_inner(C, y.p, it->second.p, acc.p, l);
  ntt_inverse(C.tab, LimbSet{acc.p, (size_t)ext * N, 2, l + 1, K, l + 1, 0, C.n_q}, C.stream);
  DevBuf v(2 * (size_t)(l + 1) * N, C.stream);
  k_moddown_spread(C, acc.p, v.p, l);
  ntt_forward(C.tab, qset(v.p, (size_t)(l + 1) * N, 2, 0, l + 1), C.stream);
  k_moddown_finish(C, acc.p, v.p, out0, out1, l, acc0, acc1);
}

std::unique_ptr<Ct> ev_mul_relin(Ctx& C, const Ct& a, const Ct& b) {
  const int l = std::min(a.level, b.level);
  auto o = ct_alloc(C, l);
  o->scale = a.scale * b.scale;
  DevBuf d2((size_t)(l + 1) * C.N, C.stream);
  k_tensor(C, a.part(0), a.part(1), b.part(0), b.part(1), o->part(0), o->part(1), d2.p, l + 1);
  key_switch(C, d2.p, l, 0, o->part(0), o->part(1), true, true);
  return o;
}

// rescale by q_l: c_i <- (c_i - [c_l]_centred) * q_l^-1 mod q_i, i < l
std::unique_ptr<Ct> ev_rescale(Ctx& C, const Ct& a) {
  const int l = a.level;
  if (l < 1) throw Error(HEDAP_ERR_LEVEL, "rescale needs level >= 1");
  const size_t N = C.N;
  const LevelConsts& LC = level_consts(C, l);
  auto o = ct_alloc(C, l - 1);
  o->scale = a.scale / (double)C.primes[l];
  DevBuf last(2 * N, C.stream);
  for (int p = 0; p < 2; ++p)
    HEDAP_CUDA(cudaMemcpyAsync(last.p + p * N, a.part(p) + (size_t)l * N, N * 8, cudaMemcpyDeviceToDevice, C.stream));
  ntt_inverse(C.tab, qset(last.p, N, 2, 0, 1, l), C.stream);
  DevBuf tmp(2 * (size_t)l * N, C.stream);
  k_rescale_spread(C, last.p, N, tmp.p, (size_t)l * N, l, LC.rescale);
  ntt_forward(C.tab, qset(tmp.p, (size_t)l * N, 2, 0, l), C.stream);
  k_rescale_finish(C, a.part(0), a.part_stride(), tmp.p, (size_t)l * N, o->part(0), o->part_stride(), l,
                   LC.rescale);
  return o;
}

std::unique_ptr<Ct> ev_mul(Ctx& C, const Ct& a, const Ct& b) { return ev_rescale(C, *ev_mul_relin(C, a, b)); }

u64 galois_for_rotation(const Ctx& C, i64 steps) {
  const i64 h = (i64)(C.N / 2);
  const i64 r = ((steps % h) + h) % h;
  return h_powmod(5, (u64)r, 2 * C.N);
}

std::unique_ptr<Ct> ev_galois(Ctx& C, const Ct& a, u64 g) {
  const int l = a.level;
  auto o = ct_alloc(C, l);
  o->scale = a.scale;
  k_automorph(C, a.part(0), a.part_stride(), o->part(0), o->part_stride(), 2, l + 1, g);
  key_switch(C, o->part(1), l, g, o->part(0), o->part(1), true, false);
  return o;
}

// Mul_P by a real constant c at plaintext scale target * q_l / scale, then rescale;
// the result's scale is set to exactly `target`.
std::unique_ptr<Ct> ev_mul_const(Ctx& C, const Ct& a, double c, double target) {
  const int l = a.level;
  if (l < 1) throw Error(HEDAP_ERR_LEVEL, "constant multiplication needs level >= 1");
  const double sp = target * (double)C.primes[l] / a.scale;
  const double v = std::round(c * sp);
  LimbConsts K;
  for (int i = 0; i <= l; ++i) {
    K.w[i] = h_double_to_mod(v, C.primes[i]);
    K.wsh[i] = h_shoup(K.w[i], C.primes[i]);
  }
  auto t = ct_alloc(C, l);
  t->scale = a.scale * sp;
  k_mul_limbconst(C, a.part(0), a.part_stride(), t->part(0), t->part_stride(), 2, l + 1, K);
  auto o = ev_rescale(C, *t);
  o->scale = target;
  return o;
}

std::unique_ptr<Ct> ev_add_const(Ctx& C, const Ct& a, double c) {
  const double v = std::round(c * a.scale);
  LimbConsts K;
  for (int i = 0; i <= a.level; ++i) K.w[i] = h_double_to_mod(v, C.primes[i]);
  auto o = ct_copy(C, a, a.level);
  k_add_limbconst(C, o->part(0), a.level + 1, K);
  return o;
}

std::unique_ptr<Ct> ev_mul_int(Ctx& C, const Ct& a, i64 m) {
  LimbConsts K;
  for (int i = 0; i <= a.level; ++i) {
    K.w[i] = h_smod(m, C.primes[i]);
    K.wsh[i] = h_shoup(K.w[i], C.primes[i]);
  }
  auto o = ct_alloc(C, a.level);
  o->scale = a.scale;
  k_mul_limbconst(C, a.part(0), a.part_stride(), o->part(0), o->part_stride(), 2, a.level + 1, K);
  return o;
}

}  // namespace hedap
