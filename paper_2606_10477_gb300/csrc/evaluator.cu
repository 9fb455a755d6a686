// Host orchestration of the CKKS operations of Sec. 2.1 over the device
// kernels: Add/Sub, Mul_C (tensor product + hybrid key switching), rescale,
// Mul_P by constants, Galois automorphisms (rotation, conjugation).
// Every operation works on a batch of ciphertexts at one level and scale (a
// single ciphertext is a batch of one); each launch covers the whole batch.
// Ciphertexts stay in the NTT domain; temporaries are stream-ordered on the
// context's stream.
#include <cmath>

#include "internal.cuh"
#include "kernels.cuh"
#include "profiler.cuh"

namespace hedap {

static LimbSet qset(u64* base, size_t part_stride, int n_parts, int first, int count, int prime_offset = 0) {
  return LimbSet{base, part_stride, n_parts, first, count, INT_MAX, prime_offset, 0};
}

std::unique_ptr<Ct> ct_alloc(Ctx& C, int level, int batch) {
  if (level < 0 || level > C.L()) throw Error(HEDAP_ERR_LEVEL, "level out of range");
  if (batch < 1 || batch > kMaxBatch) throw Error(HEDAP_ERR_ARG, "batch must lie in [1, 16]");
  auto c = std::make_unique<Ct>();
  c->owner = &C;
  c->N = C.N;
  c->cap = level + 1;
  c->level = level;
  c->batch = batch;
  c->scale = C.scale;
  c->buf = DevBuf(2 * (size_t)batch * (level + 1) * C.N, C.stream);
  return c;
}

// copy limbs 0..level of every part of a into a new (packed) batch
std::unique_ptr<Ct> ct_copy(Ctx& C, const Ct& a, int level) {
  if (level > a.level) throw Error(HEDAP_ERR_LEVEL, "cannot raise the level by copying");
  auto c = ct_alloc(C, level, a.batch);
  c->scale = a.scale;
  HEDAP_CUDA(cudaMemcpy2DAsync(c->part(0), c->part_stride() * 8, a.part(0), a.part_stride() * 8,
                               (size_t)(level + 1) * C.N * 8, a.parts(), cudaMemcpyDeviceToDevice, C.stream));
  return c;
}
std::unique_ptr<Ct> ev_drop(Ctx& C, const Ct& a, int level) {
  if (level < 0) throw Error(HEDAP_ERR_LEVEL, "negative level");
  return ct_copy(C, a, level);
}

std::unique_ptr<Ct> batch_pack(Ctx& C, const std::vector<const Ct*>& cts) {
  if (cts.empty()) throw Error(HEDAP_ERR_ARG, "empty batch");
  const Ct& f = *cts[0];
  int total = 0;
  for (const Ct* c : cts) {
    if (c->level != f.level || c->scale != f.scale) throw Error(HEDAP_ERR_ARG, "batched ciphertexts differ in level or scale");
    total += c->batch;
  }
  auto b = ct_alloc(C, f.level, total);
  b->scale = f.scale;
  int at = 0;
  for (const Ct* c : cts) {
    HEDAP_CUDA(cudaMemcpy2DAsync(b->part(2 * at), b->part_stride() * 8, c->part(0), c->part_stride() * 8,
                                 (size_t)(f.level + 1) * C.N * 8, c->parts(), cudaMemcpyDeviceToDevice, C.stream));
    at += c->batch;
  }
  return b;
}
std::unique_ptr<Ct> batch_slice(Ctx& C, const Ct& b, int first, int count) {
  if (first < 0 || count < 1 || first + count > b.batch) throw Error(HEDAP_ERR_ARG, "batch slice out of range");
  auto c = ct_alloc(C, b.level, count);
  c->scale = b.scale;
  HEDAP_CUDA(cudaMemcpy2DAsync(c->part(0), c->part_stride() * 8, b.part(2 * first), b.part_stride() * 8,
                               (size_t)(b.level + 1) * C.N * 8, 2 * count, cudaMemcpyDeviceToDevice, C.stream));
  return c;
}
std::unique_ptr<Ct> batch_unpack(Ctx& C, const Ct& b, int k) {
  if (k < 0 || k >= b.batch) throw Error(HEDAP_ERR_ARG, "batch index out of range");
  auto c = ct_alloc(C, b.level, 1);
  c->scale = b.scale;
  HEDAP_CUDA(cudaMemcpy2DAsync(c->part(0), c->part_stride() * 8, b.part(2 * k), b.part_stride() * 8,
                               (size_t)(b.level + 1) * C.N * 8, 2, cudaMemcpyDeviceToDevice, C.stream));
  return c;
}

static void check_scales(double a, double b) {
  if (std::fabs(a / b - 1.0) > 1e-12) throw Error(HEDAP_ERR_SCALE, "operand scales differ");
}
static void check_batches(const Ct& a, const Ct& b) {
  if (a.batch != b.batch) throw Error(HEDAP_ERR_ARG, "operands have different batch sizes");
}

std::unique_ptr<Ct> ev_add(Ctx& C, const Ct& a, const Ct& b, bool sub) {
  const int l = std::min(a.level, b.level);
  check_scales(a.scale, b.scale);
  check_batches(a, b);
  auto o = ct_alloc(C, l, a.batch);
  o->scale = a.scale;
  k_add_sub(C, a.part(0), a.part_stride(), b.part(0), b.part_stride(), o->part(0), o->part_stride(), a.parts(),
            l + 1, sub);
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
  const size_t nb = (size_t)dn * a * ext;  // qhat table size; its Shoup companions follow it
  std::vector<u64> v(2 * (l + 1) + 2 * nb, 0);
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
        v[2 * (l + 1) + nb + ((size_t)j * a + (i - lo)) * ext + t] = h_shoup(hm, pt);
      }
    }
  }
  L->modup = DevBuf(v.size(), C.stream);
  HEDAP_CUDA(cudaMemcpyAsync(L->modup.p, v.data(), v.size() * 8, cudaMemcpyHostToDevice, C.stream));
  // the key switch's fused ModUp: every factor divided by the key's scale (Ctx::key_scale); the factor
  // of the folded limb becomes 1 and is marked by a Shoup companion 0
  std::vector<u64> vk(v);
  double products = 0;
  const int T = C.total_primes();
  for (int j = 0; j < dn; ++j) {
    const int lo = j * a, hi = std::min(lo + a, l + 1);
    for (int t = 0; t < ext; ++t) {
      if (t >= lo && t < hi) continue;  // the digit's own limbs are not converted
      const int gt = t <= l ? t : C.n_q + (t - l - 1);
      const u64 pt = prime_of_ext(t), un = C.key_unscale[(size_t)j * T + gt];
      const int i0 = C.key_scale_i0[(size_t)j * T + gt];
      for (int i = lo; i < hi; ++i) {
        const size_t at = 2 * (l + 1) + ((size_t)j * a + (i - lo)) * ext + t;
        const u64 f = h_mulmod(v[at], un, pt);
        vk[at] = f;
        vk[at + nb] = (i == i0 && f == 1) ? 0 : h_shoup(f, pt);
        products += vk[at + nb] ? 1 : 0;
      }
    }
  }
  L->modup_products = products;
  L->modup_ks = DevBuf(vk.size(), C.stream);
  HEDAP_CUDA(cudaMemcpyAsync(L->modup_ks.p, vk.data(), vk.size() * 8, cudaMemcpyHostToDevice, C.stream));
  // the key switch's inverse NTT ends with N^-1 qhat_i^-1 instead of N^-1, so that its output is the
  // first factor [x_i qhat_i^-1]_{q_i} of the fast basis conversion
  std::vector<u64> post(2 * (l + 1));
  for (int i = 0; i <= l; ++i) {
    post[2 * i] = h_mulmod(h_invmod(C.N % q[i], q[i]), v[i], q[i]);
    post[2 * i + 1] = h_shoup(post[2 * i], q[i]);
  }
  L->intt_post = DevBuf(post.size(), C.stream);
  HEDAP_CUDA(cudaMemcpyAsync(L->intt_post.p, post.data(), post.size() * 8, cudaMemcpyHostToDevice, C.stream));
  HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  if (l >= 1) {
    const u64 ql = q[l];
    std::vector<u64> r(3 * (size_t)l);
    for (int i = 0; i < l; ++i) {
      L->rescale.ql_mod[i] = ql % q[i];
      L->rescale.inv[i] = h_invmod(ql % q[i], q[i]);
      L->rescale.inv_sh[i] = h_shoup(L->rescale.inv[i], q[i]);
      r[i] = L->rescale.ql_mod[i];
      r[l + i] = L->rescale.inv[i];
      r[2 * l + i] = L->rescale.inv_sh[i];
    }
    L->d_rescale = DevBuf(r.size(), C.stream);
    HEDAP_CUDA(cudaMemcpyAsync(L->d_rescale.p, r.data(), r.size() * 8, cudaMemcpyHostToDevice, C.stream));
    // ModDown fused with this level's rescale (ks_moddown_rescale)
    const int K = C.n_p;
    auto P_mod = [&](u64 m) {
      u64 v = 1 % m;
      for (int k = 0; k < K; ++k) v = h_mulmod(v, q[C.n_q + k] % m, m);
      return v;
    };
    std::vector<u64> w(2 * (size_t)l);
    for (int i = 0; i < l; ++i) {
      w[i] = h_mulmod(h_invmod(P_mod(q[i]), q[i]), L->rescale.inv[i], q[i]);
      w[l + i] = h_shoup(w[i], q[i]);
    }
    L->d_mdr = DevBuf(w.size(), C.stream);
    HEDAP_CUDA(cudaMemcpyAsync(L->d_mdr.p, w.data(), w.size() * 8, cudaMemcpyHostToDevice, C.stream));
    MdrLast& M = L->mdr_last;
    M = MdrLast{};
    M.K = std::min(K, 8);
    const u64 pinv = h_invmod(P_mod(ql), ql);
    for (int k = 0; k < M.K; ++k) {
      const u64 pk = q[C.n_q + k];
      u64 h = 1;  // phinv_k = (P / p_k)^-1 mod p_k
      for (int m = 0; m < K; ++m)
        if (m != k) h = h_mulmod(h, q[C.n_q + m] % pk, pk);
      const u64 phinv = h_invmod(h, pk);
      const u64 halfp = h_mulmod((P_mod(pk) + pk - 1) % pk, h_invmod(2, pk), pk);  // floor(P/2) mod p_k
      M.p[k] = pk;
      M.c[k] = h_mulmod(halfp, phinv, pk);
      M.f[k] = h_invmod(pk % ql, ql);
      M.fs[k] = h_shoup(M.f[k], ql);
    }
    const u64 halfq = h_mulmod((P_mod(ql) + ql - 1) % ql, h_invmod(2, ql), ql);  // floor(P/2) mod q_l
    M.off = (ql - h_mulmod(halfq, pinv, ql)) % ql;
    M.pinv = pinv;
    M.pinv_sh = h_shoup(pinv, ql);
    HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  }
  auto& ref = *L;
  C.lc[l] = std::move(L);
  return ref;
}

// ------------------------------------------------------------------ key switching
// Hybrid key switching (Han-Ki 2020) of a batch of polynomials with the key for
// `galois`: iNTT, ModUp of every digit to Q_l u P, NTT, inner product with the
// key digits (each key word read once for the batch), iNTT of the P limbs,
// ModDown (rounded division by P), NTT.  The ModUp is fused into the transforms:
// the inverse NTT reads d out of place and ends with N^-1 qhat_i^-1, the forward
// NTT of each extended limb loads the basis conversion directly, and a digit's
// own limbs (whose NTT is d itself) are neither converted nor transformed.
// ModUp of a batch of NTT-domain polynomials d (member stride d_stride) into NTT-domain extended
// digits [B][dn][ext][N] (a digit's own limbs are left out: they are d itself)
static DevBuf ks_modup(Ctx& C, const u64* d, size_t d_stride, int batch, int l, const KskFuse* fuse = nullptr) {
  const size_t N = C.N, nl = (size_t)l + 1;
  const int ext = l + 1 + C.n_p, dn = C.dnum(l);
  const LevelConsts& LC = level_consts(C, l);
  DevBuf dc((size_t)batch * nl * N, C.stream);  // z_i = [x_i qhat_i^-1]_{q_i}, coefficient domain
  NttAux inv{};
  inv.src = d;
  inv.src_stride = d_stride;
  inv.post = LC.intt_post.p;
  ntt_inverse(C.tab, qset(dc.p, nl * N, batch, 0, l + 1), C.stream, &inv);
  DevBuf y((size_t)batch * dn * ext * N, C.stream);
  NttAux up{};
  up.own_alpha = C.alpha;
  up.own_dn = dn;
  up.own_limit = l + 1;
  up.z = dc.p;
  up.z_stride = nl * N;
  up.bconv = LC.modup_ks.p + 2 * nl;  // factors divided by the key's folded ones
  up.bconv_sh_offset = (size_t)dn * C.alpha * ext;
  up.ext = ext;
  up.z_products = LC.modup_products * batch * (double)N;
  ntt_forward(C.tab, LimbSet{y.p, (size_t)ext * N, batch * dn, 0, ext, l + 1, 0, C.n_q}, C.stream, &up, fuse);
  return y;
}
static const DevBuf& key_for(Ctx& C, u64 galois) {
  auto it = C.keys.find(galois);
  if (it == C.keys.end()) {
    gen_galois_key(C, galois);
    it = C.keys.find(galois);
  }
  return it->second;
}
// iNTT of the P limbs of the key-switch sums acc [batch][2][ext][N], ModDown, NTT, written to / added
// into out
static void ks_moddown(Ctx& C, const DevBuf& acc, int batch, int l, u64* out, size_t out_stride, bool acc0,
                       bool acc1) {
  const size_t N = C.N, nl = (size_t)l + 1;
  const int K = C.n_p, ext = l + 1 + K;
  // ModDown: the special-prime limbs to the coefficient domain (ending with N^-1 phinv_k when the
  // conversion is fused), the conversion into every Q prime fused into the forward NTT's load, and
  // (acc - v) P^-1 (+ out) fused into its store
  const bool fuse = K <= 8;
  NttAux inv{};
  if (fuse) inv.post = C.d_moddown2.p;
  ntt_inverse(C.tab, LimbSet{acc.p, (size_t)ext * N, 2 * batch, l + 1, K, l + 1, 0, C.n_q}, C.stream, &inv);
  DevBuf v((size_t)batch * 2 * nl * N, C.stream);
  if (!fuse) k_moddown_spread(C, acc.p, v.p, 2 * batch, l);
  const u64* Pinv = C.d_moddown.p + 3 * K + (size_t)K * C.n_q;
  NttAux fw{};
  if (fuse) {
    fw.pconv = acc.p + nl * N;
    fw.pconv_stride = (size_t)ext * N;
    fw.pconv_K = K;
    fw.pconv_ld = C.n_q;
    fw.pconv_q = C.d_moddown2.p + 3 * K + (size_t)K * C.n_q;
    fw.pconv_c = C.d_moddown2.p + 2 * K;
    fw.pconv_phat = C.d_moddown.p + 3 * K;
    fw.pconv_phat_sh = C.d_moddown2.p + 3 * K;
    fw.pconv_half = C.d_moddown.p + 3 * K + (size_t)K * C.n_q + 2 * (size_t)C.n_q;
  }
  fw.fin_dst = out;
  fw.fin_dst_stride = out_stride;
  fw.fin_c = acc.p;
  fw.fin_c_stride = (size_t)ext * N;
  fw.fin_w = Pinv;
  fw.fin_wsh = Pinv + C.n_q;
  fw.fin_acc_even = acc0 ? 1 : 0;
  fw.fin_acc_odd = acc1 ? 1 : 0;
  ntt_forward(C.tab, qset(v.p, nl * N, 2 * batch, 0, l + 1), C.stream, &fw);
}

// inner product of the transformed extended digits y (permuted by X -> X^perm when perm != 0) with
// the key for `galois`, then ModDown into out
static void ks_finish(Ctx& C, const DevBuf& y, const u64* d, size_t d_stride, int batch, int l, u64 galois, u64 perm,
                      u64* out, size_t out_stride, bool acc0, bool acc1) {
  const DevBuf& key = key_for(C, galois);
  DevBuf acc((size_t)batch * 2 * (l + 1 + C.n_p) * C.N, C.stream);
  k_ksk_inner(C, y.p, d, d_stride, key.p, acc.p, batch, l, perm);
  ks_moddown(C, acc, batch, l, out, out_stride, acc0, acc1);
}

// The key switch up to the inner product: iNTT of d, the extended digits' forward transform with the
// key inner product fused into its second phase (the transformed digits are never stored).  Returns the
// sums acc [batch][2][ext][N] (NTT domain).
static DevBuf ks_inner(Ctx& C, const u64* d, size_t d_stride, int batch, int l, u64 galois) {
  const DevBuf& key = key_for(C, galois);
  const int T = C.total_primes();
  DevBuf acc((size_t)batch * 2 * (l + 1 + C.n_p) * C.N, C.stream);
  KskFuse F;
  F.d = d;
  F.d_stride = d_stride;
  F.key = key.p;
  F.key_digit_stride = (size_t)2 * T * C.N;
  F.key_a_offset = (size_t)T * C.N;
  F.acc = acc.p;
  F.acc_part_stride = (size_t)(l + 1 + C.n_p) * C.N;
  F.r64 = C.d_r64.p;
  F.batch = batch;
  ks_modup(C, d, d_stride, batch, l, &F);  // its column-phase buffer is released stream-ordered
  return acc;
}

// One key switch: the inner product, then ModDown.
void key_switch(Ctx& C, const u64* d, size_t d_stride, int batch, int l, u64 galois, u64* out, size_t out_stride,
                bool acc0, bool acc1) {
  DevBuf acc = ks_inner(C, d, d_stride, batch, l, galois);
  ks_moddown(C, acc, batch, l, out, out_stride, acc0, acc1);
}

// ModDown of the key-switch sums acc added to e (NTT domain, level l, part stride e_stride), followed
// by the rescale by q_l, written to out (level l - 1).  Separately, ModDown transforms its conversion
// v back over the l + 1 limbs and the rescale transforms the spread w of the centred last limb over
// the l remaining ones; the transforms are linear, so
//   ((e + (acc - NTT(v)) P^-1) - NTT(w)) q_l^-1 = acc (P q_l)^-1 + (e - NTT(v P^-1 + w)) q_l^-1
// and one forward transform of v P^-1 + w over l limbs does both (v P^-1 is the conversion with
// constants scaled by P^-1).  The last limb's coefficients come first: INTT(e_l + acc_l P^-1) minus
// the conversion of the special limbs into q_l scaled by P^-1.  Every residue equals that of ModDown
// followed by the rescale.
static void ks_moddown_rescale(Ctx& C, const DevBuf& acc, int batch, int l, const u64* e, size_t e_stride, u64* out,
                               size_t out_stride, bool negate = false) {
  const size_t N = C.N;
  const int K = C.n_p, ext = l + 1 + K, nq = C.n_q;
  const LevelConsts& LC = level_consts(C, l);
  NttAux inv{};
  inv.post = C.d_moddown2.p;  // the special limbs end with N^-1 phinv_k
  ntt_inverse(C.tab, LimbSet{acc.p, (size_t)ext * N, 2 * batch, l + 1, K, l + 1, 0, C.n_q}, C.stream, &inv);
  DevBuf t((size_t)2 * batch * N, C.stream), x((size_t)2 * batch * N, C.stream);
  k_mdr_last_eval(C, e + (size_t)l * N, e_stride, acc.p + (size_t)l * N, (size_t)ext * N, t.p, 2 * batch, l,
                  LC.mdr_last);
  ntt_inverse(C.tab, qset(t.p, N, 2 * batch, 0, 1, l), C.stream);
  k_mdr_last_coef(C, t.p, acc.p + (size_t)(l + 1) * N, (size_t)ext * N, x.p, 2 * batch, l, LC.mdr_last);
  DevBuf v((size_t)2 * batch * l * N, C.stream);
  NttAux fw{};
  fw.pconv = acc.p + (size_t)(l + 1) * N;
  fw.pconv_stride = (size_t)ext * N;
  fw.pconv_K = K;
  fw.pconv_ld = nq;
  fw.pconv_q = C.d_moddown2.p + 3 * K + (size_t)K * nq;
  fw.pconv_c = C.d_moddown2.p + 2 * K;
  fw.pconv_phat = C.d_mdr.p;
  fw.pconv_phat_sh = C.d_mdr.p + (size_t)K * nq;
  fw.pconv_half = C.d_mdr.p + 2 * (size_t)K * nq;
  fw.spread = x.p;
  fw.spread_stride = N;
  fw.spread_sub = LC.d_rescale.p;
  fw.spread_prime = l;
  fw.fin_dst = out;
  fw.fin_dst_stride = out_stride;
  fw.fin_c = acc.p;
  fw.fin_c_stride = (size_t)ext * N;
  fw.fin_w = LC.d_mdr.p;
  fw.fin_wsh = LC.d_mdr.p + l;
  fw.fin_e = e;
  fw.fin_e_stride = e_stride;
  fw.fin_w2 = LC.d_rescale.p + l;
  fw.fin_w2sh = LC.d_rescale.p + 2 * l;
  fw.fin_neg = negate ? 1 : 0;
  ntt_forward(C.tab, qset(v.p, (size_t)l * N, 2 * batch, 0, l), C.stream, &fw);
}

// Rotations of one (batched) ciphertext by several Galois elements sharing one ModUp of its
// second part (hoisting): the extended digits of c1 are formed once, and each rotation applies its
// automorphism to them inside the inner product.  The result differs from ev_galois (which
// converts the rotated c1) by multiples of the digit moduli in the extended basis, within the
// same noise bound.
std::vector<std::unique_ptr<Ct>> ev_galois_hoisted(Ctx& C, const Ct& a, const std::vector<u64>& gs) {
  const int l = a.level;
  for (u64 g : gs) key_for(C, g);
  const u64* d = a.part(1);
  const size_t ds = 2 * a.part_stride();
  DevBuf y = ks_modup(C, d, ds, a.batch, l);
  std::vector<std::unique_ptr<Ct>> out;
  for (u64 g : gs) {
    auto o = ct_alloc(C, l, a.batch);
    o->scale = a.scale;
    k_automorph(C, a.part(0), 2 * a.part_stride(), o->part(0), 2 * o->part_stride(), a.batch, l + 1, g);
    ks_finish(C, y, d, ds, a.batch, l, g, g, o->part(0), o->part_stride(), true, false);
    out.push_back(std::move(o));
  }
  return out;
}

std::vector<DevBuf> ev_galois_hoisted_qp(Ctx& C, const Ct& a, const std::vector<u64>& gs) {
  const int l = a.level;
  for (u64 g : gs) key_for(C, g);
  const u64* d = a.part(1);
  const size_t ds = 2 * a.part_stride();
  DevBuf y = ks_modup(C, d, ds, a.batch, l);
  std::vector<DevBuf> out;
  for (u64 g : gs) {
    DevBuf acc((size_t)a.batch * 2 * (l + 1 + C.n_p) * C.N, C.stream);
    k_ksk_inner(C, y.p, d, ds, key_for(C, g).p, acc.p, a.batch, l, g, a.part(0), ds);
    out.push_back(std::move(acc));
  }
  return out;
}
void ev_moddown_into(Ctx& C, DevBuf& acc, int batch, int level, Ct& out) {
  ks_moddown(C, acc, batch, level, out.part(0), out.part_stride(), false, false);
}

std::unique_ptr<Ct> ev_mul_relin(Ctx& C, const Ct& a, const Ct& b) {
  const int l = std::min(a.level, b.level);
  check_batches(a, b);
  auto o = ct_alloc(C, l, a.batch);
  o->scale = a.scale * b.scale;
  const size_t per = (size_t)(l + 1) * C.N;
  DevBuf d2(a.batch * per, C.stream);
  k_tensor(C, a.part(0), a.part_stride(), b.part(0), b.part_stride(), o->part(0), o->part_stride(), d2.p, a.batch,
           l + 1);
  key_switch(C, d2.p, per, a.batch, l, 0, o->part(0), o->part_stride(), true, true);
  return o;
}

// rescale by q_l: c_i <- (c_i - [c_l]_centred) * q_l^-1 mod q_i, i < l
std::unique_ptr<Ct> ev_rescale(Ctx& C, const Ct& a) {
  const int l = a.level;
  if (l < 1) throw Error(HEDAP_ERR_LEVEL, "rescale needs level >= 1");
  const size_t N = C.N;
  const int P = a.parts();
  const LevelConsts& LC = level_consts(C, l);
  auto o = ct_alloc(C, l - 1, a.batch);
  o->scale = a.scale / (double)C.primes[l];
  // the last limb to the coefficient domain (read in place), then one forward transform whose
  // load spreads its centred residue into every other prime and whose store finishes the rescale
  DevBuf last(P * N, C.stream);
  NttAux inv{};
  inv.src = a.part(0) + (size_t)l * N;
  inv.src_stride = a.part_stride();
  ntt_inverse(C.tab, qset(last.p, N, P, 0, 1, l), C.stream, &inv);
  DevBuf tmp((size_t)P * l * N, C.stream);
  NttAux fw{};
  fw.spread = last.p;
  fw.spread_stride = N;
  fw.spread_sub = LC.d_rescale.p;
  fw.spread_prime = l;
  fw.fin_dst = o->part(0);
  fw.fin_dst_stride = o->part_stride();
  fw.fin_c = a.part(0);
  fw.fin_c_stride = a.part_stride();
  fw.fin_w = LC.d_rescale.p + l;
  fw.fin_wsh = LC.d_rescale.p + 2 * l;
  ntt_forward(C.tab, qset(tmp.p, (size_t)l * N, P, 0, l), C.stream, &fw);
  return o;
}

// A relinearised product entering a linear combination that is rescaled next, as one fused
// operation: rescale(m (d01 + ModDown(acc)) + sum_j c_j t_j + c0), m the product's integer constant.
// With m = 1 the sum e = d01 + sum_j c_j t_j + c0 is formed first (one linear-combination pass) and
// ks_moddown_rescale finishes e + ModDown(acc).  With m = -1 every other constant is negated instead
// (std::round is odd, so each integer constant is exactly negated), giving -(the sum), and the fused
// rescale stores the negated residues: the centred residue is odd for an odd q_l, so rescale(-x) =
// -rescale(x) residue for residue.  Any other m, or a chain too wide for one linear-combination pass,
// takes the unfused sequence.
std::unique_ptr<Ct> ev_mul_lincomb_rescale(Ctx& C, const Ct& a, const Ct& b, double prod_scale, double prod_coef,
                                           const std::vector<std::pair<const Ct*, double>>& terms, double target,
                                           double c0) {
  const int l = std::min(a.level, b.level);
  check_batches(a, b);
  const double m = l >= 1 ? std::round(prod_coef * target * (double)C.primes[l] / prod_scale) : 0.0;
  if (l < 1 || (m != 1.0 && m != -1.0) || l + 1 > kLcLimbs || C.n_p > 8 || terms.size() + 1 > kLcTerms) {
    auto pr = ev_mul_relin(C, a, b);
    pr->scale = prod_scale;
    std::vector<std::pair<const Ct*, double>> all{{pr.get(), prod_coef}};
    all.insert(all.end(), terms.begin(), terms.end());
    return ev_rescale(C, *ev_lincomb_raw(C, all, l, target, c0));
  }
  auto d01 = ct_alloc(C, l, a.batch);
  d01->scale = prod_scale;
  const size_t per = (size_t)(l + 1) * C.N;
  DevBuf d2(a.batch * per, C.stream);
  k_tensor(C, a.part(0), a.part_stride(), b.part(0), b.part_stride(), d01->part(0), d01->part_stride(), d2.p,
           a.batch, l + 1);
  DevBuf acc = ks_inner(C, d2.p, per, a.batch, l, 0);
  std::vector<std::pair<const Ct*, double>> all{{d01.get(), m * prod_coef}};
  for (const auto& t : terms) all.emplace_back(t.first, m * t.second);
  auto e = ev_lincomb_raw(C, all, l, target, m * c0);
  auto o = ct_alloc(C, l - 1, a.batch);
  o->scale = e->scale / (double)C.primes[l];
  ks_moddown_rescale(C, acc, a.batch, l, e->part(0), e->part_stride(), o->part(0), o->part_stride(), m < 0);
  return o;
}

// HMult and rescale: the tensor product, the relinearising key switch up to its inner product, then
// ModDown and the rescale in one transform (ks_moddown_rescale); equal, residue for residue, to
// ev_rescale(ev_mul_relin(a, b)).
std::unique_ptr<Ct> ev_mul(Ctx& C, const Ct& a, const Ct& b) {
  const int l = std::min(a.level, b.level);
  if (l < 1) throw Error(HEDAP_ERR_LEVEL, "rescale needs level >= 1");
  if (C.n_p > 8) return ev_rescale(C, *ev_mul_relin(C, a, b));
  check_batches(a, b);
  auto e = ct_alloc(C, l, a.batch);
  const size_t per = (size_t)(l + 1) * C.N;
  DevBuf d2(a.batch * per, C.stream);
  k_tensor(C, a.part(0), a.part_stride(), b.part(0), b.part_stride(), e->part(0), e->part_stride(), d2.p, a.batch,
           l + 1);
  DevBuf acc = ks_inner(C, d2.p, per, a.batch, l, 0);
  auto o = ct_alloc(C, l - 1, a.batch);
  o->scale = a.scale * b.scale / (double)C.primes[l];
  ks_moddown_rescale(C, acc, a.batch, l, e->part(0), e->part_stride(), o->part(0), o->part_stride());
  return o;
}

u64 galois_for_rotation(const Ctx& C, i64 steps) {
  const i64 h = (i64)(C.N / 2);
  const i64 r = ((steps % h) + h) % h;
  return h_powmod(5, (u64)r, 2 * C.N);
}

std::unique_ptr<Ct> ev_galois(Ctx& C, const Ct& a, u64 g) {
  const int l = a.level;
  auto o = ct_alloc(C, l, a.batch);
  o->scale = a.scale;
  k_automorph(C, a.part(0), a.part_stride(), o->part(0), o->part_stride(), a.parts(), l + 1, g);
  key_switch(C, o->part(1), 2 * o->part_stride(), a.batch, l, g, o->part(0), o->part_stride(), true, false);
  return o;
}

// key switch of (c0, c1) with the key `id` (from the secret c1 multiplies to the key's target)
std::unique_ptr<Ct> ev_switch_key(Ctx& C, const Ct& a, u64 id) {
  if (!C.keys.count(id)) throw Error(HEDAP_ERR_ARG, "switching key not generated");
  const int l = a.level;
  auto o = ct_copy(C, a, l);
  key_switch(C, o->part(1), 2 * o->part_stride(), a.batch, l, id, o->part(0), o->part_stride(), true, false);
  return o;
}

// Mul_P by a real constant c at plaintext scale target * q_l / scale, then rescale;
// the result's scale is set to exactly `target`.
// Mul_P by c without the rescale: the product is labelled target * q_l (several such products at one
// level with one target add exactly and share one rescale)
std::unique_ptr<Ct> ev_mul_const_raw(Ctx& C, const Ct& a, double c, double target) {
  const int l = a.level;
  if (l < 1) throw Error(HEDAP_ERR_LEVEL, "constant multiplication needs level >= 1");
  const double sp = target * (double)C.primes[l] / a.scale;
  const double v = std::round(c * sp);
  LimbConsts K;
  for (int i = 0; i <= l; ++i) {
    K.w[i] = h_double_to_mod(v, C.primes[i]);
    K.wsh[i] = h_shoup(K.w[i], C.primes[i]);
  }
  auto t = ct_alloc(C, l, a.batch);
  t->scale = target * (double)C.primes[l];
  k_mul_limbconst(C, a.part(0), a.part_stride(), t->part(0), t->part_stride(), a.parts(), l + 1, K);
  return t;
}
std::unique_ptr<Ct> ev_lincomb_raw(Ctx& C, const std::vector<std::pair<const Ct*, double>>& terms, int level,
                                   double target, double c0) {
  if (terms.empty()) throw Error(HEDAP_ERR_ARG, "linear combination without terms");
  if (level < 1) throw Error(HEDAP_ERR_LEVEL, "constant multiplication needs level >= 1");
  const double raw = target * (double)C.primes[level];
  const int batch = terms[0].first->batch;
  for (const auto& t : terms) {
    if (t.first->level < level) throw Error(HEDAP_ERR_LEVEL, "linear combination operand below the output level");
    if (t.first->batch != batch) throw Error(HEDAP_ERR_ARG, "operands have different batch sizes");
  }
  auto o = ct_alloc(C, level, batch);
  o->scale = raw;
  if (level + 1 > kLcLimbs) {  // wide chains: one product and one addition at a time
    std::unique_ptr<Ct> acc;
    for (const auto& t : terms) {
      std::unique_ptr<Ct> d = t.first->level == level ? nullptr : ev_drop(C, *t.first, level);
      auto term = ev_mul_const_raw(C, d ? *d : *t.first, t.second, target);
      acc = acc ? ev_add(C, *acc, *term, false) : std::move(term);
    }
    acc->scale = raw;
    return ev_add_const(C, *acc, c0);
  }
  for (size_t first = 0; first < terms.size(); first += kLcTerms) {
    LinCombArgs A{};
    A.count = (int)std::min<size_t>(kLcTerms, terms.size() - first);
    A.accumulate = first > 0;
    A.add_c0 = first == 0;
    for (int j = 0; j < A.count; ++j) {
      const Ct& a = *terms[first + j].first;
      A.in[j] = a.part(0);
      A.stride[j] = a.part_stride();
      const double sp = target * (double)C.primes[level] / a.scale;  // as in ev_mul_const_raw
      const double v = std::round(terms[first + j].second * sp);
      for (int i = 0; i <= level; ++i) {
        A.w[j][i] = h_double_to_mod(v, C.primes[i]);
        A.wsh[j][i] = h_shoup(A.w[j][i], C.primes[i]);
      }
    }
    if (A.add_c0) {
      const double v0 = std::round(c0 * raw);  // as in ev_add_const on the sum
      for (int i = 0; i <= level; ++i) A.c0[i] = h_double_to_mod(v0, C.primes[i]);
    }
    k_lincomb(C, o->part(0), o->part_stride(), o->parts(), level + 1, A);
  }
  return o;
}

std::unique_ptr<Ct> ev_mul_const(Ctx& C, const Ct& a, double c, double target) {
  auto o = ev_rescale(C, *ev_mul_const_raw(C, a, c, target));
  o->scale = target;
  return o;
}

std::unique_ptr<Ct> ev_add_const(Ctx& C, const Ct& a, double c) {
  const double v = std::round(c * a.scale);
  LimbConsts K;
  for (int i = 0; i <= a.level; ++i) K.w[i] = h_double_to_mod(v, C.primes[i]);
  auto o = ct_copy(C, a, a.level);
  k_add_limbconst(C, o->part(0), 2 * o->part_stride(), a.batch, a.level + 1, K);
  return o;
}

// (a + c) * m in one pass: the constant c is added at a's scale exactly as ev_add_const adds it,
// then everything is multiplied by the integer m (same residues as the two operations in turn)
std::unique_ptr<Ct> ev_add_const_mul_int(Ctx& C, const Ct& a, double c, i64 m) {
  if (a.level + 1 > kLcLimbs) return ev_mul_int(C, *ev_add_const(C, a, c), m);
  const double v = std::round(c * a.scale);
  LinCombArgs A{};
  A.count = 1;
  A.add_c0 = 1;
  A.in[0] = a.part(0);
  A.stride[0] = a.part_stride();
  for (int i = 0; i <= a.level; ++i) {
    const u64 q = C.primes[i], mm = h_smod(m, q);
    A.w[0][i] = mm;
    A.wsh[0][i] = h_shoup(mm, q);
    A.c0[i] = h_mulmod(h_double_to_mod(v, q), mm, q);
  }
  auto o = ct_alloc(C, a.level, a.batch);
  o->scale = a.scale;
  k_lincomb(C, o->part(0), o->part_stride(), o->parts(), a.level + 1, A);
  return o;
}

std::unique_ptr<Ct> ev_mul_int(Ctx& C, const Ct& a, i64 m) {
  LimbConsts K;
  for (int i = 0; i <= a.level; ++i) {
    K.w[i] = h_smod(m, C.primes[i]);
    K.wsh[i] = h_shoup(K.w[i], C.primes[i]);
  }
  auto o = ct_alloc(C, a.level, a.batch);
  o->scale = a.scale;
  k_mul_limbconst(C, a.part(0), a.part_stride(), o->part(0), o->part_stride(), a.parts(), a.level + 1, K);
  return o;
}

}  // namespace hedap
