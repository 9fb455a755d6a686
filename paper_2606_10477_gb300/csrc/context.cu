// Context creation (prime chain, NTT tables, RNS constants), key generation,
// encoding (CKKS canonical embedding over the 5^j orbit, FP64 on the host),
// encryption and decryption.
#include <cmath>
#include <complex>

#include "internal.cuh"
#include "kernels.cuh"

namespace hedap {

typedef unsigned __int128 u128;
typedef std::complex<double> cplx;

static void upload(Ctx& C, DevBuf& dst, const std::vector<u64>& src) {
  dst = DevBuf(src.size(), C.stream);
  HEDAP_CUDA(cudaMemcpyAsync(dst.p, src.data(), src.size() * 8, cudaMemcpyHostToDevice, C.stream));
  HEDAP_CUDA(cudaStreamSynchronize(C.stream));
}

static LimbSet q_limbs(u64* base, size_t part_stride, int n_parts, int first, int count) {
  return LimbSet{base, part_stride, n_parts, first, count, INT_MAX, 0, 0};
}

Ctx* ctx_create(const hedap_params& P, u64 seed, cudaStream_t st) {
  if (P.log_n < 10 || P.log_n > 17) throw Error(HEDAP_ERR_ARG, "log_n must lie in [10, 17]");
  if (P.n_q < 1 || P.n_q > (uint32_t)kMaxLimbs || !P.q_bits) throw Error(HEDAP_ERR_ARG, "n_q must lie in [1, 64]");
  if (P.n_p < 1 || P.n_p > 8 || !P.p_bits) throw Error(HEDAP_ERR_ARG, "n_p must lie in [1, 8]");
  if (P.alpha < 1 || P.alpha > 8) throw Error(HEDAP_ERR_ARG, "alpha must lie in [1, 8]");
  if (!(P.log_scale > 0 && P.log_scale < 62)) throw Error(HEDAP_ERR_ARG, "log_scale out of range");
  if (P.secret_hw > (1u << P.log_n)) throw Error(HEDAP_ERR_ARG, "secret_hw exceeds N");
  std::unique_ptr<Ctx> C(new Ctx);
  C->log_n = (int)P.log_n;
  C->N = (size_t)1 << P.log_n;
  C->n_q = (int)P.n_q;
  C->n_p = (int)P.n_p;
  C->alpha = (int)P.alpha;
  C->hw = (int)P.secret_hw;
  C->scale = std::pow(2.0, P.log_scale);
  C->seed = seed;
  C->stream = st;
  C->home = st;

  int dev = 0;
  HEDAP_CUDA(cudaGetDevice(&dev));
  C->device = dev;
  // hedap_rescale_noalloc's scratch: resolved here, so that its module is loaded (and the array
  // allocated) now rather than inside a call that promises not to allocate
  C->noalloc_scratch = noalloc_scratch_address(dev);
  cudaMemPool_t pool;
  HEDAP_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = UINT64_MAX;
  HEDAP_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));

  std::vector<int> bits;
  for (uint32_t i = 0; i < P.n_q; ++i) bits.push_back((int)P.q_bits[i]);
  for (uint32_t i = 0; i < P.n_p; ++i) bits.push_back((int)P.p_bits[i]);
  C->primes = h_prime_chain(C->log_n, bits);
  const int T = C->total_primes();
  const size_t N = C->N;

  // NTT tables: psi^bitrev(i), psi^-bitrev(i) and Shoup companions
  std::vector<u64> psi2(2 * T * N), ipsi2(2 * T * N), ninv(T), ninv_sh(T), r64(2 * T);
  std::vector<u64> pw(N), ipw(N);
  for (int t = 0; t < T; ++t) {
    const u64 q = C->primes[t];
    C->pdev.push_back(h_prime_dev(q));
    const u64 w = h_find_psi(q, C->log_n), wi = h_invmod(w, q);
    pw[0] = ipw[0] = 1;
    for (size_t k = 1; k < N; ++k) {
      pw[k] = h_mulmod(pw[k - 1], w, q);
      ipw[k] = h_mulmod(ipw[k - 1], wi, q);
    }
    for (size_t i = 0; i < N; ++i) {
      const uint32_t r = h_bitrev((uint32_t)i, C->log_n);
      psi2[2 * (t * N + i)] = pw[r];
      psi2[2 * (t * N + i) + 1] = h_shoup(pw[r], q);
      ipsi2[2 * (t * N + i)] = ipw[r];
      ipsi2[2 * (t * N + i) + 1] = h_shoup(ipw[r], q);
    }
    ninv[t] = h_invmod(N % q, q);
    ninv_sh[t] = h_shoup(ninv[t], q);
    r64[2 * t] = (u64)(((u128)1 << 64) % q);
    r64[2 * t + 1] = h_shoup(r64[2 * t], q);
  }
  {
    std::vector<u64> pd(T * sizeof(PrimeDev) / 8);
    memcpy(pd.data(), C->pdev.data(), T * sizeof(PrimeDev));
    upload(*C, C->d_primes, pd);
  }
  upload(*C, C->d_psi2, psi2);
  upload(*C, C->d_ipsi2, ipsi2);
  upload(*C, C->d_ninv, ninv);
  upload(*C, C->d_ninv_sh, ninv_sh);
  upload(*C, C->d_r64, r64);
  C->tab = Tables{(const PrimeDev*)C->d_primes.p, (const ulonglong2*)C->d_psi2.p, (const ulonglong2*)C->d_ipsi2.p,
                  C->d_ninv.p, C->d_ninv_sh.p, C->log_n, 3, 3, 3, 3};

  // P = prod p_k; ModDown constants and P mod q_t
  const int K = C->n_p, nq = C->n_q;
  auto p_of = [&](int k) { return C->primes[nq + k]; };
  auto P_mod = [&](u64 m) {
    u64 r = 1 % m;
    for (int k = 0; k < K; ++k) r = h_mulmod(r, p_of(k) % m, m);
    return r;
  };
  auto halfP_mod = [&](u64 m) {  // (P - 1) / 2 mod m
    u64 pm = P_mod(m);
    return h_mulmod((pm + m - 1) % m, h_invmod(2, m), m);
  };
  std::vector<u64> md;
  for (int k = 0; k < K; ++k) md.push_back(halfP_mod(p_of(k)));
  std::vector<u64> phinv(K);
  for (int k = 0; k < K; ++k) {
    u64 h = 1;
    for (int m = 0; m < K; ++m)
      if (m != k) h = h_mulmod(h, p_of(m) % p_of(k), p_of(k));
    phinv[k] = h_invmod(h, p_of(k));
  }
  for (int k = 0; k < K; ++k) md.push_back(phinv[k]);
  for (int k = 0; k < K; ++k) md.push_back(h_shoup(phinv[k], p_of(k)));
  for (int k = 0; k < K; ++k)
    for (int i = 0; i < nq; ++i) {
      const u64 qi = C->primes[i];
      u64 h = 1;
      for (int m = 0; m < K; ++m)
        if (m != k) h = h_mulmod(h, p_of(m) % qi, qi);
      md.push_back(h);
    }
  std::vector<u64> pinv(nq), pinv_sh(nq), halfq(nq);
  for (int i = 0; i < nq; ++i) {
    const u64 qi = C->primes[i];
    pinv[i] = h_invmod(P_mod(qi), qi);
    pinv_sh[i] = h_shoup(pinv[i], qi);
    halfq[i] = halfP_mod(qi);
  }
  md.insert(md.end(), pinv.begin(), pinv.end());
  md.insert(md.end(), pinv_sh.begin(), pinv_sh.end());
  md.insert(md.end(), halfq.begin(), halfq.end());
  // fused ModDown: the special-prime iNTT ends with N^-1 phinv_k, the conversion adds
  // c_k = floor(P/2) phinv_k and multiplies by phat_q with Shoup companions
  std::vector<u64> md2;
  for (int k = 0; k < K; ++k) {
    const u64 pk = p_of(k), w = h_mulmod(h_invmod(N % pk, pk), phinv[k], pk);
    md2.push_back(w);
    md2.push_back(h_shoup(w, pk));
  }
  for (int k = 0; k < K; ++k) md2.push_back(h_mulmod(halfP_mod(p_of(k)), phinv[k], p_of(k)));
  for (int k = 0; k < K; ++k)
    for (int i = 0; i < nq; ++i) md2.push_back(h_shoup(md[3 * K + (size_t)k * nq + i], C->primes[i]));
  for (int k = 0; k < K; ++k) md2.push_back(p_of(k));
  upload(*C, C->d_moddown, md);
  upload(*C, C->d_moddown2, md2);
  // ModDown fused with a rescale: the conversion scaled by P^-1, i.e. phat_k P^-1 = p_k^-1 mod q_i and
  // floor(P/2) P^-1 mod q_i
  std::vector<u64> mdr((size_t)2 * K * nq + nq);
  for (int k = 0; k < K; ++k)
    for (int i = 0; i < nq; ++i) {
      const u64 qi = C->primes[i], f = h_invmod(p_of(k) % qi, qi);
      mdr[(size_t)k * nq + i] = f;
      mdr[(size_t)(K + k) * nq + i] = h_shoup(f, qi);
    }
  for (int i = 0; i < nq; ++i) mdr[(size_t)2 * K * nq + i] = h_mulmod(halfq[i], pinv[i], C->primes[i]);
  upload(*C, C->d_mdr, mdr);

  std::vector<u64> pm(T);
  for (int t = 0; t < T; ++t) pm[t] = P_mod(C->primes[t]);
  upload(*C, C->d_pmod, pm);

  // the factors folded into the switching keys (see Ctx::key_scale): for digit j and a limb t outside
  // it, the digit's smallest prime q_i0 is added to the ModUp sum unmultiplied when the sum still meets
  // the transform's input bound (q_i0 + 2 (a - 1) p_t below 8 p_t for digits of a <= 3 primes, whose
  // load reduces once, below 16 p_t otherwise); the key then carries qhat_i0 = prod_{m != i0} q_m mod p_t
  {
    const int dnL = C->dnum(C->L());
    C->key_scale.assign((size_t)dnL * T, 1);
    C->key_unscale.assign((size_t)dnL * T, 1);
    C->key_scale_i0.assign((size_t)dnL * T, -1);
    const unsigned __int128 bound = C->alpha <= 3 ? 8 : 16;
    for (int j = 0; j < dnL; ++j) {
      const int lo = j * C->alpha, hi = std::min(lo + C->alpha, nq);
      int i0 = lo;
      for (int i = lo; i < hi; ++i)
        if (C->primes[i] < C->primes[i0]) i0 = i;
      for (int t = 0; t < T; ++t) {
        if (t >= lo && t < hi) continue;
        const u64 pt = C->primes[t];
        if ((unsigned __int128)C->primes[i0] + (unsigned __int128)2 * (hi - lo - 1) * pt >= bound * pt) continue;
        u64 h = 1 % pt;
        for (int m = lo; m < hi; ++m)
          if (m != i0) h = h_mulmod(h, C->primes[m] % pt, pt);
        C->key_scale[(size_t)j * T + t] = h;
        C->key_unscale[(size_t)j * T + t] = h_invmod(h, pt);
        C->key_scale_i0[(size_t)j * T + t] = i0;
      }
    }
    std::vector<u64> ks((size_t)2 * dnL * T);
    for (size_t e = 0; e < (size_t)dnL * T; ++e) {
      ks[2 * e] = C->key_scale[e];
      ks[2 * e + 1] = h_shoup(C->key_scale[e], C->primes[e % T]);
    }
    upload(*C, C->d_key_scale, ks);
  }

  // secret key: ternary coefficients, NTT domain over every prime
  SplitMix ss(seed, tags::sk);
  C->sk = draw_ternary(ss, C->log_n, C->hw);
  std::vector<u64> skr(T * N);
  for (int t = 0; t < T; ++t)
    for (size_t i = 0; i < N; ++i) skr[t * N + i] = h_smod(C->sk[i], C->primes[t]);
  upload(*C, C->d_sk, skr);
  ntt_forward(C->tab, LimbSet{C->d_sk.p, 0, 1, 0, T, nq, 0, nq}, C->stream);
  gen_galois_key(*C, 0);
  ntt_tune(*C, 8 * C->n_q, 2, nullptr, nullptr);  // pick the NTT launch shape for this ring
  HEDAP_CUDA(cudaStreamSynchronize(C->stream));
  return C.release();
}

// Switching key with id `g` from s' to s_to (NTT domain over all primes); digit j:
// b = e - a s_to + [t in digit j] (P mod q_t) s',  a uniform (NTT domain).
void gen_switch_key(Ctx& C, u64 g, const u64* sp, const u64* s_to) {
  const int T = C.total_primes(), nq = C.n_q, dn = C.dnum(C.L());
  const size_t N = C.N;
  DevBuf key((size_t)dn * 2 * T * N, C.stream);
  std::vector<u64> ah(T * N), eh(T * N);
  std::vector<i64> e(N);
  for (int j = 0; j < dn; ++j) {
    SplitMix sa(C.seed, tags::evk_a(g, (u64)j));
    for (int t = 0; t < T; ++t)
      for (size_t i = 0; i < N; ++i) ah[t * N + i] = draw_uniform(sa, C.primes[t]);
    SplitMix se(C.seed, tags::evk_e(g, (u64)j));
    for (size_t i = 0; i < N; ++i) e[i] = draw_cbd21(se);
    for (int t = 0; t < T; ++t)
      for (size_t i = 0; i < N; ++i) eh[t * N + i] = h_smod(e[i], C.primes[t]);
    u64* b = key.p + (size_t)j * 2 * T * N;
    u64* a = b + (size_t)T * N;
    HEDAP_CUDA(cudaMemcpyAsync(b, eh.data(), T * N * 8, cudaMemcpyHostToDevice, C.stream));
    HEDAP_CUDA(cudaMemcpyAsync(a, ah.data(), T * N * 8, cudaMemcpyHostToDevice, C.stream));
    ntt_forward(C.tab, LimbSet{b, 0, 1, 0, T, nq, 0, nq}, C.stream);
    const int lo = j * C.alpha, hi = std::min(lo + C.alpha, nq);
    k_keygen_combine(C, b, a, s_to, sp, C.d_pmod.p, lo, hi);
    const u64* f = C.d_key_scale.p + (size_t)2 * j * T;  // the folded conversion factors (Ctx::key_scale)
    k_scale_limbs(C, b, T, f);
    k_scale_limbs(C, a, T, f);
    HEDAP_CUDA(cudaStreamSynchronize(C.stream));  // host buffers are reused
  }
  C.keys[g] = std::move(key);
}

// Switching key for s' -> s with s' = s^2 (g = 0) or s(X^g)
void gen_galois_key(Ctx& C, u64 g) {
  if (C.keys.count(g)) return;
  if (g != 0 && (g % 2 == 0 || g >= 2 * C.N)) throw Error(HEDAP_ERR_ARG, "galois element must be odd and < 2N");
  const int T = C.total_primes();
  DevBuf sp(T * C.N, C.stream);
  if (g == 0) k_fma(C, nullptr, C.d_sk.p, C.d_sk.p, sp.p, T, 2);
  else k_automorph(C, C.d_sk.p, 0, sp.p, 0, 1, T, g);
  gen_switch_key(C, g, sp.p, C.d_sk.p);
}

// Sparse-secret encapsulation of bootstrapping (Bossuat, Troncoso-Pastoriza and
// Hubaux 2022): an ephemeral secret s~ with h non-zero coefficients, a key from
// s to s~ (used at level 0, before ModRaise) and one from s~ back to s (used at
// the top level, after it), so that the ModRaise overflow is that of a weight-h
// secret whatever the distribution of s.
void bts_encapsulate(Ctx& C, int h) {
  if (h < 1 || (size_t)h > C.N) throw Error(HEDAP_ERR_ARG, "encapsulation weight must lie in [1, N]");
  const int T = C.total_primes();
  const size_t N = C.N;
  SplitMix ss(C.seed, tags::sk_sparse);
  const std::vector<i64> v = draw_ternary(ss, C.log_n, h);
  std::vector<u64> r(T * N);
  for (int t = 0; t < T; ++t)
    for (size_t i = 0; i < N; ++i) r[t * N + i] = h_smod(v[i], C.primes[t]);
  DevBuf d;
  upload(C, d, r);
  ntt_forward(C.tab, LimbSet{d.p, 0, 1, 0, T, C.n_q, 0, C.n_q}, C.stream);
  C.keys.erase(kKeyToSparse);
  C.keys.erase(kKeyToDense);
  gen_switch_key(C, kKeyToSparse, C.d_sk.p, d.p);
  gen_switch_key(C, kKeyToDense, d.p, C.d_sk.p);
  HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  C.d_sk_sparse = std::move(d);
  C.enc_hw = h;
}

// ------------------------------------------------------------------ encoding
// Decoding is z_j = m(zeta^(5^j)), zeta = exp(i pi / N); with n = N/2 and
// w_k = m_k + i m_{k+n} it is z = V w, V_jk = zeta^(5^j k).  V factors into the
// radix-2 stages of a decimation-in-time transform over bit-reversed input
// whose size-len sub-transforms use the root exp(2 pi i 5^j / (4 len)).
struct SpecialFFT {
  int log_n;
  size_t n;
  std::vector<cplx> root;  // exp(2 pi i k / 2N)
  explicit SpecialFFT(int logN) : log_n(logN - 1), n((size_t)1 << (logN - 1)) {
    const size_t M = 4 * n;
    root.resize(M);
    for (size_t k = 0; k < M; ++k) root[k] = std::polar(1.0, 2.0 * M_PI * (double)k / (double)M);
  }
  void bitrev_permute(std::vector<cplx>& v) const {
    for (size_t i = 0; i < n; ++i) {
      size_t r = h_bitrev((uint32_t)i, log_n);
      if (r > i) std::swap(v[i], v[r]);
    }
  }
  void forward(std::vector<cplx>& v) const {  // w -> z
    bitrev_permute(v);
    const size_t M2 = 4 * n;
    for (size_t len = 2; len <= n; len <<= 1) {
      const size_t M = 4 * len, stride = M2 / M;
      for (size_t b = 0; b < n; b += len) {
        size_t g = 1;
        for (size_t j = 0; j < len / 2; ++j) {
          const cplx r = root[(g % M) * stride];
          const cplx u = v[b + j], t = v[b + j + len / 2] * r;
          v[b + j] = u + t;
          v[b + j + len / 2] = u - t;
          g = (g * 5) % M;
        }
      }
    }
  }
  void inverse(std::vector<cplx>& v) const {  // z -> w
    const size_t M2 = 4 * n;
    for (size_t len = n; len >= 2; len >>= 1) {
      const size_t M = 4 * len, stride = M2 / M;
      for (size_t b = 0; b < n; b += len) {
        size_t g = 1;
        for (size_t j = 0; j < len / 2; ++j) {
          const cplx r = root[(g % M) * stride];
          const cplx x = v[b + j], y = v[b + j + len / 2];
          v[b + j] = (x + y) * 0.5;
          v[b + j + len / 2] = (x - y) * 0.5 / r;
          g = (g * 5) % M;
        }
      }
    }
    bitrev_permute(v);
  }
};

std::vector<double> encode_slots(const Ctx& C, const std::vector<std::complex<double>>& z, double scale) {
  const size_t n = C.N / 2;
  if (z.size() != n) throw Error(HEDAP_ERR_ARG, "encode: n_slots must equal N/2");
  std::vector<cplx> v(z);
  SpecialFFT(C.log_n).inverse(v);
  std::vector<double> m(C.N);
  for (size_t k = 0; k < n; ++k) {
    m[k] = std::round(v[k].real() * scale);
    m[k + n] = std::round(v[k].imag() * scale);
  }
  return m;
}

static std::vector<double> encode(const Ctx& C, const std::vector<double>& re, const std::vector<double>& im,
                                  double scale) {
  std::vector<cplx> v(C.N / 2);
  for (size_t j = 0; j < v.size(); ++j) v[j] = cplx(re[j], im.empty() ? 0.0 : im[j]);
  return encode_slots(C, v, scale);
}

std::unique_ptr<Ct> encrypt(Ctx& C, const std::vector<double>& re, const std::vector<double>& im, int level,
                            u64 seed) {
  if (level < 0 || level > C.L()) throw Error(HEDAP_ERR_LEVEL, "encryption level out of range");
  if (re.size() != C.N / 2) throw Error(HEDAP_ERR_ARG, "n_slots must equal N/2");
  const size_t N = C.N;
  std::vector<double> m = encode(C, re, im, C.scale);
  auto ct = ct_alloc(C, level);
  ct->scale = C.scale;
  const int nl = level + 1;
  std::vector<u64> a(nl * N), me(nl * N);
  SplitMix sa(seed, tags::enc_a);
  for (int i = 0; i < nl; ++i)
    for (size_t k = 0; k < N; ++k) a[i * N + k] = draw_uniform(sa, C.primes[i]);
  SplitMix se(seed, tags::enc_e);
  std::vector<i64> e(N);
  for (size_t k = 0; k < N; ++k) e[k] = draw_cbd21(se);
  for (int i = 0; i < nl; ++i) {
    const u64 q = C.primes[i];
    for (size_t k = 0; k < N; ++k) {
      u64 v = h_double_to_mod(m[k], q) + h_smod(e[k], q);
      me[i * N + k] = v >= q ? v - q : v;
    }
  }
  HEDAP_CUDA(cudaMemcpyAsync(ct->part(0), me.data(), nl * N * 8, cudaMemcpyHostToDevice, C.stream));
  HEDAP_CUDA(cudaMemcpyAsync(ct->part(1), a.data(), nl * N * 8, cudaMemcpyHostToDevice, C.stream));
  ntt_forward(C.tab, q_limbs(ct->part(0), 0, 1, 0, nl), C.stream);
  k_fma(C, ct->part(0), ct->part(1), C.d_sk.p, ct->part(0), nl, 0);  // c0 = (m + e) - a s
  HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  return ct;
}

// Garner mixed-radix reconstruction of the lowest k limbs, centred, as double.
// A decrypted coefficient is far below q_0 q_1 ... q_{k-1} / 2 for k = min(l+1, 8).
void decrypt(Ctx& C, const Ct& ct, std::vector<double>& re, std::vector<double>& im) {
  const size_t N = C.N;
  if (ct.batch != 1) throw Error(HEDAP_ERR_ARG, "decrypt takes one ciphertext (unpack the batch first)");
  const int l = ct.level, k = std::min(l + 1, 8);
  DevBuf m((size_t)(l + 1) * N, C.stream);
  k_fma(C, ct.part(0), ct.part(1), C.d_sk.p, m.p, l + 1, 1);  // c0 + c1 s
  ntt_inverse(C.tab, q_limbs(m.p, 0, 1, 0, k), C.stream);
  std::vector<u64> h(k * N);
  HEDAP_CUDA(cudaMemcpyAsync(h.data(), m.p, k * N * 8, cudaMemcpyDeviceToHost, C.stream));
  HEDAP_CUDA(cudaStreamSynchronize(C.stream));
  const u64* q = C.primes.data();
  std::vector<u64> inv_prefix(k, 1), half(k), dig(k);
  for (int i = 1; i < k; ++i) {
    u64 p = 1;
    for (int j = 0; j < i; ++j) p = h_mulmod(p, q[j] % q[i], q[i]);
    inv_prefix[i] = h_invmod(p, q[i]);
  }
  {  // mixed-radix digits of (Q-1)/2: Q-1 has digits q_i - 1; halve from the top
    u64 rem = 0;
    for (int i = k - 1; i >= 0; --i) {
      u128 cur = (u128)rem * q[i] + (q[i] - 1);
      half[i] = (u64)(cur / 2);
      rem = (u64)(cur % 2);
    }
  }
  std::vector<double> coef(N);
  for (size_t c = 0; c < N; ++c) {
    for (int i = 0; i < k; ++i) {
      u64 acc = 0;  // value of digits 0..i-1 modulo q_i, Horner from the top
      for (int j = i - 1; j >= 0; --j) acc = (u64)(((u128)acc * (q[j] % q[i]) + dig[j]) % q[i]);
      const u64 x = h[i * N + c] % q[i];
      dig[i] = i == 0 ? x : h_mulmod((x + q[i] - acc) % q[i], inv_prefix[i], q[i]);
    }
    int cmp = 0;
    for (int i = k - 1; i >= 0 && cmp == 0; --i) cmp = dig[i] > half[i] ? 1 : (dig[i] < half[i] ? -1 : 0);
    double v = 0;
    if (cmp <= 0) {
      for (int i = k - 1; i >= 0; --i) v = v * (double)q[i] + (double)dig[i];
    } else {  // negative: -(Q - x); Q - 1 - x has digits q_i - 1 - d_i, then + 1
      std::vector<u64> nd(k);
      u64 carry = 1;
      for (int i = 0; i < k; ++i) {
        u64 t = q[i] - 1 - dig[i] + carry;
        carry = t >= q[i];
        nd[i] = carry ? t - q[i] : t;
      }
      for (int i = k - 1; i >= 0; --i) v = v * (double)q[i] + (double)nd[i];
      v = -v;
    }
    coef[c] = v;
  }
  const size_t n = N / 2;
  std::vector<cplx> w(n);
  for (size_t j = 0; j < n; ++j) w[j] = cplx(coef[j] / ct.scale, coef[j + n] / ct.scale);
  SpecialFFT(C.log_n).forward(w);
  re.resize(n);
  im.resize(n);
  for (size_t j = 0; j < n; ++j) {
    re[j] = w[j].real();
    im[j] = w[j].imag();
  }
}

}  // namespace hedap
