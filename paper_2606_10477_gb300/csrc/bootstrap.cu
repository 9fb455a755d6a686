// Full-slot CKKS bootstrapping (BTS in the paper, Sec. 2.1: needs level >=
// l_BTS, inputs in [-1, 1], returns a ciphertext at l_afterBTS).  The paper
// treats it as a library primitive; this is the textbook construction:
//   ModRaise     level-0 coefficients (centred mod q_0) lifted to every Q prime:
//                plaintext t = m + q_0 I with |I| < K; with sparse-secret
//                encapsulation the level-0 ciphertext is first switched to an
//                ephemeral secret of small weight and the raised one back to s
//   CoeffToSlot  slots <- V^-1 slots for the decoding matrix V (z = V w), as the
//                radix-2 stages of the special FFT grouped into `cts` sparse
//                factors, each applied as a baby-step / giant-step sum of
//                plaintext diagonals times rotations (Halevi-Shoup, Chen-
//                Chillotti-Song 2019), the baby-step rotations hoisted (one
//                ModUp shared by all of them) and kept over Q_l u P: each
//                giant step sums its plaintext products there and divides by
//                P once (double hoisting, Bossuat et al. 2021); real /
//                imaginary parts split by conjugation and taken through
//                EvalMod as one batch
//   EvalMod      u = t / (q_0 K) -> sin(2 pi K u) = sin(2 pi m / q_0): Chebyshev
//                interpolant of cos(2 pi (K u - 1/4) / 2^r) and r double angles
//                (Bossuat et al. 2021)
//   SlotToCoeff  slots <- V slots (`stc` groups)
// Constant factors ride on the scale labels: ModRaise labels t with 2 q_0 K,
// and after EvalMod the label is multiplied by 2 pi s_in / q_0.
#include <cmath>
#include <complex>
#include <numeric>
#include <tuple>

#include "internal.cuh"
#include "kernels.cuh"
#include "profiler.cuh"

namespace hedap {

typedef std::complex<double> cplx;
typedef std::map<long, std::vector<cplx>> Diags;  // rotation offset (mod n) -> diagonal

// ------------------------------------------------------------------ FFT factor diagonals (host, FP64)
static std::vector<cplx> rotated(const std::vector<cplx>& v, long k) {  // out[s] = v[s + k mod n]
  const long n = (long)v.size();
  std::vector<cplx> out(n);
  const long sh = ((k % n) + n) % n;
  for (long s = 0; s < n; ++s) out[s] = v[(s + sh) % n];
  return out;
}

// stage of sub-transform length len (half h): forward
//   out_s = v_s + z_j v_{s+h} (first half), out_s = v_{s-h} - z_j v_s (second half)
// inverse
//   out_s = (v_s + v_{s+h}) / 2,            out_s = (v_{s-h} - v_s) conj(z_j) / 2
// with z_j = exp(2 pi i 5^j / (4 len)), j the position inside the half.
static Diags stage_diags(size_t n, size_t len, bool inverse) {
  const size_t h = len / 2;
  const u64 M = 4 * len;
  std::vector<cplx> self(n), up(n), down(n);
  for (size_t s = 0; s < n; ++s) {
    const size_t pos = s % len, j = pos % h;
    const cplx z = std::polar(1.0, 2.0 * M_PI * (double)h_powmod(5, j, M) / (double)M);
    const bool first = pos < h;
    if (!inverse) {
      if (first) { self[s] = 1.0; up[s] = z; } else { self[s] = -z; down[s] = 1.0; }
    } else {
      if (first) { self[s] = 0.5; up[s] = 0.5; } else { self[s] = -std::conj(z) * 0.5; down[s] = std::conj(z) * 0.5; }
    }
  }
  Diags D;
  D[0] = self;
  D[(long)h] = up;
  auto& d = D[(long)((n - h) % n)];  // equals D[h] when h = n/2: the two add
  if (d.empty()) d = down;
  else for (size_t s = 0; s < n; ++s) d[s] += down[s];
  return D;
}
// product A * B (B applied first): offset a + b gets A_a o rot(B_b, a)
static Diags diags_product(const Diags& A, const Diags& B, size_t n) {
  Diags R;
  for (const auto& a : A)
    for (const auto& b : B) {
      const long o = (a.first + b.first) % (long)n;
      const std::vector<cplx> rb = rotated(b.second, a.first);
      auto& dst = R[o];
      if (dst.empty()) dst.assign(n, cplx(0, 0));
      for (size_t s = 0; s < n; ++s) dst[s] += a.second[s] * rb[s];
    }
  return R;
}

struct LTGroup {  // one grouped factor and its baby-step / giant-step layout
  Diags d;
  long h0 = 1, kmin = 0, n1 = 1, giants = 1;
  std::map<long, const std::vector<cplx>*> by_k;  // k = offset / h0 (signed)
};

// baby-step / giant-step layout of the diagonals G.d, offsets taken mod n (signed)
static void layout_group(LTGroup& G, size_t n) {
  long h0 = 0;
  for (const auto& e : G.d) {
    const long o = e.first <= (long)n / 2 ? e.first : e.first - (long)n;
    if (o) h0 = h0 ? std::gcd(h0, std::labs(o)) : std::labs(o);
  }
  G.h0 = h0 ? h0 : 1;
  long kmax = 0;
  for (const auto& e : G.d) {
    const long o = e.first <= (long)n / 2 ? e.first : e.first - (long)n;
    const long k = o / G.h0;
    G.by_k[k] = &e.second;
    G.kmin = std::min(G.kmin, k);
    kmax = std::max(kmax, k);
  }
  // n1 baby steps: the power of two with n1^2 >= 4 span -- a giant step is a full key switch (ModUp and
  // ModDown), a baby step a hoisted rotation (inner product and ModDown only), about a quarter of the
  // transform work -- at most 16 per giant step (one diagonal MAC launch)
  const long span = kmax - G.kmin + 1;
  while (G.n1 * G.n1 < 4 * span) G.n1 <<= 1;
  G.n1 = std::min(G.n1, 16L);
  G.giants = (span + G.n1 - 1) / G.n1;
}
static std::vector<LTGroup> make_groups(size_t n, int groups, bool inverse) {
  int logn = 0;
  while (((size_t)1 << logn) < n) ++logn;
  std::vector<size_t> lens;  // in the order the stages are applied
  for (int i = 1; i <= logn; ++i) lens.push_back((size_t)1 << (inverse ? logn + 1 - i : i));
  std::vector<LTGroup> out(groups);
  size_t at = 0;
  for (int g = 0; g < groups; ++g) {
    const int stages = logn / groups + (g < logn % groups ? 1 : 0);
    Diags M = stage_diags(n, lens[at++], inverse);
    for (int k = 1; k < stages; ++k) M = diags_product(stage_diags(n, lens[at++], inverse), M, n);
    out[g].d = std::move(M);
    layout_group(out[g], n);
  }
  return out;
}
// Packed sparse slots (2n <= N/2): the last CoeffToSlot group multiplied on its output by the
// 2n-periodic mask (1 on [0, n), -i on [n, 2n)), so that s + conj(s) holds 2 Re on the first n slots
// and 2 Im on the next n; and the first SlotToCoeff group rewritten for a 2n-periodic input y whose
// slots j and j + n hold the real and imaginary parts of the n-periodic input it stands for: each
// diagonal d_k is split over offsets k and k + n with the factor 1 on the offset that reads [0, n)
// and i on the one that reads [n, 2n).
static cplx times_minus_i(cplx z) { return cplx(z.imag(), -z.real()); }
static cplx times_i(cplx z) { return cplx(-z.imag(), z.real()); }
static Diags packed_cts_last(const Diags& M, size_t n) {
  Diags R;
  for (const auto& e : M) {
    std::vector<cplx> d(2 * n);
    for (size_t j = 0; j < 2 * n; ++j) d[j] = j < n ? e.second[j] : times_minus_i(e.second[j - n]);
    R[e.first] = std::move(d);
  }
  return R;
}
static Diags packed_stc_first(const Diags& M, size_t n) {
  Diags R;
  const long P = (long)(2 * n);
  auto add = [&](long off, size_t j, cplx v) {
    auto& d = R[((off % P) + P) % P];
    if (d.empty()) d.assign(2 * n, cplx(0, 0));
    d[j] += v;
  };
  for (const auto& e : M) {
    const long k = e.first;
    for (size_t j = 0; j < 2 * n; ++j) {
      const cplx v = e.second[j % n];
      const bool lo = ((long)j + k) % P < (long)n;  // offset k reads the first n slots
      add(k, j, lo ? v : times_i(v));
      add(k + (long)n, j, lo ? times_i(v) : v);
    }
  }
  return R;
}

struct PlainSet {  // encoded, NTT-domain diagonals of one group at one level and plaintext scale
  int level = -1;
  double sp = 0;
  std::map<std::pair<long, long>, DevBuf> pt;  // (giant g, baby b) -> [level+1][N]
};

struct BtsState {
  int K = 28, r = 4, deg = 31, cts = 3, stc = 3;
  std::vector<LTGroup> cts_groups, stc_groups;      // N/2 slots
  std::map<size_t, std::pair<std::vector<LTGroup>, std::vector<LTGroup>>> sparse;  // n -> (CtS, StC) groups
  std::map<size_t, std::pair<LTGroup, LTGroup>> packed;  // n -> (last CtS group, first StC group), period 2n
  std::map<std::tuple<size_t, int, int>, PlainSet> plains;  // (slots, inverse, group) -> encoded diagonals
  std::vector<double> mod_coeffs;                  // Chebyshev coefficients of the scaled cosine
};
void BtsStateDeleter::operator()(BtsState* p) const { delete p; }

// ------------------------------------------------------------------ kernels
// ModRaise: from limb 0 in the coefficient domain (both parts, stride N) to every
// limb 0..L of out: the centred representative of x mod q_0, reduced mod q_i.
__global__ void k_mod_raise_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ x, u64* __restrict__ out,
                                   size_t os, int n_parts, int limbs, int log_n) {
  const size_t N = (size_t)1 << log_n, per = (size_t)limbs << log_n, total = n_parts * per;
  const u64 q0 = pr[0].q, h = q0 >> 1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / per);
    const size_t r = e - p * per;
    const int i = (int)(r >> log_n);
    const u64 v = x[p * N + (r & (N - 1))];
    const PrimeDev P = pr[i];
    u64 m = barrett_reduce(v, 0, P);
    if (v > h) m = sub_mod(m, barrett_reduce(q0, 0, P), P.q);
    out[p * os + r] = m;
  }
}
// multiply by X^(N/2) (factor iota_i) or X^(3N/2) (factor -iota_i), iota_i = psi_i^(N/2):
// the evaluation at psi^(2 bitrev(j) + 1) picks up iota^(2 bitrev(j)+1) = iota (-1)^bitrev(j),
// and bitrev(j) is odd exactly when j >= N/2.
__global__ void k_monomial_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ in, size_t is,
                                  u64* __restrict__ out, size_t os, int n_parts, int limbs, int log_n, LimbConsts F) {
  const size_t N = (size_t)1 << log_n, per = (size_t)limbs << log_n, total = n_parts * per;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / per);
    const size_t r = e - p * per;
    const int i = (int)(r >> log_n);
    const u64 q = pr[i].q;
    u64 v = shoup_mul(in[p * is + r], F.w[i], F.wsh[i], q);
    if ((r & (N - 1)) >= N / 2 && v) v = q - v;
    out[p * os + r] = v;
  }
}
// integer coefficients (|c| < 2^63) to residues on `limbs` limbs: limb li < q_count of prime li, the
// others of prime p_first + (li - q_count)
__global__ void k_coeffs_to_limbs_kernel(const PrimeDev* __restrict__ pr, const long long* __restrict__ c,
                                         u64* __restrict__ out, int limbs, int log_n, int q_count, int p_first) {
  const size_t N = (size_t)1 << log_n, total = (size_t)limbs << log_n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int li = (int)(e >> log_n);
    const PrimeDev P = pr[li < q_count ? li : p_first + (li - q_count)];
    const long long v = c[e & (N - 1)];
    const u64 a = barrett_reduce(v < 0 ? (u64)(-(v + 1)) + 1 : (u64)v, 0, P);
    out[e] = (v < 0 && a) ? P.q - a : a;
  }
}
// acc[p][i][k] = sum_b ct_b[p][i][k] * pt_b[i][k]  (plaintext-ciphertext products of one giant step);
// limb i < q_count has prime i, the others prime p_first + (i - q_count)
struct PtMacArgs {
  const u64* ct[16];
  size_t cs[16];
  const u64* pt[16];
  int count;
};
__global__ void k_pt_mac_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ r64s, PtMacArgs A,
                                u64* __restrict__ out, size_t os, int n_parts, int limbs, int log_n, int q_count,
                                int p_first) {
  const size_t per = (size_t)limbs << log_n, total = n_parts * per;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / per);
    const size_t r = e - p * per;
    const int li = (int)(r >> log_n), i = li < q_count ? li : p_first + (li - q_count);
    Acc128 s{0, 0};
    for (int b = 0; b < A.count; ++b) mac128(s, A.ct[b][p * A.cs[b] + r], A.pt[b][r]);
    out[p * os + r] = reduce128(s, pr[i], r64s[2 * i], r64s[2 * i + 1]);
  }
}

// ------------------------------------------------------------------ operations
std::unique_ptr<Ct> mod_raise(Ctx& C, const Ct& a) {
  if (a.level != 0) throw Error(HEDAP_ERR_LEVEL, "ModRaise needs a level-0 ciphertext");
  const size_t N = C.N;
  const int L = C.L(), P = a.parts();
  DevBuf x((size_t)P * N, C.stream);
  HEDAP_CUDA(cudaMemcpy2DAsync(x.p, N * 8, a.part(0), a.part_stride() * 8, N * 8, P, cudaMemcpyDeviceToDevice,
                               C.stream));
  ntt_inverse(C.tab, LimbSet{x.p, N, P, 0, 1, INT_MAX, 0, 0}, C.stream);
  auto o = ct_alloc(C, L, a.batch);
  o->scale = a.scale;
  {
    ProfScope prof_(PROF_ELEMENTWISE, C.stream, (1.0 + (L + 1.0)) * P * N * 8);
    prof_count_launches(1);
    k_mod_raise_kernel<<<grid_for((size_t)P * (L + 1) * N, 256), 256, 0, C.stream>>>(C.tab.pr, x.p, o->part(0),
                                                                                      o->part_stride(), P, L + 1,
                                                                                      C.log_n);
    HEDAP_LAUNCH_CHECK();
  }
  ntt_forward(C.tab, LimbSet{o->part(0), o->part_stride(), P, 0, L + 1, INT_MAX, 0, 0}, C.stream);
  return o;
}

std::unique_ptr<Ct> mul_monomial(Ctx& C, const Ct& a, u64 e) {
  const u64 n2 = C.N / 2;
  if (e != n2 && e != 3 * n2) throw Error(HEDAP_ERR_ARG, "monomial exponent must be N/2 or 3N/2");
  LimbConsts F;
  for (int i = 0; i <= a.level; ++i) {
    const u64 q = C.primes[i];
    const u64 iota = h_powmod(h_find_psi(q, C.log_n), n2, q);
    F.w[i] = e == n2 ? iota : q - iota;
    F.wsh[i] = h_shoup(F.w[i], q);
  }
  auto o = ct_alloc(C, a.level, a.batch);
  o->scale = a.scale;
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, 2.0 * a.parts() * (a.level + 1) * C.N * 8);
  prof_count_launches(1);
  k_monomial_kernel<<<grid_for((size_t)a.parts() * (a.level + 1) * C.N, 256), 256, 0, C.stream>>>(
      C.tab.pr, a.part(0), a.part_stride(), o->part(0), o->part_stride(), a.parts(), a.level + 1, C.log_n, F);
  HEDAP_LAUNCH_CHECK();
  return o;
}

static BtsState& state(Ctx& C) {
  if (!C.bts) throw Error(HEDAP_ERR_ARG, "bootstrapping is not configured on this context");
  return *C.bts;
}

// CtS (inverse) or StC groups for n slots (n = N/2, or sparse packing with period n)
static const std::vector<LTGroup>& groups_for(Ctx& C, BtsState& S, size_t n, bool inverse) {
  if (n == C.N / 2) return inverse ? S.cts_groups : S.stc_groups;
  auto it = S.sparse.find(n);
  if (it == S.sparse.end())
    it = S.sparse.emplace(n, std::make_pair(make_groups(n, S.cts, true), make_groups(n, S.stc, false))).first;
  return inverse ? it->second.first : it->second.second;
}

// encode a diagonal (n values, repeated over the N/2 slots) at plaintext scale sp onto limbs
// 0..level and the special limbs (Q_level u P, NTT domain)
static DevBuf encode_diag(Ctx& C, const std::vector<cplx>& dn, double sp, int level) {
  std::vector<cplx> d(C.N / 2);
  for (size_t s = 0; s < d.size(); ++s) d[s] = dn[s % dn.size()];
  std::vector<double> m = encode_slots(C, d, sp);
  std::vector<long long> ci(C.N);
  for (size_t k = 0; k < C.N; ++k) {
    if (!(std::fabs(m[k]) < 9.0e18)) throw Error(HEDAP_ERR_RANGE, "diagonal coefficient exceeds 63 bits");
    ci[k] = (long long)m[k];
  }
  const int ext = level + 1 + C.n_p;
  DevBuf coef(C.N, C.stream), out((size_t)ext * C.N, C.stream);
  HEDAP_CUDA(cudaMemcpyAsync(coef.p, ci.data(), C.N * 8, cudaMemcpyHostToDevice, C.stream));
  k_coeffs_to_limbs_kernel<<<grid_for((size_t)ext * C.N, 256), 256, 0, C.stream>>>(
      C.tab.pr, (const long long*)coef.p, out.p, ext, C.log_n, level + 1, C.n_q);
  HEDAP_LAUNCH_CHECK();
  prof_count_launches(1);
  ntt_forward(C.tab, LimbSet{out.p, 0, 1, 0, ext, level + 1, 0, C.n_q}, C.stream);
  HEDAP_CUDA(cudaStreamSynchronize(C.stream));  // ci is a host temporary
  return out;
}

// sum_g rot( sum_b rot(D_k, -G_g) o rot(v, b h0), G_g ),  k = kmin + g n1 + b,  G_g = h0 (kmin + g n1);
// one rescale at the end; the result's scale is `target`
// group G (diagonals of period `slots`) applied to v, its encoded diagonals cached in P
static std::unique_ptr<Ct> lt_apply(Ctx& C, const Ct& v, const LTGroup& G, PlainSet& P, double target, size_t slots) {
  const int l = v.level;
  if (l < 1) throw Error(HEDAP_ERR_LEVEL, "linear transform needs level >= 1");
  const double sp = target * (double)C.primes[l] / v.scale;
  if (P.level != l || P.sp != sp) {  // (re)encode; the cache is marked valid only once complete
    P.pt.clear();
    P.level = -1;
    for (long g = 0; g < G.giants; ++g)
      for (long b = 0; b < G.n1; ++b) {
        auto it = G.by_k.find(G.kmin + g * G.n1 + b);
        if (it == G.by_k.end()) continue;
        P.pt[{g, b}] = encode_diag(C, rotated(*it->second, -G.h0 * (G.kmin + g * G.n1)), sp, l);
      }
    P.level = l;
    P.sp = sp;
  }
  // baby steps: every rotation of v any giant step uses, hoisted (one ModUp of v) and kept over Q_l u P
  // before its ModDown (double hoisting, Bossuat et al. 2021); b = 0 is v itself, (P c0, P c1)
  const int ext = l + 1 + C.n_p;
  const size_t qp_stride = (size_t)ext * C.N;  // part stride of a pair batch [batch][2][ext][N]
  std::vector<DevBuf> baby(G.n1);
  {
    std::vector<long> need;
    for (long b = 1; b < G.n1; ++b)
      for (long g = 0; g < G.giants; ++g)
        if (P.pt.count({g, b})) {
          need.push_back(b);
          break;
        }
    std::vector<u64> gs;
    for (long b : need) gs.push_back(galois_for_rotation(C, b * G.h0));
    auto rot = ev_galois_hoisted_qp(C, v, gs);
    for (size_t i = 0; i < need.size(); ++i) baby[need[i]] = std::move(rot[i]);
    for (long g = 0; g < G.giants; ++g)
      if (P.pt.count({g, 0})) {
        baby[0] = DevBuf((size_t)v.parts() * qp_stride, C.stream);
        k_lift_qp(C, v.part(0), v.part_stride(), baby[0].p, v.parts(), l);
        break;
      }
  }
  std::unique_ptr<Ct> acc;
  const long n = (long)slots;
  for (long g = 0; g < G.giants; ++g) {
    PtMacArgs A;
    A.count = 0;
    for (long b = 0; b < G.n1; ++b) {
      auto it = P.pt.find({g, b});
      if (it == P.pt.end()) continue;
      if (A.count == 16) throw Error(HEDAP_ERR_ARG, "more than 16 baby steps");
      A.ct[A.count] = baby[b].p;
      A.cs[A.count] = qp_stride;
      A.pt[A.count] = it->second.p;
      ++A.count;
    }
    if (!A.count) continue;
    // sum_b diag o baby_b over Q_l u P, then one ModDown for the giant step
    DevBuf sum((size_t)v.parts() * qp_stride, C.stream);
    {
      ProfScope prof_(PROF_ELEMENTWISE, C.stream, (1.5 * A.count + 1.0) * v.parts() * ext * C.N * 8);
      prof_count_launches(1);
      k_pt_mac_kernel<<<grid_for((size_t)v.parts() * ext * C.N, 256), 256, 0, C.stream>>>(
          C.tab.pr, C.d_r64.p, A, sum.p, qp_stride, v.parts(), ext, C.log_n, l + 1, C.n_q);
      HEDAP_LAUNCH_CHECK();
    }
    auto inner = ct_alloc(C, l, v.batch);
    inner->scale = v.scale * sp;
    ev_moddown_into(C, sum, v.batch, l, *inner);
    const long Gs = G.h0 * (G.kmin + g * G.n1);
    std::unique_ptr<Ct> r = (((Gs % n) + n) % n) ? ev_galois(C, *inner, galois_for_rotation(C, Gs)) : std::move(inner);
    acc = acc ? ev_add(C, *acc, *r, false) : std::move(r);
  }
  auto out = ev_rescale(C, *acc);
  out->scale = target;
  return out;
}
std::unique_ptr<Ct> bts_linear_transform(Ctx& C, const Ct& v, bool inverse, int gi, double target, size_t slots) {
  BtsState& S = state(C);
  if (!slots) slots = C.N / 2;
  return lt_apply(C, v, groups_for(C, S, slots, inverse).at(gi), S.plains[{slots, inverse ? 1 : 0, gi}], target,
                  slots);
}
// the packed last CoeffToSlot group (inverse) or first SlotToCoeff group of n sparse slots, period 2n
static std::unique_ptr<Ct> lt_packed(Ctx& C, const Ct& v, bool inverse, size_t n, double target) {
  BtsState& S = state(C);
  auto it = S.packed.find(n);
  if (it == S.packed.end()) {
    it = S.packed.emplace(std::piecewise_construct, std::forward_as_tuple(n), std::forward_as_tuple()).first;
    it->second.first.d = packed_cts_last(groups_for(C, S, n, true).back().d, n);
    layout_group(it->second.first, 2 * n);
    it->second.second.d = packed_stc_first(groups_for(C, S, n, false).front().d, n);
    layout_group(it->second.second, 2 * n);
  }
  const LTGroup& G = inverse ? it->second.first : it->second.second;
  return lt_apply(C, v, G, S.plains[{2 * n, inverse ? 3 : 2, 0}], target, 2 * n);
}

// Chebyshev interpolant (first-kind nodes on [lo, hi]) of an arbitrary function
template <class F>
static std::vector<double> interp(F f, double lo, double hi, int d) {
  const int n = d + 1;
  std::vector<double> fx(n), c(n);
  for (int k = 0; k < n; ++k) fx[k] = f(0.5 * (lo + hi) + 0.5 * (hi - lo) * std::cos(M_PI * (k + 0.5) / n));
  for (int j = 0; j < n; ++j) {
    double acc = 0;
    for (int k = 0; k < n; ++k) acc += fx[k] * std::cos(M_PI * j * (k + 0.5) / n);
    c[j] = (j == 0 ? 1.0 : 2.0) / n * acc;
  }
  return c;
}

std::unique_ptr<Ct> eval_mod(Ctx& C, const Ct& u) {
  BtsState& S = state(C);
  std::unique_ptr<Ct> c = cheb_eval(C, u, S.mod_coeffs, u.scale, -1);  // fewest levels
  for (int i = 0; i < S.r; ++i)  // cos 2x = 2 cos^2 x - 1
    c = ev_add_const_mul_int(C, *ev_mul(C, *c, *c), -0.5, 2);
  return c;
}

// sum of the rotations by n, 2n, ..., N/4: the plaintext's part in Z[X^(N/2n)] times N/2n (the
// automorphisms X -> X^(5^(n j)) are those fixing that subring, since 5^(n j) = 1 mod 4n)
std::unique_ptr<Ct> sub_sum(Ctx& C, const Ct& a, size_t n) {
  if (n < 1 || n > C.N / 2 || (n & (n - 1))) throw Error(HEDAP_ERR_ARG, "slot count must be a power of two <= N/2");
  auto t = ct_copy(C, a, a.level);
  for (size_t k = n; k < C.N / 2; k *= 2) t = ev_add(C, *t, *ev_galois(C, *t, galois_for_rotation(C, (i64)k)), false);
  return t;
}

std::unique_ptr<Ct> bootstrap_core(Ctx& C, const Ct& a, int log_slots) {
  BtsState& S = state(C);
  if (a.level != 0) throw Error(HEDAP_ERR_LEVEL, "bootstrap input must be at level 0");
  if (log_slots < 0 || (log_slots && ((size_t)1 << log_slots) > C.N / 2) ||
      (log_slots && log_slots < std::max(S.cts, S.stc)))
    throw Error(HEDAP_ERR_ARG, "log_slots out of range for this bootstrapping configuration");
  const size_t n = log_slots ? (size_t)1 << log_slots : C.N / 2;
  const double s_in = a.scale, q0 = (double)C.primes[0];
  std::unique_ptr<Ct> t;
  if (C.enc_hw) {  // sparse-secret encapsulation: ModRaise under s~, then back to s at the top level
    t = ev_switch_key(C, *mod_raise(C, *ev_switch_key(C, a, kKeyToSparse)), kKeyToDense);
  } else {
    t = mod_raise(C, a);
  }
  if (n < C.N / 2) t = sub_sum(C, *t, n);  // sparse packing: project q_0 I onto the subring
  t->scale = 2.0 * q0 * S.K * (double)(C.N / 2 / n);
  if (n < C.N / 2) {  // real and imaginary parts packed in 2n slots: one EvalMod
    for (int g = 0; g + 1 < S.cts; ++g) t = bts_linear_transform(C, *t, true, g, (double)C.primes[t->level - 1], n);
    t = lt_packed(C, *t, true, n, (double)C.primes[t->level - 1]);
    auto w = eval_mod(C, *ev_add(C, *t, *ev_galois(C, *t, 2 * C.N - 1), false));  // 2 Re | 2 Im, then EvalMod
    w->scale = w->scale * 2.0 * M_PI * s_in / q0;
    w = lt_packed(C, *w, false, n, S.stc == 1 ? C.scale : (double)C.primes[w->level - 1]);
    for (int g = 1; g < S.stc; ++g)
      w = bts_linear_transform(C, *w, false, g, g + 1 == S.stc ? C.scale : (double)C.primes[w->level - 1], n);
    return w;
  }
  for (int g = 0; g < S.cts; ++g) t = bts_linear_transform(C, *t, true, g, (double)C.primes[t->level - 1], n);
  auto cj = ev_galois(C, *t, 2 * C.N - 1);
  auto re = ev_add(C, *t, *cj, false);
  auto im = mul_monomial(C, *ev_add(C, *t, *cj, true), 3 * C.N / 2);  // times -i
  if (2 * re->batch <= 16) {  // both parts through one batched EvalMod
    auto both = eval_mod(C, *batch_pack(C, {re.get(), im.get()}));
    const int B = re->batch;
    re = batch_slice(C, *both, 0, B);
    im = batch_slice(C, *both, B, B);
  } else {
    re = eval_mod(C, *re);
    im = eval_mod(C, *im);
  }
  auto w = ev_add(C, *re, *mul_monomial(C, *im, C.N / 2), false);  // re + i im
  w->scale = w->scale * 2.0 * M_PI * s_in / q0;
  for (int g = 0; g < S.stc; ++g)
    w = bts_linear_transform(C, *w, false, g, g + 1 == S.stc ? C.scale : (double)C.primes[w->level - 1], n);
  return w;
}

// y with values in [-Y, Y]: scale by 1/Y into [-1, 1], landing at level 0 with scale
// q_0 / 2^12, bootstrap, then multiply by the integer Y
std::unique_ptr<Ct> bootstrap_scaled(Ctx& C, const Ct& y, i64 Y, int log_slots) {
  if (y.level < 1) throw Error(HEDAP_ERR_LEVEL, "bootstrap needs an input at level >= 1");
  std::unique_ptr<Ct> d = y.level > 1 ? ev_drop(C, y, 1) : nullptr;
  auto a = ev_mul_const(C, d ? *d : y, 1.0 / (double)Y, (double)C.primes[0] / 4096.0);
  auto b = bootstrap_core(C, *a, log_slots);
  return Y == 1 ? std::move(b) : ev_mul_int(C, *b, Y);
}

// diagonal of a grouped factor (test access): returns false when the offset is absent
bool bts_diagonal(Ctx& C, bool inverse, int g, long offset, std::vector<std::complex<double>>& out) {
  const LTGroup& G = (inverse ? state(C).cts_groups : state(C).stc_groups).at(g);
  auto it = G.d.find(offset);
  if (it == G.d.end()) return false;
  out = it->second;
  return true;
}

int bts_setup(Ctx& C, int K, int r, int deg, int cts, int stc) {
  if (K < 1 || r < 0 || r > 8 || deg < 2 || deg > 255 || cts < 1 || stc < 1 || cts > C.log_n - 1 ||
      stc > C.log_n - 1)
    throw Error(HEDAP_ERR_ARG, "invalid bootstrapping parameters");
  int m = 0;
  while ((1 << m) < deg + 1) ++m;
  const int levels = cts + m + r + stc;  // EvalMod: the Chebyshev interpolant (m levels), r double angles
  if (C.L() - levels < 1) throw Error(HEDAP_ERR_LEVEL, "prime chain too short for bootstrapping");
  std::unique_ptr<BtsState> S(new BtsState);
  S->K = K;
  S->r = r;
  S->deg = deg;
  S->cts = cts;
  S->stc = stc;
  const size_t n = C.N / 2;
  S->cts_groups = make_groups(n, cts, true);
  S->stc_groups = make_groups(n, stc, false);
  const double Kd = K, R = std::ldexp(1.0, r);
  S->mod_coeffs = interp([&](double x) { return std::cos(2.0 * M_PI * (Kd * x - 0.25) / R); }, -1.0, 1.0, deg);
  C.bts.reset(S.release());
  return C.L() - levels;
}

}  // namespace hedap
