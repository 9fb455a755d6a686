// Internal declarations of the GB300 RNS-CKKS library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <climits>
#include <complex>
#include <cstdint>
#include <functional>
#include <map>
#include <mutex>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "hedap.h"
#include "modarith.cuh"

namespace hedap {

typedef int64_t i64;

struct Error : std::runtime_error {
  hedap_status code;
  Error(hedap_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define HEDAP_CUDA(x)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess)                                                                   \
      throw ::hedap::Error(e_ == cudaErrorMemoryAllocation ? HEDAP_ERR_OOM : HEDAP_ERR_CUDA,  \
                           std::string(#x) + ": " + cudaGetErrorString(e_));                 \
  } while (0)
#define HEDAP_LAUNCH_CHECK() HEDAP_CUDA(cudaGetLastError())

// ------------------------------------------------------------------ host math (params.cu)
u64 h_mulmod(u64 a, u64 b, u64 q);
u64 h_powmod(u64 a, u64 e, u64 q);
u64 h_invmod(u64 a, u64 q);
bool h_is_prime(u64 n);
std::vector<u64> h_prime_chain(int log_n, const std::vector<int>& bits);
u64 h_find_psi(u64 q, int log_n);
u64 h_shoup(u64 w, u64 q);  // floor(w * 2^64 / q)
PrimeDev h_prime_dev(u64 q);
uint32_t h_bitrev(uint32_t x, int bits);
u64 h_smod(i64 v, u64 q);
u64 h_double_to_mod(double x, u64 q);  // exact residue of an integer-valued double

// SplitMix64 streams (Steele, Lea, Flood 2014); a stream for (seed, tag)
// starts at mix(seed) ^ mix(tag ^ 0x5851F42D4C957F2D).
struct SplitMix {
  u64 state;
  SplitMix(u64 seed, u64 tag);
  u64 next();
};
namespace tags {
inline u64 evk_a(u64 g, u64 j) { return (2ull << 56) | (g << 8) | j; }
inline u64 evk_e(u64 g, u64 j) { return (3ull << 56) | (g << 8) | j; }
const u64 sk = 1, enc_a = 4ull << 56, enc_e = 5ull << 56, sk_sparse = 6ull << 56;
}  // namespace tags
u64 draw_uniform(SplitMix& s, u64 q);
i64 draw_cbd21(SplitMix& s);
std::vector<i64> draw_ternary(SplitMix& s, int log_n, int hw);

// ------------------------------------------------------------------ device memory
// Stream-ordered allocation from the device's default memory pool (kept
// cached: the pool's release threshold is raised at context creation).
struct DevBuf {
  u64* p = nullptr;
  size_t words = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(size_t n, cudaStream_t st);
  ~DevBuf();
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), words(o.words), s(o.s) { o.p = nullptr; o.words = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept;
};

// ------------------------------------------------------------------ tables and limb sets
struct Tables {
  const PrimeDev* pr;        // [n_primes]
  const ulonglong2* psi2;    // [n_primes][N] (psi^bitrev(i), Shoup companion)
  const ulonglong2* ipsi2;   // [n_primes][N] (psi^-bitrev(i), Shoup companion)
  const u64* ninv;           // [n_primes] N^-1
  const u64* ninv_sh;
  int log_n;
  // NTT launch shapes (see ntt_impl.cuh) per role, chosen by ntt_tune: the plain forward transform, the
  // inverse, the forward with the ModUp conversion fused into its load (the key switch's extended digits),
  // and the forward with a fused ModDown / rescale (conversion or spread load, finishing store)
  int ntt_fwd_variant;
  int ntt_inv_variant;
  int ntt_modup_variant;
  int ntt_fin_variant;
};
constexpr int kNttVariants = 8;
enum NttRole { NTT_ROLE_FORWARD = 0, NTT_ROLE_INVERSE = 1, NTT_ROLE_MODUP = 2, NTT_ROLE_FINISH = 3 };
int& ntt_role_variant(Tables& T, int role);

// A set of limbs: parts p in [0, n_parts), limbs li in [limb_begin, limb_begin+n_limbs)
// at base + p*part_stride + li*N.  Limb li < q_count uses prime prime_offset+li,
// otherwise prime p_first + (li - q_count).
struct LimbSet {
  u64* base;
  size_t part_stride;
  int n_parts;
  int limb_begin;
  int n_limbs;
  int q_count;
  int prime_offset;
  int p_first;
  __host__ __device__ int prime(int li) const {
    return li < q_count ? prime_offset + li : p_first + (li - q_count);
  }
  __host__ __device__ u64* limb(int part, int li, size_t N) const {
    return base + part * part_stride + (size_t)li * N;
  }
};

// Optional fusions of one batched transform (value-initialised: a plain in-place transform).
struct NttAux {
  // out of place: the first phase reads limb li of part p at src + p * src_stride + li * N
  const u64* src = nullptr;
  size_t src_stride = 0;
  // inverse only: the final factor of limb li is the pair post[2 r], post[2 r + 1] (value, Shoup
  // companion), r = li - limb_begin, instead of N^-1
  const u64* post = nullptr;
  // skip the limbs li of digit j = part % own_dn, li in [j own_alpha, min((j + 1) own_alpha, own_limit))
  int own_alpha = 0;
  int own_dn = 1;
  int own_limit = 0;
  // forward only: the first phase loads the fast basis conversion of digit j into the prime of limb li,
  //   sum_a z[k][j alpha + a] * bconv[j][a][li]  mod prime(li),  k = part / own_dn, alpha = own_alpha,
  // from z (limb stride N, member stride z_stride) instead of reading limb li
  const u64* z = nullptr;
  size_t z_stride = 0;
  const u64* bconv = nullptr;  // [dn][alpha][ext]; their Shoup companions at bconv + bconv_sh_offset
  size_t bconv_sh_offset = 0;  // a companion 0 marks a factor 1: z is added without a product
  int ext = 0;
  double z_products = -1;  // products of the whole launch's conversion (word x term), for the profiler
  // forward only: the first phase loads the centred residue of one coefficient-domain limb (the
  // last limb of a rescale, prime index spread_prime) into the prime of limb li:
  //   m = x mod q_li, minus spread_sub[li] when x > q_spread / 2,  x = spread[part * spread_stride + n]
  const u64* spread = nullptr;
  size_t spread_stride = 0;
  const u64* spread_sub = nullptr;
  int spread_prime = 0;
  // forward only: the first phase loads the ModDown conversion of K special limbs (coefficient
  // domain, z_k = x_k shat_k^-1 at pconv + part * pconv_stride + k * N, moduli s_k = pconv_q[k],
  // S = prod s_k) into the prime of limb li: sum_k [z_k + c_k]_{s_k} shat_k mod q_li - floor(S/2)
  const u64* pconv = nullptr;
  size_t pconv_stride = 0;
  int pconv_K = 0;
  int pconv_ld = 0;                   // row length of the per-target tables
  const u64* pconv_q = nullptr;       // [K] the special moduli s_k
  const u64* pconv_c = nullptr;       // [K] floor(S/2) shat_k^-1 mod s_k
  const u64* pconv_phat = nullptr;    // [K][ld] (S / s_k) mod q_i
  const u64* pconv_phat_sh = nullptr; // their Shoup companions
  const u64* pconv_half = nullptr;    // [ld] floor(S/2) mod q_i
  // forward only: the second phase does not store the transform v; it writes
  //   fin_dst[part][li] = (fin_c[part][li] - v) * fin_w[li]  (+ fin_dst[part][li] when the part's
  //   parity bit is set), Shoup factors fin_w / fin_wsh per limb, canonical residues
  u64* fin_dst = nullptr;
  size_t fin_dst_stride = 0;
  const u64* fin_c = nullptr;
  size_t fin_c_stride = 0;
  const u64* fin_w = nullptr;
  const u64* fin_wsh = nullptr;
  int fin_acc_even = 0, fin_acc_odd = 0;
  // with fin_e: a key switch's ModDown fused with the rescale that follows it (see ks_moddown_rescale):
  //   fin_dst[part][li] = fin_c[part][li] * fin_w[li] + (fin_e[part][li] - v) * fin_w2[li]
  // (fin_w = (P q_l)^-1, fin_w2 = q_l^-1), and the first phase loads the ModDown conversion with its
  // constants scaled by P^-1 plus the spread of the centred last limb (pconv and spread both set)
  const u64* fin_e = nullptr;
  size_t fin_e_stride = 0;
  const u64* fin_w2 = nullptr;
  const u64* fin_w2sh = nullptr;
  int fin_neg = 0;  // with fin_e: store the negated residues
};
// Forward only: the second phase of the ModUp transform of a key switch fused with the key inner
// product (k_ntt_fwd_rows_ksk): the transformed digits are multiplied by the switching key and summed
// over the digits instead of being stored.  The LimbSet's parts are (ciphertext k, digit j) = k dn + j
// (dn = NttAux::own_dn), its limbs the extended limbs t; a digit's own limbs are read from d.
struct KskFuse {
  const u64* d = nullptr;        // NTT-domain inputs: ciphertext k's limb t at d + k d_stride + t N
  size_t d_stride = 0;
  const u64* key = nullptr;      // switching key [dn][2][n_q + n_p][N] (digit j: b then a)
  size_t key_digit_stride = 0;   // 2 (n_q + n_p) N
  size_t key_a_offset = 0;       // (n_q + n_p) N
  u64* acc = nullptr;            // output: part p of ciphertext k, limb t at acc + (2k + p) acc_part_stride + t N
  size_t acc_part_stride = 0;
  const u64* r64 = nullptr;      // per prime: 2^64 mod q and its Shoup companion
  int batch = 0;
};
void ntt_forward(const Tables& T, const LimbSet& S, cudaStream_t st, const NttAux* aux = nullptr,
                 const KskFuse* fuse = nullptr);
void ntt_inverse(const Tables& T, const LimbSet& S, cudaStream_t st, const NttAux* aux = nullptr);
struct Ctx;
void ntt_tune(Ctx& C, int limbs, int reps, std::vector<float>* fwd_ms, std::vector<float>* inv_ms);
double butterfly_rate(Ctx& C);  // butterflies per second of a register-only loop

// ------------------------------------------------------------------ context and ciphertexts
// One ciphertext, or a batch of `batch` ciphertexts at one level and scale:
// [batch][2][cap][N] words, ciphertext k owning parts 2k (c0) and 2k+1 (c1).
struct Ctx;
struct Ct {
  DevBuf buf;
  const Ctx* owner = nullptr;  // the context that made it
  int cap = 0;     // limbs allocated per part
  int level = 0;
  int batch = 1;
  double scale = 1;
  size_t N = 0;
  u64* part(int p) const { return buf.p + (size_t)p * cap * N; }
  size_t part_stride() const { return (size_t)cap * N; }
  int parts() const { return 2 * batch; }
};

constexpr int kMaxLimbs = 64;
// one constant per Q limb, passed to kernels by value (w and its Shoup companion)
struct LimbConsts {
  u64 w[kMaxLimbs];
  u64 wsh[kMaxLimbs];
};
// one launch of a linear combination of ciphertexts with per-limb integer constants (k_lincomb)
constexpr int kLcTerms = 8, kLcLimbs = 32;
struct LinCombArgs {
  const u64* in[kLcTerms];  // part p of term j at in[j] + p * stride[j]
  size_t stride[kLcTerms];
  u64 w[kLcTerms][kLcLimbs];
  u64 wsh[kLcTerms][kLcLimbs];
  u64 c0[kLcLimbs];  // added to the even (c0) parts when add_c0
  int count, add_c0, accumulate;
};
// rescale by q_l: per i < l, q_l mod q_i and q_l^-1 mod q_i (+ Shoup)
struct RescaleConsts {
  u64 ql_mod[kMaxLimbs];
  u64 inv[kMaxLimbs];
  u64 inv_sh[kMaxLimbs];
};

// ModDown of limb l (prime q_l) scaled by P^-1: x - (sum_k [z_k + c_k]_{p_k} p_k^-1 + off) mod q_l
struct MdrLast {
  u64 p[8], c[8], f[8], fs[8];  // p_k, floor(P/2) phinv_k mod p_k, p_k^-1 mod q_l and its Shoup companion
  u64 off;                      // -floor(P/2) P^-1 mod q_l
  u64 pinv, pinv_sh;            // P^-1 mod q_l and its Shoup companion
  int K;
};
struct LevelConsts {  // device constants for one level (evaluator.cu)
  DevBuf modup;       // qhat_inv (+shoup) per Q prime, qhat mod target per digit (+shoup)
  DevBuf modup_ks;    // the same with every factor divided by the key's scale (key_scale); a factor 1
                      // folded into the key has Shoup companion 0 (the load adds z without a product)
  double modup_products = 0;  // products per word of one ciphertext's fused ModUp (folded terms excluded)
  DevBuf intt_post;   // per Q prime i <= l: N^-1 qhat_i^-1 mod q_i and its Shoup companion
  DevBuf d_rescale;   // [ql_mod l][inv l][inv_sh l] (the rescale constants below, on the device)
  RescaleConsts rescale;
  DevBuf d_mdr;       // ModDown fused with the rescale: [(P q_l)^-1 mod q_i][its Shoup companion], i < l
  MdrLast mdr_last;   // ... and the constants of its last limb (prime q_l)
};

struct BtsState;  // bootstrapping state (bootstrap.cu)
struct BtsStateDeleter {
  void operator()(BtsState* p) const;
};

// CUDA streams that a server's groups run on.  The context owns them (and destroys them last), so that
// a buffer allocated on one of them -- a cached table, a key built during a group's step -- can still be
// freed on it until the context goes.
struct StreamPool {
  std::vector<cudaStream_t> all, idle;
  cudaStream_t get();           // an idle stream, created on demand (non-blocking)
  void put(cudaStream_t s);     // back to the idle list (its work may still be in flight)
  ~StreamPool();                // synchronises and destroys every stream
};

struct Ctx {
  StreamPool streams;  // first member: destroyed after every buffer below
  int log_n = 0;
  size_t N = 0;
  int n_q = 0, n_p = 0, alpha = 1, hw = 0;
  double scale = 1;
  u64 seed = 0;
  cudaStream_t stream = nullptr;
  std::vector<u64> primes;
  std::vector<PrimeDev> pdev;
  DevBuf d_primes, d_psi2, d_ipsi2, d_ninv, d_ninv_sh;
  DevBuf d_moddown;   // level-independent ModDown constants
  DevBuf d_moddown2;  // fused ModDown: [N^-1 phinv_k, Shoup][K] pairs, c_k [K], phat_q Shoup [K][n_q], p_k [K]
  DevBuf d_mdr;       // ModDown scaled by P^-1 (fused with a rescale): p_k^-1 mod q_i [K][n_q], their Shoup
                      // companions [K][n_q], floor(P/2) P^-1 mod q_i [n_q]
  DevBuf d_r64;       // per prime: 2^64 mod q and its Shoup companion
  DevBuf d_pmod;      // per prime: P mod q_t (key generation)
  Tables tab{};
  std::vector<i64> sk;
  DevBuf d_sk;        // [n_q+n_p][N] NTT domain
  std::map<u64, DevBuf> keys;  // galois (0 = relinearisation; 2, 4 encapsulation) -> [dnum][2][n_q+n_p][N]
  // Limb t of key digit j, t outside the digit, is stored multiplied by key_scale[j][t]: the conversion
  // factor qhat_{i0} mod p_t of one digit limb i0 = key_scale_i0[j][t] (-1 and factor 1 where none is
  // folded), so that the ModUp conversion adds z_{i0} without a product (see ks_modup).  Exported keys
  // are multiplied back by key_unscale.  [dnum(L)][n_q + n_p] each; d_key_scale: (factor, Shoup) pairs.
  std::vector<u64> key_scale, key_unscale;
  std::vector<int> key_scale_i0;
  DevBuf d_key_scale;
  int enc_hw = 0;             // sparse-secret encapsulation of bootstrapping: weight of s~ (0 = off)
  DevBuf d_sk_sparse;         // s~, [n_q+n_p][N] NTT domain
  std::map<int, std::unique_ptr<LevelConsts>> lc;
  std::unique_ptr<BtsState, BtsStateDeleter> bts;
  int device = 0;             // the CUDA device current at creation
  cudaStream_t home = nullptr;  // the stream given at creation; `stream` is swapped while a server group steps
  u64* noalloc_scratch = nullptr;  // device address of hedap_rescale_noalloc's scratch array on `device`
  mutable std::mutex mu;      // held by every C-ABI call on this context and by a server's worker per step
  int L() const { return n_q - 1; }
  int total_primes() const { return n_q + n_p; }
  int dnum(int level) const { return (level + 1 + alpha - 1) / alpha; }
};

// ------------------------------------------------------------------ evaluator (evaluator.cu)
std::unique_ptr<Ct> ct_alloc(Ctx& C, int level, int batch = 1);
std::unique_ptr<Ct> ct_copy(Ctx& C, const Ct& a, int level);
std::unique_ptr<Ct> ev_add(Ctx& C, const Ct& a, const Ct& b, bool sub);
std::unique_ptr<Ct> ev_mul_relin(Ctx& C, const Ct& a, const Ct& b);
std::unique_ptr<Ct> ev_rescale(Ctx& C, const Ct& a);
std::unique_ptr<Ct> ev_mul(Ctx& C, const Ct& a, const Ct& b);
// Rotations of a by the Galois elements gs sharing one ModUp, each kept over Q_l u P before its ModDown:
// [batch][2][l + 1 + K][N] = (P sigma_g(c0) + ks0, ks1), NTT domain (double hoisting)
std::vector<DevBuf> ev_galois_hoisted_qp(Ctx& C, const Ct& a, const std::vector<u64>& gs);
// ModDown of such a pair batch (it is modified: its special limbs are transformed in place) into out
void ev_moddown_into(Ctx& C, DevBuf& acc, int batch, int level, Ct& out);
// rescale(lincomb({relin(a b) labelled prod_scale, prod_coef}, terms..., level min(a, b), target, c0)),
// with the key switch's ModDown fused into the rescale; residues equal the unfused sequence
std::unique_ptr<Ct> ev_mul_lincomb_rescale(Ctx& C, const Ct& a, const Ct& b, double prod_scale, double prod_coef,
                                           const std::vector<std::pair<const Ct*, double>>& terms, double target,
                                           double c0);
std::unique_ptr<Ct> ev_galois(Ctx& C, const Ct& a, u64 g);
std::vector<std::unique_ptr<Ct>> ev_galois_hoisted(Ctx& C, const Ct& a, const std::vector<u64>& gs);
std::unique_ptr<Ct> ev_drop(Ctx& C, const Ct& a, int level);
std::unique_ptr<Ct> ev_mul_const(Ctx& C, const Ct& a, double c, double target_scale);
std::unique_ptr<Ct> ev_mul_const_raw(Ctx& C, const Ct& a, double c, double target);
std::unique_ptr<Ct> ev_add_const_mul_int(Ctx& C, const Ct& a, double c, i64 m);
// sum_j c_j a_j + c0 at `level` (every a_j at level >= it), each product as ev_mul_const_raw would
// form it; the result is labelled target * q_level
std::unique_ptr<Ct> ev_lincomb_raw(Ctx& C, const std::vector<std::pair<const Ct*, double>>& terms, int level,
                                   double target, double c0);
std::unique_ptr<Ct> ev_add_const(Ctx& C, const Ct& a, double c);
std::unique_ptr<Ct> ev_mul_int(Ctx& C, const Ct& a, i64 m);
u64 galois_for_rotation(const Ctx& C, i64 steps);
// key switch of `batch` NTT-domain polynomials (limbs 0..level, ciphertext k's at d + k*d_stride):
// (ks0, ks1) of ciphertext k go to out + (2k)*out_stride and out + (2k+1)*out_stride,
// added to what is there when acc0 / acc1
void key_switch(Ctx& C, const u64* d, size_t d_stride, int batch, int level, u64 galois, u64* out, size_t out_stride,
                bool acc0, bool acc1);
std::unique_ptr<Ct> batch_pack(Ctx& C, const std::vector<const Ct*>& cts);
std::unique_ptr<Ct> batch_unpack(Ctx& C, const Ct& b, int k);
std::unique_ptr<Ct> batch_slice(Ctx& C, const Ct& b, int first, int count);  // members first .. first+count-1
void gen_galois_key(Ctx& C, u64 g);
// key ids of the sparse-secret encapsulation (even, so never a Galois element)
constexpr u64 kKeyToSparse = 2, kKeyToDense = 4;
void gen_switch_key(Ctx& C, u64 id, const u64* s_from, const u64* s_to);
void bts_encapsulate(Ctx& C, int h);
std::unique_ptr<Ct> ev_switch_key(Ctx& C, const Ct& a, u64 id);
const LevelConsts& level_consts(Ctx& C, int level);

// ------------------------------------------------------------------ context (context.cu)
Ctx* ctx_create(const hedap_params& p, u64 seed, cudaStream_t st);
std::unique_ptr<Ct> encrypt(Ctx& C, const std::vector<double>& re, const std::vector<double>& im, int level,
                            u64 seed);
void decrypt(Ctx& C, const Ct& ct, std::vector<double>& re, std::vector<double>& im);

std::vector<double> encode_slots(const Ctx& C, const std::vector<std::complex<double>>& z, double scale);

// ------------------------------------------------------------------ CryptoInvSqrt (invsqrt.cu)
std::unique_ptr<Ct> invsqrt(Ctx& C, const Ct& in, const hedap_invsqrt_cfg& cfg);
constexpr int kMaxBatchCts = 16;  // ciphertexts per batch (kernels.cuh's kMaxBatch)
// CryptoInvSqrt of single ciphertexts at their own levels, batched where their states meet (invsqrt.cu)
std::vector<std::unique_ptr<Ct>> invsqrt_mixed(Ctx& C, const std::vector<const Ct*>& in,
                                               const std::vector<hedap_invsqrt_cfg>& cfgs);
// CryptoInvSqrt in steps (construction = pre-BTS and pre-normalisation; then
// chebyshev(); then newton(i) for i = 0, 1, ...), used by invsqrt and the selector
struct InvSqrtRun {
  Ctx& C;
  hedap_invsqrt_cfg cfg;
  double lo, hi;
  i64 Y;
  std::unique_ptr<Ct> t, x, y;
  InvSqrtRun(Ctx& C, const Ct& in, const hedap_invsqrt_cfg& cfg);
  void chebyshev();
  void newton(int i);
  std::unique_ptr<Ct> result() const;  // y / sqrt(B)
};
// sum_j c_j T_j(t) at scale `target`; need < 0: the fewest-levels plan, else the fewest-products plan
// when it ends at level >= need (invsqrt.cu)
std::unique_ptr<Ct> cheb_eval(Ctx& C, const Ct& t, const std::vector<double>& coeffs, double target, int need);

// ------------------------------------------------------------------ selector (selector.cu)
int getoptiter_rule(const double* M, size_t n, double delta, double* thr_out);
int level_rule(const hedap_select_entry* D, size_t n, double theta, double target, hedap_select_entry* u1,
               hedap_select_entry* u2, hedap_select_entry* u3);
void select(Ctx& C, const hedap_select_cfg& sc, std::vector<hedap_select_entry>& D,
            std::vector<hedap_select_entry>& R, std::vector<hedap_select_trace>& trace);

// ------------------------------------------------------------------ bootstrapping (bootstrap.cu)
int bts_setup(Ctx& C, int K, int r, int deg, int cts, int stc);
std::unique_ptr<Ct> bootstrap_core(Ctx& C, const Ct& a, int log_slots = 0);
std::unique_ptr<Ct> bootstrap_scaled(Ctx& C, const Ct& y, i64 Y, int log_slots = 0);
std::unique_ptr<Ct> sub_sum(Ctx& C, const Ct& a, size_t n);
// equality of two CryptoInvSqrt configurations, field by field (the struct has padding)
inline bool same_cfg(const hedap_invsqrt_cfg& x, const hedap_invsqrt_cfg& y) {
  return x.lo == y.lo && x.hi == y.hi && x.B == y.B && x.degree == y.degree && x.newton_iters == y.newton_iters &&
         x.pre_bts == y.pre_bts && x.bts_mask == y.bts_mask && x.log_slots == y.log_slots;
}
std::unique_ptr<Ct> mod_raise(Ctx& C, const Ct& a);
std::unique_ptr<Ct> mul_monomial(Ctx& C, const Ct& a, u64 e);
std::unique_ptr<Ct> bts_linear_transform(Ctx& C, const Ct& a, bool inverse, int g, double target, size_t slots = 0);
std::unique_ptr<Ct> eval_mod(Ctx& C, const Ct& a);
bool bts_diagonal(Ctx& C, bool inverse, int g, long offset, std::vector<std::complex<double>>& out);

// thread-local message returned by hedap_last_error (capi.cu)
void set_last_error(const std::string& m);
// runs f under ctx's lock, turning exceptions into a status and the thread's last error (capi.cu)
hedap_status run_on_ctx(const hedap_ctx* ctx, const std::function<void()>& f);
// device address of hedap_rescale_noalloc's scratch array on `device` (the current device);
// looked up once per device (rescale_noalloc.cu)
u64* noalloc_scratch_address(int device);

// ------------------------------------------------------------------ launch helpers
inline int grid_for(size_t work, int threads) {
  size_t g = (work + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g ? g : 1);
}

}  // namespace hedap

// opaque ABI handles.  A live handle carries a magic word (cleared when it is freed) so that an entry
// point can refuse a pointer that is not a live handle of the right kind; a ciphertext also records
// the context it was made by (Ct::owner).
constexpr uint64_t kCtxMagic = 0x6865646170437478ull, kCtMagic = 0x6865646170437431ull;
struct hedap_ctx {
  uint64_t magic = kCtxMagic;
  hedap::Ctx* c = nullptr;
  explicit hedap_ctx(hedap::Ctx* cc) : c(cc) {}
  ~hedap_ctx() { magic = 0; }
};
struct hedap_ct {
  uint64_t magic = kCtMagic;
  std::unique_ptr<hedap::Ct> c;
  ~hedap_ct() { magic = 0; }
};
namespace hedap {
// the ciphertext behind a handle, after checking that it is a live ciphertext handle made by ctx (any
// context when ctx is null); HEDAP_ERR_ARG otherwise
Ct& ct_of(const hedap_ctx* ctx, const hedap_ct* h);
// the context behind a handle, after checking that it is a live context handle; HEDAP_ERR_ARG otherwise
Ctx& ctx_of(const hedap_ctx* ctx);
}  // namespace hedap
