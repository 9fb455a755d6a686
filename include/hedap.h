/*
 * hedap.h -- C ABI of the GB300 RNS-CKKS library behind CryptoInvSqrt.
 *
 * The operations follow the paper's statement of the problem: keys owned by
 * the server (Sec. 4.2, "the server uses its own public and secret keys"),
 * Enc(values, l) at a chosen level (Alg. 3), CryptoInvSqrt(ct, d, n) with
 * pre-normalisation by B (Alg. 1, Sec. 2.3), Dec (Alg. 2), and the CKKS
 * operations Add/Sub/Mul_P/Mul_C, level management and rotation (Sec. 2.1).
 * The ring-level conventions (prime chain, NTT order, rounding, key
 * switching, sampling) are the textbook RNS-CKKS ones; the paper states none.
 *
 * Conventions for every entry point:
 *  - Every function returns hedap_status: 0 on success, a negative code on
 *    error; nothing throws across the ABI.  hedap_last_error() gives a
 *    message for the calling thread's most recent error.
 *  - Handles (hedap_ctx, hedap_ct) are created and freed by the library.
 *    A ciphertext handle owns device memory; hedap_ct_free releases it
 *    stream-ordered on the context's stream.
 *  - Host arrays passed in are owned by the caller and copied on entry;
 *    host arrays passed out are caller-allocated with the stated capacity.
 *    Arguments named `on_device` select whether a uint64_t* points to device
 *    memory (1, accessed on the context's stream) or host memory (0).
 *  - Ciphertext limb layout: [2][level+1][N] uint64_t, part-major (c0 then
 *    c1), limb i holding residues modulo q_i in the NTT (evaluation) domain;
 *    evaluation j sits at psi_i^(2*bitrev(j)+1), psi_i a primitive 2N-th root
 *    of unity modulo q_i.
 *  - A context is single-threaded: calls on one context must not overlap.
 *    All work is issued on the context's CUDA stream; functions that return
 *    host data synchronise that stream.
 */
#ifndef HEDAP_H
#define HEDAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HEDAP_OK = 0,
  HEDAP_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, bad index)   */
  HEDAP_ERR_LEVEL = -2,    /* not enough levels left for the requested operation     */
  HEDAP_ERR_SCALE = -3,    /* operands' scales differ                                */
  HEDAP_ERR_OOM = -4,      /* device allocation failed                               */
  HEDAP_ERR_CUDA = -5,     /* a CUDA runtime call failed                             */
  HEDAP_ERR_TIMEOUT = -6,  /* a bounded device wait ran out                          */
  HEDAP_ERR_RANGE = -7,    /* input values outside the configured interval           */
  HEDAP_ERR_KEY = -8,      /* a required switching key was not generated             */
  HEDAP_ERR_CANCELLED = -9 /* the query was withdrawn (hedap_server_cancel)          */
} hedap_status;

typedef struct hedap_ctx hedap_ctx;
typedef struct hedap_ct hedap_ct;

/* CKKS parameters.  Q primes are generated in the order given (q_0 first);
 * each is the first prime 2^b + k*2N + 1, then 2^b - k*2N + 1, k = 1, 2, ...,
 * not already used; the P (special) primes follow.  Bit sizes 33..60.
 * alpha = primes per key-switching digit (dnum = ceil(n_q / alpha)).
 * secret_hw = Hamming weight of the ternary secret (0 = dense uniform). */
typedef struct {
  uint32_t log_n;
  uint32_t n_q;
  const uint32_t* q_bits;
  uint32_t n_p;
  const uint32_t* p_bits;
  uint32_t alpha;
  double log_scale;
  uint32_t secret_hw;
} hedap_params;

/* CryptoInvSqrt configuration (Alg. 1 with the pre-normalisation of Sec. 2.3):
 * inputs a lie in [lo, hi]; a/B lies in (0, 1]; the initial value is the
 * degree-`degree` Chebyshev interpolant of 1/sqrt(x) on [lo/B, hi/B];
 * `newton_iters` Newton steps y <- y (3 - (a/B) y^2) / 2 follow; the output is
 * y / sqrt(B) (applied to the scale label).  pre_bts = 1 bootstraps a/B
 * before everything (the paper's Pre-BTS indicator c); bit j < 62 of bts_mask
 * bootstraps y before Newton step j (bit 0 = right after the Chebyshev step,
 * Alg. 1); bit 63 bootstraps y lazily whenever the next step would run out of
 * levels; bit 62 (a variant, not in Alg. 1) also bootstraps ct_x = 0.5 a/B
 * whenever y is bootstrapped and ct_x has fewer than 5 levels (a Newton output
 * sits two levels below ct_x).  All need hedap_bootstrap_setup on the
 * context.  log_slots = 0: the inputs use all N/2 slots; 1..log2(N/2): they
 * hold 2^log_slots values repeated over the N/2 slots (sparse packing) and
 * every bootstrap inside is the sparse-slot one (hedap_bootstrap_slots). */
typedef struct {
  double lo, hi, B;
  uint32_t degree;
  uint32_t newton_iters;
  uint32_t pre_bts;
  uint64_t bts_mask;
  uint32_t log_slots;
} hedap_invsqrt_cfg;

const char* hedap_status_str(hedap_status s);
const char* hedap_last_error(void);

/* Context: prime chain, NTT tables, secret key and relinearisation key,
 * generated from `seed` (SplitMix64 streams).  cuda_stream may be NULL (the
 * legacy default stream) or a cudaStream_t owned by the caller that outlives
 * the context. */
hedap_status hedap_ctx_create(const hedap_params* params, uint64_t seed, void* cuda_stream, hedap_ctx** out);
void hedap_ctx_destroy(hedap_ctx* ctx);
/* primes: n_q + n_p values (Q then P) into out[cap]. */
hedap_status hedap_ctx_primes(const hedap_ctx* ctx, uint64_t* out, size_t cap);
hedap_status hedap_sync(hedap_ctx* ctx);

/* Switching keys.  Galois element g (odd, < 2N); rotation by r slots uses
 * g = 5^r mod 2N, conjugation g = 2N - 1.  Keys are generated on first use;
 * these calls generate them ahead of time. */
hedap_status hedap_gen_galois_key(hedap_ctx* ctx, uint64_t galois);
/* The Galois element of a rotation by `steps` slots (Sec. 2.1's Rotate):
 * 5^(steps mod N/2) mod 2N; with conjugate != 0 the element of complex
 * conjugation, 2N - 1 (steps ignored).  Host only. */
hedap_status hedap_galois_element(const hedap_ctx* ctx, int64_t steps, int conjugate, uint64_t* out);
/* Export digit j of the key for g (g = 0: relinearisation key) into host
 * arrays b, a of [n_q + n_p][N] words each (NTT domain), as the key is defined
 * (Sec. 2.1's hybrid key switching).  The library stores limbs outside the
 * digit multiplied by one ModUp conversion factor (so that the fused ModUp
 * skips that product); the export divides it out on the host. */
hedap_status hedap_export_key(hedap_ctx* ctx, uint64_t galois, uint32_t digit, uint64_t* b, uint64_t* a);

/* Enc (symmetric, with the server's secret key): n_slots must be N/2. */
hedap_status hedap_encrypt(hedap_ctx* ctx, const double* re, const double* im, size_t n_slots, int level,
                           uint64_t seed, hedap_ct** out);
/* Dec + decode into re/im (im may be NULL); n_slots must be N/2. */
hedap_status hedap_decrypt(hedap_ctx* ctx, const hedap_ct* ct, double* re, double* im, size_t n_slots);

/* Import [2][level+1][N] NTT-domain words from host memory (on_device = 0: the
 * call returns once they are copied; they are checked on the device to lie
 * below their primes, HEDAP_ERR_RANGE otherwise; pinned host memory copies
 * fastest) or from device memory (on_device = 1, stream ordered, unchecked). */
hedap_status hedap_ct_import(hedap_ctx* ctx, const uint64_t* limbs, int level, double scale, int on_device,
                             hedap_ct** out);
/* Export [2][level+1][N] words into out (capacity cap words). */
hedap_status hedap_ct_export(hedap_ctx* ctx, const hedap_ct* ct, uint64_t* out, size_t cap, int on_device);
hedap_status hedap_ct_info(const hedap_ct* ct, int* level, double* scale);
void hedap_ct_free(hedap_ct* ct);

/* Sec. 2.1 operations.  Binary operations first bring both operands to the
 * lower level by dropping limbs.  Add/Sub require equal scales. */
hedap_status hedap_add(hedap_ctx* ctx, const hedap_ct* a, const hedap_ct* b, hedap_ct** out);
hedap_status hedap_sub(hedap_ctx* ctx, const hedap_ct* a, const hedap_ct* b, hedap_ct** out);
/* Mul_C: tensor product + relinearisation (hybrid key switching), no rescale. */
hedap_status hedap_mul_relin(hedap_ctx* ctx, const hedap_ct* a, const hedap_ct* b, hedap_ct** out);
/* Mul_C followed by rescale (one level consumed). */
hedap_status hedap_mul(hedap_ctx* ctx, const hedap_ct* a, const hedap_ct* b, hedap_ct** out);
/* Divide by the last prime q_l with rounding; scale /= q_l, level -= 1. */
hedap_status hedap_rescale(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out);
hedap_status hedap_rotate(hedap_ctx* ctx, const hedap_ct* a, int64_t steps, hedap_ct** out);
/* n rotations of one ciphertext (out[i] by steps[i]) sharing one ModUp of its
 * second part (hoisting, as in the bootstrapping baby steps): the extended
 * digits are formed once and each rotation permutes them by its automorphism
 * before the key inner product.  Each result decrypts like hedap_rotate's
 * (they differ by multiples of the digit moduli before ModDown).  out must
 * hold n handles; on error none is returned. */
hedap_status hedap_rotate_hoisted(hedap_ctx* ctx, const hedap_ct* a, const int64_t* steps, size_t n, hedap_ct** out);
hedap_status hedap_conjugate(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out);
/* Mul_P by a real constant c, rescaled so that the result has exactly
 * scale `target_scale` (the constant is encoded at target*q_l/scale). */
hedap_status hedap_mul_const(hedap_ctx* ctx, const hedap_ct* a, double c, double target_scale, hedap_ct** out);
/* Add_P of a real constant (encoded at the ciphertext's scale). */
hedap_status hedap_add_const(hedap_ctx* ctx, const hedap_ct* a, double c, hedap_ct** out);
/* Multiply by a small integer (no level consumed). */
hedap_status hedap_mul_int(hedap_ctx* ctx, const hedap_ct* a, int64_t m, hedap_ct** out);
hedap_status hedap_drop_level(hedap_ctx* ctx, const hedap_ct* a, int level, hedap_ct** out);

/* CryptoInvSqrt (Alg. 1). */
hedap_status hedap_invsqrt(hedap_ctx* ctx, const hedap_ct* in, const hedap_invsqrt_cfg* cfg, hedap_ct** out);

/* Batches (the paper has none; many ciphertexts through one launch sequence).
 * A batch handle holds up to 16 ciphertexts at one level and scale; every
 * operation above accepts batch handles (both operands with the same batch
 * size) and applies to each ciphertext, each kernel launch covering the whole
 * batch and each switching-key word read once per batch.  hedap_decrypt,
 * hedap_ct_export/import take single ciphertexts.
 * hedap_batch_pack copies n single or batch handles (same level and scale,
 * n <= 16 ciphertexts in total) into one batch; hedap_batch_unpack copies
 * ciphertext `index` out; hedap_ct_batch_size reports the count.
 * hedap_invsqrt_batch runs CryptoInvSqrt on n single ciphertexts with their
 * own configurations: inputs with equal level, scale and configuration are
 * packed (up to 16 per batch, in input order) and run together; out[i]
 * receives input i's result.  On error every out[i] is NULL. */
hedap_status hedap_batch_pack(hedap_ctx* ctx, const hedap_ct* const* cts, size_t n, hedap_ct** out);
/* A whole batch in one copy each way: hedap_batch_import reads n (1..16)
 * ciphertexts [n][2][level+1][N] (NTT domain) into one batch handle, with
 * hedap_ct_import's semantics (host: one residue check, returns once copied;
 * device: stream ordered, unchecked); hedap_batch_export writes a batch's
 * [n][2][level+1][N] words into out (capacity cap words; host: returns once
 * copied).  HEDAP_ERR_ARG for a bad size or capacity, HEDAP_ERR_RANGE for a
 * host word not below its prime. */
hedap_status hedap_batch_import(hedap_ctx* ctx, const uint64_t* limbs, size_t n, int level, double scale,
                                int on_device, hedap_ct** out);
hedap_status hedap_batch_export(hedap_ctx* ctx, const hedap_ct* batch, uint64_t* out, size_t cap, int on_device);
hedap_status hedap_batch_unpack(hedap_ctx* ctx, const hedap_ct* batch, size_t index, hedap_ct** out);
hedap_status hedap_ct_batch_size(const hedap_ct* ct, int* n);
hedap_status hedap_invsqrt_batch(hedap_ctx* ctx, const hedap_ct* const* in, const hedap_invsqrt_cfg* cfgs, size_t n,
                                 hedap_ct** out);
/* As hedap_invsqrt_batch, for inputs at mixed levels: with level_band = W > 0,
 * inputs with equal scale and configuration whose levels fall in the same band
 * [k W, (k+1) W) form one group (up to 16, input order) and are first dropped
 * to the lowest level present in it (dropping limbs costs no precision, only
 * levels: the configuration must be feasible at that level, as it is at each
 * input's own level).  level_band = 0 is hedap_invsqrt_batch. */
hedap_status hedap_invsqrt_many(hedap_ctx* ctx, const hedap_ct* const* in, const hedap_invsqrt_cfg* cfgs, size_t n,
                                int level_band, hedap_ct** out);

/* As hedap_invsqrt_batch, for single inputs each at its own level and with its
 * own configuration, none dropped to a lower level: inputs with equal level,
 * scale and configuration form a batch (input order, up to 16); after every
 * stage of CryptoInvSqrt (the pre-normalisation with its Pre-BTS, the
 * Chebyshev step, each Newton step) batches of one configuration whose carried
 * ciphertexts stand at equal levels and scales merge (up to 16).  Inputs at
 * different levels meet where Alg. 1 brings them to one level: after a Pre-BTS
 * (c = 1), every input is at the bootstrapped level.  out[i] equals
 * hedap_invsqrt of in[i] alone, bit for bit.  On error every out[i] is NULL. */
hedap_status hedap_invsqrt_mixed(hedap_ctx* ctx, const hedap_ct* const* in, const hedap_invsqrt_cfg* cfgs, size_t n,
                                 hedap_ct** out);

/* HE-DAP provisioning (Sec. 4.2): Alg. 2 GetOptIter and Alg. 3, run on this
 * library with CUDA-event costs.  For every profiled level l (l_BTS + 1 up to
 * the level of a bootstrapped ciphertext; l_BTS = 1 here) and degree
 * d = 2^d_e - 2, d_e_min <= d_e <= d_e_max, a ciphertext of
 * linspace(A, B_max, N/2) is encrypted at level l and CryptoInvSqrt (inputs
 * in [A, B_max], pre-normalisation by B, lazy BTS) runs for up to i_max
 * Newton steps with c = 0 (when l >= l_BTS + 3) and c = 1 (Pre-BTS; when
 * bootstrapping is configured and l < l_afterBTS - 1), decrypting after each
 * step: M[i] = MRE, T[i] = accumulated HE time (ms, Dec excluded; the Pre-BTS
 * included for c = 1).  Alg. 2's rule picks I per (l, d, c) -> a D entry;
 * Alg. 3's rule picks per level u1 (fastest with m <= (floor(alpha)+theta)
 * 10^l), u2 (fastest) and, if mre_target > 0, u3 (fastest with
 * m <= mre_target).  Ties: smaller t, smaller d, c = 0, smaller i.
 * Outputs: D entries (kind 0), R entries (kind 1, 2, 3 per level), and the
 * trace of every (l, d, c, i, M[i], T[i]); counts in *n_D, *n_R, *n_trace
 * (arrays may be NULL to query counts; HEDAP_ERR_ARG if a capacity is short). */
typedef struct {
  double A, B_max, B;
  uint32_t d_e_min, d_e_max;
  uint32_t i_max;
  double theta, delta;
  double mre_target;
  int32_t level_min, level_max; /* 0 = the full range */
  uint64_t seed;                /* encryption randomness of the provisioning ciphertexts */
} hedap_select_cfg;
typedef struct {
  int32_t level;
  uint32_t degree, c, iters;
  double mre, ms;
  uint32_t kind; /* 0: D entry, 1: u1 (theta rule), 2: u2 (fastest), 3: u3 (MRE target) */
} hedap_select_entry;
typedef struct {
  int32_t level;
  uint32_t degree, c, iter;
  double mre, ms;
} hedap_select_trace;
hedap_status hedap_select(hedap_ctx* ctx, const hedap_select_cfg* cfg, hedap_select_entry* D, size_t D_cap,
                          size_t* n_D, hedap_select_entry* R, size_t R_cap, size_t* n_R, hedap_select_trace* trace,
                          size_t trace_cap, size_t* n_trace);
/* The two selection rules alone (host only, no context needed).
 * hedap_getoptiter_rule: *I = smallest 0-based i with M[i] <= MRE_delta, or -1;
 * *threshold = MRE_delta.  hedap_select_level_rule: u1, u2, u3 of one level's
 * D entries; *has_u3 = 1 when some entry meets mre_target. */
hedap_status hedap_getoptiter_rule(const double* M, size_t n, double delta, int* I, double* threshold);
hedap_status hedap_select_level_rule(const hedap_select_entry* D, size_t n, double theta, double mre_target,
                                     hedap_select_entry* u1, hedap_select_entry* u2, hedap_select_entry* u3,
                                     int* has_u3);

/* Negacyclic NTT (inverse=0) or inverse NTT with N^-1 (inverse=1) of n_limbs
 * consecutive length-N limbs in place; limb i uses prime index first_prime+i
 * (global index over Q then P). */
hedap_status hedap_ntt(hedap_ctx* ctx, uint64_t* limbs, size_t n_limbs, uint32_t first_prime, int inverse,
                       int on_device);
/* The same over n_polys consecutive polynomials of n_limbs limbs each (limb i
 * of every polynomial uses prime first_prime+i), in one launch per phase. */
hedap_status hedap_ntt_batch(hedap_ctx* ctx, uint64_t* limbs, size_t n_limbs, size_t n_polys, uint32_t first_prime,
                             int inverse, int on_device);

/* Bootstrapping (BTS, Sec. 2.1; the paper uses it as a library primitive).
 * Full-slot CKKS bootstrapping: ModRaise, CoeffToSlot (cts_levels grouped
 * special-FFT factors, baby-step/giant-step diagonals), EvalMod (Chebyshev
 * interpolant of degree mod_degree of cos(2 pi (K u - 1/4) / 2^double_angles)
 * then double_angles squarings), SlotToCoeff (stc_levels groups).  The top
 * cts_levels primes are consumed by CoeffToSlot, the next ones by EvalMod and
 * SlotToCoeff; *level_after receives the level of a bootstrapped ciphertext
 * (l_afterBTS).  K must exceed the ModRaise overflow |I| (about 7 sigma of a
 * sum of secret_hw uniform terms; 28 suits secret_hw = 192).
 * hedap_bootstrap: input at level 0 with values in [-1, 1] and scale at most
 * q_0 / 2^10; output at level_after with the context scale.
 * hedap_bootstrap_scaled: input at level >= 1 with values in [-Y, Y]; it is
 * scaled into [-1, 1] (one level, landing at scale q_0 / 2^12), bootstrapped
 * and multiplied back by the integer Y (l_BTS = 1). */
typedef struct {
  uint32_t K;
  uint32_t double_angles;
  uint32_t mod_degree;
  uint32_t cts_levels;
  uint32_t stc_levels;
} hedap_bts_params;
hedap_status hedap_bootstrap_setup(hedap_ctx* ctx, const hedap_bts_params* p, int* level_after);
/* Sparse-secret encapsulation (Bossuat, Troncoso-Pastoriza, Hubaux 2022), for
 * bootstrapping under a dense ternary secret (secret_hw = 0) with the small K
 * of a sparse one: draws an ephemeral ternary secret s~ of exactly h non-zero
 * coefficients from the context's seed and generates the switching keys s -> s~
 * and s~ -> s.  Every later bootstrap switches its level-0 input to s~, raises
 * it, and switches the raised ciphertext back to s (two key switches more; the
 * ModRaise overflow is then that of weight h).  HEDAP_ERR_ARG unless 1 <= h <= N.
 * hedap_encapsulation_switch: one of the two key switches alone (to_sparse = 1:
 * s -> s~, else s~ -> s), for parity tests; HEDAP_ERR_ARG before
 * hedap_bootstrap_encapsulate. */
hedap_status hedap_bootstrap_encapsulate(hedap_ctx* ctx, uint32_t h);
hedap_status hedap_encapsulation_switch(hedap_ctx* ctx, const hedap_ct* a, int to_sparse, hedap_ct** out);
hedap_status hedap_bootstrap(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out);
/* Sparse-slot bootstrapping: the input holds n = 2^log_slots values repeated
 * over the N/2 slots (its plaintext is a polynomial in X^(N/2n)).  After
 * ModRaise, the rotations by n, 2n, ..., N/4 are added (hedap_sub_sum; the
 * overflow q_0 I is projected onto that subring, times N/2n), then CoeffToSlot
 * and SlotToCoeff run on n slots (the transforms of the ring of dimension 2n,
 * diagonals repeated): log2(N/2n) rotations more, fewer diagonals.  Same levels
 * and output level as hedap_bootstrap; log_slots = log2(N/2) is the full-slot
 * bootstrap; HEDAP_ERR_ARG when log_slots is below cts_levels or stc_levels or
 * above log2(N/2).  hedap_bootstrap_scaled_slots is hedap_bootstrap_scaled with
 * it.  hedap_sub_sum: that sum of rotations alone, for parity tests. */
hedap_status hedap_bootstrap_slots(hedap_ctx* ctx, const hedap_ct* a, uint32_t log_slots, hedap_ct** out);
hedap_status hedap_bootstrap_scaled_slots(hedap_ctx* ctx, const hedap_ct* a, int64_t Y, uint32_t log_slots,
                                          hedap_ct** out);
hedap_status hedap_sub_sum(hedap_ctx* ctx, const hedap_ct* a, uint32_t log_slots, hedap_ct** out);
hedap_status hedap_bootstrap_scaled(hedap_ctx* ctx, const hedap_ct* a, int64_t Y, hedap_ct** out);
/* Single steps of bootstrapping, for parity tests.  hedap_mod_raise: level-0
 * input -> top level (centred lift).  hedap_mul_monomial: times X^e for
 * e in {N/2 (= i in every slot), 3N/2 (= -i)}.  hedap_bts_linear_transform:
 * group `group` of CoeffToSlot (inverse = 1) or SlotToCoeff (inverse = 0),
 * rescaled to target_scale.  hedap_eval_mod: the EvalMod polynomial and double
 * angles.  hedap_set_scale relabels a ciphertext's scale in place. */
hedap_status hedap_mod_raise(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out);
hedap_status hedap_mul_monomial(hedap_ctx* ctx, const hedap_ct* a, uint64_t e, hedap_ct** out);
hedap_status hedap_bts_linear_transform(hedap_ctx* ctx, const hedap_ct* a, int inverse, int group,
                                        double target_scale, hedap_ct** out);
hedap_status hedap_eval_mod(hedap_ctx* ctx, const hedap_ct* a, hedap_ct** out);
hedap_status hedap_set_scale(hedap_ctx* ctx, hedap_ct* a, double scale);
/* Host-side helpers for parity tests.  hedap_encode: the canonical-embedding
 * encoding of N/2 slots at `scale`, out[N] integer coefficients (|c| < 2^63).
 * hedap_bts_diagonal: diagonal `offset` (rotation offset mod N/2) of group
 * `group` of CoeffToSlot (inverse = 1) or SlotToCoeff (inverse = 0), N/2
 * complex values into re/im; HEDAP_ERR_ARG when that offset is absent. */
hedap_status hedap_encode(hedap_ctx* ctx, const double* re, const double* im, size_t n_slots, double scale,
                          int64_t* out);
hedap_status hedap_bts_diagonal(hedap_ctx* ctx, int inverse, int group, int64_t offset, double* re, double* im);

/* Steps of hybrid key switching, for parity tests (host arrays, [limb][N]).
 * hedap_modup: coefficient-domain input over q_0..q_level -> for every digit j
 *   (alpha consecutive primes) the fast basis conversion onto Q_level u P,
 *   out [dnum][level+1+n_p][N] coefficient domain (digit j's own limbs copy the input).
 * hedap_moddown: two coefficient-domain polynomials over Q_level u P,
 *   in [2][level+1+n_p][N] -> round(x / P) up to the conversion slack, out [2][level+1][N].
 * hedap_key_switch: NTT-domain d over q_0..q_level and the key for `galois`
 *   (0 = relinearisation) -> (ks0, ks1), out [2][level+1][N] NTT domain. */
hedap_status hedap_modup(hedap_ctx* ctx, const uint64_t* in, int level, uint64_t* out);
hedap_status hedap_moddown(hedap_ctx* ctx, const uint64_t* in, int level, uint64_t* out);
hedap_status hedap_key_switch(hedap_ctx* ctx, const uint64_t* d, int level, uint64_t galois, uint64_t* out);

/* Rescale without device allocation.  No counterpart in the paper: this entry
 * point exists for callers that cannot allocate device memory during an
 * operation -- a serving loop that admitted its requests against a fixed HBM
 * budget, a host framework whose allocator owns the device memory, or code
 * that must not let a cudaMalloc/cudaFree synchronise the device.
 * in:  device pointer, [2][level+1][N] words (NTT domain, as hedap_ct_export).
 * out: device pointer, [2][level][N] words; must not overlap `in`
 *      (HEDAP_ERR_ARG when the two ranges overlap).
 * Same result as hedap_rescale (scale divided by q_level is the caller's to
 * track).  Work is issued on the context's stream; the call returns without
 * synchronising.  The context's device must be the current device
 * (HEDAP_ERR_ARG otherwise).  Scratch is one library-wide device array of
 * 4 Mi words (32 MiB) per device, allocated when the first context is created
 * on that device (context creation looks up its address) and held until the
 * process exits; (2 + 2*level) * N must not exceed 4 Mi words (level <= 31 at
 * N = 2^16), otherwise HEDAP_ERR_ARG.  All calls share the array: calls whose
 * work overlaps on the GPU (other streams, other threads, other contexts on the
 * same device) race on it.  The call runs under the context's lock like every
 * other entry point, and calls no cudaMalloc, cudaFree or allocating routine
 * (with profiling off, the default). */
hedap_status hedap_rescale_noalloc(hedap_ctx* ctx, const uint64_t* in, int level, uint64_t* out);

/* Serving (the statistical workloads of Sec. 5.3: Z-score normalisation and
 * the Pearson correlation coefficient, each needing InvSqrt of an encrypted
 * variance).  A server owns a worker thread that drives the context: the
 * oldest waiting query is admitted with the later ones that can share its
 * group (one kind, input level, input scale and InvSqrt configuration; up to
 * max_batch) while the estimated device memory of the admitted queries stays
 * within hbm_budget_bytes.  Each group runs on a CUDA stream of its own, one
 * batched step at a time (statistics, pre-normalisation, Chebyshev, each
 * Newton step, the final product), the next step issued when the previous one
 * has finished on the device, so the groups in flight overlap on the GPU.  At
 * each step boundary, groups with the same signature at the same step merge
 * into one batch (up to max_batch); a group waits up to 3 steps for a later
 * one with its signature to catch up.  A query's result is bit for bit the
 * same whatever other queries share its group.
 *   z-score: x = n_ct ciphertexts holding the records in their slots (unused
 *     slots zero); result: n_ct ciphertexts z = (x - mean) * InvSqrt(var).
 *   PCC: x and y as above, record k of x paired with record k of y;
 *     result: one ciphertext with r = cov * InvSqrt(var_x * var_y) in every slot.
 * mean, var and cov are over n_records records (population moments).  All
 * inputs are single ciphertexts at one level >= 4 and one scale, and are
 * BORROWED: the caller keeps them alive and unchanged until the query is
 * done.  The InvSqrt configuration must cover the variance (z-score) or the
 * product of variances (PCC); a lazy-bootstrap mask (bit 63) needs
 * hedap_bootstrap_setup on the context, and when InvSqrt leaves the result at
 * level 0 the server bootstraps it once more for the final product.
 * hedap_server_create generates the rotation keys by 1, 2, 4, .., N/4 (kept
 * resident) and starts the worker; max_batch in [1, 16]; with start_paused
 * the worker admits nothing until hedap_server_resume (a burst submitted
 * meanwhile is grouped in arrival order).  While a server runs,
 * other calls on its context are serialised with the worker's steps.
 * hedap_server_submit returns HEDAP_ERR_OOM for a query whose own estimate
 * exceeds the budget.  hedap_server_poll: *done = 1 once finished (wait != 0
 * blocks until then); with out != NULL it hands over the result ciphertexts
 * (caller frees them with hedap_ct_free) and forgets the query; a failed query
 * reports its error once and is forgotten; *group_size = the number of queries
 * the query was grouped with (itself included).  hedap_server_estimate: the
 * admission estimate in bytes for a query of that kind, n_ct and input level.  hedap_server_stats: completion
 * latency percentiles (submit to GPU completion, ms) over all completed
 * queries and queries per second from the first submission to the last
 * completion.  hedap_server_destroy finishes every submitted query first. */
typedef struct hedap_server hedap_server;
enum { HEDAP_QUERY_ZSCORE = 1, HEDAP_QUERY_PCC = 2 };
typedef struct {
  uint32_t max_batch;        /* queries in one group, after merges too: [1, 16] */
  uint32_t start_paused;
  uint64_t hbm_budget_bytes;
  uint32_t admit_max;        /* queries admitted into one new group (0: max_batch); merges grow it later */
} hedap_server_cfg;
typedef struct {
  uint32_t kind;                 /* HEDAP_QUERY_ZSCORE or HEDAP_QUERY_PCC */
  const hedap_ct* const* x;      /* n_ct ciphertexts */
  const hedap_ct* const* y;      /* n_ct ciphertexts (PCC), else NULL */
  uint32_t n_ct;
  uint64_t n_records;            /* <= n_ct * N/2 */
  hedap_invsqrt_cfg invsqrt;
  uint32_t choice;               /* 0: invsqrt as given; 1/2/3: (degree, c, iters) from the server's
                                    HE-DAP table, entry u1/u2/u3 (see hedap_server_set_table) */
} hedap_query;
hedap_status hedap_server_create(hedap_ctx* ctx, const hedap_server_cfg* cfg, hedap_server** out);
hedap_status hedap_server_submit(hedap_server* s, const hedap_query* q, uint64_t* id);
hedap_status hedap_server_poll(hedap_server* s, uint64_t id, int wait, int* done, hedap_ct** out, size_t cap,
                               size_t* n_out, double* latency_ms, uint32_t* group_size);
hedap_status hedap_server_resume(hedap_server* s);
/* Failure handling on the host (none of it touches the GPU).
 * hedap_server_wait: blocks until query `id` is done or timeout_ms passes
 *   (HEDAP_ERR_TIMEOUT; the query goes on); the result is then taken with
 *   hedap_server_poll.
 * hedap_server_cancel: withdraws a query that is not done: a waiting one at
 *   once, one in flight at its group's next step boundary (a group whose every
 *   query is withdrawn is dropped; otherwise the others finish unchanged).  Its
 *   poll then reports HEDAP_ERR_CANCELLED; HEDAP_ERR_ARG for an unknown or
 *   finished query.
 * hedap_server_inject: fault injection; HEDAP_FAULT_ADMISSION_OOM makes the
 *   next `count` admitted groups fail as a device allocation failure at
 *   admission would: their queries end with HEDAP_ERR_OOM, their memory budget
 *   is released and the server goes on with the others.
 * hedap_server_merges: how many groups have been merged into others. */
enum { HEDAP_FAULT_ADMISSION_OOM = 1 };
hedap_status hedap_server_wait(hedap_server* s, uint64_t id, double timeout_ms);
hedap_status hedap_server_cancel(hedap_server* s, uint64_t id);
hedap_status hedap_server_inject(hedap_server* s, uint32_t fault, uint32_t count);
hedap_status hedap_server_merges(hedap_server* s, uint64_t* merged);
/* HE-DAP in serving: install the per-level table R of hedap_select (entries of
 * kind 1, 2, 3 = u1 accuracy, u2 speed, u3 absolute MRE target; copied).  A
 * query with choice k takes (degree, Pre-BTS c, Newton steps) from the kind-k
 * entry at the level its variance reaches InvSqrt (input level - 2 for z-score,
 * - 3 for PCC) or, when that level has none, at the highest tabled level below
 * it (a configuration that fits a level fits every higher one); lo, hi, B come
 * from the query's invsqrt, and bootstrapping in the Newton loop is lazy (bit
 * 63) on a context set up for it.  No such entry: HEDAP_ERR_ARG at submit. */
hedap_status hedap_server_set_table(hedap_server* s, const hedap_select_entry* R, size_t n);
hedap_status hedap_server_estimate(const hedap_server* s, uint32_t kind, uint32_t n_ct, int level, uint64_t* bytes);
hedap_status hedap_server_stats(hedap_server* s, double* p50_ms, double* p99_ms, double* qps, uint64_t* completed);
void hedap_server_destroy(hedap_server* s);

/* CryptoInvSqrt as a CUDA graph (no counterpart in the paper: a launch-overhead
 * optimisation).  hedap_invsqrt_graph_create runs InvSqrt once on a copy of
 * `example` (building every table the sequence needs) and captures the launch
 * sequence for that input level, batch and scale and that configuration; the
 * graph owns its input and output buffers.  Profiling must be off.
 * hedap_graph_run: copies `in` (if not NULL; same level, batch and scale as the
 * example, else HEDAP_ERR_ARG) into the graph's input, replays the graph on the
 * context's stream, and (if out is not NULL) returns a new ciphertext holding the
 * result, the same as hedap_invsqrt bit for bit.  Calls on the graph serialise
 * with other calls on its context.  hedap_graph_kernels: kernels one replay
 * launches.  Destroy the graph before its context. */
typedef struct hedap_graph hedap_graph;
hedap_status hedap_invsqrt_graph_create(hedap_ctx* ctx, const hedap_ct* example, const hedap_invsqrt_cfg* cfg,
                                        hedap_graph** out);
hedap_status hedap_graph_run(hedap_graph* g, const hedap_ct* in, hedap_ct** out);
/* hedap_invsqrt_mixed as one CUDA graph: captured for the examples' levels and
 * scales (n single ciphertexts) and configurations; the graph owns n input and
 * n output buffers.  hedap_graph_run_many copies in[0..n) (if in is not NULL;
 * each with its example's level and scale, else HEDAP_ERR_ARG) into the inputs,
 * replays, and (if out is not NULL) returns n new ciphertexts, equal bit for
 * bit to hedap_invsqrt_mixed's.  hedap_graph_run refuses such a graph and
 * hedap_graph_run_many a graph of one input. */
hedap_status hedap_invsqrt_mixed_graph_create(hedap_ctx* ctx, const hedap_ct* const* examples,
                                              const hedap_invsqrt_cfg* cfgs, size_t n, hedap_graph** out);
hedap_status hedap_graph_run_many(hedap_graph* g, const hedap_ct* const* in, size_t n, hedap_ct** out);
hedap_status hedap_graph_kernels(const hedap_graph* g, uint64_t* n);
void hedap_graph_destroy(hedap_graph* g);

/* NTT autotuner: times every NTT launch shape (words staged per CTA, CTAs per
 * SM, radix 16 or 8 register passes) on `limbs` limbs of scratch, forward and inverse separately (best of
 * `reps`), and makes the fastest the context's shape.  Per-variant times go
 * to fwd_ms / inv_ms (capacity cap, may be NULL); the chosen variant indices
 * to *fwd_variant / *inv_variant.  The forward transforms with a fused key-switch
 * conversion (HEDAP_NTT_ROLE_MODUP) or a fused ModDown / rescale
 * (HEDAP_NTT_ROLE_FINISH) are then tuned apart, each on an HMult with rescale of a
 * batch of 4 ciphertexts at the top level (when the relinearisation key exists);
 * hedap_ntt_get_role_variant reports their choices. */
hedap_status hedap_ntt_tune(hedap_ctx* ctx, int limbs, int reps, float* fwd_ms, float* inv_ms, int cap,
                            int* fwd_variant, int* inv_variant);
/* Butterflies per second of a register-only loop of the NTT's butterfly (no
 * memory traffic): the rate the integer pipes allow this butterfly, beside
 * which the transforms' rate is read.  Synchronises. */
hedap_status hedap_butterfly_rate(hedap_ctx* ctx, double* per_s);
/* Select NTT launch shapes directly (0 <= variant < 8); every shape computes
 * the same transform.  Context creation runs the autotuner once.
 * hedap_ntt_set_variant gives every forward role fwd_variant and the inverse
 * inv_variant; hedap_ntt_get_variant reports the plain forward and inverse shapes.
 * The per-role calls read or set one role (to persist the autotuner's choice or
 * to run one fused kernel in a given shape); HEDAP_ERR_ARG for an unknown role
 * or a variant out of range. */
#define HEDAP_NTT_ROLE_FORWARD 0 /* plain forward transform */
#define HEDAP_NTT_ROLE_INVERSE 1 /* inverse transform */
#define HEDAP_NTT_ROLE_MODUP 2   /* forward with the ModUp conversion fused into its load */
#define HEDAP_NTT_ROLE_FINISH 3  /* forward with a fused ModDown / rescale (load and store) */
#define HEDAP_NTT_ROLES 4
hedap_status hedap_ntt_set_variant(hedap_ctx* ctx, int fwd_variant, int inv_variant);
hedap_status hedap_ntt_get_variant(const hedap_ctx* ctx, int* fwd_variant, int* inv_variant);
hedap_status hedap_ntt_set_role_variant(hedap_ctx* ctx, int role, int variant);
hedap_status hedap_ntt_get_role_variant(const hedap_ctx* ctx, int role, int* variant);

/* Profiling (process-wide, not part of the paper's interface).
 * hedap_profile_enable(1) resets the counters and, until disabled, records a
 * CUDA event pair around every launch group of these kernel classes:
 * "ntt" (one forward or inverse transform of a limb batch: two launches),
 * "modup", "ksk_inner", "moddown", "tensor", "rescale", "automorph",
 * "elementwise".  hedap_profile_read synchronises and returns, for one class,
 * the number of timed groups, their summed event time in ms, and their summed
 * algorithmic bytes (each input word read once, each output word written once).
 * hedap_launch_count returns the number of kernels this library has launched
 * since it was loaded (profiling on or off). */
hedap_status hedap_profile_enable(int on);
hedap_status hedap_profile_read(const char* kernel_class, uint64_t* groups, double* ms, double* bytes);
/* The class's algorithmic multiply work over the same groups, in 32-bit
 * multiply-pipe slots (kept for "ntt": 16 per Shoup product by a constant --
 * every butterfly and every term of a fused basis conversion -- and 8 per
 * 64 x 64 -> 128-bit product of the fused key inner product). */
hedap_status hedap_profile_read_slots(const char* kernel_class, double* slots);
hedap_status hedap_launch_count(uint64_t* out);

#ifdef __cplusplus
}
#endif
#endif /* HEDAP_H */
