// Launchers of the element-wise and key-switching kernels (kernels.cu).  A batch
// of B ciphertexts is 2B parts spaced by one part stride.
#pragma once
#include "internal.cuh"

namespace hedap {

constexpr int kMaxBatch = 16;  // ciphertexts per batched operation

// sets flag[0] (device word, not cleared here) when some residue is not below its prime
void k_check_residues(const Ctx& C, const u64* a, size_t as, int n_parts, int limbs, unsigned int* flag);
void k_lincomb(const Ctx& C, u64* out, size_t os, int n_parts, int limbs, const LinCombArgs& A);
void k_add_sub(const Ctx& C, const u64* a, size_t as, const u64* b, size_t bs, u64* o, size_t os, int n_parts,
               int limbs, bool sub);
void k_tensor(const Ctx& C, const u64* a, size_t as, const u64* b, size_t bs, u64* o, size_t os, u64* d2, int batch,
              int limbs);
void k_mul_limbconst(const Ctx& C, const u64* in, size_t is, u64* out, size_t os, int n_parts, int limbs,
                     const LimbConsts& K);
void k_add_limbconst(const Ctx& C, u64* io, size_t stride, int n_parts, int limbs, const LimbConsts& K);
void k_rescale_spread(const Ctx& C, const u64* last, size_t ls, u64* tmp, size_t ts, int n_parts, int l,
                      const RescaleConsts& R);
void k_rescale_finish(const Ctx& C, const u64* in, size_t is, const u64* tmp, size_t ts, u64* out, size_t os,
                      int n_parts, int l, const RescaleConsts& R);
void k_automorph(const Ctx& C, const u64* in, size_t is, u64* out, size_t os, int n_parts, int limbs, u64 g);
void k_modup(const Ctx& C, const u64* dcoef, u64* y, int batch, int level, const u64* d_consts);
// with c0 (part 0 of the input batch, member stride c0_stride): part 0 of acc also receives P sigma_g(c0) on
// the Q limbs, the rotated ciphertext over Q_l u P before its ModDown
void k_ksk_inner(const Ctx& C, const u64* y, const u64* d, size_t d_stride, const u64* key, u64* acc, int batch,
                 int level, u64 galois_perm = 0, const u64* c0 = nullptr, size_t c0_stride = 0);
// out [n_parts][ext][N] = (P x) on the Q limbs 0..level of in (part stride is), 0 on the special limbs
void k_lift_qp(const Ctx& C, const u64* in, size_t is, u64* out, int n_parts, int level);
void k_moddown_spread(const Ctx& C, const u64* acc, u64* v, int n_parts, int level);
// ModDown fused with a rescale (evaluator.cu, ks_moddown_rescale): limb l of the ModDown output, first
// t = e_l + acc_l P^-1 (NTT domain), then, with t back in the coefficient domain, x = t minus the
// conversion of the special limbs z into q_l scaled by P^-1 (canonical)
void k_mdr_last_eval(const Ctx& C, const u64* e, size_t es, const u64* acc, size_t as, u64* t, int n_parts, int l,
                     const MdrLast& M);
void k_mdr_last_coef(const Ctx& C, const u64* t, const u64* z, size_t zs, u64* x, int n_parts, int l,
                     const MdrLast& M);
void k_moddown_finish(const Ctx& C, const u64* acc, const u64* v, u64* out, size_t os, int n_parts, int level,
                      bool acc_even, bool acc_odd);
void k_keygen_combine(const Ctx& C, u64* b, const u64* a, const u64* s, const u64* sp, const u64* pmod, int lo,
                      int hi);
// x[t][n] *= f[2t] mod prime t (Shoup companion f[2t + 1]) for the limbs t < limbs, canonical
void k_scale_limbs(const Ctx& C, u64* x, int limbs, const u64* f);
void k_fma(const Ctx& C, const u64* x, const u64* y, const u64* z, u64* out, int limbs, int op);

}  // namespace hedap
