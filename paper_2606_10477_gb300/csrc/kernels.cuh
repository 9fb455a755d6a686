// Launchers of the element-wise and key-switching kernels (kernels.cu).
#pragma once
#include "internal.cuh"

namespace hedap {

void k_add_sub(const Ctx& C, const u64* a, size_t as, const u64* b, size_t bs, u64* o, size_t os, int limbs,
               bool sub);
void k_tensor(const Ctx& C, const u64* a0, const u64* a1, const u64* b0, const u64* b1, u64* d0, u64* d1, u64* d2,
              int limbs);
void k_mul_limbconst(const Ctx& C, const u64* in, size_t is, u64* out, size_t os, int n_parts, int limbs,
                     const LimbConsts& K);
void k_add_limbconst(const Ctx& C, u64* io, int limbs, const LimbConsts& K);
void k_rescale_spread(const Ctx& C, const u64* last, size_t ls, u64* tmp, size_t ts, int l, const RescaleConsts& R);
void k_rescale_finish(const Ctx& C, const u64* in, size_t is, const u64* tmp, size_t ts, u64* out, size_t os, int l,
                      const RescaleConsts& R);
void k_automorph(const Ctx& C, const u64* in, size_t is, u64* out, size_t os, int n_parts, int limbs, u64 g);
void k_modup(const Ctx& C, const u64* dcoef, u64* y, int level, const u64* d_consts);
void k_ksk_inner(const Ctx& C, const u64* y, const u64* key, u64* acc, int level);
void k_moddown_spread(const Ctx& C, const u64* acc, u64* v, int level);
void k_moddown_finish(const Ctx& C, const u64* acc, const u64* v, u64* out0, u64* out1, int level, bool acc0,
                      bool acc1);
void k_keygen_combine(const Ctx& C, u64* b, const u64* a, const u64* s, const u64* sp, const u64* pmod, int lo,
                      int hi);
void k_fma(const Ctx& C, const u64* x, const u64* y, const u64* z, u64* out, int limbs, int op);

}  // namespace hedap
