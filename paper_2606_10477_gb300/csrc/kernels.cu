// Element-wise RNS kernels, rescale, automorphism and the hybrid key-switching
// steps (ModUp basis conversion, key inner product, ModDown), all batched.
//
// Arrays are limb-major: limb i of a part is N consecutive words.  A batch of B
// ciphertexts is 2B parts with one part stride (ciphertext k owns parts 2k, 2k+1).
// Element kernels walk the flattened (part, limb, coefficient) space two
// coefficients at a time with 128-bit loads and stores.
#include <algorithm>

#include "internal.cuh"
#include "kernels.cuh"
#include "profiler.cuh"

namespace hedap {

__device__ __forceinline__ ulonglong2 ld2(const u64* p) { return *reinterpret_cast<const ulonglong2*>(p); }
__device__ __forceinline__ void st2(u64* p, ulonglong2 v) { *reinterpret_cast<ulonglong2*>(p) = v; }

#define GRID_LOOP(var, total) \
  for (size_t var = blockIdx.x * (size_t)blockDim.x + threadIdx.x; var < (total); var += (size_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- add / sub
__global__ void k_add_sub_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ a, size_t as,
                                 const u64* __restrict__ b, size_t bs, u64* __restrict__ o, size_t os, int n_parts,
                                 int limbs, int log_n, int sub) {
  const size_t per_part = (size_t)limbs << log_n;
  GRID_LOOP(t, n_parts * per_part / 2) {
    const size_t e = 2 * t;
    const size_t p = e / per_part, r = e - p * per_part;
    const u64 q = pr[r >> log_n].q;
    ulonglong2 x = ld2(a + p * as + r), y = ld2(b + p * bs + r), z;
    z.x = sub ? sub_mod(x.x, y.x, q) : add_mod(x.x, y.x, q);
    z.y = sub ? sub_mod(x.y, y.y, q) : add_mod(x.y, y.y, q);
    st2(o + p * os + r, z);
  }
}
void k_add_sub(const Ctx& C, const u64* a, size_t as, const u64* b, size_t bs, u64* o, size_t os, int n_parts,
               int limbs, bool sub) {
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, 3.0 * n_parts * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * limbs * C.N / 2;
  k_add_sub_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, a, as, b, bs, o, os, n_parts, limbs,
                                                              C.log_n, sub);
  HEDAP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- residue range check
// flag[0] |= 1 when some word of the n_parts x limbs limbs at a (part stride as) is not below its prime
__global__ void k_check_residues_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ a, size_t as,
                                        int n_parts, int limbs, int log_n, unsigned int* flag) {
  const size_t per_part = (size_t)limbs << log_n;
  bool bad = false;
  GRID_LOOP(t, n_parts * per_part / 2) {
    const size_t e = 2 * t;
    const size_t p = e / per_part, r = e - p * per_part;
    const u64 q = pr[r >> log_n].q;
    const ulonglong2 x = ld2(a + p * as + r);
    bad |= x.x >= q || x.y >= q;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}
void k_check_residues(const Ctx& C, const u64* a, size_t as, int n_parts, int limbs, unsigned int* flag) {
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, 1.0 * n_parts * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * limbs * C.N / 2;
  k_check_residues_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, a, as, n_parts, limbs, C.log_n, flag);
  HEDAP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- tensor product
// ciphertext k: (a_2k, a_2k+1) x (b_2k, b_2k+1) -> d0 = o_2k, d1 = o_2k+1, d2 at d2 + k*limbs*N
__global__ void k_tensor_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ a, size_t as,
                                const u64* __restrict__ b, size_t bs, u64* __restrict__ o, size_t os,
                                u64* __restrict__ d2, int batch, int limbs, int log_n) {
  const size_t per = (size_t)limbs << log_n;
  GRID_LOOP(t, batch * per / 2) {
    const size_t e = 2 * t;
    const size_t k = e / per, r = e - k * per;
    const PrimeDev P = pr[r >> log_n];
    const ulonglong2 x0 = ld2(a + 2 * k * as + r), x1 = ld2(a + (2 * k + 1) * as + r);
    const ulonglong2 y0 = ld2(b + 2 * k * bs + r), y1 = ld2(b + (2 * k + 1) * bs + r);
    ulonglong2 r0, r1, r2;
    r0.x = mul_mod(x0.x, y0.x, P);
    r0.y = mul_mod(x0.y, y0.y, P);
    r1.x = add_mod(mul_mod(x0.x, y1.x, P), mul_mod(x1.x, y0.x, P), P.q);
    r1.y = add_mod(mul_mod(x0.y, y1.y, P), mul_mod(x1.y, y0.y, P), P.q);
    r2.x = mul_mod(x1.x, y1.x, P);
    r2.y = mul_mod(x1.y, y1.y, P);
    st2(o + 2 * k * os + r, r0);
    st2(o + (2 * k + 1) * os + r, r1);
    st2(d2 + k * per + r, r2);
  }
}
void k_tensor(const Ctx& C, const u64* a, size_t as, const u64* b, size_t bs, u64* o, size_t os, u64* d2, int batch,
              int limbs) {
  ProfScope prof_(PROF_TENSOR, C.stream, 7.0 * batch * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)batch * limbs * C.N / 2;
  k_tensor_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, a, as, b, bs, o, os, d2, batch, limbs,
                                                             C.log_n);
  HEDAP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- per-limb constants
__global__ void k_mul_limbconst_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ in, size_t is,
                                       u64* __restrict__ out, size_t os, int n_parts, int limbs, int log_n,
                                       LimbConsts K) {
  const size_t per_part = (size_t)limbs << log_n;
  GRID_LOOP(t, n_parts * per_part / 2) {
    const size_t e = 2 * t;
    const size_t p = e / per_part, r = e - p * per_part;
    const int i = (int)(r >> log_n);
    const u64 q = pr[i].q, w = K.w[i], wp = K.wsh[i];
    ulonglong2 x = ld2(in + p * is + r);
    x.x = shoup_mul(x.x, w, wp, q);
    x.y = shoup_mul(x.y, w, wp, q);
    st2(out + p * os + r, x);
  }
}
void k_mul_limbconst(const Ctx& C, const u64* in, size_t is, u64* out, size_t os, int n_parts, int limbs,
                     const LimbConsts& K) {
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, 2.0 * n_parts * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * limbs * C.N / 2;
  k_mul_limbconst_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, in, is, out, os, n_parts, limbs,
                                                                   C.log_n, K);
  HEDAP_LAUNCH_CHECK();
}

// out = sum_j in_j * w_j (+ c0 on the even parts, the c0 of each batch member) over limbs 0..limbs-1:
// the leaf sum of a Chebyshev evaluation in one pass (inputs read at their own part strides, so
// ciphertexts above the output level are read without a copy)
__global__ void k_lincomb_kernel(const PrimeDev* __restrict__ pr, u64* __restrict__ out, size_t os, int n_parts,
                                 int limbs, int log_n, LinCombArgs A) {
  const size_t per_part = (size_t)limbs << log_n;
  GRID_LOOP(t, n_parts * per_part / 2) {
    const size_t e = 2 * t;
    const size_t p = e / per_part, r = e - p * per_part;
    const int i = (int)(r >> log_n);
    const u64 q = pr[i].q;
    ulonglong2 s = A.accumulate ? ld2(out + p * os + r) : ulonglong2{0, 0};
    for (int j = 0; j < A.count; ++j) {
      const ulonglong2 x = ld2(A.in[j] + p * A.stride[j] + r);
      s.x = add_mod(s.x, shoup_mul(x.x, A.w[j][i], A.wsh[j][i], q), q);
      s.y = add_mod(s.y, shoup_mul(x.y, A.w[j][i], A.wsh[j][i], q), q);
    }
    if (A.add_c0 && !(p & 1)) {
      s.x = add_mod(s.x, A.c0[i], q);
      s.y = add_mod(s.y, A.c0[i], q);
    }
    st2(out + p * os + r, s);
  }
}
void k_lincomb(const Ctx& C, u64* out, size_t os, int n_parts, int limbs, const LinCombArgs& A) {
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, (A.count + 1.0 + A.accumulate) * n_parts * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * limbs * C.N / 2;
  k_lincomb_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, out, os, n_parts, limbs, C.log_n, A);
  HEDAP_LAUNCH_CHECK();
}

// add a per-limb constant to n_parts parts spaced `stride` apart (the c0 parts of a batch)
__global__ void k_add_limbconst_kernel(const PrimeDev* __restrict__ pr, u64* __restrict__ io, size_t stride,
                                       int n_parts, int limbs, int log_n, LimbConsts K) {
  const size_t per_part = (size_t)limbs << log_n;
  GRID_LOOP(t, n_parts * per_part / 2) {
    const size_t e = 2 * t;
    const size_t p = e / per_part, r = e - p * per_part;
    const int i = (int)(r >> log_n);
    const u64 q = pr[i].q, w = K.w[i];
    u64* at = io + p * stride + r;
    ulonglong2 x = ld2(at);
    x.x = add_mod(x.x, w, q);
    x.y = add_mod(x.y, w, q);
    st2(at, x);
  }
}
void k_add_limbconst(const Ctx& C, u64* io, size_t stride, int n_parts, int limbs, const LimbConsts& K) {
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, 2.0 * n_parts * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * limbs * C.N / 2;
  k_add_limbconst_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, io, stride, n_parts, limbs, C.log_n,
                                                                   K);
  HEDAP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- rescale
// last: the coefficient-domain limb l of each part (part stride ls).  For i < l the
// centred representative of last mod q_l is reduced mod q_i:
//   v <= (q_l-1)/2 -> v mod q_i,  else (v mod q_i) - (q_l mod q_i)
__global__ void k_rescale_spread_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ last, size_t ls,
                                        u64* __restrict__ tmp, size_t ts, int n_parts, int l, int log_n,
                                        RescaleConsts R) {
  const size_t N = (size_t)1 << log_n, per_part = (size_t)l << log_n;
  const u64 half = pr[l].q >> 1;
  GRID_LOOP(e, n_parts * per_part) {
    const size_t p = e / per_part, r = e - p * per_part;
    const int i = (int)(r >> log_n);
    const u64 v = last[p * ls + (r & (N - 1))];
    const PrimeDev P = pr[i];
    u64 m = barrett_reduce(v, 0, P);
    if (v > half) m = sub_mod(m, R.ql_mod[i], P.q);
    tmp[p * ts + r] = m;
  }
}
void k_rescale_spread(const Ctx& C, const u64* last, size_t ls, u64* tmp, size_t ts, int n_parts, int l,
                      const RescaleConsts& R) {
  ProfScope prof_(PROF_RESCALE, C.stream, (1.0 + l) * n_parts * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * l * C.N;
  k_rescale_spread_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, last, ls, tmp, ts, n_parts, l,
                                                                     C.log_n, R);
  HEDAP_LAUNCH_CHECK();
}
// ---------------------------------------------------------------- ModDown fused with a rescale: the last limb
__global__ void k_mdr_last_eval_kernel(const u64* __restrict__ e, size_t es, const u64* __restrict__ acc, size_t as,
                                       u64* __restrict__ t, int n_parts, int log_n, u64 q, u64 w, u64 wsh) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, (size_t)n_parts * N) {
    const size_t p = i >> log_n, n = i & (N - 1);
    t[i] = add_mod(e[p * es + n], shoup_mul(acc[p * as + n], w, wsh, q), q);
  }
}
void k_mdr_last_eval(const Ctx& C, const u64* e, size_t es, const u64* acc, size_t as, u64* t, int n_parts, int l,
                     const MdrLast& M) {
  ProfScope prof_(PROF_RESCALE, C.stream, 3.0 * n_parts * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * C.N;
  k_mdr_last_eval_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(e, es, acc, as, t, n_parts, C.log_n,
                                                                    C.primes[l], M.pinv, M.pinv_sh);
  HEDAP_LAUNCH_CHECK();
}
// x = t - (off + sum_k [z_k + c_k]_{p_k} f_k) mod q_l: the K canonical products and off sum below
// (K + 1) q_l <= 9 q_l < 2^64, reduced once
__global__ void k_mdr_last_coef_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ t,
                                       const u64* __restrict__ z, size_t zs, u64* __restrict__ x, int n_parts,
                                       int log_n, int l, MdrLast M) {
  const size_t N = (size_t)1 << log_n;
  const PrimeDev P = pr[l];
  GRID_LOOP(i, (size_t)n_parts * N) {
    const size_t p = i >> log_n, n = i & (N - 1);
    const u64* zp = z + p * zs + n;
    u64 v = M.off;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < M.K) v += shoup_mul(add_mod(zp[(size_t)k * N], M.c[k], M.p[k]), M.f[k], M.fs[k], P.q);
    x[i] = sub_mod(t[i], barrett_reduce(v, 0, P), P.q);
  }
}
void k_mdr_last_coef(const Ctx& C, const u64* t, const u64* z, size_t zs, u64* x, int n_parts, int l,
                     const MdrLast& M) {
  ProfScope prof_(PROF_RESCALE, C.stream, (2.0 + M.K) * n_parts * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * C.N;
  k_mdr_last_coef_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, t, z, zs, x, n_parts, C.log_n, l, M);
  HEDAP_LAUNCH_CHECK();
}

__global__ void k_rescale_finish_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ in, size_t is,
                                        const u64* __restrict__ tmp, size_t ts, u64* __restrict__ out, size_t os,
                                        int n_parts, int l, int log_n, RescaleConsts R) {
  const size_t per_part = (size_t)l << log_n;
  GRID_LOOP(t, n_parts * per_part / 2) {
    const size_t e = 2 * t;
    const size_t p = e / per_part, r = e - p * per_part;
    const int i = (int)(r >> log_n);
    const u64 q = pr[i].q, w = R.inv[i], wp = R.inv_sh[i];
    ulonglong2 x = ld2(in + p * is + r), y = ld2(tmp + p * ts + r);
    x.x = shoup_mul(sub_mod(x.x, y.x, q), w, wp, q);
    x.y = shoup_mul(sub_mod(x.y, y.y, q), w, wp, q);
    st2(out + p * os + r, x);
  }
}
void k_rescale_finish(const Ctx& C, const u64* in, size_t is, const u64* tmp, size_t ts, u64* out, size_t os,
                      int n_parts, int l, const RescaleConsts& R) {
  ProfScope prof_(PROF_RESCALE, C.stream, 3.0 * n_parts * l * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * l * C.N / 2;
  k_rescale_finish_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, in, is, tmp, ts, out, os, n_parts, l,
                                                                     C.log_n, R);
  HEDAP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- automorphism (NTT domain)
// evaluation j sits at psi^(2 bitrev(j) + 1); X -> X^g maps it to the evaluation at
// psi^(g (2 bitrev(j) + 1)), i.e. input index bitrev(((g e_j mod 2N) - 1) / 2).
__global__ void k_automorph_kernel(const u64* __restrict__ in, size_t is, u64* __restrict__ out, size_t os,
                                   int n_parts, int limbs, int log_n, u64 g) {
  const size_t N = (size_t)1 << log_n, per_part = (size_t)limbs << log_n;
  const u64 mask2n = 2 * N - 1;
  GRID_LOOP(e, n_parts * per_part) {
    const size_t p = e / per_part, r = e - p * per_part;
    const size_t base = r & ~(N - 1);
    const uint32_t j = (uint32_t)(r & (N - 1));
    const u64 ej = 2 * (u64)(__brev(j) >> (32 - log_n)) + 1;
    const u64 ek = (g * ej) & mask2n;
    const uint32_t k = __brev((uint32_t)((ek - 1) >> 1)) >> (32 - log_n);
    out[p * os + r] = in[p * is + base + k];
  }
}
void k_automorph(const Ctx& C, const u64* in, size_t is, u64* out, size_t os, int n_parts, int limbs, u64 g) {
  ProfScope prof_(PROF_AUTOMORPH, C.stream, 2.0 * n_parts * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * limbs * C.N;
  k_automorph_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(in, is, out, os, n_parts, limbs, C.log_n, g);
  HEDAP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- key switching
// ModUp (fast basis conversion, no correction) of every digit of the
// coefficient-domain inputs at level l into the extended basis Q_l u P:
//   y_j,t = sum_{i in digit j} [x_i * qhat_i^-1]_{q_i} * (qhat_i mod t)  mod t
// The digit's own limbs receive x itself.  dcoef: [B][l+1][N]; y: [B][dnum][l+1+K][N].
// Constants (per level): qinv[l+1], qinv_sh[l+1], then qhat[dnum][alpha][ext].
__global__ void k_modup_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ r64s,
                               const u64* __restrict__ dcoef, u64* __restrict__ y, const u64* __restrict__ cst, int l,
                               int alpha, int n_q, int K, int batch, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const int ext = l + 1 + K, dn = (l + 1 + alpha - 1) / alpha;
  const u64* qinv = cst;
  const u64* qinv_sh = cst + (l + 1);
  const u64* qhat = cst + 2 * (l + 1);
  GRID_LOOP(e, (size_t)batch * dn * N) {
    const size_t kj = e >> log_n, n = e & (N - 1);
    const int j = (int)(kj % dn);
    const size_t k = kj / dn;
    const u64* xin = dcoef + k * (size_t)(l + 1) * N;
    u64* yo = y + kj * (size_t)ext * N;
    const int lo = j * alpha, hi = min(lo + alpha, l + 1);
    u64 z[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (a < hi - lo) {
        const int i = lo + a;
        const u64 x = xin[(size_t)i * N + n];
        z[a] = shoup_mul(x, qinv[i], qinv_sh[i], pr[i].q);
        yo[(size_t)i * N + n] = x;
      }
    }
    const u64* qh = qhat + (size_t)j * alpha * ext;
    for (int t = 0; t < ext; ++t) {
      if (t >= lo && t < hi) continue;
      const int pt = t <= l ? t : n_q + (t - l - 1);
      Acc128 acc{0, 0};
#pragma unroll
      for (int a = 0; a < 8; ++a)
        if (a < hi - lo) mac128(acc, z[a], qh[(size_t)a * ext + t]);
      yo[(size_t)t * N + n] = reduce128(acc, pr[pt], r64s[2 * pt], r64s[2 * pt + 1]);
    }
  }
}
void k_modup(const Ctx& C, const u64* dcoef, u64* y, int batch, int level, const u64* d_consts) {
  if (C.alpha > 8) throw Error(HEDAP_ERR_ARG, "alpha > 8 not supported");
  const int dn = C.dnum(level), ext = level + 1 + C.n_p;
  ProfScope prof_(PROF_MODUP, C.stream, ((level + 1.0) + (double)dn * ext) * batch * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)batch * dn * C.N;
  k_modup_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, C.d_r64.p, dcoef, y, d_consts, level, C.alpha,
                                                            C.n_q, C.n_p, batch, C.log_n);
  HEDAP_LAUNCH_CHECK();
}

// inner product with the switching key:
//   acc[k][0|1][t] = sum_j y[k][j][t] * key_j[b|a][t]
// key layout: [dnum_max][2][n_q + n_p][N]; y: [B][dn][ext][N]; acc: [B][2][ext][N].
// A digit's own limbs (t in digit j) are not in y: there the extended digit equals
// the NTT-domain input itself, read from d ([B] members of stride ds, limbs of N).
// One thread per (k, t, pair of coefficients): a CTA holds the batch members of the same coefficients
// (threadIdx.y = k), so each key word comes from DRAM once and from L1 for the
// other members; few registers per thread keep many loads in flight.
// With g != 0 the extended digits enter permuted by the automorphism X -> X^g (a
// hoisted rotation: the digits were converted once, before the automorphism): the
// NTT-domain value at n is read at the index whose evaluation point is the g-th
// power of n's; within 32 consecutive indices the permutation stays inside one
// aligned group of 32, so the gather is coalesced.
__device__ __forceinline__ uint32_t galois_index(uint32_t n, u64 g, int log_n) {
  const u64 e = 2 * (u64)(__brev(n) >> (32 - log_n)) + 1;
  const u64 eg = (g * e) & ((2ull << log_n) - 1);
  return __brev((uint32_t)((eg - 1) >> 1)) >> (32 - log_n);
}
__global__ void k_ksk_inner_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ r64s,
                                   const u64* __restrict__ y, const u64* __restrict__ d, size_t ds,
                                   const u64* __restrict__ key, u64* __restrict__ acc, int l, int dn, int alpha,
                                   int n_q, int K, int log_n, u64 g, const u64* __restrict__ c0, size_t c0s,
                                   const u64* __restrict__ pmod) {
  // two consecutive coefficients per thread (16-byte loads: longer runs per DRAM page
  // across the dn x B digit streams); a permuted source is read word by word
  const size_t N = (size_t)1 << log_n;
  const int ext = l + 1 + K, total_primes = n_q + K;
  const int t = blockIdx.y, k = threadIdx.y;
  const size_t n = 2 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  const int pt = t <= l ? t : n_q + (t - l - 1);
  const int own = t <= l ? t / alpha : -1;
  const u64* kb = key + (size_t)pt * N + n;
  const u64* ka = key + ((size_t)total_primes + pt) * N + n;
  const size_t key_step = (size_t)2 * total_primes * N, y_step = (size_t)ext * N;
  const u64* yk = y + ((size_t)k * dn * ext + t) * N;
  const u64* dk = d + k * ds + (size_t)t * N;
  Acc128 a0{0, 0}, a1{0, 0}, b0{0, 0}, b1{0, 0};  // (coefficient n, n+1) x (key b, key a)
  if (!g) {
#pragma unroll 8
    for (int j = 0; j < dn; ++j) {
      const ulonglong2 v = j == own ? ld2(dk + n) : ld2(yk + j * y_step + n);
      const ulonglong2 wb = ld2(kb + j * key_step), wa = ld2(ka + j * key_step);
      mac128(a0, v.x, wb.x);
      mac128(a1, v.x, wa.x);
      mac128(b0, v.y, wb.y);
      mac128(b1, v.y, wa.y);
    }
  } else {
    const size_t s0 = galois_index((uint32_t)n, g, log_n), s1 = galois_index((uint32_t)n + 1, g, log_n);
#pragma unroll 8
    for (int j = 0; j < dn; ++j) {
      const u64* src = j == own ? dk : yk + j * y_step;
      const u64 v0 = src[s0], v1 = src[s1];
      const ulonglong2 wb = ld2(kb + j * key_step), wa = ld2(ka + j * key_step);
      mac128(a0, v0, wb.x);
      mac128(a1, v0, wa.x);
      mac128(b0, v1, wb.y);
      mac128(b1, v1, wa.y);
    }
  }
  if (c0 && t <= l) {  // the rotation kept over Q_l u P: part 0 gains P sigma_g(c0) on the Q limbs
    const u64* ck = c0 + k * c0s + (size_t)t * N;
    const size_t s0 = g ? galois_index((uint32_t)n, g, log_n) : n;
    const size_t s1 = g ? galois_index((uint32_t)n + 1, g, log_n) : n + 1;
    mac128(a0, ck[s0], pmod[pt]);
    mac128(b0, ck[s1], pmod[pt]);
  }
  const PrimeDev P = pr[pt];
  const u64 r64 = r64s[2 * pt], r64p = r64s[2 * pt + 1];
  st2(acc + (((size_t)k * 2) * ext + t) * N + n,
      ulonglong2{reduce128(a0, P, r64, r64p), reduce128(b0, P, r64, r64p)});
  st2(acc + (((size_t)k * 2 + 1) * ext + t) * N + n,
      ulonglong2{reduce128(a1, P, r64, r64p), reduce128(b1, P, r64, r64p)});
}
void k_ksk_inner(const Ctx& C, const u64* y, const u64* d, size_t d_stride, const u64* key, u64* acc, int batch,
                 int level, u64 galois_perm, const u64* c0, size_t c0_stride) {
  if (batch < 1 || batch > kMaxBatch) throw Error(HEDAP_ERR_ARG, "batch must lie in [1, 16]");
  const int dn = C.dnum(level), ext = level + 1 + C.n_p;
  ProfScope prof_(PROF_KSK_INNER, C.stream, ((double)batch * dn + 2.0 * dn + 2.0 * batch) * ext * C.N * 8);
  prof_count_launches(1);
  const unsigned tx = 32u * (unsigned)std::max(1, 8 / batch);  // about 256 threads per CTA
  const dim3 block(tx, (unsigned)batch), grid((unsigned)(C.N / 2 / tx), (unsigned)ext);
  k_ksk_inner_kernel<<<grid, block, 0, C.stream>>>(C.tab.pr, C.d_r64.p, y, d, d_stride, key, acc, level, dn, C.alpha,
                                                   C.n_q, C.n_p, C.log_n, galois_perm, c0, c0_stride, C.d_pmod.p);
  HEDAP_LAUNCH_CHECK();
}

// a batch over Q_l u P: (P c0, P c1) on the Q limbs (P mod q_i by Barrett), 0 on the special limbs
__global__ void k_lift_qp_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ pmod,
                                 const u64* __restrict__ in, size_t is, u64* __restrict__ out, int n_parts, int l,
                                 int ext, int log_n) {
  const size_t N = (size_t)1 << log_n, per = (size_t)ext << log_n;
  GRID_LOOP(e, (size_t)n_parts * per) {
    const size_t p = e / per, r = e - p * per;
    const int t = (int)(r >> log_n);
    out[e] = t <= l ? mul_mod(in[p * is + r], pmod[t], pr[t]) : 0;
  }
}
void k_lift_qp(const Ctx& C, const u64* in, size_t is, u64* out, int n_parts, int level) {
  const int ext = level + 1 + C.n_p;
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, (double)n_parts * (level + 1 + ext) * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * ext * C.N;
  k_lift_qp_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, C.d_pmod.p, in, is, out, n_parts, level,
                                                                ext, C.log_n);
  HEDAP_LAUNCH_CHECK();
}

// ModDown, first half: from the coefficient-domain P limbs of acc (n_parts parts, stride ext*N)
//   r_k = [(x_k + floor(P/2)) * phat_k^-1]_{p_k},
//   v_i = sum_k r_k * (phat_k mod q_i) - floor(P/2)  mod q_i   (coefficient domain)
// so that, after an NTT of v, x - v = x + floor(P/2) - BConv(...) on every coefficient.
// Constants (level independent, see context.cu): halfP_p[K], phinv[K], phinv_sh[K],
// phat_q[K][n_q], Pinv[n_q], Pinv_sh[n_q], halfP_q[n_q].
__global__ void k_moddown_spread_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ r64s,
                                        const u64* __restrict__ acc, u64* __restrict__ v,
                                        const u64* __restrict__ cst, int n_parts, int l, int n_q, int K, int log_n) {
  const size_t N = (size_t)1 << log_n;
  const int ext = l + 1 + K;
  const u64* halfP_p = cst;
  const u64* phinv = cst + K;
  const u64* phinv_sh = cst + 2 * K;
  const u64* phat_q = cst + 3 * K;
  const u64* halfP_q = cst + 3 * K + (size_t)K * n_q + 2 * (size_t)n_q;
  GRID_LOOP(e, (size_t)n_parts << log_n) {
    const size_t p = e >> log_n, n = e & (N - 1);
    u64 r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k < K) {
        const u64 pk = pr[n_q + k].q;
        const u64 x = acc[(p * ext + l + 1 + k) * N + n];
        r[k] = shoup_mul(add_mod(x, halfP_p[k], pk), phinv[k], phinv_sh[k], pk);
      }
    }
    for (int i = 0; i <= l; ++i) {
      Acc128 s{0, 0};
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < K) mac128(s, r[k], phat_q[(size_t)k * n_q + i]);
      const u64 conv = reduce128(s, pr[i], r64s[2 * i], r64s[2 * i + 1]);
      v[(p * (l + 1) + i) * N + n] = sub_mod(conv, halfP_q[i], pr[i].q);
    }
  }
}
void k_moddown_spread(const Ctx& C, const u64* acc, u64* v, int n_parts, int level) {
  if (C.n_p > 8) throw Error(HEDAP_ERR_ARG, "more than 8 special primes not supported");
  ProfScope prof_(PROF_MODDOWN, C.stream, (double)n_parts * (C.n_p + level + 1.0) * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * C.N;
  k_moddown_spread_kernel<<<grid_for(work, 128), 128, 0, C.stream>>>(C.tab.pr, C.d_r64.p, acc, v, C.d_moddown.p,
                                                                     n_parts, level, C.n_q, C.n_p, C.log_n);
  HEDAP_LAUNCH_CHECK();
}
// ModDown, second half (NTT domain): out_p = (acc_p - v_p) * P^-1 mod q_i, part p of the
// output at out + p * os; even parts add into the output when acc_even, odd when acc_odd
__global__ void k_moddown_finish_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ acc,
                                        const u64* __restrict__ v, u64* __restrict__ out, size_t os,
                                        const u64* __restrict__ cst, int n_parts, int l, int n_q, int K, int log_n,
                                        int acc_even, int acc_odd) {
  const size_t per_part = (size_t)(l + 1) << log_n;
  const size_t ext_stride = (size_t)(l + 1 + K) << log_n;
  const u64* Pinv = cst + 3 * K + (size_t)K * n_q;
  const u64* Pinv_sh = Pinv + n_q;
  GRID_LOOP(t, n_parts * per_part / 2) {
    const size_t e = 2 * t;
    const size_t p = e / per_part, r = e - p * per_part;
    const int i = (int)(r >> log_n);
    const u64 q = pr[i].q;
    const ulonglong2 x = ld2(acc + p * ext_stride + r);
    const ulonglong2 w = ld2(v + p * per_part + r);
    ulonglong2 z;
    z.x = shoup_mul(sub_mod(x.x, w.x, q), Pinv[i], Pinv_sh[i], q);
    z.y = shoup_mul(sub_mod(x.y, w.y, q), Pinv[i], Pinv_sh[i], q);
    u64* o = out + p * os + r;
    if ((p & 1) ? acc_odd : acc_even) {
      const ulonglong2 c = ld2(o);
      z.x = add_mod(z.x, c.x, q);
      z.y = add_mod(z.y, c.y, q);
    }
    st2(o, z);
  }
}
void k_moddown_finish(const Ctx& C, const u64* acc, const u64* v, u64* out, size_t os, int n_parts, int level,
                      bool acc_even, bool acc_odd) {
  ProfScope prof_(PROF_MODDOWN, C.stream, (3.0 + (acc_even + acc_odd) / 2.0) * n_parts * (level + 1) * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)n_parts * (level + 1) * C.N / 2;
  k_moddown_finish_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, acc, v, out, os, C.d_moddown.p,
                                                                     n_parts, level, C.n_q, C.n_p, C.log_n, acc_even,
                                                                     acc_odd);
  HEDAP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- key generation / encryption helpers
// b = e - a*s + [t in digit] * (P mod q_t) * s'   (all NTT domain, over every prime)
__global__ void k_keygen_combine_kernel(const PrimeDev* __restrict__ pr, u64* __restrict__ b,
                                        const u64* __restrict__ a, const u64* __restrict__ s,
                                        const u64* __restrict__ sp, const u64* __restrict__ pmod, int lo, int hi,
                                        int total_primes, int log_n) {
  GRID_LOOP(e, (size_t)total_primes << log_n) {
    const int t = (int)(e >> log_n);
    const PrimeDev P = pr[t];
    u64 v = sub_mod(b[e], mul_mod(a[e], s[e], P), P.q);
    if (t >= lo && t < hi) v = add_mod(v, mul_mod(pmod[t], sp[e], P), P.q);
    b[e] = v;
  }
}
void k_keygen_combine(const Ctx& C, u64* b, const u64* a, const u64* s, const u64* sp, const u64* pmod, int lo,
                      int hi) {
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, 4.0 * C.total_primes() * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)C.total_primes() * C.N;
  k_keygen_combine_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, b, a, s, sp, pmod, lo, hi,
                                                                     C.total_primes(), C.log_n);
  HEDAP_LAUNCH_CHECK();
}
__global__ void k_scale_limbs_kernel(const PrimeDev* __restrict__ pr, u64* __restrict__ x, int limbs, int log_n,
                                     const u64* __restrict__ f) {
  GRID_LOOP(e, (size_t)limbs << log_n) {
    const int t = (int)(e >> log_n);
    x[e] = shoup_mul(x[e], f[2 * t], f[2 * t + 1], pr[t].q);
  }
}
void k_scale_limbs(const Ctx& C, u64* x, int limbs, const u64* f) {
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, 2.0 * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)limbs * C.N;
  k_scale_limbs_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, x, limbs, C.log_n, f);
  HEDAP_LAUNCH_CHECK();
}
// out = x (op) y*z elementwise over `limbs` limbs (prime = limb index): op 0: x - y*z, 1: x + y*z, 2: y*z
__global__ void k_fma_kernel(const PrimeDev* __restrict__ pr, const u64* __restrict__ x, const u64* __restrict__ y,
                             const u64* __restrict__ z, u64* __restrict__ out, int limbs, int log_n, int op) {
  GRID_LOOP(e, (size_t)limbs << log_n) {
    const PrimeDev P = pr[e >> log_n];
    const u64 m = mul_mod(y[e], z[e], P);
    out[e] = op == 2 ? m : (op == 0 ? sub_mod(x[e], m, P.q) : add_mod(x[e], m, P.q));
  }
}
void k_fma(const Ctx& C, const u64* x, const u64* y, const u64* z, u64* out, int limbs, int op) {
  ProfScope prof_(PROF_ELEMENTWISE, C.stream, 4.0 * limbs * C.N * 8);
  prof_count_launches(1);
  const size_t work = (size_t)limbs * C.N;
  k_fma_kernel<<<grid_for(work, 256), 256, 0, C.stream>>>(C.tab.pr, x, y, z, out, limbs, C.log_n, op);
  HEDAP_LAUNCH_CHECK();
}

}  // namespace hedap
