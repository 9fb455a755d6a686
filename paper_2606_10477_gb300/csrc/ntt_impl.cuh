// Batched negacyclic NTT / inverse NTT over RNS limbs.
//
// Forward: out[j] = sum_i a_i psi^(i (2 bitrev(j) + 1)) mod q, computed as
// log N Cooley-Tukey stages with the psi twist merged into the twiddles
// (twiddle of stage s, butterfly block i: psi^bitrev(2^s + i)).  Inverse:
// Gentleman-Sande stages with psi^-bitrev, then N^-1.
//
// N = 2^(L1+L2) is split in two launches.  The first L1 forward stages only
// couple elements whose index agrees modulo 2^L2, so each CTA loads C such
// "columns" (rows of C consecutive words, coalesced) into shared memory and
// runs those stages there; the last L2 stages couple only elements inside
// blocks of 2^L2 consecutive words, so the second launch stages whole blocks.
// Inside a launch every thread takes groups of 2^RL elements through RL stages
// in registers between shared-memory exchanges (RL = 4: two passes per
// 256-point phase; RL = 3: three).  For a group with elements at c = high*2^(S+K) + m*2^S + low (or the
// mirrored forward form), the twiddle of every butterfly has a closed-form index
// in (high, m, u), so no per-element index arithmetic is needed.  Twiddles are
// (w, floor(w 2^64 / q)) pairs; every CTA stages the twiddles it uses in shared
// memory with its data (the column phase's 2^L1, the row phase's contiguous
// per-stage ranges for its blocks), both copied with cp.async so that all of a
// tile's copies are in flight at once.  Optional fusions (NttAux):
// the first phase may read another buffer (out of place) or compute its input as
// the fast basis conversion of a key-switching digit (ModUp fused into the load),
// the inverse may end with a per-limb factor other than N^-1, a digit's own
// limbs may be skipped, and a rescale, a ModDown or both (one transform, see
// ks_moddown_rescale) may be fused around a forward transform (conversion and
// spread into the first phase's load, the finish into the second phase's store).  Butterflies keep residues
// lazily (Harvey 2014): forward below 8q with the first operand reduced at every
// other stage, inverse in [0, 2q); the final launch writes canonical residues.
#pragma once
#include <algorithm>

#include "internal.cuh"
#include "profiler.cuh"

namespace hedap {

// Forward (Cooley-Tukey) butterfly on lazy residues.  Every stage adds at most 2q to the bound
// (t < 2q), so the first operand is brought from [0, 8q) into [0, 4q) only at even stages
// (REDUCE): an even stage leaves values below 6q, the odd stage after it below 8q (< 2^64 for
// q < 2^61), and the next even stage starts again from [0, 4q).
template <bool REDUCE>
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, const ulonglong2 w, u64 q) {
  if constexpr (REDUCE) {
    const u64 q4 = q << 2;
    if (x >= q4) x -= q4;
  }
  const u64 t = shoup_mul_lazy(y, w.x, w.y, q);  // [0, 2q)
  const u64 q2 = q << 1;
  y = x + q2 - t;
  x = x + t;
}
// stage `s` of the forward transform (global index)
__device__ __forceinline__ void ct_bfly_stage(int s, u64& x, u64& y, const ulonglong2 w, u64 q) {
  if (s % 2 == 0) ct_bfly<true>(x, y, w, q);
  else ct_bfly<false>(x, y, w, q);
}
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, const ulonglong2 w, u64 q) {
  const u64 q2 = q << 1;
  u64 s = x + y;
  if (s >= q2) s -= q2;
  const u64 d = x + q2 - y;
  y = shoup_mul_lazy(d, w.x, w.y, q);
  x = s;
}
__device__ __forceinline__ u64 reduce8q(u64 x, u64 q) {
  const u64 q4 = q << 2, q2 = q << 1;
  if (x >= q4) x -= q4;
  if (x >= q2) x -= q2;
  if (x >= q) x -= q;
  return x;
}
// asynchronous global -> shared copies (cp.async): every copy of a tile is in flight at once, with
// no register round trip; one wait_group 0 and a barrier make them visible to the CTA
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// RL: stages per register pass (radix 2^RL), a template parameter of every kernel

// true when limb li of `part` is one of its digit's own limbs (skipped, see NttAux)
__device__ __forceinline__ bool own_limb(const NttAux& A, int part, int li) {
  if (!A.own_alpha) return false;
  const int lo = (part % A.own_dn) * A.own_alpha;
  return li >= lo && li < min(lo + A.own_alpha, A.own_limit);
}
// source of limb li of `part` for the first phase (in place unless A.src)
__device__ __forceinline__ const u64* first_src(const NttAux& A, const LimbSet& S, int part, int li, size_t N) {
  return A.src ? A.src + part * A.src_stride + (size_t)li * N : S.limb(part, li, N);
}

// shared-memory index of element x of a row block: one pad word every 16
__device__ __forceinline__ uint32_t padx(uint32_t x) { return x + (x >> 4); }
// Row layout (rows of 2^L2 words, R = 2^L2 + 2^(L2-4) apart).  For the words idx = t + i TPB of an unrolled
// loop (t = threadIdx.x; TPB and 2^L2 powers of two, TPB a multiple of 16) the offset is a per-thread part
// row_off(t) plus a compile-time part row_step(i): no index arithmetic per word.
template <int L2>
__device__ __forceinline__ uint32_t row_off(uint32_t t) {
  return (t >> L2) * ((1u << L2) + (1u << (L2 - 4))) + padx(t & ((1u << L2) - 1));
}
template <int L2, int TPB>
__host__ __device__ constexpr uint32_t row_step(int i) {
  constexpr uint32_t P2 = 1u << L2, R = P2 + (P2 >> 4);
  return (uint32_t)TPB >= P2 ? (uint32_t)i * ((uint32_t)TPB >> L2) * R
                             : (uint32_t)(i / (int)(P2 / TPB)) * R + (uint32_t)(i % (int)(P2 / TPB)) * TPB +
                                   (((uint32_t)(i % (int)(P2 / TPB)) * TPB) >> 4);
}

// ---------------------------------------------------------------- forward, column phase
// element (c, col) at sm[c * C + col]; global index j = r0 + col + c * 2^L2;
// stage s couples c and c + 2^(L1-s-1); twiddle index 2^s + (c >> (L1 - s)).
template <int L1, int C, int RL, int S0>
__device__ __forceinline__ void fwd_cols_passes(u64* sm, const ulonglong2* tw, u64 q) {
  if constexpr (S0 < L1) {
    constexpr int K = (L1 - S0) < RL ? (L1 - S0) : RL;
    constexpr int TL = 1 << (L1 - S0 - K);
    constexpr int GROUPS = C << (L1 - K);
    constexpr int TPB = (C << L1) >> RL;  // threads per CTA
#pragma unroll
    for (int g = threadIdx.x; g < GROUPS; g += TPB) {
      const uint32_t col = g % C, gg = g / C;
      const uint32_t low = gg & (TL - 1), high = gg >> (L1 - S0 - K);
      const uint32_t base = (high << (L1 - S0)) | low;
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = sm[(base + m * TL) * C + col];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int half = 1 << (K - 1 - u);
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const uint32_t wi = (1u << (S0 + u)) + (high << u) + (m1 >> (K - u));
          ct_bfly_stage(S0 + u, v[m1], v[m1 + half], tw[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) sm[(base + m * TL) * C + col] = v[m];
    }
    __syncthreads();
    fwd_cols_passes<L1, C, RL, S0 + K>(sm, tw, q);
  }
}

template <int L1, int L2, int C, int TPB, int MINB, int RL>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_fwd_cols(Tables T, LimbSet S, NttAux A) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  ulonglong2* tw = reinterpret_cast<ulonglong2*>(sm + (C << L1));
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  if (own_limb(A, part, li)) return;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const ulonglong2* W = T.psi2 + (size_t)pi * N;
#pragma unroll
  for (int i = threadIdx.x; i < (1 << L1); i += TPB) cp_async16(tw + i, W + i);
  const int r0 = blockIdx.x * C;
  if (A.z) {  // fused ModUp: fast basis conversion of digit j into this limb's prime
    // sum of na <= 8 Shoup products, each in [0, 2q), brought into [0, 4q): the
    // first butterflies accept any input below 4q (a term folded into the key is z itself, below the
    // bound the key's construction checked)
    const int j = part % A.own_dn, lo = j * A.own_alpha, na = min(A.own_alpha, A.own_limit - lo);
    const u64* zk = A.z + (size_t)(part / A.own_dn) * A.z_stride + (size_t)lo * N;
    const u64* bc = A.bconv + (size_t)j * A.own_alpha * A.ext + li;
    const u64* bcs = bc + A.bconv_sh_offset;
    u64 f[8], fs[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      f[t] = t < na ? bc[(size_t)t * A.ext] : 0;
      fs[t] = t < na ? bcs[(size_t)t * A.ext] : 0;
    }
    const u64 q4 = q << 2, q8 = q << 3;
#pragma unroll
    for (int idx = threadIdx.x; idx < (C << L1); idx += TPB) {
      const int c = idx / C, col = idx % C;
      const size_t n = ((size_t)c << L2) + r0 + col;
      u64 v = 0;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t < na) v += fs[t] ? shoup_mul_lazy(zk[(size_t)t * N + n], f[t], fs[t], q) : zk[(size_t)t * N + n];
      if (v >= q8) v -= q8;
      if (v >= q4) v -= q4;
      sm[idx] = v;
    }
  } else if (A.pconv) {  // fused ModDown conversion of the special-prime limbs into this prime
    const u64* zp = A.pconv + (size_t)part * A.pconv_stride;
    u64 c[8], pk[8], f[8], fs[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const bool on = k < A.pconv_K;
      c[k] = on ? A.pconv_c[k] : 0;
      pk[k] = on ? A.pconv_q[k] : 0;
      f[k] = on ? A.pconv_phat[(size_t)k * A.pconv_ld + li] : 0;
      fs[k] = on ? A.pconv_phat_sh[(size_t)k * A.pconv_ld + li] : 0;
    }
    const u64 off = (q << 2) - A.pconv_half[li], q4 = q << 2, q8 = q << 3;
    const bool lazy = A.pconv_K <= 5;
#pragma unroll
    for (int idx = threadIdx.x; idx < (C << L1); idx += TPB) {
      const int cc = idx / C, col = idx % C;
      const size_t n = ((size_t)cc << L2) + r0 + col;
      // 4q - floor(S/2) mod q plus K products: lazy (< 2q each) for K <= 5, canonical (< q) for
      // K <= 8, so the sum stays below 16q < 2^64
      u64 v = off;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < A.pconv_K) {
          u64 term = shoup_mul_lazy(add_mod(zp[(size_t)k * N + n], c[k], pk[k]), f[k], fs[k], q);
          if (!lazy && term >= q) term -= q;
          v += term;
        }
      if (v >= q8) v -= q8;
      if (v >= q4) v -= q4;
      if (A.spread) {  // a ModDown fused with a rescale: plus the centred last limb, [0, 5q)
        const u64 x = A.spread[(size_t)part * A.spread_stride + n];
        const u64 half = T.pr[A.spread_prime].q >> 1;
        u64 m = barrett_reduce(x, 0, T.pr[pi]);
        if (x > half) m = sub_mod(m, A.spread_sub[li], q);
        v += m;
      }
      sm[idx] = v;
    }
  } else if (A.spread) {  // fused rescale spread: centred residue of the last limb in this prime
    const u64* x = A.spread + (size_t)part * A.spread_stride;
    const u64 half = T.pr[A.spread_prime].q >> 1, sub = A.spread_sub[li];
    const PrimeDev P = T.pr[pi];
#pragma unroll
    for (int idx = threadIdx.x; idx < (C << L1); idx += TPB) {
      const int c = idx / C, col = idx % C;
      const u64 v = x[((size_t)c << L2) + r0 + col];
      u64 m = barrett_reduce(v, 0, P);
      if (v > half) m = sub_mod(m, sub, q);
      sm[idx] = m;
    }
  } else {
    const u64* src = first_src(A, S, part, li, N);
#pragma unroll
    for (int idx = threadIdx.x; idx < (C << L1); idx += TPB) {
      const int c = idx / C, col = idx % C;
      cp_async8(sm + idx, src + ((size_t)c << L2) + r0 + col);
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  fwd_cols_passes<L1, C, RL, 0>(sm, tw, q);
#pragma unroll
  for (int idx = threadIdx.x; idx < (C << L1); idx += TPB) {
    const int c = idx / C, col = idx % C;
    a[((size_t)c << L2) + r0 + col] = sm[idx];
  }
}

// ---------------------------------------------------------------- forward, column phase from shared tiles, several limbs
// Three fused first phases read the same few tiles for every output limb: the ModUp of one digit
// (its na <= 3 coefficient-domain limbs z), the ModDown conversion (the K <= 3 special-prime limbs)
// and the rescale spread (the last limb).  This kernel stages those tiles once (cp.async, straight
// into shared memory) and runs the column phase of `lpc` consecutive output limbs of one part from
// there, so the wait for global memory is paid once per lpc limbs; each limb's twiddles are
// fetched with cp.async while the previous limb computes (two twiddle buffers).

template <int L1, int L2, int C, int TPB, int MINB, int RL>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_fwd_cols_shared(Tables T, LimbSet S, NttAux A, int lpc) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  constexpr int E = C << L1;
  ulonglong2* twb = reinterpret_cast<ulonglong2*>(sm + E);  // two buffers of 2^L1 pairs
  u64* zt = sm + E + 4 * (1 << L1);                         // ns staged tiles of E words
  const int groups = (S.n_limbs + lpc - 1) / lpc;
  const int part = blockIdx.y / groups, g = blockIdx.y % groups;
  const int l0 = S.limb_begin + g * lpc, l1 = min(l0 + lpc, S.limb_begin + S.n_limbs);
  // the shared tiles: ns limbs at src + t N (and, for a ModDown fused with a rescale, the last limb's
  // coefficients as tile ns)
  int ns, j = 0;
  const u64* src;
  const u64* spread_src = A.spread ? A.spread + (size_t)part * A.spread_stride : nullptr;
  if (A.z) {
    j = part % A.own_dn;
    const int lo = j * A.own_alpha;
    ns = min(A.own_alpha, A.own_limit - lo);
    src = A.z + (size_t)(part / A.own_dn) * A.z_stride + (size_t)lo * N;
  } else if (A.pconv) {
    ns = A.pconv_K;
    src = A.pconv + (size_t)part * A.pconv_stride;
  } else {
    ns = 0;
    src = nullptr;
  }
  const int nt = ns + (spread_src ? 1 : 0);
  const int r0 = blockIdx.x * C;
  // row c of tile t holds words r0 .. r0 + C - 1 of column c (16-byte copies)
  for (int idx = threadIdx.x; idx < nt * (E / 2); idx += TPB) {
    const int t = idx / (E / 2), e = 2 * (idx % (E / 2));
    const int c = e / C, col = e % C;
    const u64* base = t < ns ? src + (size_t)t * N : spread_src;
    cp_async16(zt + (size_t)t * E + e, base + ((size_t)c << L2) + r0 + col);
  }
  auto fetch_tw = [&](int li, int buf) {
    const ulonglong2* W = T.psi2 + (size_t)S.prime(li) * N;
    for (int i = threadIdx.x; i < (1 << L1); i += TPB) cp_async16(twb + buf * (1 << L1) + i, W + i);
  };
  int li = l0;
  while (li < l1 && own_limb(A, part, li)) ++li;
  if (li < l1) fetch_tw(li, 0);
  cp_async_commit();
  int buf = 0;
  for (; li < l1; buf ^= 1) {
    int next = li + 1;
    while (next < l1 && own_limb(A, part, next)) ++next;
    cp_async_wait_all();
    __syncthreads();  // the tiles and this limb's twiddles have landed; the previous limb is done
    if (next < l1) fetch_tw(next, buf ^ 1);
    cp_async_commit();
    const int pi = S.prime(li);
    const u64 q = T.pr[pi].q, q4 = q << 2, q8 = q << 3;
    if (A.z) {  // ModUp: sum of na Shoup products (each < 2q; a folded term is z) brought into [0, 4q)
      const u64* bc = A.bconv + (size_t)j * A.own_alpha * A.ext + li;
      const u64* bcs = bc + A.bconv_sh_offset;
      u64 f[3], fs[3];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        f[t] = t < ns ? bc[(size_t)t * A.ext] : 0;
        fs[t] = t < ns ? bcs[(size_t)t * A.ext] : 0;
      }
#pragma unroll
      for (int idx = threadIdx.x; idx < E; idx += TPB) {
        u64 v = 0;
#pragma unroll
        for (int t = 0; t < 3; ++t)
          if (t < ns) v += fs[t] ? shoup_mul_lazy(zt[(size_t)t * E + idx], f[t], fs[t], q) : zt[(size_t)t * E + idx];
        if (v >= q4) v -= q4;
        sm[idx] = v;
      }
    } else if (A.pconv) {  // ModDown conversion: 4q - floor(P/2) mod q plus K lazy products (< 10q)
      u64 c[3], pk[3], f[3], fs[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const bool on = k < ns;
        c[k] = on ? A.pconv_c[k] : 0;
        pk[k] = on ? A.pconv_q[k] : 0;
        f[k] = on ? A.pconv_phat[(size_t)k * A.pconv_ld + li] : 0;
        fs[k] = on ? A.pconv_phat_sh[(size_t)k * A.pconv_ld + li] : 0;
      }
      const u64 off = q4 - A.pconv_half[li];
      // a ModDown fused with a rescale adds the centred last limb (tile ns, below q): [0, 5q)
      const u64 half = spread_src ? T.pr[A.spread_prime].q >> 1 : 0, sub = spread_src ? A.spread_sub[li] : 0;
      const PrimeDev P = T.pr[pi];
#pragma unroll
      for (int idx = threadIdx.x; idx < E; idx += TPB) {
        u64 v = off;
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < ns) v += shoup_mul_lazy(add_mod(zt[(size_t)k * E + idx], c[k], pk[k]), f[k], fs[k], q);
        if (v >= q8) v -= q8;
        if (v >= q4) v -= q4;
        if (spread_src) {
          const u64 x = zt[(size_t)ns * E + idx];
          u64 m = barrett_reduce(x, 0, P);
          if (x > half) m = sub_mod(m, sub, q);
          v += m;
        }
        sm[idx] = v;
      }
    } else {  // rescale spread: centred residue of the last limb in this prime
      const u64 half = T.pr[A.spread_prime].q >> 1, sub = A.spread_sub[li];
      const PrimeDev P = T.pr[pi];
#pragma unroll
      for (int idx = threadIdx.x; idx < E; idx += TPB) {
        const u64 v = zt[idx];
        u64 m = barrett_reduce(v, 0, P);
        if (v > half) m = sub_mod(m, sub, q);
        sm[idx] = m;
      }
    }
    __syncthreads();
    fwd_cols_passes<L1, C, RL, 0>(sm, twb + buf * (1 << L1), q);
    u64* a = S.limb(part, li, N);
#pragma unroll
    for (int idx = threadIdx.x; idx < E; idx += TPB) {
      const int c = idx / C, col = idx % C;
      a[((size_t)c << L2) + r0 + col] = sm[idx];
    }
    li = next;
  }
  cp_async_wait_all();
}

// ---------------------------------------------------------------- forward, block phase
// block b, local x at sm[b * R + padx(x)]; j = (B0 + b) * 2^L2 + x; local stage s'
// couples x and x + 2^(L2-s'-1); twiddle index 2^(L1+s') + ((B0+b) << s') + (x >> (L2 - s')).
// For the CTA's blocks B0 .. B0+BPC-1 the twiddles of stage s' are the contiguous
// range starting at 2^(L1+s') + (B0 << s') of BPC 2^s' entries; they are staged in
// shared memory one stage after another (stage s' at offset BPC (2^s' - 1)), so
// twiddle (b, s', r) sits at tw[BPC (2^s' - 1) + (b << s') + r].
template <int L1, int L2, int BPC, int TPB>
__device__ __forceinline__ void fwd_rows_stage_twiddles(ulonglong2* tw, const ulonglong2* W, uint32_t B0) {
#pragma unroll
  for (int sl = 0; sl < L2; ++sl) {
    const ulonglong2* src = W + (1u << (L1 + sl)) + (B0 << sl);
    ulonglong2* dst = tw + BPC * ((1 << sl) - 1);
    for (int i = threadIdx.x; i < (BPC << sl); i += TPB) cp_async16(dst + i, src + i);
  }
}
template <int L1, int L2, int BPC, int RL, int S0>
__device__ __forceinline__ void fwd_rows_passes(u64* sm, const ulonglong2* tw, u64 q) {
  if constexpr (S0 < L2) {
    constexpr int K = (L2 - S0) < RL ? (L2 - S0) : RL;
    constexpr int TL = 1 << (L2 - S0 - K);
    constexpr int GPB = 1 << (L2 - K);
    constexpr int R = (1 << L2) + (1 << (L2 - 4));
    constexpr int TPB = (BPC << L2) >> RL;
#pragma unroll
    for (int g = threadIdx.x; g < BPC * GPB; g += TPB) {
      const uint32_t b = g / GPB, gg = g % GPB;
      const uint32_t low = gg & (TL - 1), high = gg >> (L2 - S0 - K);
      const uint32_t base = (high << (L2 - S0)) | low;
      // padx(base + m TL) = padx(base) + m TL + (m TL >> 4): base is aligned to the group's span except for
      // low < TL, so the pad words between the group's elements depend on m only
      u64* blk = sm + b * R + padx(base);
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = blk[m * TL + ((m * TL) >> 4)];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int sl = S0 + u, half = 1 << (K - 1 - u);
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const uint32_t wi = BPC * ((1u << sl) - 1) + (b << sl) + (high << u) + (m1 >> (K - u));
          ct_bfly_stage(L1 + sl, v[m1], v[m1 + half], tw[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) blk[m * TL + ((m * TL) >> 4)] = v[m];
    }
    __syncthreads();
    fwd_rows_passes<L1, L2, BPC, RL, S0 + K>(sm, tw, q);
  }
}

template <int L1, int L2, int BPC, int TPB, int MINB, int RL>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_fwd_rows(Tables T, LimbSet S, NttAux A) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  constexpr int E = BPC << L2, R = (1 << L2) + (1 << (L2 - 4));
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  if (own_limb(A, part, li)) return;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  ulonglong2* tw = reinterpret_cast<ulonglong2*>(sm + BPC * R);
  const size_t j0 = (size_t)blockIdx.x * E;
  u64* smt = sm + row_off<L2>(threadIdx.x);  // this thread's words: smt[row_step(i)] holds word t + i TPB
#pragma unroll
  for (int i = 0; i < E / TPB; ++i) cp_async8(smt + row_step<L2, TPB>(i), a + j0 + threadIdx.x + i * TPB);
  fwd_rows_stage_twiddles<L1, L2, BPC, TPB>(tw, T.psi2 + (size_t)pi * N, (uint32_t)(blockIdx.x * BPC));
  cp_async_commit();
  if (A.fin_dst) {  // the epilogue's operands: fetched into L2 while the passes run (128-byte lines)
    const u64* cp = A.fin_c + (size_t)part * A.fin_c_stride + (size_t)li * N + j0;
    const u64* dp = A.fin_e ? A.fin_e + (size_t)part * A.fin_e_stride + (size_t)li * N + j0
                            : A.fin_dst + (size_t)part * A.fin_dst_stride + (size_t)li * N + j0;
    const bool acc = A.fin_e || ((part & 1) ? A.fin_acc_odd : A.fin_acc_even);
    for (int idx = 16 * threadIdx.x; idx < E; idx += 16 * TPB) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(cp + idx));
      if (acc) asm volatile("prefetch.global.L2 [%0];" ::"l"(dp + idx));
    }
  }
  cp_async_wait_all();
  __syncthreads();
  fwd_rows_passes<L1, L2, BPC, RL, 0>(sm, tw, q);
  if (A.fin_e) {  // ModDown fused with the rescale: c (P q_l)^-1 + (e - v) q_l^-1
    const u64* cp = A.fin_c + (size_t)part * A.fin_c_stride + (size_t)li * N + j0;
    const u64* ep = A.fin_e + (size_t)part * A.fin_e_stride + (size_t)li * N + j0;
    u64* dp = A.fin_dst + (size_t)part * A.fin_dst_stride + (size_t)li * N + j0;
    const u64 w = A.fin_w[li], wp = A.fin_wsh[li], w2 = A.fin_w2[li], w2p = A.fin_w2sh[li];
#pragma unroll
    for (int i = 0; i < E / TPB; ++i) {
      const int idx = threadIdx.x + i * TPB;
      const u64 v = reduce8q(smt[row_step<L2, TPB>(i)], q);
      const u64 z = add_mod(shoup_mul(cp[idx], w, wp, q), shoup_mul(sub_mod(ep[idx], v, q), w2, w2p, q), q);
      dp[idx] = A.fin_neg ? sub_mod(0, z, q) : z;
    }
    return;
  }
  if (A.fin_dst) {  // fused epilogue of a rescale / ModDown: (c - v) * w (+ dst)
    const u64* cp = A.fin_c + (size_t)part * A.fin_c_stride + (size_t)li * N + j0;
    u64* dp = A.fin_dst + (size_t)part * A.fin_dst_stride + (size_t)li * N + j0;
    const u64 w = A.fin_w[li], wp = A.fin_wsh[li];
    const bool acc = (part & 1) ? A.fin_acc_odd : A.fin_acc_even;
#pragma unroll
    for (int i = 0; i < E / TPB; ++i) {
      const int idx = threadIdx.x + i * TPB;
      const u64 v = reduce8q(smt[row_step<L2, TPB>(i)], q);
      u64 z = shoup_mul(sub_mod(cp[idx], v, q), w, wp, q);
      if (acc) z = add_mod(z, dp[idx], q);
      dp[idx] = z;
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < E / TPB; ++i) a[j0 + threadIdx.x + i * TPB] = reduce8q(smt[row_step<L2, TPB>(i)], q);
}

// ---------------------------------------------------------------- forward, block phase fused with the key inner product
// The extended digits of a key switch are transformed and immediately consumed by the inner product
// with the switching key, so the transformed digits are never written.  A CTA owns one ciphertext k,
// one extended limb t (prime pt) and one run of BPC row blocks; it stages the twiddles of prime pt
// once and walks the dn digits: the column-phase output of digit j (or, for the digit that owns limb
// t, the NTT-domain input d itself) is copied into shared memory with cp.async (the next digit's
// copy in flight while this one computes), the row passes run, and every thread multiplies its
// words by the two key words of digit j, limb t and adds the products into 128-bit accumulators.
// One reduction per word at the end; acc[k][0/1][t] are the only stores.  Modular sums do not
// depend on order, so the result equals the separate transform and inner product bit for bit.
// Residues entering the products are canonical (< q < 2^61), so the sum of up to 64 products stays
// below 2^128.
template <int L1, int L2, int BPC, int TPB, int MINB, int RL>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_fwd_rows_ksk(Tables T, LimbSet S, NttAux A, KskFuse F) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  constexpr int E = BPC << L2, R = (1 << L2) + (1 << (L2 - 4)), PER = E / TPB;
  u64* buf[2] = {sm, sm + BPC * R};
  ulonglong2* tw = reinterpret_cast<ulonglong2*>(sm + 2 * BPC * R);
  const int k = blockIdx.x % F.batch, blk = blockIdx.x / F.batch;
  const int t = S.limb_begin + blockIdx.y, pt = S.prime(t);
  const u64 q = T.pr[pt].q;
  const size_t j0 = (size_t)blk * E;
  const int dn = A.own_dn;
  const int own = (A.own_alpha && t < A.own_limit) ? t / A.own_alpha : -1;
  const uint32_t toff = row_off<L2>(threadIdx.x);  // word t + i TPB of a buffer at toff + row_step(i)
  auto fetch = [&](int j, u64* dst) {
    const u64* src = (j == own ? F.d + (size_t)k * F.d_stride + (size_t)t * N + j0
                               : S.limb(k * dn + j, t, N) + j0) + threadIdx.x;
#pragma unroll
    for (int i = 0; i < E / TPB; ++i) cp_async8(dst + toff + row_step<L2, TPB>(i), src + i * TPB);
  };
  fwd_rows_stage_twiddles<L1, L2, BPC, TPB>(tw, T.psi2 + (size_t)pt * N, (uint32_t)(blk * BPC));
  fetch(0, buf[0]);
  cp_async_commit();
  Acc128 ab[PER], aa[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) ab[i] = aa[i] = Acc128{0, 0};
  const u64* kb = F.key + (size_t)pt * N + j0;
  for (int j = 0; j < dn; ++j) {
    u64* cur = buf[j & 1];
    if (j + 1 < dn) {
      fetch(j + 1, buf[(j + 1) & 1]);
      cp_async_commit();
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    if (j != own) fwd_rows_passes<L1, L2, BPC, RL, 0>(cur, tw, q);
    const u64* kbj = kb + (size_t)j * F.key_digit_stride;
    const u64* kaj = kbj + F.key_a_offset;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = threadIdx.x + i * TPB;  // consecutive threads, consecutive words
      const u64 v = reduce8q(cur[toff + row_step<L2, TPB>(i)], q);
      mac128(ab[i], v, __ldg(kbj + idx));
      mac128(aa[i], v, __ldg(kaj + idx));
    }
    __syncthreads();  // every thread is done with `cur` before the copy of digit j + 2 lands there
  }
  const PrimeDev P = T.pr[pt];
  const u64 r64 = F.r64[2 * pt], r64p = F.r64[2 * pt + 1];
  u64* o0 = F.acc + (size_t)(2 * k) * F.acc_part_stride + (size_t)t * N + j0;
  u64* o1 = o0 + F.acc_part_stride;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int idx = threadIdx.x + i * TPB;
    o0[idx] = reduce128(ab[i], P, r64, r64p);
    o1[idx] = reduce128(aa[i], P, r64, r64p);
  }
}

// ---------------------------------------------------------------- inverse, block phase
// GS stage with pair distance 2^lt (lt < L2): twiddle index 2^(LOGN-lt-1) + (j >> (lt+1)),
// j >> (lt+1) = ((B0+b) << (L2-lt-1)) + (x >> (lt+1)); groups x = high*2^(LT0+K) + m*2^LT0 + low.
// Staged like the forward phase: stage lt's range starts at 2^(LOGN-lt-1) + (B0 << (L2-lt-1))
// with BPC 2^(L2-lt-1) entries, at offset BPC (2^L2 - 2^(L2-lt)) in shared memory.
template <int L1, int L2, int BPC, int TPB>
__device__ __forceinline__ void inv_rows_stage_twiddles(ulonglong2* tw, const ulonglong2* W, uint32_t B0) {
#pragma unroll
  for (int lt = 0; lt < L2; ++lt) {
    const ulonglong2* src = W + (1u << (L1 + L2 - lt - 1)) + (B0 << (L2 - lt - 1));
    ulonglong2* dst = tw + BPC * ((1 << L2) - (1 << (L2 - lt)));
    for (int i = threadIdx.x; i < (BPC << (L2 - lt - 1)); i += TPB) cp_async16(dst + i, src + i);
  }
}
template <int L1, int L2, int BPC, int RL, int LT0>
__device__ __forceinline__ void inv_rows_passes(u64* sm, const ulonglong2* tw, u64 q) {
  if constexpr (LT0 < L2) {
    constexpr int K = (L2 - LT0) < RL ? (L2 - LT0) : RL;
    constexpr int GPB = 1 << (L2 - K);
    constexpr int R = (1 << L2) + (1 << (L2 - 4));
    constexpr int TPB = (BPC << L2) >> RL;
#pragma unroll
    for (int g = threadIdx.x; g < BPC * GPB; g += TPB) {
      const uint32_t b = g / GPB, gg = g % GPB;
      const uint32_t low = gg & ((1u << LT0) - 1), high = gg >> LT0;
      const uint32_t base = (high << (LT0 + K)) | low;
      u64* blk = sm + b * R + padx(base);  // as in the forward passes: the pads depend on m only
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = blk[(m << LT0) + ((m << LT0) >> 4)];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int lt = LT0 + u, half = 1 << u;
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const uint32_t wi = BPC * ((1u << L2) - (1u << (L2 - lt))) + (b << (L2 - lt - 1)) + (high << (K - u - 1)) +
                              (m1 >> (u + 1));
          gs_bfly(v[m1], v[m1 + half], tw[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) blk[(m << LT0) + ((m << LT0) >> 4)] = v[m];
    }
    __syncthreads();
    inv_rows_passes<L1, L2, BPC, RL, LT0 + K>(sm, tw, q);
  }
}

template <int L1, int L2, int BPC, int TPB, int MINB, int RL>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_inv_rows(Tables T, LimbSet S, NttAux A) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  constexpr int E = BPC << L2, R = (1 << L2) + (1 << (L2 - 4));
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  if (own_limb(A, part, li)) return;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const u64* src = first_src(A, S, part, li, N);
  ulonglong2* tw = reinterpret_cast<ulonglong2*>(sm + BPC * R);
  const size_t j0 = (size_t)blockIdx.x * E;
  u64* smt = sm + row_off<L2>(threadIdx.x);  // this thread's words: smt[row_step(i)] holds word t + i TPB
#pragma unroll
  for (int i = 0; i < E / TPB; ++i) cp_async8(smt + row_step<L2, TPB>(i), src + j0 + threadIdx.x + i * TPB);
  inv_rows_stage_twiddles<L1, L2, BPC, TPB>(tw, T.ipsi2 + (size_t)pi * N, (uint32_t)(blockIdx.x * BPC));
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  inv_rows_passes<L1, L2, BPC, RL, 0>(sm, tw, q);
#pragma unroll
  for (int i = 0; i < E / TPB; ++i) a[j0 + threadIdx.x + i * TPB] = smt[row_step<L2, TPB>(i)];  // [0, 2q)
}

// ---------------------------------------------------------------- inverse, column phase (+ N^-1)
// column distance 2^lc (lt = L2 + lc): twiddle index 2^(L1-lc-1) + (c >> (lc+1)) < 2^L1
template <int L1, int C, int RL, int LC0>
__device__ __forceinline__ void inv_cols_passes(u64* sm, const ulonglong2* tw, u64 q) {
  if constexpr (LC0 < L1) {
    constexpr int K = (L1 - LC0) < RL ? (L1 - LC0) : RL;
    constexpr int GROUPS = C << (L1 - K);
    constexpr int TPB = (C << L1) >> RL;
#pragma unroll
    for (int g = threadIdx.x; g < GROUPS; g += TPB) {
      const uint32_t col = g % C, gg = g / C;
      const uint32_t low = gg & ((1u << LC0) - 1), high = gg >> LC0;
      const uint32_t base = (high << (LC0 + K)) | low;
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = sm[(base + (m << LC0)) * C + col];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int lc = LC0 + u, half = 1 << u;
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const uint32_t wi = (1u << (L1 - lc - 1)) + (high << (K - u - 1)) + (m1 >> (u + 1));
          gs_bfly(v[m1], v[m1 + half], tw[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) sm[(base + (m << LC0)) * C + col] = v[m];
    }
    __syncthreads();
    inv_cols_passes<L1, C, RL, LC0 + K>(sm, tw, q);
  }
}

template <int L1, int L2, int C, int TPB, int MINB, int RL>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_inv_cols(Tables T, LimbSet S, NttAux A) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  ulonglong2* tw = reinterpret_cast<ulonglong2*>(sm + (C << L1));
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  if (own_limb(A, part, li)) return;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const ulonglong2* W = T.ipsi2 + (size_t)pi * N;
#pragma unroll
  for (int i = threadIdx.x; i < (1 << L1); i += TPB) cp_async16(tw + i, W + i);
  const int r0 = blockIdx.x * C;
#pragma unroll
  for (int idx = threadIdx.x; idx < (C << L1); idx += TPB) {
    const int c = idx / C, col = idx % C;
    cp_async8(sm + idx, a + ((size_t)c << L2) + r0 + col);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  inv_cols_passes<L1, C, RL, 0>(sm, tw, q);
  const int pr_ = li - S.limb_begin;
  const u64 ni = A.post ? A.post[2 * pr_] : T.ninv[pi], nip = A.post ? A.post[2 * pr_ + 1] : T.ninv_sh[pi];
#pragma unroll
  for (int idx = threadIdx.x; idx < (C << L1); idx += TPB) {
    const int c = idx / C, col = idx % C;
    a[((size_t)c << L2) + r0 + col] = shoup_mul(sm[idx], ni, nip, q);
  }
}

// ---------------------------------------------------------------- dispatch
// A variant fixes the words staged per CTA (E), the CTAs per SM the register
// allocation must allow (MINB) and the stages per register pass (RL: radix 16 or
// radix 8, the latter with half the registers per thread); threads per CTA = E / 2^RL.  The autotuner in
// ntt_tune() times every variant and keeps the fastest per direction.
// launch shape of the second phase fused with the key inner product (k_ntt_fwd_rows_ksk): 1024 words
// per CTA, radix-8 passes (128 threads, 8 words and 32 accumulator registers each), registers left
// uncapped (168 a thread, 3 CTAs per SM).  A batched HMult at the top level (N = 2^16, batch 8) took
// 3.72 ms, against 3.95 ms with 2048 words and 2 CTAs per SM (128 registers, spilling), 3.82 ms with
// 1024 words and 4 CTAs per SM (128 registers) and 3.78 ms with 512 words in radix-4 passes.
constexpr int kKskWords = 1024, kKskMinBlocks = 2, kKskRL = 3;

template <int L1, int L2, int E, int MINB, int RL>
static void launch_pair(const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse, const NttAux& A,
                        const KskFuse* F) {
  constexpr int LOGN = L1 + L2;
  constexpr int EE = E <= (1 << LOGN) ? E : (1 << LOGN);
  constexpr int C = EE >> L1, BPC = EE >> L2, TPB = EE >> RL;
  const dim3 grid((unsigned)(((size_t)1 << LOGN) / EE), (unsigned)(S.n_parts * S.n_limbs));
  const size_t smem_cols = (size_t)EE * sizeof(u64) + ((size_t)1 << L1) * sizeof(ulonglong2);
  const size_t smem_rows =
      (size_t)BPC * ((1 << L2) + (1 << (L2 - 4))) * sizeof(u64) + (size_t)BPC * (1 << L2) * sizeof(ulonglong2);
  if (grid.y == 0) return;
  static const bool attrs = [&] {  // opt in to more than 48 KB of dynamic shared memory, once per shape
    if (smem_cols > 48 * 1024) {
      HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_fwd_cols<L1, L2, C, TPB, MINB, RL>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols));
      HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_inv_cols<L1, L2, C, TPB, MINB, RL>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols));
    }
    if (smem_rows > 48 * 1024) {
      HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_fwd_rows<L1, L2, BPC, TPB, MINB, RL>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows));
      HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_inv_rows<L1, L2, BPC, TPB, MINB, RL>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows));
    }
    return true;
  }();
  (void)attrs;
  // the first phase applies src / z / spread; the second runs in place on S (or into fin_dst)
  NttAux A2 = A;
  A2.src = nullptr;
  A2.z = nullptr;
  A2.spread = nullptr;
  A2.pconv = nullptr;
  if (!inverse) {
    // staged tiles: the digit's limbs (ModUp), the special limbs (ModDown, plus the last limb when a
    // rescale is fused) or the last limb (rescale); at most 3 products per word in the load
    const int ns_max = A.z ? std::min(A.own_alpha, A.own_limit)
                           : A.pconv ? A.pconv_K + (A.spread ? 1 : 0) : A.spread ? 1 : 0;
    const int n_prod = A.z ? ns_max : A.pconv ? A.pconv_K : 0;
    if (ns_max >= 1 && ns_max <= 4 && n_prod <= 3 && !A.src) {
      // several output limbs per CTA, sharing the staged tiles: enough limb groups for about
      // four waves of 4 CTAs on 152 SMs, at most all the limbs in one group
      const size_t per_group = (size_t)grid.x * S.n_parts;
      const int groups = (int)std::min<size_t>(S.n_limbs, std::max<size_t>(1, (2432 + per_group - 1) / per_group));
      const int lpc = (S.n_limbs + groups - 1) / groups;
      const dim3 g2(grid.x, (unsigned)(S.n_parts * ((S.n_limbs + lpc - 1) / lpc)));
      const size_t smem_m = (size_t)EE * sizeof(u64) + 2 * ((size_t)1 << L1) * sizeof(ulonglong2) +
                            (size_t)ns_max * EE * sizeof(u64);
      static const bool attr_m = [&] {
        HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_fwd_cols_shared<L1, L2, C, TPB, MINB, RL>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((size_t)EE * 8 + 2 * ((size_t)1 << L1) * 16 + 4 * (size_t)EE * 8)));
        return true;
      }();
      (void)attr_m;
      k_ntt_fwd_cols_shared<L1, L2, C, TPB, MINB, RL><<<g2, TPB, smem_m, st>>>(T, S, A, lpc);
    } else {
      k_ntt_fwd_cols<L1, L2, C, TPB, MINB, RL><<<grid, TPB, smem_cols, st>>>(T, S, A);
    }
    if (F) {
      constexpr int EK = kKskWords <= (1 << LOGN) ? kKskWords : (1 << LOGN);
      constexpr int BPCK = EK >> L2, TPBK = EK >> kKskRL;
      const size_t smem_k = 2 * (size_t)BPCK * ((1 << L2) + (1 << (L2 - 4))) * sizeof(u64) +
                            (size_t)BPCK * (1 << L2) * sizeof(ulonglong2);
      static const bool attr_k = [&] {
        HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_fwd_rows_ksk<L1, L2, BPCK, TPBK, kKskMinBlocks, kKskRL>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_k));
        return true;
      }();
      (void)attr_k;
      const dim3 gk((unsigned)(F->batch * (((size_t)1 << LOGN) / EK)), (unsigned)S.n_limbs);
      k_ntt_fwd_rows_ksk<L1, L2, BPCK, TPBK, kKskMinBlocks, kKskRL><<<gk, TPBK, smem_k, st>>>(T, S, A2, *F);
    } else {
      k_ntt_fwd_rows<L1, L2, BPC, TPB, MINB, RL><<<grid, TPB, smem_rows, st>>>(T, S, A2);
    }
  } else {
    k_ntt_inv_rows<L1, L2, BPC, TPB, MINB, RL><<<grid, TPB, smem_rows, st>>>(T, S, A);
    k_ntt_inv_cols<L1, L2, C, TPB, MINB, RL><<<grid, TPB, smem_cols, st>>>(T, S, A2);
  }
  HEDAP_LAUNCH_CHECK();
}

template <int L1, int L2>
static void launch_variant(int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                           const NttAux& A, const KskFuse* F) {
  switch (v) {
    case 0: launch_pair<L1, L2, 2048, 5, 3>(S, T, st, inverse, A, F); break;
    case 1: launch_pair<L1, L2, 4096, 3, 4>(S, T, st, inverse, A, F); break;
    case 2: launch_pair<L1, L2, 2048, 4, 4>(S, T, st, inverse, A, F); break;
    case 3: launch_pair<L1, L2, 2048, 6, 4>(S, T, st, inverse, A, F); break;
    case 4: launch_pair<L1, L2, 2048, 6, 3>(S, T, st, inverse, A, F); break;
    case 5: launch_pair<L1, L2, 1024, 12, 3>(S, T, st, inverse, A, F); break;
    case 6: launch_pair<L1, L2, 2048, 4, 3>(S, T, st, inverse, A, F); break;
    default: launch_pair<L1, L2, 1024, 8, 3>(S, T, st, inverse, A, F); break;
  }
}

// one launch pair of the transform at N = 2^log_n (log_n 10 .. 16) with launch shape v; the
// instantiations are spread over the ntt_inst_*.cu translation units so that they compile in parallel
void ntt_launch(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                const NttAux& A, const KskFuse* F);

}  // namespace hedap
