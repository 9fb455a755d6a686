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
// Inside a launch every thread takes groups of 16 elements through four stages
// in registers between shared-memory exchanges (two passes per 256-point
// phase).  For a group with elements at c = high*2^(S+K) + m*2^S + low (or the
// mirrored forward form), the twiddle of every butterfly has a closed-form index
// in (high, m, u), so no per-element index arithmetic is needed.  Twiddles are
// (w, floor(w 2^64 / q)) pairs read with one 16-byte load; the column phase's
// 2^L1 distinct twiddles are staged in shared memory.  Butterflies keep residues
// lazily in [0, 4q) (forward) or [0, 2q) (inverse) following Harvey (2014);
// the final launch writes canonical residues.
#include "internal.cuh"
#include "profiler.cuh"

namespace hedap {

__device__ __forceinline__ void ct_bfly(u64& x, u64& y, const ulonglong2 w, u64 q) {
  const u64 q2 = q << 1;
  if (x >= q2) x -= q2;
  const u64 t = shoup_mul_lazy(y, w.x, w.y, q);  // [0, 2q)
  y = x + q2 - t;
  x = x + t;
}
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, const ulonglong2 w, u64 q) {
  const u64 q2 = q << 1;
  u64 s = x + y;
  if (s >= q2) s -= q2;
  const u64 d = x + q2 - y;
  y = shoup_mul_lazy(d, w.x, w.y, q);
  x = s;
}
__device__ __forceinline__ u64 reduce4q(u64 x, u64 q) {
  const u64 q2 = q << 1;
  if (x >= q2) x -= q2;
  if (x >= q) x -= q;
  return x;
}
__device__ __forceinline__ ulonglong2 ldg2(const ulonglong2* p) { return __ldg(p); }

constexpr int kRadixLog = 4;  // stages per register pass

// shared-memory index of element x of a row block: one pad word every 16
__device__ __forceinline__ uint32_t padx(uint32_t x) { return x + (x >> 4); }

// ---------------------------------------------------------------- forward, column phase
// element (c, col) at sm[c * C + col]; global index j = r0 + col + c * 2^L2;
// stage s couples c and c + 2^(L1-s-1); twiddle index 2^s + (c >> (L1 - s)).
template <int L1, int C, int S0>
__device__ __forceinline__ void fwd_cols_passes(u64* sm, const ulonglong2* tw, u64 q) {
  if constexpr (S0 < L1) {
    constexpr int K = (L1 - S0) < kRadixLog ? (L1 - S0) : kRadixLog;
    constexpr int TL = 1 << (L1 - S0 - K);
    constexpr int GROUPS = C << (L1 - K);
    for (int g = threadIdx.x; g < GROUPS; g += blockDim.x) {
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
          ct_bfly(v[m1], v[m1 + half], tw[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) sm[(base + m * TL) * C + col] = v[m];
    }
    __syncthreads();
    fwd_cols_passes<L1, C, S0 + K>(sm, tw, q);
  }
}

template <int L1, int L2, int C, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_fwd_cols(Tables T, LimbSet S) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  ulonglong2* tw = reinterpret_cast<ulonglong2*>(sm + (C << L1));
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const ulonglong2* W = T.psi2 + (size_t)pi * N;
  for (int i = threadIdx.x; i < (1 << L1); i += blockDim.x) tw[i] = ldg2(W + i);
  const int r0 = blockIdx.x * C;
  for (int idx = threadIdx.x; idx < (C << L1); idx += blockDim.x) {
    const int c = idx / C, col = idx % C;
    sm[idx] = a[((size_t)c << L2) + r0 + col];
  }
  __syncthreads();
  fwd_cols_passes<L1, C, 0>(sm, tw, q);
  for (int idx = threadIdx.x; idx < (C << L1); idx += blockDim.x) {
    const int c = idx / C, col = idx % C;
    a[((size_t)c << L2) + r0 + col] = sm[idx];
  }
}

// ---------------------------------------------------------------- forward, block phase
// block b, local x at sm[b * R + padx(x)]; j = (B0 + b) * 2^L2 + x; local stage s'
// couples x and x + 2^(L2-s'-1); twiddle index 2^(L1+s') + ((B0+b) << s') + (x >> (L2 - s')).
template <int L1, int L2, int BPC, int S0>
__device__ __forceinline__ void fwd_rows_passes(u64* sm, const ulonglong2* W, u64 q, uint32_t B0) {
  if constexpr (S0 < L2) {
    constexpr int K = (L2 - S0) < kRadixLog ? (L2 - S0) : kRadixLog;
    constexpr int TL = 1 << (L2 - S0 - K);
    constexpr int GPB = 1 << (L2 - K);
    constexpr int R = (1 << L2) + (1 << (L2 - 4));
    for (int g = threadIdx.x; g < BPC * GPB; g += blockDim.x) {
      const uint32_t b = g / GPB, gg = g % GPB;
      const uint32_t low = gg & (TL - 1), high = gg >> (L2 - S0 - K);
      const uint32_t base = (high << (L2 - S0)) | low;
      u64* blk = sm + b * R;
      const uint32_t bb = B0 + b;
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = blk[padx(base + m * TL)];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int sl = S0 + u, half = 1 << (K - 1 - u);
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const uint32_t wi = (1u << (L1 + sl)) + (bb << sl) + (high << u) + (m1 >> (K - u));
          ct_bfly(v[m1], v[m1 + half], ldg2(W + wi), q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) blk[padx(base + m * TL)] = v[m];
    }
    __syncthreads();
    fwd_rows_passes<L1, L2, BPC, S0 + K>(sm, W, q, B0);
  }
}

template <int L1, int L2, int BPC, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_fwd_rows(Tables T, LimbSet S) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  constexpr int E = BPC << L2, R = (1 << L2) + (1 << (L2 - 4));
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const size_t j0 = (size_t)blockIdx.x * E;
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x) sm[(idx >> L2) * R + padx(idx & ((1 << L2) - 1))] = a[j0 + idx];
  __syncthreads();
  fwd_rows_passes<L1, L2, BPC, 0>(sm, T.psi2 + (size_t)pi * N, q, (uint32_t)(blockIdx.x * BPC));
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x)
    a[j0 + idx] = reduce4q(sm[(idx >> L2) * R + padx(idx & ((1 << L2) - 1))], q);
}

// ---------------------------------------------------------------- inverse, block phase
// GS stage with pair distance 2^lt (lt < L2): twiddle index 2^(LOGN-lt-1) + (j >> (lt+1)),
// j >> (lt+1) = ((B0+b) << (L2-lt-1)) + (x >> (lt+1)); groups x = high*2^(LT0+K) + m*2^LT0 + low.
template <int L1, int L2, int BPC, int LT0>
__device__ __forceinline__ void inv_rows_passes(u64* sm, const ulonglong2* W, u64 q, uint32_t B0) {
  if constexpr (LT0 < L2) {
    constexpr int K = (L2 - LT0) < kRadixLog ? (L2 - LT0) : kRadixLog;
    constexpr int LOGN = L1 + L2;
    constexpr int GPB = 1 << (L2 - K);
    constexpr int R = (1 << L2) + (1 << (L2 - 4));
    for (int g = threadIdx.x; g < BPC * GPB; g += blockDim.x) {
      const uint32_t b = g / GPB, gg = g % GPB;
      const uint32_t low = gg & ((1u << LT0) - 1), high = gg >> LT0;
      const uint32_t base = (high << (LT0 + K)) | low;
      u64* blk = sm + b * R;
      const uint32_t bb = B0 + b;
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = blk[padx(base + (m << LT0))];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int lt = LT0 + u, half = 1 << u;
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const uint32_t wi = (1u << (LOGN - lt - 1)) + (bb << (L2 - lt - 1)) + (high << (K - u - 1)) + (m1 >> (u + 1));
          gs_bfly(v[m1], v[m1 + half], ldg2(W + wi), q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) blk[padx(base + (m << LT0))] = v[m];
    }
    __syncthreads();
    inv_rows_passes<L1, L2, BPC, LT0 + K>(sm, W, q, B0);
  }
}

template <int L1, int L2, int BPC, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_inv_rows(Tables T, LimbSet S) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  constexpr int E = BPC << L2, R = (1 << L2) + (1 << (L2 - 4));
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const size_t j0 = (size_t)blockIdx.x * E;
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x) sm[(idx >> L2) * R + padx(idx & ((1 << L2) - 1))] = a[j0 + idx];
  __syncthreads();
  inv_rows_passes<L1, L2, BPC, 0>(sm, T.ipsi2 + (size_t)pi * N, q, (uint32_t)(blockIdx.x * BPC));
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x)
    a[j0 + idx] = sm[(idx >> L2) * R + padx(idx & ((1 << L2) - 1))];  // [0, 2q)
}

// ---------------------------------------------------------------- inverse, column phase (+ N^-1)
// column distance 2^lc (lt = L2 + lc): twiddle index 2^(L1-lc-1) + (c >> (lc+1)) < 2^L1
template <int L1, int C, int LC0>
__device__ __forceinline__ void inv_cols_passes(u64* sm, const ulonglong2* tw, u64 q) {
  if constexpr (LC0 < L1) {
    constexpr int K = (L1 - LC0) < kRadixLog ? (L1 - LC0) : kRadixLog;
    constexpr int GROUPS = C << (L1 - K);
    for (int g = threadIdx.x; g < GROUPS; g += blockDim.x) {
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
    inv_cols_passes<L1, C, LC0 + K>(sm, tw, q);
  }
}

template <int L1, int L2, int C, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_ntt_inv_cols(Tables T, LimbSet S) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  ulonglong2* tw = reinterpret_cast<ulonglong2*>(sm + (C << L1));
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const ulonglong2* W = T.ipsi2 + (size_t)pi * N;
  for (int i = threadIdx.x; i < (1 << L1); i += blockDim.x) tw[i] = ldg2(W + i);
  const int r0 = blockIdx.x * C;
  for (int idx = threadIdx.x; idx < (C << L1); idx += blockDim.x) {
    const int c = idx / C, col = idx % C;
    sm[idx] = a[((size_t)c << L2) + r0 + col];
  }
  __syncthreads();
  inv_cols_passes<L1, C, 0>(sm, tw, q);
  const u64 ni = T.ninv[pi], nip = T.ninv_sh[pi];
  for (int idx = threadIdx.x; idx < (C << L1); idx += blockDim.x) {
    const int c = idx / C, col = idx % C;
    a[((size_t)c << L2) + r0 + col] = shoup_mul(sm[idx], ni, nip, q);
  }
}

// ---------------------------------------------------------------- dispatch
// A variant fixes the words staged per CTA (E) and the CTAs per SM the register
// allocation must allow (MINB); threads per CTA = E / 16.  The autotuner in
// ntt_tune() times every variant and keeps the fastest per direction.
template <int L1, int L2, int E, int MINB>
static void launch_pair(const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse) {
  constexpr int LOGN = L1 + L2;
  constexpr int EE = E <= (1 << LOGN) ? E : (1 << LOGN);
  constexpr int C = EE >> L1, BPC = EE >> L2, TPB = EE / 16;
  const dim3 grid((unsigned)(((size_t)1 << LOGN) / EE), (unsigned)(S.n_parts * S.n_limbs));
  const size_t smem_cols = (size_t)EE * sizeof(u64) + ((size_t)1 << L1) * sizeof(ulonglong2);
  const size_t smem_rows = (size_t)BPC * ((1 << L2) + (1 << (L2 - 4))) * sizeof(u64);
  if (grid.y == 0) return;
  static const bool attrs = [&] {  // opt in to more than 48 KB of dynamic shared memory, once per shape
    if (smem_cols > 48 * 1024) {
      HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_fwd_cols<L1, L2, C, TPB, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols));
      HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_inv_cols<L1, L2, C, TPB, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols));
    }
    if (smem_rows > 48 * 1024) {
      HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_fwd_rows<L1, L2, BPC, TPB, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows));
      HEDAP_CUDA(cudaFuncSetAttribute(k_ntt_inv_rows<L1, L2, BPC, TPB, MINB>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows));
    }
    return true;
  }();
  (void)attrs;
  if (!inverse) {
    k_ntt_fwd_cols<L1, L2, C, TPB, MINB><<<grid, TPB, smem_cols, st>>>(T, S);
    k_ntt_fwd_rows<L1, L2, BPC, TPB, MINB><<<grid, TPB, smem_rows, st>>>(T, S);
  } else {
    k_ntt_inv_rows<L1, L2, BPC, TPB, MINB><<<grid, TPB, smem_rows, st>>>(T, S);
    k_ntt_inv_cols<L1, L2, C, TPB, MINB><<<grid, TPB, smem_cols, st>>>(T, S);
  }
  HEDAP_LAUNCH_CHECK();
}

template <int L1, int L2>
static void launch_variant(int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse) {
  switch (v) {
    case 0: launch_pair<L1, L2, 4096, 1>(S, T, st, inverse); break;
    case 1: launch_pair<L1, L2, 4096, 3>(S, T, st, inverse); break;
    case 2: launch_pair<L1, L2, 2048, 4>(S, T, st, inverse); break;
    case 3: launch_pair<L1, L2, 2048, 6>(S, T, st, inverse); break;
    case 4: launch_pair<L1, L2, 8192, 1>(S, T, st, inverse); break;
    default: launch_pair<L1, L2, 1024, 8>(S, T, st, inverse); break;
  }
}

static void dispatch(const Tables& T, const LimbSet& S, cudaStream_t st, bool inverse) {
  if (S.n_parts * S.n_limbs == 0) return;
  const int v = inverse ? T.ntt_inv_variant : T.ntt_fwd_variant;
  ProfScope prof_(PROF_NTT, st, 16.0 * S.n_parts * S.n_limbs * ((size_t)1 << T.log_n));
  prof_count_launches(2);
  switch (T.log_n) {
    case 10: launch_variant<5, 5>(v, S, T, st, inverse); break;
    case 11: launch_variant<5, 6>(v, S, T, st, inverse); break;
    case 12: launch_variant<6, 6>(v, S, T, st, inverse); break;
    case 13: launch_variant<6, 7>(v, S, T, st, inverse); break;
    case 14: launch_variant<7, 7>(v, S, T, st, inverse); break;
    case 15: launch_variant<7, 8>(v, S, T, st, inverse); break;
    case 16: launch_variant<8, 8>(v, S, T, st, inverse); break;
    case 17: launch_variant<8, 9>(v, S, T, st, inverse); break;
    default: throw Error(HEDAP_ERR_ARG, "log_n must lie in [10, 17]");
  }
}

void ntt_forward(const Tables& T, const LimbSet& S, cudaStream_t st) { dispatch(T, S, st, false); }
void ntt_inverse(const Tables& T, const LimbSet& S, cudaStream_t st) { dispatch(T, S, st, true); }

// Time every variant on `limbs` limbs of scratch (forward and inverse separately,
// best of `reps` after one warm-up) and keep the fastest in C.tab.
void ntt_tune(Ctx& C, int limbs, int reps, std::vector<float>* fwd_ms, std::vector<float>* inv_ms) {
  const int n = std::max(1, std::min(limbs / C.n_q, 65535 / std::max(1, C.n_q)));
  DevBuf buf((size_t)n * C.n_q * C.N, C.stream);
  HEDAP_CUDA(cudaMemsetAsync(buf.p, 0, buf.words * 8, C.stream));
  const LimbSet S{buf.p, (size_t)C.n_q * C.N, n, 0, C.n_q, INT_MAX, 0, 0};
  cudaEvent_t a, b;
  HEDAP_CUDA(cudaEventCreate(&a));
  HEDAP_CUDA(cudaEventCreate(&b));
  for (int dir = 0; dir < 2; ++dir) {
    float best = 1e30f;
    int best_v = 0;
    for (int v = 0; v < kNttVariants; ++v) {
      Tables T = C.tab;
      T.ntt_fwd_variant = T.ntt_inv_variant = v;
      float ms = 1e30f;
      for (int r = 0; r <= reps; ++r) {
        HEDAP_CUDA(cudaEventRecord(a, C.stream));
        dispatch(T, S, C.stream, dir == 1);
        HEDAP_CUDA(cudaEventRecord(b, C.stream));
        HEDAP_CUDA(cudaEventSynchronize(b));
        float t = 0;
        HEDAP_CUDA(cudaEventElapsedTime(&t, a, b));
        if (r > 0) ms = std::min(ms, t);
      }
      if (dir == 0 && fwd_ms) fwd_ms->push_back(ms);
      if (dir == 1 && inv_ms) inv_ms->push_back(ms);
      if (ms < best) { best = ms; best_v = v; }
    }
    if (dir == 0) C.tab.ntt_fwd_variant = best_v;
    else C.tab.ntt_inv_variant = best_v;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
}

}  // namespace hedap
