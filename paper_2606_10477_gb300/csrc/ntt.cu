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
// Inside a launch every thread takes groups of 8 (or 4, 2) elements through
// up to three stages in registers between shared-memory exchanges.
// Butterflies keep residues lazily in [0, 4q) (forward) or [0, 2q) (inverse)
// following Harvey (2014); the final launch writes canonical residues.
#include "internal.cuh"
#include "profiler.cuh"

namespace hedap {

__device__ __forceinline__ void ct_bfly(u64& x, u64& y, u64 w, u64 wp, u64 q) {
  const u64 q2 = q << 1;
  if (x >= q2) x -= q2;
  u64 t = shoup_mul_lazy(y, w, wp, q);  // [0, 2q)
  y = x + q2 - t;
  x = x + t;
}
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, u64 w, u64 wp, u64 q) {
  const u64 q2 = q << 1;
  u64 s = x + y;
  if (s >= q2) s -= q2;
  u64 d = x + q2 - y;
  y = shoup_mul_lazy(d, w, wp, q);
  x = s;
}
__device__ __forceinline__ u64 reduce4q(u64 x, u64 q) {
  const u64 q2 = q << 1;
  if (x >= q2) x -= q2;
  if (x >= q) x -= q;
  return x;
}

constexpr int kThreads = 256;

// ---------------------------------------------------------------- forward, column phase
// shared layout: element (c, col) at sm[c * C + col]; global index j = r0 + col + c * 2^L2
template <int L1, int L2, int C, int S0>
__device__ __forceinline__ void fwd_cols_passes(u64* sm, const u64* W, const u64* WP, u64 q, int r0) {
  if constexpr (S0 < L1) {
    constexpr int K = (L1 - S0) < 3 ? (L1 - S0) : 3;
    constexpr int LOGN = L1 + L2;
    constexpr int TL = 1 << (L1 - S0 - K);
    constexpr int GROUPS = C << (L1 - K);
    for (int g = threadIdx.x; g < GROUPS; g += blockDim.x) {
      const int col = g % C, gg = g / C;
      const int low = gg & (TL - 1), high = gg >> (L1 - S0 - K);
      const int base = (high << (L1 - S0)) | low;
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = sm[(base + m * TL) * C + col];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int s = S0 + u, half = 1 << (K - 1 - u);
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const size_t j = (size_t)(r0 + col) + ((size_t)(base + m1 * TL) << L2);
          const size_t wi = ((size_t)1 << s) + (j >> (LOGN - s));
          ct_bfly(v[m1], v[m1 + half], W[wi], WP[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) sm[(base + m * TL) * C + col] = v[m];
    }
    __syncthreads();
    fwd_cols_passes<L1, L2, C, S0 + K>(sm, W, WP, q, r0);
  }
}

template <int L1, int L2, int C>
__global__ void __launch_bounds__(kThreads) k_ntt_fwd_cols(Tables T, LimbSet S) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const u64* W = T.psi + (size_t)pi * N;
  const u64* WP = T.psi_sh + (size_t)pi * N;
  const int r0 = blockIdx.x * C;
  for (int idx = threadIdx.x; idx < (C << L1); idx += blockDim.x) {
    const int c = idx / C, col = idx % C;
    sm[idx] = a[((size_t)c << L2) + r0 + col];
  }
  __syncthreads();
  fwd_cols_passes<L1, L2, C, 0>(sm, W, WP, q, r0);
  for (int idx = threadIdx.x; idx < (C << L1); idx += blockDim.x) {
    const int c = idx / C, col = idx % C;
    a[((size_t)c << L2) + r0 + col] = sm[idx];
  }
}

// ---------------------------------------------------------------- forward, block phase
// shared layout: block b, local x at sm[b * 2^L2 + x]; j = (B0 + b) * 2^L2 + x
template <int L1, int L2, int BPC, int S0>
__device__ __forceinline__ void fwd_rows_passes(u64* sm, const u64* W, const u64* WP, u64 q, size_t j0) {
  if constexpr (S0 < L2) {
    constexpr int K = (L2 - S0) < 3 ? (L2 - S0) : 3;
    constexpr int LOGN = L1 + L2;
    constexpr int TL = 1 << (L2 - S0 - K);
    constexpr int GPB = 1 << (L2 - K);
    for (int g = threadIdx.x; g < BPC * GPB; g += blockDim.x) {
      const int b = g / GPB, gg = g % GPB;
      const int low = gg & (TL - 1), high = gg >> (L2 - S0 - K);
      const int base = (high << (L2 - S0)) | low;
      u64* blk = sm + ((size_t)b << L2);
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = blk[base + m * TL];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int s = L1 + S0 + u, half = 1 << (K - 1 - u);
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const size_t j = j0 + ((size_t)b << L2) + base + m1 * TL;
          const size_t wi = ((size_t)1 << s) + (j >> (LOGN - s));
          ct_bfly(v[m1], v[m1 + half], W[wi], WP[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) blk[base + m * TL] = v[m];
    }
    __syncthreads();
    fwd_rows_passes<L1, L2, BPC, S0 + K>(sm, W, WP, q, j0);
  }
}

template <int L1, int L2, int BPC>
__global__ void __launch_bounds__(kThreads) k_ntt_fwd_rows(Tables T, LimbSet S) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  constexpr int E = BPC << L2;
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const size_t j0 = (size_t)blockIdx.x * E;
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x) sm[idx] = a[j0 + idx];
  __syncthreads();
  fwd_rows_passes<L1, L2, BPC, 0>(sm, T.psi + (size_t)pi * N, T.psi_sh + (size_t)pi * N, q, j0);
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x) a[j0 + idx] = reduce4q(sm[idx], q);
}

// ---------------------------------------------------------------- inverse, block phase
// GS stage with pair distance t = 2^lt: block index i = j >> (lt+1), twiddle index N/(2t) + i
template <int L1, int L2, int BPC, int LT0>
__device__ __forceinline__ void inv_rows_passes(u64* sm, const u64* W, const u64* WP, u64 q, size_t j0) {
  if constexpr (LT0 < L2) {
    constexpr int K = (L2 - LT0) < 3 ? (L2 - LT0) : 3;
    constexpr int LOGN = L1 + L2;
    constexpr int GPB = 1 << (L2 - K);
    for (int g = threadIdx.x; g < BPC * GPB; g += blockDim.x) {
      const int b = g / GPB, gg = g % GPB;
      const int low = gg & ((1 << LT0) - 1), high = gg >> LT0;
      const int base = (high << (LT0 + K)) | low;
      u64* blk = sm + ((size_t)b << L2);
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = blk[base + (m << LT0)];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int lt = LT0 + u, half = 1 << u;
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const size_t j = j0 + ((size_t)b << L2) + base + (m1 << LT0);
          const size_t wi = ((size_t)1 << (LOGN - lt - 1)) + (j >> (lt + 1));
          gs_bfly(v[m1], v[m1 + half], W[wi], WP[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) blk[base + (m << LT0)] = v[m];
    }
    __syncthreads();
    inv_rows_passes<L1, L2, BPC, LT0 + K>(sm, W, WP, q, j0);
  }
}

template <int L1, int L2, int BPC>
__global__ void __launch_bounds__(kThreads) k_ntt_inv_rows(Tables T, LimbSet S) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  constexpr int E = BPC << L2;
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const size_t j0 = (size_t)blockIdx.x * E;
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x) sm[idx] = a[j0 + idx];
  __syncthreads();
  inv_rows_passes<L1, L2, BPC, 0>(sm, T.ipsi + (size_t)pi * N, T.ipsi_sh + (size_t)pi * N, q, j0);
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x) a[j0 + idx] = sm[idx];  // [0, 2q)
}

// ---------------------------------------------------------------- inverse, column phase (+ N^-1)
template <int L1, int L2, int C, int LC0>
__device__ __forceinline__ void inv_cols_passes(u64* sm, const u64* W, const u64* WP, u64 q, int r0) {
  if constexpr (LC0 < L1) {
    constexpr int K = (L1 - LC0) < 3 ? (L1 - LC0) : 3;
    constexpr int LOGN = L1 + L2;
    constexpr int GROUPS = C << (L1 - K);
    for (int g = threadIdx.x; g < GROUPS; g += blockDim.x) {
      const int col = g % C, gg = g / C;
      const int low = gg & ((1 << LC0) - 1), high = gg >> LC0;
      const int base = (high << (LC0 + K)) | low;
      u64 v[1 << K];
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) v[m] = sm[(base + (m << LC0)) * C + col];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int lt = L2 + LC0 + u, half = 1 << u;
#pragma unroll
        for (int m1 = 0; m1 < (1 << K); ++m1) {
          if (m1 & half) continue;
          const size_t j = (size_t)(r0 + col) + ((size_t)(base + (m1 << LC0)) << L2);
          const size_t wi = ((size_t)1 << (LOGN - lt - 1)) + (j >> (lt + 1));
          gs_bfly(v[m1], v[m1 + half], W[wi], WP[wi], q);
        }
      }
#pragma unroll
      for (int m = 0; m < (1 << K); ++m) sm[(base + (m << LC0)) * C + col] = v[m];
    }
    __syncthreads();
    inv_cols_passes<L1, L2, C, LC0 + K>(sm, W, WP, q, r0);
  }
}

template <int L1, int L2, int C>
__global__ void __launch_bounds__(kThreads) k_ntt_inv_cols(Tables T, LimbSet S) {
  extern __shared__ u64 sm[];
  constexpr size_t N = (size_t)1 << (L1 + L2);
  const int y = blockIdx.y, part = y / S.n_limbs, li = S.limb_begin + y % S.n_limbs;
  const int pi = S.prime(li);
  const u64 q = T.pr[pi].q;
  u64* a = S.limb(part, li, N);
  const int r0 = blockIdx.x * C;
  for (int idx = threadIdx.x; idx < (C << L1); idx += blockDim.x) {
    const int c = idx / C, col = idx % C;
    sm[idx] = a[((size_t)c << L2) + r0 + col];
  }
  __syncthreads();
  inv_cols_passes<L1, L2, C, 0>(sm, T.ipsi + (size_t)pi * N, T.ipsi_sh + (size_t)pi * N, q, r0);
  const u64 ni = T.ninv[pi], nip = T.ninv_sh[pi];
  for (int idx = threadIdx.x; idx < (C << L1); idx += blockDim.x) {
    const int c = idx / C, col = idx % C;
    a[((size_t)c << L2) + r0 + col] = shoup_mul(sm[idx], ni, nip, q);
  }
}

// ---------------------------------------------------------------- dispatch
template <int L1, int L2>
static void launch_pair(const Tables& T, const LimbSet& S, cudaStream_t st, bool inverse) {
  constexpr int LOGN = L1 + L2;
  constexpr int E = LOGN >= 12 ? 4096 : (1 << LOGN);
  constexpr int C = E >> L1, BPC = E >> L2;
  const dim3 grid((unsigned)(((size_t)1 << LOGN) / E), (unsigned)(S.n_parts * S.n_limbs));
  const size_t smem = (size_t)E * sizeof(u64);
  if (grid.y == 0) return;
  ProfScope prof_(PROF_NTT, st, 16.0 * grid.y * ((size_t)1 << LOGN));
  prof_count_launches(2);
  if (!inverse) {
    k_ntt_fwd_cols<L1, L2, C><<<grid, kThreads, smem, st>>>(T, S);
    k_ntt_fwd_rows<L1, L2, BPC><<<grid, kThreads, smem, st>>>(T, S);
  } else {
    k_ntt_inv_rows<L1, L2, BPC><<<grid, kThreads, smem, st>>>(T, S);
    k_ntt_inv_cols<L1, L2, C><<<grid, kThreads, smem, st>>>(T, S);
  }
  HEDAP_LAUNCH_CHECK();
}

static void dispatch(const Tables& T, const LimbSet& S, cudaStream_t st, bool inverse) {
  switch (T.log_n) {
    case 10: launch_pair<5, 5>(T, S, st, inverse); break;
    case 11: launch_pair<5, 6>(T, S, st, inverse); break;
    case 12: launch_pair<6, 6>(T, S, st, inverse); break;
    case 13: launch_pair<6, 7>(T, S, st, inverse); break;
    case 14: launch_pair<7, 7>(T, S, st, inverse); break;
    case 15: launch_pair<7, 8>(T, S, st, inverse); break;
    case 16: launch_pair<8, 8>(T, S, st, inverse); break;
    case 17: launch_pair<8, 9>(T, S, st, inverse); break;
    default: throw Error(HEDAP_ERR_ARG, "log_n must lie in [10, 17]");
  }
}

void ntt_forward(const Tables& T, const LimbSet& S, cudaStream_t st) { dispatch(T, S, st, false); }
void ntt_inverse(const Tables& T, const LimbSet& S, cudaStream_t st) { dispatch(T, S, st, true); }

}  // namespace hedap
