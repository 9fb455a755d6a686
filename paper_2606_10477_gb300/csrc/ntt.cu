// Batched negacyclic NTT / inverse NTT over RNS limbs: dispatch, the launch-shape autotuner and the
// register-only butterfly rate.  The kernels and their launch shapes are in ntt_impl.cuh (see its
// header comment); their instantiations per ring size are in ntt_inst_*.cu.
#include "ntt_impl.cuh"

namespace hedap {

void ntt_launch_10_11(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                      const NttAux& A, const KskFuse* F);
void ntt_launch_12_13(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                      const NttAux& A, const KskFuse* F);
void ntt_launch_14_15(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                      const NttAux& A, const KskFuse* F);
void ntt_launch_16(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                   const NttAux& A, const KskFuse* F);
void ntt_launch_17(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                   const NttAux& A, const KskFuse* F);
void ntt_launch(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                const NttAux& A, const KskFuse* F) {
  switch (log_n) {
    case 10: case 11: ntt_launch_10_11(log_n, v, S, T, st, inverse, A, F); break;
    case 12: case 13: ntt_launch_12_13(log_n, v, S, T, st, inverse, A, F); break;
    case 14: case 15: ntt_launch_14_15(log_n, v, S, T, st, inverse, A, F); break;
    case 16: ntt_launch_16(log_n, v, S, T, st, inverse, A, F); break;
    case 17: ntt_launch_17(log_n, v, S, T, st, inverse, A, F); break;
    default: throw Error(HEDAP_ERR_ARG, "log_n must lie in [10, 17]");
  }
}

static void dispatch(const Tables& T, const LimbSet& S, cudaStream_t st, bool inverse, const NttAux* aux,
                     const KskFuse* F = nullptr) {
  if (S.n_parts * S.n_limbs == 0) return;
  const NttAux A = aux ? *aux : NttAux{};
  if (F && (inverse || !A.own_alpha || !A.z || A.fin_dst || !F->d || !F->key || !F->acc || !F->r64 ||
            F->batch < 1 || S.n_parts != F->batch * A.own_dn))
    throw Error(HEDAP_ERR_ARG, "NTT: bad key inner product fusion");
  if (A.own_alpha && (A.own_dn < 1 || A.own_alpha > 8)) throw Error(HEDAP_ERR_ARG, "NTT: bad digit layout");
  if (A.z && (inverse || !A.own_alpha || !A.bconv || !A.bconv_sh_offset)) throw Error(HEDAP_ERR_ARG, "NTT: bad ModUp fusion");
  if (A.post && !inverse) throw Error(HEDAP_ERR_ARG, "NTT: post factors apply to the inverse only");
  if ((A.spread || A.fin_dst || A.pconv) && inverse)
    throw Error(HEDAP_ERR_ARG, "NTT: fused rescale / ModDown applies to the forward only");
  if (A.pconv && (A.pconv_K < 1 || A.pconv_K > 8 || A.z || A.src || (A.spread && !A.fin_e)))
    throw Error(HEDAP_ERR_ARG, "NTT: bad ModDown fusion");
  if (A.fin_e && (!A.fin_dst || !A.fin_w2 || !A.fin_w2sh || !A.pconv || !A.spread))
    throw Error(HEDAP_ERR_ARG, "NTT: bad ModDown-rescale fusion");
  if (A.spread && (A.z || A.src || !A.spread_sub)) throw Error(HEDAP_ERR_ARG, "NTT: bad spread fusion");
  if (A.fin_dst && (!A.fin_c || !A.fin_w || !A.fin_wsh)) throw Error(HEDAP_ERR_ARG, "NTT: bad epilogue fusion");
  const int v = inverse ? T.ntt_inv_variant
                        : A.z ? T.ntt_modup_variant
                              : (A.pconv || A.spread || A.fin_dst) ? T.ntt_fin_variant : T.ntt_fwd_variant;
  // algorithmic bytes: each transformed limb read once and written once (a digit's own limbs are skipped)
  const double limbs = (double)S.n_parts * S.n_limbs - (A.own_alpha ? (double)S.n_parts / A.own_dn * A.own_limit : 0.0);
  const double n = (double)((size_t)1 << T.log_n);
  ProfScope prof_(PROF_NTT, st, 16.0 * limbs * n);
  // algorithmic multiply work in 32-bit multiply-pipe slots (one 32 x 32 -> 32 product, low or high half):
  // a Shoup product by a constant is 7 half products for the exact high half of x w' and 2 wide (2 slots each)
  // plus 4 low products for x w - qh q = 15 slots; every butterfly has one, and so does every product of a
  // fused basis conversion (ModUp: one per digit limb, less a factor folded into the key; ModDown: K per word);
  // the fused key inner product multiplies every word of every digit by two key words, a full 64 x 64 ->
  // 128-bit product of 8 half products = 8 slots each
  double shoup = limbs * n / 2 * T.log_n;
  if (A.z) shoup += A.z_products >= 0 ? A.z_products : limbs * n * std::min(A.own_alpha, A.own_limit);
  if (A.pconv) shoup += limbs * n * A.pconv_K;
  prof_.slots = 15.0 * shoup;
  if (F) prof_.slots += 8.0 * 2.0 * F->batch * (double)S.n_limbs * A.own_dn * n;
  prof_count_launches(2);
  ntt_launch(T.log_n, v, S, T, st, inverse, A, F);
}

void ntt_forward(const Tables& T, const LimbSet& S, cudaStream_t st, const NttAux* aux, const KskFuse* fuse) {
  dispatch(T, S, st, false, aux, fuse);
}
void ntt_inverse(const Tables& T, const LimbSet& S, cudaStream_t st, const NttAux* aux) {
  dispatch(T, S, st, true, aux);
}

// Register-only loop of the transform's butterfly (the rate the integer pipes allow without any
// memory or shared-memory traffic): each thread runs `iters` rounds (even, alternating the even-
// and odd-stage forms) of 4 independent lazy Cooley-Tukey butterflies on 8 residues of the
// context's first prime and stores one word.
__global__ void k_butterfly_loop(const Tables T, u64* out, int iters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const u64 q = T.pr[0].q;
  const ulonglong2 w = T.psi2[1 + (threadIdx.x & 63)];
  u64 v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = ((u64)i * 8 + m) % q;
  for (int it = 0; it < iters; it += 2) {  // an even and an odd stage
#pragma unroll
    for (int m = 0; m < 4; ++m) ct_bfly<true>(v[m], v[m + 4], w, q);
#pragma unroll
    for (int m = 0; m < 4; ++m) ct_bfly<false>(v[m], v[m + 4], w, q);
  }
  u64 s = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m) s ^= v[m];
  out[i] = s;
}
double butterfly_rate(Ctx& C) {
  int sms = 0;
  HEDAP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, C.device));
  const int threads = 256, blocks = sms * 8, iters = 512;
  DevBuf out((size_t)threads * blocks, C.stream);
  cudaEvent_t a, b;
  HEDAP_CUDA(cudaEventCreate(&a));
  HEDAP_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    HEDAP_CUDA(cudaEventRecord(a, C.stream));
    k_butterfly_loop<<<blocks, threads, 0, C.stream>>>(C.tab, out.p, iters);
    HEDAP_LAUNCH_CHECK();
    HEDAP_CUDA(cudaEventRecord(b, C.stream));
    HEDAP_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    HEDAP_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (r > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  prof_count_launches(3);
  return (double)threads * blocks * iters * 4 / (best / 1e3);
}

int& ntt_role_variant(Tables& T, int role) {
  switch (role) {
    case NTT_ROLE_FORWARD: return T.ntt_fwd_variant;
    case NTT_ROLE_INVERSE: return T.ntt_inv_variant;
    case NTT_ROLE_MODUP: return T.ntt_modup_variant;
    case NTT_ROLE_FINISH: return T.ntt_fin_variant;
    default: throw Error(HEDAP_ERR_ARG, "unknown NTT role");
  }
}

// Time every variant on `limbs` limbs of scratch (forward and inverse separately, best of `reps` after
// one warm-up) and keep the fastest in C.tab.  The fused roles run other code around the same passes
// (the ModUp conversion, the ModDown / rescale finish), and the shape that suits the plain transform
// need not suit them, so when the relinearisation key exists they are tuned on what they serve: an
// HMult with rescale of a batch of 4 at the top level (tensor, key switch, ModDown fused with the
// rescale), timed for every shape of one role with the other roles fixed.
void ntt_tune(Ctx& C, int limbs, int reps, std::vector<float>* fwd_ms, std::vector<float>* inv_ms) {
  const int n = std::max(1, std::min(limbs / C.n_q, 65535 / std::max(1, C.n_q)));
  DevBuf buf((size_t)n * C.n_q * C.N, C.stream);
  HEDAP_CUDA(cudaMemsetAsync(buf.p, 0, buf.words * 8, C.stream));
  const LimbSet S{buf.p, (size_t)C.n_q * C.N, n, 0, C.n_q, INT_MAX, 0, 0};
  cudaEvent_t a, b;
  HEDAP_CUDA(cudaEventCreate(&a));
  HEDAP_CUDA(cudaEventCreate(&b));
  auto best_of = [&](const std::function<void()>& run) {
    float ms = 1e30f;
    for (int r = 0; r <= reps; ++r) {
      HEDAP_CUDA(cudaEventRecord(a, C.stream));
      run();
      HEDAP_CUDA(cudaEventRecord(b, C.stream));
      HEDAP_CUDA(cudaEventSynchronize(b));
      float t = 0;
      HEDAP_CUDA(cudaEventElapsedTime(&t, a, b));
      if (r > 0) ms = std::min(ms, t);
    }
    return ms;
  };
  for (int dir = 0; dir < 2; ++dir) {
    float best = 1e30f;
    int best_v = 0;
    for (int v = 0; v < kNttVariants; ++v) {
      Tables T = C.tab;
      T.ntt_fwd_variant = T.ntt_inv_variant = v;
      const float ms = best_of([&] { dispatch(T, S, C.stream, dir == 1, nullptr); });
      if (dir == 0 && fwd_ms) fwd_ms->push_back(ms);
      if (dir == 1 && inv_ms) inv_ms->push_back(ms);
      if (ms < best) { best = ms; best_v = v; }
    }
    if (dir == 0) C.tab.ntt_fwd_variant = best_v;
    else C.tab.ntt_inv_variant = best_v;
  }
  C.tab.ntt_modup_variant = C.tab.ntt_fin_variant = C.tab.ntt_fwd_variant;
  if (C.keys.count(0) && C.L() >= 1) {
    const int l = C.L(), batch = 4;
    auto ct = ct_alloc(C, l, batch);
    HEDAP_CUDA(cudaMemsetAsync(ct->buf.p, 0, ct->buf.words * 8, C.stream));
    for (int role : {NTT_ROLE_MODUP, NTT_ROLE_FINISH}) {
      int& slot = ntt_role_variant(C.tab, role);
      float best = 1e30f;
      int best_v = slot;
      for (int v = 0; v < kNttVariants; ++v) {
        slot = v;
        const float ms = best_of([&] { ev_mul(C, *ct, *ct); });
        if (ms < best) { best = ms; best_v = v; }
      }
      slot = best_v;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
}

}  // namespace hedap
