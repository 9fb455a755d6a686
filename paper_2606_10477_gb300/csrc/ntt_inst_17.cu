// Instantiations of the transform kernels for N = 2^17 (see ntt_impl.cuh).
#include "ntt_impl.cuh"

namespace hedap {

void ntt_launch_17(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                   const NttAux& A, const KskFuse* F) {
  switch (log_n) {
    case 17: launch_variant<8, 9>(v, S, T, st, inverse, A, F); break;
    default: throw Error(HEDAP_ERR_ARG, "ring size not instantiated in this unit");
  }
}

}  // namespace hedap
