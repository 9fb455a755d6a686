// Instantiations of the transform kernels for N = 2^14/2^15 (see ntt_impl.cuh).
#include "ntt_impl.cuh"

namespace hedap {

void ntt_launch_14_15(int log_n, int v, const LimbSet& S, const Tables& T, cudaStream_t st, bool inverse,
                      const NttAux& A, const KskFuse* F) {
  switch (log_n) {
    case 14: launch_variant<7, 7>(v, S, T, st, inverse, A, F); break;
    case 15: launch_variant<7, 8>(v, S, T, st, inverse, A, F); break;
    default: throw Error(HEDAP_ERR_ARG, "ring size not instantiated in this unit");
  }
}

}  // namespace hedap
