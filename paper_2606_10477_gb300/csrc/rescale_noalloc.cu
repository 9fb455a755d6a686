// Rescale for callers that must not allocate device memory.
//
// hedap_rescale allocates its temporaries (the last limb in coefficient form
// and the spread residues) from the device memory pool.  Some callers cannot
// let an operation do that: a serving loop that admitted its requests against
// a fixed HBM budget (keys and ciphertexts resident) must not have an operation
// take extra device memory mid-request; a host framework whose own allocator
// owns the device memory cannot have a library allocate behind its back; and
// a cudaMalloc/cudaFree can synchronise the device and stall other streams.
// This variant takes device pointers for its input and output and keeps its
// scratch in one file-scope device array.
//
// When the array comes into being: this file is its own CUDA module (it is
// compiled apart from the kernels, without relocatable device code), and the
// runtime loads a module lazily, on the first use of something in it.  The
// first use is the cudaGetSymbolAddress below, which context creation calls
// with the context's device current; so the 32 MiB are allocated on a device
// when the first context is created there, and held until the process exits.
// hedap_rescale_noalloc itself only reads the address cached in the context.
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "kernels.cuh"

namespace {

using hedap::u64;

// 4 Mi words = 32 MiB: room for (2 + 2*level) limbs of N words, e.g. level <= 31 at N = 2^16.
constexpr size_t kScratchWords = (size_t)1 << 22;
static __device__ __align__(256) u64 g_rescale_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
u64* g_addr[kMaxDevices] = {};

}  // namespace

namespace hedap {

// Device address of the scratch array on `device`, which must be the current device.  The array's
// name is only a host-side stand-in, so the address is looked up once per device, with that device
// current, and cached.
u64* noalloc_scratch_address(int device) {
  int cur = -1;
  HEDAP_CUDA(cudaGetDevice(&cur));
  if (cur != device) throw Error(HEDAP_ERR_ARG, "scratch lookup: the device is not current");
  if (device < 0 || device >= kMaxDevices) throw Error(HEDAP_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rescale_scratch);
    if (e != cudaSuccess || !p)
      throw Error(HEDAP_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_addr[device] = (u64*)p;
  }
  return g_addr[device];
}

}  // namespace hedap

extern "C" __attribute__((visibility("default"))) hedap_status hedap_rescale_noalloc(hedap_ctx* ctx,
                                                                                       const uint64_t* in, int level,
                                                                                       uint64_t* out) {
  if (!ctx || !in || !out) {
    hedap::set_last_error("hedap_rescale_noalloc: null argument");
    return HEDAP_ERR_ARG;
  }
  return hedap::run_on_ctx(ctx, [&] {
    hedap::Ctx& C = hedap::ctx_of(ctx);
    if (level < 1 || level > C.L()) throw hedap::Error(HEDAP_ERR_LEVEL, "rescale needs 1 <= level <= L");
    const size_t N = C.N, l = (size_t)level;
    const size_t need = (2 + 2 * l) * N;
    if (need > kScratchWords)
      throw hedap::Error(HEDAP_ERR_ARG, "hedap_rescale_noalloc: (2 + 2*level) * N = " + std::to_string(need) +
                                           " words exceeds the scratch maximum of " + std::to_string(kScratchWords));
    // [in, in + 2(l+1)N) and [out, out + 2lN) must be disjoint: the last kernel reads one and writes the other
    const uintptr_t i0 = (uintptr_t)in, i1 = i0 + 2 * (l + 1) * N * 8, o0 = (uintptr_t)out, o1 = o0 + 2 * l * N * 8;
    if (i0 < o1 && o0 < i1) throw hedap::Error(HEDAP_ERR_ARG, "hedap_rescale_noalloc: out overlaps in");
    int cur = -1;
    HEDAP_CUDA(cudaGetDevice(&cur));
    if (cur != C.device)
      throw hedap::Error(HEDAP_ERR_ARG, "hedap_rescale_noalloc: the context's device is not the current device");
    u64* scratch = C.noalloc_scratch;
    if (!scratch) throw hedap::Error(HEDAP_ERR_CUDA, "hedap_rescale_noalloc: scratch address not set up");
    u64* last = scratch;          // [2][N]: limb `level` of each part, coefficient domain
    u64* tmp = scratch + 2 * N;   // [2][level][N]: centred residues, then their NTT
    // every word of last and tmp is written before it is read: nothing to clear
    for (int p = 0; p < 2; ++p)
      HEDAP_CUDA(cudaMemcpyAsync(last + p * N, in + (p * (l + 1) + l) * N, N * 8, cudaMemcpyDeviceToDevice,
                                 C.stream));
    hedap::ntt_inverse(C.tab, hedap::LimbSet{last, N, 2, 0, 1, INT_MAX, level, 0}, C.stream);
    hedap::RescaleConsts R;
    const u64 ql = C.primes[l];
    for (size_t i = 0; i < l; ++i) {
      const u64 qi = C.primes[i];
      R.ql_mod[i] = ql % qi;
      R.inv[i] = hedap::h_invmod(ql % qi, qi);
      R.inv_sh[i] = hedap::h_shoup(R.inv[i], qi);
    }
    hedap::k_rescale_spread(C, last, N, tmp, l * N, 2, level, R);
    hedap::ntt_forward(C.tab, hedap::LimbSet{tmp, l * N, 2, 0, level, INT_MAX, 0, 0}, C.stream);
    hedap::k_rescale_finish(C, in, (l + 1) * N, tmp, l * N, out, l * N, 2, level, R);
  });
}
