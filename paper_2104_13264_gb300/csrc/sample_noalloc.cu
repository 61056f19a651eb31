// tnmc_sample_noalloc: the SIMT sampler of tnmc_sample, run with its per-thread
// right-vector stacks in a fixed, file-scope device array instead of memory the
// library allocates.
//
// Why: tnmc_sample grows its scratch with cudaMallocAsync / cudaFreeAsync the
// first time it needs more.  Some callers must not have the library allocate:
// code that runs under a fixed device-memory budget owned by another allocator,
// and latency-sensitive loops where an allocation (or the device-wide
// synchronisation a cudaFree implies) is not acceptable.  This entry point
// allocates nothing; the caller still passes every input and output.
//
// The scratch is one static __device__ array of kNoAllocScratchBytes.  Every GPU
// that loads the library holds it until the process exits.  All calls on a device
// share it, and it keeps the previous call's contents: calls that overlap on the
// GPU (two streams, or two threads) race and must be ordered by the caller.  The
// kernel writes every scratch word before it reads it, so nothing has to be
// cleared between calls.
//
// Host code cannot use the array's name as a device address (in host code it is
// a host-side stand-in).  The first call on each device therefore looks the
// address up with cudaGetSymbolAddress while that device is current and caches
// it; make that first call before any stream capture.
#include <mutex>

#include "common.cuh"
#include "sample_simt_kernel.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device (set-up on first use).
tnmc_status scratch_address(void** out) {
  int dev = 0;
  TNMC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    tnmc_set_error("device ordinal %d is beyond the %d devices tnmc_sample_noalloc supports", dev, kMaxDevices);
    return TNMC_E_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      tnmc_set_error("cudaGetSymbolAddress of the no-alloc scratch failed on device %d: %s", dev,
                     cudaGetErrorString(e));
      return TNMC_E_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TNMC_OK;
}

template <typename T, int NT>
tnmc_status launch_noalloc(const tnmc_env* env, const T* L, const T* R, const T* fe, int64_t B, uint64_t seed,
                           uint64_t offset, int8_t* spins, double* logq, double* energy, int32_t* flags,
                           cudaStream_t stream) {
  using namespace tnmc;
  const DeviceEnv& d = env->d;
  const size_t per_cta = (size_t)(d.Lx + 1) * d.P * NT * sizeof(T);
  if (per_cta > kNoAllocScratchBytes) {
    tnmc_set_error("tnmc_sample_noalloc: one CTA needs %zu bytes of scratch for this %d x %d lattice "
                   "(chi padding %d) but the fixed scratch holds %zu bytes; use tnmc_sample",
                   per_cta, d.Ly, d.Lx, d.P, kNoAllocScratchBytes);
    return TNMC_E_INVALID_ARG;
  }
  void* scratch = nullptr;
  tnmc_status st = scratch_address(&scratch);
  if (st != TNMC_OK) return st;
  const int W = (d.Lx + 31) / 32;
  const size_t smem = (size_t)3 * d.P * NT * sizeof(T) + (size_t)2 * W * NT * sizeof(uint32_t);
  auto kern = sample_simt_kernel<T, NT>;
  int dev = 0, nsm = 0, max_optin = 0;
  TNMC_CUDA_TRY(cudaGetDevice(&dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)max_optin) {
    tnmc_set_error("sampler needs %zu bytes of shared memory per CTA (device allows %d)", smem, max_optin);
    return TNMC_E_UNSUPPORTED;
  }
  TNMC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TNMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = (B + NT - 1) / NT;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  const int64_t fit = (int64_t)(kNoAllocScratchBytes / per_cta);   // CTAs whose stacks fit
  if (grid > fit) grid = fit;
  if (grid < 1) grid = 1;
  SampleArgs<T> a;
  a.e = d;
  a.L = L;
  a.Rt = R;
  a.fe = fe;
  a.B = B;
  a.seed = seed;
  a.offset = offset;
  a.spins_in = nullptr;
  a.spins_out = spins;
  a.logq = logq;
  a.energy = energy;
  a.flags = flags;
  a.scratch = static_cast<T*>(scratch);
  kern<<<(unsigned)grid, NT, smem, stream>>>(a);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

}  // namespace

extern "C" tnmc_status tnmc_sample_noalloc(const tnmc_env* env, int precision, int64_t B, uint64_t seed,
                                           uint64_t sample_offset, int8_t* spins, double* logq, double* energy,
                                           int32_t* flags, void* stream) {
  tnmc_set_error("%s", "");
  if (!env) {
    tnmc_set_error("env must be non-null");
    return TNMC_E_INVALID_ARG;
  }
  if (B < 0 || (B > 0 && !(spins && logq && energy))) {
    tnmc_set_error("B must be >= 0 and spins, logq, energy non-null");
    return TNMC_E_INVALID_ARG;
  }
  if (precision != TNMC_F64 && precision != TNMC_F32) {
    tnmc_set_error("tnmc_sample_noalloc supports TNMC_F64 and TNMC_F32 only");
    return TNMC_E_UNSUPPORTED;
  }
  if (!(env->precision_mask & (1 << precision))) {
    tnmc_set_error("the env was built without the sampler copy for precision %d", precision);
    return TNMC_E_UNSUPPORTED;
  }
  if (B == 0) return TNMC_OK;
  const tnmc::DeviceEnv& d = env->d;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == TNMC_F64)
    return launch_noalloc<double, 64>(env, d.M64, d.R64, d.fe, B, seed, sample_offset, spins, logq, energy, flags, s);
  return launch_noalloc<float, 128>(env, d.L32, d.R32, d.fe32, B, seed, sample_offset, spins, logq, energy, flags, s);
}
