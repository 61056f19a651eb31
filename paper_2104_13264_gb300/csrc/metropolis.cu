// Single-instance Metropolis sweeps of chain states and link overlaps of replica pairs
// (Sec. 3, "Equilibration"): tnmc_metropolis, tnmc_link_overlap.
#include "metropolis_kernel.cuh"

namespace tnmc {
namespace {

// One CTA per chain: the chain's spins in shared memory for all sweeps.
__global__ void metropolis_kernel(MetroInst I, int64_t C, int8_t* chains, uint64_t seed, uint64_t chain_offset,
                                  uint32_t sweep0, int sweeps) {
  extern __shared__ int8_t sm[];
  const int n = I.Lx * I.Ly;
  for (int64_t i = blockIdx.x; i < C; i += gridDim.x) {
    int8_t* g = chains + i * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) sm[k] = g[k];
    __syncthreads();
    metropolis_chain(I, sm, seed, (uint32_t)(chain_offset + (uint64_t)i), sweep0, sweeps);
    for (int k = threadIdx.x; k < n; k += blockDim.x) g[k] = sm[k];
    __syncthreads();
  }
}

__global__ void link_overlap_kernel(int Lx, int Ly, int64_t pairs, const int8_t* chains, double* out) {
  __shared__ long long red[32];
  const int64_t n = (int64_t)Lx * Ly;
  for (int64_t k = blockIdx.x; k < pairs; k += gridDim.x) {
    const double q = link_overlap_pair(Lx, Ly, chains + 2 * k * n, chains + (2 * k + 1) * n, red);
    if (threadIdx.x == 0) out[k] = q;
  }
}

}  // namespace
}  // namespace tnmc

tnmc_status tnmc_launch_metropolis(const tnmc_env* env, int64_t C, int8_t* chains, uint64_t seed,
                                   uint64_t chain_offset, uint64_t sweep_offset, int sweeps, cudaStream_t stream) {
  using namespace tnmc;
  if (C == 0 || sweeps == 0) return TNMC_OK;
  const DeviceEnv& d = env->d;
  MetroInst I{d.Jh, d.Jv, d.h, d.beta, d.Lx, d.Ly, 0};
  const size_t smem = (size_t)d.Lx * d.Ly;
  if (smem > 48 * 1024) TNMC_CUDA_TRY(cudaFuncSetAttribute(metropolis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)(C < 65535 ? C : 65535);
  metropolis_kernel<<<grid, 256, smem, stream>>>(I, C, chains, seed, chain_offset, (uint32_t)sweep_offset, sweeps);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_launch_link_overlap(int Lx, int Ly, int64_t pairs, const int8_t* chains, double* out,
                                     cudaStream_t stream) {
  using namespace tnmc;
  if (pairs == 0) return TNMC_OK;
  const unsigned grid = (unsigned)(pairs < 65535 ? pairs : 65535);
  link_overlap_kernel<<<grid, 256, 0, stream>>>(Lx, Ly, pairs, chains, out);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}
