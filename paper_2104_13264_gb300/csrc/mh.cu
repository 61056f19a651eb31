// Metropolis-Hastings scan (eq. mh-acc with the independence prior of eq.
// tns-prior; Algorithm 1) and the random start of the chains.
#include <math.h>

#include "common.cuh"

namespace tnmc {
namespace {

// One thread per chain, sequential over its T proposals (proposal t = i*T + j).
__global__ void mh_scan_kernel(int64_t C, int64_t T, double beta, const double* __restrict__ prop_logq,
                               const double* __restrict__ prop_E, double* chain_logq, double* chain_E,
                               uint64_t seed, uint64_t step_offset, uint8_t* accepted, int64_t* last,
                               int64_t* n_accepted) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= C) return;
  double lq = chain_logq[i], E = chain_E[i];
  int64_t lastt = -1, cnt = 0;
  for (int64_t j = 0; j < T; ++j) {
    const int64_t t = i * T + j;
    const double u = mh_uniform(seed, step_offset + (uint64_t)j, (uint32_t)i);
    const double lqt = prop_logq[t], Et = prop_E[t];
    const double d = -beta * (Et - E) + (lq - lqt);
    const bool ok = isfinite(lqt) && !isnan(d);
    // a state with log q = -inf (only a random start can be one) takes the first valid proposal
    const bool acc = ok && (lq == -INFINITY || u < exp(fmin(d, 0.0)));
    if (accepted) accepted[t] = acc ? 1 : 0;
    if (acc) {
      lq = lqt;
      E = Et;
      lastt = t;
      ++cnt;
    }
  }
  chain_logq[i] = lq;
  chain_E[i] = E;
  last[i] = lastt;
  if (n_accepted && cnt) atomicAdd(reinterpret_cast<unsigned long long*>(n_accepted), (unsigned long long)cnt);
}

// Copy the last accepted proposal of each chain into the chain state (one CTA per chain).
__global__ void mh_copy_kernel(int64_t C, int64_t n, const int64_t* last, const int8_t* __restrict__ prop,
                               int8_t* chain) {
  for (int64_t i = blockIdx.x; i < C; i += gridDim.x) {
    const int64_t t = last[i];
    if (t < 0) continue;
    const int8_t* src = prop + t * n;
    int8_t* dst = chain + i * n;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 && (n & 15) == 0;
    if (vec) {
      const int4* s4 = reinterpret_cast<const int4*>(src);
      int4* d4 = reinterpret_cast<int4*>(dst);
      for (int64_t k = threadIdx.x; k < n / 16; k += blockDim.x) d4[k] = s4[k];
    } else {
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
    }
  }
}

// Random +-1 start: spin = +1 iff bit (site % 128) of Philox(site / 128, i_lo, i_hi, 2) is set.
__global__ void init_bits_kernel(int64_t C, int64_t n, uint64_t seed, int8_t* spins) {
  const int64_t total = C * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / n, site = idx % n;
    U4 c{(uint32_t)(site >> 7), (uint32_t)i, (uint32_t)((uint64_t)i >> 32), 2u};
    const U4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const int j = (int)(site & 127);
    const uint32_t word = (j < 32) ? o.x : (j < 64) ? o.y : (j < 96) ? o.z : o.w;
    spins[idx] = ((word >> (j & 31)) & 1u) ? 1 : -1;
  }
}

}  // namespace
}  // namespace tnmc

tnmc_status tnmc_launch_mh_core(int64_t n, double beta, const tnmc::Allocator& alloc, int64_t C, int64_t T,
                                const int8_t* prop_spins, const double* prop_logq, const double* prop_energy,
                                int8_t* chain_spins, double* chain_logq, double* chain_energy, uint64_t seed,
                                uint64_t step_offset, uint8_t* accepted, int64_t* n_accepted, cudaStream_t stream) {
  using namespace tnmc;
  if (C == 0 || T == 0) return TNMC_OK;
  int64_t* last = static_cast<int64_t*>(dev_alloc(alloc, C * sizeof(int64_t), stream));
  if (!last) {
    tnmc_set_error("cannot allocate %zu bytes for the MH scan", (size_t)C * sizeof(int64_t));
    return TNMC_E_NOMEM;
  }
  const int threads = 128;
  const int64_t blocks = (C + threads - 1) / threads;
  mh_scan_kernel<<<(unsigned)blocks, threads, 0, stream>>>(C, T, beta, prop_logq, prop_energy, chain_logq,
                                                           chain_energy, seed, step_offset, accepted, last,
                                                           n_accepted);
  TNMC_CUDA_TRY(cudaGetLastError());
  const int64_t cb = C < 65535 ? C : 65535;
  mh_copy_kernel<<<(unsigned)cb, 256, 0, stream>>>(C, n, last, prop_spins, chain_spins);
  TNMC_CUDA_TRY(cudaGetLastError());
  dev_free(alloc, last, C * sizeof(int64_t), stream);
  return TNMC_OK;
}

tnmc_status tnmc_launch_mh(const tnmc_env* env, int64_t C, int64_t T, const int8_t* prop_spins,
                           const double* prop_logq, const double* prop_energy, int8_t* chain_spins,
                           double* chain_logq, double* chain_energy, uint64_t seed, uint64_t step_offset,
                           uint8_t* accepted, int64_t* n_accepted, cudaStream_t stream) {
  return tnmc_launch_mh_core((int64_t)env->d.Lx * env->d.Ly, env->d.beta, env->alloc, C, T, prop_spins, prop_logq,
                             prop_energy, chain_spins, chain_logq, chain_energy, seed, step_offset, accepted,
                             n_accepted, stream);
}

tnmc_status tnmc_launch_init_bits_core(int64_t n, int64_t C, uint64_t seed, int8_t* spins, cudaStream_t stream) {
  using namespace tnmc;
  if (C == 0) return TNMC_OK;
  init_bits_kernel<<<1024, 256, 0, stream>>>(C, n, seed, spins);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_launch_init_bits(const tnmc_env* env, int64_t C, uint64_t seed, int8_t* spins,
                                  cudaStream_t stream) {
  return tnmc_launch_init_bits_core((int64_t)env->d.Lx * env->d.Ly, C, seed, spins, stream);
}
