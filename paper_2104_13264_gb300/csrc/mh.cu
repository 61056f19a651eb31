// Metropolis-Hastings scan (eq. mh-acc with the independence prior of eq.
// tns-prior; Algorithm 1) and the random start of the chains.
#include <math.h>

#include "common.cuh"

namespace tnmc {
namespace {

// u < exp(min(0, d)) (eq. mh-acc), decided without the FP64 exp wherever the answer is
// already certain, with the same result as evaluating it:
//   d >= 0: exp(0) = 1 > u (u <= 1 - 2^-53) -- accept;
//   d < -40, u > 0: exp(d) < 4.3e-18 < 2^-53 <= u -- reject;
//   otherwise the FP32 exp of d is within 3e-6 relative of exp(d) (expf is within 2 ulp, and
//   rounding |d| <= 40 to float moves exp(d) by at most 2.4e-6 relative), so a u outside
//   e (1 -+ 1e-5) falls on the same side as for exp(d); u inside that band (and u = 0) goes
//   to the FP64 exp.
__device__ __forceinline__ bool mh_below(double u, double d) {
  if (d >= 0.0) return true;
  if (u > 0.0) {
    if (d < -40.0) return false;
    const double e = (double)expf((float)d);
    if (u < e * (1.0 - 1e-5)) return true;
    if (u > e * (1.0 + 1e-5)) return false;
  }
  return u < exp(d);
}

// The MH uniforms of every (chain, proposal), drawn in parallel: they do not depend on the
// chain state, so the sequential scan below only carries the dependent arithmetic.
// Also the log target-over-proposal weight a = -beta E - log q of every proposal (rounded
// once each step, no contraction), so that Delta = a(prop) - a(cur) is one subtraction.
__device__ __forceinline__ double mh_weight(double beta, double E, double lq) {
  return __dsub_rn(__dmul_rn(-beta, E), lq);
}

__global__ void mh_uniforms_kernel(int64_t C, int64_t T, uint64_t seed, uint64_t step_offset, double beta,
                                   const double* __restrict__ prop_logq, const double* __restrict__ prop_E,
                                   double* u, double* w) {
  const int64_t total = C * T;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / T, j = t % T;
    u[t] = mh_uniform(seed, step_offset + (uint64_t)j, (uint32_t)i);
    w[t] = mh_weight(beta, prop_E[t], prop_logq[t]);
  }
}

// One thread per chain, sequential over its T proposals (proposal t = i*T + j), with the
// uniforms u[t] precomputed.
__global__ void mh_scan_kernel(int64_t C, int64_t T, double beta, const double* __restrict__ prop_logq,
                               const double* __restrict__ prop_E, const double* __restrict__ u_all,
                               const double* __restrict__ w_all, double* __restrict__ chain_logq,
                               double* __restrict__ chain_E, uint8_t* __restrict__ accepted,
                               int64_t* __restrict__ last, int64_t* n_accepted) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= C) return;
  double lq = chain_logq[i], E = chain_E[i];
  double wc = mh_weight(beta, E, lq);
  int64_t lastt = -1, cnt = 0;
#pragma unroll 4
  for (int64_t j = 0; j < T; ++j) {
    const int64_t t = i * T + j;
    const double u = u_all[t];
    const double lqt = prop_logq[t], Et = prop_E[t], wt = w_all[t];
    const double d = __dsub_rn(wt, wc);
    const bool ok = isfinite(lqt) && !isnan(d);
    // a state with log q = -inf (only a random start can be one) takes the first valid proposal
    const bool acc = ok && (lq == -INFINITY || mh_below(u, d));
    if (accepted) accepted[t] = acc ? 1 : 0;
    if (acc) {
      lq = lqt;
      E = Et;
      wc = wt;
      lastt = t;
      ++cnt;
    }
  }
  chain_logq[i] = lq;
  chain_E[i] = E;
  last[i] = lastt;
  if (n_accepted && cnt) atomicAdd(reinterpret_cast<unsigned long long*>(n_accepted), (unsigned long long)cnt);
}

// The same scan with one warp per chain: the lanes load 32 proposals at a time, each
// proposal's values are broadcast by shuffle, and every lane takes the decision with the
// arithmetic of mh_scan_kernel (so the decisions are identical); the loads of a block of
// 32 proceed together instead of one at a time on the dependent chain.
__global__ void mh_scan_warp_kernel(int64_t C, int64_t T, double beta, const double* __restrict__ prop_logq,
                                    const double* __restrict__ prop_E, const double* __restrict__ u_all,
                                    const double* __restrict__ w_all,
                                    double* __restrict__ chain_logq, double* __restrict__ chain_E,
                                    uint8_t* __restrict__ accepted, int64_t* __restrict__ last,
                                    int64_t* n_accepted) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= C) return;      // warp-uniform
  double lq = chain_logq[i], E = chain_E[i];
  double wc = mh_weight(beta, E, lq);
  int64_t lastt = -1, cnt = 0;
  for (int64_t base = 0; base < T; base += 32) {
    const int64_t n = (T - base) < 32 ? (T - base) : 32;
    const int64_t tl = i * T + base + lane;
    double ul = 0.0, lql = 0.0, El = 0.0, wl = 0.0;
    if (lane < n) {
      ul = u_all[tl];
      lql = prop_logq[tl];
      El = prop_E[tl];
      wl = w_all[tl];
    }
    for (int k = 0; k < (int)n; ++k) {
      const double u = __shfl_sync(0xffffffffu, ul, k);
      const double lqt = __shfl_sync(0xffffffffu, lql, k);
      const double Et = __shfl_sync(0xffffffffu, El, k);
      const double wt = __shfl_sync(0xffffffffu, wl, k);
      const double d = __dsub_rn(wt, wc);
      const bool ok = isfinite(lqt) && !isnan(d);
      const bool acc = ok && (lq == -INFINITY || mh_below(u, d));
      if (accepted && lane == k) accepted[tl] = acc ? 1 : 0;
      if (acc) {
        lq = lqt;
        E = Et;
        wc = wt;
        lastt = i * T + base + k;
        ++cnt;
      }
    }
  }
  if (lane == 0) {
    chain_logq[i] = lq;
    chain_E[i] = E;
    last[i] = lastt;
    if (n_accepted && cnt) atomicAdd(reinterpret_cast<unsigned long long*>(n_accepted), (unsigned long long)cnt);
  }
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
  const size_t bytes = (size_t)C * sizeof(int64_t) + (size_t)C * T * 2 * sizeof(double);
  char* buf = static_cast<char*>(dev_alloc(alloc, bytes, stream));
  if (!buf) {
    tnmc_set_error("cannot allocate %zu bytes for the MH scan", bytes);
    return TNMC_E_NOMEM;
  }
  double* u = reinterpret_cast<double*>(buf);
  double* w = u + (size_t)C * T;
  int64_t* last = reinterpret_cast<int64_t*>(buf + (size_t)C * T * 2 * sizeof(double));
  mh_uniforms_kernel<<<1024, 256, 0, stream>>>(C, T, seed, step_offset, beta, prop_logq, prop_energy, u, w);
  TNMC_CUDA_TRY(cudaGetLastError());
  const int threads = 128;
  if (C <= 65536) {   // one warp per chain
    const int64_t blocks = (C * 32 + threads - 1) / threads;
    mh_scan_warp_kernel<<<(unsigned)blocks, threads, 0, stream>>>(C, T, beta, prop_logq, prop_energy, u, w,
                                                                  chain_logq, chain_energy, accepted, last, n_accepted);
  } else {            // one thread per chain
    const int64_t blocks = (C + threads - 1) / threads;
    mh_scan_kernel<<<(unsigned)blocks, threads, 0, stream>>>(C, T, beta, prop_logq, prop_energy, u, w, chain_logq,
                                                             chain_energy, accepted, last, n_accepted);
  }
  TNMC_CUDA_TRY(cudaGetLastError());
  const int64_t cb = C < 65535 ? C : 65535;
  mh_copy_kernel<<<(unsigned)cb, 256, 0, stream>>>(C, n, last, prop_spins, chain_spins);
  TNMC_CUDA_TRY(cudaGetLastError());
  dev_free(alloc, buf, bytes, stream);
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
