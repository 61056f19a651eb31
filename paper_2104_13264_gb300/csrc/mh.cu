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

// The log target-over-proposal weight a = -beta E - log q of a state (each step rounded
// once, no contraction), so that Delta = a(prop) - a(cur) is one subtraction.
__device__ __forceinline__ double mh_weight(double beta, double E, double lq) {
  return __dsub_rn(__dmul_rn(-beta, E), lq);
}

// The rule itself, in FP64: proposal t of chain i against the current weight wc.  A state
// with log q = -inf (only a random start can be one) takes the first valid proposal.
__device__ __noinline__ bool mh_exact(double beta, uint64_t seed, uint64_t step, uint32_t chain, double lqt,
                                      double Et, double wc, bool start) {
  const double d = __dsub_rn(mh_weight(beta, Et, lqt), wc);
  const bool ok = isfinite(lqt) && !isnan(d);
  return ok && (start || mh_below(mh_uniform(seed, step, chain), d));
}

// Order-preserving map of the doubles (NaN excluded) onto int64: key(x) <= key(y) implies
// x <= y, and x < y implies key(x) < key(y).
__device__ __forceinline__ int64_t mh_key(double x) {
  const int64_t b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ INT64_MAX);
}
__device__ __forceinline__ double mh_unkey(int64_t k) { return __longlong_as_double(k >= 0 ? k : (k ^ INT64_MAX)); }

// Per proposal, in parallel (nothing here depends on the chain state): its weight key kt and
// an acceptance band on the current weight wc, so that the sequential scan decides with two
// integer compares:
//   key(wc) <= lo  -> accept,   key(wc) >= hi  -> reject,   otherwise the FP64 rule.
// With theta = a' - log u (the wc at which Delta = log u), lo = max(key(theta - m), kt),
// hi = key(theta + m), m = 1e-12 (1 + |theta|):
//   - wc <= a' gives Delta >= 0 (the rounded difference keeps the sign): accepted.
//   - |wc - theta| >= m puts Delta at least 9.9e-13 away from log u, while the roundings of
//     log u, theta and Delta and the error of exp (|log u| <= 36.8 since u >= 2^-53) sum to
//     below 1e-14, so u < exp(Delta) has the answer the side of theta says.
// A proposal with non-finite log q is never accepted (lo = hi = INT64_MIN); u = 0 or a
// non-finite weight leaves every wc to the FP64 rule (lo = INT64_MIN, hi = INT64_MAX).
__global__ void mh_bands_kernel(int64_t C, int64_t T, uint64_t seed, uint64_t step_offset, double beta,
                                const double* __restrict__ prop_logq, const double* __restrict__ prop_E,
                                int64_t* __restrict__ band_lo, int64_t* __restrict__ band_hi,
                                int64_t* __restrict__ key_w) {
  const int64_t total = C * T;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / T, j = t % T;
    const double lqt = prop_logq[t];
    const double wt = mh_weight(beta, prop_E[t], lqt);
    const int64_t kt = mh_key(wt);
    int64_t lo = INT64_MIN, hi = INT64_MIN;
    if (isfinite(lqt)) {
      const double u = mh_uniform(seed, step_offset + (uint64_t)j, (uint32_t)i);
      hi = INT64_MAX;
      if (isfinite(wt) && u > 0.0) {
        const double theta = wt - log(u);
        const double m = 1e-12 * (1.0 + fabs(theta));
        const int64_t kl = mh_key(theta - m);
        lo = kl > kt ? kl : kt;
        hi = mh_key(theta + m);
      }
    }
    band_lo[t] = lo;
    band_hi[t] = hi;
    key_w[t] = kt;
  }
}

// The state a chain carries through the scan: its weight key, and whether it sits at a
// random start (log q = -inf) or at a NaN weight, where every decision takes the FP64 rule
// until the first acceptance.
struct ScanState {
  int64_t kc;
  bool start, slow;
};

// Decides proposals j0 .. j0+cnt-1 (cnt <= kGrp) of one chain from their bands, held in
// registers.  A speculative pass takes every decision by the compares alone (a compare and
// a select per proposal on the dependent path); if one of them falls inside its band, or the
// chain is slow, the group is decided again from its entry state, with the FP64 rule where
// the band leaves it open.  Returns the group's acceptance bits.
constexpr int kGrp = 8;
__device__ __forceinline__ uint32_t mh_group(ScanState& st, const long long (&l)[kGrp], const long long (&h)[kGrp],
                                             const long long (&w)[kGrp], int cnt, double beta, uint64_t seed,
                                             uint64_t step0, uint32_t chain, const double* lq_row,
                                             const double* E_row) {
  int64_t kc = st.kc;
  bool unc = st.slow;
  uint32_t m = 0;
#pragma unroll
  for (int g = 0; g < kGrp; ++g) {
    const bool in = g < cnt;
    const bool a = in && kc <= l[g];
    unc |= in && !a && kc < h[g];
    kc = a ? w[g] : kc;
    m |= (uint32_t)a << g;
  }
  if (!unc) {
    st.kc = kc;
    return m;
  }
  kc = st.kc;
  m = 0;
#pragma unroll
  for (int g = 0; g < kGrp; ++g) {
    if (g < cnt) {
      bool a;
      if (!st.slow && kc <= l[g]) a = true;
      else if (!st.slow && kc >= h[g]) a = false;
      else a = mh_exact(beta, seed, step0 + (uint64_t)g, chain, lq_row[g], E_row[g], mh_unkey(kc), st.start);
      if (a) {
        kc = w[g];
        st.start = st.slow = false;
      }
      m |= (uint32_t)a << g;
    }
  }
  st.kc = kc;
  return m;
}

__device__ __forceinline__ ScanState mh_scan_start(double beta, double lq0, double E0) {
  const double w0 = mh_weight(beta, E0, lq0);
  ScanState st;
  st.kc = mh_key(w0);
  st.start = lq0 == -INFINITY;
  st.slow = st.start || isnan(w0);
  return st;
}

// One thread per chain, sequential over its T proposals (proposal t = i*T + j), in groups of
// kGrp whose bands are loaded together.
__global__ void mh_scan_kernel(int64_t C, int64_t T, double beta, uint64_t seed, uint64_t step_offset,
                               const double* __restrict__ prop_logq, const double* __restrict__ prop_E,
                               const int64_t* __restrict__ band_lo, const int64_t* __restrict__ band_hi,
                               const int64_t* __restrict__ key_w, double* __restrict__ chain_logq,
                               double* __restrict__ chain_E, uint8_t* __restrict__ accepted,
                               int64_t* __restrict__ last, int64_t* n_accepted) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= C) return;
  ScanState st = mh_scan_start(beta, chain_logq[i], chain_E[i]);
  const int64_t row = i * T;
  int64_t lastt = -1, cnt = 0;
  for (int64_t j0 = 0; j0 < T; j0 += kGrp) {
    const int n = (T - j0) < kGrp ? (int)(T - j0) : kGrp;
    long long l[kGrp], h[kGrp], w[kGrp];
#pragma unroll
    for (int g = 0; g < kGrp; ++g) {
      const bool in = g < n;
      l[g] = in ? band_lo[row + j0 + g] : 0;
      h[g] = in ? band_hi[row + j0 + g] : 0;
      w[g] = in ? key_w[row + j0 + g] : 0;
    }
    const uint32_t m = mh_group(st, l, h, w, n, beta, seed, step_offset + (uint64_t)j0, (uint32_t)i,
                                prop_logq + row + j0, prop_E + row + j0);
    if (m) {
      cnt += __popc(m);
      lastt = row + j0 + (31 - __clz(m));
    }
    if (accepted) {
#pragma unroll
      for (int g = 0; g < kGrp; ++g)
        if (g < n) accepted[row + j0 + g] = (m >> g) & 1u;
    }
  }
  if (lastt >= 0) {
    chain_logq[i] = prop_logq[lastt];
    chain_E[i] = prop_E[lastt];
  }
  last[i] = lastt;
  if (n_accepted && cnt) atomicAdd(reinterpret_cast<unsigned long long*>(n_accepted), (unsigned long long)cnt);
}

// The same scan with one warp per chain, for up to 65536 chains: the lanes load the bands of
// 128 proposals (4 per lane, coalesced) and stage them in the warp's shared memory; the next
// 128 are loaded while these are scanned.  Every lane runs the scan on the staged bands (the
// same values, read by broadcast), lanes 0-7 record each group's acceptance bits, and the
// flags of the 128 leave in one coalesced store.
constexpr int kScanR = 4;
constexpr int kScanWarps = 4;
__global__ void __launch_bounds__(32 * kScanWarps)
    mh_scan_warp_kernel(int64_t C, int64_t T, double beta, uint64_t seed, uint64_t step_offset,
                        const double* __restrict__ prop_logq, const double* __restrict__ prop_E,
                        const int64_t* __restrict__ band_lo, const int64_t* __restrict__ band_hi,
                        const int64_t* __restrict__ key_w, double* __restrict__ chain_logq,
                        double* __restrict__ chain_E, uint8_t* __restrict__ accepted,
                        int64_t* __restrict__ last, int64_t* n_accepted) {
  constexpr int kBlk = 32 * kScanR;
  __shared__ long long s_band[kScanWarps][3][kBlk];
  __shared__ uint8_t s_acc[kScanWarps][kBlk];
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (i >= C) return;      // warp-uniform
  ScanState st = mh_scan_start(beta, chain_logq[i], chain_E[i]);
  int64_t lastt = -1, cnt = 0;
  const int64_t row = i * T;
  long long lo[kScanR], hi[kScanR], kt[kScanR];
#pragma unroll
  for (int r = 0; r < kScanR; ++r) {
    const int64_t j = r * 32 + lane;
    const bool in = j < T;
    lo[r] = in ? band_lo[row + j] : 0;
    hi[r] = in ? band_hi[row + j] : 0;
    kt[r] = in ? key_w[row + j] : 0;
  }
  for (int64_t base = 0; base < T; base += kBlk) {
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kScanR; ++r) {
      s_band[wid][0][r * 32 + lane] = lo[r];
      s_band[wid][1][r * 32 + lane] = hi[r];
      s_band[wid][2][r * 32 + lane] = kt[r];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kScanR; ++r) {   // the next block's bands, in flight during this one
      const int64_t j = base + kBlk + r * 32 + lane;
      const bool in = j < T;
      lo[r] = in ? band_lo[row + j] : 0;
      hi[r] = in ? band_hi[row + j] : 0;
      kt[r] = in ? key_w[row + j] : 0;
    }
    const int n = (T - base) < kBlk ? (int)(T - base) : kBlk;
    for (int k = 0; k < n; k += kGrp) {
      long long l[kGrp], h[kGrp], w[kGrp];
#pragma unroll
      for (int g = 0; g < kGrp; ++g) {
        l[g] = s_band[wid][0][k + g];
        h[g] = s_band[wid][1][k + g];
        w[g] = s_band[wid][2][k + g];
      }
      const int c = (n - k) < kGrp ? (n - k) : kGrp;
      const uint32_t m = mh_group(st, l, h, w, c, beta, seed, step_offset + (uint64_t)(base + k), (uint32_t)i,
                                  prop_logq + row + base + k, prop_E + row + base + k);
      if (m) {
        cnt += __popc(m);
        lastt = row + base + k + (31 - __clz(m));
      }
      if (lane < kGrp) s_acc[wid][k + lane] = (m >> lane) & 1u;
    }
    __syncwarp();
    if (accepted) {
#pragma unroll
      for (int r = 0; r < kScanR; ++r) {
        const int j = r * 32 + lane;
        if (j < n) accepted[row + base + j] = s_acc[wid][j];
      }
    }
  }
  if (lane == 0) {
    if (lastt >= 0) {
      chain_logq[i] = prop_logq[lastt];
      chain_E[i] = prop_E[lastt];
    }
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
  const size_t bytes = (size_t)C * sizeof(int64_t) + (size_t)C * T * 3 * sizeof(int64_t);
  char* buf = static_cast<char*>(dev_alloc(alloc, bytes, stream));
  if (!buf) {
    tnmc_set_error("cannot allocate %zu bytes for the MH scan", bytes);
    return TNMC_E_NOMEM;
  }
  int64_t* band_lo = reinterpret_cast<int64_t*>(buf);
  int64_t* band_hi = band_lo + (size_t)C * T;
  int64_t* key_w = band_hi + (size_t)C * T;
  int64_t* last = key_w + (size_t)C * T;
  mh_bands_kernel<<<1024, 256, 0, stream>>>(C, T, seed, step_offset, beta, prop_logq, prop_energy, band_lo, band_hi,
                                            key_w);
  TNMC_CUDA_TRY(cudaGetLastError());
  const int threads = 128;   // 4 warps: the warp form's shared-memory layout
  if (C <= 65536) {   // one warp per chain
    const int64_t blocks = (C * 32 + threads - 1) / threads;
    mh_scan_warp_kernel<<<(unsigned)blocks, threads, 0, stream>>>(C, T, beta, seed, step_offset, prop_logq,
                                                                  prop_energy, band_lo, band_hi, key_w, chain_logq,
                                                                  chain_energy, accepted, last, n_accepted);
  } else {            // one thread per chain
    const int64_t blocks = (C + threads - 1) / threads;
    mh_scan_kernel<<<(unsigned)blocks, threads, 0, stream>>>(C, T, beta, seed, step_offset, prop_logq, prop_energy,
                                                             band_lo, band_hi, key_w, chain_logq, chain_energy,
                                                             accepted, last, n_accepted);
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
