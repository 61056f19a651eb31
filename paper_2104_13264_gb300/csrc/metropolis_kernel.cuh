// Single-spin-flip Metropolis sweeps of chain states and the link overlap of replica
// pairs: the sweeps the paper intersperses between proposals, and the quantity of its
// equilibration diagnostic (Sec. 3, "Equilibration", eq. Delta).
//
// A sweep updates the sites with (r + c) even, then those with (r + c) odd.  Sites of
// one colour share no bond, so each is updated against the current spins of the other
// colour: site i flips iff u < exp(-beta dE), dE = 2 s_i (h_i + sum_j J_ij s_j), with
// u = (x >> 11) 2^-53 from Philox4x32-10 words (0, 1) of the counter
// (site, chain id, sweep, 5).  The local field is summed in the order h, right, left,
// below, above (every term is exact: a coupling times +-1).
#pragma once

#include <math.h>

#include "common.cuh"

namespace tnmc {

struct MetroInst {
  const double* Jh;     // [Ly][Lx-1]
  const double* Jv;     // [Ly-1][Lx]
  const double* h;      // [Ly][Lx]
  double beta;
  int Lx, Ly;
  int64_t chain_spin;   // byte offset of the instance's chains in a chain arena
};

__device__ inline double sweep_uniform(uint64_t seed, uint32_t site, uint32_t chain, uint32_t sweep) {
  const U4 o = philox4x32_10(U4{site, chain, sweep, 5u}, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t x = (uint64_t)o.x | ((uint64_t)o.y << 32);
  return (double)(x >> 11) * 0x1.0p-53;
}

// `sweeps` sweeps of one chain by one CTA; `s` is the chain's spins in shared memory.
__device__ inline void metropolis_chain(const MetroInst& I, int8_t* s, uint64_t seed, uint32_t chain,
                                        uint32_t sweep0, int sweeps) {
  const int Lx = I.Lx, Ly = I.Ly, n = Lx * Ly;
  for (int k = 0; k < sweeps; ++k) {
    const uint32_t sweep = sweep0 + (uint32_t)k;
    for (int colour = 0; colour < 2; ++colour) {
      for (int site = threadIdx.x; site < n; site += blockDim.x) {
        const int r = site / Lx, c = site - r * Lx;
        if (((r + c) & 1) != colour) continue;
        double f = I.h[site];
        if (c + 1 < Lx) f += I.Jh[r * (Lx - 1) + c] * (double)s[site + 1];
        if (c > 0) f += I.Jh[r * (Lx - 1) + c - 1] * (double)s[site - 1];
        if (r + 1 < Ly) f += I.Jv[r * Lx + c] * (double)s[site + Lx];
        if (r > 0) f += I.Jv[(r - 1) * Lx + c] * (double)s[site - Lx];
        const double dE = 2.0 * (double)s[site] * f;
        const double u = sweep_uniform(seed, (uint32_t)site, chain, sweep);
        if (u < exp(-I.beta * dE)) s[site] = (int8_t)(-s[site]);
      }
      __syncthreads();
    }
  }
}

// sum over the bonds of s_i^a s_j^a s_i^b s_j^b, by one CTA (exact integer count).
__device__ inline double link_overlap_pair(int Lx, int Ly, const int8_t* a, const int8_t* b, long long* red) {
  const int n = Lx * Ly;
  long long acc = 0;
  for (int site = threadIdx.x; site < n; site += blockDim.x) {
    const int r = site / Lx, c = site - r * Lx;
    const int ab = a[site] * b[site];
    if (c + 1 < Lx) acc += ab * a[site + 1] * b[site + 1];
    if (r + 1 < Ly) acc += ab * a[site + Lx] * b[site + Lx];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  long long tot = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  __syncthreads();
  return (double)tot;
}

}  // namespace tnmc
