// Internal definitions shared by the CUDA translation units of libtnmc.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/tnmc.h"

namespace tnmc {

constexpr int kMaxChi = 64;       // largest supported bond dimension
constexpr int kMaxPad = 64;       // padded bond stride P <= 64

// ---------------------------------------------------------------------------
// Environment held on the device.
//   M64   FP64 master, [Ly][Lx][P][2][P]  M[a][s][b]      (left layout)
//   L{T}  sampler copy in precision T, same layout as M64
//   R{T}  sampler copy in precision T, [Ly][Lx][P][P][2]  MT[b][a][s]
//   L16 / R16 (BF16) instead hold the tensor-core operand tiles: per (r, c) two
//         128 x 64 K-major 128-byte-swizzled tiles, hi = bf16(M) then
//         lo = bf16(M - hi) (left: n = s*64 + b, k = a; right: n = s*64 + a, k = b),
//         zero-padded to 64.
//   fe    FP64 [Ly][Lx][2]: exp(-beta Jv[r-1][c]), exp(+beta Jv[r-1][c]); 1 for r = 0
//   fe32  same in FP32
// ---------------------------------------------------------------------------
struct DeviceEnv {
  int Lx, Ly, chi, P;
  double beta;
  int integer_couplings;
  int z2;             // 1 when every field is zero: the builder uses parity sectors
  int gauge;          // 0: spin basis; 1: bond basis (rows sampled from the untruncated 2 chi MPS)
  int sweeps;         // two-site variational rounds after successive SVD (0: successive SVD only)
  int order;          // site order of the samplers: TNMC_ORDER_RASTER, TNMC_ORDER_SNAKE
  const double* Jh;   // device copies of the couplings
  const double* Jv;
  const double* h;
  const double* fe;
  const float* fe32;
  const int32_t* bond;   // [Ly][Lx+1]
  const double* M64;
  const double* R64;
  const float* L32;
  const float* R32;
  const __nv_bfloat16* L16;
  const __nv_bfloat16* R16;
  int32_t* status;       // device status word
};

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// The device-memory hook an object allocates and frees through (tnmc_set_allocator).
struct Allocator {
  tnmc_alloc_fn alloc = nullptr;   // nullptr: cudaMallocAsync / cudaFreeAsync
  tnmc_free_fn free = nullptr;
  void* ctx = nullptr;
};

Allocator current_allocator();
void* dev_alloc(const Allocator& A, size_t bytes, cudaStream_t s);   // nullptr on failure
void dev_free(const Allocator& A, void* p, size_t bytes, cudaStream_t s);

}  // namespace tnmc

struct tnmc_env {
  tnmc::DeviceEnv d;
  int precision_mask;
  cudaStream_t build_stream;
  // device allocations owned by the env
  void* arena = nullptr;
  size_t arena_bytes = 0;
  double* log_scale = nullptr;   // [Ly]
  double* sv = nullptr;          // [Ly][Lx+1][P]
  double* discarded = nullptr;   // [Ly][Lx+1]
  double* logZ = nullptr;        // scalar
  int32_t* esz = nullptr;        // [Ly][Lx+1] even-sector size per bond (Z2 builder)
  float* h32 = nullptr;          // FP32 couplings for the tensor-core sampler's energy
  float* Jh32 = nullptr;
  float* Jv32 = nullptr;
  tnmc::Scratch scratch;         // sampler scratch (grown on demand)
  tnmc::Allocator alloc;         // the hook current when the env was created
};

namespace tnmc {
// Grow env->scratch to at least `need` bytes (the old block is released in stream order).
tnmc_status grow_scratch(tnmc_env* env, size_t need, cudaStream_t s, const char* what);
}  // namespace tnmc

namespace tnmc {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// two-multiplication bijection, key bumped by the Weyl constants between rounds.
struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (i > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t p0 = (uint64_t)M0 * c.x;
    const uint64_t p1 = (uint64_t)M1 * c.z;
    U4 n;
    n.x = (uint32_t)(p1 >> 32) ^ c.y ^ k0;
    n.y = (uint32_t)p1;
    n.z = (uint32_t)(p0 >> 32) ^ c.w ^ k1;
    n.w = (uint32_t)p0;
    c = n;
  }
  return c;
}

// 64-bit draw for (site, sample) on stream 0.
__device__ inline uint64_t draw_word(uint64_t seed, int64_t site, uint64_t sample) {
  U4 c{(uint32_t)(site >> 1), (uint32_t)sample, (uint32_t)(sample >> 32), 0u};
  U4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return (site & 1) ? ((uint64_t)o.z | ((uint64_t)o.w << 32)) : ((uint64_t)o.x | ((uint64_t)o.y << 32));
}

__device__ inline double mh_uniform(uint64_t seed, uint64_t t, uint32_t chain) {
  U4 c{(uint32_t)t, (uint32_t)(t >> 32), chain, 1u};
  U4 o = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  uint64_t x = (uint64_t)o.x | ((uint64_t)o.y << 32);
  return (double)(x >> 11) * 0x1.0p-53;
}

// Spin draw: +1 iff x < floor(p_plus 2^64); p_plus >= 1 always gives +1.
__device__ inline bool draw_plus(double pplus, uint64_t x) {
  if (pplus >= 1.0) return true;
  if (!(pplus > 0.0)) return false;
  return x < __double2ull_rz(pplus * 0x1.0p64);
}
__device__ inline bool draw_plus(float pplus, uint64_t x) {
  if (pplus >= 1.0f) return true;
  if (!(pplus > 0.0f)) return false;
  return x < __float2ull_rz(pplus * 0x1.0p64f);
}

inline int pad4(int x) { return (x + 3) & ~3; }

inline int bond_dim_host(int chi, int Lx, int Ly, int r, int c) {
  if (c <= 0 || c >= Lx) return 1;
  int e = c;
  if (Lx - c < e) e = Lx - c;
  if (Ly - r < e) e = Ly - r;
  if (e > 30) e = 30;
  int v = 1 << e;
  return chi < v ? chi : v;
}

// status word helpers
__device__ inline void set_status(int32_t* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

}  // namespace tnmc

// error plumbing (api.cu)
void tnmc_set_error(const char* fmt, ...);
#define TNMC_CUDA_TRY(expr)                                                        \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      tnmc_set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__); \
      return TNMC_E_CUDA;                                                          \
    }                                                                              \
  } while (0)

// launchers implemented in the kernel translation units
tnmc_status tnmc_launch_build(tnmc_env* env, cudaStream_t stream, void* work, size_t work_bytes);
tnmc_status tnmc_launch_build_batched(tnmc_env* const* envs, int n, void* work, const size_t* work_offsets,
                                      void* args_dev, cudaStream_t stream);
size_t tnmc_build_args_bytes();
size_t tnmc_build_work_bytes(int Lx, int Ly, int P, int sweeps);
tnmc_status tnmc_launch_derive(tnmc_env* env, int precision_mask, cudaStream_t stream);
tnmc_status tnmc_launch_mh_core(int64_t n, double beta, const tnmc::Allocator& alloc, int64_t C, int64_t T,
                                const int8_t* prop_spins, const double* prop_logq, const double* prop_energy,
                                int8_t* chain_spins, double* chain_logq, double* chain_energy, uint64_t seed,
                                uint64_t step_offset, uint8_t* accepted, int64_t* n_accepted, cudaStream_t stream);
tnmc_status tnmc_launch_init_bits_core(int64_t n, int64_t C, uint64_t seed, int8_t* spins, cudaStream_t stream);
tnmc_status tnmc_launch_bond_sampling(tnmc_env* env, cudaStream_t stream);
tnmc_status tnmc_launch_sample(const tnmc_env* env, int precision, int64_t B, uint64_t seed,
                               uint64_t sample_offset, const int8_t* spins_in, int8_t* spins_out,
                               double* logq, double* energy, int32_t* flags, cudaStream_t stream);
tnmc_status tnmc_launch_derive_tc(tnmc_env* env, cudaStream_t stream);
size_t tnmc_tc_tile_bytes();
tnmc_status tnmc_launch_sample_tc(const tnmc_env* env, int64_t B, uint64_t seed, uint64_t offset,
                                  const int8_t* spins_in, int8_t* spins_out, double* logq, double* energy,
                                  int32_t* flags, cudaStream_t stream);
tnmc_status tnmc_launch_logq_grad(const tnmc_env* env, int64_t B, const int8_t* spins, const float* weights,
                                  float* grad, cudaStream_t stream);
tnmc_status tnmc_launch_rederive_f32(tnmc_env* env, cudaStream_t stream);
tnmc_status tnmc_launch_mh(const tnmc_env* env, int64_t C, int64_t T, const int8_t* prop_spins,
                           const double* prop_logq, const double* prop_energy, int8_t* chain_spins,
                           double* chain_logq, double* chain_energy, uint64_t seed,
                           uint64_t step_offset, uint8_t* accepted, int64_t* n_accepted,
                           cudaStream_t stream);
tnmc_status tnmc_launch_init_bits(const tnmc_env* env, int64_t C, uint64_t seed, int8_t* spins,
                                  cudaStream_t stream);
tnmc_status tnmc_launch_metropolis(const tnmc_env* env, int64_t C, int8_t* chains, uint64_t seed,
                                   uint64_t chain_offset, uint64_t sweep_offset, int sweeps, cudaStream_t stream);
tnmc_status tnmc_launch_link_overlap(int Lx, int Ly, int64_t pairs, const int8_t* chains, double* out,
                                     cudaStream_t stream);
