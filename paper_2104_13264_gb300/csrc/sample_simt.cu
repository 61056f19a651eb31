// SIMT sampler / evaluator of q = pi~ (Sec. 2, eqs. bayes, pi-approx, tns-prior;
// App. A) in FP64 or FP32, and the kernel that derives the sampler copies of the
// environment.
//
// One thread owns one sample.  For every row r it
//   (right sweep) builds R_{Lx} = 1, R_c = sum_s f_c(s) M_c[:, s, :] R_{c+1}
//                 for c = Lx-1 .. 1, each rescaled by a power of two and pushed
//                 to a per-thread stack in global scratch;
//   (left sweep)  walks c = 0 .. Lx-1:  U[s] = Lambda_c M_c[:, s, :],
//                 w(s) = f_c(s) <U[s], R_{c+1}>, clamps at 0, normalises,
//                 draws the spin from the 64-bit Philox word (or reads it in
//                 forced mode), accumulates log q and the energy, and sets
//                 Lambda_{c+1} = f_c(s) U[s], rescaled by a power of two.
// f_c(s) = exp(beta Jv[r-1][c] s_{r-1,c} s) carries the (exactly contracted)
// product state of the rows above.  Environment tensors are read through the
// read-only cache: every thread of a CTA reads the same element at the same
// time, so each load is a broadcast.  Per-thread vectors live in shared memory
// laid out [k][thread] (conflict free).
#include <math.h>

#include "common.cuh"
#include "sample_simt_kernel.cuh"

namespace tnmc {
namespace {

// Sampler copies: L (same layout as M64), R ([b][a][s]) and the field table.
template <typename T>
__global__ void derive_kernel(DeviceEnv e, T* L, T* R, size_t ntens) {
  const int P = e.P;
  const size_t per = (size_t)P * 2 * P;
  const size_t total = ntens * per;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t t = i / per;
    const int rem = (int)(i % per);
    const int b = rem % P, s = (rem / P) & 1, aa = rem / (2 * P);
    const T v = (T)e.M64[i];
    if (L) L[i] = v;
    R[t * per + ((size_t)b * P + aa) * 2 + s] = v;
  }
}

__global__ void fields_kernel(DeviceEnv e, double* fe, float* fe32) {
  const int Lx = e.Lx, Ly = e.Ly;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Lx * Ly; i += gridDim.x * blockDim.x) {
    const int r = i / Lx, c = i % Lx;
    double d = 1.0, s = 1.0;
    if (r > 0) {
      const double jv = e.Jv[(r - 1) * Lx + c];
      d = exp(-e.beta * jv);
      s = exp(e.beta * jv);
    }
    fe[2 * i] = d;
    fe[2 * i + 1] = s;
    fe32[2 * i] = (float)d;
    fe32[2 * i + 1] = (float)s;
  }
}

template <typename T, int NT>
tnmc_status launch_sample_t(const tnmc_env* env, const T* L, const T* R, const T* fe, int64_t B,
                            uint64_t seed, uint64_t offset, const int8_t* spins_in, int8_t* spins_out,
                            double* logq, double* energy, int32_t* flags, cudaStream_t stream) {
  const DeviceEnv& d = env->d;
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
  if (grid < 1) grid = 1;
  const size_t need = (size_t)grid * (d.Lx + 1) * d.P * NT * sizeof(T);
  tnmc_env* me = const_cast<tnmc_env*>(env);
  {
    const tnmc_status gs = grow_scratch(me, need, stream, "sampler");
    if (gs != TNMC_OK) return gs;
  }
  SampleArgs<T> a;
  a.e = d;
  a.L = L;
  a.Rt = R;
  a.fe = fe;
  a.B = B;
  a.seed = seed;
  a.offset = offset;
  a.spins_in = spins_in;
  a.spins_out = spins_out;
  a.logq = logq;
  a.energy = energy;
  a.flags = flags;
  a.scratch = static_cast<T*>(me->scratch.ptr);
  kern<<<(unsigned)grid, NT, smem, stream>>>(a);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

}  // namespace
}  // namespace tnmc

tnmc_status tnmc_launch_derive(tnmc_env* env, int mask, cudaStream_t stream) {
  using namespace tnmc;
  DeviceEnv& d = env->d;
  const size_t ntens = (size_t)d.Lx * d.Ly;
  fields_kernel<<<256, 256, 0, stream>>>(d, const_cast<double*>(d.fe), const_cast<float*>(d.fe32));
  TNMC_CUDA_TRY(cudaGetLastError());
  derive_kernel<double><<<1024, 256, 0, stream>>>(d, nullptr, const_cast<double*>(d.R64), ntens);
  TNMC_CUDA_TRY(cudaGetLastError());
  if (mask & (1 << TNMC_F32)) {
    derive_kernel<float><<<1024, 256, 0, stream>>>(d, const_cast<float*>(d.L32), const_cast<float*>(d.R32), ntens);
    TNMC_CUDA_TRY(cudaGetLastError());
  }
  return TNMC_OK;
}

namespace tnmc {
namespace {
// transposed FP32 copy [b][a][s] from the left layout [a][s][b]
__global__ void rederive_f32_kernel(const float* L, float* R, int P, size_t ntens) {
  const size_t per = (size_t)P * 2 * P;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ntens * per; i += (size_t)gridDim.x * blockDim.x) {
    const size_t t = i / per;
    const int rem = (int)(i % per);
    const int b = rem % P, s = (rem / P) & 1, aa = rem / (2 * P);
    R[t * per + ((size_t)b * P + aa) * 2 + s] = L[i];
  }
}
}  // namespace
}  // namespace tnmc

tnmc_status tnmc_launch_rederive_f32(tnmc_env* env, cudaStream_t stream) {
  using namespace tnmc;
  DeviceEnv& d = env->d;
  rederive_f32_kernel<<<1024, 256, 0, stream>>>(d.L32, const_cast<float*>(d.R32), d.P, (size_t)d.Lx * d.Ly);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_launch_sample(const tnmc_env* env, int precision, int64_t B, uint64_t seed,
                               uint64_t offset, const int8_t* spins_in, int8_t* spins_out, double* logq,
                               double* energy, int32_t* flags, cudaStream_t stream) {
  using namespace tnmc;
  const DeviceEnv& d = env->d;
  if (B == 0) return TNMC_OK;
  if (precision == TNMC_F64)
    return launch_sample_t<double, 64>(env, d.M64, d.R64, d.fe, B, seed, offset, spins_in, spins_out, logq,
                                       energy, flags, stream);
  if (precision == TNMC_F32) {
    // 128 samples per CTA, or 64 when that leaves SMs without a tile (one thread per sample
    // either way, so every sample's arithmetic is the same)
    int dev = 0, nsm = 0;
    TNMC_CUDA_TRY(cudaGetDevice(&dev));
    TNMC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if ((B + 127) / 128 < 2 * (int64_t)nsm)
      return launch_sample_t<float, 64>(env, d.L32, d.R32, d.fe32, B, seed, offset, spins_in, spins_out, logq,
                                        energy, flags, stream);
    return launch_sample_t<float, 128>(env, d.L32, d.R32, d.fe32, B, seed, offset, spins_in, spins_out, logq,
                                       energy, flags, stream);
  }
  if (precision == TNMC_BF16)
    return tnmc_launch_sample_tc(env, B, seed, offset, spins_in, spins_out, logq, energy, flags, stream);
  tnmc_set_error("unknown precision %d", precision);
  return TNMC_E_UNSUPPORTED;
}
