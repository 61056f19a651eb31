// C-ABI entry points of libtnmc: argument checking, device memory of the
// environment, and the launches.  No C++ exception crosses the boundary.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"

static thread_local char g_err[512] = "";

void tnmc_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

namespace tnmc {

static Allocator g_alloc;   // process-wide hook (tnmc_set_allocator)

Allocator current_allocator() { return g_alloc; }

void* dev_alloc(const Allocator& A, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 1;
  if (A.alloc) return A.alloc(bytes, s, A.ctx);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(const Allocator& A, void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (A.free) {
    A.free(p, bytes, s, A.ctx);
    return;
  }
  if (cudaFreeAsync(p, s) != cudaSuccess) (void)cudaGetLastError();
}

tnmc_status grow_scratch(tnmc_env* env, size_t need, cudaStream_t s, const char* what) {
  if (env->scratch.bytes >= need) return TNMC_OK;
  dev_free(env->alloc, env->scratch.ptr, env->scratch.bytes, s);
  env->scratch.ptr = nullptr;
  env->scratch.bytes = 0;
  void* p = dev_alloc(env->alloc, need, s);
  if (!p) {
    tnmc_set_error("cannot allocate %zu bytes of %s scratch", need, what);
    return TNMC_E_NOMEM;
  }
  env->scratch.ptr = p;
  env->scratch.bytes = need;
  return TNMC_OK;
}

}  // namespace tnmc

#define CHECK_ARG(cond, ...)          \
  do {                                \
    if (!(cond)) {                    \
      tnmc_set_error(__VA_ARGS__);    \
      return TNMC_E_INVALID_ARG;      \
    }                                 \
  } while (0)

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool is_integer_array(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (p[i] != floor(p[i])) return false;
  return true;
}

}  // namespace

namespace {

// Checks the arguments, allocates the environment's arena and uploads the
// couplings; the tensors are written by a later builder launch.
tnmc_status env_create(const tnmc_lattice* lat, double beta, int chi, int precision_mask, int gauge, int sweeps,
                       cudaStream_t s, tnmc_env** out) {
  using namespace tnmc;
  *out = nullptr;
  CHECK_ARG(lat, "lattice must be non-null");
  const int Lx = lat->Lx, Ly = lat->Ly;
  CHECK_ARG(Lx >= 1 && Ly >= 1 && Lx <= 4096 && Ly <= 4096, "lattice %d x %d out of range", Ly, Lx);
  CHECK_ARG(chi >= 1 && chi <= kMaxChi, "chi = %d must be in [1, %d]", chi, kMaxChi);
  CHECK_ARG(gauge == 0 || chi <= kMaxChi / 2, "the bond basis samples from 2 chi bonds: chi = %d must be <= %d", chi,
            kMaxChi / 2);
  CHECK_ARG(sweeps >= 0 && sweeps <= 64, "variational sweeps = %d must be in [0, 64]", sweeps);
  CHECK_ARG(sweeps == 0 || gauge == 0, "variational compression is built for the spin basis only");
  CHECK_ARG(isfinite(beta) && beta >= 0.0, "beta must be finite and >= 0");
  CHECK_ARG(lat->h, "h must be non-null");
  CHECK_ARG(Lx == 1 || lat->Jh, "Jh must be non-null when Lx > 1");
  CHECK_ARG(Ly == 1 || lat->Jv, "Jv must be non-null when Ly > 1");
  CHECK_ARG((precision_mask & ~7) == 0, "unknown precision bits in mask 0x%x", precision_mask);
  const size_t nJh = (size_t)Ly * (Lx - 1), nJv = (size_t)(Ly - 1) * Lx, nh = (size_t)Ly * Lx;
  for (size_t i = 0; i < nJh; ++i) CHECK_ARG(isfinite(lat->Jh[i]), "Jh[%zu] is not finite", i);
  for (size_t i = 0; i < nJv; ++i) CHECK_ARG(isfinite(lat->Jv[i]), "Jv[%zu] is not finite", i);
  for (size_t i = 0; i < nh; ++i) CHECK_ARG(isfinite(lat->h[i]), "h[%zu] is not finite", i);
  const int mask = precision_mask | (1 << TNMC_F64);
  // padded bond stride
  int maxb = 1;
  for (int r = 0; r < Ly; ++r)
    for (int c = 0; c <= Lx; ++c) {
      const int b = bond_dim_host(chi, Lx, Ly, r, c);
      if (b > maxb) maxb = b;
    }
  // the bond basis samples each row from its untruncated MPS: bonds up to 2 chi
  const int P = pad4(gauge ? 2 * maxb : maxb);
  const size_t ntens = (size_t)Lx * Ly;
  const size_t tens = ntens * P * 2 * P;
  // arena layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t oJh = take((nJh ? nJh : 1) * 8), oJv = take((nJv ? nJv : 1) * 8), oh = take(nh * 8);
  const size_t ofe = take(nh * 2 * 8), ofe32 = take(nh * 2 * 4);
  const size_t obond = take((size_t)Ly * (Lx + 1) * 4), oesz = take((size_t)Ly * (Lx + 1) * 4);
  const size_t oM64 = take(tens * 8), oR64 = take(tens * 8);
  const size_t oL32 = (mask & (1 << TNMC_F32)) ? take(tens * 4) : 0;
  const size_t oR32 = (mask & (1 << TNMC_F32)) ? take(tens * 4) : 0;
  const size_t oL16 = (mask & (1 << TNMC_BF16)) ? take(ntens * tnmc_tc_tile_bytes()) : 0;
  const size_t oR16 = (mask & (1 << TNMC_BF16)) ? take(ntens * tnmc_tc_tile_bytes()) : 0;
  const size_t oh32 = take(nh * 4), oJh32 = take((nJh ? nJh : 1) * 4), oJv32 = take((nJv ? nJv : 1) * 4);
  const size_t ols = take((size_t)Ly * 8), osv = take((size_t)Ly * (Lx + 1) * P * 8);
  const size_t odisc = take((size_t)Ly * (Lx + 1) * 8), ologZ = take(8), ostat = take(8);
  const size_t total = off;

  tnmc_env* env = new (std::nothrow) tnmc_env();
  if (!env) {
    tnmc_set_error("host allocation failed");
    return TNMC_E_NOMEM;
  }
  env->alloc = current_allocator();
  char* base = static_cast<char*>(dev_alloc(env->alloc, total, s));
  if (!base) {
    delete env;
    tnmc_set_error("cannot allocate %zu bytes for the environment", total);
    return TNMC_E_NOMEM;
  }
  env->arena = base;
  env->arena_bytes = total;
  env->precision_mask = mask;
  env->build_stream = s;
  DeviceEnv& d = env->d;
  d.Lx = Lx;
  d.Ly = Ly;
  d.chi = chi;
  d.P = P;
  d.beta = beta;
  d.integer_couplings = is_integer_array(lat->h, nh) && (nJh == 0 || is_integer_array(lat->Jh, nJh)) &&
                        (nJv == 0 || is_integer_array(lat->Jv, nJv));
  {
    bool zero_field = true;
    for (size_t i = 0; i < nh; ++i) zero_field = zero_field && (lat->h[i] == 0.0);
    const char* force = getenv("TNMC_DENSE_BUILDER");   // testing knob: the dense path on h = 0 lattices
    d.z2 = zero_field && !(force && force[0] == '1') && gauge == 0 && sweeps == 0;
  }
  d.gauge = gauge;
  d.sweeps = sweeps;
  d.Jh = reinterpret_cast<const double*>(base + oJh);
  d.Jv = reinterpret_cast<const double*>(base + oJv);
  d.h = reinterpret_cast<const double*>(base + oh);
  d.fe = reinterpret_cast<const double*>(base + ofe);
  d.fe32 = reinterpret_cast<const float*>(base + ofe32);
  d.bond = reinterpret_cast<const int32_t*>(base + obond);
  d.M64 = reinterpret_cast<const double*>(base + oM64);
  d.R64 = reinterpret_cast<const double*>(base + oR64);
  d.L32 = oL32 ? reinterpret_cast<const float*>(base + oL32) : nullptr;
  d.R32 = oR32 ? reinterpret_cast<const float*>(base + oR32) : nullptr;
  d.L16 = oL16 ? reinterpret_cast<const __nv_bfloat16*>(base + oL16) : nullptr;
  d.R16 = oR16 ? reinterpret_cast<const __nv_bfloat16*>(base + oR16) : nullptr;
  d.status = reinterpret_cast<int32_t*>(base + ostat);
  env->log_scale = reinterpret_cast<double*>(base + ols);
  env->sv = reinterpret_cast<double*>(base + osv);
  env->discarded = reinterpret_cast<double*>(base + odisc);
  env->logZ = reinterpret_cast<double*>(base + ologZ);
  env->esz = reinterpret_cast<int32_t*>(base + oesz);
  env->h32 = reinterpret_cast<float*>(base + oh32);
  env->Jh32 = reinterpret_cast<float*>(base + oJh32);
  env->Jv32 = reinterpret_cast<float*>(base + oJv32);

  tnmc_status st = TNMC_OK;
  do {
    if (cudaMemsetAsync(base, 0, total, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    if (nJh && cudaMemcpyAsync(const_cast<double*>(d.Jh), lat->Jh, nJh * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    if (nJv && cudaMemcpyAsync(const_cast<double*>(d.Jv), lat->Jv, nJv * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    if (cudaMemcpyAsync(const_cast<double*>(d.h), lat->h, nh * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    // the host arrays may be released as soon as this call returns
    if (cudaStreamSynchronize(s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
  } while (0);
  if (st != TNMC_OK) {
    if (!g_err[0]) tnmc_set_error("CUDA error while uploading the couplings: %s", cudaGetErrorString(cudaGetLastError()));
    (void)cudaStreamSynchronize(s);
    dev_free(env->alloc, base, total, s);
    delete env;
    return st;
  }
  *out = env;
  return TNMC_OK;
}

void env_destroy(tnmc_env* env, cudaStream_t s) {
  if (!env) return;
  (void)cudaStreamSynchronize(s);
  dev_free(env->alloc, env->scratch.ptr, env->scratch.bytes, s);
  dev_free(env->alloc, env->arena, env->arena_bytes, s);
  (void)cudaStreamSynchronize(s);
  delete env;
}

// The sampler copies of a built environment.
tnmc_status env_derive(tnmc_env* env, cudaStream_t s) {
  tnmc_status st = tnmc_launch_derive(env, env->precision_mask, s);
  if (st == TNMC_OK && (env->precision_mask & (1 << TNMC_BF16))) st = tnmc_launch_derive_tc(env, s);
  return st;
}

}  // namespace

extern "C" {

const char* tnmc_last_error(void) { return g_err; }

static tnmc_status build_env_variant(const tnmc_lattice* lat, double beta, int chi, int precision_mask, int gauge,
                                     int sweeps, void* stream, tnmc_env** out) {
  using namespace tnmc;
  g_err[0] = 0;
  CHECK_ARG(lat && out, "lat and out must be non-null");
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tnmc_env* env = nullptr;
  tnmc_status st = env_create(lat, beta, chi, precision_mask, gauge, sweeps, s, &env);
  if (st != TNMC_OK) return st;
  const DeviceEnv& d = env->d;
  void* work = nullptr;
  const size_t wbytes = tnmc_build_work_bytes(d.Lx, d.Ly, d.P, d.sweeps);
  do {
    work = dev_alloc(env->alloc, wbytes, s);
    if (!work) {
      st = TNMC_E_NOMEM;
      tnmc_set_error("cannot allocate %zu bytes of builder scratch", wbytes);
      break;
    }
    st = tnmc_launch_build(env, s, work, wbytes);
    if (st != TNMC_OK) break;
    if (gauge == 1) st = tnmc_launch_bond_sampling(env, s);
    if (st != TNMC_OK) break;
    st = env_derive(env, s);
  } while (0);
  dev_free(env->alloc, work, wbytes, s);
  if (st != TNMC_OK) {
    if (st == TNMC_E_CUDA && !g_err[0]) tnmc_set_error("CUDA error while building: %s", cudaGetErrorString(cudaGetLastError()));
    env_destroy(env, s);
    return st;
  }
  *out = env;
  return TNMC_OK;
}

tnmc_status tnmc_build_env(const tnmc_lattice* lat, double beta, int chi, int precision_mask, void* stream,
                           tnmc_env** out) {
  return build_env_variant(lat, beta, chi, precision_mask, 0, 0, stream, out);
}

tnmc_status tnmc_build_env_bond(const tnmc_lattice* lat, double beta, int chi, int precision_mask, void* stream,
                                tnmc_env** out) {
  return build_env_variant(lat, beta, chi, precision_mask, 1, 0, stream, out);
}

tnmc_status tnmc_build_env_variational(const tnmc_lattice* lat, double beta, int chi, int sweeps, int precision_mask,
                                       void* stream, tnmc_env** out) {
  return build_env_variant(lat, beta, chi, precision_mask, 0, sweeps, stream, out);
}

tnmc_status tnmc_build_env_batched(int n, const tnmc_lattice* lats, const double* beta, const int* chi,
                                   int precision_mask, void* stream, tnmc_env** out) {
  using namespace tnmc;
  g_err[0] = 0;
  CHECK_ARG(n >= 0, "n = %d must be >= 0", n);
  CHECK_ARG(n == 0 || (lats && beta && chi && out), "lats, beta, chi and out must be non-null");
  if (n == 0) return TNMC_OK;
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<tnmc_env*> envs(n, nullptr);
  std::vector<size_t> woff(n);
  tnmc_status st = TNMC_OK;
  size_t wtotal = 0;
  for (int i = 0; i < n && st == TNMC_OK; ++i) {
    st = env_create(&lats[i], beta[i], chi[i], precision_mask, 0, 0, s, &envs[i]);
    if (st != TNMC_OK) {
      char msg[512];
      snprintf(msg, sizeof msg, "instance %d: %s", i, g_err);
      tnmc_set_error("%s", msg);
      break;
    }
    const DeviceEnv& d = envs[i]->d;
    woff[i] = wtotal;
    wtotal += align256(tnmc_build_work_bytes(d.Lx, d.Ly, d.P, d.sweeps));
  }
  const Allocator A = current_allocator();
  void* work = nullptr;
  void* args = nullptr;
  if (st == TNMC_OK) {
    do {
      work = dev_alloc(A, wtotal, s);
      args = work ? dev_alloc(A, (size_t)n * tnmc_build_args_bytes(), s) : nullptr;
      if (!work || !args) {
        st = TNMC_E_NOMEM;
        tnmc_set_error("cannot allocate %zu bytes of builder scratch", wtotal);
        break;
      }
      st = tnmc_launch_build_batched(envs.data(), n, work, woff.data(), args, s);
      for (int i = 0; i < n && st == TNMC_OK; ++i) st = env_derive(envs[i], s);
    } while (0);
  }
  dev_free(A, work, wtotal, s);
  dev_free(A, args, (size_t)n * tnmc_build_args_bytes(), s);
  if (st != TNMC_OK) {
    if (st == TNMC_E_CUDA && !g_err[0]) tnmc_set_error("CUDA error while building: %s", cudaGetErrorString(cudaGetLastError()));
    for (int i = 0; i < n; ++i) env_destroy(envs[i], s);
    return st;
  }
  for (int i = 0; i < n; ++i) out[i] = envs[i];
  return TNMC_OK;
}

tnmc_status tnmc_env_free(tnmc_env* env) {
  if (!env) return TNMC_OK;
  cudaDeviceSynchronize();
  dev_free(env->alloc, env->scratch.ptr, env->scratch.bytes, nullptr);
  dev_free(env->alloc, env->arena, env->arena_bytes, nullptr);
  cudaDeviceSynchronize();
  delete env;
  return TNMC_OK;
}

tnmc_status tnmc_set_allocator(tnmc_alloc_fn alloc_fn, tnmc_free_fn free_fn, void* ctx) {
  g_err[0] = 0;
  CHECK_ARG((alloc_fn == nullptr) == (free_fn == nullptr), "alloc_fn and free_fn must both be set or both be NULL");
  tnmc::g_alloc.alloc = alloc_fn;
  tnmc::g_alloc.free = free_fn;
  tnmc::g_alloc.ctx = alloc_fn ? ctx : nullptr;
  return TNMC_OK;
}

tnmc_status tnmc_env_info(const tnmc_env* env, tnmc_env_info_t* info) {
  CHECK_ARG(env && info, "env and info must be non-null");
  TNMC_CUDA_TRY(cudaStreamSynchronize(env->build_stream));
  double logZ = 0.0;
  TNMC_CUDA_TRY(cudaMemcpy(&logZ, env->logZ, sizeof(double), cudaMemcpyDeviceToHost));
  info->Lx = env->d.Lx;
  info->Ly = env->d.Ly;
  info->chi = env->d.chi;
  info->pad = env->d.P;
  info->precision_mask = env->precision_mask;
  info->integer_couplings = env->d.integer_couplings;
  info->beta = env->d.beta;
  info->logZ = logZ;
  info->bytes = (int64_t)(env->arena_bytes + env->scratch.bytes);
  return TNMC_OK;
}

tnmc_status tnmc_env_export(const tnmc_env* env, double* tensors, double* log_scale, double* sv, double* discarded,
                            int32_t* bond_dims) {
  CHECK_ARG(env, "env must be non-null");
  const tnmc::DeviceEnv& d = env->d;
  TNMC_CUDA_TRY(cudaStreamSynchronize(env->build_stream));
  const size_t tens = (size_t)d.Lx * d.Ly * d.P * 2 * d.P;
  if (tensors) TNMC_CUDA_TRY(cudaMemcpy(tensors, d.M64, tens * 8, cudaMemcpyDeviceToHost));
  if (log_scale) TNMC_CUDA_TRY(cudaMemcpy(log_scale, env->log_scale, (size_t)d.Ly * 8, cudaMemcpyDeviceToHost));
  if (sv) TNMC_CUDA_TRY(cudaMemcpy(sv, env->sv, (size_t)d.Ly * (d.Lx + 1) * d.P * 8, cudaMemcpyDeviceToHost));
  if (discarded) TNMC_CUDA_TRY(cudaMemcpy(discarded, env->discarded, (size_t)d.Ly * (d.Lx + 1) * 8, cudaMemcpyDeviceToHost));
  if (bond_dims) TNMC_CUDA_TRY(cudaMemcpy(bond_dims, d.bond, (size_t)d.Ly * (d.Lx + 1) * 4, cudaMemcpyDeviceToHost));
  return TNMC_OK;
}

tnmc_status tnmc_env_status(const tnmc_env* env, int32_t* status) {
  CHECK_ARG(env && status, "env and status must be non-null");
  TNMC_CUDA_TRY(cudaDeviceSynchronize());
  TNMC_CUDA_TRY(cudaMemcpy(status, env->d.status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return TNMC_OK;
}

static tnmc_status check_precision(const tnmc_env* env, int precision) {
  CHECK_ARG(precision >= 0 && precision <= 2, "unknown precision %d", precision);
  if (!(env->precision_mask & (1 << precision))) {
    tnmc_set_error("the env was built without the sampler copy for precision %d", precision);
    return TNMC_E_UNSUPPORTED;
  }
  if (env->d.order == TNMC_ORDER_SNAKE && precision == TNMC_BF16) {
    tnmc_set_error("the BF16 tensor-core sampler runs in raster order only");
    return TNMC_E_UNSUPPORTED;
  }
  return TNMC_OK;
}

tnmc_status tnmc_env_set_order(tnmc_env* env, int order) {
  g_err[0] = 0;
  CHECK_ARG(env, "env must be non-null");
  CHECK_ARG(order == TNMC_ORDER_RASTER || order == TNMC_ORDER_SNAKE, "unknown site order %d", order);
  env->d.order = order;
  return TNMC_OK;
}

tnmc_status tnmc_sample(const tnmc_env* env, int precision, int64_t B, uint64_t seed, uint64_t sample_offset,
                        int8_t* spins, double* logq, double* energy, int32_t* flags, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env, "env must be non-null");
  CHECK_ARG(B >= 0, "B must be >= 0");
  CHECK_ARG(B == 0 || (spins && logq && energy), "spins, logq and energy must be non-null");
  tnmc_status st = check_precision(env, precision);
  if (st != TNMC_OK) return st;
  return tnmc_launch_sample(env, precision, B, seed, sample_offset, nullptr, spins, logq, energy, flags,
                            static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc_logq(const tnmc_env* env, int precision, int64_t B, const int8_t* spins, double* logq,
                      double* energy, int32_t* flags, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env, "env must be non-null");
  CHECK_ARG(B >= 0, "B must be >= 0");
  CHECK_ARG(B == 0 || (spins && logq && energy), "spins, logq and energy must be non-null");
  tnmc_status st = check_precision(env, precision);
  if (st != TNMC_OK) return st;
  return tnmc_launch_sample(env, precision, B, 0, 0, spins, nullptr, logq, energy, flags,
                            static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc_init_chains(const tnmc_env* env, int precision, int64_t C, uint64_t seed, int8_t* chain_spins,
                             double* chain_logq, double* chain_energy, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env, "env must be non-null");
  CHECK_ARG(C >= 0 && C < ((int64_t)1 << 32), "C out of range");
  CHECK_ARG(C == 0 || (chain_spins && chain_logq && chain_energy), "chain arrays must be non-null");
  tnmc_status st = check_precision(env, precision);
  if (st != TNMC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = tnmc_launch_init_bits(env, C, seed, chain_spins, s);
  if (st != TNMC_OK) return st;
  return tnmc_launch_sample(env, precision, C, 0, 0, chain_spins, nullptr, chain_logq, chain_energy, nullptr, s);
}

tnmc_status tnmc_mh_step(const tnmc_env* env, int64_t C, int64_t T, const int8_t* prop_spins,
                         const double* prop_logq, const double* prop_energy, int8_t* chain_spins,
                         double* chain_logq, double* chain_energy, uint64_t seed, uint64_t step_offset,
                         uint8_t* accepted, int64_t* n_accepted, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env, "env must be non-null");
  CHECK_ARG(C >= 0 && C < ((int64_t)1 << 32) && T >= 0, "C or T out of range");
  CHECK_ARG(C == 0 || T == 0 ||
                (prop_spins && prop_logq && prop_energy && chain_spins && chain_logq && chain_energy),
            "proposal and chain arrays must be non-null");
  return tnmc_launch_mh(env, C, T, prop_spins, prop_logq, prop_energy, chain_spins, chain_logq, chain_energy, seed,
                        step_offset, accepted, n_accepted, static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc_metropolis(const tnmc_env* env, int precision, int64_t C, int8_t* chain_spins, double* chain_logq,
                            double* chain_energy, uint64_t seed, uint64_t chain_offset, uint64_t sweep_offset,
                            int sweeps, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env, "env must be non-null");
  CHECK_ARG(C >= 0 && C < ((int64_t)1 << 32), "C out of range");
  CHECK_ARG(sweeps >= 0, "sweeps must be >= 0");
  CHECK_ARG(C == 0 || (chain_spins && chain_logq && chain_energy), "chain arrays must be non-null");
  CHECK_ARG((size_t)env->d.Lx * env->d.Ly <= 200 * 1024, "a chain of %d sites does not fit in shared memory",
            env->d.Lx * env->d.Ly);
  tnmc_status st = check_precision(env, precision);
  if (st != TNMC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = tnmc_launch_metropolis(env, C, chain_spins, seed, chain_offset, sweep_offset, sweeps, s);
  if (st != TNMC_OK) return st;
  // the chain states changed: their log q and energy, as tnmc_logq computes them
  return tnmc_launch_sample(env, precision, C, 0, 0, chain_spins, nullptr, chain_logq, chain_energy, nullptr, s);
}

tnmc_status tnmc_link_overlap(const tnmc_env* env, int64_t C, const int8_t* chain_spins, double* overlap,
                              void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env, "env must be non-null");
  CHECK_ARG(C >= 0 && C % 2 == 0, "C = %lld must be even (replica pairs)", (long long)C);
  CHECK_ARG(C == 0 || (chain_spins && overlap), "chain_spins and overlap must be non-null");
  return tnmc_launch_link_overlap(env->d.Lx, env->d.Ly, C / 2, chain_spins, overlap,
                                  static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc_logq_backward(const tnmc_env* env, int64_t B, const int8_t* spins, const float* weights,
                               float* grad, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env, "env must be non-null");
  CHECK_ARG(B >= 0, "B must be >= 0");
  CHECK_ARG(grad && (B == 0 || (spins && weights)), "spins, weights and grad must be non-null");
  tnmc_status st = check_precision(env, TNMC_F32);
  if (st != TNMC_OK) return st;
  if (env->d.order != TNMC_ORDER_RASTER) {
    tnmc_set_error("tnmc_logq_backward differentiates the raster-order q only");
    return TNMC_E_UNSUPPORTED;
  }
  if (env->d.P > 64) {
    tnmc_set_error("tnmc_logq_backward supports padded bond dimension P <= 64 (got %d)", env->d.P);
    return TNMC_E_UNSUPPORTED;
  }
  return tnmc_launch_logq_grad(env, B, spins, weights, grad, static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc_env_get_params(const tnmc_env* env, float* dst, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env && dst, "env and dst must be non-null");
  tnmc_status st = check_precision(env, TNMC_F32);
  if (st != TNMC_OK) return st;
  const size_t n = (size_t)env->d.Lx * env->d.Ly * env->d.P * 2 * env->d.P;
  TNMC_CUDA_TRY(cudaMemcpyAsync(dst, env->d.L32, n * sizeof(float), cudaMemcpyDeviceToDevice,
                                static_cast<cudaStream_t>(stream)));
  return TNMC_OK;
}

tnmc_status tnmc_env_set_tensors(tnmc_env* env, const double* src, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env && src, "env and src must be non-null");
  const size_t n = (size_t)env->d.Lx * env->d.Ly * env->d.P * 2 * env->d.P;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TNMC_CUDA_TRY(cudaMemcpyAsync(const_cast<double*>(env->d.M64), src, n * sizeof(double), cudaMemcpyDefault, s));
  return env_derive(env, s);
}

tnmc_status tnmc_env_set_params(tnmc_env* env, const float* src, void* stream) {
  g_err[0] = 0;
  CHECK_ARG(env && src, "env and src must be non-null");
  tnmc_status st = check_precision(env, TNMC_F32);
  if (st != TNMC_OK) return st;
  const size_t n = (size_t)env->d.Lx * env->d.Ly * env->d.P * 2 * env->d.P;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TNMC_CUDA_TRY(cudaMemcpyAsync(const_cast<float*>(env->d.L32), src, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return tnmc_launch_rederive_f32(env, s);
}

}  // extern "C"
