// Batched persistent form: many independent disorder instances of uneven size
// and bond dimension sampled in one launch (the independence sampler of
// Sec. 2, eqs. pi-approx and tns-prior, applied to every instance), with the
// Metropolis-Hastings scan of eq. mh-acc / Algorithm 1 run for every chain of
// every instance in one launch.
//
// A plan fixes the instances, the proposals per instance B_i, the chains per
// instance C, the precision (FP64 or FP32), the tile width NT and the order of
// the work items.  One work item is one tile of NT samples of one instance;
// the items sit in a device list (instance order, or longest-first by the
// instance's per-sample cost) and a persistent grid of nSM x (CTAs per SM)
// pulls them from an atomic counter, so that instances whose costs differ by
// two orders of magnitude still fill the machine.  Each item runs the same
// per-tile body as the single-instance SIMT sampler, so its outputs equal the
// single-instance call at the same sample indices bit for bit.
//
// Sample indices: instance i at step k draws samples (i << 40) + k B_i + b;
// its MH uniforms use t = (i << 40) + k T_i + j with T_i = B_i / C.  The pair
// (seed, k) lives in device memory, so that a captured CUDA graph replays
// fresh steps after tnmc_batch_advance.
#include <algorithm>
#include <new>
#include <numeric>
#include <string.h>
#include <vector>

#include "common.cuh"
#include "metropolis_kernel.cuh"
#include "sample_simt_kernel.cuh"

namespace tnmc {
namespace {

struct MhInst {
  double beta;
  int64_t n_sites;
  int64_t T;            // proposals per chain
  int64_t prop_row;     // first proposal row of the instance
  int64_t prop_spin;    // byte offset of its proposals in the spin arena
  int64_t chain_spin;   // byte offset of its chains in the chain arena
};

constexpr int kSampleOffsetShift = 40;

// Per-call fields of the per-instance sampler arguments (one thread per instance).
template <typename T>
__global__ void batch_prepare_kernel(SampleArgs<T>* tab, int n, const int64_t* row_off, const int64_t* spin_off,
                                     const uint64_t* params, const int8_t* spins_in, int8_t* spins_out,
                                     double* logq, double* energy, int32_t* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  SampleArgs<T>& a = tab[i];
  a.seed = params[0];
  a.offset = ((uint64_t)i << kSampleOffsetShift) + params[1] * (uint64_t)a.B;
  a.spins_in = spins_in ? spins_in + spin_off[i] : nullptr;
  a.spins_out = spins_out ? spins_out + spin_off[i] : nullptr;
  a.logq = logq + row_off[i];
  a.energy = energy + row_off[i];
  a.flags = flags ? flags + row_off[i] : nullptr;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// cta_ns[2 i], cta_ns[2 i + 1]: when CTA i started and when it found no item left (global
// timer, ns): the load balance of the launch is sum(busy) / (grid x makespan).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) sample_batched_kernel(const SampleArgs<T>* __restrict__ tab,
                                                            const int2* __restrict__ items, int64_t nitems,
                                                            unsigned int* counter, T* scratch, size_t stack_elems,
                                                            uint64_t* cta_ns) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int2 item;
  T* stack = scratch + (size_t)blockIdx.x * stack_elems;
  if (threadIdx.x == 0) cta_ns[2 * blockIdx.x] = global_ns();
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int k = atomicAdd(counter, 1u);
      item = (k < (uint64_t)nitems) ? items[k] : make_int2(-1, -1);
    }
    __syncthreads();
    const int2 it = item;
    __syncthreads();
    if (it.x < 0) break;
    const SampleArgs<T> a = tab[it.x];
    sample_simt_tile<T, NT>(a, it.y, smem_raw, stack);
  }
  if (threadIdx.x == 0) cta_ns[2 * blockIdx.x + 1] = global_ns();
}

// One thread per chain (g = i C + c), sequential over the chain's T_i proposals.
__global__ void mh_batched_scan_kernel(const MhInst* __restrict__ inst, int64_t total, int64_t C,
                                       const uint64_t* params, const double* __restrict__ prop_logq,
                                       const double* __restrict__ prop_E, double* chain_logq, double* chain_E,
                                       uint8_t* accepted, int64_t* last, int64_t* n_accepted) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int64_t i = g / C, c = g % C;
  const MhInst I = inst[i];
  const uint64_t seed = params[0];
  const uint64_t t0 = ((uint64_t)i << kSampleOffsetShift) + params[1] * (uint64_t)I.T;
  double lq = chain_logq[g], E = chain_E[g];
  // Delta = a(prop) - a(cur), a = -beta E - log q, each step rounded once (eq. mh-acc)
  double wc = __dsub_rn(__dmul_rn(-I.beta, E), lq);
  int64_t lastj = -1, cnt = 0;
  for (int64_t j = 0; j < I.T; ++j) {
    const int64_t row = I.prop_row + c * I.T + j;
    const double u = mh_uniform(seed, t0 + (uint64_t)j, (uint32_t)c);
    const double lqt = prop_logq[row], Et = prop_E[row];
    const double wt = __dsub_rn(__dmul_rn(-I.beta, Et), lqt);
    const double d = __dsub_rn(wt, wc);
    const bool ok = isfinite(lqt) && !isnan(d);
    // a state with log q = -inf (only a random start can be one) takes the first valid proposal
    const bool acc = ok && (lq == -INFINITY || u < exp(fmin(d, 0.0)));
    if (accepted) accepted[row] = acc ? 1 : 0;
    if (acc) {
      lq = lqt;
      E = Et;
      wc = wt;
      lastj = c * I.T + j;
      ++cnt;
    }
  }
  chain_logq[g] = lq;
  chain_E[g] = E;
  last[g] = lastj;
  if (n_accepted && cnt) atomicAdd(reinterpret_cast<unsigned long long*>(n_accepted + i), (unsigned long long)cnt);
}

// The last accepted proposal of every chain becomes its state (one CTA per chain).
__global__ void mh_batched_copy_kernel(const MhInst* __restrict__ inst, int64_t total, int64_t C,
                                       const int64_t* last, const int8_t* __restrict__ prop, int8_t* chain) {
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int64_t t = last[g];
    if (t < 0) continue;
    const int64_t i = g / C, c = g % C;
    const MhInst I = inst[i];
    const int8_t* src = prop + I.prop_spin + t * I.n_sites;
    int8_t* dst = chain + I.chain_spin + c * I.n_sites;
    for (int64_t k = threadIdx.x; k < I.n_sites; k += blockDim.x) dst[k] = src[k];
  }
}

// Random +-1 start of chain c of instance i: chain id (i << 32) | c in the
// counter (site / 128, id_lo, id_hi, 2), spin = +1 iff bit site % 128 is set.
__global__ void init_batched_kernel(const MhInst* __restrict__ inst, int64_t total, int64_t C, uint64_t seed,
                                    int8_t* chain) {
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int64_t i = g / C, c = g % C;
    const MhInst I = inst[i];
    int8_t* dst = chain + I.chain_spin + c * I.n_sites;
    for (int64_t site = threadIdx.x; site < I.n_sites; site += blockDim.x) {
      U4 ctr{(uint32_t)(site >> 7), (uint32_t)c, (uint32_t)i, 2u};
      const U4 o = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
      const int j = (int)(site & 127);
      const uint32_t word = (j < 32) ? o.x : (j < 64) ? o.y : (j < 96) ? o.z : o.w;
      dst[site] = ((word >> (j & 31)) & 1u) ? 1 : -1;
    }
  }
}

// Metropolis sweeps of every chain (one CTA per chain at a time): chain c of instance i
// has id i C + c and, at plan step k, runs sweeps k * sweeps .. k * sweeps + sweeps - 1.
__global__ void metropolis_batched_kernel(const MetroInst* __restrict__ inst, int64_t total, int64_t C,
                                          const uint64_t* params, int sweeps, int8_t* chains) {
  extern __shared__ int8_t sm[];
  const uint64_t seed = params[0];
  const uint32_t sweep0 = (uint32_t)(params[1] * (uint64_t)sweeps);
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int64_t i = g / C, c = g % C;
    const MetroInst I = inst[i];
    const int n = I.Lx * I.Ly;
    int8_t* dst = chains + I.chain_spin + c * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) sm[k] = dst[k];
    __syncthreads();
    metropolis_chain(I, sm, seed, (uint32_t)g, sweep0, sweeps);
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = sm[k];
    __syncthreads();
  }
}

// Link overlap of replica pair k of instance i (output row i * half + k).
__global__ void link_overlap_batched_kernel(const MetroInst* __restrict__ inst, int64_t total, int64_t half,
                                            const int8_t* chains, double* out) {
  __shared__ long long red[32];
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int64_t i = g / half, k = g % half;
    const MetroInst I = inst[i];
    const int64_t n = (int64_t)I.Lx * I.Ly;
    const int8_t* a = chains + I.chain_spin + 2 * k * n;
    const double q = link_overlap_pair(I.Lx, I.Ly, a, a + n, red);
    if (threadIdx.x == 0) out[g] = q;
  }
}

__global__ void set_params_kernel(uint64_t* params, uint64_t seed, uint64_t step) {
  params[0] = seed;
  params[1] = step;
}

__global__ void advance_kernel(uint64_t* params) { params[1] += 1; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Per-sample work of one instance in units of multiply-adds: both sweeps touch
// every padded dc x dc1 block twice per spin value.
double instance_cost(const DeviceEnv& d) {
  double w = 0.0;
  for (int r = 0; r < d.Ly; ++r)
    for (int c = 0; c < d.Lx; ++c) {
      const int a = pad4(bond_dim_host(d.chi, d.Lx, d.Ly, r, c));
      const int b = pad4(bond_dim_host(d.chi, d.Lx, d.Ly, r, c + 1));
      w += 4.0 * a * b + 16.0;
    }
  return w;
}

}  // namespace
}  // namespace tnmc

struct tnmc_batch {
  int n = 0, precision = 0, tile = 0, order = 0;
  int64_t chains = 0;
  std::vector<tnmc_env*> envs;
  std::vector<int64_t> B, prop_row, prop_spin, chain_row, chain_spin;
  int64_t prop_rows = 0, prop_bytes = 0, chain_rows = 0, chain_bytes = 0;
  int64_t items_prop = 0, items_chain = 0;
  int grid = 0;
  size_t smem = 0, stack_elems = 0, scratch_bytes = 0, arena_bytes = 0;
  tnmc::Allocator alloc;   // the hook current when the plan was created
  // device memory: one arena for the tables, one for the per-CTA stacks
  void* arena = nullptr;
  void* scratch = nullptr;
  void* tab_prop = nullptr;    // SampleArgs<T>[n]
  void* tab_chain = nullptr;   // SampleArgs<T>[n]
  int64_t* d_prop_row = nullptr;
  int64_t* d_prop_spin = nullptr;
  int64_t* d_chain_row = nullptr;
  int64_t* d_chain_spin = nullptr;
  int2* d_items_prop = nullptr;
  int2* d_items_chain = nullptr;
  tnmc::MhInst* d_mh = nullptr;
  tnmc::MetroInst* d_metro = nullptr;
  int max_sites = 0;
  unsigned int* d_counter = nullptr;
  uint64_t* d_params = nullptr;
  int64_t* d_last = nullptr;
  uint64_t* d_cta_ns = nullptr;   // [grid][2] timers of the last sampling launch
};

namespace {

using tnmc::SampleArgs;

template <typename T>
const T* env_L(const tnmc_env* e);
template <>
const double* env_L<double>(const tnmc_env* e) { return e->d.M64; }
template <>
const float* env_L<float>(const tnmc_env* e) { return e->d.L32; }
template <typename T>
const T* env_R(const tnmc_env* e);
template <>
const double* env_R<double>(const tnmc_env* e) { return e->d.R64; }
template <>
const float* env_R<float>(const tnmc_env* e) { return e->d.R32; }
template <typename T>
const T* env_fe(const tnmc_env* e);
template <>
const double* env_fe<double>(const tnmc_env* e) { return e->d.fe; }
template <>
const float* env_fe<float>(const tnmc_env* e) { return e->d.fe32; }

template <typename T, int NT>
tnmc_status plan_kernel_setup(tnmc_batch* p, int max_P, int max_W) {
  using namespace tnmc;
  auto kern = sample_batched_kernel<T, NT>;
  p->smem = (size_t)3 * max_P * NT * sizeof(T) + (size_t)2 * max_W * NT * sizeof(uint32_t);
  int dev = 0, nsm = 0, max_optin = 0;
  TNMC_CUDA_TRY(cudaGetDevice(&dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (p->smem + sizeof(int2) > (size_t)max_optin) {
    tnmc_set_error("batched sampler needs %zu bytes of shared memory per CTA (device allows %d)", p->smem, max_optin);
    return TNMC_E_UNSUPPORTED;
  }
  TNMC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem));
  int per_sm = 0;
  TNMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, p->smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)nsm * per_sm;
  const int64_t most = std::max(p->items_prop, p->items_chain);
  if (grid > most) grid = most;
  if (grid < 1) grid = 1;
  p->grid = (int)grid;
  p->scratch_bytes = (size_t)grid * p->stack_elems * sizeof(T);
  return TNMC_OK;
}

template <typename T>
void fill_table(const tnmc_batch* p, std::vector<SampleArgs<T>>& tab, bool chains) {
  tab.resize(p->n);
  for (int i = 0; i < p->n; ++i) {
    SampleArgs<T>& a = tab[i];
    memset(&a, 0, sizeof(a));
    a.e = p->envs[i]->d;
    a.L = env_L<T>(p->envs[i]);
    a.Rt = env_R<T>(p->envs[i]);
    a.fe = env_fe<T>(p->envs[i]);
    a.B = chains ? p->chains : p->B[i];
    a.scratch = nullptr;
  }
}

template <typename T, int NT>
tnmc_status launch_batched(tnmc_batch* p, bool chains, const int8_t* spins_in, int8_t* spins_out, double* logq,
                           double* energy, int32_t* flags, cudaStream_t s) {
  using namespace tnmc;
  const int64_t nitems = chains ? p->items_chain : p->items_prop;
  if (nitems == 0) return TNMC_OK;
  auto* tab = static_cast<SampleArgs<T>*>(chains ? p->tab_chain : p->tab_prop);
  const int64_t* row = chains ? p->d_chain_row : p->d_prop_row;
  const int64_t* spin = chains ? p->d_chain_spin : p->d_prop_spin;
  batch_prepare_kernel<T><<<(p->n + 127) / 128, 128, 0, s>>>(tab, p->n, row, spin, p->d_params, spins_in,
                                                             spins_out, logq, energy, flags);
  TNMC_CUDA_TRY(cudaGetLastError());
  unsigned int* counter = p->d_counter + (chains ? 1 : 0);
  TNMC_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
  sample_batched_kernel<T, NT><<<p->grid, NT, p->smem, s>>>(tab, chains ? p->d_items_chain : p->d_items_prop, nitems,
                                                            counter, static_cast<T*>(p->scratch), p->stack_elems,
                                                            p->d_cta_ns);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status dispatch_batched(tnmc_batch* p, bool chains, const int8_t* spins_in, int8_t* spins_out, double* logq,
                             double* energy, int32_t* flags, cudaStream_t s) {
  if (p->precision == TNMC_F64)
    return p->tile == 64 ? launch_batched<double, 64>(p, chains, spins_in, spins_out, logq, energy, flags, s)
                         : launch_batched<double, 128>(p, chains, spins_in, spins_out, logq, energy, flags, s);
  return p->tile == 64 ? launch_batched<float, 64>(p, chains, spins_in, spins_out, logq, energy, flags, s)
                       : launch_batched<float, 128>(p, chains, spins_in, spins_out, logq, energy, flags, s);
}

#define CHECK_ARG(cond, ...)       \
  do {                             \
    if (!(cond)) {                 \
      tnmc_set_error(__VA_ARGS__); \
      return TNMC_E_INVALID_ARG;   \
    }                              \
  } while (0)

void free_plan(tnmc_batch* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  tnmc::dev_free(p->alloc, p->scratch, p->scratch_bytes, nullptr);
  tnmc::dev_free(p->alloc, p->arena, p->arena_bytes, nullptr);
  cudaDeviceSynchronize();
  delete p;
}

}  // namespace

extern "C" {

tnmc_status tnmc_batch_create(int n, tnmc_env* const* envs, const int64_t* B, int64_t chains, int precision,
                              int tile, int order, void* stream, tnmc_batch** out) {
  using namespace tnmc;
  tnmc_set_error("");
  CHECK_ARG(out, "out must be non-null");
  *out = nullptr;
  CHECK_ARG(n >= 1 && n <= (1 << 20), "n = %d must be in [1, 2^20]", n);
  CHECK_ARG(envs && B, "envs and B must be non-null");
  CHECK_ARG(chains >= 1, "chains = %lld must be >= 1", (long long)chains);
  CHECK_ARG(precision == TNMC_F64 || precision == TNMC_F32, "the batched sampler runs in FP64 or FP32");
  CHECK_ARG(tile == 64 || tile == 128, "tile = %d must be 64 or 128", tile);
  CHECK_ARG(order == 0 || order == 1, "order = %d must be 0 (instance) or 1 (longest first)", order);
  for (int i = 0; i < n; ++i) {
    CHECK_ARG(envs[i], "envs[%d] is null", i);
    CHECK_ARG(envs[i]->precision_mask & (1 << precision), "envs[%d] was built without this precision", i);
    CHECK_ARG(B[i] >= 0 && B[i] % chains == 0, "B[%d] = %lld must be a non-negative multiple of chains", i,
              (long long)B[i]);
    CHECK_ARG(B[i] < ((int64_t)1 << kSampleOffsetShift), "B[%d] too large", i);
  }
  tnmc_batch* p = new (std::nothrow) tnmc_batch();
  if (!p) {
    tnmc_set_error("host allocation failed");
    return TNMC_E_NOMEM;
  }
  p->n = n;
  p->precision = precision;
  p->tile = tile;
  p->order = order;
  p->chains = chains;
  p->envs.assign(envs, envs + n);
  p->B.assign(B, B + n);
  p->prop_row.resize(n);
  p->prop_spin.resize(n);
  p->chain_row.resize(n);
  p->chain_spin.resize(n);
  int max_P = 1, max_W = 1;
  size_t max_stack = 1;
  std::vector<double> cost(n);
  std::vector<tnmc::MhInst> mh(n);
  std::vector<tnmc::MetroInst> metro(n);
  for (int i = 0; i < n; ++i) {
    const DeviceEnv& d = envs[i]->d;
    const int64_t ns = (int64_t)d.Lx * d.Ly;
    p->prop_row[i] = p->prop_rows;
    p->prop_spin[i] = p->prop_bytes;
    p->chain_row[i] = p->chain_rows;
    p->chain_spin[i] = p->chain_bytes;
    p->prop_rows += B[i];
    p->prop_bytes += B[i] * ns;
    p->chain_rows += chains;
    p->chain_bytes += chains * ns;
    p->items_prop += (B[i] + tile - 1) / tile;
    p->items_chain += (chains + tile - 1) / tile;
    max_P = std::max(max_P, d.P);
    max_W = std::max(max_W, (d.Lx + 31) / 32);
    max_stack = std::max(max_stack, (size_t)(d.Lx + 1) * d.P * tile);
    cost[i] = instance_cost(d);
    mh[i] = tnmc::MhInst{d.beta, ns, B[i] / chains, p->prop_row[i], p->prop_spin[i], p->chain_spin[i]};
    metro[i] = tnmc::MetroInst{d.Jh, d.Jv, d.h, d.beta, d.Lx, d.Ly, p->chain_spin[i]};
    p->max_sites = std::max(p->max_sites, (int)ns);
  }
  if (p->items_prop >= (1ll << 31) || p->items_chain >= (1ll << 31)) {
    delete p;
    tnmc_set_error("too many work items");
    return TNMC_E_INVALID_ARG;
  }
  p->stack_elems = max_stack;
  // work items: (instance, tile); longest first orders by per-sample cost, ties by instance
  auto make_items = [&](bool ch) {
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    if (order == 1) std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<int2> items;
    for (int i : idx) {
      const int64_t cnt = ch ? chains : B[i];
      for (int64_t t = 0; t * tile < cnt; ++t) items.push_back(make_int2(i, (int)t));
    }
    return items;
  };
  const std::vector<int2> ip = make_items(false), ic = make_items(true);

  tnmc_status st = (precision == TNMC_F64)
                       ? (tile == 64 ? plan_kernel_setup<double, 64>(p, max_P, max_W)
                                     : plan_kernel_setup<double, 128>(p, max_P, max_W))
                       : (tile == 64 ? plan_kernel_setup<float, 64>(p, max_P, max_W)
                                     : plan_kernel_setup<float, 128>(p, max_P, max_W));
  if (st != TNMC_OK) {
    delete p;
    return st;
  }
  const size_t tab_bytes = (size_t)n * (precision == TNMC_F64 ? sizeof(SampleArgs<double>) : sizeof(SampleArgs<float>));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes ? bytes : 1);
    return o;
  };
  const size_t o_tp = take(tab_bytes), o_tc = take(tab_bytes);
  const size_t o_pr = take(n * 8), o_ps = take(n * 8), o_cr = take(n * 8), o_cs = take(n * 8);
  const size_t o_ip = take(ip.size() * sizeof(int2)), o_ic = take(ic.size() * sizeof(int2));
  const size_t o_mh = take(n * sizeof(tnmc::MhInst)), o_cnt = take(2 * sizeof(unsigned int));
  const size_t o_metro = take(n * sizeof(tnmc::MetroInst));
  const size_t o_par = take(2 * sizeof(uint64_t)), o_last = take((size_t)p->chain_rows * 8);
  const size_t o_ns = take((size_t)p->grid * 2 * sizeof(uint64_t));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  p->alloc = current_allocator();
  char* base = static_cast<char*>(dev_alloc(p->alloc, off, s));
  p->scratch = base ? dev_alloc(p->alloc, p->scratch_bytes, s) : nullptr;
  if (!base || !p->scratch) {
    const size_t sb = p->scratch_bytes;
    dev_free(p->alloc, base, off, s);
    (void)cudaStreamSynchronize(s);
    delete p;
    tnmc_set_error("cannot allocate the batch plan (%zu + %zu bytes)", off, sb);
    return TNMC_E_NOMEM;
  }
  p->arena = base;
  p->arena_bytes = off;
  p->tab_prop = base + o_tp;
  p->tab_chain = base + o_tc;
  p->d_prop_row = reinterpret_cast<int64_t*>(base + o_pr);
  p->d_prop_spin = reinterpret_cast<int64_t*>(base + o_ps);
  p->d_chain_row = reinterpret_cast<int64_t*>(base + o_cr);
  p->d_chain_spin = reinterpret_cast<int64_t*>(base + o_cs);
  p->d_items_prop = reinterpret_cast<int2*>(base + o_ip);
  p->d_items_chain = reinterpret_cast<int2*>(base + o_ic);
  p->d_mh = reinterpret_cast<tnmc::MhInst*>(base + o_mh);
  p->d_metro = reinterpret_cast<tnmc::MetroInst*>(base + o_metro);
  p->d_counter = reinterpret_cast<unsigned int*>(base + o_cnt);
  p->d_params = reinterpret_cast<uint64_t*>(base + o_par);
  p->d_last = reinterpret_cast<int64_t*>(base + o_last);
  p->d_cta_ns = reinterpret_cast<uint64_t*>(base + o_ns);

  // host images of the tables, uploaded once; the call returns after the upload
  std::vector<char> tp(tab_bytes), tc(tab_bytes);
  if (precision == TNMC_F64) {
    std::vector<SampleArgs<double>> a, b;
    fill_table<double>(p, a, false);
    fill_table<double>(p, b, true);
    memcpy(tp.data(), a.data(), tab_bytes);
    memcpy(tc.data(), b.data(), tab_bytes);
  } else {
    std::vector<SampleArgs<float>> a, b;
    fill_table<float>(p, a, false);
    fill_table<float>(p, b, true);
    memcpy(tp.data(), a.data(), tab_bytes);
    memcpy(tc.data(), b.data(), tab_bytes);
  }
  cudaError_t e = cudaMemsetAsync(base, 0, off, s);
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  };
  up(p->tab_prop, tp.data(), tab_bytes);
  up(p->tab_chain, tc.data(), tab_bytes);
  up(p->d_prop_row, p->prop_row.data(), n * 8);
  up(p->d_prop_spin, p->prop_spin.data(), n * 8);
  up(p->d_chain_row, p->chain_row.data(), n * 8);
  up(p->d_chain_spin, p->chain_spin.data(), n * 8);
  up(p->d_items_prop, ip.data(), ip.size() * sizeof(int2));
  up(p->d_items_chain, ic.data(), ic.size() * sizeof(int2));
  up(p->d_mh, mh.data(), n * sizeof(tnmc::MhInst));
  up(p->d_metro, metro.data(), n * sizeof(tnmc::MetroInst));
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    tnmc_set_error("batch plan upload failed: %s", cudaGetErrorString(e));
    free_plan(p);
    return TNMC_E_CUDA;
  }
  *out = p;
  return TNMC_OK;
}

tnmc_status tnmc_batch_free(tnmc_batch* p) {
  free_plan(p);
  return TNMC_OK;
}

tnmc_status tnmc_batch_info(const tnmc_batch* p, tnmc_batch_info_t* info) {
  CHECK_ARG(p && info, "plan and info must be non-null");
  info->n = p->n;
  info->precision = p->precision;
  info->tile = p->tile;
  info->order = p->order;
  info->grid = p->grid;
  info->chains = p->chains;
  info->proposal_rows = p->prop_rows;
  info->proposal_bytes = p->prop_bytes;
  info->chain_rows = p->chain_rows;
  info->chain_bytes = p->chain_bytes;
  info->items = p->items_prop;
  info->smem_bytes = (int64_t)p->smem;
  info->scratch_bytes = (int64_t)p->scratch_bytes;
  return TNMC_OK;
}

tnmc_status tnmc_batch_balance(const tnmc_batch* p, double* efficiency, double* makespan_ms) {
  CHECK_ARG(p && efficiency, "plan and efficiency must be non-null");
  std::vector<uint64_t> t((size_t)p->grid * 2);
  TNMC_CUDA_TRY(cudaDeviceSynchronize());
  TNMC_CUDA_TRY(cudaMemcpy(t.data(), p->d_cta_ns, t.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  uint64_t lo = UINT64_MAX, hi = 0;
  double busy = 0.0;
  for (int i = 0; i < p->grid; ++i) {
    const uint64_t a = t[2 * i], b = t[2 * i + 1];
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
    busy += (b > a) ? (double)(b - a) : 0.0;
  }
  const double span = (hi > lo) ? (double)(hi - lo) : 0.0;
  *efficiency = span > 0.0 ? busy / ((double)p->grid * span) : 0.0;
  if (makespan_ms) *makespan_ms = span * 1e-6;
  return TNMC_OK;
}

tnmc_status tnmc_batch_layout(const tnmc_batch* p, int64_t* prop_row, int64_t* prop_spin, int64_t* chain_row,
                              int64_t* chain_spin) {
  CHECK_ARG(p, "plan must be non-null");
  for (int i = 0; i < p->n; ++i) {
    if (prop_row) prop_row[i] = p->prop_row[i];
    if (prop_spin) prop_spin[i] = p->prop_spin[i];
    if (chain_row) chain_row[i] = p->chain_row[i];
    if (chain_spin) chain_spin[i] = p->chain_spin[i];
  }
  return TNMC_OK;
}

tnmc_status tnmc_batch_set_step(tnmc_batch* p, uint64_t seed, uint64_t step, void* stream) {
  CHECK_ARG(p, "plan must be non-null");
  tnmc::set_params_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(p->d_params, seed, step);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_batch_advance(tnmc_batch* p, void* stream) {
  CHECK_ARG(p, "plan must be non-null");
  tnmc::advance_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(p->d_params);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_sample_batched(tnmc_batch* p, int8_t* prop_spins, double* prop_logq, double* prop_energy,
                                int32_t* flags, void* stream) {
  CHECK_ARG(p, "plan must be non-null");
  CHECK_ARG(p->prop_rows == 0 || (prop_spins && prop_logq && prop_energy),
            "prop_spins, prop_logq and prop_energy must be non-null");
  return dispatch_batched(p, false, nullptr, prop_spins, prop_logq, prop_energy, flags,
                          static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc_logq_batched(tnmc_batch* p, const int8_t* prop_spins, double* prop_logq, double* prop_energy,
                              int32_t* flags, void* stream) {
  CHECK_ARG(p, "plan must be non-null");
  CHECK_ARG(p->prop_rows == 0 || (prop_spins && prop_logq && prop_energy),
            "prop_spins, prop_logq and prop_energy must be non-null");
  return dispatch_batched(p, false, prop_spins, nullptr, prop_logq, prop_energy, flags,
                          static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc_batch_init_chains(tnmc_batch* p, uint64_t seed, int8_t* chain_spins, double* chain_logq,
                                   double* chain_energy, void* stream) {
  using namespace tnmc;
  CHECK_ARG(p, "plan must be non-null");
  CHECK_ARG(chain_spins && chain_logq && chain_energy, "chain arrays must be non-null");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t total = p->chain_rows;
  init_batched_kernel<<<(unsigned)std::min<int64_t>(total, 65535), 256, 0, s>>>(p->d_mh, total, p->chains, seed,
                                                                               chain_spins);
  TNMC_CUDA_TRY(cudaGetLastError());
  return dispatch_batched(p, true, chain_spins, nullptr, chain_logq, chain_energy, nullptr, s);
}

tnmc_status tnmc_mh_batched(tnmc_batch* p, const int8_t* prop_spins, const double* prop_logq,
                            const double* prop_energy, int8_t* chain_spins, double* chain_logq,
                            double* chain_energy, uint8_t* accepted, int64_t* n_accepted, void* stream) {
  using namespace tnmc;
  CHECK_ARG(p, "plan must be non-null");
  CHECK_ARG(prop_spins && prop_logq && prop_energy && chain_spins && chain_logq && chain_energy,
            "proposal and chain arrays must be non-null");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t total = p->chain_rows;
  mh_batched_scan_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(
      p->d_mh, total, p->chains, p->d_params, prop_logq, prop_energy, chain_logq, chain_energy, accepted, p->d_last,
      n_accepted);
  TNMC_CUDA_TRY(cudaGetLastError());
  mh_batched_copy_kernel<<<(unsigned)std::min<int64_t>(total, 65535), 256, 0, s>>>(p->d_mh, total, p->chains,
                                                                                  p->d_last, prop_spins, chain_spins);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_metropolis_batched(tnmc_batch* p, int8_t* chain_spins, double* chain_logq, double* chain_energy,
                                    int sweeps, void* stream) {
  using namespace tnmc;
  CHECK_ARG(p, "plan must be non-null");
  CHECK_ARG(sweeps >= 0, "sweeps must be >= 0");
  CHECK_ARG(chain_spins && chain_logq && chain_energy, "chain arrays must be non-null");
  CHECK_ARG(p->max_sites <= 200 * 1024, "a chain of %d sites does not fit in shared memory", p->max_sites);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t total = p->chain_rows;
  if (sweeps > 0) {
    const size_t smem = (size_t)p->max_sites;
    if (smem > 48 * 1024)
      TNMC_CUDA_TRY(cudaFuncSetAttribute(metropolis_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    metropolis_batched_kernel<<<(unsigned)std::min<int64_t>(total, 65535), 256, smem, s>>>(
        p->d_metro, total, p->chains, p->d_params, sweeps, chain_spins);
    TNMC_CUDA_TRY(cudaGetLastError());
  }
  return dispatch_batched(p, true, chain_spins, nullptr, chain_logq, chain_energy, nullptr, s);
}

tnmc_status tnmc_link_overlap_batched(tnmc_batch* p, const int8_t* chain_spins, double* overlap, void* stream) {
  using namespace tnmc;
  CHECK_ARG(p, "plan must be non-null");
  CHECK_ARG(p->chains % 2 == 0, "chains = %lld must be even (replica pairs)", (long long)p->chains);
  CHECK_ARG(chain_spins && overlap, "chain_spins and overlap must be non-null");
  const int64_t half = p->chains / 2;
  const int64_t total = (int64_t)p->n * half;
  if (total == 0) return TNMC_OK;
  link_overlap_batched_kernel<<<(unsigned)std::min<int64_t>(total, 65535), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      p->d_metro, total, half, chain_spins, overlap);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

}  // extern "C"
