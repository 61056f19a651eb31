// BF16 tensor-core sampler / evaluator of q = pi~ (Sec. 2, eqs. bayes, pi-approx;
// App. A) for sm_103a: tcgen05.mma with the accumulator in TMEM, environment tiles
// streamed into shared memory by bulk async copies, FP32 accumulation.
//
// A CTA owns a tile of 128 samples (UMMA M = 128): sample t is TMEM lane t.  Per
// site one UMMA 128 x 128 x 64 forms, for all samples at once,
//   right sweep  D[t][(u, a)] = sum_b R_{c+1}[t][b] Mt^(u)_c[a][b]   -> R_c = D(u_t, -)
//   left sweep   D[t][(s, b)] = sum_a Lambda_c[t][a] M_c[a][s][b]     -> U[s] = D(s, -)
// where Mt^(u) = sum_s f_u(s) M[:, s, :] is the site tensor with the field factor of the
// spin above (u) already applied (both u at once; the epilogue keeps the sample's own),
// with the vectors (A operand, 128 x 64) in shared memory and the environment tile
// (B operand, 128 x 64) loaded from a pre-swizzled copy of the environment.  Both
// operands are BF16 hi + lo pairs; the three products hi*hi + lo*hi + hi*lo keep
// about 16 significant bits (the lo*lo term is below that).
//
// 256 threads: thread (t, h) = (tid % 128, tid / 128) runs the epilogue of sample t
// for the components k in [32h, 32h + 32) -- warps w and w + 4 read the same TMEM
// lanes (lane quadrant w % 4) at different columns, 16 columns per load.  The two
// halves exchange their partial maxima (right steps) or partial dot products (left
// steps) through shared memory under a named barrier per warp pair, and take
// identical decisions from identical sums.  Every rescaling is by a power of two,
// which leaves the arithmetic of q unchanged: right vectors by their max, left vectors
// by the drawn weight w(s) (which the left step has already summed).
//
// The left sweep needs R_{c+1} in the reverse of the order the right sweep makes it:
// the right sweep writes every R_c into a shared buffer, from which one 32 KB bulk store
// moves it to a per-CTA stack in global memory (Lx x 32 KB per tile and row) during the
// next step's UMMA; the left sweep brings it back with one bulk copy into the buffer,
// issued with the step's UMMA (and prefetched into L2 a step earlier).  The
// environment tile of the next step is copied as soon as the UMMA has read the current
// one, while the epilogue runs.  Steps per row: (Lx - 1) right + Lx left.
#include <math.h>
#include <stdlib.h>

#include "common.cuh"
#include "umma.cuh"

namespace tnmc {
namespace {

constexpr int kTile = 128;          // samples per CTA (UMMA M)
constexpr int kThreads = 256;       // two epilogue threads per sample
constexpr int kK = 64;              // padded bond dimension (UMMA K per site)
constexpr int kN = 128;             // 2 x 64 outputs (UMMA N)
constexpr uint32_t kTileBytes = kN * kK * 2;   // 16 KiB: one BF16 operand tile
constexpr uint32_t kStageBytes = 2 * kTileBytes;   // hi + lo tiles of one (r, c)
constexpr uint32_t kVecBytes = kTile * kK * 2;  // 16 KiB (one BF16 A operand)
constexpr uint32_t kRBytes = kTile * kK * 4;    // 32 KiB: R_{c+1} of the tile, FP32
constexpr uint32_t kPollLimit = 1u << 16;    // polls of a bounded wait ...
constexpr uint32_t kPollHintNs = 1u << 16;   // ... each parked up to ~65 us: at most ~4 s

struct TcArgs {
  DeviceEnv e;
  const __nv_bfloat16* TR;   // [Ly*Lx] right-sweep tiles (n = s*64 + a, k = b), SW128
  const __nv_bfloat16* TL;   // [Ly*Lx] left-sweep tiles  (n = s*64 + b, k = a), SW128
  const float* fe;           // [Ly][Lx][2]
  const float* h32;          // [Ly][Lx]
  const float* Jh32;         // [Ly][Lx-1]
  const float* Jv32;         // [Ly-1][Lx]
  int64_t B;
  uint64_t seed, offset;
  const int8_t* spins_in;
  int8_t* spins_out;
  double* logq;
  double* energy;
  int32_t* flags;
  float4* stack;             // per CTA: [Lx][2 halves][8 chunks][128 samples] float4
  const double* h64;         // FP64 couplings: the energy of non-integer instances
  const double* Jh64;
  const double* Jv64;
  uint32_t poll_limit;       // polls of each wait inside the sampling loop (kPollLimit;
                             // 0 makes every such wait give up at once)
};

__device__ inline float pow2f(int e) { return __int_as_float((e + 127) << 23); }   // 2^e, |e| < 127
__device__ inline int ilogb_f(float x) { return ((__float_as_int(x) >> 23) & 0xff) - 127; }   // x normal, > 0

// Split 8 FP32 values (components k0 .. k0+7, k0 a multiple of 8) into BF16 hi + lo and
// store them in row t of the two swizzled A operands (one 16-byte chunk each).
__device__ inline void store_split8(unsigned char* sHi, unsigned char* sLo, int t, int k0, const float* v) {
  uint32_t wh[4], wl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = v[2 * q], x1 = v[2 * q + 1];
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - __low2float(h2), x1 - __high2float(h2));
    wh[q] = *reinterpret_cast<const uint32_t*>(&h2);
    wl[q] = *reinterpret_cast<const uint32_t*>(&l2);
  }
  const uint32_t off = umma::sw128_offset(t, k0);
  *reinterpret_cast<uint4*>(sHi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
  *reinterpret_cast<uint4*>(sLo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

// Split 32 FP32 values (components 32h .. 32h+31) into BF16 hi + lo and store them in
// row t of the two swizzled A operands.
__device__ inline void store_split_half(unsigned char* sHi, unsigned char* sLo, int t, int h, const float* v) {
#pragma unroll
  for (int j = 0; j < 4; ++j) store_split8(sHi, sLo, t, 32 * h + 8 * j, v + 8 * j);
}

// e_0 restricted to this thread's half
__device__ inline void unit_half(float* v, int h) {
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = (h == 0 && q == 0) ? 1.0f : 0.0f;
}

// Bulk store shared -> global (one group per call), and the waits on it.
__device__ inline void bulk_s2g(void* dst, uint32_t src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src_smem), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ inline void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ inline void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ inline void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ inline void pair_sync(int warp) {
  asm volatile("bar.sync %0, 64;" ::"r"(1 + (warp & 3)) : "memory");
}

__global__ void __launch_bounds__(kThreads, 2) sample_tc_kernel(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* sHi = base;
  unsigned char* sLo = base + kVecBytes;
  unsigned char* sB = base + 2 * kVecBytes;                                   // environment tile (hi, lo)
  float4* sR = reinterpret_cast<float4*>(sB + kStageBytes);                  // [2][8][128] float4
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStageBytes + kRBytes);  // [0] tile, [1] UMMA, [2] R
  uint32_t* misc = reinterpret_cast<uint32_t*>(bars + 3);                    // [0] tmem base, [1] abort, [2] tile ok
  // thread 0's copy counters live in shared memory (registers are the scarce resource):
  // [0] environment tiles copied, [1] R copies issued, [2] R copies waited for
  int64_t* cnt = reinterpret_cast<int64_t*>(misc + 4);
  float* xw = reinterpret_cast<float*>(misc + 10);   // left steps: [2 halves][2][128] partial w(-), w(+)
  float* xmb = xw + 4 * kTile;                      // right steps: [2 steps][2 halves][128] partial max
  const int Lx = a.e.Lx, Ly = a.e.Ly;
  const int W = (Lx + 31) >> 5;
  uint32_t* xs = reinterpret_cast<uint32_t*>(xw + 8 * kTile);   // [2][128]: the site's 64-bit uniform
  uint32_t* bits_prev = xs + 2 * kTile;
  uint32_t* bits_cur = bits_prev + W * kTile;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int t = tid & (kTile - 1), h = tid >> 7;
  const int64_t ntiles = (a.B + kTile - 1) / kTile;
  const int S = 2 * Lx - 1;
  const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
  const int64_t total_steps = my_tiles * (int64_t)Ly * S;
  const int n = Lx * Ly;
  float4* stk_cta = a.stack + (size_t)blockIdx.x * Lx * (2 * 8 * kTile);
  float4* stk = stk_cta + (size_t)h * (8 * kTile) + t;
  const uint32_t idesc = umma::idesc_bf16_f32(kTile, kN);

  if (warp == 0) umma::tmem_alloc(umma::smem_u32(&misc[0]), kN);
  if (tid == 0) {
    // the UMMA barrier completes on the commit and on thread 0, once the bulk store of the
    // step (if any) has read the R buffer
    for (int s = 0; s < 3; ++s) umma::mbar_init(umma::smem_u32(&bars[s]), s == 1 ? 2 : 1);
    umma::fence_mbar_init();
    misc[1] = 0;
    misc[2] = 1;
    cnt[0] = cnt[1] = cnt[2] = 0;
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = misc[0];
  const uint32_t tlane = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * h;

  // producer position (row, step within the row) of the next tile to load
  int prod_r = 0, prod_i = 0;
  auto next_tile = [&]() -> const __nv_bfloat16* {
    const bool left = prod_i >= Lx - 1;
    const int c = left ? prod_i - (Lx - 1) : Lx - 1 - prod_i;
    const __nv_bfloat16* T = (left ? a.TL : a.TR) + ((size_t)prod_r * Lx + c) * (2 * kN * kK);
    if (++prod_i == S) {
      prod_i = 0;
      if (++prod_r == Ly) prod_r = 0;
    }
    return T;
  };

  uint32_t nr = 0;                   // R copies consumed (every thread)
  if (tid == 0 && total_steps > 0) {
    umma::mbar_expect_tx(umma::smem_u32(&bars[0]), kStageBytes);
    umma::bulk_g2s(umma::smem_u32(sB), next_tile(), kStageBytes, umma::smem_u32(&bars[0]));
    cnt[0] = 1;
  }

  int64_t g = 0;
  bool abort = false;
  for (int64_t tile = blockIdx.x; tile < ntiles && !abort; tile += gridDim.x) {
    const int64_t b = tile * kTile + t;
    const bool active = b < a.B;
    const uint64_t sample = a.offset + (uint64_t)b;
    double lq = 0.0, E = 0.0;
    int flag = 0;
    if (h == 0)
      for (int wd = 0; wd < W; ++wd) bits_prev[wd * kTile + t] = 0u;
    uint64_t pair_word = 0;
    int64_t pair_id = -1;
    for (int r = 0; r < Ly && !abort; ++r) {
      const float* fe_row = a.fe + (size_t)r * Lx * 2;
      const float* h_row = a.h32 + (size_t)r * Lx;
      const float* jh_row = a.Jh32 + (size_t)r * (Lx - 1);
      const float* jv_row = a.Jv32 + (size_t)(r > 0 ? r - 1 : 0) * Lx;
      if (a.spins_in && h == 0) {
        for (int wd = 0; wd < W; ++wd) bits_cur[wd * kTile + t] = 0u;
        if (active) {
          const int8_t* src = a.spins_in + (size_t)b * n + (size_t)r * Lx;
          for (int c = 0; c < Lx; ++c)
            if (src[c] > 0) bits_cur[(c >> 5) * kTile + t] |= 1u << (c & 31);
        }
      }
      // row start: A = R_{Lx} = e_0 (Lx > 1) or Lambda_0 = e_0 (Lx = 1), whose max is 1
      {
        float v[32];
        unit_half(v, h);
        store_split_half(sHi, sLo, t, h, v);
        xmb[((g + 1) & 1) * (2 * kTile) + h * kTile + t] = 1.0f;
      }
      float prod = 1.0f;
      int pexp = 0;
      float Erow = 0.0f;      // integer couplings: exact in FP32 (others: FP64 at the row end)
      int s_left = 0;
      umma::fence_proxy_async();
      umma::fence_before_sync();
      __syncthreads();
      for (int i = 0; i < S; ++i, ++g) {
        const bool left = i >= Lx - 1;
        const int c = left ? i - (Lx - 1) : Lx - 1 - i;
        // R_1 is still in the buffer when the left sweep starts; later R_{c+1} come back by copy
        const bool rcopy = left && c >= 1 && c + 1 < Lx;
        umma::fence_after_sync();
        if (tid == 0) {
          if (rcopy) {   // R_{c+1} of the whole tile: the buffer was last read before the step's barrier
            bulk_wait_all();   // the stack stores of the right sweep have landed
            umma::mbar_expect_tx(umma::smem_u32(&bars[2]), kRBytes);
            umma::bulk_g2s(umma::smem_u32(sR), stk_cta + (size_t)(c + 1) * (2 * 8 * kTile), kRBytes,
                           umma::smem_u32(&bars[2]));
            ++cnt[1];
          }
          const bool tile_ok = umma::mbar_wait_parked(umma::smem_u32(&bars[0]), (uint32_t)(g & 1), a.poll_limit,
                                                      kPollHintNs);
          misc[2] = tile_ok;
          if (!tile_ok) {
            set_status(a.e.status, TNMC_E_TIMEOUT);
            misc[1] = 1;
          } else {
            const uint64_t ah = umma::sw128_desc(umma::smem_u32(sHi));
            const uint64_t al = umma::sw128_desc(umma::smem_u32(sLo));
            const uint64_t bh = umma::sw128_desc(umma::smem_u32(sB));
            const uint64_t bl = umma::sw128_desc(umma::smem_u32(sB + kTileBytes));
#pragma unroll
            for (int k = 0; k < kK / 16; ++k) umma::mma_bf16(tmem, ah + 2 * k, bh + 2 * k, idesc, k > 0);
#pragma unroll
            for (int k = 0; k < kK / 16; ++k) umma::mma_bf16(tmem, al + 2 * k, bh + 2 * k, idesc, 1);
#pragma unroll
            for (int k = 0; k < kK / 16; ++k) umma::mma_bf16(tmem, ah + 2 * k, bl + 2 * k, idesc, 1);
          }
          umma::mma_commit(umma::smem_u32(&bars[1]));
          const int c_prev = Lx - i;   // site of the previous step when it was a right step
          if (i >= 1 && i - 1 < Lx - 1 && c_prev >= 2) {
            // R_{c_prev}, written to the buffer by the previous epilogue, goes to the stack
            bulk_s2g(stk_cta + (size_t)c_prev * (2 * 8 * kTile), umma::smem_u32(sR), kRBytes);
            bulk_wait_read();
          }
          mbar_arrive(umma::smem_u32(&bars[1]));
        }
        // work that does not need the accumulator, overlapped with the UMMA
        const bool up = (r > 0) && ((bits_prev[(c >> 5) * kTile + t] >> (c & 31)) & 1u);
        const float fsame = (r == 0) ? 1.0f : fe_row[2 * c + 1];
        const float fdiff = (r == 0) ? 1.0f : fe_row[2 * c];
        const float fm = up ? fdiff : fsame;   // s = -1
        const float fp = up ? fsame : fdiff;   // s = +1
        uint64_t x = 0;
        // couplings of the site's energy term, read while the UMMA runs (FP32: exact for
        // integer couplings; other couplings are read in FP64 where the term is added)
        float e_h = 0.0f, e_jh = 0.0f, e_jv = 0.0f;
        if (left && h == 0 && a.e.integer_couplings) {
          e_h = h_row[c];
          if (c > 0) e_jh = jh_row[c - 1];
          if (r > 0) e_jv = jv_row[c];
        }
        if (left) {
          if (c + 2 < Lx) {
            // R_{c+2} into L2 one step ahead: each lane fetches one of its warp's 32 lines
            const int lane = tid & 31;
            const float4* pf = stk - t + 32 * (warp & 3) + (size_t)(c + 2) * (2 * 8 * kTile) +
                               (size_t)(lane >> 2) * kTile + 8 * (lane & 3);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pf));
          }
          if (!a.spins_in && h == 0) {   // half 0 draws the word, half 1 receives it with the dots
            const int64_t site = (int64_t)r * Lx + c;
            if ((site & 1) && (site >> 1) == pair_id) {
              x = pair_word;
            } else {
              pair_id = site >> 1;
              const U4 o = philox4x32_10(U4{(uint32_t)pair_id, (uint32_t)sample, (uint32_t)(sample >> 32), 0u},
                                         (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
              const uint64_t even = (uint64_t)o.x | ((uint64_t)o.y << 32);
              const uint64_t odd = (uint64_t)o.z | ((uint64_t)o.w << 32);
              x = (site & 1) ? odd : even;
              pair_word = odd;
            }
          }
        }
        const bool mma_ok = umma::mbar_wait_parked(umma::smem_u32(&bars[1]), (uint32_t)(g & 1), a.poll_limit, kPollHintNs);
        if (!mma_ok) {
          set_status(a.e.status, TNMC_E_TIMEOUT);
          misc[1] = 1;
        }
        umma::fence_after_sync();
        if (tid == 0 && mma_ok && misc[2] && cnt[0] < total_steps) {
          // the UMMA has read the tile: the next step's tile lands while the epilogue runs
          // (not after a failed wait: the UMMA, or the tile's own copy, may still use sB)
          umma::mbar_expect_tx(umma::smem_u32(&bars[0]), kStageBytes);
          umma::bulk_g2s(umma::smem_u32(sB), next_tile(), kStageBytes, umma::smem_u32(&bars[0]));
          ++cnt[0];
        }
        float v[32];
        if (!left) {
          // ---- right-sweep epilogue: R_c = Mt^(u)_c R_{c+1} for this sample's u (the spin
          // above): the UMMA formed both u halves, the epilogue selects one ----
          const uint32_t col = up ? 1u : 0u;
          uint32_t d0[16], d1[16], e0[16], e1[16];
          umma::tmem_ld16_issue(tlane, d0);
          umma::tmem_ld16_issue(tlane + 16, d1);
          umma::tmem_ld16_issue(tlane + 64, e0);
          umma::tmem_ld16_issue(tlane + 80, e1);
          // the power of two that rescales R_c comes from the full max of the previous A
          // operand (both halves' partial maxima, exchanged through the step barrier), so no
          // pair barrier is needed here: A(c) = raw_c 2^(-ilogb(max |A(c+1)|)) stays within
          // one step's growth of [1, 2)
          const float* mrd = xmb + ((g + 1) & 1) * (2 * kTile);   // written by the previous step
          const float mprev = fmaxf(mrd[t], mrd[kTile + t]);
          const float sc = (mprev > 0x1.0p-126f && mprev < INFINITY) ? pow2f(-ilogb_f(mprev)) : 1.0f;
          umma::tmem_wait_ld();
          umma::tmem_hold16(d0);
          umma::tmem_hold16(d1);
          umma::tmem_hold16(e0);
          umma::tmem_hold16(e1);
          float m4[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // four independent chains (max is exact)
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            v[q] = __uint_as_float(col ? e0[q] : d0[q]) * sc;
            v[16 + q] = __uint_as_float(col ? e1[q] : d1[q]) * sc;
            m4[q & 3] = fmaxf(m4[q & 3], fmaxf(fabsf(v[q]), fabsf(v[16 + q])));
          }
          float4* dst = sR + h * (8 * kTile) + t;   // to the stack by a bulk store next step
#pragma unroll
          for (int j = 0; j < 8; ++j) dst[j * kTile] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          if (c == 1) unit_half(v, h);           // the left sweep starts from Lambda_0 = e_0
          store_split_half(sHi, sLo, t, h, v);
          // this half's max of the new A operand, read by both halves in the next step (the
          // buffers alternate by step, so this write cannot meet this step's reads)
          xmb[(g & 1) * (2 * kTile) + h * kTile + t] = fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3]));
        } else {
          // ---- left-sweep epilogue: w(s) = f(s) <U[s], R_{c+1}>, draw, Lambda_{c+1} ----
          if (rcopy) {
            if (!umma::mbar_wait_parked(umma::smem_u32(&bars[2]), nr & 1u, a.poll_limit, kPollHintNs)) {
              set_status(a.e.status, TNMC_E_TIMEOUT);
              misc[1] = 1;
            } else if (tid == 0) {
              ++cnt[2];
            }
            ++nr;
          }
          // pass 1: partial dot products over this half, 16 components at a time
          float a0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, a1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
          const float4* src = sR + h * (8 * kTile) + t;
#pragma unroll
          for (int ch = 0; ch < 2; ++ch) {
            uint32_t p0[16], p1[16];
            umma::tmem_ld16_issue(tlane + 16 * ch, p0);
            umma::tmem_ld16_issue(tlane + 64 + 16 * ch, p1);
            umma::tmem_wait_ld();
            umma::tmem_hold16(p0);
            umma::tmem_hold16(p1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              float4 q4 = make_float4((h == 0 && ch == 0 && j == 0) ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f);
              if (c + 1 < Lx) q4 = src[(4 * ch + j) * kTile];
              const float r4[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
              for (int z = 0; z < 4; ++z) {
                a0[z] = fmaf(__uint_as_float(p0[4 * j + z]), r4[z], a0[z]);
                a1[z] = fmaf(__uint_as_float(p1[4 * j + z]), r4[z], a1[z]);
              }
            }
          }
          xw[(2 * h) * kTile + t] = (a0[0] + a0[1]) + (a0[2] + a0[3]);
          xw[(2 * h + 1) * kTile + t] = (a1[0] + a1[1]) + (a1[2] + a1[3]);
          if (h == 0) {
            xs[t] = (uint32_t)x;
            xs[kTile + t] = (uint32_t)(x >> 32);
          }
          uint32_t p0[16], p1[16];
          umma::tmem_ld16_issue(tlane, p0);
          umma::tmem_ld16_issue(tlane + 64, p1);
          pair_sync(warp);
          if (h == 1) x = (uint64_t)xs[t] | ((uint64_t)xs[kTile + t] << 32);
          float w0 = xw[t] + xw[2 * kTile + t];            // half 0 + half 1, same order in both
          float w1 = xw[kTile + t] + xw[3 * kTile + t];
          w0 = fmaxf(w0 * fm, 0.0f);
          w1 = fmaxf(w1 * fp, 0.0f);
          const float tot = w0 + w1;
          const bool bad = !(tot > 0.0f) || !isfinite(tot);
          const float pplus = bad ? 0.5f : w1 / tot;
          const float pminus = bad ? 0.5f : w0 / tot;
          bool plus;
          if (a.spins_in) plus = (bits_cur[(c >> 5) * kTile + t] >> (c & 31)) & 1u;
          else plus = draw_plus(pplus, x);
          if (h == 0) {
            if (!a.spins_in) {
              if (plus) bits_cur[(c >> 5) * kTile + t] |= 1u << (c & 31);
              else bits_cur[(c >> 5) * kTile + t] &= ~(1u << (c & 31));
            }
            prod *= plus ? pplus : pminus;
            if (prod < 0x1.0p-60f && prod > 0.0f) {
              prod *= 0x1.0p60f;
              pexp -= 60;
            }
            flag |= bad ? TNMC_FLAG_NUMERIC : 0;
            float loc = e_h;
            if (c > 0) loc += e_jh * (s_left ? 1.0f : -1.0f);
            if (r > 0) loc += e_jv * (up ? 1.0f : -1.0f);
            Erow -= (plus ? 1.0f : -1.0f) * loc;
            s_left = plus;
          }
          // Lambda_{c+1} = f(s) U[s] times a power of two: any such factor leaves q's
          // arithmetic unchanged, so it is taken from w(s) = f(s) <U[s], R_{c+1}> (already
          // summed) rather than from max |U[s]|: <Lambda_{c+1}, R_{c+1}> lands in [1, 2)
          const float ws = plus ? w1 : w0;
          const float mult = (plus ? fp : fm) * ((ws > 0x1.0p-126f && ws < INFINITY) ? pow2f(-ilogb_f(ws)) : 1.0f);
          umma::tmem_wait_ld();
          umma::tmem_hold16(p0);
          umma::tmem_hold16(p1);
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(plus ? p1[q] : p0[q]) * mult;
          umma::tmem_ld16_issue(tlane + 16, p0);
          umma::tmem_ld16_issue(tlane + 80, p1);
          umma::tmem_wait_ld();
          umma::tmem_hold16(p0);
          umma::tmem_hold16(p1);
#pragma unroll
          for (int q = 0; q < 16; ++q) v[16 + q] = __uint_as_float(plus ? p1[q] : p0[q]) * mult;
          store_split_half(sHi, sLo, t, h, v);
        }
        // the shared A operand and R buffer become visible to the UMMA and the bulk store
        umma::fence_proxy_async();
        umma::fence_before_sync();
        __syncthreads();

        if (misc[1]) {
          abort = true;
          break;
        }
      }
      // end of row: log q, energy, spins; this row becomes the previous row
      if (h == 0) {
        lq += log((double)prod) + (double)pexp * 0.69314718055994530942;
        if (a.e.integer_couplings) {
          E += (double)Erow;
        } else {
          // the row's terms of eq. ising in FP64 from its spins and the row above
          for (int c = 0; c < Lx; ++c) {
            const bool sc = (bits_cur[(c >> 5) * kTile + t] >> (c & 31)) & 1u;
            double loc = a.h64[(size_t)r * Lx + c];
            if (c > 0)
              loc += a.Jh64[(size_t)r * (Lx - 1) + c - 1] *
                     (((bits_cur[((c - 1) >> 5) * kTile + t] >> ((c - 1) & 31)) & 1u) ? 1.0 : -1.0);
            if (r > 0)
              loc += a.Jv64[(size_t)(r - 1) * Lx + c] * (((bits_prev[(c >> 5) * kTile + t] >> (c & 31)) & 1u) ? 1.0 : -1.0);
            E -= (sc ? 1.0 : -1.0) * loc;
          }
        }
        if (active && a.spins_out && !a.spins_in) {
          int8_t* dst = a.spins_out + (size_t)b * n + (size_t)r * Lx;
          if ((Lx & 15) == 0 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
            for (int c0 = 0; c0 < Lx; c0 += 16) {
              const uint32_t wb = bits_cur[(c0 >> 5) * kTile + t] >> (c0 & 31);
              uint32_t wv[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                uint32_t word = 0;
#pragma unroll
                for (int z = 0; z < 4; ++z) word |= (uint32_t)(((wb >> (4 * q + z)) & 1u) ? 0x01u : 0xFFu) << (8 * z);
                wv[q] = word;
              }
              *reinterpret_cast<uint4*>(dst + c0) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
          } else {
            for (int c = 0; c < Lx; ++c) dst[c] = ((bits_cur[(c >> 5) * kTile + t] >> (c & 31)) & 1u) ? 1 : -1;
          }
        }
        for (int wd = 0; wd < W; ++wd) bits_prev[wd * kTile + t] = bits_cur[wd * kTile + t];
      }
      __syncthreads();   // bits_prev is read by both halves in the next row
    }
    if (h == 0 && active && !abort) {
      a.logq[b] = lq;   // flagged samples too: the log of the probability they were drawn with
      a.energy[b] = E;
      if (a.flags) a.flags[b] = flag;
      if (flag) set_status(a.e.status, TNMC_E_NUMERIC);
    }
  }
  // teardown (after the last step, or after a wait gave up): let the copies still in
  // flight land and the last committed UMMA finish (bounded waits with the full limit),
  // then free TMEM.  Thread 0 observes the tile and R barriers in order and refills a
  // buffer only after a successful wait, so at most one phase of each is outstanding.
  if (tid == 0) {
    // steps thread 0 committed (g counts finished steps; an aborted step committed too),
    // and tiles it saw land
    const int64_t committed = g + (abort ? 1 : 0);
    const int64_t tiles_seen = g + ((abort && misc[2]) ? 1 : 0);
    for (int64_t q = tiles_seen; q < cnt[0]; ++q)
      (void)umma::mbar_wait_parked(umma::smem_u32(&bars[0]), (uint32_t)(q & 1), kPollLimit, kPollHintNs);
    for (int64_t q = cnt[2]; q < cnt[1]; ++q)
      (void)umma::mbar_wait_parked(umma::smem_u32(&bars[2]), (uint32_t)(q & 1), kPollLimit, kPollHintNs);
    if (committed > 0)
      (void)umma::mbar_wait_parked(umma::smem_u32(&bars[1]), (uint32_t)((committed - 1) & 1), kPollLimit,
                                   kPollHintNs);
    bulk_wait_all();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(tmem, kN);
}

// Pre-swizzled BF16 operand tiles of every (r, c).  Left sweep: M itself (n = s*64 + b,
// k = a).  Right sweep: the field-combined tensor of each value u of the spin above,
//   Mt^(u)[a][b] = sum_s f_u(s) M[a][s][b],  f_u(s) = exp(beta Jv[r-1][c] u s)  (1 on row 0),
// formed in FP64 (n = u*64 + a, k = b), so that R_c = Mt^(u) R_{c+1} is one half of the
// UMMA output.  Both are zero outside the bond dimensions and stored as BF16 hi + lo.
__global__ void derive_tc_kernel(DeviceEnv e, __nv_bfloat16* TR, __nv_bfloat16* TL, size_t ntens) {
  const int P = e.P;
  const size_t per = (size_t)kN * kK;
  const size_t total = ntens * per;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t tt = i / per;
    const int rem = (int)(i % per);
    const int nn = rem / kK, k = rem % kK;
    const int s = nn >> 6, x = nn & 63;
    const double* M = e.M64 + tt * (size_t)P * 2 * P;
    const double fmin = e.fe[2 * tt], fplus = e.fe[2 * tt + 1];   // exp(-beta Jv), exp(+beta Jv); 1 on row 0
    // right tile: u = s (0: spin above -1), a = x, b = k ; left tile: s, b = x, a = k
    double vr = 0.0;
    if (x < P && k < P) {
      const double m0 = M[((size_t)x * 2 + 0) * P + k], m1 = M[((size_t)x * 2 + 1) * P + k];
      vr = s ? (fmin * m0 + fplus * m1) : (fplus * m0 + fmin * m1);
    }
    const double vl = (x < P && k < P) ? M[((size_t)k * 2 + s) * P + x] : 0.0;
    // hi = bf16(v), lo = bf16(v - hi): the pair carries about 16 significant bits
    const size_t off = tt * 2 * per + umma::sw128_offset(nn, k) / 2;
    const __nv_bfloat16 rh = __double2bfloat16(vr), lh = __double2bfloat16(vl);
    TR[off] = rh;
    TR[off + per] = __double2bfloat16(vr - (double)__bfloat162float(rh));
    TL[off] = lh;
    TL[off + per] = __double2bfloat16(vl - (double)__bfloat162float(lh));
  }
}

__global__ void couplings32_kernel(DeviceEnv e, float* h32, float* Jh32, float* Jv32) {
  const int Lx = e.Lx, Ly = e.Ly;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Lx * Ly; i += gridDim.x * blockDim.x) {
    const int r = i / Lx, c = i % Lx;
    h32[i] = (float)e.h[i];
    if (c < Lx - 1) Jh32[r * (Lx - 1) + c] = (float)e.Jh[r * (Lx - 1) + c];
    if (r < Ly - 1) Jv32[i] = (float)e.Jv[i];
  }
}

}  // namespace
}  // namespace tnmc

size_t tnmc_tc_tile_bytes() { return tnmc::kStageBytes; }

tnmc_status tnmc_launch_derive_tc(tnmc_env* env, cudaStream_t stream) {
  using namespace tnmc;
  DeviceEnv& d = env->d;
  const size_t ntens = (size_t)d.Lx * d.Ly;
  couplings32_kernel<<<256, 256, 0, stream>>>(d, env->h32, env->Jh32, env->Jv32);
  TNMC_CUDA_TRY(cudaGetLastError());
  derive_tc_kernel<<<2048, 256, 0, stream>>>(d, const_cast<__nv_bfloat16*>(d.R16), const_cast<__nv_bfloat16*>(d.L16),
                                             ntens);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_launch_sample_tc(const tnmc_env* env, int64_t B, uint64_t seed, uint64_t offset,
                                  const int8_t* spins_in, int8_t* spins_out, double* logq, double* energy,
                                  int32_t* flags, cudaStream_t stream) {
  using namespace tnmc;
  const DeviceEnv& d = env->d;
  if (d.P > kK) {
    tnmc_set_error("the tensor-core sampler supports chi <= 64");
    return TNMC_E_UNSUPPORTED;
  }
  const int W = (d.Lx + 31) / 32;
  const size_t smem = 1024 + 2 * kVecBytes + kStageBytes + kRBytes + 3 * 8 + 40 +
                      (size_t)10 * kTile * sizeof(float) + (size_t)2 * W * kTile * sizeof(uint32_t);
  int dev = 0, nsm = 0, max_optin = 0;
  TNMC_CUDA_TRY(cudaGetDevice(&dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)max_optin) {
    tnmc_set_error("tensor-core sampler needs %zu bytes of shared memory (device allows %d)", smem, max_optin);
    return TNMC_E_UNSUPPORTED;
  }
  TNMC_CUDA_TRY(cudaFuncSetAttribute(sample_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TNMC_CUDA_TRY(cudaFuncSetAttribute(sample_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  TNMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_tc_kernel, kThreads, smem));
  {
    // cross-check the occupancy query against the shared-memory budget of an SM
    int smem_sm = 0, regs_sm = 0;
    TNMC_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    TNMC_CUDA_TRY(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    cudaFuncAttributes fa;
    TNMC_CUDA_TRY(cudaFuncGetAttributes(&fa, sample_tc_kernel));
    const int by_smem = smem_sm / (int)(smem + 1024);
    const int by_regs = regs_sm / (((fa.numRegs + 7) & ~7) * kThreads);
    const int est = by_smem < by_regs ? by_smem : by_regs;
    if (est > per_sm) per_sm = est;
  }
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;   // TMEM: 4 x 128 columns per SM
  const int64_t ntiles = (B + kTile - 1) / kTile;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  const size_t need = (size_t)grid * d.Lx * kTile * kK * sizeof(float);
  tnmc_env* me = const_cast<tnmc_env*>(env);
  {
    const tnmc_status gs = grow_scratch(me, need, stream, "sampler");
    if (gs != TNMC_OK) return gs;
  }
  TcArgs a;
  a.e = d;
  a.TR = d.R16;
  a.TL = d.L16;
  a.fe = d.fe32;
  a.h32 = env->h32;
  a.Jh32 = env->Jh32;
  a.Jv32 = env->Jv32;
  a.B = B;
  a.seed = seed;
  a.offset = offset;
  a.spins_in = spins_in;
  a.spins_out = spins_out;
  a.logq = logq;
  a.energy = energy;
  a.flags = flags;
  a.stack = static_cast<float4*>(me->scratch.ptr);
  a.h64 = d.h;
  a.Jh64 = d.Jh;
  a.Jv64 = d.Jv;
  a.poll_limit = kPollLimit;
  {
    // test hook: TNMC_DEBUG_POLL_LIMIT=<n> caps the polls of the in-loop waits (0: they
    // give up at once), so that the timeout path can be exercised without a stuck copy
    const char* pl = getenv("TNMC_DEBUG_POLL_LIMIT");
    if (pl && *pl) a.poll_limit = (uint32_t)strtoul(pl, nullptr, 10);
  }
  sample_tc_kernel<<<(unsigned)grid, kThreads, smem, stream>>>(a);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}
