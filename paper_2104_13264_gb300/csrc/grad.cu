// Backward of sum_b w_b log q(s_b) with respect to every environment tensor
// M^(r)_c (the FP32 sampler copy), by reverse-mode differentiation of the forced
// evaluation (Sec. 2, eq. pi-approx; App. A): per-site normalised, clamped
// conditionals, power-of-two rescalings treated as constants.
//
// One thread owns one sample, a CTA owns 128 samples.  Per row r:
//   1. forward right sweep  R_c = k'_c sum_s f_c(s) M_c[s] R_{c+1}      (stack)
//   2. forward left sweep   Lambda_{c+1} = k_c f_c(s_c) Lambda_c M_c[s_c]   (stack),
//      raw weights w_c(s) = f_c(s) <Lambda_c M_c[s], R_{c+1}>
//   3. g_c(s) = d/dw_c(s) [w log w_c(s_c) - w log(w_+ + w_-)], zero where clamped
//   4. right-to-left adjoint of Lambda:
//        Lbar_c = sum_s g_c(s) M_c[s] R_{c+1} + k_c f_c(s_c) M_c[s_c] Lbar_{c+1}
//   5. left-to-right adjoint of R and the gradient of site c:
//        Rbar_{c+1} = sum_s g_c(s) (Lambda_c M_c[s]) + k'_c sum_s f_c(s) M_c[s]^T Rbar_c
//        G_c[a,s,b] += sum_t Lambda_c[a] Y_s[b] + Rbar_c[a] Z_s[b]
//          Y_s = g_c(s) R_{c+1} + [s = s_c] k_c f_c(s) Lbar_{c+1},  Z_s = k'_c f_c(s) R_{c+1}
//      The sum over the CTA's samples is a small (P x 2*128) . (2*128 x P) contraction
//      per site done in shared memory; each CTA adds its partial with one atomic per
//      element.
#include <math.h>

#include "common.cuh"

namespace tnmc {
namespace {

// NT samples per CTA (one per thread); vectors live in shared memory with stride NT + 1
// (conflict free).  128 up to P = 52 for large batches; 64 above P = 52 (so that P = 64 fits
// the shared memory) and for batches too small to give every SM two 128-sample tiles.

struct GradArgs {
  DeviceEnv e;
  const float* L;       // [Ly][Lx][P][2][P]
  const float* Rt;      // [Ly][Lx][P][P][2]
  const float* fe;      // [Ly][Lx][2]
  int64_t B;
  const int8_t* spins;
  const float* weights;
  float* grad;          // [Ly][Lx][P][2][P], accumulated
  float* scratch;       // per CTA: 3 stacks [Lx+1][P][NT] + 4 x [Lx][NT]
};

__device__ inline float scale2f(float x, int e) { return scalbnf(x, e); }

template <int kNT>
__global__ void __launch_bounds__(kNT) logq_grad_kernel(GradArgs a) {
  constexpr int kSP = kNT + 1;
  extern __shared__ float sm[];
  const int Lx = a.e.Lx, Ly = a.e.Ly, P = a.e.P;
  const int W = (Lx + 31) >> 5;
  const int t = threadIdx.x;
  float* V0 = sm;                        // [P][SP]  Lambda_c (P1)
  float* V2 = V0 + P * kSP;              // [P][SP]  Rbar_c (P2)
  float* V3 = V2 + P * kSP;              // [P][SP]  scratch vector
  float* Y = V3 + P * kSP;               // [2][P][SP]
  float* Z = Y + 2 * P * kSP;            // [2][P][SP]
  uint32_t* bits_prev = reinterpret_cast<uint32_t*>(Z + 2 * P * kSP);   // [W][NT]
  uint32_t* bits_cur = bits_prev + W * kNT;
  const int64_t tile = blockIdx.x;
  const int64_t b = tile * kNT + t;
  const bool active = b < a.B;
  const int n = Lx * Ly;
  const size_t stack = (size_t)(Lx + 1) * P * kNT;
  float* Rs = a.scratch + (size_t)blockIdx.x * (3 * stack + 4 * (size_t)Lx * kNT);
  float* Ls = Rs + stack;
  float* LBs = Ls + stack;
  float* w0s = LBs + stack;              // [Lx][NT] raw w(-)
  float* w1s = w0s + (size_t)Lx * kNT;   // [Lx][NT] raw w(+)
  int* ek = reinterpret_cast<int*>(w1s + (size_t)Lx * kNT);    // exponent of k_c (Lambda_{c+1})
  int* ekp = ek + (size_t)Lx * kNT;                           // exponent of k'_c (R_c)
  const float wt = active ? a.weights[b] : 0.0f;

  for (int wd = 0; wd < W; ++wd) bits_prev[wd * kNT + t] = 0u;
  for (int r = 0; r < Ly; ++r) {
    const int32_t* bond = a.e.bond + r * (Lx + 1);
    const float* fer = a.fe + (size_t)r * Lx * 2;
    for (int wd = 0; wd < W; ++wd) bits_cur[wd * kNT + t] = 0u;
    if (active) {
      const int8_t* src = a.spins + (size_t)b * n + (size_t)r * Lx;
      for (int c = 0; c < Lx; ++c)
        if (src[c] > 0) bits_cur[(c >> 5) * kNT + t] |= 1u << (c & 31);
    }
    auto fval = [&](int c, int s) -> float {
      if (r == 0) return 1.0f;
      const bool up = (bits_prev[(c >> 5) * kNT + t] >> (c & 31)) & 1u;
      return ((up ? 1 : 0) == s) ? fer[2 * c + 1] : fer[2 * c];
    };
    auto spin = [&](int c) -> int { return (bits_cur[(c >> 5) * kNT + t] >> (c & 31)) & 1u; };
    // ---- 1. right sweep ----
    for (int k = 0; k < P; ++k) Rs[((size_t)Lx * P + k) * kNT + t] = (k == 0) ? 1.0f : 0.0f;
    for (int c = Lx - 1; c >= 1; --c) {
      const int dc = bond[c], dc1 = bond[c + 1];
      const float f0 = fval(c, 0), f1 = fval(c, 1);
      const float* M = a.L + ((size_t)r * Lx + c) * P * 2 * P;
      const float* Rn = Rs + (size_t)(c + 1) * P * kNT;
      float mx = 0.0f;
      for (int aa = 0; aa < dc; ++aa) {
        float s0 = 0.0f, s1 = 0.0f;
        for (int bb = 0; bb < dc1; ++bb) {
          const float rb = Rn[bb * kNT + t];
          s0 = fmaf(__ldg(M + ((size_t)aa * 2) * P + bb), rb, s0);
          s1 = fmaf(__ldg(M + ((size_t)aa * 2 + 1) * P + bb), rb, s1);
        }
        const float v = f0 * s0 + f1 * s1;
        V3[aa * kSP + t] = v;
        mx = fmaxf(mx, fabsf(v));
      }
      const int e = (mx > 0.0f) ? -ilogbf(mx) : 0;
      ekp[(size_t)c * kNT + t] = e;
      float* Rc = Rs + (size_t)c * P * kNT;
      for (int aa = 0; aa < P; ++aa) Rc[aa * kNT + t] = (aa < dc) ? scale2f(V3[aa * kSP + t], e) : 0.0f;
    }
    // ---- 2. left sweep (forced) ----
    for (int k = 0; k < P; ++k) Ls[(size_t)k * kNT + t] = (k == 0) ? 1.0f : 0.0f;
    for (int c = 0; c < Lx; ++c) {
      const int dc = bond[c], dc1 = bond[c + 1];
      const float f0 = fval(c, 0), f1 = fval(c, 1);
      const int s = spin(c);
      const float* M = a.L + ((size_t)r * Lx + c) * P * 2 * P;
      const float* Lc = Ls + (size_t)c * P * kNT;
      const float* Rn = Rs + (size_t)(c + 1) * P * kNT;
      float w0 = 0.0f, w1 = 0.0f, mx = 0.0f;
      for (int bb = 0; bb < dc1; ++bb) {
        float u0 = 0.0f, u1 = 0.0f;
        for (int aa = 0; aa < dc; ++aa) {
          const float la = Lc[aa * kNT + t];
          u0 = fmaf(la, __ldg(M + ((size_t)aa * 2) * P + bb), u0);
          u1 = fmaf(la, __ldg(M + ((size_t)aa * 2 + 1) * P + bb), u1);
        }
        const float rb = Rn[bb * kNT + t];
        w0 = fmaf(u0, rb, w0);
        w1 = fmaf(u1, rb, w1);
        const float us = (s ? u1 : u0) * (s ? f1 : f0);
        V3[bb * kSP + t] = us;
        mx = fmaxf(mx, fabsf(us));
      }
      w0s[(size_t)c * kNT + t] = w0 * f0;
      w1s[(size_t)c * kNT + t] = w1 * f1;
      const int e = (mx > 0.0f) ? -ilogbf(mx) : 0;
      ek[(size_t)c * kNT + t] = e;
      float* Ln = Ls + (size_t)(c + 1) * P * kNT;
      for (int bb = 0; bb < P; ++bb) Ln[bb * kNT + t] = (bb < dc1) ? scale2f(V3[bb * kSP + t], e) : 0.0f;
    }
    // per-site weight adjoints g_c(s); a sample with a non-positive normaliser, or with
    // q = 0, contributes nothing (its log q is not differentiable)
    bool ok = wt != 0.0f;
    for (int c = 0; c < Lx && ok; ++c) {
      const float w0 = fmaxf(w0s[(size_t)c * kNT + t], 0.0f), w1 = fmaxf(w1s[(size_t)c * kNT + t], 0.0f);
      const float ws = spin(c) ? w1 : w0;
      ok = (w0 + w1 > 0.0f) && isfinite(w0 + w1) && ws > 0.0f;
    }
    auto gw = [&](int c, int s_) -> float {
      if (!ok) return 0.0f;
      const float w0r = w0s[(size_t)c * kNT + t], w1r = w1s[(size_t)c * kNT + t];
      const float w0 = fmaxf(w0r, 0.0f), w1 = fmaxf(w1r, 0.0f);
      const int sc = spin(c);
      const float ws = sc ? w1 : w0;
      float g = -1.0f / (w0 + w1);
      if (s_ == sc) g += 1.0f / ws;
      const float raw = s_ ? w1r : w0r;
      return (raw > 0.0f) ? wt * g * fval(c, s_) : 0.0f;
    };
    // ---- 4. Lambda adjoint, right to left: LBs[c] = Lbar_c (c = 1..Lx) ----
    for (int k = 0; k < P; ++k) LBs[((size_t)Lx * P + k) * kNT + t] = 0.0f;
    for (int c = Lx - 1; c >= 1; --c) {
      const int dc = bond[c], dc1 = bond[c + 1];
      const int s = spin(c);
      const float g0 = gw(c, 0), g1 = gw(c, 1);
      const float kf = scale2f(1.0f, ek[(size_t)c * kNT + t]) * fval(c, s);
      const float* M = a.L + ((size_t)r * Lx + c) * P * 2 * P;
      const float* Rn = Rs + (size_t)(c + 1) * P * kNT;
      const float* LBn = LBs + (size_t)(c + 1) * P * kNT;
      float* LBc = LBs + (size_t)c * P * kNT;
      for (int aa = 0; aa < P; ++aa) {
        float acc = 0.0f;
        if (aa < dc) {
          for (int bb = 0; bb < dc1; ++bb) {
            const float m0 = __ldg(M + ((size_t)aa * 2) * P + bb), m1 = __ldg(M + ((size_t)aa * 2 + 1) * P + bb);
            const float rb = Rn[bb * kNT + t];
            acc = fmaf(g0 * m0 + g1 * m1, rb, acc);
            acc = fmaf(kf * (s ? m1 : m0), LBn[bb * kNT + t], acc);
          }
        }
        LBc[aa * kNT + t] = acc;
      }
    }
    // ---- 5. R adjoint left to right, and the site gradients ----
    for (int k = 0; k < P; ++k) V2[k * kSP + t] = 0.0f;   // Rbar_0 (unused: R_0 is never formed)
    for (int c = 0; c < Lx; ++c) {
      const int dc = bond[c], dc1 = bond[c + 1];
      const int s = spin(c);
      const float f0 = fval(c, 0), f1 = fval(c, 1);
      const float g0 = gw(c, 0), g1 = gw(c, 1);
      const float kf = scale2f(1.0f, ek[(size_t)c * kNT + t]) * (s ? f1 : f0);
      const float kp = (c >= 1) ? scale2f(1.0f, ekp[(size_t)c * kNT + t]) : 0.0f;
      const float* M = a.L + ((size_t)r * Lx + c) * P * 2 * P;
      const float* Lc = Ls + (size_t)c * P * kNT;
      const float* Rn = Rs + (size_t)(c + 1) * P * kNT;
      const float* LBn = LBs + (size_t)(c + 1) * P * kNT;
      // operands of G_c: P1 = Lambda_c, P2 = Rbar_c, Y_s, Z_s
      for (int k = 0; k < P; ++k) {
        V0[k * kSP + t] = Lc[k * kNT + t];
        const float rb = Rn[k * kNT + t];
        const float lb = (c + 1 < Lx) ? LBn[k * kNT + t] : 0.0f;
        Y[(0 * P + k) * kSP + t] = g0 * rb + (s == 0 ? kf * lb : 0.0f);
        Y[(1 * P + k) * kSP + t] = g1 * rb + (s == 1 ? kf * lb : 0.0f);
        Z[(0 * P + k) * kSP + t] = kp * f0 * rb;
        Z[(1 * P + k) * kSP + t] = kp * f1 * rb;
      }
      __syncthreads();
      // G_c partial over the CTA's samples: thread -> (a, s, b) entries
      float* G = a.grad + ((size_t)r * Lx + c) * P * 2 * P;
      for (int idx = t; idx < dc * 2 * dc1; idx += kNT) {
        const int bb = idx % dc1, s_ = (idx / dc1) & 1, aa = idx / (2 * dc1);
        const float* y = Y + (size_t)(s_ * P + bb) * kSP;
        const float* z = Z + (size_t)(s_ * P + bb) * kSP;
        const float* p1 = V0 + (size_t)aa * kSP;
        const float* p2 = V2 + (size_t)aa * kSP;
        float acc = 0.0f;
        for (int q = 0; q < kNT; ++q) acc = fmaf(p1[q], y[q], fmaf(p2[q], z[q], acc));
        if (acc != 0.0f) atomicAdd(G + ((size_t)aa * 2 + s_) * P + bb, acc);
      }
      __syncthreads();
      // Rbar_{c+1} = sum_s g(s) Lambda_c M_c[s] + k'_c sum_s f(s) M_c[s]^T Rbar_c
      if (c + 1 < Lx) {
        for (int bb = 0; bb < dc1; ++bb) {
          float acc = 0.0f;
          for (int aa = 0; aa < dc; ++aa) {
            const float m0 = __ldg(M + ((size_t)aa * 2) * P + bb), m1 = __ldg(M + ((size_t)aa * 2 + 1) * P + bb);
            acc = fmaf(Lc[aa * kNT + t], g0 * m0 + g1 * m1, acc);
            acc = fmaf(V2[aa * kSP + t], kp * (f0 * m0 + f1 * m1), acc);
          }
          V3[bb * kSP + t] = acc;
        }
        __syncthreads();
        for (int k = 0; k < P; ++k) V2[k * kSP + t] = (k < dc1) ? V3[k * kSP + t] : 0.0f;
      }
      __syncthreads();
    }
    for (int wd = 0; wd < W; ++wd) bits_prev[wd * kNT + t] = bits_cur[wd * kNT + t];
  }
}

}  // namespace
}  // namespace tnmc

tnmc_status tnmc_launch_logq_grad(const tnmc_env* env, int64_t B, const int8_t* spins, const float* weights,
                                  float* grad, cudaStream_t stream) {
  using namespace tnmc;
  const DeviceEnv& d = env->d;
  const size_t gsz = (size_t)d.Lx * d.Ly * d.P * 2 * d.P;
  TNMC_CUDA_TRY(cudaMemsetAsync(grad, 0, gsz * sizeof(float), stream));
  if (B == 0) return TNMC_OK;
  const int W = (d.Lx + 31) / 32;
  int dev = 0, max_optin = 0;
  TNMC_CUDA_TRY(cudaGetDevice(&dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  auto smem_of = [&](int nt) {
    return (size_t)7 * d.P * (nt + 1) * sizeof(float) + (size_t)2 * W * nt * sizeof(uint32_t);
  };
  int nsm = 0;
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // 128 samples per CTA; 64 when P > 52 (shared memory) or when 128 would leave SMs idle
  const int kNT = (smem_of(128) <= (size_t)max_optin && (B + 127) / 128 >= 2 * (int64_t)nsm) ? 128 : 64;
  const size_t smem = smem_of(kNT);
  if (smem > (size_t)max_optin) {
    tnmc_set_error("gradient kernel needs %zu bytes of shared memory (device allows %d)", smem, max_optin);
    return TNMC_E_UNSUPPORTED;
  }
  if (kNT == 128)
    TNMC_CUDA_TRY(cudaFuncSetAttribute(logq_grad_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  else
    TNMC_CUDA_TRY(cudaFuncSetAttribute(logq_grad_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t ntiles = (B + kNT - 1) / kNT;
  const size_t per_cta = (size_t)3 * (d.Lx + 1) * d.P * kNT + (size_t)4 * d.Lx * kNT;
  const size_t need = (size_t)ntiles * per_cta * sizeof(float);
  tnmc_env* me = const_cast<tnmc_env*>(env);
  {
    const tnmc_status gs = grow_scratch(me, need, stream, "gradient");
    if (gs != TNMC_OK) return gs;
  }
  GradArgs a;
  a.e = d;
  a.L = d.L32;
  a.Rt = d.R32;
  a.fe = d.fe32;
  a.B = B;
  a.spins = spins;
  a.weights = weights;
  a.grad = grad;
  a.scratch = static_cast<float*>(me->scratch.ptr);
  if (kNT == 128) logq_grad_kernel<128><<<(unsigned)ntiles, 128, smem, stream>>>(a);
  else logq_grad_kernel<64><<<(unsigned)ntiles, 64, smem, stream>>>(a);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}
