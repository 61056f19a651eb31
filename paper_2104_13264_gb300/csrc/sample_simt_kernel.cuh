// SIMT sampler / evaluator kernel template (FP64 or FP32), shared by the
// translation units that launch it.  See sample_simt.cu for the algorithm.
#pragma once

#include <math.h>

#include "common.cuh"

namespace tnmc {
namespace {

template <typename T>
struct SampleArgs {
  DeviceEnv e;
  const T* L;     // [Ly][Lx][P][2][P]
  const T* Rt;    // [Ly][Lx][P][P][2]
  const T* fe;    // [Ly][Lx][2]
  int64_t B;
  uint64_t seed, offset;
  const int8_t* spins_in;   // forced mode when non-null
  int8_t* spins_out;        // may be null in forced mode
  double* logq;
  double* energy;
  int32_t* flags;
  T* scratch;               // per CTA: [Lx+1][P][NT]
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ inline void load(const float* p, float* o) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
};
template <>
struct Vec4<double> {
  static __device__ inline void load(const double* p, double* o) {
    const double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
    const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
  }
};

__device__ inline int ilogb_pos(double x) { return ilogb(x); }
__device__ inline int ilogb_pos(float x) { return ilogbf(x); }
__device__ inline double scale2(double x, int e) { return scalbn(x, e); }
__device__ inline float scale2(float x, int e) { return scalbnf(x, e); }

// log-probability accumulator: FP64 sums logs; FP32 keeps a product with a
// separate binary exponent and takes one FP64 log per row.
template <typename T>
struct LogAcc;
template <>
struct LogAcc<double> {
  double lq = 0.0;
  __device__ void mul(double p) { lq += log(p); }
  __device__ void flush() {}
  __device__ double value() const { return lq; }
};
template <>
struct LogAcc<float> {
  double lq = 0.0;
  float prod = 1.0f;
  int ex = 0;
  __device__ void mul(float p) {
    prod *= p;
    if (prod < 0x1.0p-60f && prod > 0.0f) {
      prod *= 0x1.0p60f;
      ex -= 60;
    }
  }
  __device__ void flush() {
    lq += log((double)prod) + (double)ex * 0.69314718055994530942;
    prod = 1.0f;
    ex = 0;
  }
  __device__ double value() const { return lq; }
};

// One tile of NT samples of one instance.  Shared memory: VA, VB, VC [P][NT] and the
// two bit rows [W][NT] carved from `smem` for this instance's P and W; `stack` is the
// calling CTA's right-vector stack [Lx+1][P][NT].
template <typename T, int NT>
__device__ void sample_simt_tile(const SampleArgs<T>& a, int64_t tile, unsigned char* smem, T* stack) {
  const int Lx = a.e.Lx, Ly = a.e.Ly, P = a.e.P;
  const int W = (Lx + 31) >> 5;
  T* VA = reinterpret_cast<T*>(smem);               // [P][NT]   Lambda / R ping
  T* VB = VA + (size_t)P * NT;                       // [P][NT]   R pong / U[-1]
  T* VC = VB + (size_t)P * NT;                       // [P][NT]   U[+1]
  uint32_t* bits_prev = reinterpret_cast<uint32_t*>(VC + (size_t)P * NT);   // [W][NT]
  uint32_t* bits_cur = bits_prev + (size_t)W * NT;                            // [W][NT]
  const int tid = threadIdx.x;
  const int n = Lx * Ly;
  {
    const int64_t b = tile * NT + tid;
    const bool active = b < a.B;
    const uint64_t sample = a.offset + (uint64_t)b;
    LogAcc<T> acc;
    double E = 0.0;
    int flag = 0;
    for (int wd = 0; wd < W; ++wd) bits_prev[wd * NT + tid] = 0u;

    for (int r = 0; r < Ly; ++r) {
      const int32_t* bond = a.e.bond + r * (Lx + 1);
      const T* fer = a.fe + (size_t)r * Lx * 2;
      if (a.spins_in) {
        for (int wd = 0; wd < W; ++wd) bits_cur[wd * NT + tid] = 0u;
        if (active) {
          const int8_t* src = a.spins_in + (size_t)b * n + (size_t)r * Lx;
          for (int c = 0; c < Lx; ++c)
            if (src[c] > 0) bits_cur[(c >> 5) * NT + tid] |= 1u << (c & 31);
        }
      }
      if (a.e.order == 1 && (r & 1)) {
        // ---- snake order, odd row: right to left ----
        // forward sweep: V_{c+1} = sum_s f(s) V_c M_c[:, s, :] (sites < c+1 summed), V_c in stack[c]
        {
          T* V0 = stack;
          for (int k = 0; k < P; ++k) {
            const T v = (k == 0) ? T(1) : T(0);
            V0[k * NT + tid] = v;
            VA[k * NT + tid] = v;
          }
        }
        T* Vin = VA;
        T* Vout = VB;
        for (int c = 0; c + 1 < Lx; ++c) {
          const int dc = (bond[c] + 3) & ~3, dc1 = (bond[c + 1] + 3) & ~3;
          const bool up = (r > 0) && ((bits_prev[(c >> 5) * NT + tid] >> (c & 31)) & 1u);
          const T fsame = fer[2 * c + 1], fdiff = fer[2 * c];
          const T fm = up ? fdiff : fsame;
          const T fp = up ? fsame : fdiff;
          const T* M = a.L + ((size_t)r * Lx + c) * P * 2 * P;
          T mx = T(0);
          for (int b0 = 0; b0 < dc1; b0 += 4) {
            T u0[4] = {T(0), T(0), T(0), T(0)}, u1[4] = {T(0), T(0), T(0), T(0)};
            for (int aa = 0; aa < dc; ++aa) {
              const T la = Vin[aa * NT + tid];
              T m0[4], m1[4];
              Vec4<T>::load(M + ((size_t)aa * 2) * P + b0, m0);
              Vec4<T>::load(M + ((size_t)aa * 2 + 1) * P + b0, m1);
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                u0[i] = fma(la, m0[i], u0[i]);
                u1[i] = fma(la, m1[i], u1[i]);
              }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const T v = fm * u0[i] + fp * u1[i];
              Vout[(b0 + i) * NT + tid] = v;
              mx = fmax(mx, fabs(v));
            }
          }
          const int e = (mx > T(0)) ? -ilogb_pos(mx) : 0;
          T* Vs = stack + (size_t)(c + 1) * P * NT;
          for (int k = 0; k < dc1; ++k) {
            const T v = scale2(Vout[k * NT + tid], e);
            Vout[k * NT + tid] = v;
            Vs[k * NT + tid] = v;
          }
          T* t = Vin;
          Vin = Vout;
          Vout = t;
        }
        // draws from the right: Lambda' holds the drawn sites > c (VA), U'[a][s] in VB / VC
        for (int k = 0; k < P; ++k) VA[k * NT + tid] = (k == 0) ? T(1) : T(0);
        int s_right = 0;
        for (int c = Lx - 1; c >= 0; --c) {
          const int dc = (bond[c] + 3) & ~3, dc1 = (bond[c + 1] + 3) & ~3;
          const bool up = (r > 0) && ((bits_prev[(c >> 5) * NT + tid] >> (c & 31)) & 1u);
          const T fsame = fer[2 * c + 1], fdiff = fer[2 * c];
          const T fm = up ? fdiff : fsame;
          const T fp = up ? fsame : fdiff;
          const T* MT = a.Rt + ((size_t)r * Lx + c) * P * P * 2;
          const T* Vl = stack + (size_t)c * P * NT;
          T w0 = T(0), w1 = T(0);
          for (int a0 = 0; a0 < dc; a0 += 4) {
            T s0[4] = {T(0), T(0), T(0), T(0)}, s1[4] = {T(0), T(0), T(0), T(0)};
            for (int bb = 0; bb < dc1; ++bb) {
              const T rb = VA[bb * NT + tid];
              T m[8];
              Vec4<T>::load(MT + ((size_t)bb * P + a0) * 2, m);
              Vec4<T>::load(MT + ((size_t)bb * P + a0) * 2 + 4, m + 4);
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                s0[i] = fma(m[2 * i], rb, s0[i]);
                s1[i] = fma(m[2 * i + 1], rb, s1[i]);
              }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const T vl = Vl[(a0 + i) * NT + tid];
              w0 = fma(vl, s0[i], w0);
              w1 = fma(vl, s1[i], w1);
              VB[(a0 + i) * NT + tid] = s0[i];
              VC[(a0 + i) * NT + tid] = s1[i];
            }
          }
          w0 *= fm;
          w1 *= fp;
          w0 = fmax(w0, T(0));
          w1 = fmax(w1, T(0));
          const T tot = w0 + w1;
          const bool bad = !(tot > T(0)) || !isfinite(tot);
          const T pplus = bad ? T(0.5) : w1 / tot;
          const T pminus = bad ? T(0.5) : w0 / tot;
          const int64_t site = (int64_t)r * Lx + c;
          bool plus;
          if (a.spins_in) {
            plus = (bits_cur[(c >> 5) * NT + tid] >> (c & 31)) & 1u;
          } else {
            plus = draw_plus(pplus, draw_word(a.seed, site, sample));
            if (plus) bits_cur[(c >> 5) * NT + tid] |= 1u << (c & 31);
            else bits_cur[(c >> 5) * NT + tid] &= ~(1u << (c & 31));
          }
          acc.mul(plus ? pplus : pminus);
          flag |= bad ? TNMC_FLAG_NUMERIC : 0;
          {
            const double sv = plus ? 1.0 : -1.0;
            double loc = a.e.h[r * Lx + c];
            if (c + 1 < Lx) loc += a.e.Jh[r * (Lx - 1) + c] * (s_right ? 1.0 : -1.0);
            loc += a.e.Jv[(r - 1) * Lx + c] * (up ? 1.0 : -1.0);
            E -= sv * loc;
          }
          s_right = plus;
          const T fs = plus ? fp : fm;
          const T* U = plus ? VC : VB;
          T mx = T(0);
          for (int k = 0; k < dc; ++k) mx = fmax(mx, fabs(U[k * NT + tid] * fs));
          const int e = (mx > T(0)) ? -ilogb_pos(mx) : 0;
          for (int k = 0; k < dc; ++k) VA[k * NT + tid] = scale2(U[k * NT + tid] * fs, e);
        }
      } else {
        // ---- right sweep ----
        {
          T* Rl = stack + (size_t)Lx * P * NT;
          for (int k = 0; k < P; ++k) {
            const T v = (k == 0) ? T(1) : T(0);
            Rl[k * NT + tid] = v;
            VA[k * NT + tid] = v;
          }
        }
        T* Rin = VA;
        T* Rout = VB;
        for (int c = Lx - 1; c >= 1; --c) {
          const int dc = (bond[c] + 3) & ~3, dc1 = (bond[c + 1] + 3) & ~3;
          const bool up = (r > 0) && ((bits_prev[(c >> 5) * NT + tid] >> (c & 31)) & 1u);
          // f(s) with s_up * s = +1 -> fer[1], -1 -> fer[0]
          const T fsame = fer[2 * c + 1], fdiff = fer[2 * c];
          const T fm = (r == 0) ? T(1) : (up ? fdiff : fsame);   // s = -1
          const T fp = (r == 0) ? T(1) : (up ? fsame : fdiff);   // s = +1
          const T* MT = a.Rt + ((size_t)r * Lx + c) * P * P * 2;
          T mx = T(0);
          for (int a0 = 0; a0 < dc; a0 += 4) {
            T s0[4] = {T(0), T(0), T(0), T(0)}, s1[4] = {T(0), T(0), T(0), T(0)};
            for (int bb = 0; bb < dc1; ++bb) {
              const T rb = Rin[bb * NT + tid];
              T m[8];
              Vec4<T>::load(MT + ((size_t)bb * P + a0) * 2, m);
              Vec4<T>::load(MT + ((size_t)bb * P + a0) * 2 + 4, m + 4);
  #pragma unroll
              for (int i = 0; i < 4; ++i) {
                s0[i] = fma(m[2 * i], rb, s0[i]);
                s1[i] = fma(m[2 * i + 1], rb, s1[i]);
              }
            }
  #pragma unroll
            for (int i = 0; i < 4; ++i) {
              const T v = fm * s0[i] + fp * s1[i];
              Rout[(a0 + i) * NT + tid] = v;
              mx = fmax(mx, fabs(v));
            }
          }
          const int e = (mx > T(0)) ? -ilogb_pos(mx) : 0;
          T* Rs = stack + (size_t)c * P * NT;
          for (int k = 0; k < dc; ++k) {
            const T v = scale2(Rout[k * NT + tid], e);
            Rout[k * NT + tid] = v;
            Rs[k * NT + tid] = v;
          }
          T* t = Rin;
          Rin = Rout;
          Rout = t;
        }
        // ---- left sweep ----
        for (int k = 0; k < P; ++k) VA[k * NT + tid] = (k == 0) ? T(1) : T(0);
        int s_left = 0;
        for (int c = 0; c < Lx; ++c) {
          const int dc = (bond[c] + 3) & ~3, dc1 = (bond[c + 1] + 3) & ~3;
          const bool up = (r > 0) && ((bits_prev[(c >> 5) * NT + tid] >> (c & 31)) & 1u);
          const T fsame = fer[2 * c + 1], fdiff = fer[2 * c];
          const T fm = (r == 0) ? T(1) : (up ? fdiff : fsame);
          const T fp = (r == 0) ? T(1) : (up ? fsame : fdiff);
          const T* M = a.L + ((size_t)r * Lx + c) * P * 2 * P;
          const T* Rn = stack + (size_t)(c + 1) * P * NT;
          T w0 = T(0), w1 = T(0);
          for (int b0 = 0; b0 < dc1; b0 += 4) {
            T u0[4] = {T(0), T(0), T(0), T(0)}, u1[4] = {T(0), T(0), T(0), T(0)};
            for (int aa = 0; aa < dc; ++aa) {
              const T la = VA[aa * NT + tid];
              T m0[4], m1[4];
              Vec4<T>::load(M + ((size_t)aa * 2) * P + b0, m0);
              Vec4<T>::load(M + ((size_t)aa * 2 + 1) * P + b0, m1);
  #pragma unroll
              for (int i = 0; i < 4; ++i) {
                u0[i] = fma(la, m0[i], u0[i]);
                u1[i] = fma(la, m1[i], u1[i]);
              }
            }
  #pragma unroll
            for (int i = 0; i < 4; ++i) {
              const T rb = Rn[(b0 + i) * NT + tid];
              w0 = fma(u0[i], rb, w0);
              w1 = fma(u1[i], rb, w1);
              VB[(b0 + i) * NT + tid] = u0[i];
              VC[(b0 + i) * NT + tid] = u1[i];
            }
          }
          w0 *= fm;
          w1 *= fp;
          w0 = fmax(w0, T(0));
          w1 = fmax(w1, T(0));
          const T tot = w0 + w1;
          const bool bad = !(tot > T(0)) || !isfinite(tot);
          const T pplus = bad ? T(0.5) : w1 / tot;
          const T pminus = bad ? T(0.5) : w0 / tot;
          const int64_t site = (int64_t)r * Lx + c;
          bool plus;
          if (a.spins_in) {
            plus = (bits_cur[(c >> 5) * NT + tid] >> (c & 31)) & 1u;
          } else {
            plus = draw_plus(pplus, draw_word(a.seed, site, sample));
            if (plus) bits_cur[(c >> 5) * NT + tid] |= 1u << (c & 31);
            else bits_cur[(c >> 5) * NT + tid] &= ~(1u << (c & 31));
          }
          acc.mul(plus ? pplus : pminus);
          flag |= bad ? TNMC_FLAG_NUMERIC : 0;
          // energy (eq. ising), FP64
          {
            const double sv = plus ? 1.0 : -1.0;
            double loc = a.e.h[r * Lx + c];
            if (c > 0) loc += a.e.Jh[r * (Lx - 1) + c - 1] * (s_left ? 1.0 : -1.0);
            if (r > 0) loc += a.e.Jv[(r - 1) * Lx + c] * (up ? 1.0 : -1.0);
            E -= sv * loc;
          }
          s_left = plus;
          // Lambda_{c+1} = f(s) U[s], rescaled
          const T fs = plus ? fp : fm;
          const T* U = plus ? VC : VB;
          T mx = T(0);
          for (int k = 0; k < dc1; ++k) mx = fmax(mx, fabs(U[k * NT + tid] * fs));
          const int e = (mx > T(0)) ? -ilogb_pos(mx) : 0;
          for (int k = 0; k < dc1; ++k) VA[k * NT + tid] = scale2(U[k * NT + tid] * fs, e);
        }
      }
      acc.flush();
      // ---- row output: spins, then this row becomes the previous row ----
      if (active && a.spins_out && !a.spins_in) {
        int8_t* dst = a.spins_out + (size_t)b * n + (size_t)r * Lx;
        if ((Lx & 3) == 0 && ((reinterpret_cast<uintptr_t>(dst) & 3) == 0)) {
          for (int c = 0; c < Lx; c += 4) {
            const uint32_t wbits = bits_cur[(c >> 5) * NT + tid] >> (c & 31);
            uint32_t word = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) word |= (uint32_t)(((wbits >> i) & 1u) ? 0x01u : 0xFFu) << (8 * i);
            *reinterpret_cast<uint32_t*>(dst + c) = word;
          }
        } else {
          for (int c = 0; c < Lx; ++c)
            dst[c] = ((bits_cur[(c >> 5) * NT + tid] >> (c & 31)) & 1u) ? 1 : -1;
        }
      }
      for (int wd = 0; wd < W; ++wd) bits_prev[wd * NT + tid] = bits_cur[wd * NT + tid];
    }
    if (active) {
      // a flagged sample keeps the log of the probability it was drawn with (log 1/2 at a
      // site whose normaliser failed): q stays the exact law of the sampler
      a.logq[b] = acc.value();
      a.energy[b] = E;
      if (a.flags) a.flags[b] = flag;
      if (flag) set_status(a.e.status, TNMC_E_NUMERIC);
    }
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) sample_simt_kernel(SampleArgs<T> a) {
  extern __shared__ unsigned char smem_raw[];
  const int64_t ntiles = (a.B + NT - 1) / NT;
  T* stack = a.scratch + (size_t)blockIdx.x * (a.e.Lx + 1) * a.e.P * NT;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) sample_simt_tile<T, NT>(a, tile, smem_raw, stack);
}

}  // namespace
}  // namespace tnmc
