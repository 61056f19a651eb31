// TNMH on three-dimensional Ising lattices (Sec. 3D; App. A, the three-dimensional
// paragraph and Figs. peps-cutoff2, peps-cutoff).
//
// Layer environments: PEPS of bond D over the spins of one layer, built bottom-up as
//   env_{Lz-1} = the exact weight of the last layer,  env_z = T_D[ D_z H_z V_z env_{z+1} ],
// V_z summing layer z+1 through the vertical bond weights (no bond growth), D_z the
// fields, H_z the in-layer bonds as copy structure (each in-layer bond doubles: the spin
// of the site on the left / above travels along the bond and is weighted at the other
// end).  T_D reads every column as an MPS (bonds: the column's vertical bonds; physical
// index: the spin with the two horizontal bonds) and compresses it by successive SVD,
// then every row likewise along its horizontal bonds.
//
// Sampling (one thread per sample; every tensor is small and all samples share their
// shapes, so a warp runs in lockstep): layer z is sampled with the spins of layer z-1
// as fields f(s) = exp(beta Jz s_up s).  Row y of the layer is sampled from the
// sandwich  Top_y (rows < y, drawn spins; MPS of bond chi) x row y x Bot_y (rows > y,
// spins summed; MPS of bond chi):
//   Bot_{Ly-1} = 1, Bot_y = T_chi[S_{y+1} Bot_{y+1}], S = sum_s A f;
//   Top_0 = 1,      Top_{y+1} = T_chi[Top_y F_y],    F = A f at the drawn spins.
// The site conditionals come from the right vectors R_x (sites > x summed) and the
// left vector Lambda (sites < x drawn), clamped at zero and normalised, drawn with the
// Philox word of site (z Ly + y) Lx + x.  The per-sample scratch lives in HBM with the
// sample index fastest (element i of sample b at base[i * Bc + b]), so every load and
// store of a warp is coalesced.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "common.cuh"

struct tnmc3d_env {
  int Lx, Ly, Lz, D, chi;
  double beta;
  double* Jx;   // [Lz][Ly][Lx-1]
  double* Jy;   // [Lz][Ly-1][Lx]
  double* Jz;   // [Lz-1][Ly][Lx]
  double* h;    // [Lz][Ly][Lx]
  double* A64;  // [Lz][Ly][Lx][2][D][D][D][D]
  float* A32;
  int32_t* dims;   // [Lz][Ly][Lx][4]: du, dl, dd, dr
  int gauge = 0;   // 1: bond basis (layers sampled from their uncompressed PEPS)
  int Ds = 0;      // pad of the sampling tensors: D (spin basis) or 2 D (bond basis)
  double* S64;     // sampling tensors [Lz][Ly][Lx][2][Ds]^4 (the A64 arena in the spin basis)
  float* S32;
  int32_t* sdims;
  double* log_scale;
  int32_t* status;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  tnmc::Allocator alloc;
};

namespace tnmc {
namespace {

constexpr int kMaxSide3 = 64;
constexpr int kMaxRows3 = 64;
constexpr int kSweeps3 = 60;

template <typename T>
struct V {
  T* p;
  int64_t s;
  __device__ __forceinline__ T& operator[](int64_t i) const { return p[i * s]; }
  __device__ __forceinline__ V at(int64_t off) const { return V{p + off * s, s}; }
};

template <typename T>
struct Tol3;
template <>
struct Tol3<double> {
  static constexpr double rot = 1e-13, null = 1e-13, big = 1e150, qr = 1e-12;
};
template <>
struct Tol3<float> {
  static constexpr float rot = 2e-6f, null = 1e-6f, big = 1e15f, qr = 1e-5f;
};

// One-sided (Hestenes) Jacobi on the m rows (length n, row-major) of J, cyclic order.
// On return J's rows are orthogonal and d[i] holds their 2-norms.  Rows below `null`
// of the largest are left out of the rotations.  Returns false when the last sweep
// still rotated.
template <typename T>
__device__ bool orth_rows(V<T> J, int m, int n, V<T> d) {
  bool converged = false;
  for (int sweep = 0; sweep < kSweeps3 && !converged; ++sweep) {
    T dmax = 0;
    for (int i = 0; i < m; ++i) {
      T s = 0;
      for (int x = 0; x < n; ++x) s += J[(int64_t)i * n + x] * J[(int64_t)i * n + x];
      d[i] = s;
      dmax = s > dmax ? s : dmax;
    }
    const T dnull = Tol3<T>::null * Tol3<T>::null * dmax;
    bool rotated = false;
    for (int p = 0; p + 1 < m; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const T al = d[p], be = d[q];
        if (al <= dnull || be <= dnull) continue;
        T ga = 0;
        for (int x = 0; x < n; ++x) ga += J[(int64_t)p * n + x] * J[(int64_t)q * n + x];
        if (!(ga * ga > Tol3<T>::rot * Tol3<T>::rot * al * be)) continue;
        const T zeta = (be - al) / (T(2) * ga);
        const T az = zeta < 0 ? -zeta : zeta;
        const T t = az > Tol3<T>::big ? T(0.5) / zeta : (zeta >= 0 ? T(1) : T(-1)) / (az + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
        for (int x = 0; x < n; ++x) {
          const T u = J[(int64_t)p * n + x], v = J[(int64_t)q * n + x];
          J[(int64_t)p * n + x] = c * u - sn * v;
          J[(int64_t)q * n + x] = sn * u + c * v;
        }
        d[p] = al - t * ga;
        d[q] = be + t * ga;
        rotated = true;
      }
    }
    converged = !rotated;
  }
  for (int i = 0; i < m; ++i) {
    T s = 0;
    for (int x = 0; x < n; ++x) s += J[(int64_t)i * n + x] * J[(int64_t)i * n + x];
    d[i] = sqrt(s);
  }
  return converged;
}

// sel[0..k) = the k rows of largest norm (descending; ties by index).
template <typename T>
__device__ void select_rows(V<T> d, int m, int k, int* sel) {
  for (int i = 0; i < m; ++i) {
    int rank = 0;
    const T di = d[i];
    for (int j = 0; j < m; ++j) {
      const T dj = d[j];
      rank += (dj > di) || (dj == di && j < i);
    }
    if (rank < k) sel[rank] = i;
  }
}

// Successive SVD of an MPS of ns sites (site i at M.at(i * cap), layout [dl][p][dr]):
// QR sweep left to right (classical Gram-Schmidt applied twice, bond min(dl p, dr)), then
// SVD sweep right to left keeping min(kmax, dl, p dr) values;
// site 0 is left with unit norm.  Scratch: J >= rows x len of every step, d >= rows,
// sm >= Kraw^2, tmp >= cap.  Returns 0 or TNMC_E_NUMERIC; *logs gets the removed scale.
template <typename T>
__device__ int mps_compress(V<T> M, int64_t cap, int ns, int* dl, const int* pp, int* dr, int kmax, V<T> J, V<T> d,
                            V<T> sm, V<T> tmp, double* logs) {
  int sel[kMaxRows3];
  int err = 0;
  double lg = 0.0;
  for (int i = 0; i + 1 < ns; ++i) {
    const int a = dl[i], p = pp[i], b = dr[i], len = a * p;
    V<T> Mi = M.at(i * cap);
    const int k = len < b ? len : b;
    // Q R = X (len x b, X[x][c] = Mi[x b + c]) by classical Gram-Schmidt applied twice: the
    // columns of Q (rows of J) are orthonormal; a column numerically inside the span of the
    // earlier ones adds no basis vector, and the basis is padded with zero vectors to k
    // (the bond width min(len, b) of a thin QR), so X = Q R still holds.
    for (int e = 0; e < k * b; ++e) sm[e] = T(0);
    int acc = 0;
    for (int j = 0; j < b; ++j) {
      T nx = 0;
      for (int x = 0; x < len; ++x) {
        const T v = Mi[(int64_t)x * b + j];
        tmp[x] = v;
        nx += v * v;
      }
      for (int pass = 0; pass < 2; ++pass)
        for (int q = 0; q < acc; ++q) {
          T r = 0;
          for (int x = 0; x < len; ++x) r += J[(int64_t)q * len + x] * tmp[x];
          for (int x = 0; x < len; ++x) tmp[x] -= r * J[(int64_t)q * len + x];
          sm[(int64_t)q * b + j] += r;
        }
      T nv = 0;
      for (int x = 0; x < len; ++x) nv += tmp[x] * tmp[x];
      nv = sqrt(nv);
      if (acc < k && nv > Tol3<T>::qr * sqrt(nx) && nv > 0) {
        const T inv = T(1) / nv;
        for (int x = 0; x < len; ++x) J[(int64_t)acc * len + x] = tmp[x] * inv;
        sm[(int64_t)acc * b + j] = nv;
        ++acc;
      }
    }
    for (int q = acc; q < k; ++q)
      for (int x = 0; x < len; ++x) J[(int64_t)q * len + x] = T(0);
    T sc = 0;
    for (int e = 0; e < k * b; ++e) {
      const T aa = sm[e] < 0 ? -sm[e] : sm[e];
      sc = aa > sc ? aa : sc;
    }
    if (!(sc > 0) || !isfinite((double)sc)) return TNMC_E_NUMERIC;
    lg += log((double)sc);
    for (int q = 0; q < k; ++q)
      for (int x = 0; x < len; ++x) Mi[(int64_t)x * k + q] = J[(int64_t)q * len + x];
    V<T> Mn = M.at((i + 1) * cap);
    const int rest = pp[i + 1] * dr[i + 1];
    const T isc = T(1) / sc;
    for (int j = 0; j < k; ++j)
      for (int y = 0; y < rest; ++y) {
        T acc = 0;
        for (int c = 0; c < b; ++c) acc += sm[(int64_t)j * b + c] * Mn[(int64_t)c * rest + y];
        tmp[(int64_t)j * rest + y] = acc * isc;
      }
    for (int e = 0; e < k * rest; ++e) Mn[e] = tmp[e];
    dr[i] = k;
    dl[i + 1] = k;
  }
  for (int i = ns - 1; i >= 1; --i) {
    const int a = dl[i], p = pp[i], b = dr[i], len = p * b;
    V<T> Mi = M.at(i * cap);
    if (a > kMaxRows3) return TNMC_E_NUMERIC;
    for (int e = 0; e < a * len; ++e) J[e] = Mi[e];
    if (!orth_rows(J, a, len, d)) err = TNMC_E_NUMERIC;
    int k = a < len ? a : len;
    k = kmax < k ? kmax : k;
    select_rows(d, a, k, sel);
    const T smax = d[sel[0]];
    if (!(smax > 0) || !isfinite((double)smax)) return TNMC_E_NUMERIC;
    for (int j = 0; j < k; ++j) {
      const T nj = d[sel[j]];
      const T inv = nj > Tol3<T>::null * smax ? T(1) / nj : T(0);
      for (int y = 0; y < len; ++y) tmp[(int64_t)j * len + y] = J[(int64_t)sel[j] * len + y] * inv;
    }
    const T is = T(1) / smax;
    for (int r = 0; r < a; ++r)
      for (int j = 0; j < k; ++j) {
        T acc = 0;
        for (int y = 0; y < len; ++y) acc += Mi[(int64_t)r * len + y] * tmp[(int64_t)j * len + y];
        sm[(int64_t)r * k + j] = acc * is;
      }
    lg += log((double)smax);
    for (int e = 0; e < k * len; ++e) Mi[e] = tmp[e];
    V<T> Mp = M.at((i - 1) * cap);
    const int rows = dl[i - 1] * pp[i - 1];
    for (int z = 0; z < rows; ++z)
      for (int j = 0; j < k; ++j) {
        T acc = 0;
        for (int r = 0; r < a; ++r) acc += Mp[(int64_t)z * a + r] * sm[(int64_t)r * k + j];
        tmp[(int64_t)z * k + j] = acc;
      }
    for (int e = 0; e < rows * k; ++e) Mp[e] = tmp[e];
    dl[i] = k;
    dr[i - 1] = k;
  }
  {
    const int n0 = dl[0] * pp[0] * dr[0];
    T s = 0;
    for (int e = 0; e < n0; ++e) s += M[e] * M[e];
    const T nrm = sqrt(s);
    if (!(nrm > 0) || !isfinite((double)nrm)) return TNMC_E_NUMERIC;
    const T inv = T(1) / nrm;
    for (int e = 0; e < n0; ++e) M[e] *= inv;
    lg += log((double)nrm);
  }
  *logs = lg;
  return err;
}

// ---------------------------------------------------------------------------
// Builder (FP64)
// ---------------------------------------------------------------------------
// The split W = B T of a vertical bond weight W[s][s'] = exp(beta J s s') (App. A), index
// 0 <-> s = -1: eigenvectors u_0 = (1, 1)/sqrt 2, u_1 = (1, -1)/sqrt 2, eigenvalues
// 2 cosh(beta J), 2 sinh(beta J); B[s][rho] = u_rho(s) sqrt|lambda_rho|,
// T[rho][s] = sign(lambda_rho) sqrt|lambda_rho| u_rho(s).
__device__ inline double bsplit3(double bj, int s, int rho) {
  const double lam = rho ? 2.0 * sinh(bj) : 2.0 * cosh(bj);
  const double u = (rho && s) ? -0.70710678118654752440 : 0.70710678118654752440;
  return u * sqrt(fabs(lam));
}
__device__ inline double tsplit3(double bj, int rho, int s) {
  const double lam = rho ? 2.0 * sinh(bj) : 2.0 * cosh(bj);
  const double u = (rho && s) ? -0.70710678118654752440 : 0.70710678118654752440;
  return (lam < 0.0 ? -1.0 : 1.0) * sqrt(fabs(lam)) * u;
}

struct Build3 {
  int Lx, Ly, Lz, D, RP;   // RP = 2 D: pad of the uncompressed layer
  int gauge;               // 1: env_{z+1} carries the vertical bond index; V' applies B
  double beta;
  const double* Jx;
  const double* Jy;
  const double* Jz;
  const double* h;
  double* A;         // compressed layers, pad D
  int32_t* dims;     // [Lz][Ly][Lx][4]
  double* raw;       // one uncompressed layer, [Ly][Lx][2][RP]^4
  int32_t* rdims;    // [Ly][Lx][4]
  double* work;      // per-thread scratch (AoS)
  int64_t work_per;  // doubles per thread
  double* logs;      // [Lx + Ly]
  double* log_scale;
  int32_t* status;
};

__device__ __forceinline__ int64_t pad_index(int P, int s, int u, int l, int d, int r) {
  return ((((int64_t)s * P + u) * P + l) * P + d) * P + r;
}

__device__ __forceinline__ double spin_of(int i) { return i ? 1.0 : -1.0; }

// D_z H_z V_z env_{z+1} into `raw` (grid-stride over every padded entry of the layer).
__global__ void layer_raw_kernel(Build3 a, int z) {
  const int Lx = a.Lx, Ly = a.Ly, RP = a.RP, D = a.D;
  const int64_t per = 2LL * RP * RP * RP * RP;
  const int64_t total = (int64_t)Lx * Ly * per;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int site = (int)(idx / per);
    int64_t e = idx % per;
    const int R = (int)(e % RP); e /= RP;
    const int Dd = (int)(e % RP); e /= RP;
    const int L = (int)(e % RP); e /= RP;
    const int U = (int)(e % RP); e /= RP;
    const int s = (int)e;
    const int y = site / Lx, x = site % Lx;
    const bool last = (z == a.Lz - 1);
    int nu = 1, nl = 1, nd = 1, nr = 1;
    const int32_t* nd4 = last ? nullptr : a.dims + (((int64_t)(z + 1) * Ly + y) * Lx + x) * 4;
    if (!last) {
      nu = nd4[0];
      nl = nd4[1];
      nd = nd4[2];
      nr = nd4[3];
    }
    const int ku = (y > 0) ? 2 : 1, kl = (x > 0) ? 2 : 1, kd = (y < Ly - 1) ? 2 : 1, kr = (x < Lx - 1) ? 2 : 1;
    const int du = nu * ku, dl = nl * kl, ddim = nd * kd, dr = nr * kr;
    if (e == 0 && U == 0 && L == 0 && Dd == 0 && R == 0 && s == 0) {
      int32_t* rd = a.rdims + (int64_t)site * 4;
      rd[0] = du;
      rd[1] = dl;
      rd[2] = ddim;
      rd[3] = dr;
    }
    double val = 0.0;
    if (U < du && L < dl && Dd < ddim && R < dr) {
      const int u = (ku == 2) ? U >> 1 : U, cu = U & 1;
      const int l = (kl == 2) ? L >> 1 : L, cl = L & 1;
      const int d = (kd == 2) ? Dd >> 1 : Dd, cd = Dd & 1;
      const int r = (kr == 2) ? R >> 1 : R, cr = R & 1;
      bool ok = true;
      if (kd == 2 && cd != s) ok = false;
      if (kr == 2 && cr != s) ok = false;
      if (ok) {
        const double sv = spin_of(s);
        double base;
        if (last) {
          base = (u == 0 && l == 0 && d == 0 && r == 0) ? 1.0 : 0.0;
        } else {
          const double bj = a.beta * a.Jz[((int64_t)z * Ly + y) * Lx + x];
          const double* An = a.A + (((int64_t)(z + 1) * Ly + y) * Lx + x) * 2 * D * D * D * D;
          if (a.gauge == 1)
            base = bsplit3(bj, s, 0) * An[pad_index(D, 0, u, l, d, r)] + bsplit3(bj, s, 1) * An[pad_index(D, 1, u, l, d, r)];
          else
            base = exp(bj * sv * -1.0) * An[pad_index(D, 0, u, l, d, r)] + exp(bj * sv) * An[pad_index(D, 1, u, l, d, r)];
        }
        val = base * exp(a.beta * a.h[((int64_t)z * Ly + y) * Lx + x] * sv);
        if (ku == 2) val *= exp(a.beta * a.Jy[((int64_t)z * (Ly - 1) + y - 1) * Lx + x] * spin_of(cu) * sv);
        if (kl == 2) val *= exp(a.beta * a.Jx[((int64_t)z * Ly + y) * (Lx - 1) + x - 1] * spin_of(cl) * sv);
      }
    }
    a.raw[idx] = val;
  }
}

// Builder scratch of one thread: MPS (L sites x cap), J, d, sm, tmp.
__device__ inline void build_scratch(const Build3& a, int t, int64_t cap, V<double>& M, V<double>& J, V<double>& d,
                                     V<double>& sm, V<double>& tmp) {
  const int L = a.Lx > a.Ly ? a.Lx : a.Ly;
  double* base = a.work + (int64_t)t * a.work_per;
  M = V<double>{base, 1};
  J = V<double>{base + L * cap, 1};
  tmp = V<double>{base + (L + 1) * cap, 1};
  sm = V<double>{base + (L + 2) * cap, 1};
  d = V<double>{base + (L + 2) * cap + (int64_t)a.RP * a.RP, 1};
}

// Columns of the uncompressed layer: vertical bonds to <= D (one thread per column).
__global__ void compress_cols_kernel(Build3 a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.Lx) return;
  const int RP = a.RP, Ly = a.Ly, Lx = a.Lx;
  const int64_t cap = 2LL * RP * RP * RP * RP;
  const int64_t per = cap;
  V<double> M, J, d, sm, tmp;
  build_scratch(a, x, cap, M, J, d, sm, tmp);
  int dl[kMaxSide3], pp[kMaxSide3], dr[kMaxSide3];
  for (int y = 0; y < Ly; ++y) {
    const int32_t* rd = a.rdims + ((int64_t)y * Lx + x) * 4;
    const int du = rd[0], dlh = rd[1], dd = rd[2], drh = rd[3];
    const int p = 2 * dlh * drh;
    dl[y] = du;
    pp[y] = p;
    dr[y] = dd;
    const double* src = a.raw + ((int64_t)y * Lx + x) * per;
    V<double> My = M.at(y * cap);
    for (int s = 0; s < 2; ++s)
      for (int u = 0; u < du; ++u)
        for (int l = 0; l < dlh; ++l)
          for (int dd2 = 0; dd2 < dd; ++dd2)
            for (int r = 0; r < drh; ++r)
              My[((int64_t)u * p + (s * dlh + l) * drh + r) * dd + dd2] = src[pad_index(RP, s, u, l, dd2, r)];
  }
  double lg = 0.0;
  const int err = mps_compress(M, cap, Ly, dl, pp, dr, a.D, J, d, sm, tmp, &lg);
  if (err) set_status(a.status, err);
  a.logs[x] = lg;
  for (int y = 0; y < Ly; ++y) {
    int32_t* rd = a.rdims + ((int64_t)y * Lx + x) * 4;
    const int dlh = rd[1], drh = rd[3];
    const int p = 2 * dlh * drh, du = dl[y], dd = dr[y];
    double* dst = a.raw + ((int64_t)y * Lx + x) * per;
    V<double> My = M.at(y * cap);
    for (int s = 0; s < 2; ++s)
      for (int u = 0; u < du; ++u)
        for (int l = 0; l < dlh; ++l)
          for (int dd2 = 0; dd2 < dd; ++dd2)
            for (int r = 0; r < drh; ++r)
              dst[pad_index(RP, s, u, l, dd2, r)] = My[((int64_t)u * p + (s * dlh + l) * drh + r) * dd + dd2];
    rd[0] = du;
    rd[2] = dd;
  }
}

// Rows: horizontal bonds to <= D, result into layer z of the environment (pad D).
__global__ void compress_rows_kernel(Build3 a, int z) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= a.Ly) return;
  const int RP = a.RP, D = a.D, Lx = a.Lx;
  const int64_t cap = 2LL * RP * RP * RP * RP;
  const int64_t per = cap;
  V<double> M, J, d, sm, tmp;
  build_scratch(a, y, cap, M, J, d, sm, tmp);
  int dl[kMaxSide3], pp[kMaxSide3], dr[kMaxSide3];
  for (int x = 0; x < Lx; ++x) {
    const int32_t* rd = a.rdims + ((int64_t)y * Lx + x) * 4;
    const int du = rd[0], dlh = rd[1], dd = rd[2], drh = rd[3];
    const int p = 2 * du * dd;
    dl[x] = dlh;
    pp[x] = p;
    dr[x] = drh;
    const double* src = a.raw + ((int64_t)y * Lx + x) * per;
    V<double> Mx = M.at(x * cap);
    for (int s = 0; s < 2; ++s)
      for (int u = 0; u < du; ++u)
        for (int l = 0; l < dlh; ++l)
          for (int dd2 = 0; dd2 < dd; ++dd2)
            for (int r = 0; r < drh; ++r)
              Mx[((int64_t)l * p + (s * du + u) * dd + dd2) * drh + r] = src[pad_index(RP, s, u, l, dd2, r)];
  }
  double lg = 0.0;
  const int err = mps_compress(M, cap, Lx, dl, pp, dr, D, J, d, sm, tmp, &lg);
  if (err) set_status(a.status, err);
  a.logs[a.Lx + y] = lg;
  for (int x = 0; x < Lx; ++x) {
    const int32_t* rd = a.rdims + ((int64_t)y * Lx + x) * 4;
    const int du = rd[0], dd = rd[2];
    const int p = 2 * du * dd, dlh = dl[x], drh = dr[x];
    if (du > D || dd > D || dlh > D || drh > D) set_status(a.status, TNMC_E_NUMERIC);
    const int64_t site = ((int64_t)z * a.Ly + y) * Lx + x;
    double* dst = a.A + site * 2 * D * D * D * D;
    V<double> Mx = M.at(x * cap);
    for (int s = 0; s < 2; ++s)
      for (int u = 0; u < D; ++u)
        for (int l = 0; l < D; ++l)
          for (int dd2 = 0; dd2 < D; ++dd2)
            for (int r = 0; r < D; ++r) {
              const bool in = u < du && l < dlh && dd2 < dd && r < drh;
              dst[pad_index(D, s, u, l, dd2, r)] = in ? Mx[((int64_t)l * p + (s * du + u) * dd + dd2) * drh + r] : 0.0;
            }
    int32_t* od = a.dims + site * 4;
    od[0] = du;
    od[1] = dlh;
    od[2] = dd;
    od[3] = drh;
  }
}

// Bond basis: the uncompressed layer is layer z's sampling PEPS (pad RP, its dims).
__global__ void keep_sampling_kernel(Build3 a, int z, double* S, int32_t* sdims) {
  const int64_t n = (int64_t)a.Ly * a.Lx * 2 * a.RP * a.RP * a.RP * a.RP;
  double* dst = S + (int64_t)z * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = a.raw[i];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)a.Ly * a.Lx * 4;
       i += (int64_t)gridDim.x * blockDim.x)
    sdims[(int64_t)z * a.Ly * a.Lx * 4 + i] = a.rdims[i];
}

// Bond basis: the upper factor T of the vertical bonds (z-1, z) on the physical leg of the
// uncompressed layer, before it is compressed: X[rho] = sum_s T[rho][s] M[s].
__global__ void apply_upper_factor_kernel(Build3 a, int z) {
  const int RP = a.RP;
  const int64_t half = (int64_t)RP * RP * RP * RP;
  const int64_t total = (int64_t)a.Ly * a.Lx * half;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t site = i / half, e = i % half;
    const int y = (int)(site / a.Lx), x = (int)(site % a.Lx);
    const double bj = a.beta * a.Jz[((int64_t)(z - 1) * a.Ly + y) * a.Lx + x];
    double* t = a.raw + site * 2 * half;
    const double v0 = t[e], v1 = t[half + e];
    t[e] = tsplit3(bj, 0, 0) * v0 + tsplit3(bj, 0, 1) * v1;
    t[half + e] = tsplit3(bj, 1, 0) * v0 + tsplit3(bj, 1, 1) * v1;
  }
}

__global__ void layer_logscale_kernel(Build3 a, int z) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < a.Lx + a.Ly; ++i) s += a.logs[i];
    a.log_scale[z] = s;
  }
}

__global__ void to_f32_kernel(const double* src, float* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// ---------------------------------------------------------------------------
// Sampler (one thread per sample)
// ---------------------------------------------------------------------------
struct Samp3 {
  int Lx, Ly, Lz, D, chi;
  double beta;
  const double* Jx;
  const double* Jy;
  const double* Jz;
  const double* h;
  const void* A;        // T tensors, pad D
  const int32_t* dims;
  int32_t* status;
  int64_t b0, Bc;       // first sample of the chunk, samples in the chunk
  uint64_t seed, offset;
  int forced;
  int8_t* spins;        // [B][Lz][Ly][Lx]
  double* logq;
  double* energy;
  int32_t* flags;
  void* scr;            // T scratch, SoA
  int32_t* iscr;        // int scratch, SoA: bot bonds [Ly][Lx+1]
};

struct Lay3 {   // offsets (in elements) of one sample's scratch
  int64_t capS, capW;
  int64_t bot, top, w, J, d, sm, tmp, R, lam, U1, U2, total;
};

__host__ __device__ inline Lay3 lay3(int Lx, int Ly, int D, int chi) {
  Lay3 o;
  const int64_t K = (int64_t)D * chi;
  o.capS = (int64_t)chi * D * chi;
  o.capW = K * D * K;
  int64_t off = 0;
  o.bot = off; off += (int64_t)Ly * Lx * o.capS;
  o.top = off; off += (int64_t)Lx * o.capS;
  o.w = off;   off += (int64_t)Lx * o.capW;
  o.J = off;   off += K * K * D;
  o.d = off;   off += K;
  o.sm = off;  off += K * K;
  o.tmp = off; off += o.capW;
  o.R = off;   off += (int64_t)(Lx + 1) * o.capS;
  o.lam = off; off += o.capS;
  o.U1 = off;  off += (int64_t)D * chi * D * chi;
  o.U2 = off;  off += (int64_t)D * D * chi * D * chi;
  o.total = off;
  return o;
}

template <typename T>
__device__ __forceinline__ T field3(const Samp3& a, int z, int y, int x, int s, const int8_t* sp) {
  if (z == 0) return T(1);
  const double up = (double)sp[(((int64_t)(z - 1) * a.Ly + y) * a.Lx + x)];
  return (T)exp(a.beta * a.Jz[((int64_t)(z - 1) * a.Ly + y) * a.Lx + x] * up * spin_of(s));
}

template <typename T>
__device__ __forceinline__ T absT(T v) {
  return v < 0 ? -v : v;
}

template <typename T>
__global__ void __launch_bounds__(128, 4) sample3d_kernel(Samp3 a) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= a.Bc) return;
  const int64_t g = a.b0 + b;
  const int Lx = a.Lx, Ly = a.Ly, Lz = a.Lz, D = a.D, chi = a.chi;
  const Lay3 o = lay3(Lx, Ly, D, chi);
  const V<T> base{static_cast<T*>(a.scr) + b, a.Bc};
  const V<T> Bot = base.at(o.bot), Top = base.at(o.top), W = base.at(o.w), J = base.at(o.J), dv = base.at(o.d);
  const V<T> sm = base.at(o.sm), tmp = base.at(o.tmp), R = base.at(o.R), lam = base.at(o.lam);
  const V<T> U1 = base.at(o.U1), U2 = base.at(o.U2);
  const V<int32_t> botb{a.iscr + b, a.Bc};
  const T* A = static_cast<const T*>(a.A);
  const int64_t site_sz = 2LL * D * D * D * D;
  int8_t* sp = a.spins + g * (int64_t)Lx * Ly * Lz;
  const uint64_t sample = a.offset + (uint64_t)g;
  double lq = 0.0;
  int flag = 0, err = 0;
  int wl[kMaxSide3 + 1], wp[kMaxSide3 + 1], wr[kMaxSide3 + 1], tb[kMaxSide3 + 1];
  for (int z = 0; z < Lz; ++z) {
    auto Aof = [&](int y, int x) { return A + (((int64_t)z * Ly + y) * Lx + x) * site_sz; };
    auto dimof = [&](int y, int x, int k) { return (int)a.dims[(((int64_t)z * Ly + y) * Lx + x) * 4 + k]; };
    // bottom boundaries, Bot[y][x] = [bl][d][br] at Bot.at((y * Lx + x) * capS), bonds botb[y][x]
    for (int x = 0; x <= Lx; ++x) botb[(int64_t)(Ly - 1) * (Lx + 1) + x] = 1;
    for (int x = 0; x < Lx; ++x) Bot.at(((int64_t)(Ly - 1) * Lx + x) * o.capS)[0] = T(1);
    for (int y = Ly - 2; y >= 0; --y) {
      for (int x = 0; x < Lx; ++x) {
        const T* As = Aof(y + 1, x);
        const int du = dimof(y + 1, x, 0), dl = dimof(y + 1, x, 1), dd = dimof(y + 1, x, 2), dr = dimof(y + 1, x, 3);
        const int bl = botb[(int64_t)(y + 1) * (Lx + 1) + x], br = botb[(int64_t)(y + 1) * (Lx + 1) + x + 1];
        const T f0 = field3<T>(a, z, y + 1, x, 0, sp), f1 = field3<T>(a, z, y + 1, x, 1, sp);
        const V<T> Bn = Bot.at(((int64_t)(y + 1) * Lx + x) * o.capS);
        const V<T> Wx = W.at(x * o.capW);
        const int ncol = dr * br;
        for (int l = 0; l < dl; ++l)
          for (int p = 0; p < bl; ++p)
            for (int u = 0; u < du; ++u)
              for (int r = 0; r < dr; ++r)
                for (int q = 0; q < br; ++q) {
                  T acc = 0;
                  for (int d = 0; d < dd; ++d) {
                    const T S = f0 * As[pad_index(D, 0, u, l, d, r)] + f1 * As[pad_index(D, 1, u, l, d, r)];
                    acc += S * Bn[((int64_t)p * dd + d) * br + q];
                  }
                  Wx[((int64_t)(l * bl + p) * du + u) * ncol + r * br + q] = acc;
                }
        wl[x] = dl * bl;
        wp[x] = du;
        wr[x] = ncol;
      }
      double lg;
      const int e = mps_compress(W, o.capW, Lx, wl, wp, wr, chi, J, dv, sm, tmp, &lg);
      err = err ? err : e;
      for (int x = 0; x < Lx; ++x) {
        const V<T> Bd = Bot.at(((int64_t)y * Lx + x) * o.capS);
        const V<T> Wx = W.at(x * o.capW);
        const int n = wl[x] * wp[x] * wr[x];
        for (int i = 0; i < n; ++i) Bd[i] = Wx[i];
        botb[(int64_t)y * (Lx + 1) + x] = wl[x];
      }
      botb[(int64_t)y * (Lx + 1) + Lx] = 1;
    }
    // rows of the layer
    for (int x = 0; x <= Lx; ++x) tb[x] = 1;
    for (int x = 0; x < Lx; ++x) Top.at(x * o.capS)[0] = T(1);
    for (int y = 0; y < Ly; ++y) {
      const int64_t brow = (int64_t)y * (Lx + 1);
      R.at((int64_t)Lx * o.capS)[0] = T(1);
      for (int x = Lx - 1; x >= 1; --x) {
        const T* As = Aof(y, x);
        const int du = dimof(y, x, 0), dl = dimof(y, x, 1), dd = dimof(y, x, 2), dr = dimof(y, x, 3);
        const int ta = tb[x], tc = tb[x + 1], pb = botb[brow + x], qb = botb[brow + x + 1];
        const T f0 = field3<T>(a, z, y, x, 0, sp), f1 = field3<T>(a, z, y, x, 1, sp);
        const V<T> Tx = Top.at(x * o.capS), Bx = Bot.at(((int64_t)y * Lx + x) * o.capS);
        const V<T> Rn = R.at((int64_t)(x + 1) * o.capS), Rx = R.at((int64_t)x * o.capS);
        // U1 = T1[a][u][r][q] = sum_c Top[a][u][c] Rn[c][r][q]
        for (int aa = 0; aa < ta; ++aa)
          for (int u = 0; u < du; ++u)
            for (int r = 0; r < dr; ++r)
              for (int q = 0; q < qb; ++q) {
                T acc = 0;
                for (int c = 0; c < tc; ++c) acc += Tx[((int64_t)aa * du + u) * tc + c] * Rn[((int64_t)c * dr + r) * qb + q];
                U1[(((int64_t)aa * du + u) * dr + r) * qb + q] = acc;
              }
        // U2 = T2[a][l][d][q] = sum_{u,r} S[u][l][d][r] T1[a][u][r][q]
        for (int aa = 0; aa < ta; ++aa)
          for (int l = 0; l < dl; ++l)
            for (int d = 0; d < dd; ++d)
              for (int q = 0; q < qb; ++q) {
                T acc = 0;
                for (int u = 0; u < du; ++u)
                  for (int r = 0; r < dr; ++r) {
                    const T S = f0 * As[pad_index(D, 0, u, l, d, r)] + f1 * As[pad_index(D, 1, u, l, d, r)];
                    acc += S * U1[(((int64_t)aa * du + u) * dr + r) * qb + q];
                  }
                U2[(((int64_t)aa * dl + l) * dd + d) * qb + q] = acc;
              }
        // R_x[a][l][p] = sum_{d,q} T2[a][l][d][q] Bot[p][d][q], rescaled by its largest entry
        T mx = 0;
        for (int aa = 0; aa < ta; ++aa)
          for (int l = 0; l < dl; ++l)
            for (int p = 0; p < pb; ++p) {
              T acc = 0;
              for (int d = 0; d < dd; ++d)
                for (int q = 0; q < qb; ++q)
                  acc += U2[(((int64_t)aa * dl + l) * dd + d) * qb + q] * Bx[((int64_t)p * dd + d) * qb + q];
              Rx[((int64_t)aa * dl + l) * pb + p] = acc;
              mx = absT(acc) > mx ? absT(acc) : mx;
            }
        if (mx > 0 && isfinite((double)mx)) {
          const T inv = T(1) / mx;
          for (int i = 0; i < ta * dl * pb; ++i) Rx[i] *= inv;
        }
      }
      lam[0] = T(1);
      for (int x = 0; x < Lx; ++x) {
        const T* As = Aof(y, x);
        const int du = dimof(y, x, 0), dl = dimof(y, x, 1), dd = dimof(y, x, 2), dr = dimof(y, x, 3);
        const int ta = tb[x], tc = tb[x + 1], pb = botb[brow + x], qb = botb[brow + x + 1];
        const V<T> Tx = Top.at(x * o.capS), Bx = Bot.at(((int64_t)y * Lx + x) * o.capS);
        const V<T> Rn = R.at((int64_t)(x + 1) * o.capS);
        // U1[l][p][u][c] = sum_a lam[a][l][p] Top[a][u][c]
        for (int l = 0; l < dl; ++l)
          for (int p = 0; p < pb; ++p)
            for (int u = 0; u < du; ++u)
              for (int c = 0; c < tc; ++c) {
                T acc = 0;
                for (int aa = 0; aa < ta; ++aa) acc += lam[((int64_t)aa * dl + l) * pb + p] * Tx[((int64_t)aa * du + u) * tc + c];
                U1[(((int64_t)l * pb + p) * du + u) * tc + c] = acc;
              }
        // U2[l][u][c][d][q] = sum_p U1[l][p][u][c] Bot[p][d][q]
        for (int l = 0; l < dl; ++l)
          for (int u = 0; u < du; ++u)
            for (int c = 0; c < tc; ++c)
              for (int d = 0; d < dd; ++d)
                for (int q = 0; q < qb; ++q) {
                  T acc = 0;
                  for (int p = 0; p < pb; ++p)
                    acc += U1[(((int64_t)l * pb + p) * du + u) * tc + c] * Bx[((int64_t)p * dd + d) * qb + q];
                  U2[((((int64_t)l * du + u) * tc + c) * dd + d) * qb + q] = acc;
                }
        // w(s) = f(s) sum_{l,u,d,r} A[s][u][l][d][r] U3[l][u][d][r] with
        // U3[l][u][d][r] = sum_{c,q} U2[l][u][c][d][q] R_{x+1}[c][r][q], each U3 entry formed
        // on the fly (it never goes to the scratch)
        T w[2];
        {
          T p0 = 0, p1 = 0;
          for (int l = 0; l < dl; ++l)
            for (int u = 0; u < du; ++u)
              for (int d = 0; d < dd; ++d)
                for (int r = 0; r < dr; ++r) {
                  T u3 = 0;
                  for (int c = 0; c < tc; ++c)
                    for (int q = 0; q < qb; ++q)
                      u3 += U2[((((int64_t)l * du + u) * tc + c) * dd + d) * qb + q] * Rn[((int64_t)c * dr + r) * qb + q];
                  p0 += As[pad_index(D, 0, u, l, d, r)] * u3;
                  p1 += As[pad_index(D, 1, u, l, d, r)] * u3;
                }
          w[0] = p0 * field3<T>(a, z, y, x, 0, sp);
          w[1] = p1 * field3<T>(a, z, y, x, 1, sp);
          if (!(w[0] > 0)) w[0] = 0;
          if (!(w[1] > 0)) w[1] = 0;
        }
        const T tot = w[0] + w[1];
        const bool bad = !(tot > 0) || !isfinite((double)tot);
        const T pplus = bad ? T(0.5) : w[1] / tot;
        const T pminus = bad ? T(0.5) : w[0] / tot;
        const int64_t si = ((int64_t)z * Ly + y) * Lx + x;
        bool plus;
        if (a.forced) {
          plus = sp[si] > 0;
        } else {
          plus = draw_plus(pplus, draw_word(a.seed, si, sample));
          sp[si] = plus ? 1 : -1;
        }
        lq += log((double)(plus ? pplus : pminus));
        if (bad) flag = TNMC_FLAG_NUMERIC;
        // lam'[c][r][q] = f(s) sum_{l,u,d} U2[l][u][c][d][q] A[s][u][l][d][r], rescaled
        const int s = plus ? 1 : 0;
        const T fs = field3<T>(a, z, y, x, s, sp);
        T mx = 0;
        for (int c = 0; c < tc; ++c)
          for (int r = 0; r < dr; ++r)
            for (int q = 0; q < qb; ++q) {
              T acc = 0;
              for (int l = 0; l < dl; ++l)
                for (int u = 0; u < du; ++u)
                  for (int d = 0; d < dd; ++d)
                    acc += U2[((((int64_t)l * du + u) * tc + c) * dd + d) * qb + q] * As[pad_index(D, s, u, l, d, r)];
              acc *= fs;
              tmp[((int64_t)c * dr + r) * qb + q] = acc;
              mx = absT(acc) > mx ? absT(acc) : mx;
            }
        const T inv = (mx > 0 && isfinite((double)mx)) ? T(1) / mx : T(1);
        for (int i = 0; i < tc * dr * qb; ++i) lam[i] = tmp[i] * inv;
      }
      if (y + 1 < Ly) {
        // Top_{y+1} = T_chi[Top_y F_y]: site [(a,l)][d][(c,r)]
        for (int x = 0; x < Lx; ++x) {
          const T* As = Aof(y, x);
          const int du = dimof(y, x, 0), dl = dimof(y, x, 1), dd = dimof(y, x, 2), dr = dimof(y, x, 3);
          const int ta = tb[x], tc = tb[x + 1];
          const int s = sp[((int64_t)z * Ly + y) * Lx + x] > 0 ? 1 : 0;
          const T fs = field3<T>(a, z, y, x, s, sp);
          const V<T> Tx = Top.at(x * o.capS), Wx = W.at(x * o.capW);
          const int ncol = tc * dr;
          for (int aa = 0; aa < ta; ++aa)
            for (int l = 0; l < dl; ++l)
              for (int d = 0; d < dd; ++d)
                for (int c = 0; c < tc; ++c)
                  for (int r = 0; r < dr; ++r) {
                    T acc = 0;
                    for (int u = 0; u < du; ++u)
                      acc += Tx[((int64_t)aa * du + u) * tc + c] * As[pad_index(D, s, u, l, d, r)];
                    Wx[((int64_t)(aa * dl + l) * dd + d) * ncol + c * dr + r] = acc * fs;
                  }
          wl[x] = ta * dl;
          wp[x] = dd;
          wr[x] = ncol;
        }
        double lg;
        const int e = mps_compress(W, o.capW, Lx, wl, wp, wr, chi, J, dv, sm, tmp, &lg);
        err = err ? err : e;
        for (int x = 0; x < Lx; ++x) {
          const V<T> Tx = Top.at(x * o.capS), Wx = W.at(x * o.capW);
          const int n = wl[x] * wp[x] * wr[x];
          for (int i = 0; i < n; ++i) Tx[i] = Wx[i];
          tb[x] = wl[x];
        }
        tb[Lx] = 1;
      }
    }
  }
  // energy (eq. ising), FP64
  double E = 0.0;
  for (int z = 0; z < Lz; ++z)
    for (int y = 0; y < Ly; ++y)
      for (int x = 0; x < Lx; ++x) {
        const double s = sp[((int64_t)z * Ly + y) * Lx + x];
        E -= a.h[((int64_t)z * Ly + y) * Lx + x] * s;
        if (x + 1 < Lx) E -= a.Jx[((int64_t)z * Ly + y) * (Lx - 1) + x] * s * sp[((int64_t)z * Ly + y) * Lx + x + 1];
        if (y + 1 < Ly) E -= a.Jy[((int64_t)z * (Ly - 1) + y) * Lx + x] * s * sp[((int64_t)z * Ly + y + 1) * Lx + x];
        if (z + 1 < Lz) E -= a.Jz[((int64_t)z * Ly + y) * Lx + x] * s * sp[((int64_t)(z + 1) * Ly + y) * Lx + x];
      }
  a.logq[g] = lq;
  a.energy[g] = E;
  if (a.flags) a.flags[g] = flag;
  if (err) set_status(a.status, err);
}


// ---------------------------------------------------------------------------
// Sampler, one group of G lanes per sample (G = 8, 16 or 32: larger bonds).  The same
// algorithm and arithmetic order per output element as sample3d_kernel; lane l owns the
// entries x = l mod G of every vector it updates, so the elementwise steps need no
// synchronisation, and only the scalars (dots, norms, maxima) go through reductions over
// the group.  Samples in one warp may take different numbers of Jacobi sweeps, so every
// shuffle and __syncwarp names the group's own lanes.  The small QR / SVD matrices
// and the sandwich buffers live in this warp's slice of shared memory; the MPS being
// compressed, the boundaries and the right vectors stay in HBM, contiguous per sample.
// ---------------------------------------------------------------------------
template <int G, typename T>
__device__ __forceinline__ T wsum(T v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gm, v, o);
  return v;
}
template <int G, typename T>
__device__ __forceinline__ T wmax(T v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const T u = __shfl_xor_sync(gm, v, o);
    v = u > v ? u : v;
  }
  return v;
}

struct WLay {   // per-warp shared-memory slice (elements of T, then ints)
  int64_t J, d, sm, tmp, lam, U1, U2, nT, nI;
};
__host__ __device__ inline WLay wlay(int D, int chi) {
  WLay w;
  const int64_t K = (int64_t)D * chi;
  int64_t off = 0;
  w.J = off;   off += K * K * D;
  w.d = off;   off += K;
  w.sm = off;  off += K * K;
  w.tmp = off; off += K * D * K;
  w.lam = off; off += (int64_t)chi * D * chi;
  w.U1 = off;  off += (int64_t)D * chi * D * chi;
  w.U2 = off;  off += (int64_t)D * D * chi * D * chi;
  w.nT = (off + 1) & ~(int64_t)1;    // keep the int tail 8-byte aligned
  w.nI = K;
  return w;
}
// bytes of one warp's slice, a multiple of 16
__host__ __device__ inline size_t wslice_bytes(const WLay& w, size_t esz) {
  return ((size_t)w.nT * esz + (size_t)w.nI * sizeof(int) + 15) & ~(size_t)15;
}

template <int G, typename T>
__device__ bool orth_rows_w(T* J, int m, int n, T* d, int lane, unsigned gm) {
  bool converged = false;
  for (int sweep = 0; sweep < kSweeps3 && !converged; ++sweep) {
    T dmax = 0;
    for (int i = 0; i < m; ++i) {
      T s = 0;
      for (int x = lane; x < n; x += G) s += J[(int64_t)i * n + x] * J[(int64_t)i * n + x];
      s = wsum<G>(s, gm);
      if (lane == 0) d[i] = s;
      dmax = s > dmax ? s : dmax;
    }
    __syncwarp(gm);
    const T dnull = Tol3<T>::null * Tol3<T>::null * dmax;
    bool rotated = false;
    for (int p = 0; p + 1 < m; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const T al = d[p], be = d[q];
        if (al <= dnull || be <= dnull) continue;
        T ga = 0;
        for (int x = lane; x < n; x += G) ga += J[(int64_t)p * n + x] * J[(int64_t)q * n + x];
        ga = wsum<G>(ga, gm);
        if (!(ga * ga > Tol3<T>::rot * Tol3<T>::rot * al * be)) continue;
        const T zeta = (be - al) / (T(2) * ga);
        const T az = zeta < 0 ? -zeta : zeta;
        const T t = az > Tol3<T>::big ? T(0.5) / zeta : (zeta >= 0 ? T(1) : T(-1)) / (az + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
        for (int x = lane; x < n; x += G) {
          const T u = J[(int64_t)p * n + x], v = J[(int64_t)q * n + x];
          J[(int64_t)p * n + x] = c * u - sn * v;
          J[(int64_t)q * n + x] = sn * u + c * v;
        }
        __syncwarp(gm);
        if (lane == 0) {
          d[p] = al - t * ga;
          d[q] = be + t * ga;
        }
        __syncwarp(gm);
        rotated = true;
      }
    }
    converged = !rotated;
  }
  for (int i = 0; i < m; ++i) {
    T s = 0;
    for (int x = lane; x < n; x += G) s += J[(int64_t)i * n + x] * J[(int64_t)i * n + x];
    s = wsum<G>(s, gm);
    if (lane == 0) d[i] = sqrt(s);
  }
  __syncwarp(gm);
  return converged;
}

template <int G, typename T>
__device__ int mps_compress_w(T* M, int64_t cap, int ns, int* dl, const int* pp, int* dr, int kmax, T* J, T* d,
                              T* sm, T* tmp, int* sel, int lane, unsigned gm, double* logs) {
  int err = 0;
  double lg = 0.0;
  for (int i = 0; i + 1 < ns; ++i) {
    const int a = dl[i], p = pp[i], b = dr[i], len = a * p;
    T* Mi = M + i * cap;
    const int k = len < b ? len : b;
    if (b > kMaxRows3) return TNMC_E_NUMERIC;
    for (int e = lane; e < k * b; e += G) sm[e] = T(0);
    __syncwarp(gm);
    int acc = 0;
    for (int j = 0; j < b; ++j) {
      T nx = 0;
      for (int x = lane; x < len; x += G) {
        const T v = Mi[(int64_t)x * b + j];
        tmp[x] = v;
        nx += v * v;
      }
      nx = wsum<G>(nx, gm);
      for (int pass = 0; pass < 2; ++pass)
        for (int q = 0; q < acc; ++q) {
          T r = 0;
          for (int x = lane; x < len; x += G) r += J[(int64_t)q * len + x] * tmp[x];
          r = wsum<G>(r, gm);
          for (int x = lane; x < len; x += G) tmp[x] -= r * J[(int64_t)q * len + x];
          if (lane == 0) sm[(int64_t)q * b + j] += r;
        }
      T nv = 0;
      for (int x = lane; x < len; x += G) nv += tmp[x] * tmp[x];
      nv = sqrt(wsum<G>(nv, gm));
      if (acc < k && nv > Tol3<T>::qr * sqrt(nx) && nv > 0) {
        const T inv = T(1) / nv;
        for (int x = lane; x < len; x += G) J[(int64_t)acc * len + x] = tmp[x] * inv;
        if (lane == 0) sm[(int64_t)acc * b + j] = nv;
        ++acc;
      }
    }
    for (int q = acc; q < k; ++q)
      for (int x = lane; x < len; x += G) J[(int64_t)q * len + x] = T(0);
    __syncwarp(gm);
    T sc = 0;
    for (int e = lane; e < k * b; e += G) {
      const T aa = sm[e] < 0 ? -sm[e] : sm[e];
      sc = aa > sc ? aa : sc;
    }
    sc = wmax<G>(sc, gm);
    if (!(sc > 0) || !isfinite((double)sc)) return TNMC_E_NUMERIC;
    lg += log((double)sc);
    for (int e = lane; e < k * len; e += G) {
      const int x = e / k, q = e % k;
      Mi[e] = J[(int64_t)q * len + x];
    }
    T* Mn = M + (i + 1) * cap;
    const int rest = pp[i + 1] * dr[i + 1];
    const T isc = T(1) / sc;
    for (int e = lane; e < k * rest; e += G) {
      const int j = e / rest, y = e % rest;
      T accv = 0;
      for (int c = 0; c < b; ++c) accv += sm[(int64_t)j * b + c] * Mn[(int64_t)c * rest + y];
      tmp[e] = accv * isc;
    }
    __syncwarp(gm);
    for (int e = lane; e < k * rest; e += G) Mn[e] = tmp[e];
    __syncwarp(gm);
    dr[i] = k;
    dl[i + 1] = k;
  }
  for (int i = ns - 1; i >= 1; --i) {
    const int a = dl[i], p = pp[i], b = dr[i], len = p * b;
    T* Mi = M + i * cap;
    if (a > kMaxRows3) return TNMC_E_NUMERIC;
    for (int e = lane; e < a * len; e += G) J[e] = Mi[e];
    __syncwarp(gm);
    if (!orth_rows_w<G>(J, a, len, d, lane, gm)) err = TNMC_E_NUMERIC;
    int k = a < len ? a : len;
    k = kmax < k ? kmax : k;
    if (lane == 0) {
      for (int r = 0; r < a; ++r) {
        int rank = 0;
        const T dr_ = d[r];
        for (int j = 0; j < a; ++j) rank += (d[j] > dr_) || (d[j] == dr_ && j < r);
        if (rank < k) sel[rank] = r;
      }
    }
    __syncwarp(gm);
    const T smax = d[sel[0]];
    if (!(smax > 0) || !isfinite((double)smax)) return TNMC_E_NUMERIC;
    for (int e = lane; e < k * len; e += G) {
      const int j = e / len, y = e % len;
      const T nj = d[sel[j]];
      tmp[e] = nj > Tol3<T>::null * smax ? J[(int64_t)sel[j] * len + y] / nj : T(0);
    }
    __syncwarp(gm);
    const T is = T(1) / smax;
    for (int e = lane; e < a * k; e += G) {
      const int r = e / k, j = e % k;
      T accv = 0;
      for (int y = 0; y < len; ++y) accv += Mi[(int64_t)r * len + y] * tmp[(int64_t)j * len + y];
      sm[e] = accv * is;
    }
    __syncwarp(gm);
    lg += log((double)smax);
    for (int e = lane; e < k * len; e += G) Mi[e] = tmp[e];
    T* Mp = M + (i - 1) * cap;
    const int rows = dl[i - 1] * pp[i - 1];
    __syncwarp(gm);
    for (int e = lane; e < rows * k; e += G) {
      const int z = e / k, j = e % k;
      T accv = 0;
      for (int r = 0; r < a; ++r) accv += Mp[(int64_t)z * a + r] * sm[(int64_t)r * k + j];
      tmp[e] = accv;
    }
    __syncwarp(gm);
    for (int e = lane; e < rows * k; e += G) Mp[e] = tmp[e];
    __syncwarp(gm);
    dl[i] = k;
    dr[i - 1] = k;
  }
  {
    const int n0 = dl[0] * pp[0] * dr[0];
    T s = 0;
    for (int e = lane; e < n0; e += G) s += M[e] * M[e];
    const T nrm = sqrt(wsum<G>(s, gm));
    if (!(nrm > 0) || !isfinite((double)nrm)) return TNMC_E_NUMERIC;
    const T inv = T(1) / nrm;
    for (int e = lane; e < n0; e += G) M[e] *= inv;
    __syncwarp(gm);
    lg += log((double)nrm);
  }
  *logs = lg;
  return err;
}

template <typename T, int G>
__global__ void __launch_bounds__(128) sample3d_warp_kernel(Samp3 a) {
  extern __shared__ unsigned char smem3[];
  const int lane = threadIdx.x & (G - 1);
  // the G lanes of one sample: their mask within the warp
  const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;   // one sample per group of G lanes
  if (b >= a.Bc) return;      // uniform within the group
  const int64_t g = a.b0 + b;
  const int Lx = a.Lx, Ly = a.Ly, Lz = a.Lz, D = a.D, chi = a.chi;
  const Lay3 o = lay3(Lx, Ly, D, chi);
  const WLay wl = wlay(D, chi);
  T* ws = reinterpret_cast<T*>(smem3 + (size_t)(threadIdx.x / G) * wslice_bytes(wl, sizeof(T)));
  T *J = ws + wl.J, *dv = ws + wl.d, *sm = ws + wl.sm, *tmp = ws + wl.tmp, *lam = ws + wl.lam;
  T *U1 = ws + wl.U1, *U2 = ws + wl.U2;
  int* sel = reinterpret_cast<int*>(ws + wl.nT);
  T* base = static_cast<T*>(a.scr) + b * o.total;       // this sample's HBM scratch, contiguous
  T *Bot = base + o.bot, *Top = base + o.top, *W = base + o.w, *R = base + o.R;
  int32_t* botb = a.iscr + b * (int64_t)Ly * (Lx + 1);
  const T* A = static_cast<const T*>(a.A);
  const int64_t site_sz = 2LL * D * D * D * D;
  int8_t* sp = a.spins + g * (int64_t)Lx * Ly * Lz;
  const uint64_t sample = a.offset + (uint64_t)g;
  double lq = 0.0;
  int flag = 0, err = 0;
  int wlv[kMaxSide3 + 1], wp[kMaxSide3 + 1], wr[kMaxSide3 + 1], tb[kMaxSide3 + 1];
  for (int z = 0; z < Lz; ++z) {
    auto Aof = [&](int y, int x) { return A + (((int64_t)z * Ly + y) * Lx + x) * site_sz; };
    auto dimof = [&](int y, int x, int k) { return (int)a.dims[(((int64_t)z * Ly + y) * Lx + x) * 4 + k]; };
    for (int x = lane; x <= Lx; x += G) botb[(int64_t)(Ly - 1) * (Lx + 1) + x] = 1;
    for (int x = lane; x < Lx; x += G) Bot[((int64_t)(Ly - 1) * Lx + x) * o.capS] = T(1);
    __syncwarp(gm);
    for (int y = Ly - 2; y >= 0; --y) {
      for (int x = 0; x < Lx; ++x) {
        const T* As = Aof(y + 1, x);
        const int du = dimof(y + 1, x, 0), dl = dimof(y + 1, x, 1), dd = dimof(y + 1, x, 2), dr = dimof(y + 1, x, 3);
        const int bl = botb[(int64_t)(y + 1) * (Lx + 1) + x], br = botb[(int64_t)(y + 1) * (Lx + 1) + x + 1];
        const T f0 = field3<T>(a, z, y + 1, x, 0, sp), f1 = field3<T>(a, z, y + 1, x, 1, sp);
        const T* Bn = Bot + ((int64_t)(y + 1) * Lx + x) * o.capS;
        T* Wx = W + x * o.capW;
        const int ncol = dr * br;
        const int total = dl * bl * du * ncol;
        for (int e = lane; e < total; e += G) {
          int t = e;
          const int q = t % br; t /= br;
          const int r = t % dr; t /= dr;
          const int u = t % du; t /= du;
          const int p = t % bl; t /= bl;
          const int l = t;
          T acc = 0;
          for (int d = 0; d < dd; ++d) {
            const T S = f0 * As[pad_index(D, 0, u, l, d, r)] + f1 * As[pad_index(D, 1, u, l, d, r)];
            acc += S * Bn[((int64_t)p * dd + d) * br + q];
          }
          Wx[((int64_t)(l * bl + p) * du + u) * ncol + r * br + q] = acc;
        }
        wlv[x] = dl * bl;
        wp[x] = du;
        wr[x] = ncol;
      }
      __syncwarp(gm);
      double lg;
      const int e = mps_compress_w<G>(W, o.capW, Lx, wlv, wp, wr, chi, J, dv, sm, tmp, sel, lane, gm, &lg);
      err = err ? err : e;
      for (int x = 0; x < Lx; ++x) {
        T* Bd = Bot + ((int64_t)y * Lx + x) * o.capS;
        const T* Wx = W + x * o.capW;
        const int n = wlv[x] * wp[x] * wr[x];
        for (int i = lane; i < n; i += G) Bd[i] = Wx[i];
        if (lane == 0) botb[(int64_t)y * (Lx + 1) + x] = wlv[x];
      }
      if (lane == 0) botb[(int64_t)y * (Lx + 1) + Lx] = 1;
      __syncwarp(gm);
    }
    for (int x = 0; x <= Lx; ++x) tb[x] = 1;
    for (int x = lane; x < Lx; x += G) Top[x * o.capS] = T(1);
    __syncwarp(gm);
    for (int y = 0; y < Ly; ++y) {
      const int64_t brow = (int64_t)y * (Lx + 1);
      if (lane == 0) R[(int64_t)Lx * o.capS] = T(1);
      __syncwarp(gm);
      for (int x = Lx - 1; x >= 1; --x) {
        const T* As = Aof(y, x);
        const int du = dimof(y, x, 0), dl = dimof(y, x, 1), dd = dimof(y, x, 2), dr = dimof(y, x, 3);
        const int ta = tb[x], tc = tb[x + 1], pb = botb[brow + x], qb = botb[brow + x + 1];
        const T f0 = field3<T>(a, z, y, x, 0, sp), f1 = field3<T>(a, z, y, x, 1, sp);
        const T *Tx = Top + x * o.capS, *Bx = Bot + ((int64_t)y * Lx + x) * o.capS;
        const T* Rn = R + (int64_t)(x + 1) * o.capS;
        T* Rx = R + (int64_t)x * o.capS;
        for (int e = lane; e < ta * du * dr * qb; e += G) {
          int t = e;
          const int q = t % qb; t /= qb;
          const int r = t % dr; t /= dr;
          const int u = t % du;
          const int aa = t / du;
          T acc = 0;
          for (int c = 0; c < tc; ++c) acc += Tx[((int64_t)aa * du + u) * tc + c] * Rn[((int64_t)c * dr + r) * qb + q];
          U1[e] = acc;
        }
        __syncwarp(gm);
        for (int e = lane; e < ta * dl * dd * qb; e += G) {
          int t = e;
          const int q = t % qb; t /= qb;
          const int d = t % dd; t /= dd;
          const int l = t % dl;
          const int aa = t / dl;
          T acc = 0;
          for (int u = 0; u < du; ++u)
            for (int r = 0; r < dr; ++r) {
              const T S = f0 * As[pad_index(D, 0, u, l, d, r)] + f1 * As[pad_index(D, 1, u, l, d, r)];
              acc += S * U1[(((int64_t)aa * du + u) * dr + r) * qb + q];
            }
          U2[e] = acc;
        }
        __syncwarp(gm);
        T mx = 0;
        for (int e = lane; e < ta * dl * pb; e += G) {
          const int p = e % pb, l = (e / pb) % dl, aa = e / (pb * dl);
          T acc = 0;
          for (int d = 0; d < dd; ++d)
            for (int q = 0; q < qb; ++q)
              acc += U2[(((int64_t)aa * dl + l) * dd + d) * qb + q] * Bx[((int64_t)p * dd + d) * qb + q];
          Rx[e] = acc;
          mx = absT(acc) > mx ? absT(acc) : mx;
        }
        mx = wmax<G>(mx, gm);
        __syncwarp(gm);
        if (mx > 0 && isfinite((double)mx)) {
          const T inv = T(1) / mx;
          for (int e = lane; e < ta * dl * pb; e += G) Rx[e] *= inv;
        }
        __syncwarp(gm);
      }
      if (lane == 0) lam[0] = T(1);
      __syncwarp(gm);
      for (int x = 0; x < Lx; ++x) {
        const T* As = Aof(y, x);
        const int du = dimof(y, x, 0), dl = dimof(y, x, 1), dd = dimof(y, x, 2), dr = dimof(y, x, 3);
        const int ta = tb[x], tc = tb[x + 1], pb = botb[brow + x], qb = botb[brow + x + 1];
        const T *Tx = Top + x * o.capS, *Bx = Bot + ((int64_t)y * Lx + x) * o.capS;
        const T* Rn = R + (int64_t)(x + 1) * o.capS;
        for (int e = lane; e < dl * pb * du * tc; e += G) {
          int t = e;
          const int c = t % tc; t /= tc;
          const int u = t % du; t /= du;
          const int p = t % pb;
          const int l = t / pb;
          T acc = 0;
          for (int aa = 0; aa < ta; ++aa) acc += lam[((int64_t)aa * dl + l) * pb + p] * Tx[((int64_t)aa * du + u) * tc + c];
          U1[e] = acc;
        }
        __syncwarp(gm);
        for (int e = lane; e < dl * du * tc * dd * qb; e += G) {
          int t = e;
          const int q = t % qb; t /= qb;
          const int d = t % dd; t /= dd;
          const int c = t % tc; t /= tc;
          const int u = t % du;
          const int l = t / du;
          T acc = 0;
          for (int p = 0; p < pb; ++p)
            acc += U1[(((int64_t)l * pb + p) * du + u) * tc + c] * Bx[((int64_t)p * dd + d) * qb + q];
          U2[e] = acc;
        }
        __syncwarp(gm);
        // w(s) = f(s) sum_{l,u,d,r} A[s][u][l][d][r] U3[l][u][d][r], U3 = sum_{c,q} U2 R_{x+1}:
        // each lane forms its U3 entries on the fly (no U3 buffer)
        T w[2];
        {
          T p0 = 0, p1 = 0;
          for (int e = lane; e < dl * du * dd * dr; e += G) {
            int t = e;
            const int r = t % dr; t /= dr;
            const int d = t % dd; t /= dd;
            const int u = t % du;
            const int l = t / du;
            T u3 = 0;
            for (int c = 0; c < tc; ++c)
              for (int q = 0; q < qb; ++q)
                u3 += U2[((((int64_t)l * du + u) * tc + c) * dd + d) * qb + q] * Rn[((int64_t)c * dr + r) * qb + q];
            p0 += As[pad_index(D, 0, u, l, d, r)] * u3;
            p1 += As[pad_index(D, 1, u, l, d, r)] * u3;
          }
          w[0] = wsum<G>(p0, gm) * field3<T>(a, z, y, x, 0, sp);
          w[1] = wsum<G>(p1, gm) * field3<T>(a, z, y, x, 1, sp);
          if (!(w[0] > 0)) w[0] = 0;
          if (!(w[1] > 0)) w[1] = 0;
        }
        const T tot = w[0] + w[1];
        const bool bad = !(tot > 0) || !isfinite((double)tot);
        const T pplus = bad ? T(0.5) : w[1] / tot;
        const T pminus = bad ? T(0.5) : w[0] / tot;
        const int64_t si = ((int64_t)z * Ly + y) * Lx + x;
        bool plus;
        if (a.forced) {
          plus = sp[si] > 0;
        } else {
          plus = draw_plus(pplus, draw_word(a.seed, si, sample));
          __syncwarp(gm);
          if (lane == 0) sp[si] = plus ? 1 : -1;
        }
        __syncwarp(gm);
        lq += log((double)(plus ? pplus : pminus));
        if (bad) flag = TNMC_FLAG_NUMERIC;
        const int s = plus ? 1 : 0;
        const T fs = field3<T>(a, z, y, x, s, sp);
        T mx = 0;
        for (int e = lane; e < tc * dr * qb; e += G) {
          const int q = e % qb, r = (e / qb) % dr, c = e / (qb * dr);
          T acc = 0;
          for (int l = 0; l < dl; ++l)
            for (int u = 0; u < du; ++u)
              for (int d = 0; d < dd; ++d)
                acc += U2[((((int64_t)l * du + u) * tc + c) * dd + d) * qb + q] * As[pad_index(D, s, u, l, d, r)];
          acc *= fs;
          tmp[e] = acc;
          mx = absT(acc) > mx ? absT(acc) : mx;
        }
        mx = wmax<G>(mx, gm);
        __syncwarp(gm);
        const T inv = (mx > 0 && isfinite((double)mx)) ? T(1) / mx : T(1);
        for (int i = lane; i < tc * dr * qb; i += G) lam[i] = tmp[i] * inv;
        __syncwarp(gm);
      }
      if (y + 1 < Ly) {
        for (int x = 0; x < Lx; ++x) {
          const T* As = Aof(y, x);
          const int du = dimof(y, x, 0), dl = dimof(y, x, 1), dd = dimof(y, x, 2), dr = dimof(y, x, 3);
          const int ta = tb[x], tc = tb[x + 1];
          const int s = sp[((int64_t)z * Ly + y) * Lx + x] > 0 ? 1 : 0;
          const T fs = field3<T>(a, z, y, x, s, sp);
          const T* Tx = Top + x * o.capS;
          T* Wx = W + x * o.capW;
          const int ncol = tc * dr;
          for (int e = lane; e < ta * dl * dd * tc * dr; e += G) {
            int t = e;
            const int r = t % dr; t /= dr;
            const int c = t % tc; t /= tc;
            const int d = t % dd; t /= dd;
            const int l = t % dl;
            const int aa = t / dl;
            T acc = 0;
            for (int u = 0; u < du; ++u) acc += Tx[((int64_t)aa * du + u) * tc + c] * As[pad_index(D, s, u, l, d, r)];
            Wx[((int64_t)(aa * dl + l) * dd + d) * ncol + c * dr + r] = acc * fs;
          }
          wlv[x] = ta * dl;
          wp[x] = dd;
          wr[x] = ncol;
        }
        __syncwarp(gm);
        double lg;
        const int e = mps_compress_w<G>(W, o.capW, Lx, wlv, wp, wr, chi, J, dv, sm, tmp, sel, lane, gm, &lg);
        err = err ? err : e;
        for (int x = 0; x < Lx; ++x) {
          T* Tx = Top + x * o.capS;
          const T* Wx = W + x * o.capW;
          const int n = wlv[x] * wp[x] * wr[x];
          for (int i = lane; i < n; i += G) Tx[i] = Wx[i];
          tb[x] = wlv[x];
        }
        tb[Lx] = 1;
        __syncwarp(gm);
      }
    }
  }
  if (lane == 0) {
    double E = 0.0;
    for (int z = 0; z < Lz; ++z)
      for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
          const double s = sp[((int64_t)z * Ly + y) * Lx + x];
          E -= a.h[((int64_t)z * Ly + y) * Lx + x] * s;
          if (x + 1 < Lx) E -= a.Jx[((int64_t)z * Ly + y) * (Lx - 1) + x] * s * sp[((int64_t)z * Ly + y) * Lx + x + 1];
          if (y + 1 < Ly) E -= a.Jy[((int64_t)z * (Ly - 1) + y) * Lx + x] * s * sp[((int64_t)z * Ly + y + 1) * Lx + x];
          if (z + 1 < Lz) E -= a.Jz[((int64_t)z * Ly + y) * Lx + x] * s * sp[((int64_t)(z + 1) * Ly + y) * Lx + x];
        }
    a.logq[g] = lq;
    a.energy[g] = E;
    if (a.flags) a.flags[g] = flag;
    if (err) set_status(a.status, err);
  }
}
}  // namespace
}  // namespace tnmc

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
#define CHECK3(cond, ...)          \
  do {                             \
    if (!(cond)) {                 \
      tnmc_set_error(__VA_ARGS__); \
      return TNMC_E_INVALID_ARG;   \
    }                              \
  } while (0)

static size_t align256_3(size_t b) { return (b + 255) & ~(size_t)255; }

// One launch of the group-per-sample sampler: spb samples (spb G threads) per CTA.
template <typename T, int G>
static tnmc_status launch_group(const tnmc::Samp3& a, int spb, size_t wbytes, cudaStream_t s) {
  const size_t smem = (size_t)spb * wbytes;
  TNMC_CUDA_TRY(cudaFuncSetAttribute(tnmc::sample3d_warp_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  const unsigned blocks = (unsigned)((a.Bc + spb - 1) / spb);
  tnmc::sample3d_warp_kernel<T, G><<<blocks, spb * G, smem, s>>>(a);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

extern "C" {

static tnmc_status build3d(const tnmc_lattice3d* lat, double beta, int D, int chi, int gauge, void* stream,
                           tnmc3d_env** out) {
  using namespace tnmc;
  CHECK3(lat && out, "lat and out must be non-null");
  *out = nullptr;
  const int Lx = lat->Lx, Ly = lat->Ly, Lz = lat->Lz;
  CHECK3(Lx >= 1 && Ly >= 1 && Lz >= 1 && Lx <= kMaxSide3 && Ly <= kMaxSide3 && Lz <= 4096,
         "lattice %d x %d x %d out of range (in-layer sides <= %d)", Lz, Ly, Lx, kMaxSide3);
  CHECK3(D >= 1 && D <= 8, "D = %d must be in [1, 8]", D);
  const int Ds = gauge ? 2 * D : D;
  CHECK3(chi >= 1 && chi <= 32 && Ds * chi <= kMaxRows3, "chi = %d must be in [1, 32] with %sD chi <= %d", chi,
         gauge ? "2 " : "", kMaxRows3);
  CHECK3(isfinite(beta) && beta >= 0.0, "beta must be finite and >= 0");
  CHECK3(lat->h && (Lx == 1 || lat->Jx) && (Ly == 1 || lat->Jy) && (Lz == 1 || lat->Jz), "couplings must be non-null");
  const size_t nJx = (size_t)Lz * Ly * (Lx - 1), nJy = (size_t)Lz * (Ly - 1) * Lx, nJz = (size_t)(Lz - 1) * Ly * Lx;
  const size_t nh = (size_t)Lz * Ly * Lx;
  for (size_t i = 0; i < nJx; ++i) CHECK3(isfinite(lat->Jx[i]), "Jx[%zu] is not finite", i);
  for (size_t i = 0; i < nJy; ++i) CHECK3(isfinite(lat->Jy[i]), "Jy[%zu] is not finite", i);
  for (size_t i = 0; i < nJz; ++i) CHECK3(isfinite(lat->Jz[i]), "Jz[%zu] is not finite", i);
  for (size_t i = 0; i < nh; ++i) CHECK3(isfinite(lat->h[i]), "h[%zu] is not finite", i);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t site = 2 * (size_t)D * D * D * D;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256_3(bytes);
    return o;
  };
  const size_t oJx = take((nJx ? nJx : 1) * 8), oJy = take((nJy ? nJy : 1) * 8), oJz = take((nJz ? nJz : 1) * 8);
  const size_t oh = take(nh * 8), oA64 = take(nh * site * 8), oA32 = take(nh * site * 4);
  const size_t odims = take(nh * 4 * 4), ols = take((size_t)Lz * 8), ost = take(8);
  const size_t ssite = 2 * (size_t)Ds * Ds * Ds * Ds;
  const size_t oS64 = gauge ? take(nh * ssite * 8) : 0, oS32 = gauge ? take(nh * ssite * 4) : 0;
  const size_t osd = gauge ? take(nh * 4 * 4) : 0;
  tnmc3d_env* env = new (std::nothrow) tnmc3d_env();
  if (!env) {
    tnmc_set_error("host allocation failed");
    return TNMC_E_NOMEM;
  }
  env->alloc = current_allocator();
  char* base = static_cast<char*>(dev_alloc(env->alloc, off, s));
  if (!base) {
    delete env;
    tnmc_set_error("cannot allocate %zu bytes for the 3D environment", off);
    return TNMC_E_NOMEM;
  }
  env->arena = base;
  env->arena_bytes = off;
  env->Lx = Lx;
  env->Ly = Ly;
  env->Lz = Lz;
  env->D = D;
  env->chi = chi;
  env->beta = beta;
  env->Jx = reinterpret_cast<double*>(base + oJx);
  env->Jy = reinterpret_cast<double*>(base + oJy);
  env->Jz = reinterpret_cast<double*>(base + oJz);
  env->h = reinterpret_cast<double*>(base + oh);
  env->A64 = reinterpret_cast<double*>(base + oA64);
  env->A32 = reinterpret_cast<float*>(base + oA32);
  env->dims = reinterpret_cast<int32_t*>(base + odims);
  env->log_scale = reinterpret_cast<double*>(base + ols);
  env->status = reinterpret_cast<int32_t*>(base + ost);
  env->gauge = gauge;
  env->Ds = Ds;
  env->S64 = gauge ? reinterpret_cast<double*>(base + oS64) : env->A64;
  env->S32 = gauge ? reinterpret_cast<float*>(base + oS32) : env->A32;
  env->sdims = gauge ? reinterpret_cast<int32_t*>(base + osd) : env->dims;
  // builder scratch
  const int RP = 2 * D;
  const int L = Lx > Ly ? Lx : Ly;
  const int64_t cap = 2LL * RP * RP * RP * RP;
  const int64_t per_thread = (L + 2) * cap + (int64_t)RP * RP + RP;
  const size_t wraw = (size_t)Ly * Lx * cap * 8, wrd = (size_t)Ly * Lx * 4 * 4;
  const size_t wthr = (size_t)L * per_thread * 8, wlogs = (size_t)(Lx + Ly) * 8;
  const size_t wbytes = align256_3(wraw) + align256_3(wrd) + align256_3(wthr) + align256_3(wlogs);
  char* work = static_cast<char*>(dev_alloc(env->alloc, wbytes, s));
  tnmc_status st = TNMC_OK;
  do {
    if (!work) {
      st = TNMC_E_NOMEM;
      tnmc_set_error("cannot allocate %zu bytes of 3D builder scratch", wbytes);
      break;
    }
    if (cudaMemsetAsync(base, 0, off, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    if (nJx && cudaMemcpyAsync(env->Jx, lat->Jx, nJx * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    if (nJy && cudaMemcpyAsync(env->Jy, lat->Jy, nJy * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    if (nJz && cudaMemcpyAsync(env->Jz, lat->Jz, nJz * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    if (cudaMemcpyAsync(env->h, lat->h, nh * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
    Build3 a;
    a.Lx = Lx;
    a.Ly = Ly;
    a.Lz = Lz;
    a.D = D;
    a.RP = RP;
    a.gauge = gauge;
    a.beta = beta;
    a.Jx = env->Jx;
    a.Jy = env->Jy;
    a.Jz = env->Jz;
    a.h = env->h;
    a.A = env->A64;
    a.dims = env->dims;
    a.raw = reinterpret_cast<double*>(work);
    a.rdims = reinterpret_cast<int32_t*>(work + align256_3(wraw));
    a.work = reinterpret_cast<double*>(work + align256_3(wraw) + align256_3(wrd));
    a.work_per = per_thread;
    a.logs = reinterpret_cast<double*>(work + align256_3(wraw) + align256_3(wrd) + align256_3(wthr));
    a.log_scale = env->log_scale;
    a.status = env->status;
    for (int z = Lz - 1; z >= 0 && st == TNMC_OK; --z) {
      layer_raw_kernel<<<1024, 256, 0, s>>>(a, z);
      if (gauge) {
        keep_sampling_kernel<<<1024, 256, 0, s>>>(a, z, env->S64, env->sdims);
        if (z == 0) break;            // env'_0 is never used
        apply_upper_factor_kernel<<<1024, 256, 0, s>>>(a, z);
      }
      compress_cols_kernel<<<1, Lx, 0, s>>>(a);
      compress_rows_kernel<<<1, Ly, 0, s>>>(a, z);
      layer_logscale_kernel<<<1, 32, 0, s>>>(a, z);
      if (cudaGetLastError() != cudaSuccess) st = TNMC_E_CUDA;
    }
    if (st == TNMC_OK && cudaGetLastError() != cudaSuccess) st = TNMC_E_CUDA;
    if (st != TNMC_OK) break;
    to_f32_kernel<<<1024, 256, 0, s>>>(env->A64, env->A32, (int64_t)(nh * site));
    if (gauge) to_f32_kernel<<<1024, 256, 0, s>>>(env->S64, env->S32, (int64_t)(nh * ssite));
    if (cudaGetLastError() != cudaSuccess) { st = TNMC_E_CUDA; break; }
    if (cudaStreamSynchronize(s) != cudaSuccess) { st = TNMC_E_CUDA; break; }
  } while (0);
  if (work) dev_free(env->alloc, work, wbytes, s);
  if (st != TNMC_OK) {
    // a refused allocation keeps its own message
    if (st == TNMC_E_CUDA) tnmc_set_error("3D build failed: %s", cudaGetErrorString(cudaGetLastError()));
    (void)cudaStreamSynchronize(s);
    dev_free(env->alloc, base, off, s);
    delete env;
    return st;
  }
  *out = env;
  return TNMC_OK;
}

tnmc_status tnmc3d_build_env(const tnmc_lattice3d* lat, double beta, int D, int chi, void* stream, tnmc3d_env** out) {
  return build3d(lat, beta, D, chi, 0, stream, out);
}

tnmc_status tnmc3d_build_env_bond(const tnmc_lattice3d* lat, double beta, int D, int chi, void* stream,
                                  tnmc3d_env** out) {
  return build3d(lat, beta, D, chi, 1, stream, out);
}

tnmc_status tnmc3d_env_free(tnmc3d_env* env) {
  if (!env) return TNMC_OK;
  (void)cudaDeviceSynchronize();
  tnmc::dev_free(env->alloc, env->arena, env->arena_bytes, 0);
  (void)cudaDeviceSynchronize();
  delete env;
  return TNMC_OK;
}

tnmc_status tnmc3d_env_status(const tnmc3d_env* env, int32_t* status) {
  CHECK3(env && status, "env and status must be non-null");
  TNMC_CUDA_TRY(cudaDeviceSynchronize());
  TNMC_CUDA_TRY(cudaMemcpy(status, env->status, 4, cudaMemcpyDeviceToHost));
  return TNMC_OK;
}

tnmc_status tnmc3d_env_export(const tnmc3d_env* env, double* tensors, int32_t* dims, double* log_scale) {
  CHECK3(env, "env must be non-null");
  TNMC_CUDA_TRY(cudaDeviceSynchronize());
  const size_t nh = (size_t)env->Lz * env->Ly * env->Lx;
  const size_t site = 2 * (size_t)env->Ds * env->Ds * env->Ds * env->Ds;
  if (tensors) TNMC_CUDA_TRY(cudaMemcpy(tensors, env->S64, nh * site * 8, cudaMemcpyDeviceToHost));
  if (dims) TNMC_CUDA_TRY(cudaMemcpy(dims, env->sdims, nh * 16, cudaMemcpyDeviceToHost));
  if (log_scale) TNMC_CUDA_TRY(cudaMemcpy(log_scale, env->log_scale, (size_t)env->Lz * 8, cudaMemcpyDeviceToHost));
  return TNMC_OK;
}

static tnmc_status run3d(const tnmc3d_env* env, int precision, int64_t B, uint64_t seed, uint64_t offset, int forced,
                         int8_t* spins, double* logq, double* energy, int32_t* flags, cudaStream_t s) {
  using namespace tnmc;
  CHECK3(env, "env must be non-null");
  CHECK3(precision == TNMC_F64 || precision == TNMC_F32, "the 3D sampler runs in TNMC_F64 or TNMC_F32");
  CHECK3(B >= 0, "B must be >= 0");
  if (B == 0) return TNMC_OK;
  CHECK3(spins && logq && energy, "spins, logq and energy must be non-null");
  const Lay3 o = lay3(env->Lx, env->Ly, env->Ds, env->chi);
  const size_t esz = precision == TNMC_F64 ? 8 : 4;
  const size_t per = o.total * esz + (size_t)env->Ly * (env->Lx + 1) * 4;
  const size_t budget = (size_t)4 << 30;
  int64_t Bc = (int64_t)(budget / per);
  if (Bc > B) Bc = B;
  if (Bc > 128) Bc -= Bc % 128;
  if (Bc < 1) Bc = 1;
  const size_t fbytes = align256_3((size_t)Bc * o.total * esz), ibytes = align256_3((size_t)Bc * env->Ly * (env->Lx + 1) * 4);
  char* scr = static_cast<char*>(dev_alloc(env->alloc, fbytes + ibytes, s));
  if (!scr) {
    tnmc_set_error("cannot allocate %zu bytes of 3D sampler scratch", fbytes + ibytes);
    return TNMC_E_NOMEM;
  }
  Samp3 a;
  a.Lx = env->Lx;
  a.Ly = env->Ly;
  a.Lz = env->Lz;
  a.D = env->Ds;
  a.chi = env->chi;
  a.beta = env->beta;
  a.Jx = env->Jx;
  a.Jy = env->Jy;
  a.Jz = env->Jz;
  a.h = env->h;
  a.A = precision == TNMC_F64 ? static_cast<const void*>(env->S64) : static_cast<const void*>(env->S32);
  a.dims = env->sdims;
  a.status = env->status;
  a.seed = seed;
  a.offset = offset;
  a.forced = forced;
  a.spins = spins;
  a.logq = logq;
  a.energy = energy;
  a.flags = flags;
  a.scr = scr;
  a.iscr = reinterpret_cast<int32_t*>(scr + fbytes);
  // one warp per sample from D chi = 16 (its QR / SVD matrices in shared memory), one
  // thread per sample below.  Measured on the 16^3 bond-basis (2, 2) line (D chi = 8):
  // one thread 15.9 s per step, groups of 8 lanes 29.3 s, of 16 lanes 41.5 s (the per-step
  // reductions and syncs cost more than the lanes gain on 8-wide vectors); at D chi = 16 the
  // warp form is the faster one.  TNMC_3D_KERNEL=thread|warp|group8|group16 overrides.
  const WLay wl = wlay(env->Ds, env->chi);
  const size_t wbytes = wslice_bytes(wl, esz);
  int dev = 0, max_optin = 0;
  TNMC_CUDA_TRY(cudaGetDevice(&dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int64_t K = (int64_t)env->Ds * env->chi;
  int G = K >= 16 ? 32 : 0;
  const char* force = getenv("TNMC_3D_KERNEL");
  if (force && force[0] == 't') G = 0;
  if (force && force[0] == 'w') G = 32;
  if (force && strcmp(force, "group8") == 0) G = 8;
  if (force && strcmp(force, "group16") == 0) G = 16;
  // samples per CTA: up to 128 / G, in whole warps, within the shared memory
  int spb = 0;
  if (G) {
    const int per_warp = 32 / G;
    const int fit = (int)((size_t)max_optin / wbytes);
    spb = 128 / G < fit ? 128 / G : fit;
    spb -= spb % per_warp;
    if (spb < per_warp) G = 0;
  }
  tnmc_status st = TNMC_OK;
  for (int64_t b0 = 0; b0 < B && st == TNMC_OK; b0 += Bc) {
    a.b0 = b0;
    a.Bc = (B - b0) < Bc ? (B - b0) : Bc;
    if (G) {
      const bool f64 = precision == TNMC_F64;
      st = G == 32 ? (f64 ? launch_group<double, 32>(a, spb, wbytes, s) : launch_group<float, 32>(a, spb, wbytes, s))
         : G == 16 ? (f64 ? launch_group<double, 16>(a, spb, wbytes, s) : launch_group<float, 16>(a, spb, wbytes, s))
                   : (f64 ? launch_group<double, 8>(a, spb, wbytes, s) : launch_group<float, 8>(a, spb, wbytes, s));
    } else {
      const int threads = 128;
      const unsigned blocks = (unsigned)((a.Bc + threads - 1) / threads);
      if (precision == TNMC_F64) sample3d_kernel<double><<<blocks, threads, 0, s>>>(a);
      else sample3d_kernel<float><<<blocks, threads, 0, s>>>(a);
      if (cudaGetLastError() != cudaSuccess) {
        tnmc_set_error("3D sampler launch failed");
        st = TNMC_E_CUDA;
      }
    }
  }
  dev_free(env->alloc, scr, fbytes + ibytes, s);
  return st;
}

tnmc_status tnmc3d_sample(const tnmc3d_env* env, int precision, int64_t B, uint64_t seed, uint64_t sample_offset,
                          int8_t* spins, double* logq, double* energy, int32_t* flags, void* stream) {
  return run3d(env, precision, B, seed, sample_offset, 0, spins, logq, energy, flags, static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc3d_logq(const tnmc3d_env* env, int precision, int64_t B, const int8_t* spins, double* logq,
                        double* energy, int32_t* flags, void* stream) {
  return run3d(env, precision, B, 0, 0, 1, const_cast<int8_t*>(spins), logq, energy, flags,
               static_cast<cudaStream_t>(stream));
}

tnmc_status tnmc3d_init_chains(const tnmc3d_env* env, int precision, int64_t C, uint64_t seed, int8_t* chain_spins,
                               double* chain_logq, double* chain_energy, void* stream) {
  CHECK3(env && chain_spins && chain_logq && chain_energy, "arguments must be non-null");
  CHECK3(C >= 0, "C must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = (int64_t)env->Lx * env->Ly * env->Lz;
  tnmc_status st = tnmc_launch_init_bits_core(n, C, seed, chain_spins, s);
  if (st != TNMC_OK) return st;
  return run3d(env, precision, C, 0, 0, 1, chain_spins, chain_logq, chain_energy, nullptr, s);
}

tnmc_status tnmc3d_mh_step(const tnmc3d_env* env, int64_t C, int64_t T, const int8_t* prop_spins,
                           const double* prop_logq, const double* prop_energy, int8_t* chain_spins,
                           double* chain_logq, double* chain_energy, uint64_t seed, uint64_t step_offset,
                           uint8_t* accepted, int64_t* n_accepted, void* stream) {
  CHECK3(env, "env must be non-null");
  CHECK3(C >= 0 && T >= 0, "C and T must be >= 0");
  CHECK3((C == 0 || T == 0) || (prop_spins && prop_logq && prop_energy && chain_spins && chain_logq && chain_energy),
         "arguments must be non-null");
  const int64_t n = (int64_t)env->Lx * env->Ly * env->Lz;
  return tnmc_launch_mh_core(n, env->beta, env->alloc, C, T, prop_spins, prop_logq, prop_energy, chain_spins,
                             chain_logq, chain_energy, seed, step_offset, accepted, n_accepted,
                             static_cast<cudaStream_t>(stream));
}

}  // extern "C"
