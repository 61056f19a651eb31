// FP64 boundary-MPS builder (App. A, eq. braket-top-tm-bot; "successive SVD").
//
// One CTA builds every row environment of one instance, bottom-up:
//   env_{Ly-1} = exact weight of row Ly-1;  env_r = T_chi[ D_r H_r V_r env_{r+1} ].
// Per row:
//   1. MPO application (V_r vertical bonds, D_r fields, H_r horizontal bonds as a
//      bond-2 copy MPO): site c becomes a (Dl x 2 x Dr) tensor with doubled bonds;
//      the right index (b, k') carries a copy k' of the site's own spin.
//   2. Left-to-right Householder QR sweep.  Because k' copies the spin, each
//      site matrix (Dl*2) x Dr is block diagonal in (s, k'), so it is factored as
//      two (Dl x Dr/2) QRs; R is absorbed into the next site.
//   3. Right-to-left SVD sweep: one-sided Jacobi (Hestenes) on the rows of the
//      (Dl x 2 Dr) site matrix, keep the chi_c largest rows (= sigma_i v_i^T), the
//      normalised rows become the right-orthonormal site, U S = A V_k is absorbed
//      into the left neighbour.
//   4. Site 0 is divided by its Frobenius norm; every positive factor removed on
//      the way is accumulated in log_scale[r].
// Working tensors live in global scratch slots (L2 resident); the linear algebra
// of one site runs in shared memory.  All arithmetic is FP64.
#include <math.h>

#include <new>

#include "common.cuh"

namespace tnmc {
namespace {

constexpr int kBuildThreads = 256;
constexpr int kWarps = kBuildThreads / 32;

struct BuildArgs {
  int Lx, Ly, chi, P;
  double beta;
  const double* Jh;
  const double* Jv;
  const double* h;
  double* M64;
  int32_t* bond;
  double* log_scale;
  double* sv;
  double* disc;
  double* logZ;
  double* work;   // (Lx + 2) slots of 8 P^2 doubles
  int32_t* status;
  int32_t* esz;   // [Ly][Lx+1] even-sector size of every bond (Z2 builder)
  int z2;         // parity-sector builder (all fields zero)
  int gauge;      // 1: bond basis (vertical bonds split as W = B T)
  int sweeps;     // > 0: two-site variational rounds after successive SVD (dense builder)
  double* vw;     // their scratch (after the Lx + 2 slots of `work`)
};

// The split W = B T of a vertical bond weight W[s][s'] = exp(beta J s s') (App. A): W has
// eigenvectors u_0 = (1, 1)/sqrt 2, u_1 = (1, -1)/sqrt 2 (index 0 <-> s = -1) with
// eigenvalues 2 cosh(beta J), 2 sinh(beta J); B[s][rho] = u_rho(s) sqrt|lambda_rho|,
// T[rho][s] = sign(lambda_rho) sqrt|lambda_rho| u_rho(s).
__host__ __device__ inline double split_B(double bj, int s, int rho) {
  const double lam = rho ? 2.0 * sinh(bj) : 2.0 * cosh(bj);
  const double u = (rho && s) ? -0.70710678118654752440 : 0.70710678118654752440;
  return u * sqrt(fabs(lam));
}
__host__ __device__ inline double split_T(double bj, int rho, int s) {
  const double lam = rho ? 2.0 * sinh(bj) : 2.0 * cosh(bj);
  const double u = (rho && s) ? -0.70710678118654752440 : 0.70710678118654752440;
  return (lam < 0.0 ? -1.0 : 1.0) * sqrt(fabs(lam)) * u;
}


__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ inline int bond_dim_dev(int chi, int Lx, int Ly, int r, int c) {
  if (c <= 0 || c >= Lx) return 1;
  int e = min(min(c, Lx - c), min(Ly - r, 30));
  return min(chi, 1 << e);
}

struct Shared {
  double* W;     // work area
  int* slot;     // [Lx + 2]
  int* dl;       // [Lx + 1]
  int* dr;       // [Lx + 1]
  int* sel;      // [2P]
  double* red;   // [64] block reduction scratch
  int* flag;     // [4]
};

// Block-wide max of v (all threads must call).
__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = red[0];
  for (int i = 1; i < kWarps; ++i) r = fmax(r, red[i]);
  __syncthreads();
  return r;
}
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < kWarps; ++i) r += red[i];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// 1. MPO application of row r into slots 0..Lx-1.
// ---------------------------------------------------------------------------
__device__ void apply_row_mpo(const BuildArgs& a, Shared& sh, int r) {
  const int Lx = a.Lx, P = a.P;
  const size_t slot_sz = (size_t)8 * P * P;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = w; c < Lx; c += kWarps) {
    const bool last_row = (r == a.Ly - 1);
    const int Dl0 = last_row ? 1 : a.bond[(r + 1) * (Lx + 1) + c];
    const int Dr0 = last_row ? 1 : a.bond[(r + 1) * (Lx + 1) + c + 1];
    const int kl = (c > 0) ? 2 : 1, kr = (c < Lx - 1) ? 2 : 1;
    const int Dl = Dl0 * kl, Dr = Dr0 * kr;
    const double hv = a.h[r * Lx + c];
    const double hp = exp(a.beta * hv), hm = exp(-a.beta * hv);
    double vs = 1.0, vd = 1.0, gs = 1.0, gd = 1.0;
    if (!last_row) {
      const double jv = a.Jv[r * Lx + c];
      vs = exp(a.beta * jv);
      vd = exp(-a.beta * jv);
    }
    if (c > 0) {
      const double jh = a.Jh[r * (Lx - 1) + c - 1];
      gs = exp(a.beta * jh);
      gd = exp(-a.beta * jh);
    }
    const double* Mn = last_row ? nullptr : a.M64 + ((size_t)(r + 1) * Lx + c) * P * 2 * P;
    double* out = a.work + (size_t)c * slot_sz;
    const int total = Dl * 2 * Dr;
    const double bjd = last_row ? 0.0 : a.beta * a.Jv[r * Lx + c];              // bond (r, r+1)
    const double bju = (r > 0) ? a.beta * a.Jv[(r - 1) * Lx + c] : 0.0;         // bond (r-1, r)
    // site value for row-r spin s (before any upper factor)
    auto site = [&](int s, int aa, int k, int b, int kp) -> double {
      if (!(kr == 1 || kp == s)) return 0.0;
      double n;
      if (last_row) {
        n = 1.0;
      } else if (a.gauge == 1) {
        // the lower factor of bond (r, r+1) on the boundary MPS's bond index rho
        n = split_B(bjd, s, 0) * Mn[((size_t)aa * 2 + 0) * P + b] + split_B(bjd, s, 1) * Mn[((size_t)aa * 2 + 1) * P + b];
      } else {
        // sum over the spin s' of row r+1: W[s][s'] = exp(beta Jv s s')
        const double m0 = Mn[((size_t)aa * 2 + 0) * P + b];
        const double m1 = Mn[((size_t)aa * 2 + 1) * P + b];
        n = s ? (vd * m0 + vs * m1) : (vs * m0 + vd * m1);
      }
      double val = n * (s ? hp : hm);
      if (kl == 2) val *= (k == s) ? gs : gd;
      return val;
    };
    for (int idx = lane; idx < total; idx += 32) {
      const int rr = idx % Dr;
      const int s = (idx / Dr) & 1;
      const int l = idx / (2 * Dr);
      int aa = l, k = 0, b = rr, kp = 0;
      if (kl == 2) { aa = l >> 1; k = l & 1; }
      if (kr == 2) { b = rr >> 1; kp = rr & 1; }
      double val;
      if (a.gauge == 1 && r > 0) {
        // bond basis: the physical index becomes rho of bond (r-1, r), through its upper factor
        val = split_T(bju, s, 0) * site(0, aa, k, b, kp) + split_T(bju, s, 1) * site(1, aa, k, b, kp);
      } else {
        val = site(s, aa, k, b, kp);
      }
      out[idx] = val;
    }
    if (lane == 0) {
      sh.dl[c] = Dl;
      sh.dr[c] = Dr;
      sh.slot[c] = c;
    }
  }
  if (threadIdx.x == 0) {
    sh.slot[Lx] = Lx;
    sh.slot[Lx + 1] = Lx + 1;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Householder QR of a column-major m x n matrix A (lda = m) in shared memory.
// On exit: R (k x n, k = min(m, n)) in Rout (row-major, ld n), Q (m x k) in Q
// (column-major, ld m).  Reflector j is stored in A[j*m + j .. ], tau[j].
// ---------------------------------------------------------------------------
__device__ void householder_qr(double* A, int m, int n, double* Q, double* Rout, double* tau,
                               double* diag) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = min(m, n);
  for (int j = 0; j < k; ++j) {
    if (w == 0) {
      double s = 0.0;
      for (int i = j + lane; i < m; i += 32) s += A[j * m + i] * A[j * m + i];
      s = warp_sum(s);
      if (lane == 0) {
        const double x0 = A[j * m + j];
        const double nrm = sqrt(s);
        if (nrm == 0.0) {
          tau[j] = 0.0;
          diag[j] = 0.0;
        } else {
          const double alpha = (x0 > 0.0) ? -nrm : nrm;
          const double v0 = x0 - alpha;
          A[j * m + j] = v0;
          tau[j] = -1.0 / (alpha * v0);
          diag[j] = alpha;
        }
      }
    }
    __syncthreads();
    const double t = tau[j];
    if (t != 0.0) {
      for (int l = j + 1 + w; l < n; l += kWarps) {
        double d = 0.0;
        for (int i = j + lane; i < m; i += 32) d += A[j * m + i] * A[l * m + i];
        d = warp_sum(d) * t;
        for (int i = j + lane; i < m; i += 32) A[l * m + i] -= d * A[j * m + i];
      }
    }
    __syncthreads();
  }
  // R
  for (int idx = threadIdx.x; idx < k * n; idx += blockDim.x) {
    const int j = idx / n, l = idx % n;
    Rout[idx] = (l < j) ? 0.0 : (l == j ? diag[j] : A[l * m + j]);
  }
  // Q = H_0 ... H_{k-1} [I_k; 0]
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) {
    const int l = idx / m, i = idx % m;
    Q[idx] = (i == l) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t != 0.0) {
      for (int l = j + w; l < k; l += kWarps) {
        double d = 0.0;
        for (int i = j + lane; i < m; i += 32) d += A[j * m + i] * Q[l * m + i];
        d = warp_sum(d) * t;
        for (int i = j + lane; i < m; i += 32) Q[l * m + i] -= d * A[j * m + i];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 2. Left-to-right QR sweep.  Returns the accumulated log of removed scales.
// ---------------------------------------------------------------------------
// Bond basis: the upper factor T mixes the physical index, so the site tensors lose the
// copy structure (physical spin == right horizontal copy) that qr_sweep factors block
// by block.  Here each site is one (2 m) x Dr matrix, rows (left, physical), and its QR
// gives a new bond of min(2 m, Dr).  Dims stay <= 2 max_bond <= P, so A and Q fit in
// 2 P^2 doubles each and R in P^2.
__device__ double qr_sweep_dense(const BuildArgs& a, Shared& sh) {
  const int Lx = a.Lx, P = a.P;
  const size_t slot_sz = (size_t)8 * P * P;
  double logs = 0.0;
  double* A = sh.W;
  double* Q = sh.W + 2 * P * P;
  double* Rb = sh.W + 4 * P * P;
  double* tau = sh.W + 6 * P * P;
  double* diag = tau + P;
  for (int c = 0; c < Lx - 1; ++c) {
    const int M = 2 * sh.dl[c];
    const int Dr = sh.dr[c];
    const int k = min(M, Dr);
    const double* X = a.work + (size_t)sh.slot[c] * slot_sz;
    double* Tn = a.work + (size_t)sh.slot[Lx] * slot_sz;   // new site c: [dl][2][k]
    for (int idx = threadIdx.x; idx < M * Dr; idx += blockDim.x) {
      const int l = idx / M, q = idx % M;   // column-major A[l*M + q]
      A[idx] = X[(size_t)q * Dr + l];
    }
    __syncthreads();
    householder_qr(A, M, Dr, Q, Rb, tau, diag);
    __syncthreads();
    for (int idx = threadIdx.x; idx < M * k; idx += blockDim.x) {
      const int j = idx / M, q = idx % M;
      Tn[(size_t)q * k + j] = Q[j * M + q];
    }
    double mx = 0.0;
    for (int idx = threadIdx.x; idx < k * Dr; idx += blockDim.x) mx = fmax(mx, fabs(Rb[idx]));
    mx = block_max(mx, sh.red);
    if (!(mx > 0.0) || !isfinite(mx)) {
      if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
      mx = 1.0;
    }
    logs += log(mx);
    const double inv = 1.0 / mx;
    // absorb R into site c+1: new[j][x'] = sum_{b >= j} R[j][b] old[b][x']
    const double* O = a.work + (size_t)sh.slot[c + 1] * slot_sz;
    double* Nn = a.work + (size_t)sh.slot[Lx + 1] * slot_sz;
    const int ncol = 2 * sh.dr[c + 1];
    for (int idx = threadIdx.x; idx < k * ncol; idx += blockDim.x) {
      const int j = idx / ncol, col = idx % ncol;
      double acc = 0.0;
      for (int b = j; b < Dr; ++b) acc += Rb[j * Dr + b] * O[(size_t)b * ncol + col];
      Nn[idx] = acc * inv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = sh.slot[c];
      sh.slot[c] = sh.slot[Lx];
      sh.slot[Lx] = t;
      t = sh.slot[c + 1];
      sh.slot[c + 1] = sh.slot[Lx + 1];
      sh.slot[Lx + 1] = t;
      sh.dr[c] = k;
      sh.dl[c + 1] = k;
    }
    __syncthreads();
  }
  return logs;
}

__device__ double qr_sweep(const BuildArgs& a, Shared& sh) {
  if (a.gauge == 1) return qr_sweep_dense(a, sh);
  const int Lx = a.Lx, P = a.P;
  const size_t slot_sz = (size_t)8 * P * P;
  double logs = 0.0;
  double* A = sh.W;
  double* Q = sh.W + 2 * P * P;
  double* Rb = sh.W + 4 * P * P;   // R_0 at Rb, R_1 at Rb + P*P
  double* tau = sh.W + 6 * P * P;
  double* diag = tau + P;
  for (int c = 0; c < Lx - 1; ++c) {
    const int m = sh.dl[c];
    const int Dr = sh.dr[c];
    const int nb = Dr / 2;
    const int k = min(m, nb);
    const double* X = a.work + (size_t)sh.slot[c] * slot_sz;
    double* Tn = a.work + (size_t)sh.slot[Lx] * slot_sz;   // new site c: [m][2][2k]
    for (int sp = 0; sp < 2; ++sp) {
      for (int idx = threadIdx.x; idx < m * nb; idx += blockDim.x) {
        const int l = idx / m, i = idx % m;   // column-major A[l*m + i]
        A[idx] = X[((size_t)i * 2 + sp) * Dr + l * 2 + sp];
      }
      __syncthreads();
      householder_qr(A, m, nb, Q, Rb + sp * P * P, tau, diag);
      __syncthreads();
      // new tensor entries (i, s, (j, s')) with s == s' == sp
      for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) {
        const int j = idx / m, i = idx % m;
        Tn[((size_t)i * 2 + sp) * (2 * k) + j * 2 + sp] = Q[j * m + i];
        Tn[((size_t)i * 2 + sp) * (2 * k) + j * 2 + (1 - sp)] = 0.0;
      }
      __syncthreads();
    }
    // scale of R
    double mx = 0.0;
    for (int idx = threadIdx.x; idx < k * nb; idx += blockDim.x)
      mx = fmax(mx, fmax(fabs(Rb[idx]), fabs(Rb[P * P + idx])));
    mx = block_max(mx, sh.red);
    if (!(mx > 0.0) || !isfinite(mx)) {
      if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
      mx = 1.0;
    }
    logs += log(mx);
    const double inv = 1.0 / mx;
    // absorb R into site c+1: new[(j,k')][x'] = sum_b R_k'[j][b] old[(b,k')][x']
    const double* O = a.work + (size_t)sh.slot[c + 1] * slot_sz;
    double* Nn = a.work + (size_t)sh.slot[Lx + 1] * slot_sz;
    const int ncol = 2 * sh.dr[c + 1];
    for (int idx = threadIdx.x; idx < 2 * k * ncol; idx += blockDim.x) {
      const int row = idx / ncol, col = idx % ncol;
      const int j = row >> 1, kp = row & 1;
      const double* Rk = Rb + kp * P * P + j * nb;
      double acc = 0.0;
      for (int b = j; b < nb; ++b) acc += Rk[b] * O[((size_t)b * 2 + kp) * ncol + col];
      Nn[idx] = acc * inv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = sh.slot[c];
      sh.slot[c] = sh.slot[Lx];
      sh.slot[Lx] = t;
      t = sh.slot[c + 1];
      sh.slot[c + 1] = sh.slot[Lx + 1];
      sh.slot[Lx + 1] = t;
      sh.dr[c] = 2 * k;
      sh.dl[c + 1] = 2 * k;
    }
    __syncthreads();
  }
  return logs;
}

// Round-robin tournament: round t of N-1 (N even), pair i of N/2.
__device__ inline void tournament(int t, int i, int N, int& p, int& q) {
  if (i == 0) {
    p = N - 1;
    q = t;
  } else {
    p = (t + i) % (N - 1);
    q = (t - i + (N - 1)) % (N - 1);
  }
}

// One-sided Jacobi (Hestenes): orthogonalise the m <= 128 rows (length n, stride
// ld) of J.  Round-robin pairing; a group of L lanes owns one pair, with L chosen
// so that all m/2 pairs of a round run at once on the CTA's threads.  Squared row
// norms d[] are maintained through the exact update alpha' = alpha - t gamma,
// beta' = beta + t gamma and recomputed at the start of every sweep.  A pair is
// rotated while |gamma| > tol sqrt(alpha beta), tol = 1e-13 (above the rounding
// level of a dot product of length <= 128).  Rows whose norm is below 1e-13 of
// the largest are at the rounding level of the matrix: they carry no information
// and are left out of the rotations (callers treat them as zero rows).  Returns
// false when the last of kJacobiSweeps sweeps still rotated (not converged); the
// value is the same on every thread.
constexpr double kJacobiTol = 1e-13;
constexpr int kJacobiSweeps = 40;
constexpr double kNullRel = 1e-13;

__device__ bool jacobi_rows(double* J, int m, int n, int ld, double* d, int* flag) {
  const int N = m + (m & 1);
  const int npairs = N / 2;
  // blockDim.x / 64 lanes per pair (a power of two): all m/2 <= 64 pairs of a round
  // at once; the per-pair scalar work is repeated on every lane of a group
  const int L = blockDim.x / 64;
  const int grp = threadIdx.x / L, gl = threadIdx.x % L;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double s = 0.0;
      for (int x = 0; x < n; ++x) s += J[(size_t)i * ld + x] * J[(size_t)i * ld + x];
      d[i] = s;
    }
    if (threadIdx.x == 0) flag[0] = 0;
    __syncthreads();
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) dmax = fmax(dmax, d[i]);
    const double dnull = kNullRel * kNullRel * dmax;
    for (int t = 0; t < N - 1; ++t) {
      {
        // every lane runs the group shuffles below (full-warp masks); groups beyond
        // the round's pairs only contribute zeros.  m <= 128 gives at most 64 pairs,
        // one per group of lanes.
        int p = m, q = m;
        if (grp < npairs) tournament(t, grp, N, p, q);
        const bool live = p < m && q < m;
        double ga = 0.0;
        double* rp = J + (size_t)(live ? p : 0) * ld;
        double* rq = J + (size_t)(live ? q : 0) * ld;
        if (live)
          for (int x = gl; x < n; x += L) ga += rp[x] * rq[x];
        for (int o = 1; o < L; o <<= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        if (live) {
          const double al = d[p], be = d[q];
          if (ga != 0.0 && al > dnull && be > dnull && ga * ga > kJacobiTol * kJacobiTol * al * be) {
            // tangent of the rotation angle in FP32 (its accuracy only sets the
            // convergence rate); cos from it by two FP64 Newton steps for 1/sqrt, so the
            // applied rotation is orthogonal to FP64 rounding whatever t is
            float zeta = (float)(be - al) / (2.0f * (float)ga);
            if (!isfinite(zeta)) zeta = (float)((be - al) / (2.0 * ga));   // outside FP32 range
            float tf;
            if (fabsf(zeta) > 1e18f) tf = 0.5f / zeta;
            else tf = (zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
            const double tt = (double)tf;
            const double x = fma(tt, tt, 1.0);
            double cs = (double)rsqrtf((float)x);
            cs = cs * fma(-0.5 * x, cs * cs, 1.5);
            cs = cs * fma(-0.5 * x, cs * cs, 1.5);
            const double sn = cs * tt;
            for (int xx = gl; xx < n; xx += L) {
              const double u = rp[xx], v = rq[xx];
              rp[xx] = cs * u - sn * v;
              rq[xx] = sn * u + cs * v;
            }
            if (gl == 0) {
              const double c2 = cs * cs;
              d[p] = c2 * fma(tt * tt, be, fma(-2.0 * tt, ga, al));
              d[q] = c2 * fma(tt * tt, al, fma(2.0 * tt, ga, be));
              flag[0] = 1;
            }
          }
        }
      }
      __syncthreads();
    }
    const int rotated = flag[0];
    __syncthreads();
    if (!rotated) return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// 3. Right-to-left SVD sweep with truncation.
// ---------------------------------------------------------------------------
__device__ double svd_sweep(const BuildArgs& a, Shared& sh, int r) {
  const int Lx = a.Lx, P = a.P;
  const size_t slot_sz = (size_t)8 * P * P;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double logs = 0.0;
  for (int c = Lx - 1; c >= 1; --c) {
    const int m = sh.dl[c];
    const int n = 2 * sh.dr[c];
    const int ld = n + 1;
    double* J = sh.W;
    double* US = sh.W + 4 * P * P + 2 * P;
    double* nrm = sh.W + 6 * P * P + 2 * P;
    const double* A = a.work + (size_t)sh.slot[c] * slot_sz;
    const int kk = bond_dim_dev(a.chi, Lx, a.Ly, r, c);
    if (kk > min(m, n)) {
      if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
      return logs;
    }
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) J[(idx / n) * ld + idx % n] = A[idx];
    __syncthreads();
    if (!jacobi_rows(J, m, n, ld, nrm, sh.flag) && threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
    for (int i = w; i < m; i += kWarps) {
      double s = 0.0;
      for (int x = lane; x < n; x += 32) s += J[i * ld + x] * J[i * ld + x];
      s = warp_sum(s);
      if (lane == 0) nrm[i] = sqrt(s);
    }
    __syncthreads();
    // rank of each row by norm (descending; ties by index) -> sel[rank] = row
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      int rank = 0;
      const double ni = nrm[i];
      for (int j = 0; j < m; ++j) {
        const double nj = nrm[j];
        rank += (nj > ni) || (nj == ni && j < i);
      }
      if (rank < kk) sh.sel[rank] = i;
    }
    __syncthreads();
    // singular-value record
    double tot = 0.0, dsc = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) tot += nrm[i] * nrm[i];
    tot = block_sum(tot, sh.red);
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      // rows not selected
      int rank = 0;
      for (int i = 0; i < m; ++i) rank += (nrm[i] > nrm[j]) || (nrm[i] == nrm[j] && i < j);
      if (rank >= kk) dsc += nrm[j] * nrm[j];
    }
    dsc = block_sum(dsc, sh.red);
    const double smax = nrm[sh.sel[0]];
    if (!(smax > 0.0) || !isfinite(smax)) {
      if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
      return logs;
    }
    double* svr = a.sv + ((size_t)r * (Lx + 1) + c) * P;
    for (int j = threadIdx.x; j < P; j += blockDim.x) svr[j] = (j < kk) ? nrm[sh.sel[j]] / sqrt(tot) : 0.0;
    if (threadIdx.x == 0) a.disc[r * (Lx + 1) + c] = dsc / tot;
    // V_k^T rows into the spare slot: new site c, [kk][2][dr]
    double* Vt = a.work + (size_t)sh.slot[Lx] * slot_sz;
    for (int idx = threadIdx.x; idx < kk * n; idx += blockDim.x) {
      const int j = idx / n, x = idx % n;
      const int i = sh.sel[j];
      const double nv = nrm[i];
      Vt[idx] = (nv > kNullRel * smax) ? J[i * ld + x] / nv : 0.0;
    }
    __syncthreads();
    // kept rows at the rounding level (norm <= 1e-13 of the largest) stay zero rows:
    // they carry no weight, so the MPS and q are unchanged
    // US = A V_k / smax  (m x kk), A from the original slot
    const double inv = 1.0 / smax;
    for (int idx = threadIdx.x; idx < m * kk; idx += blockDim.x) {
      const int i = idx / kk, j = idx % kk;
      double acc = 0.0;
      for (int x = 0; x < n; ++x) acc += A[(size_t)i * n + x] * Vt[(size_t)j * n + x];
      US[idx] = acc * inv;
    }
    __syncthreads();
    logs += log(smax);
    // absorb into site c-1: rows (l, s) of length m -> length kk
    const double* O = a.work + (size_t)sh.slot[c - 1] * slot_sz;
    double* Nn = a.work + (size_t)sh.slot[Lx + 1] * slot_sz;
    const int rows = sh.dl[c - 1] * 2;
    for (int idx = threadIdx.x; idx < rows * kk; idx += blockDim.x) {
      const int q = idx / kk, j = idx % kk;
      double acc = 0.0;
      for (int i = 0; i < m; ++i) acc += O[(size_t)q * m + i] * US[i * kk + j];
      Nn[idx] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = sh.slot[c];
      sh.slot[c] = sh.slot[Lx];
      sh.slot[Lx] = t;
      t = sh.slot[c - 1];
      sh.slot[c - 1] = sh.slot[Lx + 1];
      sh.slot[Lx + 1] = t;
      sh.dl[c] = kk;
      sh.dr[c - 1] = kk;
    }
    __syncthreads();
  }
  return logs;
}

// ---------------------------------------------------------------------------
// 4. Two-site variational compression (App. A names it beside successive SVD).
//
// X is the exact row (the MPO-MPS product, saved before the QR sweep), Y the
// successive-SVD result in the slots.  Each round is a left-to-right and a
// right-to-left pass over the pairs (c, c+1).  With the sites outside the pair
// isometries, the closest Y to X has the two-site tensor
//   Theta[(a,s),(t,b)] = sum Lenv[a][a'] X_c[a'][s][x] X_{c+1}[x][t][b'] Renv[b][b'],
// and the best one of rank k at bond c+1 is its truncated SVD.  Going right,
// Y_c = U (one-sided Jacobi on the rows of Theta^T gives u_j to working accuracy
// however small s_j is) and Y_{c+1} = U^T Theta; going left, Y_{c+1} = V^T (Jacobi
// on the rows of Theta) and Y_c = Theta V.  Overlap environments are rescaled by
// their largest entry; the log of the scale of Renv[2] plus the norm of the final
// Y_0 is the row's log-scale.  Scratch (a.vw): X store (Lx slots), T1, T2, Theta
// (one slot each), Lenv[c] and Renv[c] (2 P^2 each, c <= Lx), log-scales of Renv, dims.
// Sites left of a pair are untouched by a right-to-left pass until it reaches them,
// so the Lenv[c] of the left-to-right pass serve it.
// ---------------------------------------------------------------------------
struct VarWork {
  double* X;      // [Lx] slots
  double* T1;
  double* T2;
  double* Th;
  double* Lenv;   // [Lx + 1][2 P^2]
  double* Renv;   // [Lx + 1][2 P^2]
  double* lR;     // [Lx + 1]
  int* xdl;       // [Lx] left / right dims of X_c
  int* xdr;
};

__device__ inline VarWork var_work(const BuildArgs& a) {
  const size_t slot_sz = (size_t)8 * a.P * a.P;
  VarWork v;
  v.X = a.vw;
  v.T1 = v.X + (size_t)a.Lx * slot_sz;
  v.T2 = v.T1 + slot_sz;
  v.Th = v.T2 + slot_sz;
  v.Lenv = v.Th + slot_sz;
  v.Renv = v.Lenv + (size_t)(a.Lx + 1) * 2 * a.P * a.P;
  v.lR = v.Renv + (size_t)(a.Lx + 1) * 2 * a.P * a.P;
  v.xdl = reinterpret_cast<int*>(v.lR + a.Lx + 1);
  v.xdr = v.xdl + a.Lx;
  return v;
}

size_t var_work_doubles(int Lx, int P) {
  const size_t slot_sz = (size_t)8 * P * P;
  return (size_t)(Lx + 3) * slot_sz + (size_t)(Lx + 1) * 4 * P * P + (Lx + 1) + Lx;   // + 2 Lx ints
}

// The exact row X (slots as apply_row_mpo left them) into the X store.
__device__ void var_save_x(const BuildArgs& a, Shared& sh) {
  const VarWork v = var_work(a);
  const size_t slot_sz = (size_t)8 * a.P * a.P;
  for (int c = 0; c < a.Lx; ++c) {
    const double* src = a.work + (size_t)sh.slot[c] * slot_sz;
    double* dst = v.X + (size_t)c * slot_sz;
    const int n = sh.dl[c] * 2 * sh.dr[c];
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
      v.xdl[c] = sh.dl[c];
      v.xdr[c] = sh.dr[c];
    }
  }
  __syncthreads();
}

// Renv_out[ay][ax] = sum_{t, by, bx} Y[ay][t][by] X[ax][t][bx] Renv_in[by][bx]; returns the
// log of the largest entry, divided out.  tmp: [ax][t][by].
__device__ double var_right_overlap(const BuildArgs& a, Shared& sh, const double* Y, int ay, int by, const double* X,
                                    int ax, int bx, const double* Rin, double* tmp, double* Rout) {
  for (int idx = threadIdx.x; idx < ax * 2 * by; idx += blockDim.x) {
    const int b = idx % by, q = idx / by;   // q = (x, t)
    double acc = 0.0;
    for (int k = 0; k < bx; ++k) acc += X[(size_t)q * bx + k] * Rin[(size_t)b * bx + k];
    tmp[idx] = acc;
  }
  __syncthreads();
  double mx = 0.0;
  for (int idx = threadIdx.x; idx < ay * ax; idx += blockDim.x) {
    const int i = idx / ax, x = idx % ax;
    double acc = 0.0;
    for (int t = 0; t < 2; ++t)
      for (int b = 0; b < by; ++b) acc += Y[((size_t)i * 2 + t) * by + b] * tmp[((size_t)x * 2 + t) * by + b];
    Rout[idx] = acc;
    mx = fmax(mx, fabs(acc));
  }
  mx = block_max(mx, sh.red);
  if (!(mx > 0.0) || !isfinite(mx)) {
    if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
    mx = 1.0;
  }
  const double inv = 1.0 / mx;
  for (int idx = threadIdx.x; idx < ay * ax; idx += blockDim.x) Rout[idx] *= inv;
  __syncthreads();
  return log(mx);
}

// Theta of pair (c, c+1) into v.Th (m x n row-major, m = 2 ay, n = 2 by); T1 = Lenv X_c kept.
__device__ void var_theta(const BuildArgs& a, const VarWork& v, int c, int ay, int by) {
  const size_t slot_sz = (size_t)8 * a.P * a.P;
  const double* Xc = v.X + (size_t)c * slot_sz;
  const double* Xn = v.X + (size_t)(c + 1) * slot_sz;
  const double* R = v.Renv + (size_t)(c + 2) * 2 * a.P * a.P;
  const double* Le = v.Lenv + (size_t)c * 2 * a.P * a.P;
  const int ax = v.xdl[c], xm = v.xdr[c], bx = v.xdr[c + 1];
  // T1[ay][s][x] = sum_ax' Lenv[ay][ax'] X_c[ax'][s][x]
  for (int idx = threadIdx.x; idx < ay * 2 * xm; idx += blockDim.x) {
    const int i = idx / (2 * xm), q = idx % (2 * xm);
    double acc = 0.0;
    for (int k = 0; k < ax; ++k) acc += Le[(size_t)i * ax + k] * Xc[(size_t)k * 2 * xm + q];
    v.T1[idx] = acc;
  }
  __syncthreads();
  // T2[(ay,s)][t][bx] = sum_x T1[(ay,s)][x] X_{c+1}[x][t][bx]
  for (int idx = threadIdx.x; idx < ay * 2 * 2 * bx; idx += blockDim.x) {
    const int row = idx / (2 * bx), q = idx % (2 * bx);
    double acc = 0.0;
    for (int k = 0; k < xm; ++k) acc += v.T1[(size_t)row * xm + k] * Xn[(size_t)k * 2 * bx + q];
    v.T2[idx] = acc;
  }
  __syncthreads();
  // Theta[(ay,s)][(t,by)] = sum_bx T2[(ay,s)][t][bx] Renv[by][bx]
  const int n = 2 * by;
  for (int idx = threadIdx.x; idx < ay * 2 * n; idx += blockDim.x) {
    const int row = idx / n, col = idx % n;
    const int t = col / by, b = col % by;
    double acc = 0.0;
    for (int k = 0; k < bx; ++k) acc += v.T2[((size_t)row * 2 + t) * bx + k] * R[(size_t)b * bx + k];
    v.Th[idx] = acc;
  }
  __syncthreads();
}

// Truncated SVD of Theta (m x n) to kk: one-sided Jacobi on the rows of Theta^T
// (right) or of Theta (left).  Writes the new Y_c ([m/2][2][kk]) and Y_{c+1}
// ([kk][2][n/2]); when `record`, the singular-value record of bond c+1.
__device__ void var_split(const BuildArgs& a, Shared& sh, const VarWork& v, int r, int c, int m, int n, int kk,
                          bool right, bool record, double* Yc, double* Yn) {
  const int P = a.P;
  const int rows = right ? n : m, len = right ? m : n;
  const int ld = len + 1;
  double* J = sh.W;
  double* nrm = sh.W + 6 * P * P + 2 * P;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (kk > min(m, n) || rows > 128) {
    if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
    return;
  }
  for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
    const int i = idx / n, x = idx % n;
    if (right) J[(size_t)x * ld + i] = v.Th[idx];
    else J[(size_t)i * ld + x] = v.Th[idx];
  }
  __syncthreads();
  if (!jacobi_rows(J, rows, len, ld, nrm, sh.flag) && threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
  for (int i = w; i < rows; i += kWarps) {
    double s = 0.0;
    for (int x = lane; x < len; x += 32) s += J[i * ld + x] * J[i * ld + x];
    s = warp_sum(s);
    if (lane == 0) nrm[i] = sqrt(s);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    int rank = 0;
    const double ni = nrm[i];
    for (int j = 0; j < rows; ++j) {
      const double nj = nrm[j];
      rank += (nj > ni) || (nj == ni && j < i);
    }
    if (rank < kk) sh.sel[rank] = i;
  }
  __syncthreads();
  const double smax = nrm[sh.sel[0]];
  if (!(smax > 0.0) || !isfinite(smax)) {
    if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
    return;
  }
  if (record) {
    double tot = 0.0, dsc = 0.0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) tot += nrm[i] * nrm[i];
    tot = block_sum(tot, sh.red);
    for (int j = threadIdx.x; j < rows; j += blockDim.x) {
      int rank = 0;
      for (int i = 0; i < rows; ++i) rank += (nrm[i] > nrm[j]) || (nrm[i] == nrm[j] && i < j);
      if (rank >= kk) dsc += nrm[j] * nrm[j];
    }
    dsc = block_sum(dsc, sh.red);
    double* svr = a.sv + ((size_t)r * (a.Lx + 1) + c + 1) * P;
    for (int j = threadIdx.x; j < P; j += blockDim.x) svr[j] = (j < kk) ? nrm[sh.sel[j]] / sqrt(tot) : 0.0;
    if (threadIdx.x == 0) a.disc[r * (a.Lx + 1) + c + 1] = dsc / tot;
  }
  // the isometry: kept rows normalised (rows at the rounding level stay zero)
  double* iso = right ? v.T2 : Yn;   // right: U^T rows (kk x m) staged in T2; left: V^T = Y_{c+1}
  for (int idx = threadIdx.x; idx < kk * len; idx += blockDim.x) {
    const int j = idx / len, x = idx % len;
    const int i = sh.sel[j];
    const double nv = nrm[i];
    iso[idx] = (nv > kNullRel * smax) ? J[i * ld + x] / nv : 0.0;
  }
  __syncthreads();
  if (right) {
    // Y_c[q][j] = u_j[q];  Y_{c+1}[j][x] = sum_q u_j[q] Theta[q][x]
    for (int idx = threadIdx.x; idx < m * kk; idx += blockDim.x) {
      const int q = idx / kk, j = idx % kk;
      Yc[idx] = iso[(size_t)j * m + q];
    }
    for (int idx = threadIdx.x; idx < kk * n; idx += blockDim.x) {
      const int j = idx / n, x = idx % n;
      double acc = 0.0;
      for (int q = 0; q < m; ++q) acc += iso[(size_t)j * m + q] * v.Th[(size_t)q * n + x];
      Yn[idx] = acc;
    }
  } else {
    // Y_c[q][j] = sum_x Theta[q][x] v_j[x]
    for (int idx = threadIdx.x; idx < m * kk; idx += blockDim.x) {
      const int q = idx / kk, j = idx % kk;
      double acc = 0.0;
      for (int x = 0; x < n; ++x) acc += v.Th[(size_t)q * n + x] * iso[(size_t)j * n + x];
      Yc[idx] = acc;
    }
  }
  __syncthreads();
}

// Returns the row's log-scale; Y_0 (unnormalised, norm = the removed scale's
// remainder) and the right-orthonormal Y_1.. are left in the slots.
__device__ double variational_sweeps(const BuildArgs& a, Shared& sh, int r) {
  const int Lx = a.Lx, P = a.P;
  const size_t slot_sz = (size_t)8 * P * P;
  const size_t env_sz = (size_t)2 * P * P;
  const VarWork v = var_work(a);
  auto Yp = [&](int c) { return a.work + (size_t)sh.slot[c] * slot_sz; };
  // right environments of the successive-SVD start
  if (threadIdx.x == 0) {
    v.Renv[(size_t)Lx * env_sz] = 1.0;
    v.lR[Lx] = 0.0;
  }
  __syncthreads();
  for (int c = Lx - 1; c >= 2; --c) {
    const double l = var_right_overlap(a, sh, Yp(c), sh.dl[c], sh.dr[c], v.X + (size_t)c * slot_sz, v.xdl[c], v.xdr[c],
                                       v.Renv + (size_t)(c + 1) * env_sz, v.T1, v.Renv + (size_t)c * env_sz);
    if (threadIdx.x == 0) v.lR[c] = v.lR[c + 1] + l;
    __syncthreads();
  }
  for (int sweep = 0; sweep < a.sweeps; ++sweep) {
    if (threadIdx.x == 0) v.Lenv[0] = 1.0;
    __syncthreads();
    for (int c = 0; c < Lx - 1; ++c) {
      const int ay = sh.dl[c], by = sh.dr[c + 1];
      const int kk = bond_dim_dev(a.chi, Lx, a.Ly, r, c + 1);
      var_theta(a, v, c, ay, by);
      var_split(a, sh, v, r, c, 2 * ay, 2 * by, kk, true, false, Yp(c), Yp(c + 1));
      if (threadIdx.x == 0) {
        sh.dr[c] = kk;
        sh.dl[c + 1] = kk;
      }
      __syncthreads();
      if (c + 1 < Lx - 1) {
        // Lenv[c+1][j][x] = sum_{a, s} Y_c[a][s][j] T1[a][s][x]  (T1 = Lenv[c] X_c, still in place)
        const int xm = v.xdr[c];
        const double* Yc = Yp(c);
        double* Lo = v.Lenv + (size_t)(c + 1) * env_sz;
        double mx = 0.0;
        for (int idx = threadIdx.x; idx < kk * xm; idx += blockDim.x) {
          const int j = idx / xm, x = idx % xm;
          double acc = 0.0;
          for (int q = 0; q < 2 * ay; ++q) acc += Yc[(size_t)q * kk + j] * v.T1[(size_t)q * xm + x];
          Lo[idx] = acc;
          mx = fmax(mx, fabs(acc));
        }
        mx = block_max(mx, sh.red);
        if (!(mx > 0.0) || !isfinite(mx)) {
          if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
          mx = 1.0;
        }
        const double inv = 1.0 / mx;
        for (int idx = threadIdx.x; idx < kk * xm; idx += blockDim.x) Lo[idx] *= inv;
        __syncthreads();
      }
    }
    for (int c = Lx - 2; c >= 0; --c) {
      const int ay = sh.dl[c], by = sh.dr[c + 1];
      const int kk = bond_dim_dev(a.chi, Lx, a.Ly, r, c + 1);
      var_theta(a, v, c, ay, by);
      var_split(a, sh, v, r, c, 2 * ay, 2 * by, kk, false, true, Yp(c), Yp(c + 1));
      if (threadIdx.x == 0) {
        sh.dr[c] = kk;
        sh.dl[c + 1] = kk;
      }
      __syncthreads();
      if (c > 0) {
        const double l = var_right_overlap(a, sh, Yp(c + 1), kk, sh.dr[c + 1], v.X + (size_t)(c + 1) * slot_sz,
                                           v.xdl[c + 1], v.xdr[c + 1], v.Renv + (size_t)(c + 2) * env_sz, v.T1,
                                           v.Renv + (size_t)(c + 1) * env_sz);
        if (threadIdx.x == 0) v.lR[c + 1] = v.lR[c + 2] + l;
        __syncthreads();
      }
    }
  }
  return v.lR[2];
}

__device__ void build_env_body(const BuildArgs& a, double* smem) {
  const int Lx = a.Lx, P = a.P;
  Shared sh;
  sh.W = smem;
  sh.red = smem + 6 * P * P + 4 * P;
  int* ip = reinterpret_cast<int*>(sh.red + 64);
  sh.slot = ip;
  sh.dl = ip + (Lx + 2);
  sh.dr = sh.dl + (Lx + 1);
  sh.sel = sh.dr + (Lx + 1);
  sh.flag = sh.sel + 2 * P;
  const size_t slot_sz = (size_t)8 * P * P;

  for (int r = a.Ly - 1; r >= 0; --r) {
    apply_row_mpo(a, sh, r);
    if (a.sweeps > 0) var_save_x(a, sh);
    double logs = qr_sweep(a, sh);
    logs += svd_sweep(a, sh, r);
    if (a.sweeps > 0 && Lx >= 2) logs = variational_sweeps(a, sh, r);
    // normalise site 0
    {
      const double* T0 = a.work + (size_t)sh.slot[0] * slot_sz;
      const int cnt = sh.dl[0] * 2 * sh.dr[0];
      double s = 0.0;
      for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) s += T0[idx] * T0[idx];
      s = block_sum(s, sh.red);
      const double n0 = sqrt(s);
      if (!(n0 > 0.0) || !isfinite(n0)) {
        if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
      }
      logs += log(n0);
      // write the row into the padded FP64 arena
      for (int c = 0; c < Lx; ++c) {
        const int Dl = sh.dl[c], Dr = sh.dr[c];
        const double* T = a.work + (size_t)sh.slot[c] * slot_sz;
        double* out = a.M64 + ((size_t)r * Lx + c) * P * 2 * P;
        const double scale = (c == 0) ? 1.0 / n0 : 1.0;
        for (int idx = threadIdx.x; idx < P * 2 * P; idx += blockDim.x) {
          const int b = idx % P, s2 = (idx / P) & 1, aa = idx / (2 * P);
          out[idx] = (aa < Dl && b < Dr) ? T[((size_t)aa * 2 + s2) * Dr + b] * scale : 0.0;
        }
        if (threadIdx.x == 0) {
          a.bond[r * (Lx + 1) + c] = Dl;
          if (Dl != bond_dim_dev(a.chi, Lx, a.Ly, r, c)) set_status(a.status, TNMC_E_NUMERIC);
        }
      }
      if (threadIdx.x == 0) {
        a.bond[r * (Lx + 1) + Lx] = 1;
        a.log_scale[r] = logs;
      }
    }
    __syncthreads();
  }
  // log Z~ = sum_r log_scale[r] + log sum_sigma env_0(sigma)  (row 0 has no field from above)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double* v = sh.W;          // [P]
    double* v2 = sh.W + P;     // [P]
    for (int i = lane; i < P; i += 32) v[i] = (i == 0) ? 1.0 : 0.0;
    __syncwarp();
    double logv = 0.0;
    for (int c = 0; c < Lx; ++c) {
      const double* M = a.M64 + (size_t)c * P * 2 * P;
      const int Dl = a.bond[c], Dr = a.bond[c + 1];
      double mx = 0.0;
      for (int b = lane; b < Dr; b += 32) {
        double acc = 0.0;
        for (int aa = 0; aa < Dl; ++aa) acc += v[aa] * (M[((size_t)aa * 2) * P + b] + M[((size_t)aa * 2 + 1) * P + b]);
        v2[b] = acc;
        mx = fmax(mx, fabs(acc));
      }
      mx = warp_max(mx);
      __syncwarp();
      for (int b = lane; b < P; b += 32) v[b] = (b < Dr && mx > 0.0) ? v2[b] / mx : 0.0;
      if (mx > 0.0) logv += log(mx);
      __syncwarp();
    }
    if (lane == 0) {
      double tot = 0.0;
      for (int r = 0; r < a.Ly; ++r) tot += a.log_scale[r];
      *a.logZ = (v[0] > 0.0) ? tot + logv + log(v[0]) : NAN;
    }
  }
}

// ===========================================================================
// Z2-symmetric builder (all fields h = 0).
//
// With h = 0 the Boltzmann weight is invariant under a global spin flip, so every
// environment is an even function of its row.  In the parity basis
// |0> = (|-1> + |+1>)/sqrt2, |1> = (|-1> - |+1>)/sqrt2 of each site the vertical
// transfer exp(beta J s s') is diagonal (2 cosh, 2 sinh), a horizontal bond is
// cosh I(x)I + sinh X(x)X (X flips the parity), and every bond index carries a
// parity.  Each site matrix of the QR sweep and of the SVD sweep is then block
// diagonal with one block per parity sector; the sectors are factored separately
// (the SVD blocks are half the size of the dense ones, a quarter of the Jacobi
// work) and the chi largest singular values are kept across both sectors.  The
// truncated MPS is the dense algorithm's up to gauge.  Bonds store their even
// sector first: index i of a bond with e even states has parity (i >= e).
// The finished row is written back in the spin basis.
// ===========================================================================

struct ShZ2 {
  double* W;
  int* slot;     // [Lx + 2]
  int* bdim;     // [Lx + 1] dimension of bond c
  int* bev;      // [Lx + 1] even-sector size of bond c
  int* sel;      // [2P] kept rows by global rank
  int* sec;      // [2P] scratch: (sector, rank within sector) per kept row
  double* red;
  int* flag;
};

// position of (a, k) in a doubled bond built from a bond of size D with e even states
__device__ inline int dbl_idx(int a, int k, int D, int e) {
  const bool odd = a >= e;
  if (k == 0) return odd ? D + (a - e) : a;
  return odd ? a : D + (D - e) + a;
}
__device__ inline void dbl_inv(int l, int D, int e, int& a, int& k) {
  if (l < D) {
    a = l;
    k = (l < e) ? 0 : 1;
  } else {
    const int j = l - D;
    if (j < D - e) { a = e + j; k = 0; }
    else { a = j - (D - e); k = 1; }
  }
}

__device__ void apply_row_mpo_z2(const BuildArgs& a, ShZ2& sh, int r) {
  const int Lx = a.Lx, P = a.P;
  const size_t slot_sz = (size_t)8 * P * P;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double isq2 = 0.70710678118654752440;
  for (int c = w; c < Lx; c += kWarps) {
    const bool last_row = (r == a.Ly - 1);
    const int Dl0 = last_row ? 1 : a.bond[(r + 1) * (Lx + 1) + c];
    const int Dr0 = last_row ? 1 : a.bond[(r + 1) * (Lx + 1) + c + 1];
    const int el0 = last_row ? 1 : a.esz[(r + 1) * (Lx + 1) + c];
    const int er0 = last_row ? 1 : a.esz[(r + 1) * (Lx + 1) + c + 1];
    const bool kl = c > 0, kr = c < Lx - 1;
    const int Dl = kl ? 2 * Dl0 : Dl0, Dr = kr ? 2 * Dr0 : Dr0;
    double lam0 = 1.0, lam1 = 1.0, w0 = 1.0, w1 = 0.0;
    if (!last_row) {
      const double jv = a.Jv[r * Lx + c];
      lam0 = exp(a.beta * jv) + exp(-a.beta * jv);
      lam1 = exp(a.beta * jv) - exp(-a.beta * jv);
    }
    if (kr) {
      const double jh = a.Jh[r * (Lx - 1) + c];
      w0 = 0.5 * (exp(a.beta * jh) + exp(-a.beta * jh));
      w1 = 0.5 * (exp(a.beta * jh) - exp(-a.beta * jh));
    }
    const double* Mn = last_row ? nullptr : a.M64 + ((size_t)(r + 1) * Lx + c) * P * 2 * P;
    double* out = a.work + (size_t)c * slot_sz;
    const int total = Dl * 2 * Dr;
    for (int idx = lane; idx < total; idx += 32) {
      const int rr = idx % Dr, tau = (idx / Dr) & 1, l = idx / (2 * Dr);
      int aa = l, kin = 0, b = rr, kout = 0;
      if (kl) dbl_inv(l, Dl0, el0, aa, kin);
      if (kr) dbl_inv(rr, Dr0, er0, b, kout);
      const int tp = tau ^ kin ^ kout;   // X^(kin + kout) acting on the site
      double n;
      if (last_row) {
        n = (tp == 0) ? 1.4142135623730950488 : 0.0;
      } else {
        const double m0 = Mn[((size_t)aa * 2 + 0) * P + b];
        const double m1 = Mn[((size_t)aa * 2 + 1) * P + b];
        n = (tp == 0) ? lam0 * (m0 + m1) * isq2 : lam1 * (m0 - m1) * isq2;
      }
      out[idx] = kr ? (kout ? w1 : w0) * n : n;
    }
    if (lane == 0) {
      sh.slot[c] = c;
      sh.bdim[c] = Dl;
      sh.bev[c] = kl ? Dl0 : el0;
      if (c == Lx - 1) {
        sh.bdim[Lx] = Dr;
        sh.bev[Lx] = er0;
      }
    }
  }
  if (threadIdx.x == 0) {
    sh.slot[Lx] = Lx;
    sh.slot[Lx + 1] = Lx + 1;
  }
  __syncthreads();
}

__device__ double qr_sweep_z2(const BuildArgs& a, ShZ2& sh) {
  const int Lx = a.Lx, P = a.P;
  const size_t slot_sz = (size_t)8 * P * P;
  double logs = 0.0;
  double* A = sh.W;
  double* Q = sh.W + 2 * P * P;
  double* Rb = sh.W + 4 * P * P;
  double* tau = sh.W + 6 * P * P;
  double* diag = tau + P;
  for (int c = 0; c < Lx - 1; ++c) {
    const int Dl = sh.bdim[c], el = sh.bev[c], Dr = sh.bdim[c + 1], er = sh.bev[c + 1];
    const int n0 = er, n1 = Dr - er;
    const int k0 = min(Dl, n0), k1 = min(Dl, n1), K = k0 + k1;
    const double* X = a.work + (size_t)sh.slot[c] * slot_sz;
    double* Tn = a.work + (size_t)sh.slot[Lx] * slot_sz;   // new site c: [Dl][2][K]
    for (int idx = threadIdx.x; idx < Dl * 2 * K; idx += blockDim.x) Tn[idx] = 0.0;
    __syncthreads();
    for (int s = 0; s < 2; ++s) {
      const int ns = s ? n1 : n0, col0 = s ? er : 0, ks = s ? k1 : k0, j0 = s ? k0 : 0;
      if (ns == 0) continue;
      for (int idx = threadIdx.x; idx < Dl * ns; idx += blockDim.x) {
        const int j = idx / Dl, l = idx % Dl;
        const int tl = s ^ (l >= el ? 1 : 0);
        A[idx] = X[((size_t)l * 2 + tl) * Dr + col0 + j];
      }
      __syncthreads();
      householder_qr(A, Dl, ns, Q, Rb + s * P * P, tau, diag);
      __syncthreads();
      for (int idx = threadIdx.x; idx < Dl * ks; idx += blockDim.x) {
        const int j = idx / Dl, l = idx % Dl;
        const int tl = s ^ (l >= el ? 1 : 0);
        Tn[((size_t)l * 2 + tl) * K + j0 + j] = Q[j * Dl + l];
      }
      __syncthreads();
    }
    double mx = 0.0;
    for (int idx = threadIdx.x; idx < k0 * n0; idx += blockDim.x) mx = fmax(mx, fabs(Rb[idx]));
    for (int idx = threadIdx.x; idx < k1 * n1; idx += blockDim.x) mx = fmax(mx, fabs(Rb[P * P + idx]));
    mx = block_max(mx, sh.red);
    if (!(mx > 0.0) || !isfinite(mx)) {
      if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
      mx = 1.0;
    }
    logs += log(mx);
    const double inv = 1.0 / mx;
    const double* O = a.work + (size_t)sh.slot[c + 1] * slot_sz;
    double* Nn = a.work + (size_t)sh.slot[Lx + 1] * slot_sz;
    const int ncol = 2 * sh.bdim[c + 2 > Lx ? Lx : c + 2];   // (tau, x) of site c+1
    for (int idx = threadIdx.x; idx < K * ncol; idx += blockDim.x) {
      const int jp = idx / ncol, col = idx % ncol;
      const int s = jp >= k0 ? 1 : 0;
      const int j = s ? jp - k0 : jp;
      const int ns = s ? n1 : n0, col0 = s ? er : 0;
      const double* Rk = Rb + s * P * P + j * ns;
      double acc = 0.0;
      for (int i = j; i < ns; ++i) acc += Rk[i] * O[(size_t)(col0 + i) * ncol + col];
      Nn[idx] = acc * inv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = sh.slot[c];
      sh.slot[c] = sh.slot[Lx];
      sh.slot[Lx] = t;
      t = sh.slot[c + 1];
      sh.slot[c + 1] = sh.slot[Lx + 1];
      sh.slot[Lx + 1] = t;
      sh.bdim[c + 1] = K;
      sh.bev[c + 1] = k0;
    }
    __syncthreads();
  }
  return logs;
}

// column j of parity block s of a site matrix with right bond (Dr, er): (tau, x)
__device__ inline int z2_col(int s, int j, int Dr, int er) {
  const int ns0 = s ? Dr - er : er;              // tau = 0 part: x in sector s
  if (j < ns0) return (s ? er : 0) + j;           // tau = 0
  return Dr + (s ? 0 : er) + (j - ns0);           // tau = 1, x in sector 1 - s
}

// Both parity sectors of a site at once: the first half of the threads orthogonalises
// the m0 rows of J0, the second half the m1 rows of J1 (m0, m1 <= 64; same n, ld), each
// with the rounds, tolerances and arithmetic of jacobi_rows (blockDim.x / 64 lanes per
// pair, a power of two).  Sweeps continue until neither
// sector rotates; a converged sector's extra sweep rotates nothing.
__device__ bool jacobi_rows2(double* J0, int m0, double* J1, int m1, int n, int ld, double* d0, double* d1,
                             int* flag) {
  const int half = blockDim.x >> 1;          // threads per sector
  const int sec = threadIdx.x >= half;
  const int lt = threadIdx.x - sec * half;
  double* J = sec ? J1 : J0;
  double* d = sec ? d1 : d0;
  const int m = sec ? m1 : m0;
  const int N = m + (m & 1);
  const int npairs = N / 2;
  const int Nmax = max(m0 + (m0 & 1), m1 + (m1 & 1));
  const int L = half / 32;                   // lanes per pair: all 32 pairs of a round at once
  const int grp = lt / L, gl = lt % L;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    for (int i = lt; i < m; i += half) {
      double s = 0.0;
      for (int x = 0; x < n; ++x) s += J[(size_t)i * ld + x] * J[(size_t)i * ld + x];
      d[i] = s;
    }
    if (threadIdx.x == 0) {
      flag[0] = 0;
      flag[2] = 0;
    }
    __syncthreads();
    double dmax = 0.0;
    for (int i = 0; i < m; ++i) dmax = fmax(dmax, d[i]);
    const double dnull = kNullRel * kNullRel * dmax;
    for (int t = 0; t < Nmax - 1; ++t) {
      {
        // groups beyond this sector's pairs (or rounds) only contribute zeros to the shuffles
        int p = m, q = m;
        if (grp < npairs && t < N - 1) tournament(t, grp, N, p, q);
        const bool live = p < m && q < m;
        double ga = 0.0;
        double* rp = J + (size_t)(live ? p : 0) * ld;
        double* rq = J + (size_t)(live ? q : 0) * ld;
        if (live)
          for (int x = gl; x < n; x += L) ga += rp[x] * rq[x];
        for (int o = 1; o < L; o <<= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        if (live) {
          const double al = d[p], be = d[q];
          if (ga != 0.0 && al > dnull && be > dnull && ga * ga > kJacobiTol * kJacobiTol * al * be) {
            float zeta = (float)(be - al) / (2.0f * (float)ga);
            if (!isfinite(zeta)) zeta = (float)((be - al) / (2.0 * ga));
            float tf;
            if (fabsf(zeta) > 1e18f) tf = 0.5f / zeta;
            else tf = (zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
            const double tt = (double)tf;
            const double x = fma(tt, tt, 1.0);
            double cs = (double)rsqrtf((float)x);
            cs = cs * fma(-0.5 * x, cs * cs, 1.5);
            cs = cs * fma(-0.5 * x, cs * cs, 1.5);
            const double sn = cs * tt;
            for (int xx = gl; xx < n; xx += L) {
              const double u = rp[xx], v = rq[xx];
              rp[xx] = cs * u - sn * v;
              rq[xx] = sn * u + cs * v;
            }
            if (gl == 0) {
              const double c2 = cs * cs;
              d[p] = c2 * fma(tt * tt, be, fma(-2.0 * tt, ga, al));
              d[q] = c2 * fma(tt * tt, al, fma(2.0 * tt, ga, be));
              flag[2 * sec] = 1;
            }
          }
        }
      }
      __syncthreads();
    }
    const int rotated = flag[0] | flag[2];
    __syncthreads();
    if (!rotated) return true;
  }
  return false;
}

__device__ double svd_sweep_z2(const BuildArgs& a, ShZ2& sh, int r) {
  const int Lx = a.Lx, P = a.P;
  const size_t slot_sz = (size_t)8 * P * P;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double logs = 0.0;
  for (int c = Lx - 1; c >= 1; --c) {
    const int Dl = sh.bdim[c], el = sh.bev[c], Dr = sh.bdim[c + 1], er = sh.bev[c + 1];
    const int n = Dr;                 // columns of each parity block
    const int ld = n + 1;
    double* J = sh.W;                 // [Dl][ld]: sector-0 rows, then sector-1 rows
    double* US = sh.W + 4 * P * P + 2 * P;
    double* nrm = sh.W + 6 * P * P + 2 * P;
    const double* A = a.work + (size_t)sh.slot[c] * slot_sz;   // [Dl][2][Dr]
    const int kk = bond_dim_dev(a.chi, Lx, a.Ly, r, c);
    if (kk > Dl) {
      if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
      return logs;
    }
    for (int idx = threadIdx.x; idx < Dl * n; idx += blockDim.x) {
      const int l = idx / n, j = idx % n;
      const int s = l >= el ? 1 : 0;
      const int col = z2_col(s, j, Dr, er);     // tau * Dr + x
      J[l * ld + j] = A[(size_t)l * 2 * Dr + col];
    }
    __syncthreads();
    bool converged = true;
    if (el <= 64 && Dl - el <= 64) {
      converged = jacobi_rows2(J, el, J + (size_t)el * ld, Dl - el, n, ld, nrm, nrm + el, sh.flag);
    } else {
      if (el > 0) converged = jacobi_rows(J, el, n, ld, nrm, sh.flag);
      if (Dl - el > 0) converged = jacobi_rows(J + (size_t)el * ld, Dl - el, n, ld, nrm + el, sh.flag) && converged;
    }
    if (!converged && threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
    for (int i = w; i < Dl; i += kWarps) {
      double sq = 0.0;
      for (int x = lane; x < n; x += 32) sq += J[i * ld + x] * J[i * ld + x];
      sq = warp_sum(sq);
      if (lane == 0) nrm[i] = sqrt(sq);
    }
    __syncthreads();
    // global rank (descending norm, ties by index); kept rows listed sector by sector
    for (int i = threadIdx.x; i < Dl; i += blockDim.x) {
      int rank = 0, rs = 0;
      const double ni = nrm[i];
      const int si = i >= el;
      for (int j = 0; j < Dl; ++j) {
        const double nj = nrm[j];
        const int before = (nj > ni) || (nj == ni && j < i);
        rank += before;
        if (before && ((j >= el) == si)) ++rs;   // kept-candidates of the same sector ranked above
      }
      sh.sec[i] = (rank < kk) ? (si << 16 | rs) : -1;
      if (rank < kk) sh.sel[rank] = i;
    }
    __syncthreads();
    // sector counts of the kept rows
    if (threadIdx.x == 0) {
      int k0 = 0;
      for (int q = 0; q < kk; ++q) k0 += (sh.sel[q] < el);
      sh.flag[1] = k0;
    }
    __syncthreads();
    const int k0 = sh.flag[1];
    double tot = 0.0, dsc = 0.0;
    for (int i = threadIdx.x; i < Dl; i += blockDim.x) {
      tot += nrm[i] * nrm[i];
      if (sh.sec[i] < 0) dsc += nrm[i] * nrm[i];
    }
    tot = block_sum(tot, sh.red);
    dsc = block_sum(dsc, sh.red);
    const double smax = nrm[sh.sel[0]];
    if (!(smax > 0.0) || !isfinite(smax)) {
      if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
      return logs;
    }
    double* svr = a.sv + ((size_t)r * (Lx + 1) + c) * P;
    for (int j = threadIdx.x; j < P; j += blockDim.x) svr[j] = (j < kk) ? nrm[sh.sel[j]] / sqrt(tot) : 0.0;
    if (threadIdx.x == 0) a.disc[r * (Lx + 1) + c] = dsc / tot;
    // new site c: [kk][2][Dr]; kept row i of sector s with in-sector rank j sits at s ? k0 + j : j
    double* Vt = a.work + (size_t)sh.slot[Lx] * slot_sz;
    for (int idx = threadIdx.x; idx < kk * 2 * Dr; idx += blockDim.x) Vt[idx] = 0.0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < Dl * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      const int code = sh.sec[i];
      if (code < 0) continue;
      const int s = code >> 16, rs = code & 0xFFFF;
      const int row = s ? k0 + rs : rs;
      const double nv = nrm[i];
      Vt[(size_t)row * 2 * Dr + z2_col(s, j, Dr, er)] = (nv > kNullRel * smax) ? J[i * ld + j] / nv : 0.0;
    }
    __syncthreads();
    // kept rows at the rounding level stay zero rows (no weight; q unchanged)
    // US (Dl x kk, block diagonal) = A V / smax
    const double inv = 1.0 / smax;
    for (int idx = threadIdx.x; idx < Dl * kk; idx += blockDim.x) {
      const int i = idx / kk, jp = idx % kk;
      const int si = i >= el, sj = jp >= k0;
      double acc = 0.0;
      if (si == sj) {
        const double* Ar = A + (size_t)i * 2 * Dr;
        const double* Vr = Vt + (size_t)jp * 2 * Dr;
        for (int j = 0; j < n; ++j) {
          const int col = z2_col(si, j, Dr, er);
          acc += Ar[col] * Vr[col];
        }
      }
      US[idx] = acc * inv;
    }
    __syncthreads();
    logs += log(smax);
    // absorb into site c-1: rows (y, tau) of length Dl -> kk, block by block
    const double* O = a.work + (size_t)sh.slot[c - 1] * slot_sz;
    double* Nn = a.work + (size_t)sh.slot[Lx + 1] * slot_sz;
    const int rows = sh.bdim[c - 1] * 2;
    for (int idx = threadIdx.x; idx < rows * kk; idx += blockDim.x) {
      const int q = idx / kk, jp = idx % kk;
      const int sj = jp >= k0;
      const int i0 = sj ? el : 0, i1 = sj ? Dl : el;
      double acc = 0.0;
      for (int i = i0; i < i1; ++i) acc += O[(size_t)q * Dl + i] * US[i * kk + jp];
      Nn[idx] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = sh.slot[c];
      sh.slot[c] = sh.slot[Lx];
      sh.slot[Lx] = t;
      t = sh.slot[c - 1];
      sh.slot[c - 1] = sh.slot[Lx + 1];
      sh.slot[Lx + 1] = t;
      sh.bdim[c] = kk;
      sh.bev[c] = k0;
    }
    __syncthreads();
  }
  return logs;
}

__device__ void build_env_z2_body(const BuildArgs& a, double* smem) {
  const int Lx = a.Lx, P = a.P;
  ShZ2 sh;
  sh.W = smem;
  sh.red = smem + 6 * P * P + 4 * P;
  int* ip = reinterpret_cast<int*>(sh.red + 64);
  sh.slot = ip;
  sh.bdim = ip + (Lx + 2);
  sh.bev = sh.bdim + (Lx + 1);
  sh.sel = sh.bev + (Lx + 1);
  sh.sec = sh.sel + 2 * P;
  sh.flag = sh.sec + 2 * P;
  const size_t slot_sz = (size_t)8 * P * P;
  const double isq2 = 0.70710678118654752440;

  for (int r = a.Ly - 1; r >= 0; --r) {
    apply_row_mpo_z2(a, sh, r);
    double logs = qr_sweep_z2(a, sh);
    logs += svd_sweep_z2(a, sh, r);
    const double* T0 = a.work + (size_t)sh.slot[0] * slot_sz;
    const int cnt = sh.bdim[0] * 2 * sh.bdim[1];
    double sq = 0.0;
    for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) sq += T0[idx] * T0[idx];
    sq = block_sum(sq, sh.red);
    const double n0 = sqrt(sq);
    if (!(n0 > 0.0) || !isfinite(n0)) {
      if (threadIdx.x == 0) set_status(a.status, TNMC_E_NUMERIC);
    }
    logs += log(n0);
    // write the row in the spin basis: M[.][-1][.] = (T0 + T1)/sqrt2, M[.][+1][.] = (T0 - T1)/sqrt2
    for (int c = 0; c < Lx; ++c) {
      const int Dl = sh.bdim[c], Dr = sh.bdim[c + 1];
      const double* T = a.work + (size_t)sh.slot[c] * slot_sz;
      double* out = a.M64 + ((size_t)r * Lx + c) * P * 2 * P;
      const double scale = ((c == 0) ? 1.0 / n0 : 1.0) * isq2;
      for (int idx = threadIdx.x; idx < P * 2 * P; idx += blockDim.x) {
        const int b = idx % P, s2 = (idx / P) & 1, aa = idx / (2 * P);
        double v = 0.0;
        if (aa < Dl && b < Dr) {
          const double t0 = T[((size_t)aa * 2 + 0) * Dr + b], t1 = T[((size_t)aa * 2 + 1) * Dr + b];
          v = (s2 == 0 ? t0 + t1 : t0 - t1) * scale;
        }
        out[idx] = v;
      }
      if (threadIdx.x == 0) {
        a.bond[r * (Lx + 1) + c] = Dl;
        a.esz[r * (Lx + 1) + c] = sh.bev[c];
        if (Dl != bond_dim_dev(a.chi, Lx, a.Ly, r, c)) set_status(a.status, TNMC_E_NUMERIC);
      }
    }
    if (threadIdx.x == 0) {
      a.bond[r * (Lx + 1) + Lx] = 1;
      a.esz[r * (Lx + 1) + Lx] = 1;
      a.log_scale[r] = logs;
    }
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double* v = sh.W;
    double* v2 = sh.W + P;
    for (int i = lane; i < P; i += 32) v[i] = (i == 0) ? 1.0 : 0.0;
    __syncwarp();
    double logv = 0.0;
    for (int c = 0; c < Lx; ++c) {
      const double* M = a.M64 + (size_t)c * P * 2 * P;
      const int Dl = a.bond[c], Dr = a.bond[c + 1];
      double mx = 0.0;
      for (int b = lane; b < Dr; b += 32) {
        double acc = 0.0;
        for (int aa = 0; aa < Dl; ++aa) acc += v[aa] * (M[((size_t)aa * 2) * P + b] + M[((size_t)aa * 2 + 1) * P + b]);
        v2[b] = acc;
        mx = fmax(mx, fabs(acc));
      }
      mx = warp_max(mx);
      __syncwarp();
      for (int b = lane; b < P; b += 32) v[b] = (b < Dr && mx > 0.0) ? v2[b] / mx : 0.0;
      if (mx > 0.0) logv += log(mx);
      __syncwarp();
    }
    if (lane == 0) {
      double tot = 0.0;
      for (int r = 0; r < a.Ly; ++r) tot += a.log_scale[r];
      *a.logZ = (v[0] > 0.0) ? tot + logv + log(v[0]) : NAN;
    }
  }
}

__global__ void __launch_bounds__(kBuildThreads) build_env_kernel(BuildArgs a) {
  extern __shared__ double smem[];
  build_env_body(a, smem);
}
__global__ void __launch_bounds__(kBuildThreads) build_env_z2_kernel(BuildArgs a) {
  extern __shared__ double smem[];
  build_env_z2_body(a, smem);
}
// Many instances in one launch, one CTA each (independent problems).
__global__ void __launch_bounds__(kBuildThreads) build_env_batched_kernel(const BuildArgs* list) {
  extern __shared__ double smem[];
  const BuildArgs a = list[blockIdx.x];
  if (a.z2) build_env_z2_body(a, smem);
  else build_env_body(a, smem);
}

// Bond basis: the sampling tensors M'_r = D_r H_r V'_r env'_{r+1} of every row (the
// untruncated MPS of the row's spins, bond up to 2 chi), from the bond-basis boundary MPS
// env' the builder left in M64 (bond dims in `bond`), into `out` ([Ly][Lx][P][2][P], zero
// padded), and their bond dims into `nb`.  Same index layout as the builder's row MPO.
__global__ void bond_sampling_kernel(DeviceEnv d, const int32_t* bond, double* out, int32_t* nb) {
  const int Lx = d.Lx, Ly = d.Ly, P = d.P;
  const size_t per = (size_t)P * 2 * P;
  const size_t total = (size_t)Lx * Ly * per;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t t = i / per;
    const int rem = (int)(i % per);
    const int rr = rem % P, s = (rem / P) & 1, l = rem / (2 * P);
    const int r = (int)(t / Lx), c = (int)(t % Lx);
    const bool last_row = (r == Ly - 1);
    const int Dl0 = last_row ? 1 : bond[(r + 1) * (Lx + 1) + c];
    const int Dr0 = last_row ? 1 : bond[(r + 1) * (Lx + 1) + c + 1];
    const int kl = (c > 0) ? 2 : 1, kr = (c < Lx - 1) ? 2 : 1;
    const int Dl = Dl0 * kl, Dr = Dr0 * kr;
    if (rem == 0) {
      nb[r * (Lx + 1) + c] = Dl;
      if (c == Lx - 1) nb[r * (Lx + 1) + Lx] = 1;
    }
    double val = 0.0;
    if (l < Dl && rr < Dr) {
      int aa = l, k = 0, b = rr, kp = 0;
      if (kl == 2) { aa = l >> 1; k = l & 1; }
      if (kr == 2) { b = rr >> 1; kp = rr & 1; }
      if (kr == 1 || kp == s) {
        double n = 1.0;
        if (!last_row) {
          const double bj = d.beta * d.Jv[r * Lx + c];
          const double* Mn = d.M64 + ((size_t)(r + 1) * Lx + c) * per;
          n = split_B(bj, s, 0) * Mn[((size_t)aa * 2 + 0) * P + b] + split_B(bj, s, 1) * Mn[((size_t)aa * 2 + 1) * P + b];
        }
        const double hv = d.beta * d.h[r * Lx + c];
        val = n * exp(s ? hv : -hv);
        if (kl == 2) val *= exp(d.beta * d.Jh[r * (Lx - 1) + c - 1] * ((k == s) ? 1.0 : -1.0));
      }
    }
    out[i] = val;
  }
}

// log Z~ of the bond basis: sum_{r >= 1} log_scale[r] + log of the contraction of M'_0 over
// row 0's spins (one warp).
__global__ void bond_logz_kernel(DeviceEnv d, const double* log_scale, double* logZ) {
  const int lane = threadIdx.x, Lx = d.Lx, P = d.P;
  __shared__ double v[kMaxPad], v2[kMaxPad];
  for (int i = lane; i < P; i += 32) v[i] = (i == 0) ? 1.0 : 0.0;
  __syncwarp();
  double logv = 0.0;
  for (int c = 0; c < Lx; ++c) {
    const double* M = d.M64 + (size_t)c * P * 2 * P;
    const int Dl = d.bond[c], Dr = d.bond[c + 1];
    double mx = 0.0;
    for (int b = lane; b < Dr; b += 32) {
      double acc = 0.0;
      for (int aa = 0; aa < Dl; ++aa) acc += v[aa] * (M[((size_t)aa * 2) * P + b] + M[((size_t)aa * 2 + 1) * P + b]);
      v2[b] = acc;
      mx = fmax(mx, fabs(acc));
    }
    mx = warp_max(mx);
    __syncwarp();
    for (int b = lane; b < P; b += 32) v[b] = (b < Dr && mx > 0.0) ? v2[b] / mx : 0.0;
    if (mx > 0.0) logv += log(mx);
    __syncwarp();
  }
  if (lane == 0) {
    double tot = 0.0;
    for (int r = 1; r < d.Ly; ++r) tot += log_scale[r];
    *logZ = (v[0] > 0.0) ? tot + logv + log(v[0]) : NAN;
  }
}

}  // namespace
}  // namespace tnmc

tnmc_status tnmc_launch_bond_sampling(tnmc_env* env, cudaStream_t stream) {
  using namespace tnmc;
  DeviceEnv& d = env->d;
  const size_t bytes = (size_t)d.Lx * d.Ly * d.P * 2 * d.P * sizeof(double);
  const size_t bb = (size_t)d.Ly * (d.Lx + 1) * sizeof(int32_t);
  // R64 (derived later) is free scratch now; esz is unused by the dense builder
  bond_sampling_kernel<<<1024, 256, 0, stream>>>(d, d.bond, const_cast<double*>(d.R64), env->esz);
  TNMC_CUDA_TRY(cudaGetLastError());
  TNMC_CUDA_TRY(cudaMemcpyAsync(const_cast<double*>(d.M64), d.R64, bytes, cudaMemcpyDeviceToDevice, stream));
  TNMC_CUDA_TRY(cudaMemcpyAsync(const_cast<int32_t*>(d.bond), env->esz, bb, cudaMemcpyDeviceToDevice, stream));
  bond_logz_kernel<<<1, 32, 0, stream>>>(d, env->log_scale, env->logZ);
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

size_t tnmc_build_work_bytes(int Lx, int Ly, int P, int sweeps) {
  (void)Ly;
  const size_t base = (size_t)(Lx + 2) * 8 * P * P * sizeof(double);
  return sweeps > 0 ? base + tnmc::var_work_doubles(Lx, P) * sizeof(double) : base;
}

static size_t build_smem_bytes(int Lx, int P) {
  return (size_t)(6 * P * P + 4 * P + 64) * sizeof(double) + (size_t)(3 * Lx + 4 + 4 * P + 8) * sizeof(int);
}

static tnmc::BuildArgs make_build_args(tnmc_env* env, void* work) {
  using namespace tnmc;
  const DeviceEnv& d = env->d;
  BuildArgs a;
  a.Lx = d.Lx;
  a.Ly = d.Ly;
  a.chi = d.chi;
  a.P = d.P;
  a.beta = d.beta;
  a.Jh = d.Jh;
  a.Jv = d.Jv;
  a.h = d.h;
  a.M64 = const_cast<double*>(d.M64);
  a.bond = const_cast<int32_t*>(d.bond);
  a.log_scale = env->log_scale;
  a.sv = env->sv;
  a.disc = env->discarded;
  a.logZ = env->logZ;
  a.work = static_cast<double*>(work);
  a.status = d.status;
  a.esz = env->esz;
  a.z2 = d.z2;
  a.gauge = d.gauge;
  a.sweeps = d.sweeps;
  a.vw = d.sweeps > 0 ? a.work + (size_t)(d.Lx + 2) * 8 * d.P * d.P : nullptr;
  return a;
}

tnmc_status tnmc_launch_build(tnmc_env* env, cudaStream_t stream, void* work, size_t work_bytes) {
  using namespace tnmc;
  const DeviceEnv& d = env->d;
  if (work_bytes < tnmc_build_work_bytes(d.Lx, d.Ly, d.P, d.sweeps)) {
    tnmc_set_error("build scratch too small");
    return TNMC_E_INVALID_ARG;
  }
  BuildArgs a = make_build_args(env, work);
  const size_t smem = build_smem_bytes(d.Lx, d.P);
  int dev = 0, max_optin = 0;
  TNMC_CUDA_TRY(cudaGetDevice(&dev));
  TNMC_CUDA_TRY(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)max_optin) {
    tnmc_set_error("builder needs %zu bytes of shared memory (device allows %d): Lx too large", smem, max_optin);
    return TNMC_E_UNSUPPORTED;
  }
  if (d.z2) {
    TNMC_CUDA_TRY(cudaFuncSetAttribute(build_env_z2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    build_env_z2_kernel<<<1, kBuildThreads, smem, stream>>>(a);
  } else {
    TNMC_CUDA_TRY(cudaFuncSetAttribute(build_env_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    build_env_kernel<<<1, kBuildThreads, smem, stream>>>(a);
  }
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_launch_build_batched(tnmc_env* const* envs, int n, void* work, const size_t* work_offsets,
                                      void* args_dev, cudaStream_t stream) {
  using namespace tnmc;
  if (n <= 0) return TNMC_OK;
  BuildArgs* host = new (std::nothrow) BuildArgs[n];
  if (!host) {
    tnmc_set_error("host allocation failed");
    return TNMC_E_NOMEM;
  }
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    host[i] = make_build_args(envs[i], static_cast<char*>(work) + work_offsets[i]);
    const size_t si = build_smem_bytes(envs[i]->d.Lx, envs[i]->d.P);
    if (si > smem) smem = si;
  }
  int dev = 0, max_optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess && smem > (size_t)max_optin) {
    delete[] host;
    tnmc_set_error("builder needs %zu bytes of shared memory (device allows %d)", smem, max_optin);
    return TNMC_E_UNSUPPORTED;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(args_dev, host, sizeof(BuildArgs) * n, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // `host` is released below
  delete[] host;
  if (e != cudaSuccess) {
    tnmc_set_error("batched build setup failed: %s", cudaGetErrorString(e));
    return TNMC_E_CUDA;
  }
  TNMC_CUDA_TRY(cudaFuncSetAttribute(build_env_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  build_env_batched_kernel<<<n, kBuildThreads, smem, stream>>>(static_cast<const BuildArgs*>(args_dev));
  TNMC_CUDA_TRY(cudaGetLastError());
  return TNMC_OK;
}

size_t tnmc_build_args_bytes() { return sizeof(tnmc::BuildArgs); }
