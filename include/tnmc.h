/*
 * tnmc.h -- C ABI of libtnmc.so, the GB300 (sm_103a) path of the TNMH method of
 * Frias-Perez, Marien, Perez-Garcia, Banuls, Iblisdir, "Collective Monte Carlo
 * updates through tensor network renormalization" (arXiv:2104.13264).
 *
 * Conventions shared by every entry point
 *   - Lattice Ly x Lx with open boundaries; site (r, c), row r = 0 first;
 *     site index r*Lx + c.  Spins are int8 -1/+1, layout [sample][Ly][Lx].
 *   - Couplings (eq. ising):  H = -sum h s - sum J s s with
 *       Jh [Ly][Lx-1] bond (r,c)-(r,c+1),  Jv [Ly-1][Lx] bond (r,c)-(r+1,c),
 *       h  [Ly][Lx]   field; all row-major FP64.
 *   - Every call returns a tnmc_status.  Argument errors are reported
 *     synchronously (nothing is launched); tnmc_last_error() then returns a
 *     thread-local message.  No C++ exception crosses the ABI.
 *   - Device pointers are caller-owned (for instance torch tensors'
 *     data_ptr()), host pointers are read before the call returns.  Work is
 *     enqueued on `stream` (a cudaStream_t; NULL = legacy default stream).
 *   - A tnmc_env is opaque and library-owned; free it with tnmc_env_free.
 *     Calls that use one env share its device scratch, so they must be
 *     ordered on one stream (calls that overlap on the GPU race).
 *   - Numerical trouble found on the device (a non-positive or non-finite
 *     conditional normaliser, a zero environment) is reported per sample in
 *     `flags` and in the env's status word, read with tnmc_env_status.  A flagged
 *     sample keeps a finite log q (the probability it was drawn with) and takes part
 *     in MH like any other; it contributes nothing to tnmc_logq_backward.
 *   - Random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     the 64-bit seed; counters:
 *       draw of (site, sample) (site/2, sample_lo, sample_hi, 0), words
 *           (0,1) for even sites, (2,3) for odd ones, as x = lo | hi << 32;
 *           spin = +1 iff x < floor(p_+ 2^64)  (always when p_+ >= 1);
 *       MH uniform of proposal t of chain i  (t_lo, t_hi, i, 1), words (0,1),
 *           u = (x >> 11) 2^-53;
 *       random start of chain i  (site/128, i_lo, i_hi, 2), bit site % 128.
 */
#ifndef TNMC_H
#define TNMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TNMC_OK = 0,
  TNMC_E_INVALID_ARG = 1,
  TNMC_E_NOMEM = 2,
  TNMC_E_CUDA = 3,
  TNMC_E_NUMERIC = 4,
  TNMC_E_TIMEOUT = 5,
  TNMC_E_UNSUPPORTED = 6
} tnmc_status;

/* Arithmetic of the sampler copy of the environment (the builder is always FP64). */
typedef enum { TNMC_F64 = 0, TNMC_F32 = 1, TNMC_BF16 = 2 } tnmc_precision;

/* Site order of the samplers (defines q; App. A's labelling of the sites is not fixed by
 * the text).  Raster: every row left to right.  Snake: even rows left to right, odd rows
 * right to left. */
typedef enum { TNMC_ORDER_RASTER = 0, TNMC_ORDER_SNAKE = 1 } tnmc_order;

/* Per-sample flag bits. */
#define TNMC_FLAG_NUMERIC 1

typedef struct tnmc_env tnmc_env;
typedef struct tnmc_batch tnmc_batch;

typedef struct {
  int Lx, Ly;
  const double* Jh; /* host [Ly][Lx-1] */
  const double* Jv; /* host [Ly-1][Lx] */
  const double* h;  /* host [Ly][Lx]   */
} tnmc_lattice;

typedef struct {
  int Lx, Ly, chi;
  int pad;                /* P: padded bond stride of every stored tensor          */
  int precision_mask;     /* bit (1 << p) set when the sampler copy p is present   */
  int integer_couplings;  /* 1 when every J and h is an integer                    */
  double beta;
  double logZ;            /* log Z~ of the truncated contraction                   */
  int64_t bytes;          /* device bytes held by the env                          */
} tnmc_env_info_t;

typedef struct {
  int n;                   /* instances                                           */
  int precision;           /* TNMC_F64 or TNMC_F32                                */
  int tile;                /* samples per work item (64 or 128)                   */
  int order;               /* 0 instance order, 1 longest instance first          */
  int grid;                /* CTAs of the persistent launch                       */
  int64_t chains;          /* chains per instance C                               */
  int64_t proposal_rows;   /* sum_i B_i                                           */
  int64_t proposal_bytes;  /* sum_i B_i Lx_i Ly_i (the proposal spin arena)       */
  int64_t chain_rows;      /* n C                                                 */
  int64_t chain_bytes;     /* sum_i C Lx_i Ly_i (the chain spin arena)            */
  int64_t items;           /* work items of one proposal launch                   */
  int64_t smem_bytes;      /* dynamic shared memory per CTA                       */
  int64_t scratch_bytes;   /* device bytes of the per-CTA right-vector stacks     */
} tnmc_batch_info_t;

/*
 * Device-memory hook.  Every device allocation the library makes (environment
 * arenas, sampler and gradient scratch, builder work space, batch plans, the MH
 * scan's temporary) goes through alloc_fn / free_fn, so that a caller's allocator
 * (for instance PyTorch's caching allocator) can own the memory.  alloc_fn returns
 * a device pointer of at least `bytes` bytes, usable in stream order on `stream`
 * (a cudaStream_t, possibly NULL), or NULL on failure; free_fn releases a pointer
 * it returned (`stream` is the stream of the last use, or NULL once the device has
 * been synchronised).  Objects keep the hook that was current when they were
 * created and free through it.  Passing NULL, NULL restores the default
 * (cudaMallocAsync / cudaFreeAsync).  Set it before creating objects, from one
 * thread; it applies process-wide.  The paper has no counterpart: this is plumbing
 * for callers that manage device memory themselves.
 */
typedef void* (*tnmc_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*tnmc_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
tnmc_status tnmc_set_allocator(tnmc_alloc_fn alloc_fn, tnmc_free_fn free_fn, void* ctx);

/* Thread-local text of the last error (empty string if none). */
const char* tnmc_last_error(void);

/*
 * Build the chi-truncated boundary-MPS row environments of one instance in
 * FP64 on the GPU (App. A, eq. braket-top-tm-bot; "successive SVD").
 *   env_{Ly-1} is row Ly-1's exact weight; for r < Ly-1
 *   env_r = T_chi[ D_r H_r V_r env_{r+1} ]:  V_r sums row r+1 with the
 *   vertical bond weights, D_r applies the fields, H_r the horizontal bonds
 *   (a bond-2 copy MPO), T_chi is a left-to-right Householder QR sweep then a
 *   right-to-left one-sided Jacobi SVD sweep keeping
 *   chi_c = min(chi, 2^c, 2^(Lx-c), 2^(Ly-r)) values per bond.  When every
 *   field is zero the sweeps run block by block in the Z2 parity basis (same
 *   truncation up to gauge).  One CTA builds the whole instance: the row
 *   sweeps are sequential, and the cost is bound by the FP64 pipe of one SM
 *   (about 9.5 min for 256 x 256 at chi = 64).
 * lat         host lattice (Lx, Ly >= 1; Jh, Jv may be NULL when their size is 0)
 * beta        inverse temperature, finite, >= 0
 * chi         1 <= chi <= 64
 * precision_mask  bit (1 << TNMC_F64 | 1 << TNMC_F32 | 1 << TNMC_BF16): which
 *             sampler copies to derive (FP64 is always kept)
 * out         receives the new env (device memory allocated here)
 * Asynchronous on `stream`; tnmc_env_info / tnmc_env_export synchronise it.
 */
tnmc_status tnmc_build_env(const tnmc_lattice* lat, double beta, int chi, int precision_mask,
                           void* stream, tnmc_env** out);

/*
 * The same environments in the paper's bond-basis gauge (App. A, eqs. pf_bond_description
 * to pf_vertex_description), a builder variant that defines another q.  Each vertical bond
 * weight is split as W = B T by its SVD (W = sum_rho lambda_rho u_rho u_rho^T with
 * u_0 = (1,1)/sqrt 2, u_1 = (1,-1)/sqrt 2, index 0 <-> s = -1, lambda = 2 cosh, 2 sinh of
 * beta J; B[s][rho] = u_rho(s) sqrt|lambda_rho|, T[rho][s] = sign(lambda_rho) sqrt|lambda_rho|
 * u_rho(s)), and the boundary MPS carries the vertical bond index rho:
 *   env'_r = T_chi[ T_{r-1} D_r H_r V'_r env'_{r+1} ]   (V' applies B; T_{r-1} the upper factor
 *   of the bonds above row r, on the physical leg, before truncating),
 * while row r is sampled from the untruncated M'_r = D_r H_r V'_r env'_{r+1}, an MPS of the
 * row's spins with bonds up to 2 chi (the rows above enter through the same field factors
 * f(s) = W(s_up, s)).  The samplers, MH and backward run on it unchanged.  log Z~ (env_info)
 * is this gauge's; log_scale, sv and discarded (env_export) describe the truncations of
 * env'_r for r >= 1 (row 0's entries are not used).  chi <= 32 (bonds up to 64); always the
 * dense (non-parity) builder.  Arguments as tnmc_build_env.
 */
tnmc_status tnmc_build_env_bond(const tnmc_lattice* lat, double beta, int chi, int precision_mask, void* stream,
                                tnmc_env** out);

/*
 * The same environments with each row compressed by two-site variational sweeps
 * (App. A names two-site variational compression beside successive SVD): a builder
 * variant that defines another q.  T_chi starts from the successive-SVD result; each of
 * `sweeps` rounds is a left-to-right and a right-to-left pass over the neighbour pairs
 * (c, c+1), replacing the pair by the truncated SVD of the two-site tensor that is
 * closest to the exact row D_r H_r V_r env_{r+1} with the other sites fixed (exact
 * overlap environments; bond dims as successive SVD).  No update increases the
 * 2-norm distance to the exact row.  sv / discarded (env_export) record each bond's last
 * update.  sweeps in [0, 64] (0 is tnmc_build_env); always the dense (non-parity)
 * builder.  Scratch: the builder's plus about (2 Lx) x 8 P^2 doubles.  Other arguments as
 * tnmc_build_env.
 */
tnmc_status tnmc_build_env_variational(const tnmc_lattice* lat, double beta, int chi, int sweeps, int precision_mask,
                                       void* stream, tnmc_env** out);

tnmc_status tnmc_env_free(tnmc_env* env);

/*
 * Site order of every later sample / logq / init_chains / metropolis call on this env (and
 * of batch plans created afterwards), TNMC_ORDER_RASTER (default) or TNMC_ORDER_SNAKE.  The
 * environments do not depend on the order.  In snake order an odd row r is drawn from
 * c = Lx-1 down to 0: a forward sweep V_{c+1} = sum_s f_c(s) V_c M_c[:, s, :] (sites < c
 * summed) is stored, then w(s) = f_c(s) <V_c M_c[:, s, :], Lambda'_{c+1}> with Lambda' the
 * drawn sites > c; draws, log q and energy otherwise as tnmc_sample (site r*Lx + c keeps its
 * Philox counter).  The BF16 tensor-core sampler and tnmc_logq_backward support raster
 * order only and return TNMC_E_UNSUPPORTED.  Not synchronised with work in flight: call it
 * between launches.
 */
tnmc_status tnmc_env_set_order(tnmc_env* env, int order);

/* Synchronises the env's build stream and fills `info`. */
tnmc_status tnmc_env_info(const tnmc_env* env, tnmc_env_info_t* info);

/*
 * Copy the FP64 environment to host memory (synchronous).  Any pointer may be NULL.
 * tensors    [Ly][Lx][P][2][P]  M^(r)_c[a][sigma][b], zero outside the bond dims
 * log_scale  [Ly]   log of the factor removed while building row r
 * sv         [Ly][Lx+1][P]  kept singular values at bond c divided by the 2-norm
 *                           of all singular values of that SVD step (0 elsewhere)
 * discarded  [Ly][Lx+1]     discarded squared-weight fraction at bond c
 * bond_dims  [Ly][Lx+1]     chi_c^(r)
 */
tnmc_status tnmc_env_export(const tnmc_env* env, double* tensors, double* log_scale, double* sv,
                            double* discarded, int32_t* bond_dims);

/* Synchronises and reads the env's device status word (0 = clean; else tnmc_status). */
tnmc_status tnmc_env_status(const tnmc_env* env, int32_t* status);

/*
 * Draw B independent proposals from q = pi~ (Sec. 2, eqs. bayes, pi-approx,
 * tns-prior): raster order, one site at a time, each conditional
 *   w(s) = f_c(s) <Lambda_c M_c[s], R_{c+1}>,  clamped at 0 and normalised,
 * with f_c(s) = exp(beta Jv[r-1][c] s_{r-1,c} s) (the rows above are a
 * product state, App. A).  Also returns the exact log q of each draw and its
 * energy H (eq. ising; exact integers when all couplings are integers).
 * precision   which sampler copy to use (must be present in the env)
 * B           number of proposals, >= 0; sample index of row b is sample_offset + b
 * spins       device int8 [B][Ly][Lx] (output)
 * logq        device double [B] (output).  A site whose normaliser w_+ + w_- is not
 *             positive or not finite is drawn with p_+ = 1/2 and contributes log 1/2;
 *             the sample is flagged, and its log q is still the log of the probability
 *             it was drawn with, so q is the exact law of the sampler.
 * energy      device double [B] (output)
 * flags       device int32 [B] or NULL (output; TNMC_FLAG_NUMERIC)
 * The first call on an env may allocate device scratch for the per-sample
 * right-vector stacks (grown, never shrunk, freed with the env).  FP64/FP32:
 * (Lx+1) * P * 64 * 8 or (Lx+1) * P * 128 * 4 bytes per resident CTA.  BF16
 * (tensor cores, chi <= 64): Lx * 32 KiB per resident CTA, e.g. 2.5 GB for
 * Lx = 256 on a 152-SM GPU; the BF16 path also reads the pre-swizzled operand
 * tiles derived at build time (64 KiB per site).
 */
tnmc_status tnmc_sample(const tnmc_env* env, int precision, int64_t B, uint64_t seed,
                        uint64_t sample_offset, int8_t* spins, double* logq, double* energy,
                        int32_t* flags, void* stream);

/*
 * tnmc_sample without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot let the library allocate -- code that
 * runs under a fixed device-memory budget owned by another allocator, and
 * latency-sensitive loops where an allocation, or the device-wide
 * synchronisation a cudaFree implies, is not acceptable.
 * Same arguments, arithmetic and outputs as tnmc_sample (precision TNMC_F64 or
 * TNMC_F32).  The per-sample right-vector stacks live in one fixed 64 MiB
 * static device array that every GPU loading the library holds until the
 * process exits; when the stacks of all CTAs do not fit, fewer CTAs run (slower,
 * same results).  A lattice whose single-CTA stack exceeds 64 MiB
 * ((Lx+1) * P * 64 * 8 bytes in FP64, (Lx+1) * P * 128 * 4 in FP32) is rejected
 * with TNMC_E_INVALID_ARG.  All calls on a device share the array: calls that
 * overlap on the GPU race, so order them on one stream.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make it before any stream capture.
 */
tnmc_status tnmc_sample_noalloc(const tnmc_env* env, int precision, int64_t B, uint64_t seed,
                                uint64_t sample_offset, int8_t* spins, double* logq, double* energy,
                                int32_t* flags, void* stream);

/*
 * Forced ("teacher") evaluation of log q and H for given configurations
 * (App. A, product of conditional ratios); same arithmetic as tnmc_sample.
 * spins       device int8 [B][Ly][Lx], values -1/+1 (input)
 */
tnmc_status tnmc_logq(const tnmc_env* env, int precision, int64_t B, const int8_t* spins,
                      double* logq, double* energy, int32_t* flags, void* stream);

/*
 * Random +-1 start of C chains (Algorithm 1, second step) with their forced
 * log q (sampler copy `precision`) and energy.
 */
tnmc_status tnmc_init_chains(const tnmc_env* env, int precision, int64_t C, uint64_t seed,
                             int8_t* chain_spins, double* chain_logq, double* chain_energy,
                             void* stream);

/*
 * Metropolis-Hastings scan (eq. mh-acc with g(w'|w) = q(w'), Algorithm 1):
 * chain i consumes proposals i*T .. i*T+T-1 in order.  For proposal t
 *   Delta = a_t - a_cur,  a = (-beta * E) - log q  (each operation rounded once),
 *   accept iff log q_t is finite and u < exp(min(0, Delta)),
 * u from the MH stream at step (step_offset + j).  A chain whose log q is -inf
 * (a random start outside q's support) takes its first valid proposal.  On exit
 * each chain holds its last accepted proposal (spins, log q, energy).  The
 * decisions are those of the FP64 rule, most of them taken by integer compares
 * against per-proposal bands computed beforehand.
 * prop_*      device [C*T] (spins [C*T][Ly][Lx])
 * chain_*     device [C] in/out (spins [C][Ly][Lx])
 * accepted    device uint8 [C*T] or NULL (output)
 * n_accepted  device int64 scalar or NULL; the number accepted is ADDED to it
 * Scratch: 24 C T + 8 C bytes from the env's allocator (TNMC_E_NOMEM if refused),
 * freed on the stream before return.
 */
tnmc_status tnmc_mh_step(const tnmc_env* env, int64_t C, int64_t T, const int8_t* prop_spins,
                         const double* prop_logq, const double* prop_energy, int8_t* chain_spins,
                         double* chain_logq, double* chain_energy, uint64_t seed,
                         uint64_t step_offset, uint8_t* accepted, int64_t* n_accepted,
                         void* stream);

/*
 * Single-spin-flip Metropolis sweeps of chain states, the moves the paper intersperses
 * between proposals (Sec. 3, "Equilibration"; Table hb: TNMH + Metropolis).  Each of
 * the C chains gets `sweeps` checkerboard sweeps: first the sites with (r + c) even,
 * then the odd ones, each updated against the current spins of the other colour.  Site
 * i flips iff u < exp(-beta dE), dE = 2 s_i (h_i + sum_j J_ij s_j) (eq. ising), with
 * u = (x >> 11) 2^-53 from Philox words (0, 1) of the counter (i, chain id, sweep, 5):
 * chain k has id (uint32)(chain_offset + k), and the sweeps are sweep_offset .. +sweeps-1
 * (low 32 bits).  The sweeps leave the Boltzmann distribution invariant, so a chain that
 * alternates them with tnmc_mh_step still samples pi exactly.  Afterwards the chains'
 * log q (sampler copy `precision`) and energy are recomputed, as tnmc_logq does, so the
 * next MH step sees consistent chain states.
 * chain_spins   device int8 [C][Ly][Lx], in/out;  chain_logq, chain_energy  device [C], out
 * The lattice must fit in shared memory (Lx * Ly <= 200 KiB).
 */
tnmc_status tnmc_metropolis(const tnmc_env* env, int precision, int64_t C, int8_t* chain_spins, double* chain_logq,
                            double* chain_energy, uint64_t seed, uint64_t chain_offset, uint64_t sweep_offset,
                            int sweeps, void* stream);

/*
 * Link overlap of replica pairs (Sec. 3, eq. Delta): for chains (2k, 2k + 1),
 *   overlap[k] = sum over the bonds <ij> of s_i^a s_j^a s_i^b s_j^b   (exact integers),
 * an estimate of sum_<ij> <s_i s_j>^2.  With the chains' mean energy it gives the
 * equilibration diagnostic (1/|V|)(<H> + beta (|E| - sum_<ij> <s_i s_j>^2)), whose
 * average over Gaussian disorder vanishes at equilibrium.
 * C even; chain_spins device int8 [C][Ly][Lx]; overlap device double [C / 2]
 */
tnmc_status tnmc_link_overlap(const tnmc_env* env, int64_t C, const int8_t* chain_spins, double* overlap,
                              void* stream);

/*
 * Gradient of sum_b weights[b] log q(spins[b]) with respect to every tensor of the
 * FP32 sampler copy (the parameters of tnmc_env_get_params), by reverse-mode
 * differentiation of the forced evaluation (Sec. 2, eq. pi-approx; App. A):
 * per-site normalised, clamped conditionals; the power-of-two rescalings are
 * constants.  The per-row forward vectors are recomputed, not stored.  Used to
 * tune the proposal (maximise the mean log q of accepted chain samples); the MH
 * step keeps the chain exact whatever q is.
 * spins    device int8 [B][Ly][Lx]
 * weights  device float [B]; samples whose log q is -inf must have weight 0
 * grad     device float, same layout as the parameters ([Ly][Lx][P][2][P]);
 *          overwritten.  Requires the TNMC_F32 copy and P <= 64 (64 samples per CTA above P = 52).
 */
tnmc_status tnmc_logq_backward(const tnmc_env* env, int64_t B, const int8_t* spins, const float* weights,
                               float* grad, void* stream);

/*
 * The FP32 sampler copy as a flat parameter vector: [Ly][Lx][P][2][P] floats,
 * M^(r)_c[a][s][b] zero-padded to P.  get copies it into `dst`; set copies `src`
 * into the env and re-derives the transposed copy the right sweep reads, so
 * tnmc_sample / tnmc_logq / tnmc_logq_backward with TNMC_F32 use the new tensors
 * (the FP64 master and the BF16 tiles keep the built values).  Device pointers,
 * asynchronous on `stream`.
 */
tnmc_status tnmc_env_get_params(const tnmc_env* env, float* dst, void* stream);
tnmc_status tnmc_env_set_params(tnmc_env* env, const float* src, void* stream);

/*
 * Replace the FP64 environment tensors M^(r)_c the samplers use, and re-derive every
 * sampler copy the env holds (FP64 transposed, FP32, BF16 operand tiles) from them.
 * The builder's other outputs (log Z~, log-scales, singular values) are kept.  Any
 * normalisation of the tensors gives a valid proposal: each conditional is
 * normalised by w_+ + w_- (Sec. 2, eq. pi-approx), so q sums to one whatever the
 * tensors are.  This serves environments made elsewhere (another compression of
 * App. A, a tuned FP64 set) and tests that run the samplers on given tensors.
 * src     [Ly][Lx][P][2][P] doubles, M^(r)_c[a][sigma][b], ZERO outside the bond
 *         dimensions chi_c^(r) x 2 x chi_{c+1}^(r) (P from tnmc_env_info); host or
 *         device memory (copied with cudaMemcpyAsync, kind default).
 * Asynchronous on `stream`; a host `src` must stay valid until the stream reaches
 * the copy.
 */
tnmc_status tnmc_env_set_tensors(tnmc_env* env, const double* src, void* stream);

/* ---------------------------------------------------------------------------
 * Batched persistent form: many independent instances (for instance disorder
 * realisations of uneven L and chi) in single launches.  Each instance follows
 * exactly the single-instance definitions above; batching changes only how the
 * work is scheduled.
 * ------------------------------------------------------------------------- */

/*
 * Build n instances' environments in ONE builder launch (one CTA per
 * instance), then derive their sampler copies.  Arguments are arrays of n
 * (lattices, betas, chis) with the meaning of tnmc_build_env; out[n] receives
 * the envs (free each with tnmc_env_free).  On error nothing is returned and
 * the message names the instance.
 */
tnmc_status tnmc_build_env_batched(int n, const tnmc_lattice* lats, const double* beta, const int* chi,
                                   int precision_mask, void* stream, tnmc_env** out);

/*
 * A plan over n built envs (which must outlive it): B[i] proposals per step
 * for instance i (a multiple of `chains`), `chains` Markov chains per instance
 * (chain c of instance i consumes proposals c*T_i .. c*T_i+T_i-1 of that
 * instance, T_i = B[i] / chains), sampler arithmetic `precision` (TNMC_F64 or
 * TNMC_F32; every env must hold that copy), `tile` samples per work item (64
 * or 128) and the item `order` (0: instance order; 1: instances with the
 * largest per-sample cost first).  Work items are (instance, tile) pairs taken
 * by a persistent grid from an atomic counter.  Allocates the plan's device
 * tables and per-CTA scratch; synchronises `stream` before returning.
 * Proposal arrays are concatenated by instance: instance i's proposals are rows
 * prop_row[i] .. prop_row[i]+B[i]-1 of logq / energy / flags and bytes
 * prop_spin[i] .. of the spin arena (layout [B_i][Ly_i][Lx_i]); chains
 * likewise (see tnmc_batch_layout).  A plan serves one stream at a time.
 */
tnmc_status tnmc_batch_create(int n, tnmc_env* const* envs, const int64_t* B, int64_t chains, int precision,
                              int tile, int order, void* stream, tnmc_batch** out);
tnmc_status tnmc_batch_free(tnmc_batch* plan);
tnmc_status tnmc_batch_info(const tnmc_batch* plan, tnmc_batch_info_t* info);

/* Host arrays [n] (any may be NULL): first proposal row, proposal spin byte
 * offset, first chain row (= i * chains), chain spin byte offset per instance. */
tnmc_status tnmc_batch_layout(const tnmc_batch* plan, int64_t* prop_row, int64_t* prop_spin,
                              int64_t* chain_row, int64_t* chain_spin);

/*
 * The plan's device-resident (seed, step k).  At step k instance i draws the
 * samples (i << 40) + k B_i + b, b < B_i (so its proposals equal tnmc_sample
 * with sample_offset (i << 40) + k B_i), and its MH scan uses step offsets
 * (i << 40) + k T_i (tnmc_mh_step's step_offset).  set writes both values;
 * advance adds 1 to k on the device, so a captured CUDA graph of
 * sample + mh + advance replays successive steps.
 */
/*
 * Load balance of the plan's last persistent sampling launch (proposals or chains):
 * every CTA records the global timer when it starts and when it finds no item left;
 * efficiency = sum over CTAs of their busy time / (grid x makespan), in (0, 1].
 * Synchronises the device.  makespan_ms may be NULL.
 */
tnmc_status tnmc_batch_balance(const tnmc_batch* plan, double* efficiency, double* makespan_ms);

tnmc_status tnmc_batch_set_step(tnmc_batch* plan, uint64_t seed, uint64_t step, void* stream);
tnmc_status tnmc_batch_advance(tnmc_batch* plan, void* stream);

/*
 * One persistent launch drawing every instance's B_i proposals (spins, exact
 * log q, exact energy, flags as tnmc_sample).  Issues no allocation and no
 * synchronisation, so it may be captured in a CUDA graph.
 * prop_spins  device int8, proposal_bytes (output); prop_logq / prop_energy
 * device double [proposal_rows]; flags device int32 [proposal_rows] or NULL.
 */
tnmc_status tnmc_sample_batched(tnmc_batch* plan, int8_t* prop_spins, double* prop_logq, double* prop_energy,
                                int32_t* flags, void* stream);

/* Forced evaluation (tnmc_logq) of a whole proposal arena in one persistent launch. */
tnmc_status tnmc_logq_batched(tnmc_batch* plan, const int8_t* prop_spins, double* prop_logq,
                              double* prop_energy, int32_t* flags, void* stream);

/*
 * Random +-1 start of every chain (Algorithm 1, second step): chain c of
 * instance i takes the random-start stream with chain id (i << 32) | c, then its
 * forced log q and energy.  chain_spins device int8 [chain_bytes];
 * chain_logq / chain_energy device double [chain_rows].
 */
tnmc_status tnmc_batch_init_chains(tnmc_batch* plan, uint64_t seed, int8_t* chain_spins, double* chain_logq,
                                   double* chain_energy, void* stream);

/*
 * The MH scan (eq. mh-acc, Algorithm 1) of every chain of every instance in
 * one launch, with the plan's (seed, step); per instance identical to
 * tnmc_mh_step(env_i, chains, T_i, ..., seed, (i << 40) + k T_i, ...).
 * accepted  device uint8 [proposal_rows] or NULL
 * n_accepted  device int64 [n] or NULL; instance i's count is ADDED to entry i
 */
tnmc_status tnmc_mh_batched(tnmc_batch* plan, const int8_t* prop_spins, const double* prop_logq,
                            const double* prop_energy, int8_t* chain_spins, double* chain_logq,
                            double* chain_energy, uint8_t* accepted, int64_t* n_accepted, void* stream);

/*
 * tnmc_metropolis for every chain of every instance in one launch, then the forced log q
 * and energy of the whole chain arena in one persistent launch.  At plan step k chain c of
 * instance i has chain id (uint32)(i * chains + c) and runs sweeps k * sweeps .. +sweeps-1
 * with the plan's seed: per instance identical to tnmc_metropolis(env_i, plan precision,
 * chains, ..., seed, i * chains, k * sweeps, sweeps).  Allocates nothing (capturable).
 */
tnmc_status tnmc_metropolis_batched(tnmc_batch* plan, int8_t* chain_spins, double* chain_logq, double* chain_energy,
                                    int sweeps, void* stream);

/*
 * tnmc_link_overlap of every instance's replica pairs: overlap [n][chains / 2] (device
 * double), instance-major; chains must be even.
 */
tnmc_status tnmc_link_overlap_batched(tnmc_batch* plan, const int8_t* chain_spins, double* overlap, void* stream);

/* ------------------------------------------------------------------------------------
 * Three-dimensional lattices (Sec. 3D; App. A, three-dimensional paragraph and Figs.
 * peps-cutoff2, peps-cutoff).
 *
 * Lattice Lz x Ly x Lx, open boundaries, site (z, y, x), index (z*Ly + y)*Lx + x; layer
 * z = 0 is sampled first, each layer in raster order.  Spins int8 [sample][Lz][Ly][Lx].
 * H = -sum h s - sum J s s with Jx [Lz][Ly][Lx-1] bond (z,y,x)-(z,y,x+1),
 * Jy [Lz][Ly-1][Lx] bond (z,y,x)-(z,y+1,x), Jz [Lz-1][Ly][Lx] bond (z,y,x)-(z+1,y,x),
 * h [Lz][Ly][Lx]; row-major FP64 host arrays.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  int Lx, Ly, Lz;
  const double* Jx;
  const double* Jy;
  const double* Jz;
  const double* h;
} tnmc_lattice3d;

typedef struct tnmc3d_env tnmc3d_env;

/*
 * Layer environments: PEPS of bond D over the spins of each layer, bottom-up,
 *   env_{Lz-1} = the exact weight of the last layer,
 *   env_z = T_D[ D_z H_z V_z env_{z+1} ]
 * (V_z: the sum over layer z+1 through exp(beta Jz s s'); D_z: fields; H_z: the in-layer
 * bonds as copy structure, each doubling its bond).  T_D is the paper's renormalisation
 * (Fig. peps-cutoff2): every column is read as an MPS with the column's vertical bonds as
 * MPS bonds and the spin and the two horizontal bonds as physical index, compressed by
 * successive SVD keeping min(D, rank bound) values per bond; then every row likewise
 * along its horizontal bonds.  `chi` is the boundary-MPS bond used by the sampler.
 * The build is synchronous.  Limits: Lx, Ly <= 64; D <= 8; chi <= 32; D chi <= 64.
 * Errors: TNMC_E_INVALID_ARG (arguments), TNMC_E_NOMEM, TNMC_E_CUDA; numerical trouble
 * (a zero column, a Jacobi SVD that does not converge) sets the env's status word.
 */
tnmc_status tnmc3d_build_env(const tnmc_lattice3d* lat, double beta, int D, int chi, void* stream, tnmc3d_env** out);
/*
 * The same in the bond basis (App. A: vertex tensors from split bond weights): each
 * vertical bond weight is split W = B T as in tnmc_build_env_bond, the layer PEPS carries
 * the index of the vertical bonds above it,
 *   env'_z = T_D[ T_{z-1} D_z H_z V'_z env'_{z+1} ]   (V' applies B),
 * and layer z is sampled from its uncompressed PEPS M'_z = D_z H_z V'_z env'_{z+1}
 * (in-layer bonds up to 2 D); the layer above enters through the same fields.  The
 * sampler, MH and forced evaluation run on it unchanged.  Limits as tnmc3d_build_env with
 * 2 D chi <= 64; env_export returns the sampling tensors, padded to 2 D.
 */
tnmc_status tnmc3d_build_env_bond(const tnmc_lattice3d* lat, double beta, int D, int chi, void* stream,
                                  tnmc3d_env** out);
tnmc_status tnmc3d_env_free(tnmc3d_env* env);
/* Synchronises and reads the status word (0 = clean; else a tnmc_status). */
tnmc_status tnmc3d_env_status(const tnmc3d_env* env, int32_t* status);
/*
 * Host copies (synchronous; any pointer may be NULL) of the tensors the sampler reads:
 * tensors [Lz][Ly][Lx][2][P][P][P][P] with P = D (tnmc3d_build_env) or 2 D (bond basis),
 * A[s][u][l][d][r] (u: bond to row y-1, l: to column x-1, d: to row y+1, r: to column
 * x+1; zero outside the dims), dims [Lz][Ly][Lx][4] = (du, dl, dd, dr), log_scale [Lz]
 * (log of the factor removed while compressing layer z).
 */
tnmc_status tnmc3d_env_export(const tnmc3d_env* env, double* tensors, int32_t* dims, double* log_scale);

/*
 * Draw B proposals from the 3D q.  Layer z is sampled with the spins of layer z-1 as
 * fields f(s) = exp(beta Jz s_up s); row y of the layer from the sandwich of Top_y (rows
 * < y at their drawn spins, an MPS of bond chi over the row's upper bonds) x row y x
 * Bot_y (rows > y summed, an MPS of bond chi over its lower bonds), both rebuilt for
 * every sample by successive SVD (Bot_y = T_chi[S_{y+1} Bot_{y+1}], S = sum_s A f;
 * Top_{y+1} = T_chi[Top_y F_y], F = A f at the drawn spins).  Site conditionals are
 * clamped at zero and normalised; sample b (index sample_offset + b) draws site i with
 * the Philox word of (i, sample) as in two dimensions.  Also returns the exact log q of
 * each draw (sum of the logs of the probabilities used) and its energy (FP64).  One
 * thread per sample; the samples' scratch (about 8 (L^2 chi^2 D + L (D chi)^2 D) bytes
 * each) is taken from the env's allocator in chunks of at most 4 GiB.
 * precision  TNMC_F64 or TNMC_F32 (the FP32 copy of the environment, FP32 arithmetic)
 * spins      device int8 [B][Lz][Ly][Lx] (output); logq, energy device double [B];
 * flags      device int32 [B] or NULL (TNMC_FLAG_NUMERIC: a site drawn at p = 1/2).
 */
tnmc_status tnmc3d_sample(const tnmc3d_env* env, int precision, int64_t B, uint64_t seed, uint64_t sample_offset,
                          int8_t* spins, double* logq, double* energy, int32_t* flags, void* stream);
/* Forced evaluation: log q and energy of given configurations (same arithmetic). */
tnmc_status tnmc3d_logq(const tnmc3d_env* env, int precision, int64_t B, const int8_t* spins, double* logq,
                        double* energy, int32_t* flags, void* stream);
/* Random +-1 start of C chains (counter as tnmc_init_chains) and their forced log q, energy. */
tnmc_status tnmc3d_init_chains(const tnmc3d_env* env, int precision, int64_t C, uint64_t seed, int8_t* chain_spins,
                               double* chain_logq, double* chain_energy, void* stream);
/* The MH scan of tnmc_mh_step on 3D configurations (n = Lz Ly Lx spins each). */
tnmc_status tnmc3d_mh_step(const tnmc3d_env* env, int64_t C, int64_t T, const int8_t* prop_spins,
                           const double* prop_logq, const double* prop_energy, int8_t* chain_spins,
                           double* chain_logq, double* chain_energy, uint64_t seed, uint64_t step_offset,
                           uint8_t* accepted, int64_t* n_accepted, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TNMC_H */
