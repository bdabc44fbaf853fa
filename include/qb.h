/*
 * qb.h -- C ABI of the GB300 fixed-precision randomized QB library.
 *
 * The library computes A ~= Q B with Q (m x rank) orthonormal, B = Q^T A (rank x n), and picks the
 * rank adaptively so that ||A - QB||_F < eps, using the error indicator of Theorem 1:
 * E = ||A||_F^2 - sum_i ||B_i||_F^2 (Algorithm 1), updated row by row (Sect. 3.1).
 * Two generators of the blocks Q_i, B_i are offered (Yu, Gu, Li, arXiv:1606.09402):
 *   randQB_EI  (Algorithm 2): per block, sketch A Omega_i, project against Q, orthonormalise,
 *              re-orthogonalise, B_i = Q_i^T A.  2 + 2P passes over A per block.
 *   randQB_FP  (Algorithm 4): G = A Omega and H = A^T G for l~ columns, then the blocked loop
 *              builds Q, B from G, H, Omega only (the re-orthogonalised B_i formula of
 *              Sect. 4.2).  Remark 4.2 forms G and H in one read of a row-major A; this library
 *              forms them in two kernels, each reading A once, so a batch (or chunk, see
 *              QB_FLAG_WHOLE_BATCH) costs 2 + 2P reads of A where Table 1 counts 1 + 2P.
 *              qb_info.passes counts every read.
 *
 * Conventions shared by every entry point
 *   - All matrix pointers are DEVICE pointers unless stated otherwise; the caller owns every
 *     buffer (A, Q, B, workspace).  The library never allocates device memory.
 *   - Dense A is row-major: element (i, j) at a[i * ld + j], ld >= n.
 *   - Q is column-major m x rank_cap: element (i, j) at Q[i + j * ldq], ldq >= m.
 *   - B is row-major rank_cap x n:    element (i, j) at B[i * ldb + j], ldb >= n.
 *   - Q and B are double when opts.prec == QB_PREC_FP64 and float when QB_PREC_MIXED.
 *   - Work is ordered on the given CUDA stream (a cudaStream_t passed as void*, NULL = legacy
 *     default stream).  The tolerance test needs E on the host once per block, so the call
 *     synchronises that stream once per block and returns after all its work has completed.
 *   - Omega is defined by opts.seed alone: Omega(j, c) is a Philox4x32-10 Box-Muller normal of
 *     row j and global column c (block i of EI and batch q of FP address the same columns).
 *   - Return value: negative = error, no valid output; 0 = converged; positive = valid output with
 *     a warning (QB_NOT_CONVERGED: rank cap or Omega budget reached first, Q and B hold the
 *     valid partial factorisation of info->rank columns; QB_WARN_TOL_FLOOR: the tolerance is
 *     below the Theorem 3 floor sqrt(4 u / 0.01) ||A||_F, so E may be less accurate than 1%;
 *     u = 2^-53 on the float64 path, 2^-24 on the mixed path, where Q and B are float32).
 *   - Mixed path stopping rule: E < eps^2 - 2 u ||A||_F^2 (u = 2^-24).  The margin covers the
 *     rounding of ||B||^2 that Theorem 3 bounds and, for B = Q^T A, the term
 *     tr(B^T (Q^T Q - I) B) by which a float32 Q moves the true error away from E (measured
 *     0.7 u ||A||_F^2 on the 40000 x 20000 benchmark); the tests check ||A - QB||_F < eps on
 *     every mixed result.  The batched path adds that term to E itself.
 */
#ifndef GB300_QB_H
#define GB300_QB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QB_OK = 0,
    QB_NOT_CONVERGED = 1,
    QB_WARN_TOL_FLOOR = 2,
    QB_ERR_INVALID_ARG = -1,
    QB_ERR_NONFINITE = -2,   /* A holds NaN or Inf */
    QB_ERR_CUDA = -3,        /* a CUDA call failed; qb_last_cuda_error() names it */
    QB_ERR_BREAKDOWN = -4,   /* reserved: panel factorisation produced non-finite values */
    QB_ERR_WORKSPACE = -5,   /* ws_bytes below the matching *_workspace() query */
    QB_ERR_TIMEOUT = -6,     /* a bounded device-side wait ran out (tensor-core pipelines, grid
                                barriers of the fused CholeskyQR, the batched graph) */
    QB_ERR_UNSUPPORTED = -7  /* dtype / precision combination not provided */
} qb_status;

/* status_bits in qb_info */
#define QB_BIT_BREAKDOWN 1      /* a Cholesky pivot fell below the breakdown threshold and was clamped */
#define QB_BIT_TOL_FLOOR 2      /* tolerance below the Theorem 3 floor */
#define QB_BIT_NOT_CONVERGED 4  /* rank cap reached before E < eps^2 */

typedef enum { QB_F64 = 0, QB_F32 = 1, QB_BF16 = 2, QB_BF16X2 = 3 } qb_dtype;

typedef enum {
    QB_PREC_FP64 = 0,  /* every step in float64 (A must be QB_F64 or CSR float64) */
    QB_PREC_MIXED = 1  /* BF16 tensor-core passes over A, float32 Q/B, float64 indicator,
                          float64 b x b Cholesky and triangular inverse */
} qb_prec;

/* Dense row-major A.  dtype QB_BF16X2 stores A = a_hi + a_lo as two bf16 arrays with the same
 * ld (see qb_quantize_bf16x2); sketch passes read a_hi only, the passes that form B_i (EI) or
 * H (FP) read both.  src_norm2 = ||A_src||_F^2 of the float64 source the bf16 arrays were made
 * from; pass a NaN to have the library compute ||A||_F^2 from the stored A.
 * a_lo_ready: NULL, or a cudaEvent_t (as void*) recorded after the last write of a_lo on another
 * stream.  The call makes its stream wait on the event right before its first read of a_lo, so
 * a_lo may still be arriving (a host-to-device copy on a second stream) while the sketches of
 * randQB_FP's power scheme run on a_hi.  Ignored by the batched path. */
typedef struct {
    int64_t m, n, ld;
    int32_t dtype;
    int32_t reserved;
    const void* a;
    const void* a_lo;
    double src_norm2;
    const void* a_lo_ready;
} qb_dense;

/* CSR A: rowptr[m+1], colind[nnz] (int32, zero-based, any order inside a row), val[nnz] of
 * dtype QB_F64 or QB_F32. */
typedef struct {
    int64_t m, n, nnz;
    const int32_t* rowptr;
    const int32_t* colind;
    int32_t dtype;
    int32_t reserved;
    const void* val;
} qb_csr;

typedef struct {
    double tol;          /* eps (absolute) or eps / ||A||_F when relative != 0 (Sect. 5.4) */
    int32_t relative;    /* nonzero: eps = tol * ||A||_F */
    int32_t b;           /* block size, 1 <= b <= 64 */
    int32_t P;           /* power parameter, 0 <= P <= 8 */
    int32_t row_by_row;  /* nonzero: stop at the row of B_i that meets the tolerance (Sect. 3.1) */
    uint64_t seed;       /* Omega seed (Philox key) */
    int64_t rank_cap;    /* capacity of Q and B in columns/rows; <= 0 means min(m, n) */
    int64_t l_tilde;     /* FP only: Omega batch width; <= 0 means 50 b (Sect. 5.4) */
    int32_t prec;        /* qb_prec */
    int32_t flags;       /* QB_FLAG_* bits, 0 by default */
} qb_opts;

/* qb_opts.flags: run the passes over a bf16 A on the SIMT kernels instead of the tensor cores
 * (float32 FMA on the same bf16 data; slower, used to cross-check the tensor-core kernels). */
#define QB_FLAG_SIMT_APASS 1
/* qb_opts.flags: record CUDA events around the phases of the call (adds a synchronisation at the
 * end); read the device milliseconds with qb_profile_last(). */
#define QB_FLAG_PROFILE 2
/* qb_opts.flags (randQB_FP): form each Omega batch of l~ columns in one go as Algorithm 4 is
 * written: 1 + 2P reads of A for the power scheme and G, plus one read per 512-column piece of
 * H (formed as the blocked loop reaches it).  By default the batch is formed in chunks of 512
 * columns as the blocked loop reaches them (P <= 1): the same Q and B up to rounding (orth is
 * column-causal), the columns after the stopping block are never formed, at 2 + 2P reads of A per
 * chunk.  With P > 1 the batch is always formed in one go. */
#define QB_FLAG_WHOLE_BATCH 4

typedef struct {
    int64_t rank;        /* columns of Q / rows of B that are valid */
    double err2_est;     /* E at exit (may be slightly negative through rounding) */
    double err_est;      /* sqrt(max(E, 0)) */
    double normA2;       /* ||A||_F^2 used by the indicator */
    int64_t passes;      /* reads of A by the kernels (Table 1's unit; G and H count two) */
    int64_t omega_cols;  /* global Omega columns drawn */
    int32_t status_bits; /* QB_BIT_* */
    int32_t blocks;      /* blocks of the loop that ran */
    int64_t launches;    /* kernels launched by this call */
} qb_info;

/* Human-readable name of a qb_status value. Never NULL. */
const char* qb_status_str(int32_t status);

/* Name of the last CUDA error seen by the library in this process ("" if none). */
const char* qb_last_cuda_error(void);

/* Total kernels launched by the library in this process (all calls). */
int64_t qb_launch_count(void);

/* Device milliseconds per phase of the last call made with QB_FLAG_PROFILE (or of the last
 * qb_apass_sketch / qb_apass_trans call, which always records its pass), in this order:
 * 0 Omega generation, 1 sketch passes over A (A X), 2 transposed passes over A (A^T X),
 * 3 power-scheme orthonormalisation, 4 projections against Q and B, 5 CholeskyQR2 of the new
 * block (with its re-orthogonalisation), 6 randQB_FP's B_i formula, 7 indicator and host
 * round trip.  Writes min(n, phases) values; returns the number of phases. */
int32_t qb_profile_last(double* ms, int32_t n);

/* ---------------------------------------------------------------------------------------------
 * Dense fixed-precision QB.  algo: 0 = randQB_EI (Algorithm 2), 1 = randQB_FP (Algorithm 4).
 * Workspace: bytes needed for (A shape, opts, algo); returns 0 on invalid arguments.
 * Q: ldq >= m, capacity rank_cap columns; B: ldb >= n, capacity rank_cap rows.
 * ------------------------------------------------------------------------------------------- */
size_t qb_dense_workspace(const qb_dense* A, const qb_opts* opts, int32_t algo);

/* randQB_EI, Algorithm 2 with the row-by-row stop of Sect. 3.1 and, for P > 0, the power
 * scheme applied per block to the implicit residual A - QB. */
int32_t qb_ei_dense(const qb_dense* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                    int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream);

/* randQB_FP, Algorithm 4 (power scheme on the whole Omega batch, G = A Omega and H = A^T G,
 * blocked loop with the re-orthogonalised B_i of Sect. 4.2).  When l~ columns do not
 * reach the tolerance the next batch of l~ global Omega columns is drawn (Sect. 4.3), its power
 * iterations act on the implicit residual, and the loop continues with the same Q, B. */
int32_t qb_fp_dense(const qb_dense* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                    int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Sparse CSR A (the sparse experiments of Sect. 5.1).  Same semantics as the dense calls; the
 * workspace holds a CSC copy of A built on the device for the A^T products.
 * ------------------------------------------------------------------------------------------- */
size_t qb_csr_workspace(const qb_csr* A, const qb_opts* opts, int32_t algo);
int32_t qb_ei_csr(const qb_csr* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                  int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream);
int32_t qb_fp_csr(const qb_csr* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                  int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Sparse COO A (Sect. 5.1: a coordinate-format copy of the sparse matrix lets randQB_FP spread
 * its work more evenly than CSR).  Triplets (row[e], col[e], val[e]), e < nnz, int32 zero-based
 * indices, val of dtype QB_F64 or QB_F32; each (row, col) at most once (||A||_F^2 is the sum of
 * val^2); any order is accepted and entries sorted by row are fastest.  The passes give every warp the same number of nonzeros whatever
 * the row and column lengths; A^T products run on a column-sorted copy the call builds in its
 * workspace.  Same semantics, outputs and statuses as the dense and CSR calls.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    int64_t m, n, nnz;
    const int32_t* row;
    const int32_t* col;
    int32_t dtype;
    int32_t reserved;
    const void* val;
} qb_coo;

size_t qb_coo_workspace(const qb_coo* A, const qb_opts* opts, int32_t algo);
int32_t qb_ei_coo(const qb_coo* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                  int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream);
int32_t qb_fp_coo(const qb_coo* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                  int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Single passes over dense A (the hot step of both algorithms, exposed for measurement and
 * verification).  Same kernels the drivers use; float64 A runs the float64 kernels, bf16 / bf16x2
 * A the tensor-core kernels (float32 V and outputs).
 *   qb_apass_sketch: Y (m x w, column-major, ldy) = A V, V n x w column-major (ldv)
 *                    (G = A Omega of Algorithm 4, A Omega_i of Algorithm 2); a bf16x2 A is read
 *                    through its hi part only.
 *   qb_apass_trans:  Z (n x w, column-major, ldz) = A^T V, V m x w column-major (ldv)
 *                    (H = A^T G of Algorithm 4, B_i^T = A^T Q_i of Algorithm 2).  For a bf16x2 A:
 *                    precise = 0: A_hi^T bf16(V) (sketch precision);
 *                    precise = 1: (A_hi + A_lo)^T V, V split exactly into three bf16 terms;
 *                    precise = 2: (A_hi + A_lo)^T bf16(V);
 *                    precise = 3: (A_hi + A_lo)^T (V_hi + V_lo), V_hi = bf16(V),
 *                                 V_lo = bf16(V - V_hi) (exact for V with 16 significant bits).
 *                    With precise != 0 the leading product A_hi^T V_hi is summed per MMA in
 *                    float32 registers with round-to-nearest (the precision the indicator
 *                    needs; a single tensor-core accumulation chain would bias it toward zero).
 *                    Float64 A ignores precise.
 * Workspace: qb_apass_workspace(A, w) bytes.
 * ------------------------------------------------------------------------------------------- */
size_t qb_apass_workspace(const qb_dense* A, int64_t w);
int32_t qb_apass_sketch(const qb_dense* A, const void* V, int64_t ldv, int64_t w, void* Y,
                        int64_t ldy, void* ws, size_t ws_bytes, void* stream);
int32_t qb_apass_trans(const qb_dense* A, const void* V, int64_t ldv, int64_t w, int32_t precise,
                       void* Z, int64_t ldz, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Batched randQB_EI (Algorithm 2 with P = 0 and the row-by-row stop) over `count` independent
 * float32 matrices of any shapes, each with its own tolerance tols[t] (relative when
 * opts->relative) and Omega seed opts->seed + t.  Every stage of one iteration is a single launch
 * over all matrices still running; the iteration is captured in a CUDA graph whose conditional
 * WHILE node repeats it until every matrix has converged or reached its rank cap (matrices that
 * finish early drop out of the work lists).  Requirements: opts->b == 16, opts->P == 0,
 * opts->prec == QB_PREC_MIXED, As[t].dtype == QB_F32.  As, tols, Qs, ldqs, Bs, ldbs, infos are
 * HOST arrays of `count` entries (the matrices they point to live on the device): Q_t is
 * column-major m_t x cap_t (ldqs[t] >= m_t), B_t row-major cap_t x n_t (ldbs[t] >= n_t),
 * cap_t = min(m_t, n_t, rank_cap).  Q and B are float32; the indicator is float64 and the stop
 * test keeps the 2 u ||A_t||^2 margin of the mixed path.  infos[t] receives each result; the
 * return value is the worst status over the batch.  Synchronises the stream.  Calls that share a
 * workspace must not overlap (the kept graph of a call reads the workspace it was captured on).
 * ------------------------------------------------------------------------------------------- */
size_t qb_ei_batched_workspace(int32_t count, const qb_dense* As, const qb_opts* opts);
/* Launch plan of the batched call's two A-streaming stages (the sketch Y = A Omega and the pass
 * B_i = Y^T A): tile shape and grid size.  The first call that meets a batch-shape bucket (log2
 * of the count, of the mean m and of the mean n) times every candidate on its own matrices (tile
 * shapes 64 / 128 rows per sketch tile and 64 / 128 columns per B tile, 4 / 8 / 16 CTAs per SM;
 * both stages are pure functions of their inputs, so the extra runs change no result) and keeps
 * the fastest of each stage for the bucket; later calls reuse it.  The iteration graph of a call
 * is kept (up to 4, keyed by workspace address, shapes, plan, seed and stop rule) and relaunched
 * by a later call with the same key instead of being captured again.
 *   qb_batched_set_plan(cfg): cfg = {rows per thread (1|2), columns per thread (1|2), sketch
 *     CTAs per SM, B-pass CTAs per SM} pins the plan for later calls; NULL returns to the tuner.
 *   qb_batched_last_plan(out, n): the last call's {rows per thread, columns per thread, sketch
 *     grid, B-pass grid, 1 if it tuned, 1 if it reused a graph, tuner cache entries}; returns 7.
 * The tile shape changes no summation order: results are identical under every plan. */
int32_t qb_batched_set_plan(const int32_t* cfg);
int32_t qb_batched_last_plan(int32_t* out, int32_t n);
int32_t qb_ei_batched(int32_t count, const qb_dense* As, const double* tols,
                      const qb_opts* opts, void* const* Qs, const int64_t* ldqs,
                      void* const* Bs, const int64_t* ldbs, void* ws, size_t ws_bytes,
                      qb_info* infos, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Fixed-rank QB map and its adjoint (reverse-mode derivative; the paper has no adjoint, the map
 * is k columns of randQB / randQB_EI / randQB_FP at P = 0 by Proposition 2).
 *   forward:  Omega = the Philox columns 0..k-1 of seed (bf16-rounded on the mixed path),
 *             Y = A Omega, Y = Q R with diag(R) > 0, B = Q^T A.
 *             Q column-major m x k (ldq), B row-major k x n (ldb), R column-major k x k upper (ldr).
 *   backward: for L with dL/dQ = G_Q (column-major m x k) and dL/dB = G_B (row-major k x n),
 *             dL/dA (row-major m x n, ldga) = Q G_B + Ybar Omega^T, where
 *             Qbar = G_Q + A G_B^T, M = -Qbar^T Q, Ybar = (Qbar + Q (tril(M) + tril(M,-1)^T)) R^-T;
 *             Y is not stored: Omega is regenerated from the seed.
 *   prec QB_PREC_FP64 (float64 A and buffers) or QB_PREC_MIXED (bf16 / bf16x2 A, float32
 *   buffers, tensor-core sketch, round-to-nearest B pass).  1 <= k <= min(m, n).
 *   The QR of Y is blocked over panels of 64 columns: each panel is projected twice against the
 *   finished ones, then orthonormalised by CholeskyQR2.  On the mixed path the projections run on
 *   the tensor cores against three-term bf16 copies of the finished panels (float32 accuracy;
 *   the workspace holds them), and a panel's diagonal block of R is the float32 inverse of the
 *   product of its two CholeskyQR factors' inverses.
 *   Both calls synchronise the stream before returning.
 * ------------------------------------------------------------------------------------------- */
size_t qb_fixed_rank_workspace(const qb_dense* A, int64_t k, int32_t prec);
int32_t qb_fixed_rank_fwd(const qb_dense* A, int64_t k, uint64_t seed, int32_t prec, void* Q,
                          int64_t ldq, void* B, int64_t ldb, void* R, int64_t ldr, void* ws,
                          size_t ws_bytes, void* stream);
int32_t qb_fixed_rank_bwd(const qb_dense* A, int64_t k, uint64_t seed, int32_t prec,
                          const void* Q, int64_t ldq, const void* R, int64_t ldr, const void* GQ,
                          int64_t ldgq, const void* GB, int64_t ldgb, void* GA, int64_t ldga,
                          void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------------
 * SVD from a QB factorisation (Sect. 2, the approximate SVD A ~ Q B = (Q U~) S~ V~^T): the SVD of
 * the small k x n B, B = U~ S~ V~^T, then U = Q U~.  The first columns of U, V and the leading
 * entries of S approximate A's singular triplets; with randQB_FP at P = 0 (Algorithm 3: G and H
 * from the same Omega, which the paper forms in one sweep over a row-major A and this library
 * in two reads) this is the single-pass SVD of Sect. 5.3.
 *   Q: m x k column-major (ldq >= m), B: k x n row-major (ldb >= n), both float64 (prec
 *   QB_PREC_FP64) or float32 (QB_PREC_MIXED): the outputs of qb_*_dense / qb_*_csr.
 *   S: k doubles (device), descending, S[j] = sqrt(lambda_j) of W = B B^T (float64).
 *   U: m x k column-major (ldu), V: n x k column-major (ldv), in Q's type; either may be NULL.
 * Method: W = B B^T (float64 sums; float32 B with exact products in float32-pair sums), cyclic
 * Jacobi eigendecomposition of W in float64 (one cooperative launch, bounded barrier waits), V =
 * B^T U~ S~^-1 (zero columns where S~ = 0).  Singular values are accurate to about
 * u (s_1 / s_j)^2 relative (W squares the condition number).  1 <= k <= min(m, n, 4096).
 * Workspace: qb_svd_workspace(m, n, k, prec) bytes.  Returns QB_OK, QB_NOT_CONVERGED (40 Jacobi
 * sweeps did not settle; S, U, V hold the last iterate), QB_ERR_TIMEOUT or another error; *sweeps
 * (nullable, host) receives the sweeps run.  Synchronises the stream.
 * ------------------------------------------------------------------------------------------- */
size_t qb_svd_workspace(int64_t m, int64_t n, int64_t k, int32_t prec);
int32_t qb_svd_from_qb(int64_t m, int64_t n, int64_t k, int32_t prec, const void* Q, int64_t ldq,
                       const void* B, int64_t ldb, double* S, void* U, int64_t ldu, void* V,
                       int64_t ldv, void* ws, size_t ws_bytes, int32_t* sweeps, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Allocation-free sketch pass (no counterpart in the paper; a deployment convenience).
 * Y (m x w, column-major, float32, ldy) = A_hi V, V float32 column-major n x w (ldv), A a
 * bf16 or bf16x2 dense A with ld % 8 == 0 and a 16-byte aligned base, m, n >= 128: the same
 * tensor-core kernel as qb_apass_sketch, for callers that can neither allocate device memory nor
 * pass a workspace (a process whose device memory is entirely carved up by its own pool, a plug-in
 * that must not call the device allocator).  Its scratch is one 16 MiB file-scope device array
 * that every GPU loading the library reserves until exit.  Limits: w <= 64, and the bf16 copy of
 * V (align8(n) * w * 2 bytes, rounded up to 256) plus 10 MiB + 256 bytes of partial tiles and
 * flag must fit in the 16 MiB, so n <= 49144 at w = 64.  Larger calls return QB_ERR_WORKSPACE
 * before anything is launched.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) and keeps it.  All calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race.  Every call ends by
 * copying the kernel's timeout flag to the host and synchronising the stream, so it returns
 * only after its work has completed.
 * ------------------------------------------------------------------------------------------- */
int32_t qb_apass_sketch_noalloc(const qb_dense* A, const float* V, int64_t ldv, int64_t w,
                                float* Y, int64_t ldy, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Omega generator (exposed for verification).  Writes Omega rows 0..n-1, global columns
 * col0..col0+w-1 column-major into out (ld >= n), dtype QB_F64 (float64 Box-Muller on 53-bit
 * uniforms), QB_F32 (float32 Box-Muller on 24-bit uniforms) or QB_BF16 (the QB_F32 value
 * rounded to nearest even).
 * ------------------------------------------------------------------------------------------- */
int32_t qb_omega(int64_t n, int64_t col0, int64_t w, uint64_t seed, int32_t dtype, void* out,
                 int64_t ld, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Quantisation of a float64 row-major source into bf16 hi + lo arrays (A = hi + lo to ~2^-17
 * relative per entry), with the float64 norms the mixed path needs:
 *   norms[0] = ||A_src||_F^2, norms[1] = ||A_src - hi - lo||_F^2, norms[2] = ||A_src - hi||_F^2.
 * norms is a HOST pointer (3 doubles); the call synchronises the stream.  ws must hold
 * qb_quantize_workspace() bytes.
 * ------------------------------------------------------------------------------------------- */
size_t qb_quantize_workspace(int64_t m, int64_t n);
int32_t qb_quantize_bf16x2(const double* src, int64_t m, int64_t n, int64_t ld_src, void* hi,
                           void* lo, int64_t ld, double* norms, void* ws, size_t ws_bytes,
                           void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_QB_H */
