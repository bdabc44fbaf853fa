// Internal declarations shared by the translation units of libqb.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <atomic>
#include <stdexcept>
#include <string>

#include "qb.h"

namespace qb {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------------------------ errors
struct Error {
    int32_t code;
    std::string what;
};

void record_cuda_error(cudaError_t e, const char* where);
void count_launch();
int64_t launches_total();

#define QB_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e__ = (call);                                            \
        if (e__ != cudaSuccess) {                                            \
            ::qb::record_cuda_error(e__, #call);                             \
            throw ::qb::Error{QB_ERR_CUDA, cudaGetErrorString(e__)};         \
        }                                                                    \
    } while (0)

#define QB_LAUNCHED()                                                        \
    do {                                                                     \
        ::qb::count_launch();                                                \
        cudaError_t e__ = cudaGetLastError();                                \
        if (e__ != cudaSuccess) {                                            \
            ::qb::record_cuda_error(e__, __func__);                          \
            throw ::qb::Error{QB_ERR_CUDA, cudaGetErrorString(e__)};         \
        }                                                                    \
    } while (0)

// Raise kernel KERN's dynamic shared-memory limit to `bytes`, once per device (the attribute
// outlives the call); later calls cost one cudaGetDevice.
template <auto KERN>
void smem_limit_once(size_t bytes) {
    static std::atomic<unsigned> done{0};   // bit d: set on device d (devices 0..31)
    int dev = 0;
    QB_CUDA(cudaGetDevice(&dev));
    const unsigned bit = dev < 32 ? 1u << dev : 0u;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return;
    QB_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(KERN),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
    done.fetch_or(bit, std::memory_order_relaxed);
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t align_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

int num_sms();

// ------------------------------------------------------------------------------------ workspace
// Bump allocator over the caller's workspace.  With base == nullptr it only measures.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    template <class T>
    T* get(int64_t count) {
        size_t off = (used + 255) & ~size_t(255);
        size_t bytes = size_t(count > 0 ? count : 1) * sizeof(T);
        used = off + bytes;
        if (base == nullptr) return nullptr;
        if (used > cap) throw Error{QB_ERR_WORKSPACE, "workspace too small"};
        return reinterpret_cast<T*>(base + off);
    }
};

// ------------------------------------------------------------------------------------ GEMM
// C (M x N, column-major, ldc) = alpha * op(X) * Y + beta * C, Y is K x N column-major (ldy).
//   xt == true : op(X) = X^T with X column-major K x M (ldx)   ("TN": both operands K-contiguous)
//   xt == false: op(X) = X   with X column-major M x K (ldx)   ("NN")
// Accumulation: ACC_D float64, ACC_F float32, ACC_DF float32 pair (exact products, ~48-bit sums).
// ACC_D: float64; ACC_F: float32; ACC_DF: float32 pair with exact products (~48 bits);
// ACC_F2: float32 per 16-step stage, stage sums into a float32 pair
enum Acc { ACC_D = 0, ACC_F = 1, ACC_DF = 2, ACC_F2 = 3 };
enum XKind { X_F64 = 0, X_F32 = 1, X_BF16 = 2, X_BF16X2 = 3 };

struct GemmScratch {
    void* part = nullptr;   // split-K partials
    size_t part_bytes = 0;
};

// X given as a typed pointer pair (lo only for X_BF16X2).
struct XOp {
    XKind kind;
    const void* p;
    const void* lo;
    int64_t ld;
};

void gemm(cudaStream_t st, bool xt, int64_t M, int64_t N, int64_t K, double alpha, XOp X,
          const void* Y, bool y_f64, int64_t ldy, double beta, void* C, bool c_f64, int64_t ldc,
          Acc acc, const GemmScratch& scr);
// W (MAXB x MAXB, symmetric, zero outside bi x bi) = P^T P for the rows x bi panel P (column-major,
// float64 when f64 else float32), bi <= MAXB; partials in scr
void gram(cudaStream_t st, const void* P, int64_t ldp, int64_t rows, int bi, bool f64, Acc acc,
          double* W, const GemmScratch& scr);
// bytes of split-K partial storage needed by gemm() for any (M, N) with M * N <= mn_max
size_t gemm_scratch_bytes(int64_t mn_max);
// Z (n x w, col-major) = (A_hi + A_lo)^T V in float32 with round-to-nearest sums (SIMT)
void trans_precise(cudaStream_t st, const bf16* Ahi, const bf16* Alo, int64_t lda, int64_t m,
                   int64_t n, const float* V, int64_t ldv, int64_t w, float* Z, int64_t ldz,
                   const GemmScratch& scr);

// ------------------------------------------------------------------------------------ tcgen05
// BF16 tensor-core passes over dense A (row-major m x n, bf16 hi [+ lo]).
//   sketch: Y (m x w, col-major, float) = A_hi * V, V given as bf16 column-major n x w
//   trans : Z (n x w, col-major, float) = A^T V with V float column-major m x w:
//           mode 1: A_hi^T bf16(V), float32 tensor-core accumulation (sketch precision);
//           mode 2: (A_hi [+ A_lo])^T bf16(V) (exact operand for bf16-valued V);
//           mode 3: (A_hi [+ A_lo])^T V with V = V_hi + V_mid + V_lo split exactly on the fly;
//           mode 4: (A_hi [+ A_lo])^T V for V holding two-term bf16 values (V = hi + lo exactly).
//           Modes 2-4 sum the leading product per MMA in registers (round-to-nearest).
bool tc_available();
// scratch layout starts with a 256-byte error area: word 0 is set when a bounded wait timed out
size_t tc_scratch_bytes(int64_t m, int64_t n, int64_t w);
int* tc_error_flag(void* scratch);
// Vt_lo (nullable): second bf16 operand; Y = A_hi (V_hi + V_lo) as two products
void tc_sketch(cudaStream_t st, const bf16* A, int64_t lda, int64_t m, int64_t n,
               const bf16* Vt, const bf16* Vt_lo, int64_t ldv, int64_t w, float* Y, int64_t ldy,
               void* scratch, size_t scratch_bytes);
// Tensor-core products with a column-major X held as bf16 hi [+ lo] (rows % 8 == 0):
//   tc_xtp:        T (j0 x bw) = X[:, :j0]^T P
//   tc_p_minus_xt: P (rows x bw) -= X[:, :j0] T
void tc_xtp(cudaStream_t st, const bf16* Xhi, const bf16* Xlo, int64_t ldx, int64_t rows,
            int64_t j0, const float* P, int64_t ldp, int64_t bw, float* T, int64_t ldt,
            void* scratch, size_t scratch_bytes);
void tc_p_minus_xt(cudaStream_t st, const bf16* Xhi, const bf16* Xlo, int64_t ldx, int64_t rows,
                   int64_t j0, const float* T, int64_t ldt, int64_t bw, float* P, int64_t ldp,
                   void* scratch, size_t scratch_bytes);
// V (rows x w float, col-major) -> bf16 hi (and lo = bf16(V - hi) when lo != nullptr)
void split_bf16(cudaStream_t st, const float* V, int64_t ldv, int64_t rows, int64_t w, bf16* hi,
                bf16* lo, int64_t ldo);
void tc_trans(cudaStream_t st, const bf16* A_hi, const bf16* A_lo, int64_t lda, int64_t m,
              int64_t n, const float* V, int64_t ldv, int64_t w, float* Z, int64_t ldz, int mode,
              void* scratch, size_t scratch_bytes);
// D (M x N <= 64, col-major) = alpha op(A) V + beta D on the tensor cores at float32 accuracy:
// A as na exact bf16 terms (trans = false: A row-major M x K; trans = true: A row-major K x M,
// op(A) = A^T), V float32 column-major K x N split exactly into three bf16 terms on the fly.
void tc_prec_gemm(cudaStream_t st, bool trans, const bf16* const* A, int na, int64_t lda,
                  int64_t M, int64_t K, const float* V, int64_t ldv, int64_t N, float alpha,
                  float beta, float* D, int64_t ldd, void* scratch, size_t scratch_bytes);
// The same with V = [V1 | V2] (two column blocks with their own ld, N1 + N2 <= 128): one pass
// over A's terms for both; the scratch must hold the split of K x (N1 + N2).
void tc_prec_gemm2(cudaStream_t st, bool trans, const bf16* const* A, int na, int64_t lda,
                   int64_t M, int64_t K, const float* V1, int64_t ldv1, int64_t N1,
                   const float* V2, int64_t ldv2, int64_t N2, float alpha, float beta, float* D,
                   int64_t ldd, void* scratch, size_t scratch_bytes);
// hi + mid + lo == X exactly (three bf16 terms of a float32 column-major block)
void split3_bf16(cudaStream_t st, const float* X, int64_t ldx, int64_t rows, int64_t cols, bf16* hi,
                 bf16* mid, bf16* lo, int64_t ldo);
// X <- bf16(X) (pairs 1) or bf16(X) + bf16(X - bf16(X)) (pairs 2), elementwise, in place
void round_bf16_inplace(cudaStream_t st, float* X, int64_t ldx, int64_t rows, int64_t cols,
                        int pairs);

// ------------------------------------------------------------------------------------ misc kernels
void omega_gen(cudaStream_t st, int64_t n, int64_t col0, int64_t w, uint64_t seed, int dtype,
               void* out, int64_t ld);
void to_bf16(cudaStream_t st, const float* X, int64_t ldx, int64_t rows, int64_t cols, bf16* Y,
             int64_t ldy);
// ||A||^2 of a dense row-major A; flags[0] |= 1 on a non-finite entry.  part: >= 1024 doubles
void dense_norm2(cudaStream_t st, XOp A, int64_t m, int64_t n, double* part, double* out,
                 int* flags);
void vec_norm2(cudaStream_t st, const void* v, bool f64, int64_t count, double* part,
               double* out, int* flags);
void quantize_bf16x2(cudaStream_t st, const double* src, int64_t m, int64_t n, int64_t lds,
                     bf16* hi, bf16* lo, int64_t ld, double* part, double* out3);
// copy a column-major rows x cols block (f64 or f32)
void copy_cols(cudaStream_t st, bool f64, const void* X, int64_t ldx, int64_t rows,
               int64_t cols, void* Y, int64_t ldy);
void fill_zero(cudaStream_t st, void* p, size_t bytes);
// Y (cols x rows) = X^T, column-major blocks
void transpose(cudaStream_t st, bool f64, const void* X, int64_t ldx, int64_t rows, int64_t cols,
               void* Y, int64_t ldy);
// hi (row-major, ld ldo) columns [off, off + cols) = bf16(X) of the float32 column-major rows x cols
// block X, row r of the output holding row r of X; lo = bf16(X - hi); either may be null
void pack_rows_bf16(cudaStream_t st, const float* X, int64_t ldx, int64_t rows, int64_t cols,
                    bf16* hi, bf16* lo, int64_t ldo, int64_t off);
// C = tril(M) + tril(M, -1)^T (k x k, ld k)
void copyltu(cudaStream_t st, bool f64, const void* M, int64_t k, void* C);
// Y = X converted from float64 (column-major blocks)
void from_f64(cudaStream_t st, bool f64, const double* X, int64_t ldx, int64_t rows, int64_t cols,
              void* Y, int64_t ldy);
// Y += alpha X (column-major blocks)
void axpy(cudaStream_t st, bool f64, int64_t rows, int64_t cols, double alpha, const void* X,
          int64_t ldx, void* Y, int64_t ldy);
// X = R^-1 for upper-triangular k x k R (any k)
void tri_inv_big(cudaStream_t st, bool f64, const void* R, int64_t ldr, int64_t k, void* X,
                 int64_t ldx);
// X = R^-1 for a float64 upper-triangular k x k R (k <= 229), written as float64 (f64, computed
// in float64) or float32 (computed in float32)
void tri_inv_from_f64(cudaStream_t st, bool f64, const double* R, int64_t ldr, int64_t k, void* X,
                      int64_t ldx);

// ------------------------------------------------------------------------------------ panel
// Small b x b float64 matrices are column-major with ld = 64.
constexpr int MAXB = 64;
// W (bi x bi Gram, col-major ld 64) -> R (upper, W = R^T R) and Rinv; breakdown clamps the pivot
// and sets flags[1]; R_acc <- R * R_acc if R_acc != nullptr (R_acc starts as identity).
// CHOL_F64: factor and inverse in float64 (the float64 path); CHOL_F64_INV_F32: float64 factor,
// float32 inverse (the mixed path, which applies Rinv in float32); CHOL_F32: both in float32 (the
// orthonormalisation inside the power scheme, where only the span matters); CHOL_ADAPTIVE: float32
// when every pivot keeps >= 1e-4 of its column's squared norm, else as CHOL_F64_INV_F32.
// R may be null.
enum CholPrec { CHOL_F64 = 0, CHOL_F64_INV_F32 = 1, CHOL_F32 = 2, CHOL_ADAPTIVE = 3 };
// `passes` CholeskyQR passes on a float32 rows x bi panel in one cooperative launch; precise =
// false: float32 Gram and factor (power scheme); precise = true: two-level Gram and float32 factor,
// exact-product Gram and float64 factor for a panel with weak pivots.  rinv_out (nullable)
// receives rinv_prev R_1^-1 ... R_passes^-1 (MAXB x MAXB, float64; rinv_prev null = identity; the
// two may be the same buffer).
// bar: two zero-initialised words kept across calls; err is set if a grid barrier timed out.
// out_hi (nullable): also write bf16(P) there (ld ldo), and bf16(P - bf16(P)) to out_lo when given.
// Slices taller than the rows a CTA holds in shared memory are streamed through it in tiles.
// Returns false (nothing launched) when no cooperative launch is possible or the scratch is short.
size_t cholqr_coop_scratch_bytes();
bool cholqr_coop(cudaStream_t st, float* P, int64_t ldp, int64_t rows, int bi, int passes,
                 bool precise, double tau, const double* rinv_prev, double* rinv_out,
                 void* scratch, size_t scratch_bytes, unsigned* bar, int* flags, int* err,
                 bf16* out_hi = nullptr, bf16* out_lo = nullptr, int64_t ldo = 0);
void chol_rinv(cudaStream_t st, const double* W, int bi, double tau_rel, double* R,
               double* Rinv, double* R_acc, int* flags, CholPrec prec);
void set_identity(cudaStream_t st, double* R, int bi);
// P (m x bi, col-major, f32/f64) <- P * Rinv (upper triangular)
void apply_rinv(cudaStream_t st, bool f64, void* P, int64_t ldp, int64_t m, int bi,
                const double* Rinv);
// rn[j] = ||B(j, :)||^2 for rows j < rows of a row-major B (ld), float64 sums
void row_norm2(cudaStream_t st, bool f64, const void* B, int64_t ldb, int rows, int64_t n,
               double* rn);
// state = {E, keep, stop, ...}: E -= rn[j] row by row until E < eps2 (see Sect. 3.1); with
// Wq = Q_i^T Q_i and Gb = B_i B_i^T (MAXB x MAXB, nullable) the rows also carry the correction
// for Q's departure from orthonormality, tr(B_i^T (Q_i^T Q_i - I) B_i), row by row
void indicator(cudaStream_t st, double* state, const double* rn, int rows, double eps2,
               int row_by_row, const double* Wq = nullptr, const double* Gb = nullptr);

// ------------------------------------------------------------------------------------ CSR
struct CsrDev {
    int64_t m, n, nnz;
    const int32_t* rowptr;
    const int32_t* colind;
    const void* val;
    bool f64;
};
// staging bytes for csr_spmm on an m x n matrix (either orientation)
size_t csr_stage_bytes(int64_t m, int64_t n, bool f64);
// CSC copy of A: colptr[n+1], rowind[nnz], cval[nnz]; cnt: 2 n int32 scratch.  Entries inside a
// column come in no particular order (atomic scatter).
void csr_to_csc(cudaStream_t st, const CsrDev& A, int32_t* colptr, int32_t* rowind, void* cval,
                int32_t* cnt);
// Rows of a compressed matrix longer than CSR_SEG nonzeros are cut into CSR_SEG-nonzero segments:
// segment s covers [beg[s], min(beg[s] + CSR_SEG, ptr[row[s] + 1])) of row row[s]; *count
// segments (device int), at most cap.
constexpr int CSR_SEG = 256;
struct CsrSegs {
    int32_t* row = nullptr;
    int32_t* beg = nullptr;
    int32_t* count = nullptr;
    int64_t cap = 0;
};
// upper bound on the segments of any matrix with nnz nonzeros
int64_t csr_seg_cap(int64_t nnz);
// fills segs.row / segs.beg (caller-owned, segs.cap entries each); off: rows + 1 int32 (count is
// off[rows]); tmp: 2 rows int32 scratch
void csr_segments(cudaStream_t st, const int32_t* ptr, int64_t rows, int32_t* off, int32_t* tmp,
                  CsrSegs& segs);
// Y (rows x w, col-major) = S X, S given by (ptr, idx, val) compressed along its rows,
// X (cols x w, col-major); segs: the long-row table of S (nullptr: one warp per row throughout)
void csr_spmm(cudaStream_t st, bool f64, const int32_t* ptr, const int32_t* idx, const void* val,
              int64_t rows, int64_t cols, const CsrSegs* segs, const void* X, int64_t ldx,
              int64_t w, void* Y, int64_t ldy, void* stage);

// ------------------------------------------------------------------------------------ COO
struct CooDev {
    int64_t m, n, nnz;
    const int32_t* row;
    const int32_t* col;
    const void* val;
    bool f64;
};
// Column-sorted copy of COO triplets (counting sort by column; order inside a column is not
// fixed): ocol, orow, oval (nnz each); colptr n + 1 int32; cnt: 2 n int32 scratch.
void coo_by_column(cudaStream_t st, const CooDev& A, int32_t* ocol, int32_t* orow, void* oval,
                   int32_t* colptr, int32_t* cnt);
// Y (rows x w, col-major) = S X for S given by nnz triplets (key = row of S, idx = column of S,
// val), any order (sorted by key is fastest); X (cols x w, col-major); stage as for csr_spmm.
void coo_spmm(cudaStream_t st, bool f64, const int32_t* key, const int32_t* idx, const void* val,
              int64_t nnz, int64_t rows, int64_t cols, const void* X, int64_t ldx, int64_t w,
              void* Y, int64_t ldy, void* stage);

}  // namespace qb
