// Host drivers of randQB_EI (Algorithm 2) and randQB_FP (Algorithm 4) over the kernels of this
// library, and the C ABI declared in include/qb.h.
//
// The drivers are stream-ordered: all arithmetic runs in the library's kernels; the host only
// sequences launches and, once per block, reads back {E, rows kept, stop} (24 bytes) to decide
// whether to continue (Algorithm 1's "if E < eps^2 then stop").
#include "qb_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

namespace qb {

// ------------------------------------------------------------------------------------ process state
static std::atomic<int64_t> g_launches{0};
static char g_last_err[256] = "";
static std::mutex g_err_mu;

void record_cuda_error(cudaError_t e, const char* where) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    std::snprintf(g_last_err, sizeof g_last_err, "%s: %s", where, cudaGetErrorString(e));
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(); }

int num_sms() {
    static int cache[64] = {0};
    int dev = 0;
    QB_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && cache[dev]) return cache[dev];
    int v = 0;
    QB_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 64) cache[dev] = v;
    return v;
}

// ------------------------------------------------------------------------------------ phase profile
enum Phase { PH_OMEGA = 0, PH_SKETCH, PH_TRANS, PH_ORTHW, PH_PROJ, PH_CHOLQR, PH_BFORM, PH_IND,
             PH_COUNT };
static double g_prof_ms[PH_COUNT] = {0};
static std::mutex g_prof_mu;

namespace {

constexpr double U64 = 1.1102230246251565e-16;   // 2^-53
constexpr double U32 = 5.9604644775390625e-08;   // 2^-24
constexpr double THM3_DELTA = 0.01;
constexpr int64_t H_CHUNK = 512;    // randQB_FP: columns of H = A^T G formed at a time
constexpr int64_t FP_CHUNK = 512;   // randQB_FP: Omega columns carried through the power scheme together

// ------------------------------------------------------------------------------------ context
struct Ctx {
    cudaStream_t st = nullptr;
    bool f64 = true;        // work precision of Q, B, G, H, Omega
    size_t es = 8;
    GemmScratch scr;
    double* W = nullptr;    // 64 x 64 Gram
    double* R = nullptr;
    double* Rinv = nullptr;
    double* Racc = nullptr;
    double* Rchain = nullptr; // 4 x (64 x 64): inverses of the CholeskyQR factors of one block
    int nchain = 0;
    bool chain_fused = false;   // the last Rchain slot holds a product formed by coop_precise
    double* rn = nullptr;   // 64 row norms
    double* state = nullptr;  // E, keep, stop, E_prev
    double* part = nullptr;   // 3 x 1024 reduction partials
    int* flags = nullptr;     // [0] non-finite, [1] breakdown, [2] grid-barrier timeout,
                              // [4..5] grid-barrier words of the fused CholeskyQR
    void* coop_scr = nullptr; // fused CholeskyQR partial Grams
    size_t coop_bytes = 0;
    double tau = 1e-14;       // Cholesky breakdown threshold (relative to max Gram diagonal)
    Acc acc_gram = ACC_D;     // Grams of panels
    Acc acc_proj = ACC_D;     // projections / updates
    Acc acc_fine = ACC_D;     // cancellation-prone products (FP's B_i formula, re-orth coefficients)
    bool simt_apass = false;  // QB_FLAG_SIMT_APASS
    // tensor-core projections for the power-scheme orthonormalisation (mixed path)
    void* tcs = nullptr;
    size_t tcs_bytes = 0;
    // three-term bf16 shadows of Q (m x cap) and B^T (n x cap) for the tensor-core projections
    bf16* qs[3] = {nullptr, nullptr, nullptr};
    bf16* bs[3] = {nullptr, nullptr, nullptr};
    int64_t ldqs = 0, ldbs = 0;
    // bf16 shadows of the power-scheme panels finished so far: set 0 for G (hi), set 1 for Omega
    // (hi, lo); separate, because the chunks of a batch alternate between the two orthonormalisations
    bf16* xb_hi[2] = {nullptr, nullptr};
    bf16* xb_lo[2] = {nullptr, nullptr};
    int64_t xb_ld = 0;
    bool prof = false;        // QB_FLAG_PROFILE: CUDA events around the phases of the loop
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> events;
    struct Scope {
        Ctx* c;
        int ph;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        Scope(Ctx& cc, int p) : c(&cc), ph(p) {
            if (!c->prof) return;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, c->st);
        }
        ~Scope() {
            if (!c->prof) return;
            cudaEventRecord(e1, c->st);
            c->events.push_back({ph, {e0, e1}});
        }
    };
    void flush_profile() {
        if (!prof) return;
        cudaStreamSynchronize(st);
        double acc[PH_COUNT] = {0};
        for (auto& e : events) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e.second.first, e.second.second);
            acc[e.first] += ms;
            cudaEventDestroy(e.second.first);
            cudaEventDestroy(e.second.second);
        }
        events.clear();
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (int i = 0; i < PH_COUNT; ++i) g_prof_ms[i] = acc[i];
    }

    void alloc(Arena& ar, int64_t mn_max) {
        scr.part_bytes = gemm_scratch_bytes(mn_max);
        scr.part = ar.get<char>(int64_t(scr.part_bytes));
        W = ar.get<double>(MAXB * MAXB);
        R = ar.get<double>(MAXB * MAXB);
        Rinv = ar.get<double>(MAXB * MAXB);
        Racc = ar.get<double>(MAXB * MAXB);
        Rchain = ar.get<double>(4 * MAXB * MAXB);
        rn = ar.get<double>(MAXB);
        state = ar.get<double>(8);
        part = ar.get<double>(3 * 1024);
        flags = ar.get<int>(8);
        coop_scr = ar.get<char>(int64_t(cholqr_coop_scratch_bytes()));
        coop_bytes = cholqr_coop_scratch_bytes();
    }
    XOp x(const void* p, int64_t ld) const { return XOp{f64 ? X_F64 : X_F32, p, nullptr, ld}; }

    // C (M x N) = alpha * X^T Y + beta C, X (K x M), Y (K x N), work precision, col-major
    void tn(int64_t M, int64_t N, int64_t K, double alpha, const void* X, int64_t ldx, const void* Y,
            int64_t ldy, double beta, void* C, int64_t ldc, Acc acc) {
        if (M <= 0 || N <= 0) return;
        gemm(st, true, M, N, K, alpha, x(X, ldx), Y, f64, ldy, beta, C, f64, ldc, f64 ? ACC_D : acc, scr);
    }
    // C (M x N) = alpha * X Y + beta C, X (M x K), Y (K x N)
    void nn(int64_t M, int64_t N, int64_t K, double alpha, const void* X, int64_t ldx, const void* Y,
            int64_t ldy, double beta, void* C, int64_t ldc, Acc acc) {
        if (M <= 0 || N <= 0) return;
        gemm(st, false, M, N, K, alpha, x(X, ldx), Y, f64, ldy, beta, C, f64, ldc, f64 ? ACC_D : acc, scr);
    }
    void copy_cols_(const void* X, int64_t ldx, int64_t rows, int64_t cols, void* Y, int64_t ldy) {
        copy_cols(st, f64, X, ldx, rows, cols, Y, ldy);
    }
    char* col(void* base, int64_t ld, int64_t j) const {
        return reinterpret_cast<char*>(base) + size_t(j) * size_t(ld) * es;
    }
    const char* col(const void* base, int64_t ld, int64_t j) const {
        return reinterpret_cast<const char*>(base) + size_t(j) * size_t(ld) * es;
    }

    // One CholeskyQR pass: W = P^T P (float64 or float32-pair accumulation), W = R^T R,
    // P <- P R^-1; with acc_r the factor's inverse is kept in Rchain (in order) for the B_i formula.  sketch: the basis only has to span the same space
    // (the power scheme), so the Gram is accumulated and factored in float32.
    // Fused float32 CholeskyQR passes for the power-scheme orthonormalisation (one launch).
    bool coop(void* P, int64_t ld, int64_t rows, int bi, int passes, bf16* out_hi = nullptr,
              bf16* out_lo = nullptr, int64_t ldo = 0) {
        return cholqr_coop(st, reinterpret_cast<float*>(P), ld, rows, bi, passes, false, 1e-10,
                           nullptr, nullptr, coop_scr, coop_bytes,
                           reinterpret_cast<unsigned*>(flags + 4), flags, flags + 2, out_hi,
                           out_lo, ldo);
    }
    // Fused CholeskyQR2 of a Q_i panel on the mixed path (adaptive factor).  With acc_r the
    // product of the inverses joins the Rchain: multiplied into the last slot when that slot came
    // from this path too (the slots are applied in order, so a product of consecutive ones is the
    // same), else into a new slot.
    bool coop_precise(void* P, int64_t ld, int64_t rows, int bi, bool acc_r, int passes = 2) {
        if (f64 || (acc_r && nchain >= 4)) return false;
        const bool merge = acc_r && nchain > 0 && chain_fused;
        double* slot = acc_r ? Rchain + size_t(merge ? nchain - 1 : nchain) * MAXB * MAXB : nullptr;
        if (!cholqr_coop(st, reinterpret_cast<float*>(P), ld, rows, bi, passes, true, tau,
                         merge ? slot : nullptr, slot, coop_scr, coop_bytes,
                         reinterpret_cast<unsigned*>(flags + 4), flags, flags + 2))
            return false;
        if (acc_r && !merge) ++nchain;
        if (acc_r) chain_fused = true;
        return true;
    }
    void cholqr(void* P, int64_t ld, int64_t rows, int bi, bool acc_r, bool sketch = false) {
        const bool fast = sketch && !f64;
        if (fast && !acc_r && coop(P, ld, rows, bi, 1)) return;
        gram(st, P, ld, rows, bi, f64, f64 ? ACC_D : (fast ? ACC_F : acc_gram), W, scr);
        double* ri = Rinv;
        if (acc_r && nchain < 4) {
            ri = Rchain + size_t(nchain++) * MAXB * MAXB;
            chain_fused = false;
        }
        chol_rinv(st, W, bi, fast ? 1e-10 : tau, nullptr, ri, nullptr, flags,
                  f64 ? CHOL_F64 : (fast ? CHOL_F32 : CHOL_ADAPTIVE));
        apply_rinv(st, f64, P, ld, rows, bi, ri);
    }
    // Fused CholeskyQR2 with the adaptive factor on the mixed path; Rinv receives
    // R_1^-1 R_2^-1 = (R_2 R_1)^-1 (the fixed-rank map inverts it to keep R).  False: not launched.
    bool coop_rinv(void* P, int64_t ld, int64_t rows, int bi) {
        if (f64) return false;
        return cholqr_coop(st, reinterpret_cast<float*>(P), ld, rows, bi, 2, true, tau, nullptr,
                           Rinv, coop_scr, coop_bytes, reinterpret_cast<unsigned*>(flags + 4), flags,
                           flags + 2);
    }
    // CholeskyQR pass accumulating the factor: Racc <- R Racc (the fixed-rank map keeps R)
    void cholqr_racc(void* P, int64_t ld, int64_t rows, int bi) {
        gram(st, P, ld, rows, bi, f64, f64 ? ACC_D : acc_gram, W, scr);
        chol_rinv(st, W, bi, tau, nullptr, Rinv, Racc, flags, f64 ? CHOL_F64 : CHOL_F64_INV_F32);
        apply_rinv(st, f64, P, ld, rows, bi, Rinv);
    }
    // orth(P): CholeskyQR2 (two passes); with acc_r the factors' inverses go to Rchain.
    void cholqr2(void* P, int64_t ld, int64_t rows, int bi, bool acc_r, bool sketch = false) {
        Scope sc(*this, sketch ? PH_ORTHW : PH_CHOLQR);
        if (sketch && !f64 && !acc_r && coop(P, ld, rows, bi, 2)) return;
        if (!sketch && coop_precise(P, ld, rows, bi, acc_r)) return;
        cholqr(P, ld, rows, bi, acc_r, sketch);
        cholqr(P, ld, rows, bi, acc_r, sketch);
    }
    // orth(P) of a block that is re-orthogonalised and orthonormalised again right after: one
    // CholeskyQR pass on the mixed path (the passes after the re-orthogonalisation restore
    // float32 orthogonality), CholeskyQR2 on the float64 path
    void cholqr_pre(void* P, int64_t ld, int64_t rows, int bi, bool acc_r) {
        if (f64) {
            cholqr2(P, ld, rows, bi, acc_r);
            return;
        }
        Scope sc(*this, PH_CHOLQR);
        if (coop_precise(P, ld, rows, bi, acc_r, 1)) return;
        cholqr(P, ld, rows, bi, acc_r);
    }
    // orth(P) inside a power step, where only the span matters: one float32 CholeskyQR pass on
    // the mixed path (a well-conditioned basis is enough for the next application of A or A^T),
    // CholeskyQR2 on the float64 path
    void orth_span(void* P, int64_t ld, int64_t rows, int bi) {
        if (f64) {
            cholqr2(P, ld, rows, bi, false);
            return;
        }
        Scope sc(*this, PH_ORTHW);
        cholqr(P, ld, rows, bi, false, true);
    }
    // P <- P - Qk (Qk^T P), Qk = first k columns of Q (ld ldq); T: k x bi scratch (ld k)
    void project_out(const void* Q, int64_t ldq, int64_t k, void* P, int64_t ldp, int64_t rows, int bi,
                     void* T, bool sketch = false) {
        if (k <= 0) return;
        Scope sc(*this, sketch ? PH_ORTHW : PH_PROJ);
        tn(k, bi, rows, 1.0, Q, ldq, P, ldp, 0.0, T, k, sketch ? ACC_F : acc_fine);
        nn(rows, bi, k, -1.0, Q, ldq, T, k, 1.0, P, ldp, acc_proj);
    }
    // ---- products with the current Q (m x k, ld ldq) and B (k x n row-major = n x k column-major,
    // ld ldb); tensor cores (float32 accuracy) when the three-term shadows exist, SIMT otherwise.
    bool tcg() const { return qs[0] != nullptr; }
    const bf16* const* qsp() const { return qs; }
    // T (k x bi, ld ldt) = Q^T X + beta T, X m x bi
    void qt_x(int64_t k, int bi, const void* Q, int64_t ldq, int64_t m, const void* X, int64_t ldx,
              double beta, void* T, int64_t ldt, Acc acc) {
        if (k <= 0) return;
        if (tcg()) {
            tc_prec_gemm(st, false, qs, 3, ldqs, k, m, reinterpret_cast<const float*>(X), ldx, bi,
                         1.f, float(beta), reinterpret_cast<float*>(T), ldt, tcs, tcs_bytes);
            return;
        }
        tn(k, bi, m, 1.0, Q, ldq, X, ldx, beta, T, ldt, acc);
    }
    // [T1 | T2] (k x 2 bi, ld ldt) += Q^T [X1 | X2] (X1, X2: m x bi) in one pass over Q's shadows
    // (tensor-core path only)
    void qt_x2(int64_t k, int bi, int64_t m, const void* X1, int64_t ldx1, const void* X2,
               int64_t ldx2, void* T, int64_t ldt) {
        tc_prec_gemm2(st, false, qs, 3, ldqs, k, m, reinterpret_cast<const float*>(X1), ldx1, bi,
                      reinterpret_cast<const float*>(X2), ldx2, bi, 1.f, 1.f,
                      reinterpret_cast<float*>(T), ldt, tcs, tcs_bytes);
    }
    // Y (m x bi) += alpha Q T, T k x bi
    void q_t(int64_t k, int bi, const void* Q, int64_t ldq, int64_t m, double alpha, const void* T,
             int64_t ldt, void* Y, int64_t ldy, Acc acc) {
        if (k <= 0) return;
        if (tcg()) {
            tc_prec_gemm(st, true, qs, 3, ldqs, m, k, reinterpret_cast<const float*>(T), ldt, bi,
                         float(alpha), 1.f, reinterpret_cast<float*>(Y), ldy, tcs, tcs_bytes);
            return;
        }
        nn(m, bi, k, alpha, Q, ldq, T, ldt, 1.0, Y, ldy, acc);
    }
    // T (k x bi) = B X + beta T, X n x bi
    void b_x(int64_t k, int bi, const void* B, int64_t ldb, int64_t n, const void* X, int64_t ldx,
             double beta, void* T, int64_t ldt, Acc acc) {
        if (k <= 0) return;
        if (tcg()) {
            tc_prec_gemm(st, false, bs, 3, ldbs, k, n, reinterpret_cast<const float*>(X), ldx, bi,
                         1.f, float(beta), reinterpret_cast<float*>(T), ldt, tcs, tcs_bytes);
            return;
        }
        tn(k, bi, n, 1.0, B, ldb, X, ldx, beta, T, ldt, acc);
    }
    // Z (n x bi) += alpha B^T T, T k x bi
    void bt_t(int64_t k, int bi, const void* B, int64_t ldb, int64_t n, double alpha, const void* T,
              int64_t ldt, void* Z, int64_t ldz, Acc acc) {
        if (k <= 0) return;
        if (tcg()) {
            tc_prec_gemm(st, true, bs, 3, ldbs, n, k, reinterpret_cast<const float*>(T), ldt, bi,
                         float(alpha), 1.f, reinterpret_cast<float*>(Z), ldz, tcs, tcs_bytes);
            return;
        }
        nn(n, bi, k, alpha, B, ldb, T, ldt, 1.0, Z, ldz, acc);
    }
    // re-orthogonalise P (m x bi) against Q: P -= Q (Q^T P); T: k x bi scratch
    void reorth_q(int64_t k, const void* Q, int64_t ldq, int64_t m, void* P, int64_t ldp, int bi,
                  void* T) {
        if (k <= 0) return;
        if (!tcg()) {
            project_out(Q, ldq, k, P, ldp, m, bi, T);
            return;
        }
        Scope sc(*this, PH_PROJ);
        qt_x(k, bi, Q, ldq, m, P, ldp, 0.0, T, k, acc_fine);
        q_t(k, bi, Q, ldq, m, -1.0, T, k, P, ldp, acc_proj);
    }
    // a block is final: record its three-term shadows (Q_i: m x bi at column k; B_i^T: n x bi)
    void shadow(int64_t k, int bi, const void* Qi, int64_t ldq, int64_t m, const void* BiT,
                int64_t ldb, int64_t n) {
        if (!tcg()) return;
        split3_bf16(st, reinterpret_cast<const float*>(Qi), ldq, m, bi, qs[0] + k * ldqs,
                    qs[1] + k * ldqs, qs[2] + k * ldqs, ldqs);
        split3_bf16(st, reinterpret_cast<const float*>(BiT), ldb, n, bi, bs[0] + k * ldbs,
                    bs[1] + k * ldbs, bs[2] + k * ldbs, ldbs);
    }
    // Orthonormalise the rows x w matrix X (column-major) panel by panel for the power scheme:
    // block Gram-Schmidt with re-orthogonalisation, CholeskyQR per panel of width b.  Only the
    // span matters here, so the mixed path works in float32 throughout.  T: w x b scratch.
    //
    // On the mixed path with a TMA-compatible layout the projections run on the tensor cores
    // against a bf16 shadow of the finished panels: bf16 only for G (one pass; any well-conditioned
    // basis will do), bf16 hi + lo with three products for Omega (its residual overlap with earlier
    // panels leaks sigma_1^2-sized terms into the B_i formula).
    // Panels from column j_begin on are orthonormalised against all columns before them (the
    // columns before j_begin are already final): the result is column-causal, the first k columns
    // depend only on the first k input columns.
    void orth_wide(void* X, int64_t ld, int64_t rows, int64_t w, int b, void* T, bool reorth = true,
                   int64_t j_begin = 0) {
        const int set = reorth ? 1 : 0;
        bf16* hi = xb_hi[set];
        const bool tc = !f64 && hi && rows % 8 == 0 && rows <= xb_ld;
        bf16* lo = reorth ? xb_lo[set] : nullptr;
        auto project = [&](int64_t j0, char* Pj, int bj) {
            if (j0 <= 0) return;
            if (!tc) {
                project_out(X, ld, j0, Pj, ld, rows, bj, T, true);
                return;
            }
            Scope sc(*this, PH_ORTHW);
            tc_xtp(st, hi, lo, xb_ld, rows, j0, reinterpret_cast<const float*>(Pj), ld, bj,
                   reinterpret_cast<float*>(T), j0, tcs, tcs_bytes);
            tc_p_minus_xt(st, hi, lo, xb_ld, rows, j0, reinterpret_cast<const float*>(T), j0,
                          bj, reinterpret_cast<float*>(Pj), ld, tcs, tcs_bytes);
        };
        for (int64_t j0 = j_begin; j0 < w; j0 += b) {
            const int bj = int(std::min<int64_t>(b, w - j0));
            char* Pj = col(X, ld, j0);
            // the last orthonormalisation of the panel also writes its bf16 shadow when fused
            bf16* shi = tc ? hi + j0 * xb_ld : nullptr;
            bf16* slo = tc && lo ? lo + j0 * xb_ld : nullptr;
            const bool again = j0 > 0 && (reorth || f64);
            bool shadow = false;
            auto fused = [&](int passes, bf16* h) {
                Scope sc(*this, PH_ORTHW);
                return !f64 && coop(Pj, ld, rows, bj, passes, h, slo, xb_ld);
            };
            project(j0, Pj, bj);
            // a panel that is projected again gets one CholeskyQR pass before the second
            // projection and one after it (the second pass restores float32 orthogonality);
            // without re-orthogonalisation (G of the power scheme, which only has to be a
            // well-conditioned basis for the next application of A^T) one pass in all on the
            // mixed path; otherwise CholeskyQR2 here
            const bool one = again || !reorth;
            if (fused(one ? 1 : 2, again ? nullptr : shi)) shadow = !again;
            else if (one && !f64) cholqr(Pj, ld, rows, bj, false, true);
            else cholqr2(Pj, ld, rows, bj, false, true);
            if (again) {
                project(j0, Pj, bj);
                if (f64) cholqr2(Pj, ld, rows, bj, false, true);
                else if (fused(1, shi)) shadow = true;
                else cholqr(Pj, ld, rows, bj, false, true);
            }
            if (tc && !shadow)
                split_bf16(st, reinterpret_cast<const float*>(Pj), ld, rows, bj, shi, slo, xb_ld);
        }
    }
    struct Step { double E; int keep; int stop; };
    Step indicator_step(const void* Bslot, int64_t ldb, int bi, int64_t n, double eps2, int rbr) {
        Scope sc(*this, PH_IND);
        row_norm2(st, f64, Bslot, ldb, bi, n, rn);
        indicator(st, state, rn, bi, eps2, rbr);
        double h[3];
        QB_CUDA(cudaMemcpyAsync(h, state, sizeof h, cudaMemcpyDeviceToHost, st));
        QB_CUDA(cudaStreamSynchronize(st));
        return Step{h[0], int(h[1]), int(h[2])};
    }
    int read_flags(int* h) {
        QB_CUDA(cudaMemcpyAsync(h, flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        QB_CUDA(cudaStreamSynchronize(st));
        return 0;
    }
};

// ------------------------------------------------------------------------------------ A operators
struct AOp {
    int64_t m = 0, n = 0;
    virtual ~AOp() = default;
    virtual void reserve(Arena& ar, const Ctx& c, int64_t wmax) = 0;
    virtual void prepare(Ctx& c) = 0;
    // Y (m x w) = A X (X: n x w); sketch passes may use the reduced representation of A.
    // pairs = 2: X was rounded to two bf16 terms and both are used (randQB_FP's final G).
    virtual void apply(Ctx& c, const void* X, int64_t ldx, int64_t w, void* Y, int64_t ldy,
                       int pairs = 1) = 0;
    // Y (n x w) = A^T X (X: m x w).  mode 1: sketch precision; mode 2: full A with an operand
    // already rounded by round_operand(); mode 3: full A and full-precision operand (B_i = Q_i^T A);
    // mode 4: full A with an operand rounded to two bf16 terms (round_operand(.., 2))
    virtual void apply_t(Ctx& c, const void* X, int64_t ldx, int64_t w, void* Y, int64_t ldy,
                         int mode) = 0;
    // Round an operand of the coming passes to the precision the passes consume (bf16 on the
    // tensor-core path), in place, so that the projections against Q, B use the same values.
    virtual void round_operand(Ctx&, void*, int64_t, int64_t, int64_t, int pairs = 1) {}
    // ||A||_F^2 (float64); non-finite entries raise c.flags[0]
    virtual double norm2(Ctx& c) = 0;
    // true when a bounded device-side wait of this operator's kernels ran out
    virtual bool timed_out(Ctx&) { return false; }
    // tensor-core scratch of this operator, if it has one
    virtual bool tc_scratch(void**, size_t*) { return false; }
};

struct DenseOp : AOp {
    qb_dense d;
    bool use_tc = false;
    void* tc_scr = nullptr;
    size_t tc_bytes = 0;
    bf16* Xb = nullptr;      // bf16 copy of the sketch operand (tensor-core path)
    int64_t wmax = 0;
    bool lo_waited = false;
    explicit DenseOp(const qb_dense& dd) : d(dd) { m = dd.m; n = dd.n; }
    // before the first read of a_lo: wait for the caller's event (a_lo may still be arriving)
    void wait_lo(Ctx& c) {
        if (d.a_lo_ready && d.a_lo && !lo_waited) {
            cudaEvent_t ev = reinterpret_cast<cudaEvent_t>(const_cast<void*>(d.a_lo_ready));
            QB_CUDA(cudaStreamWaitEvent(c.st, ev, 0));
            lo_waited = true;
        }
    }
    XOp xa(bool precise) const {
        switch (d.dtype) {
            case QB_F64: return XOp{X_F64, d.a, nullptr, d.ld};
            case QB_F32: return XOp{X_F32, d.a, nullptr, d.ld};
            case QB_BF16: return XOp{X_BF16, d.a, nullptr, d.ld};
            default: return precise ? XOp{X_BF16X2, d.a, d.a_lo, d.ld} : XOp{X_BF16, d.a, nullptr, d.ld};
        }
    }
    bool bf16_storage() const { return d.dtype == QB_BF16 || d.dtype == QB_BF16X2; }
    // The tensor-core path needs TMA-compatible A: 16-byte aligned rows and base, and at least
    // one full 128-row tile each way.
    bool tc_ok() const {
        auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
        return bf16_storage() && d.ld % 8 == 0 && al(d.a) && (!d.a_lo || al(d.a_lo)) &&
               m >= 128 && n >= 128;
    }
    void reserve(Arena& ar, const Ctx& c, int64_t w) override {
        wmax = w;
        use_tc = !c.f64 && !c.simt_apass && tc_ok() && (ar.base == nullptr || tc_available());
        if (use_tc) {
            tc_bytes = tc_scratch_bytes(m, n, w);
            tc_scr = ar.get<char>(int64_t(tc_bytes));
            Xb = ar.get<bf16>(2 * align_up(n, 8) * w);
        }
    }
    void prepare(Ctx& c) override {
        if (use_tc) QB_CUDA(cudaMemsetAsync(tc_error_flag(tc_scr), 0, 256, c.st));
    }
    bool tc_scratch(void** p, size_t* b) override {
        if (!use_tc) return false;
        *p = tc_scr;
        *b = tc_bytes;
        return true;
    }
    bool timed_out(Ctx& c) override {
        if (!use_tc) return false;
        int h = 0;
        QB_CUDA(cudaMemcpyAsync(&h, tc_error_flag(tc_scr), sizeof h, cudaMemcpyDeviceToHost, c.st));
        QB_CUDA(cudaStreamSynchronize(c.st));
        return h != 0;
    }
    void apply(Ctx& c, const void* X, int64_t ldx, int64_t w, void* Y, int64_t ldy,
               int pairs) override {
        Ctx::Scope sc(c, PH_SKETCH);
        if (use_tc) {
            const int64_t ldb = align_up(n, 8);
            bf16* lo = pairs == 2 ? Xb + ldb * wmax : nullptr;
            split_bf16(c.st, reinterpret_cast<const float*>(X), ldx, n, w, Xb, lo, ldb);
            tc_sketch(c.st, reinterpret_cast<const bf16*>(d.a), d.ld, m, n, Xb, lo, ldb, w,
                      reinterpret_cast<float*>(Y), ldy, tc_scr, tc_bytes);
            return;
        }
        // Y = (A viewed column-major n x m)^T X
        gemm(c.st, true, m, w, n, 1.0, xa(false), X, c.f64, ldx, 0.0, Y, c.f64, ldy,
             c.f64 ? ACC_D : ACC_F, c.scr);
    }
    void apply_t(Ctx& c, const void* X, int64_t ldx, int64_t w, void* Y, int64_t ldy,
                 int mode) override {
        Ctx::Scope sc(c, PH_TRANS);
        if (mode >= 2) wait_lo(c);                 // mode 1 reads a_hi only
        if (use_tc && mode >= 2) {
            // The passes that feed the indicator (B_i = Q_i^T A, H = A^T G): full A, the operand
            // split exactly into bf16 terms, the leading product summed per MMA in registers with
            // round-to-nearest (tensor-core float32 accumulation is not round-to-nearest and
            // would bias ||B_i||^2 low on long reductions).
            tc_trans(c.st, reinterpret_cast<const bf16*>(d.a),
                     d.dtype == QB_BF16X2 ? reinterpret_cast<const bf16*>(d.a_lo) : nullptr, d.ld,
                     m, n, reinterpret_cast<const float*>(X), ldx, w, reinterpret_cast<float*>(Y),
                     ldy, mode, tc_scr, tc_bytes);
            return;
        }
        if (!c.f64 && mode >= 2 && bf16_storage()) {
            // round-to-nearest float32 sums on the SIMT cores
            trans_precise(c.st, reinterpret_cast<const bf16*>(d.a),
                          d.dtype == QB_BF16X2 ? reinterpret_cast<const bf16*>(d.a_lo) : nullptr,
                          d.ld, m, n,
                          reinterpret_cast<const float*>(X), ldx, w, reinterpret_cast<float*>(Y),
                          ldy, c.scr);
            return;
        }
        if (use_tc) {
            tc_trans(c.st, reinterpret_cast<const bf16*>(d.a), reinterpret_cast<const bf16*>(d.a_lo),
                     d.ld, m, n, reinterpret_cast<const float*>(X), ldx, w,
                     reinterpret_cast<float*>(Y), ldy, 1, tc_scr, tc_bytes);
            return;
        }
        gemm(c.st, false, n, w, m, 1.0, xa(mode > 1), X, c.f64, ldx, 0.0, Y, c.f64, ldy,
             c.f64 ? ACC_D : ACC_F, c.scr);
    }
    void round_operand(Ctx& c, void* X, int64_t ldx, int64_t rows, int64_t w,
                       int pairs) override {
        if (use_tc) round_bf16_inplace(c.st, reinterpret_cast<float*>(X), ldx, rows, w, pairs);
    }
    double norm2(Ctx& c) override {
        if (!std::isnan(d.src_norm2)) return d.src_norm2;
        wait_lo(c);
        dense_norm2(c.st, xa(true), m, n, c.part, c.state + 4, c.flags);
        double h = 0;
        QB_CUDA(cudaMemcpyAsync(&h, c.state + 4, sizeof h, cudaMemcpyDeviceToHost, c.st));
        QB_CUDA(cudaStreamSynchronize(c.st));
        return h;
    }
};

struct CsrOp : AOp {
    qb_csr s;
    int32_t* colptr = nullptr;
    int32_t* rowind = nullptr;
    void* cval = nullptr;
    int32_t* cnt = nullptr;
    void* stage = nullptr;
    CsrSegs seg_r, seg_c;            // long rows of A, long columns of A (rows of the CSC copy)
    int32_t* off_r = nullptr;
    int32_t* off_c = nullptr;
    // The passes over A are SIMT gathers; on the float32 path the projections against Q and B
    // still run on tensor cores (three-term bf16 shadows), which needs the tensor-core scratch.
    bool use_tc = false;
    void* tc_scr = nullptr;
    size_t tc_bytes = 0;
    explicit CsrOp(const qb_csr& ss) : s(ss) { m = ss.m; n = ss.n; }
    bool f64v() const { return s.dtype == QB_F64; }
    void reserve(Arena& ar, const Ctx& c, int64_t w) override {
        use_tc = !c.f64 && !c.simt_apass && m >= 128 && n >= 128 &&
                 (ar.base == nullptr || tc_available());
        if (use_tc) {
            tc_bytes = tc_scratch_bytes(m, n, w);
            tc_scr = ar.get<char>(int64_t(tc_bytes));
        }
        colptr = ar.get<int32_t>(n + 1);
        rowind = ar.get<int32_t>(s.nnz);
        cval = ar.get<char>(s.nnz * (f64v() ? 8 : 4));
        cnt = ar.get<int32_t>(2 * std::max(m, n));
        stage = ar.get<char>(int64_t(csr_stage_bytes(m, n, f64v())));
        for (CsrSegs* g : {&seg_r, &seg_c}) {
            g->cap = csr_seg_cap(s.nnz);
            g->row = ar.get<int32_t>(g->cap);
            g->beg = ar.get<int32_t>(g->cap);
        }
        off_r = ar.get<int32_t>(m + 1);
        off_c = ar.get<int32_t>(n + 1);
    }
    bool tc_scratch(void** p, size_t* b) override {
        if (!use_tc) return false;
        *p = tc_scr;
        *b = tc_bytes;
        return true;
    }
    bool timed_out(Ctx& c) override {
        if (!use_tc) return false;
        int h = 0;
        QB_CUDA(cudaMemcpyAsync(&h, tc_error_flag(tc_scr), sizeof h, cudaMemcpyDeviceToHost, c.st));
        QB_CUDA(cudaStreamSynchronize(c.st));
        return h != 0;
    }
    void prepare(Ctx& c) override {
        if (use_tc) QB_CUDA(cudaMemsetAsync(tc_error_flag(tc_scr), 0, 256, c.st));
        CsrDev A{m, n, s.nnz, s.rowptr, s.colind, s.val, f64v()};
        csr_to_csc(c.st, A, colptr, rowind, cval, cnt);
        csr_segments(c.st, s.rowptr, m, off_r, cnt, seg_r);
        csr_segments(c.st, colptr, n, off_c, cnt, seg_c);
    }
    void apply(Ctx& c, const void* X, int64_t ldx, int64_t w, void* Y, int64_t ldy, int) override {
        Ctx::Scope sc(c, PH_SKETCH);
        csr_spmm(c.st, f64v(), s.rowptr, s.colind, s.val, m, n, &seg_r, X, ldx, w, Y, ldy, stage);
    }
    void apply_t(Ctx& c, const void* X, int64_t ldx, int64_t w, void* Y, int64_t ldy, int) override {
        Ctx::Scope sc(c, PH_TRANS);
        csr_spmm(c.st, f64v(), colptr, rowind, cval, n, m, &seg_c, X, ldx, w, Y, ldy, stage);
    }
    double norm2(Ctx& c) override {
        vec_norm2(c.st, s.val, f64v(), s.nnz, c.part, c.state + 4, c.flags);
        double h = 0;
        QB_CUDA(cudaMemcpyAsync(&h, c.state + 4, sizeof h, cudaMemcpyDeviceToHost, c.st));
        QB_CUDA(cudaStreamSynchronize(c.st));
        return h;
    }
};

// Sparse A as COO triplets (Sect. 5.1: COO instead of CSR).  A X runs the nonzero-balanced
// segmented kernel on the caller's triplets (fastest sorted by row); A^T X on a column-sorted copy
// built once per call.  No row pointer is needed and no row or column length sets the load of a
// warp: every warp takes 256 nonzeros.
struct CooOp : AOp {
    qb_coo s;
    int32_t* ocol = nullptr;
    int32_t* orow = nullptr;
    void* oval = nullptr;
    int32_t* colptr = nullptr;
    int32_t* cnt = nullptr;
    void* stage = nullptr;
    bool use_tc = false;
    void* tc_scr = nullptr;
    size_t tc_bytes = 0;
    explicit CooOp(const qb_coo& ss) : s(ss) { m = ss.m; n = ss.n; }
    bool f64v() const { return s.dtype == QB_F64; }
    void reserve(Arena& ar, const Ctx& c, int64_t w) override {
        use_tc = !c.f64 && !c.simt_apass && m >= 128 && n >= 128 &&
                 (ar.base == nullptr || tc_available());
        if (use_tc) {
            tc_bytes = tc_scratch_bytes(m, n, w);
            tc_scr = ar.get<char>(int64_t(tc_bytes));
        }
        ocol = ar.get<int32_t>(s.nnz);
        orow = ar.get<int32_t>(s.nnz);
        oval = ar.get<char>(s.nnz * (f64v() ? 8 : 4));
        colptr = ar.get<int32_t>(n + 1);
        cnt = ar.get<int32_t>(2 * std::max<int64_t>(n, 1));
        stage = ar.get<char>(int64_t(csr_stage_bytes(m, n, f64v())));
    }
    bool tc_scratch(void** p, size_t* b) override {
        if (!use_tc) return false;
        *p = tc_scr;
        *b = tc_bytes;
        return true;
    }
    bool timed_out(Ctx& c) override {
        if (!use_tc) return false;
        int h = 0;
        QB_CUDA(cudaMemcpyAsync(&h, tc_error_flag(tc_scr), sizeof h, cudaMemcpyDeviceToHost, c.st));
        QB_CUDA(cudaStreamSynchronize(c.st));
        return h != 0;
    }
    void prepare(Ctx& c) override {
        if (use_tc) QB_CUDA(cudaMemsetAsync(tc_error_flag(tc_scr), 0, 256, c.st));
        CooDev A{m, n, s.nnz, s.row, s.col, s.val, f64v()};
        coo_by_column(c.st, A, ocol, orow, oval, colptr, cnt);
    }
    void apply(Ctx& c, const void* X, int64_t ldx, int64_t w, void* Y, int64_t ldy, int) override {
        Ctx::Scope sc(c, PH_SKETCH);
        coo_spmm(c.st, f64v(), s.row, s.col, s.val, s.nnz, m, n, X, ldx, w, Y, ldy, stage);
    }
    void apply_t(Ctx& c, const void* X, int64_t ldx, int64_t w, void* Y, int64_t ldy, int) override {
        Ctx::Scope sc(c, PH_TRANS);
        coo_spmm(c.st, f64v(), ocol, orow, oval, s.nnz, n, m, X, ldx, w, Y, ldy, stage);
    }
    double norm2(Ctx& c) override {
        vec_norm2(c.st, s.val, f64v(), s.nnz, c.part, c.state + 4, c.flags);
        double h = 0;
        QB_CUDA(cudaMemcpyAsync(&h, c.state + 4, sizeof h, cudaMemcpyDeviceToHost, c.st));
        QB_CUDA(cudaStreamSynchronize(c.st));
        return h;
    }
};

// ------------------------------------------------------------------------------------ shared setup
struct Plan {
    int64_t m, n, cap, lt;
    int b, P;
};

bool valid_opts(const qb_opts* o) {
    return o && o->b >= 1 && o->b <= MAXB && o->P >= 0 && o->P <= 8 && std::isfinite(o->tol) &&
           o->tol >= 0.0 && (o->prec == QB_PREC_FP64 || o->prec == QB_PREC_MIXED);
}

Plan make_plan(int64_t m, int64_t n, const qb_opts& o, bool fp) {
    Plan p;
    p.m = m;
    p.n = n;
    p.b = o.b;
    p.P = o.P;
    p.cap = std::min(m, n);
    if (o.rank_cap > 0) p.cap = std::min<int64_t>(p.cap, o.rank_cap);
    p.lt = o.l_tilde > 0 ? o.l_tilde : 50LL * o.b;
    p.lt = std::max<int64_t>(1, std::min(p.lt, std::max<int64_t>(p.cap, 1)));
    if (!fp) p.lt = o.b;
    return p;
}

void setup_ctx(Ctx& c, bool f64) {
    c.f64 = f64;
    c.es = f64 ? 8 : 4;
    c.tau = f64 ? 1e-14 : 1e-12;
    c.acc_gram = f64 ? ACC_D : ACC_DF;
    c.acc_proj = f64 ? ACC_D : ACC_F;
    c.acc_fine = f64 ? ACC_D : ACC_F2;
}

struct Bufs {
    char* Om = nullptr;   // n x lt
    char* Z = nullptr;    // n x b (EI power) or n x b S (FP)
    char* G = nullptr;    // m x lt (FP): G = A Omega of the processed Omega
    char* Gp = nullptr;   // m x lt (FP, P > 0): the power scheme's orthonormal G; kept apart
                          // from G because later chunks project against its earlier columns
    char* H = nullptr;    // n x lt (FP)
    char* Ys = nullptr;   // m x b (FP)
    char* T1 = nullptr;   // cap x lt
    char* C2 = nullptr;   // cap x b
    char* Tw = nullptr;   // lt x b (orth_wide)
    char* TT = nullptr;   // cap x 2b (FP, tensor-core path): [Q^T Q_i | B Omega_i + Q^T Y_i]
};

void reserve_all(Arena& ar, Ctx& c, AOp& A, const Plan& p, bool fp, Bufs& bf) {
    const int64_t es = int64_t(c.es);
    const int64_t wmax = fp ? p.lt : p.b;
    c.alloc(ar, std::max({p.m, p.n, p.cap, wmax}) * std::max<int64_t>(wmax, p.b));
    bf.Om = ar.get<char>(p.n * wmax * es);
    bf.Z = ar.get<char>(p.n * p.b * es);
    bf.T1 = ar.get<char>(std::max<int64_t>(p.cap, 1) * wmax * es);
    bf.C2 = ar.get<char>(std::max<int64_t>(p.cap, 1) * p.b * es);
    if (fp) {
        bf.G = ar.get<char>(p.m * p.lt * es);
        if (p.P > 0) bf.Gp = ar.get<char>(p.m * p.lt * es);
        bf.H = ar.get<char>(p.n * p.lt * es);
        bf.Ys = ar.get<char>(p.m * p.b * es);
        bf.Tw = ar.get<char>(p.lt * p.b * es);
    }
    A.reserve(ar, c, wmax);
    if (!c.f64 && A.tc_scratch(&c.tcs, &c.tcs_bytes)) {
        if (fp && p.P > 0) {
            c.xb_ld = align_up(std::max(p.m, p.n), 8);
            c.xb_hi[0] = ar.get<bf16>(c.xb_ld * p.lt);
            c.xb_hi[1] = ar.get<bf16>(c.xb_ld * p.lt);
            c.xb_lo[1] = ar.get<bf16>(c.xb_ld * p.lt);
        }
        const int64_t cap = std::max<int64_t>(p.cap, 1);
        c.ldqs = align_up(p.m, 8);
        c.ldbs = align_up(p.n, 8);
        for (int t = 0; t < 3; ++t) c.qs[t] = ar.get<bf16>(c.ldqs * cap);
        for (int t = 0; t < 3; ++t) c.bs[t] = ar.get<bf16>(c.ldbs * cap);
        // the merged Q^T [Q_i | Y_i] product splits 2b columns into the scratch sized for lt
        if (fp && p.lt >= 2 * p.b) bf.TT = ar.get<char>(cap * 2 * p.b * es);
    }
}

struct RunOut {
    int64_t rank = 0;
    double E = 0, normA2 = 0;
    int64_t passes = 0, omega_cols = 0;
    int blocks = 0;
    bool converged = false;
};

// ------------------------------------------------------------------------------------ randQB_EI
void run_ei(Ctx& c, AOp& A, const Plan& p, const qb_opts& o, Bufs& bf, void* Q, int64_t ldq,
            void* B, int64_t ldb, double eps2, RunOut& out) {
    const int64_t m = p.m, n = p.n;
    int64_t k = 0;
    const int omega_dt = c.f64 ? QB_F64 : QB_F32;
    while (k < p.cap) {
        const int bi = int(std::min<int64_t>(p.b, p.cap - k));
        out.omega_cols = k + bi;
        // Omega_i = randn(n, b), global columns [k, k + bi)
        {
            Ctx::Scope so(c, PH_OMEGA);
            omega_gen(c.st, n, k, bi, o.seed, omega_dt, bf.Om, n);
            A.round_operand(c, bf.Om, n, n, bi);
        }
        // Y = A Omega_i - Q (B Omega_i), computed in the slot of Q_i
        char* Y = c.col(Q, ldq, k);
        A.apply(c, bf.Om, n, bi, Y, ldq);
        out.passes += 1;
        if (k > 0) {
            Ctx::Scope sp(c, PH_PROJ);
            c.b_x(k, bi, B, ldb, n, bf.Om, n, 0.0, bf.T1, k, c.acc_proj);          // B Omega_i
            c.q_t(k, bi, Q, ldq, m, -1.0, bf.T1, k, Y, ldq, c.acc_proj);          // Y -= Q (.)
        }
        for (int it = 0; it < p.P; ++it) {
            c.orth_span(Y, ldq, m, bi);                                           // Y = orth(Y)
            A.round_operand(c, Y, ldq, m, bi);
            A.apply_t(c, Y, ldq, bi, bf.Z, n, 1);                                 // Z = A^T Y
            out.passes += 1;
            if (k > 0) {
                Ctx::Scope sp(c, PH_PROJ);
                c.qt_x(k, bi, Q, ldq, m, Y, ldq, 0.0, bf.T1, k, c.acc_proj);      // Q^T Y
                c.bt_t(k, bi, B, ldb, n, -1.0, bf.T1, k, bf.Z, n, c.acc_proj);    // Z -= B^T (.)
            }
            c.orth_span(bf.Z, n, n, bi);                                          // Z = orth(Z)
            A.round_operand(c, bf.Z, n, n, bi);
            A.apply(c, bf.Z, n, bi, Y, ldq);                                      // Y = A Z
            out.passes += 1;
            if (k > 0) {
                Ctx::Scope sp(c, PH_PROJ);
                c.b_x(k, bi, B, ldb, n, bf.Z, n, 0.0, bf.T1, k, c.acc_proj);      // B Z
                c.q_t(k, bi, Q, ldq, m, -1.0, bf.T1, k, Y, ldq, c.acc_proj);      // Y -= Q (.)
            }
        }
        if (k > 0) c.cholqr_pre(Y, ldq, m, bi, false);                            // Q_i = orth(Y)
        else c.cholqr2(Y, ldq, m, bi, false);
        if (k > 0) {                                                              // re-orthogonalise
            c.reorth_q(k, Q, ldq, m, Y, ldq, bi, bf.T1);
            c.cholqr2(Y, ldq, m, bi, false);
        }
        // B_i = Q_i^T A, written as rows k.. of B (= column-major n x bi with ld ldb)
        char* Bs = c.col(B, ldb, k);
        A.apply_t(c, Y, ldq, bi, Bs, ldb, 3);
        out.passes += 1;
        c.shadow(k, bi, Y, ldq, m, Bs, ldb, n);
        const Ctx::Step s = c.indicator_step(Bs, ldb, bi, n, eps2, o.row_by_row);
        out.blocks += 1;
        out.E = s.E;
        k += s.keep;
        if (s.stop) { out.converged = true; break; }
    }
    out.rank = k;
}

// ------------------------------------------------------------------------------------ randQB_FP
void run_fp(Ctx& c, AOp& A, const Plan& p, const qb_opts& o, Bufs& bf, void* Q, int64_t ldq,
            void* B, int64_t ldb, double eps2, RunOut& out) {
    const int64_t m = p.m, n = p.n;
    const int omega_dt = c.f64 ? QB_F64 : QB_F32;
    // chunks need every earlier column at the same power iteration as the chunk's own: with one
    // iteration the earlier chunks' G and Omega panels are exactly that; with more, the whole batch
    const bool whole = (o.flags & QB_FLAG_WHOLE_BATCH) != 0 || p.P > 1;
    int64_t k = 0;
    int64_t q = 0;
    bool stop = false;
    while (k < p.cap && !stop) {
        const int64_t w = std::min<int64_t>(p.lt, p.cap - k);
        const int64_t col0 = q * p.lt;
        const int64_t kb = k;   // Q, B at the start of the batch: the implicit residual A - Q B
        // The batch's l~ columns are processed in chunks of FP_CHUNK columns, each carried
        // through the power scheme, G = A Omega and H = A^T G before the blocked loop reaches
        // it.  orth is column-causal (panel Gram-Schmidt / CholeskyQR), so every column comes out
        // as in Algorithm 4 on the whole batch; the chunks after the stopping block are never
        // formed.  QB_FLAG_WHOLE_BATCH forms the whole batch at once: 1 + 2P passes over A for
        // the power scheme and G, plus one per H_CHUNK-column piece of H.
        const int64_t chunk = whole ? w : std::min<int64_t>(FP_CHUNK, w);
        for (int64_t cc = 0; cc < w && !stop; cc += chunk) {
            const int64_t cw = std::min<int64_t>(chunk, w - cc);
            char* Om_c = c.col(bf.Om, n, cc);
            char* G_c = c.col(bf.G, m, cc);
            char* Gp_c = p.P > 0 ? c.col(bf.Gp, m, cc) : nullptr;
            out.omega_cols = col0 + cc + cw;
            omega_gen(c.st, n, col0 + cc, cw, o.seed, omega_dt, Om_c, n);   // Omega = randn(n, l~)
            A.round_operand(c, Om_c, n, n, cw);
            for (int it = 0; it < p.P; ++it) {                                // power scheme
                A.apply(c, Om_c, n, cw, Gp_c, m);                             // G = A Omega
                out.passes += 1;
                if (kb > 0) {
                    c.tn(kb, cw, n, 1.0, B, ldb, Om_c, n, 0.0, bf.T1, kb, c.acc_proj);
                    c.nn(m, cw, kb, -1.0, Q, ldq, bf.T1, kb, 1.0, Gp_c, m, c.acc_proj);
                }
                // G only has to be a well-conditioned basis for the next application of A^T:
                // one Gram-Schmidt pass per panel on the mixed path
                c.orth_wide(bf.Gp, m, m, cc + cw, p.b, bf.Tw, false, cc);      // G = orth(.)
                A.round_operand(c, Gp_c, m, m, cw);
                A.apply_t(c, Gp_c, m, cw, Om_c, n, 1);                        // Omega = A^T G
                out.passes += 1;
                if (kb > 0) {
                    c.tn(kb, cw, m, 1.0, Q, ldq, Gp_c, m, 0.0, bf.T1, kb, c.acc_proj);
                    c.nn(n, cw, kb, -1.0, B, ldb, bf.T1, kb, 1.0, Om_c, n, c.acc_proj);
                }
                c.orth_wide(bf.Om, n, n, cc + cw, p.b, bf.Tw, true, cc);       // Omega = orth(.)
                // The B_i formula cancels the components of H_i = A^T G_i along singular vectors
                // already in Q; a bf16-rounded Omega (2^-9) would leak sigma_1^2-sized terms into
                // every H_i, so the processed Omega keeps two bf16 terms (16 bits).
                A.round_operand(c, Om_c, n, n, cw, 2);
            }
            A.apply(c, Om_c, n, cw, G_c, m, p.P > 0 ? 2 : 1);                 // G = A Omega
            out.passes += 1;
            // The B_i formula needs H = A^T G exactly for the G it uses, not G = A Omega exactly:
            // keep G as two-term bf16 values (16 bits) so the precise pass takes four products
            A.round_operand(c, G_c, m, m, cw, 2);
            // H = A^T G for the stored G, in the precision the B_i formula needs, formed in
            // pieces of at most H_CHUNK columns as the loop reaches them
            int64_t h_done = cc;
            for (int64_t c0 = cc; c0 < cc + cw && !stop; c0 += p.b) {
                const int bi = int(std::min<int64_t>(p.b, cc + cw - c0));
                if (c0 + bi > h_done) {
                    const int64_t hw =
                        std::min<int64_t>(std::max<int64_t>(H_CHUNK, bi), cc + cw - h_done);
                    A.apply_t(c, c.col(bf.G, m, h_done), m, hw, c.col(bf.H, n, h_done), n, 4);
                    // every piece of H is a read of A of its own: G and H are two launches here
                    // (Remark 4.2's single read would need all n x w of H held on chip)
                    out.passes += 1;
                    h_done += hw;
                }
                const char* Om_i = c.col(bf.Om, n, c0);
                // with the tensor-core products, Q^T Q_i (re-orthogonalisation) and Q^T Y_i (B_i
                // formula) come from one pass over Q's shadows: T1 then sits right after the
                // coefficients' bi columns in TT
                const bool merged = k > 0 && bf.TT && c.tcg();
                char* T1 = merged ? bf.TT + size_t(bi) * size_t(k) * c.es : bf.T1;   // ld k
                // Y_i = G_i - Q (B Omega_i), kept for the B_i formula
                c.copy_cols_(c.col(bf.G, m, c0), m, m, bi, bf.Ys, m);
                if (k > 0) {
                    Ctx::Scope sc(c, PH_PROJ);
                    c.b_x(k, bi, B, ldb, n, Om_i, n, 0.0, T1, k, c.acc_proj);
                    c.q_t(k, bi, Q, ldq, m, -1.0, T1, k, bf.Ys, m, c.acc_proj);
                }
                // [Q_i, R_i] = qr(Y_i) in the slot of Q_i; the inverses of the factors go to Rchain
                char* Qi = c.col(Q, ldq, k);
                c.copy_cols_(bf.Ys, m, m, bi, Qi, ldq);
                c.nchain = 0;
                c.chain_fused = false;
                if (k > 0) c.cholqr_pre(Qi, ldq, m, bi, true);
                else c.cholqr2(Qi, ldq, m, bi, true);
                if (k > 0) {
                    // [Q_i, R~_i] = qr(Q_i - Q (Q^T Q_i)), R_i = R~_i R_i
                    if (merged) {
                        Ctx::Scope sp(c, PH_PROJ);
                        QB_CUDA(cudaMemsetAsync(bf.TT, 0, size_t(bi) * size_t(k) * c.es, c.st));
                        c.qt_x2(k, bi, m, Qi, ldq, bf.Ys, m, bf.TT, k);   // T1 += Q^T Y_i too
                        c.q_t(k, bi, Q, ldq, m, -1.0, bf.TT, k, Qi, ldq, c.acc_proj);
                    } else {
                        c.reorth_q(k, Q, ldq, m, Qi, ldq, bi, bf.C2);
                    }
                    c.cholqr2(Qi, ldq, m, bi, true);
                }
                char* Bs = c.col(B, ldb, k);
                {
                    Ctx::Scope scb(c, PH_BFORM);
                    // S^T = H_i - B^T (Q^T Y_i + B Omega_i), i.e. S = H_i^T - Y_i^T Q B - Omega_i^T B^T B,
                    // formed in place in H_i's columns (H_i is read only here)
                    char* S = c.col(bf.H, n, c0);
                    if (k > 0) {
                        // T1 still holds B Omega_i from the projection of Y_i
                        if (!merged)
                            c.qt_x(k, bi, Q, ldq, m, bf.Ys, m, 1.0, T1, k, c.acc_fine); // += Q^T Y_i
                        c.bt_t(k, bi, B, ldb, n, -1.0, T1, k, S, n, c.acc_fine);        // S^T -= B^T T1
                    }
                    // B_i = R_i^-T S  <=>  B_i^T = S^T R_i^-1, R_i the product of the CholeskyQR
                    // factors (R~_2 R~_1 R_1 on the mixed path, R~_2 R~_1 R_2 R_1 on the float64
                    // path): apply their inverses in turn (Rchain, consecutive fused ones merged)
                    for (int f = 0; f < c.nchain; ++f)
                        apply_rinv(c.st, c.f64, S, n, n, bi, c.Rchain + size_t(f) * MAXB * MAXB);
                    c.copy_cols_(S, n, n, bi, Bs, ldb);
                }
                c.shadow(k, bi, Qi, ldq, m, Bs, ldb, n);
                const Ctx::Step s = c.indicator_step(Bs, ldb, bi, n, eps2, o.row_by_row);
                out.blocks += 1;
                out.E = s.E;
                k += s.keep;
                if (s.stop) { stop = true; out.converged = true; }
            }
        }
        ++q;
    }
    out.rank = k;
}

// ------------------------------------------------------------------------------------ common entry
int32_t run_common(AOp& A, const qb_opts* opts, bool fp, void* Q, int64_t ldq, void* B,
                   int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream,
                   size_t* measure) {
    if (!valid_opts(opts)) return QB_ERR_INVALID_ARG;
    const qb_opts& o = *opts;
    if (A.m < 0 || A.n < 0) return QB_ERR_INVALID_ARG;
    const Plan p = make_plan(A.m, A.n, o, fp);
    Ctx c;
    setup_ctx(c, o.prec == QB_PREC_FP64);
    c.simt_apass = (o.flags & QB_FLAG_SIMT_APASS) != 0;
    c.prof = (o.flags & QB_FLAG_PROFILE) != 0;
    c.st = reinterpret_cast<cudaStream_t>(stream);
    Bufs bf;
    Arena ar;
    if (measure) {
        reserve_all(ar, c, A, p, fp, bf);
        *measure = ar.used + 4096;
        return QB_OK;
    }
    if (!Q || !B || ldq < A.m || ldb < A.n) return QB_ERR_INVALID_ARG;
    ar.base = reinterpret_cast<char*>(ws);
    ar.cap = ws_bytes;
    const int64_t l0 = launches_total();
    reserve_all(ar, c, A, p, fp, bf);
    QB_CUDA(cudaMemsetAsync(c.flags, 0, 8 * sizeof(int), c.st));
    A.prepare(c);
    const double normA2 = A.norm2(c);
    int hf[4];
    c.read_flags(hf);
    RunOut out;
    out.normA2 = normA2;
    auto fill_info = [&](int32_t bits) {
        if (!info) return;
        info->rank = out.rank;
        info->err2_est = out.E;
        info->err_est = std::sqrt(std::max(out.E, 0.0));
        info->normA2 = out.normA2;
        info->passes = out.passes;
        info->omega_cols = out.omega_cols;
        info->status_bits = bits;
        info->blocks = out.blocks;
        info->launches = launches_total() - l0;
    };
    if (hf[0] || !std::isfinite(normA2)) {
        fill_info(0);
        return QB_ERR_NONFINITE;
    }
    const double eps = o.relative ? o.tol * std::sqrt(normA2) : o.tol;
    // Theorem 3 bounds the rounding error of E by 2u(||A||^2 + ||B||^2).  ||A||^2 is exact to
    // float64 here; on the mixed path the rows of B carry float32 rounding (u = 2^-24), so the
    // stop test keeps a margin 2 u ||A||^2 >= 2 u ||B||^2 to guarantee ||A - QB|| < eps.
    const double u_work = o.prec == QB_PREC_FP64 ? U64 : U32;
    const double margin = o.prec == QB_PREC_FP64 ? 0.0 : 2.0 * U32 * normA2;
    const double eps2 = eps * eps - margin;
    if (normA2 == 0.0 || p.cap == 0) {
        out.E = normA2;
        out.converged = normA2 < eps * eps || normA2 == 0.0;
        fill_info(out.converged ? 0 : QB_BIT_NOT_CONVERGED);
        return out.converged ? QB_OK : QB_NOT_CONVERGED;
    }
    double st0[4] = {normA2, 0, 0, normA2};
    QB_CUDA(cudaMemcpyAsync(c.state, st0, sizeof st0, cudaMemcpyHostToDevice, c.st));
    if (fp) run_fp(c, A, p, o, bf, Q, ldq, B, ldb, eps2, out);
    else run_ei(c, A, p, o, bf, Q, ldq, B, ldb, eps2, out);
    c.flush_profile();
    c.read_flags(hf);
    if (A.timed_out(c) || hf[2]) {
        fill_info(0);
        return QB_ERR_TIMEOUT;
    }
    int32_t bits = 0;
    if (hf[1]) bits |= QB_BIT_BREAKDOWN;
    const double floor = std::sqrt(4.0 * u_work / THM3_DELTA) * std::sqrt(normA2);
    int32_t status = QB_OK;
    if (!out.converged) {
        bits |= QB_BIT_NOT_CONVERGED;
        status = QB_NOT_CONVERGED;
    } else if (eps <= floor) {
        bits |= QB_BIT_TOL_FLOOR;
        status = QB_WARN_TOL_FLOOR;
    }
    fill_info(bits);
    return status;
}

// ------------------------------------------------------------------------------------ fixed-rank map
// The fixed-rank QB map A -> (Q, B) with Omega fixed (Omega = Philox columns 0..k-1): Y = A Omega,
// Y = Q R (diag R > 0), B = Q^T A.  In exact arithmetic this is k columns of randQB / EI / FP at
// P = 0 (Proposition 2); the QR is blocked (Gram-Schmidt with re-orthogonalisation over panels of
// 64, CholeskyQR2 per panel) and keeps R.
struct FixedBufs {
    char* Om = nullptr;   // n x k
    char* T = nullptr;    // k x 64
    char* M = nullptr;    // k x k
    char* C = nullptr;    // k x k
    char* Ri = nullptr;   // k x k
    char* Qb = nullptr;   // m x k
    char* Yb = nullptr;   // m x k
    char* Qt = nullptr;   // k x m
    char* Gb = nullptr;   // n x k (mixed: rounded copy of G_B^T)
    bf16* P1 = nullptr;   // mixed, tensor-core path: n x kp rows [G_B^T hi | G_B^T lo | Omega | 0]
    bf16* P2h = nullptr;  // m x kp rows [Q | Q | Ybar | 0], bf16 hi terms ...
    bf16* P2l = nullptr;  // ... and lo terms
    int64_t kp = 0;
};

void fixed_reserve(Arena& ar, Ctx& c, DenseOp& A, int64_t k, FixedBufs& f, bool bwd) {
    const int64_t m = A.m, n = A.n, es = int64_t(c.es);
    c.alloc(ar, std::max({m, n, k}) * std::max<int64_t>(k, 64));
    f.Om = ar.get<char>(n * k * es);
    f.T = ar.get<char>(k * MAXB * es);
    if (bwd) {
        f.M = ar.get<char>(k * k * es);
        f.C = ar.get<char>(k * k * es);
        f.Ri = ar.get<char>(k * k * es);
        f.Qb = ar.get<char>(m * k * es);
        f.Yb = ar.get<char>(m * k * es);
        f.Qt = ar.get<char>(k * m * es);
        f.Gb = ar.get<char>(n * k * es);
    }
    A.reserve(ar, c, k);
    if (!c.f64 && A.tc_scratch(&c.tcs, &c.tcs_bytes)) {
        // three-term bf16 shadows of the finished panels of Q: the forward's Gram-Schmidt
        // projections run on the tensor cores at float32 accuracy
        c.ldqs = align_up(m, 8);
        for (int t = 0; t < 3; ++t) c.qs[t] = ar.get<bf16>(c.ldqs * k);
    }
    if (bwd && A.use_tc && n >= 128 && m >= 1) {
        f.kp = std::max<int64_t>(align_up(3 * k, 64), 128);   // at least one 128-wide K tile
        f.P1 = ar.get<bf16>(n * f.kp);
        f.P2h = ar.get<bf16>(m * f.kp);
        f.P2l = ar.get<bf16>(m * f.kp);
    }
}

void fixed_fwd(Ctx& c, DenseOp& A, int64_t k, uint64_t seed, FixedBufs& f, void* Q, int64_t ldq,
               void* B, int64_t ldb, void* R, int64_t ldr) {
    const int64_t m = A.m, n = A.n;
    omega_gen(c.st, n, 0, k, seed, c.f64 ? QB_F64 : QB_F32, f.Om, n);
    A.round_operand(c, f.Om, n, n, k, 1);                       // the map's Omega (bf16 on the mixed path)
    A.apply(c, f.Om, n, k, Q, ldq, 1);                          // Y = A Omega, in Q
    QB_CUDA(cudaMemset2DAsync(R, size_t(ldr) * c.es, 0, size_t(k) * c.es, size_t(k), c.st));
    for (int64_t j0 = 0; j0 < k; j0 += MAXB) {
        const int bj = int(std::min<int64_t>(MAXB, k - j0));
        char* Pj = c.col(Q, ldq, j0);
        char* Rj = c.col(R, ldr, j0);                           // R(0:j0, j0:j0+bj)
        if (j0 > 0) {
            for (int pass = 0; pass < 2; ++pass) {              // Gram-Schmidt, then re-orthogonalise
                c.qt_x(j0, bj, Q, ldq, m, Pj, ldq, 0.0, f.T, j0, c.acc_fine);
                c.q_t(j0, bj, Q, ldq, m, -1.0, f.T, j0, Pj, ldq, c.acc_proj);
                axpy(c.st, c.f64, j0, bj, 1.0, f.T, j0, Rj, ldr);
            }
        }
        char* Rjj = reinterpret_cast<char*>(Rj) + size_t(j0) * c.es;
        if (c.coop_rinv(Pj, ldq, m, bj)) {                      // Q_j R_jj = P_j
            tri_inv_from_f64(c.st, false, c.Rinv, MAXB, bj, Rjj, ldr);
        } else {
            set_identity(c.st, c.Racc, bj);
            c.cholqr_racc(Pj, ldq, m, bj);
            c.cholqr_racc(Pj, ldq, m, bj);
            from_f64(c.st, c.f64, c.Racc, MAXB, bj, bj, Rjj, ldr);
        }
        if (c.tcg() && j0 + bj < k)
            split3_bf16(c.st, reinterpret_cast<const float*>(Pj), ldq, m, bj, c.qs[0] + j0 * c.ldqs,
                        c.qs[1] + j0 * c.ldqs, c.qs[2] + j0 * c.ldqs, c.ldqs);
    }
    A.apply_t(c, Q, ldq, k, B, ldb, 3);                         // B = Q^T A
}

// Abar = Q G_B + Ybar Omega^T with Qbar = G_Q + A G_B^T, M = -Qbar^T Q,
// Ybar = (Qbar + Q copyltu(M)) R^-T (reverse mode through B = Q^T A, Y = Q R, Y = A Omega).
void fixed_bwd(Ctx& c, DenseOp& A, int64_t k, uint64_t seed, FixedBufs& f, const void* Q,
               int64_t ldq, const void* R, int64_t ldr, const void* GQ, int64_t ldgq,
               const void* GB, int64_t ldgb, void* GA, int64_t ldga) {
    const int64_t m = A.m, n = A.n;
    omega_gen(c.st, n, 0, k, seed, c.f64 ? QB_F64 : QB_F32, f.Om, n);
    A.round_operand(c, f.Om, n, n, k, 1);
    // Qbar = G_Q + A G_B^T  (G_B row-major k x n = column-major n x k)
    c.copy_cols_(GB, ldgb, n, k, f.Gb, n);
    A.round_operand(c, f.Gb, n, n, k, 2);
    A.apply(c, f.Gb, n, k, f.Qb, m, 2);
    axpy(c.st, c.f64, m, k, 1.0, GQ, ldgq, f.Qb, m);
    // M = -Qbar^T Q; C = copyltu(M); Z = Qbar + Q C (in Qbar)
    c.tn(k, k, m, -1.0, f.Qb, m, Q, ldq, 0.0, f.M, k, c.acc_fine);
    copyltu(c.st, c.f64, f.M, k, f.C);
    c.nn(m, k, k, 1.0, Q, ldq, f.C, k, 1.0, f.Qb, m, c.acc_proj);
    // Ybar = Z R^-T  =  Z (R^-1)^T
    tri_inv_big(c.st, c.f64, R, ldr, k, f.Ri, k);
    transpose(c.st, c.f64, f.Ri, k, k, k, f.M, k);              // M <- R^-T
    c.nn(m, k, k, 1.0, f.Qb, m, f.M, k, 0.0, f.Yb, m, c.acc_proj);
    if (f.P1) {
        // Abar = Q G_B + Ybar Omega^T as ONE tensor-core product with K = 3k: Abar^T (n x m,
        // column-major = Abar row-major) = [G_B^T hi | G_B^T lo | Omega] [Q | Q | Ybar]^T, the
        // right factor in two bf16 terms (two products); G_B's lo term carries its float32 part,
        // Omega is bf16-valued on this path (exact).  Padding columns are zero on both sides.
        const int64_t kp = f.kp;
        if (kp > 3 * k) {      // zero padding columns (the packs write the rest)
            const size_t pw = sizeof(bf16) * size_t(kp - 3 * k), pitch = sizeof(bf16) * size_t(kp);
            QB_CUDA(cudaMemset2DAsync(f.P1 + 3 * k, pitch, 0, pw, size_t(n), c.st));
            QB_CUDA(cudaMemset2DAsync(f.P2h + 3 * k, pitch, 0, pw, size_t(m), c.st));
            QB_CUDA(cudaMemset2DAsync(f.P2l + 3 * k, pitch, 0, pw, size_t(m), c.st));
        }
        const float* gb = reinterpret_cast<const float*>(GB);
        pack_rows_bf16(c.st, gb, ldgb, n, k, f.P1, nullptr, kp, 0);
        pack_rows_bf16(c.st, gb, ldgb, n, k, nullptr, f.P1, kp, k);     // G_B's lo term
        pack_rows_bf16(c.st, reinterpret_cast<const float*>(f.Om), n, n, k, f.P1, nullptr, kp,
                       2 * k);
        const float* qf = reinterpret_cast<const float*>(Q);
        pack_rows_bf16(c.st, qf, ldq, m, k, f.P2h, f.P2l, kp, 0);
        pack_rows_bf16(c.st, qf, ldq, m, k, f.P2h, f.P2l, kp, k);
        pack_rows_bf16(c.st, reinterpret_cast<const float*>(f.Yb), m, m, k, f.P2h, f.P2l, kp,
                       2 * k);
        tc_sketch(c.st, f.P1, kp, n, kp, f.P2h, f.P2l, kp, m, reinterpret_cast<float*>(GA), ldga,
                  A.tc_scr, A.tc_bytes);
        return;
    }
    // Abar^T (n x m, column-major = Abar row-major) = G_B^T Q^T + Omega Ybar^T
    transpose(c.st, c.f64, Q, ldq, m, k, f.Qt, k);
    c.nn(n, m, k, 1.0, GB, ldgb, f.Qt, k, 0.0, GA, ldga, c.acc_proj);
    transpose(c.st, c.f64, f.Yb, m, m, k, f.Qt, k);
    c.nn(n, m, k, 1.0, f.Om, n, f.Qt, k, 1.0, GA, ldga, c.acc_proj);
}

template <class F>
int32_t guarded(F&& f) {
    try {
        return f();
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return QB_ERR_CUDA;
    }
}

bool valid_dense(const qb_dense* A, const qb_opts* o) {
    if (!A || !o || A->m < 0 || A->n < 0 || A->ld < A->n || !A->a) return false;
    if (A->dtype == QB_BF16X2 && !A->a_lo) return false;
    if (o->prec == QB_PREC_FP64 && A->dtype != QB_F64) return false;
    if (o->prec == QB_PREC_MIXED && A->dtype == QB_F64) return false;
    return A->dtype >= QB_F64 && A->dtype <= QB_BF16X2;
}

bool valid_csr(const qb_csr* A, const qb_opts* o) {
    if (!A || !o || A->m < 0 || A->n < 0 || A->nnz < 0 || A->nnz > INT32_MAX) return false;
    if (!A->rowptr || (A->nnz > 0 && (!A->colind || !A->val))) return false;
    if (A->dtype != QB_F64 && A->dtype != QB_F32) return false;
    if (o->prec == QB_PREC_FP64 && A->dtype != QB_F64) return false;
    if (o->prec == QB_PREC_MIXED && A->dtype != QB_F32) return false;
    return true;
}

bool valid_coo(const qb_coo* A, const qb_opts* o) {
    if (!A || !o || A->m < 0 || A->n < 0 || A->nnz < 0 || A->nnz > INT32_MAX) return false;
    if (A->nnz > 0 && (!A->row || !A->col || !A->val)) return false;
    if (A->dtype != QB_F64 && A->dtype != QB_F32) return false;
    if (o->prec == QB_PREC_FP64 && A->dtype != QB_F64) return false;
    if (o->prec == QB_PREC_MIXED && A->dtype != QB_F32) return false;
    return true;
}

}  // namespace

}  // namespace qb

// ======================================================================================== C ABI
using namespace qb;

extern "C" {

const char* qb_status_str(int32_t s) {
    switch (s) {
        case QB_OK: return "QB_OK";
        case QB_NOT_CONVERGED: return "QB_NOT_CONVERGED";
        case QB_WARN_TOL_FLOOR: return "QB_WARN_TOL_FLOOR";
        case QB_ERR_INVALID_ARG: return "QB_ERR_INVALID_ARG";
        case QB_ERR_NONFINITE: return "QB_ERR_NONFINITE";
        case QB_ERR_CUDA: return "QB_ERR_CUDA";
        case QB_ERR_BREAKDOWN: return "QB_ERR_BREAKDOWN";
        case QB_ERR_WORKSPACE: return "QB_ERR_WORKSPACE";
        case QB_ERR_TIMEOUT: return "QB_ERR_TIMEOUT";
        case QB_ERR_UNSUPPORTED: return "QB_ERR_UNSUPPORTED";
        default: return "QB_UNKNOWN_STATUS";
    }
}

const char* qb_last_cuda_error(void) { return g_last_err; }

int64_t qb_launch_count(void) { return launches_total(); }

int32_t qb_profile_last(double* ms, int32_t n) {
    if (!ms || n < 0) return QB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int i = 0; i < n && i < PH_COUNT; ++i) ms[i] = g_prof_ms[i];
    return PH_COUNT;
}

size_t qb_dense_workspace(const qb_dense* A, const qb_opts* opts, int32_t algo) {
    if (!valid_dense(A, opts) || !valid_opts(opts) || (algo != 0 && algo != 1)) return 0;
    size_t bytes = 0;
    DenseOp op(*A);
    int32_t rc = guarded([&] {
        return run_common(op, opts, algo == 1, nullptr, 0, nullptr, 0, nullptr, 0, nullptr,
                          nullptr, &bytes);
    });
    return rc == QB_OK ? bytes : 0;
}

int32_t qb_ei_dense(const qb_dense* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                    int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream) {
    if (!valid_dense(A, opts)) return QB_ERR_INVALID_ARG;
    DenseOp op(*A);
    return guarded([&] {
        return run_common(op, opts, false, Q, ldq, B, ldb, ws, ws_bytes, info, stream, nullptr);
    });
}

int32_t qb_fp_dense(const qb_dense* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                    int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream) {
    if (!valid_dense(A, opts)) return QB_ERR_INVALID_ARG;
    DenseOp op(*A);
    return guarded([&] {
        return run_common(op, opts, true, Q, ldq, B, ldb, ws, ws_bytes, info, stream, nullptr);
    });
}

size_t qb_csr_workspace(const qb_csr* A, const qb_opts* opts, int32_t algo) {
    if (!valid_csr(A, opts) || !valid_opts(opts) || (algo != 0 && algo != 1)) return 0;
    size_t bytes = 0;
    CsrOp op(*A);
    int32_t rc = guarded([&] {
        return run_common(op, opts, algo == 1, nullptr, 0, nullptr, 0, nullptr, 0, nullptr,
                          nullptr, &bytes);
    });
    return rc == QB_OK ? bytes : 0;
}

int32_t qb_ei_csr(const qb_csr* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                  int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream) {
    if (!valid_csr(A, opts)) return QB_ERR_INVALID_ARG;
    CsrOp op(*A);
    return guarded([&] {
        return run_common(op, opts, false, Q, ldq, B, ldb, ws, ws_bytes, info, stream, nullptr);
    });
}

int32_t qb_fp_csr(const qb_csr* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                  int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream) {
    if (!valid_csr(A, opts)) return QB_ERR_INVALID_ARG;
    CsrOp op(*A);
    return guarded([&] {
        return run_common(op, opts, true, Q, ldq, B, ldb, ws, ws_bytes, info, stream, nullptr);
    });
}

size_t qb_coo_workspace(const qb_coo* A, const qb_opts* opts, int32_t algo) {
    if (!valid_coo(A, opts) || !valid_opts(opts) || (algo != 0 && algo != 1)) return 0;
    size_t bytes = 0;
    CooOp op(*A);
    int32_t rc = guarded([&] {
        return run_common(op, opts, algo == 1, nullptr, 0, nullptr, 0, nullptr, 0, nullptr,
                          nullptr, &bytes);
    });
    return rc == QB_OK ? bytes : 0;
}

int32_t qb_ei_coo(const qb_coo* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                  int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream) {
    if (!valid_coo(A, opts)) return QB_ERR_INVALID_ARG;
    CooOp op(*A);
    return guarded([&] {
        return run_common(op, opts, false, Q, ldq, B, ldb, ws, ws_bytes, info, stream, nullptr);
    });
}

int32_t qb_fp_coo(const qb_coo* A, const qb_opts* opts, void* Q, int64_t ldq, void* B,
                  int64_t ldb, void* ws, size_t ws_bytes, qb_info* info, void* stream) {
    if (!valid_coo(A, opts)) return QB_ERR_INVALID_ARG;
    CooOp op(*A);
    return guarded([&] {
        return run_common(op, opts, true, Q, ldq, B, ldb, ws, ws_bytes, info, stream, nullptr);
    });
}

int32_t qb_omega(int64_t n, int64_t col0, int64_t w, uint64_t seed, int32_t dtype, void* out,
                 int64_t ld, void* stream) {
    if (n < 0 || col0 < 0 || w < 0 || ld < n || (n > 0 && w > 0 && !out)) return QB_ERR_INVALID_ARG;
    if (dtype != QB_F64 && dtype != QB_F32 && dtype != QB_BF16) return QB_ERR_INVALID_ARG;
    return guarded([&] {
        omega_gen(reinterpret_cast<cudaStream_t>(stream), n, col0, w, seed, dtype, out, ld);
        return int32_t(QB_OK);
    });
}

size_t qb_apass_workspace(const qb_dense* A, int64_t w) {
    if (!A || A->m < 0 || A->n < 0 || w < 0) return 0;
    qb_opts o{};
    o.b = 1;
    o.prec = A->dtype == QB_F64 ? QB_PREC_FP64 : QB_PREC_MIXED;
    if (!valid_dense(A, &o)) return 0;
    try {
        Ctx c;
        setup_ctx(c, o.prec == QB_PREC_FP64);
        Arena ar;   // measuring arena
        c.alloc(ar, std::max(A->m, A->n) * std::max<int64_t>(w, 1));
        DenseOp op(*A);
        op.reserve(ar, c, std::max<int64_t>(w, 1));
        return ar.used + 4096;
    } catch (...) {
        return 0;
    }
}

static int32_t apass(const qb_dense* A, bool trans, const void* V, int64_t ldv, int64_t w,
                     int32_t precise, void* Y, int64_t ldy, void* ws, size_t ws_bytes,
                     void* stream) {
    qb_opts o{};
    o.b = 1;
    o.prec = (A && A->dtype == QB_F64) ? QB_PREC_FP64 : QB_PREC_MIXED;
    if (!valid_dense(A, &o) || w < 0 || !V || !Y) return QB_ERR_INVALID_ARG;
    const int64_t rows_in = trans ? A->m : A->n, rows_out = trans ? A->n : A->m;
    if (ldv < rows_in || ldy < rows_out) return QB_ERR_INVALID_ARG;
    return guarded([&] {
        Ctx c;
        setup_ctx(c, o.prec == QB_PREC_FP64);
        c.st = reinterpret_cast<cudaStream_t>(stream);
        Arena ar;
        ar.base = reinterpret_cast<char*>(ws);
        ar.cap = ws_bytes;
        c.alloc(ar, std::max(A->m, A->n) * std::max<int64_t>(w, 1));
        DenseOp op(*A);
        op.reserve(ar, c, std::max<int64_t>(w, 1));
        op.prepare(c);
        c.prof = true;   // the pass's device time, read back with qb_profile_last
        if (trans)
            op.apply_t(c, V, ldv, w, Y, ldy,
                       precise == 0 ? 1 : (precise == 2 ? 2 : (precise == 3 ? 4 : 3)));
        else op.apply(c, V, ldv, w, Y, ldy, 1);
        const bool to = op.timed_out(c);
        c.flush_profile();
        return int32_t(to ? QB_ERR_TIMEOUT : QB_OK);
    });
}

int32_t qb_apass_sketch(const qb_dense* A, const void* V, int64_t ldv, int64_t w, void* Y,
                        int64_t ldy, void* ws, size_t ws_bytes, void* stream) {
    return apass(A, false, V, ldv, w, 0, Y, ldy, ws, ws_bytes, stream);
}

int32_t qb_apass_trans(const qb_dense* A, const void* V, int64_t ldv, int64_t w, int32_t precise,
                       void* Z, int64_t ldz, void* ws, size_t ws_bytes, void* stream) {
    return apass(A, true, V, ldv, w, precise, Z, ldz, ws, ws_bytes, stream);
}

static bool valid_fixed(const qb_dense* A, int64_t k, int32_t prec) {
    qb_opts o{};
    o.b = 1;
    o.prec = prec;
    return (prec == QB_PREC_FP64 || prec == QB_PREC_MIXED) && valid_dense(A, &o) && k >= 1 &&
           k <= std::min(A->m, A->n);
}

size_t qb_fixed_rank_workspace(const qb_dense* A, int64_t k, int32_t prec) {
    if (!valid_fixed(A, k, prec)) return 0;
    try {
        Ctx c;
        setup_ctx(c, prec == QB_PREC_FP64);
        Arena ar;
        DenseOp op(*A);
        FixedBufs f;
        fixed_reserve(ar, c, op, k, f, true);
        return ar.used + 4096;
    } catch (...) {
        return 0;
    }
}

int32_t qb_fixed_rank_fwd(const qb_dense* A, int64_t k, uint64_t seed, int32_t prec, void* Q,
                          int64_t ldq, void* B, int64_t ldb, void* R, int64_t ldr, void* ws,
                          size_t ws_bytes, void* stream) {
    if (!valid_fixed(A, k, prec) || !Q || !B || !R || ldq < A->m || ldb < A->n || ldr < k)
        return QB_ERR_INVALID_ARG;
    return guarded([&] {
        Ctx c;
        setup_ctx(c, prec == QB_PREC_FP64);
        c.st = reinterpret_cast<cudaStream_t>(stream);
        Arena ar;
        ar.base = reinterpret_cast<char*>(ws);
        ar.cap = ws_bytes;
        DenseOp op(*A);
        FixedBufs f;
        fixed_reserve(ar, c, op, k, f, false);
        QB_CUDA(cudaMemsetAsync(c.flags, 0, 8 * sizeof(int), c.st));
        op.prepare(c);
        fixed_fwd(c, op, k, seed, f, Q, ldq, B, ldb, R, ldr);
        if (op.timed_out(c)) return int32_t(QB_ERR_TIMEOUT);
        QB_CUDA(cudaStreamSynchronize(c.st));
        return int32_t(QB_OK);
    });
}

int32_t qb_fixed_rank_bwd(const qb_dense* A, int64_t k, uint64_t seed, int32_t prec,
                          const void* Q, int64_t ldq, const void* R, int64_t ldr, const void* GQ,
                          int64_t ldgq, const void* GB, int64_t ldgb, void* GA, int64_t ldga,
                          void* ws, size_t ws_bytes, void* stream) {
    if (!valid_fixed(A, k, prec) || !Q || !R || !GQ || !GB || !GA || ldq < A->m || ldr < k ||
        ldgq < A->m || ldgb < A->n || ldga < A->n)
        return QB_ERR_INVALID_ARG;
    return guarded([&] {
        Ctx c;
        setup_ctx(c, prec == QB_PREC_FP64);
        c.st = reinterpret_cast<cudaStream_t>(stream);
        Arena ar;
        ar.base = reinterpret_cast<char*>(ws);
        ar.cap = ws_bytes;
        DenseOp op(*A);
        FixedBufs f;
        fixed_reserve(ar, c, op, k, f, true);
        op.prepare(c);
        fixed_bwd(c, op, k, seed, f, Q, ldq, R, ldr, GQ, ldgq, GB, ldgb, GA, ldga);
        if (op.timed_out(c)) return int32_t(QB_ERR_TIMEOUT);
        QB_CUDA(cudaStreamSynchronize(c.st));
        return int32_t(QB_OK);
    });
}

size_t qb_quantize_workspace(int64_t, int64_t) { return (3 * 1024 + 8) * sizeof(double); }

int32_t qb_quantize_bf16x2(const double* src, int64_t m, int64_t n, int64_t ld_src, void* hi,
                           void* lo, int64_t ld, double* norms, void* ws, size_t ws_bytes,
                           void* stream) {
    if (m < 0 || n < 0 || ld_src < n || ld < n || !norms) return QB_ERR_INVALID_ARG;
    if (m > 0 && n > 0 && (!src || !hi || !lo)) return QB_ERR_INVALID_ARG;
    if (!ws || ws_bytes < qb_quantize_workspace(m, n)) return QB_ERR_WORKSPACE;
    return guarded([&] {
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        double* part = reinterpret_cast<double*>(ws);   // 3 x 1024 partial sums
        double* res = part + 3 * 1024;                 // 3 results
        quantize_bf16x2(st, src, m, n, ld_src, reinterpret_cast<bf16*>(hi),
                        reinterpret_cast<bf16*>(lo), ld, part, res);
        QB_CUDA(cudaMemcpyAsync(norms, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        QB_CUDA(cudaStreamSynchronize(st));
        return int32_t(QB_OK);
    });
}

}  // extern "C"
