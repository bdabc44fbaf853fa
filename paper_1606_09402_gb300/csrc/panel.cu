// CholeskyQR panel pieces (b x b float64 Cholesky, triangular inverse, R accumulation, applying
// R^-1 to an m x b panel) and the Frobenius-norm indicator of Theorem 1 with the row-by-row
// stopping rule of Sect. 3.1.
#include "qb_internal.cuh"

namespace qb {
namespace {

constexpr int LDS = MAXB + 1;

// Cholesky of a bi x bi Gram W (bi <= 64) by one CTA (at least CHOL_THREADS threads): W = R^T R
// (upper R) factored in TF, R^-1 formed in TI.
// Breakdown: a pivot d <= tau_rel * max_diag(W) (or NaN) is replaced by tau_rel * max_diag (or
// the smallest normal number) and flags[1] is raised; the column it produces has norm <= 1.
//
// One elimination sweep gives both factors: W = L D L^T (L unit lower), R = D^1/2 L^T and
// R^-1 = L^-T D^-1/2.  Step j removes row j from the rows a > j of [W | I] (Gaussian elimination
// without pivoting, multipliers m_a = W[j][a] / d_j read from the symmetric upper part), so the
// trailing upper triangle becomes the Schur complement and the right half becomes L^-1.
//
// Work split: the 64 x 64 matrices are cut into 4 x 4 tiles held in registers.  Threads 0..135
// own the upper tiles of W in row-major order (so the tiles that are finished form a prefix and
// whole warps drop out), threads 160..295 the lower tiles of L^-1.  After step j the owners of
// row j + 1 publish it (W in TF and in TI, L^-1 in TI) to shared memory, the owner of its diagonal
// also its pivot; one barrier per step.
constexpr int CLD = MAXB + 4;          // shared row stride: rows stay 16-byte aligned
// Pivot test of the adaptive factorisation: a float32 factor is kept when every pivot keeps at
// least this fraction of its column's squared norm (kappa of the panel below about 100, so the
// float32 factor leaves the first CholeskyQR pass orthogonal to ~64 u32 kappa^2 < 0.04 and the
// second pass restores it); otherwise the panel is refactored in float64.
constexpr double CHOL_WEAK_REL = 1e-4;
constexpr int CHOL_THREADS = 320;
constexpr int CHOL_TILES = 136;        // 4 x 4 tiles in a triangle of the 16 x 16 tile grid
constexpr int CHOL_L0 = 160;           // first thread of the L^-1 tiles

template <class TF, class TI>
struct CholShared {
    TF (*S)[CLD];    // rows W'[j][.] of the elimination as they are finished (TF)
    TI (*Sf)[CLD];   // the same rows in TI (multipliers of the L^-1 update)
    TI (*Li)[CLD];   // rows of L^-1 as they are finished
    TF* dpiv;        // [MAXB] pivots d_j
    TF* invd;        // [MAXB] 1 / d_j
    TF* idiag;       // [MAXB] 1 / sqrt(d_j)
    TF* diag0;       // [MAXB] diagonal of W
    TF* dmax;        // [1]
    int* weak;       // [1] set when some pivot fell below weak_rel * W[j][j]
};

// tile t of a triangle of the 16 x 16 tile grid, row-major: (ti, tj) with ti <= tj
__device__ __forceinline__ void tri_tile(int t, int& ti, int& tj) {
    ti = 0;
    while (t >= 16 - ti) { t -= 16 - ti; ++ti; }
    tj = ti + t;
}

template <class T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = p[q];
}
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
template <class T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = v[q];
}
template <>
__device__ __forceinline__ void st4<float>(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// load(i, j) returns W[i][j] for i <= j < bi.  On return (after a barrier) S rows hold W'[j][.]
// in their upper part, dpiv / idiag the pivots, and an L^-1 tile owner (threadIdx.x in
// [CHOL_L0, CHOL_L0 + 136)) has in l[r][q] the entry L^-1[4 lr + r][4 lc + q] (lr >= lc).
// weak_rel > 0: *sh.weak is set when a pivot d_j < weak_rel * W[j][j] (a conditioning test).
//
// The tile updates need no per-element predicates: the multiplier of a row a <= j is zero, the
// entries of row j beyond bi are zero, row j of L^-1 is zero beyond column j, and the lower part
// of the diagonal tiles of W (which picks up rounding garbage) is never read.
template <class TF, class TI, class Load>
__device__ void chol_core(int bi, double tau_rel, double weak_rel, int* flags, Load load,
                          CholShared<TF, TI> sh, TI (&l)[4][4], int& lr, int& lc) {
    TF (*S)[CLD] = sh.S;
    TI (*Sf)[CLD] = sh.Sf;
    TI (*Li)[CLD] = sh.Li;
    const int tid = threadIdx.x;
    const bool wown = tid < CHOL_TILES;
    const bool lown = tid >= CHOL_L0 && tid < CHOL_L0 + CHOL_TILES;
    int wi = 0, wj = 0;                // W tile (rows 4 wi.., cols 4 wj..), wi <= wj
    if (wown) tri_tile(tid, wi, wj);
    lr = 0;
    lc = 0;                            // L^-1 tile (rows 4 lr.., cols 4 lc..), lr >= lc
    if (lown) tri_tile(tid - CHOL_L0, lc, lr);
    TF w[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int a = 4 * wi + r, c = 4 * wj + q;
            w[r][q] = (wown && a <= c && c < bi) ? TF(load(a, c)) : TF(0);
            const int la = 4 * lr + r, lcc = 4 * lc + q;
            l[r][q] = (lown && la == lcc && la < bi) ? TI(1) : TI(0);
        }
    if (wown) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            TI f[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) f[q] = TI(w[r][q]);
            st4(&S[4 * wi + r][4 * wj], w[r]);
            st4(&Sf[4 * wi + r][4 * wj], f);
            if (wi == wj) sh.diag0[4 * wi + r] = w[r][r];
        }
    }
    if (lown) {
#pragma unroll
        for (int r = 0; r < 4; ++r) st4(&Li[4 * lr + r][4 * lc], l[r]);
    }
    if (tid == 0) sh.weak[0] = 0;
    __syncthreads();
    if (tid < 32) {
        TF m = TF(0);
        for (int i = tid; i < bi; i += 32) m = sh.diag0[i] > m ? sh.diag0[i] : m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const TF v = __shfl_xor_sync(0xffffffffu, m, o);
            m = v > m ? v : m;
        }
        if (tid == 0) sh.dmax[0] = m;
    }
    __syncthreads();
    const TF dmax = sh.dmax[0];
    const TF tiny = sizeof(TF) == 8 ? TF(2.2250738585072014e-308) : TF(1.1754943508222875e-38);
    const TF floor_piv = TF(tau_rel) * dmax > tiny ? TF(tau_rel) * dmax : tiny;
    // pivot of row j from its (updated) diagonal value; called by one thread
    auto pivot = [&](int j, TF d) {
        if (!(d >= TF(weak_rel) * sh.diag0[j])) sh.weak[0] = 1;
        if (!(d > TF(tau_rel) * dmax)) {
            d = floor_piv;
            sh.weak[0] = 1;
            if (flags) atomicOr(flags + 1, 1);
        }
        sh.dpiv[j] = d;
        sh.invd[j] = TF(1) / d;
    };
    if (tid == 0 && bi > 0) pivot(0, S[0][0]);
    __syncthreads();
    for (int j = 0; j < bi; ++j) {
        const int jn = j + 1;
        if (wown && 4 * wi + 3 > j) {
            // W'[a][c] -= W'[j][a] * (W'[j][c] / d_j) for j < a <= c
            const TF inv = sh.invd[j];
            TF m[4], t[4];
            ld4(&S[j][4 * wi], m);
            ld4(&S[j][4 * wj], t);
#pragma unroll
            for (int r = 0; r < 4; ++r) m[r] = 4 * wi + r > j ? m[r] : TF(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) t[q] *= inv;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) w[r][q] = fma(-m[r], t[q], w[r][q]);
            if ((jn >> 2) == wi) {
                const int r = jn & 3;
                TF v[4];
                TI f[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[q] = r == 0 ? w[0][q] : r == 1 ? w[1][q] : r == 2 ? w[2][q] : w[3][q];
                    f[q] = TI(v[q]);
                }
                st4(&S[jn][4 * wj], v);
                st4(&Sf[jn][4 * wj], f);
                if (wi == wj && jn < bi) pivot(jn, r == 0 ? v[0] : r == 1 ? v[1] : r == 2 ? v[2] : v[3]);
            }
        }
        if (lown && 4 * lr + 3 > j && 4 * lc <= j) {
            // L^-1[a][c] -= (W'[j][a] / d_j) * L^-1[j][c] for a > j >= c
            const TI inv = TI(sh.invd[j]);
            TI m[4], u[4];
            ld4(&Sf[j][4 * lr], m);
            ld4(&Li[j][4 * lc], u);
#pragma unroll
            for (int r = 0; r < 4; ++r) m[r] = 4 * lr + r > j ? m[r] * inv : TI(0);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) l[r][q] = fma(-m[r], u[q], l[r][q]);
        }
        if (lown && (jn >> 2) == lr) {
            const int r = jn & 3;
            TI v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v[q] = r == 0 ? l[0][q] : r == 1 ? l[1][q] : r == 2 ? l[2][q] : l[3][q];
            st4(&Li[jn][4 * lc], v);
        }
        __syncthreads();
    }
    if (tid < bi) sh.idiag[tid] = TF(1) / sqrt(sh.dpiv[tid]);
    __syncthreads();
}

// Rinv = R^-1 (and R, R_acc <- R R_acc when given), all MAXB x MAXB column-major, from the state
// chol_core leaves.  X: MAXB x CLD scratch of TF.
template <class TF, class TI>
__device__ void chol_outputs(int bi, const TI (&l)[4][4], int lr, int lc, TF (*S)[CLD],
                             TF (*X)[CLD], const TF* dpiv, const TF* idiag, double* Rout,
                             double* Rinv, double* Racc) {
    const int tid = threadIdx.x;
    if (Rinv) {
        // R^-1[c][a] = L^-1[a][c] / sqrt(d_a); strictly lower tiles of R^-1 are zero
        for (int e = tid; e < MAXB * MAXB; e += blockDim.x)
            if (((e % MAXB) >> 2) > ((e / MAXB) >> 2)) Rinv[e] = 0.0;
        if (tid >= CHOL_L0 && tid < CHOL_L0 + CHOL_TILES) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int a = 4 * lr + r, c = 4 * lc + q;
                    Rinv[c + a * MAXB] = (a < bi && c < bi) ? double(l[r][q] * TI(idiag[a])) : 0.0;
                }
        }
    }
    if (!Rout && !Racc) return;
    // R: R[j][j] = sqrt(d_j), R[j][c] = W'[j][c] / sqrt(d_j) (c > j), zero elsewhere
    for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
        const int a = e / MAXB, c = e % MAXB;
        X[a][c] = (a < bi && c < bi && a <= c) ? (a == c ? sqrt(dpiv[a]) : S[a][c] * idiag[a])
                                               : TF(0);
    }
    __syncthreads();
    for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
        const int a = e / MAXB, c = e % MAXB;
        S[a][c] = X[a][c];
    }
    __syncthreads();
    if (Rout) {
        for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
            const int a = e % MAXB, c = e / MAXB;
            Rout[a + c * MAXB] = double(S[a][c]);
        }
    }
    if (Racc) {
        // Racc <- R * Racc (both upper triangular); X holds the old Racc
        for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
            const int i = e % MAXB, jj = e / MAXB;
            X[i][jj] = TF(Racc[i + jj * MAXB]);
        }
        __syncthreads();
        for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
            const int i = e % MAXB, jj = e / MAXB;
            TF acc = TF(0);
            if (i < bi && jj < bi)
                for (int q = i; q <= jj; ++q) acc = fma(S[i][q], X[q][jj], acc);
            Racc[i + jj * MAXB] = double(acc);
        }
    }
}


// Standalone factorisation.  ADAPT: float32 first, float64 (TF) when a pivot is weak.
template <class TF, class TI, bool ADAPT>
__global__ void __launch_bounds__(CHOL_THREADS)
k_chol(const double* __restrict__ W, int bi, double tau_rel, double* __restrict__ Rout,
       double* __restrict__ Rinv, double* __restrict__ Racc, int* flags) {
    extern __shared__ __align__(16) unsigned char chol_smem[];
    TF (*S)[CLD] = reinterpret_cast<TF (*)[CLD]>(chol_smem);
    TF (*X)[CLD] = reinterpret_cast<TF (*)[CLD]>(chol_smem + sizeof(TF) * MAXB * CLD);
    TI (*Sf)[CLD] = reinterpret_cast<TI (*)[CLD]>(chol_smem + 2 * sizeof(TF) * MAXB * CLD);
    TI (*Li)[CLD] = reinterpret_cast<TI (*)[CLD]>(chol_smem + (2 * sizeof(TF) + sizeof(TI)) * MAXB * CLD);
    __shared__ TF dpiv[MAXB];
    __shared__ TF invd[MAXB];
    __shared__ TF idiag[MAXB];
    __shared__ TF diag0[MAXB];
    __shared__ TF dmax_s;
    __shared__ int weak;
    auto ldw = [&](int i, int j) { return W[i + j * MAXB]; };
    TI l[4][4];
    int lr, lc;
    if (ADAPT) {
        // float32 attempt in the same shared memory (float views of S, X; TI is float here)
        float (*Sg)[CLD] = reinterpret_cast<float (*)[CLD]>(chol_smem);
        float (*Xg)[CLD] = reinterpret_cast<float (*)[CLD]>(chol_smem + sizeof(float) * MAXB * CLD);
        __shared__ float fpiv[MAXB], finvd[MAXB], fidiag[MAXB], fdiag0[MAXB], fdmax;
        float lf[4][4];
        chol_core<float, float>(bi, tau_rel, CHOL_WEAK_REL, nullptr, ldw,
                                CholShared<float, float>{Sg, reinterpret_cast<float (*)[CLD]>(Sf),
                                                         reinterpret_cast<float (*)[CLD]>(Li),
                                                         fpiv, finvd, fidiag, fdiag0, &fdmax, &weak},
                                lf, lr, lc);
        if (!weak) {
            chol_outputs<float, float>(bi, lf, lr, lc, Sg, Xg, fpiv, fidiag, Rout, Rinv, Racc);
            return;
        }
        __syncthreads();
    }
    chol_core<TF, TI>(bi, tau_rel, 0.0, flags, ldw,
                      CholShared<TF, TI>{S, Sf, Li, dpiv, invd, idiag, diag0, &dmax_s, &weak}, l,
                      lr, lc);
    chol_outputs<TF, TI>(bi, l, lr, lc, S, X, dpiv, idiag, Rout, Rinv, Racc);
}

// ---------------------------------------------------------------- fused CholeskyQR (float32 panel)
// One cooperative launch runs `passes` CholeskyQR passes on a float32 rows x bi panel: every CTA
// keeps its slice of rows in shared memory for the whole call, forms the partial Gram of the slice,
// the CTAs sum the partials (each CTA an equal share of the entries, in CTA order), every CTA
// factors the 64 x 64 Gram itself (the same arithmetic in every CTA, so the same R), and applies
// R^-1 to its rows.  The panel is read and written once when every slice fits in shared memory
// (COOP_ROWS rows per CTA); a taller slice is streamed through it in tiles of COOP_ROWS rows,
// re-read in each phase.  Grid-wide barriers use a global arrive counter and generation word;
// every wait is bounded and a timeout sets err.
//
// PRECISE = false (power scheme, only the span matters): float32 Gram and factor.
// PRECISE = true (Q_i of the randQB loops): the Gram is summed in two levels (float32 over 8 rows,
// then a float32 pair) and factored in float32 when every pivot keeps >= CHOL_WEAK_REL of its
// column's squared norm (the panel's kappa is then below ~100 and a float32-accurate Gram is
// enough); otherwise the Gram is formed again with exact products and float32-pair sums and
// factored in float64, as the unfused path does.
constexpr int COOP_THREADS = 512;
constexpr int COOP_ROWS = 440;      // rows per CTA held in shared memory
constexpr int COOP_MAX_CTAS = 256;
constexpr int PLD = MAXB + 1;       // shared row stride of the panel slice
constexpr uint64_t COOP_WAIT_NS = 2000000000ull;
// dynamic shared memory: panel slice, then S (float64 size), Sf, Li, Rs
constexpr size_t COOP_SMEM = sizeof(float) * COOP_ROWS * PLD + sizeof(double) * MAXB * CLD +
                             4 * sizeof(float) * MAXB * CLD;

struct CoopArgs {
    float* P;
    int64_t ldp, rows, rows_per;
    int bi, passes;
    double tau;
    const double* rinv_prev;  // MAXB x MAXB or null (identity)
    double* rinv_out;   // rinv_prev R_1^-1 ... R_passes^-1 (MAXB x MAXB) or null
    double* part;       // gridDim.x x (MAXB x MAXB) partial Grams
    double* wred;       // MAXB x MAXB summed Gram
    unsigned* bar;      // [0] arrivals, [1] generation
    int* flags;         // flags[1]: breakdown
    int* err;           // set when a grid barrier wait timed out
    bf16* out_hi;       // optional bf16 copy of the result: hi = bf16(P) ...
    bf16* out_lo;       // ... lo = bf16(P - hi) (nullable)
    int64_t ldo;
};

__device__ __forceinline__ uint64_t coop_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch; false when a wait ran out (err set) or err was set.
__device__ bool coop_sync(unsigned* bar, int* err) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = *reinterpret_cast<volatile int*>(err) == 0;
        if (ok) {
            volatile unsigned* gen = bar + 1;
            const unsigned g = *gen;
            __threadfence();
            if (atomicAdd(bar, 1u) == gridDim.x - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const uint64_t t0 = coop_timer();
                while (*gen == g) {
                    if (coop_timer() - t0 > COOP_WAIT_NS ||
                        *reinterpret_cast<volatile int*>(err) != 0) {
                        atomicOr(err, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// float32 pair accumulation of exact products (the float32-pair Gram)
__device__ __forceinline__ void df_add(float& hi, float& lo, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    lo += ((hi - (s - bb)) + (p - bb)) + e;
    hi = s;
}
__device__ __forceinline__ void df_add_sum(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

template <bool PRECISE>
__global__ void __launch_bounds__(COOP_THREADS, 1) k_cholqr_coop(CoopArgs p) {
    extern __shared__ __align__(16) unsigned char coop_smem[];
    float (*Ps)[PLD] = reinterpret_cast<float (*)[PLD]>(coop_smem);
    unsigned char* rest = coop_smem + sizeof(float) * COOP_ROWS * PLD;
    unsigned char* sreg = rest;                                           // S (float or double)
    float (*Sf)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + sizeof(double) * MAXB * CLD);
    float (*Li)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + (sizeof(double) + sizeof(float)) * MAXB * CLD);
    float (*Rs)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + (sizeof(double) + 2 * sizeof(float)) * MAXB * CLD);
    float (*Pc)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + (sizeof(double) + 3 * sizeof(float)) * MAXB * CLD);
    double* scratch = reinterpret_cast<double*>(rest);   // Gram combine space (S and Sf regions)
    // CTA 0 keeps the running product rinv_prev R_1^-1 R_2^-1 ... of the passes
    const bool chain = blockIdx.x == 0 && p.rinv_out != nullptr;
    if (chain) {
        for (int e = threadIdx.x; e < MAXB * MAXB; e += COOP_THREADS) {
            const int i = e % MAXB, j = e / MAXB;
            Pc[i][j] = p.rinv_prev ? float(p.rinv_prev[e]) : (i == j ? 1.f : 0.f);
        }
    }
    __shared__ float fpiv[MAXB], finvd[MAXB], fidiag[MAXB], fdiag0[MAXB], fdmax;
    __shared__ double dpiv[MAXB], dinvd[MAXB], didiag[MAXB], ddiag0[MAXB], ddmax;
    __shared__ int weak_s;
    __shared__ double red[16][32];
    const int tid = threadIdx.x;
    const int G = gridDim.x, cta = blockIdx.x;
    const int bi = p.bi;
    const int64_t r0 = int64_t(cta) * p.rows_per;
    const int64_t r_end = p.rows < r0 + p.rows_per ? p.rows : r0 + p.rows_per;
    const int nr = r_end > r0 ? int(r_end - r0) : 0;
    // A slice taller than COOP_ROWS is streamed through shared memory in tiles of COOP_ROWS rows
    // (each phase re-reads it from global memory); a slice of one tile stays resident throughout.
    const int ntile = nr > 0 ? (nr + COOP_ROWS - 1) / COOP_ROWS : 1;
    auto tile_rows = [&](int t) { return min(COOP_ROWS, nr - t * COOP_ROWS); };
    auto load_tile = [&](int t) {
        const int tn = tile_rows(t);
        const int64_t rb = r0 + int64_t(t) * COOP_ROWS;
        for (int e = tid; e < tn * MAXB; e += COOP_THREADS) {
            const int r = e % tn, col = e / tn;
            Ps[r][col] = col < bi ? p.P[rb + r + int64_t(col) * p.ldp] : 0.f;
        }
    };
    // write the tile back; the final write also emits the optional bf16 shadow
    auto store_tile = [&](int t, bool final) {
        const int tn = tile_rows(t);
        const int64_t rb = r0 + int64_t(t) * COOP_ROWS;
        for (int e = tid; e < tn * MAXB; e += COOP_THREADS) {
            const int r = e % tn, col = e / tn;
            if (col >= bi) continue;
            const float v = Ps[r][col];
            p.P[rb + r + int64_t(col) * p.ldp] = v;
            if (final && p.out_hi) {
                const bf16 h = __float2bfloat16_rn(v);
                p.out_hi[rb + r + int64_t(col) * p.ldo] = h;
                if (p.out_lo)
                    p.out_lo[rb + r + int64_t(col) * p.ldo] = __float2bfloat16_rn(v - __bfloat162float(h));
            }
        }
    };
    if (ntile == 1) load_tile(0);
    // Gram block of thread t < 3 * 136: the (t % 136)-th 4 x 4 block of the upper triangle over
    // rows t / 136, t / 136 + 3, ...
    const int blk = tid % 136, grp = tid / 136;
    int gi = 0, gj = 0;
    {
        int t = blk;
        while (t >= 16 - gi) { t -= 16 - gi; ++gi; }
        gj = gi + t;
    }
    // partial Gram of the slice into p.part[cta]; mode 0 float32, 1 two-level, 2 exact products
    auto gram = [&](int mode) {
        __syncthreads();
        float hi[4][4], lo[4][4], ch[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = ch[a][b] = 0.f;
        int cnt = 0;
        for (int t = 0; t < ntile; ++t) {
            if (ntile > 1) {
                __syncthreads();
                load_tile(t);
                __syncthreads();
            }
            const int tn = ntile > 1 ? tile_rows(t) : nr;
            if (grp >= 3) continue;
            for (int r = grp; r < tn; r += 3) {
                float x[4], y[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    x[q] = Ps[r][gi * 4 + q];
                    y[q] = Ps[r][gj * 4 + q];
                }
                if (mode == 2) {
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) df_add(hi[a][b], lo[a][b], x[a], y[b]);
                } else {
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) ch[a][b] = fmaf(x[a], y[b], ch[a][b]);
                    if (mode == 1 && ++cnt == 8) {
                        cnt = 0;
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                df_add_sum(hi[a][b], lo[a][b], ch[a][b]);
                                ch[a][b] = 0.f;
                            }
                    }
                }
            }
        }
        // the Gram scratch aliases S / Sf, free here: the factor of the previous pass is done
        __syncthreads();
        if (grp < 3) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const double v = mode == 0 ? double(ch[a][b])
                                               : double(hi[a][b]) + double(lo[a][b]) + double(ch[a][b]);
                    scratch[(grp * 136 + blk) * 16 + a * 4 + b] = v;
                }
        }
        __syncthreads();
        if (tid < 136) {
            double* out = p.part + int64_t(cta) * MAXB * MAXB;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const double v = scratch[blk * 16 + q] + scratch[(136 + blk) * 16 + q] +
                                 scratch[(272 + blk) * 16 + q];
                out[(gi * 4 + q / 4) + (gj * 4 + q % 4) * MAXB] = v;
            }
        }
    };
    // sum the partials: this CTA owns an equal share of the upper entries
    auto reduce = [&]() {
        const int per = (MAXB * MAXB + G - 1) / G;
        const int e0 = cta * per, e1 = min(MAXB * MAXB, e0 + per);
        const int lane = tid & 31, sub = tid >> 5;   // 16 subsets of the partials
        for (int eb = e0; eb < e1; eb += 32) {
            const int e = eb + lane;
            double v = 0.0;
            if (e < e1 && e % MAXB <= e / MAXB)
                for (int q = sub; q < G; q += 16) v += __ldcg(p.part + int64_t(q) * MAXB * MAXB + e);
            red[sub][lane] = v;
            __syncthreads();
            if (sub == 0 && e < e1) {
                double t = 0.0;
#pragma unroll
                for (int q = 0; q < 16; ++q) t += red[q][lane];
                p.wred[e] = t;
            }
            __syncthreads();
        }
    };
    auto ldw = [&](int i, int j) { return __ldcg(p.wred + i + j * MAXB); };
    for (int pass = 0; pass < p.passes; ++pass) {
        gram(PRECISE ? 1 : 0);
        if (!coop_sync(p.bar, p.err)) return;
        reduce();
        if (!coop_sync(p.bar, p.err)) return;
        // ---- every CTA factors the summed Gram
        float l[4][4];
        int lr, lc;
        float (*Sfl)[CLD] = reinterpret_cast<float (*)[CLD]>(sreg);
        chol_core<float, float>(bi, p.tau, PRECISE ? CHOL_WEAK_REL : 0.0,
                                (cta == 0 && !PRECISE) ? p.flags : nullptr, ldw,
                                CholShared<float, float>{Sfl, Sf, Li, fpiv, finvd, fidiag, fdiag0,
                                                         &fdmax, &weak_s},
                                l, lr, lc);
        bool dbl = false;
        if (PRECISE && weak_s) {
            // ill-conditioned panel: exact-product Gram, float64 factor
            dbl = true;
            gram(2);
            if (!coop_sync(p.bar, p.err)) return;
            reduce();
            if (!coop_sync(p.bar, p.err)) return;
            double (*Sd)[CLD] = reinterpret_cast<double (*)[CLD]>(sreg);
            chol_core<double, float>(bi, p.tau, 0.0, cta == 0 ? p.flags : nullptr, ldw,
                                     CholShared<double, float>{Sd, Sf, Li, dpiv, dinvd, didiag,
                                                               ddiag0, &ddmax, &weak_s},
                                     l, lr, lc);
        }
        // R^-1[c][a] = L^-1[a][c] / sqrt(d_a); strictly lower tiles are zero
        for (int e = tid; e < MAXB * MAXB; e += COOP_THREADS) {
            const int i = e % MAXB, jj = e / MAXB;
            if ((i >> 2) > (jj >> 2)) Rs[i][jj] = 0.f;
        }
        if (tid >= CHOL_L0 && tid < CHOL_L0 + CHOL_TILES) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int a = 4 * lr + r, c = 4 * lc + q;
                    const float id = dbl ? float(didiag[a < MAXB ? a : 0]) : fidiag[a < MAXB ? a : 0];
                    Rs[c][a] = (a < bi && c < bi) ? l[r][q] * id : 0.f;
                }
        }
        __syncthreads();
        if (chain) {
            // Pc <- Pc R^-1 (thread: row i, 8 consecutive columns)
            const int i = tid & 63, c0 = (tid >> 6) * 8;
            float acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = 0.f;
            for (int l2 = 0; l2 < MAXB; ++l2) {
                const float v = Pc[i][l2];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = fmaf(v, Rs[l2][c0 + q], acc[q]);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 8; ++q) Pc[i][c0 + q] = acc[q];
        }
        // ---- rows <- rows * R^-1, 128 rows at a time (thread: one row, 16 columns)
        const bool last = pass + 1 == p.passes;
        for (int t = 0; t < ntile; ++t) {
            if (ntile > 1) {
                __syncthreads();
                load_tile(t);
                __syncthreads();
            }
            const int tn = ntile > 1 ? tile_rows(t) : nr;
            const int i = tid & 127, c0 = (tid >> 7) * 16;
            for (int rb = 0; rb < tn; rb += 128) {
                const int r = rb + i;
                float acc[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = 0.f;
                if (r < tn) {
                    for (int q2 = 0; q2 < bi; ++q2) {
                        const float v = Ps[r][q2];
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc[q] = fmaf(v, Rs[q2][c0 + q], acc[q]);
                    }
                }
                __syncthreads();
                if (r < tn) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) Ps[r][c0 + q] = acc[q];
                }
                __syncthreads();
            }
            if (ntile > 1) store_tile(t, last);
        }
    }
    __syncthreads();
    if (chain) {
        for (int e = tid; e < MAXB * MAXB; e += COOP_THREADS)
            p.rinv_out[e] = double(Pc[e % MAXB][e / MAXB]);
    }
    if (ntile == 1) store_tile(0, true);
}

__global__ void k_identity(double* R, int bi) {
    for (int e = threadIdx.x; e < MAXB * MAXB; e += blockDim.x) {
        const int i = e % MAXB, j = e / MAXB;
        R[e] = (i == j && i < bi) ? 1.0 : 0.0;
    }
}

__global__ void k_tri_inv(const double* __restrict__ Rg, int bi, double* __restrict__ Xg) {
    extern __shared__ double smem[];
    double (*R)[LDS] = reinterpret_cast<double (*)[LDS]>(smem);
    double (*X)[LDS] = reinterpret_cast<double (*)[LDS]>(smem + MAXB * LDS);
    for (int e = threadIdx.x; e < MAXB * MAXB; e += blockDim.x) {
        const int i = e % MAXB, j = e / MAXB;
        R[i][j] = Rg[i + j * MAXB];
        X[i][j] = 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < bi; c += blockDim.x) {
        X[c][c] = 1.0 / R[c][c];
        for (int i = c - 1; i >= 0; --i) {
            double s = 0.0;
            for (int l = i + 1; l <= c; ++l) s = fma(R[i][l], X[l][c], s);
            X[i][c] = -s / R[i][i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < MAXB * MAXB; e += blockDim.x) {
        const int i = e % MAXB, j = e / MAXB;
        Xg[i + j * MAXB] = X[i][j];
    }
}

// P (rows x bi) <- P * Rinv, in place, 128 rows per CTA (each CTA owns its rows).  Thread t
// computes rows t % 64 and t % 64 + 64 for columns 16 (t / 64) .. 16 (t / 64) + 15; Rinv rows are
// read as broadcast vectors.  Terms run l = 0, 1, ... (the zero lower part of Rinv adds exact
// zeros).
constexpr int APPLY_ROWS = 128;
template <class T>
__global__ void __launch_bounds__(256)
k_apply_rinv(T* __restrict__ P, int64_t ldp, int64_t m, int bi, const double* __restrict__ Rinv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*Rs)[MAXB] = reinterpret_cast<T (*)[MAXB]>(smem_raw);                           // [l][c]
    T (*Ps)[LDS] = reinterpret_cast<T (*)[LDS]>(smem_raw + sizeof(T) * MAXB * MAXB);   // [row][l]
    const int64_t r0 = int64_t(blockIdx.x) * APPLY_ROWS;
    const int tid = threadIdx.x;
    for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
        const int i = e % MAXB, j = e / MAXB;
        Rs[i][j] = (i < bi && j < bi) ? T(Rinv[i + j * MAXB]) : T(0);
    }
    for (int e = tid; e < APPLY_ROWS * MAXB; e += blockDim.x) {
        const int i = e % APPLY_ROWS, j = e / APPLY_ROWS;
        const int64_t gr = r0 + i;
        Ps[i][j] = (gr < m && j < bi) ? P[gr + int64_t(j) * ldp] : T(0);
    }
    __syncthreads();
    const int i = tid & 63, c0 = (tid >> 6) * 16;
    T acc[2][16];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[h][k] = T(0);
    for (int l = 0; l < bi; ++l) {
        const T p0 = Ps[i][l], p1 = Ps[i + 64][l];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const T r = Rs[l][c0 + k];
            acc[0][k] = fma(p0, r, acc[0][k]);
            acc[1][k] = fma(p1, r, acc[1][k]);
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t gr = r0 + i + 64 * h;
        if (gr >= m) continue;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (c0 + k < bi) P[gr + int64_t(c0 + k) * ldp] = acc[h][k];
    }
}

template <class T>
__global__ void k_row_norm2(const T* __restrict__ B, int64_t ldb, int64_t n, double* rn) {
    const int j = blockIdx.x;
    double s = 0.0;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
        const double v = double(B[int64_t(j) * ldb + c]);
        s = fma(v, v, s);
    }
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[w];
        rn[j] = t;
    }
}

// state[0] = E, state[1] = rows kept, state[2] = stop flag, state[3] = E before the block.
// With Wq = Q_i^T Q_i and Gb = B_i B_i^T of the block (MAXB x MAXB, ld MAXB), row j also adds
// (Wq_jj - 1) Gb_jj + 2 sum_{p<j} Wq_pj Gb_pj: for B = Q^T A, ||A - Q B||^2 = E +
// tr(B^T (Q^T Q - I) B), and a float32 Q is orthonormal only to a few u, which on the leading
// rows is a few u ||A||^2, as large as the stop margin.  (Terms between blocks are second order
// after the re-orthogonalisation.)  rn[j] = Gb_jj then.
__global__ void k_indicator(double* state, const double* rn, int rows, double eps2,
                            int row_by_row, const double* Wq, const double* Gb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double E = state[0];
    state[3] = E;
    int keep = rows;
    int stop = 0;
    auto row_term = [&](int j) {
        if (!Wq) return rn[j];
        double c = (Wq[j + j * MAXB] - 1.0) * Gb[j + j * MAXB];
        for (int p = 0; p < j; ++p) c += 2.0 * Wq[p + j * MAXB] * Gb[p + j * MAXB];
        return Gb[j + j * MAXB] - c;
    };
    if (row_by_row) {
        for (int j = 0; j < rows; ++j) {
            E -= row_term(j);
            if (E < eps2) { keep = j + 1; stop = 1; break; }
        }
    } else {
        double s = 0.0;
        for (int j = 0; j < rows; ++j) s += row_term(j);
        E -= s;
        stop = E < eps2;
    }
    state[0] = E;
    state[1] = double(keep);
    state[2] = double(stop);
}

}  // namespace

template <class TF, class TI>
constexpr size_t chol_smem() {
    return (2 * sizeof(TF) + 2 * sizeof(TI)) * MAXB * CLD;
}
constexpr size_t TRI_SMEM = sizeof(double) * 2 * MAXB * LDS;

template <class K>
void allow_smem(K kernel, size_t bytes) {
    // idempotent, cheap; called before every launch so each device gets it
    QB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
}

void chol_rinv(cudaStream_t st, const double* W, int bi, double tau_rel, double* R, double* Rinv,
               double* R_acc, int* flags, CholPrec prec) {
    switch (prec) {
        case CHOL_F64: {
            constexpr size_t sm = chol_smem<double, double>();
            allow_smem(k_chol<double, double, false>, sm);
            k_chol<double, double, false><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv,
                                                                       R_acc, flags);
            break;
        }
        case CHOL_F64_INV_F32: {
            constexpr size_t sm = chol_smem<double, float>();
            allow_smem(k_chol<double, float, false>, sm);
            k_chol<double, float, false><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv,
                                                                      R_acc, flags);
            break;
        }
        case CHOL_ADAPTIVE: {
            constexpr size_t sm = chol_smem<double, float>();
            allow_smem(k_chol<double, float, true>, sm);
            k_chol<double, float, true><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv,
                                                                     R_acc, flags);
            break;
        }
        default: {
            constexpr size_t sm = chol_smem<float, float>();
            allow_smem(k_chol<float, float, false>, sm);
            k_chol<float, float, false><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv,
                                                                     R_acc, flags);
            break;
        }
    }
    QB_LAUNCHED();
}

size_t cholqr_coop_scratch_bytes() {
    return size_t(COOP_MAX_CTAS) * MAXB * MAXB * sizeof(double) + MAXB * MAXB * sizeof(double) + 256;
}

bool cholqr_coop(cudaStream_t st, float* P, int64_t ldp, int64_t rows, int bi, int passes,
                 bool precise, double tau, const double* rinv_prev, double* rinv_out,
                 void* scratch, size_t scratch_bytes, unsigned* bar, int* flags, int* err,
                 bf16* out_hi, bf16* out_lo, int64_t ldo) {
    static int max_ctas[2] = {-1, -1};
    const int v = precise ? 1 : 0;
    auto kern = precise ? k_cholqr_coop<true> : k_cholqr_coop<false>;
    if (max_ctas[v] < 0) {
        int dev = 0, coop = 0, per_sm = 0;
        QB_CUDA(cudaGetDevice(&dev));
        QB_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        QB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(COOP_SMEM)));
        QB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, COOP_THREADS,
                                                               COOP_SMEM));
        max_ctas[v] = coop ? std::min(per_sm * num_sms(), COOP_MAX_CTAS) : 0;
    }
    if (max_ctas[v] <= 0 || bi < 1 || bi > MAXB || rows <= 0 || passes < 1) return false;
    int G = int(std::min<int64_t>(max_ctas[v], cdiv(rows, 64)));
    const int64_t rows_per = cdiv(rows, G);
    // slices taller than COOP_ROWS are streamed in tiles (int row indices inside a slice)
    if (rows_per > (int64_t(1) << 28)) return false;
    G = int(cdiv(rows, rows_per));
    if (scratch_bytes < cholqr_coop_scratch_bytes()) return false;
    CoopArgs a;
    a.P = P;
    a.ldp = ldp;
    a.rows = rows;
    a.rows_per = rows_per;
    a.bi = bi;
    a.passes = passes;
    a.tau = tau;
    a.rinv_prev = rinv_prev;
    a.rinv_out = rinv_out;
    a.part = reinterpret_cast<double*>(scratch);
    a.wred = a.part + size_t(COOP_MAX_CTAS) * MAXB * MAXB;
    a.bar = bar;
    a.flags = flags;
    a.err = err;
    a.out_hi = out_hi;
    a.out_lo = out_hi ? out_lo : nullptr;
    a.ldo = ldo;
    void* args[] = {&a};
    QB_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), dim3(G), dim3(COOP_THREADS),
                                        args, COOP_SMEM, st));
    QB_LAUNCHED();
    return true;
}

void set_identity(cudaStream_t st, double* R, int bi) {
    k_identity<<<1, 256, 0, st>>>(R, bi);
    QB_LAUNCHED();
}

void tri_inv(cudaStream_t st, const double* R, int bi, double* Rinv) {
    allow_smem(k_tri_inv, TRI_SMEM);
    k_tri_inv<<<1, 64, TRI_SMEM, st>>>(R, bi, Rinv);
    QB_LAUNCHED();
}

void apply_rinv(cudaStream_t st, bool f64, void* P, int64_t ldp, int64_t m, int bi,
                const double* Rinv) {
    if (m <= 0) return;
    const unsigned g = unsigned(cdiv(m, APPLY_ROWS));
    if (f64) {
        const size_t sm = sizeof(double) * (MAXB * MAXB + APPLY_ROWS * LDS);
        allow_smem(k_apply_rinv<double>, sm);
        k_apply_rinv<double><<<g, 256, sm, st>>>(reinterpret_cast<double*>(P), ldp, m, bi, Rinv);
    } else {
        const size_t sm = sizeof(float) * (MAXB * MAXB + APPLY_ROWS * LDS);
        allow_smem(k_apply_rinv<float>, sm);
        k_apply_rinv<float><<<g, 256, sm, st>>>(reinterpret_cast<float*>(P), ldp, m, bi, Rinv);
    }
    QB_LAUNCHED();
}

void row_norm2(cudaStream_t st, bool f64, const void* B, int64_t ldb, int rows, int64_t n,
               double* rn) {
    if (rows <= 0) return;
    if (f64) k_row_norm2<double><<<rows, 256, 0, st>>>(reinterpret_cast<const double*>(B), ldb, n, rn);
    else k_row_norm2<float><<<rows, 256, 0, st>>>(reinterpret_cast<const float*>(B), ldb, n, rn);
    QB_LAUNCHED();
}

void indicator(cudaStream_t st, double* state, const double* rn, int rows, double eps2,
               int row_by_row, const double* Wq, const double* Gb) {
    k_indicator<<<1, 32, 0, st>>>(state, rn, rows, eps2, row_by_row, Wq, Gb);
    QB_LAUNCHED();
}

}  // namespace qb
