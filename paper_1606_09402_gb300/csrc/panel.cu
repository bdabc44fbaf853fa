// CholeskyQR panel pieces (b x b float64 Cholesky, triangular inverse, R accumulation, applying
// R^-1 to an m x b panel) and the Frobenius-norm indicator of Theorem 1 with the row-by-row
// stopping rule of Sect. 3.1.
#include <type_traits>
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
// whole warps drop out), threads 160..295 the lower tiles of L^-1.  The elimination takes the four
// pivots of a tile row per block barrier (a quad step): the tile row waits in shared memory with
// every earlier update applied; every thread factors its 4 x 4 diagonal block and brings the block
// rows up to date at the indices it needs (the same arithmetic as their owners), then applies the
// four rank-one updates to its tile; the owners publish the tile row (final) and the next one
// (pending).
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
    TI (*Sf)[CLD];   // scratch of MAXB rows of TI: holds the two-slot rings of pending tile rows
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
// reciprocal of a pivot: float32 by the fast hardware reciprocal (an error of ~2 ulp in a
// multiplier is rounding of the elimination itself, and the float32 factor feeds CholeskyQR2),
// float64 correctly rounded (the float64 path's parity with the float64 oracle)
__device__ __forceinline__ float rcp_rn(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

template <class TF, class TI, class Load>
__device__ void chol_core(int bi, double tau_rel, double weak_rel, int* flags, Load load,
                          CholShared<TF, TI> sh, TI (&l)[4][4], int& lr, int& lc) {
    TF (*S)[CLD] = sh.S;
    TI (*Li)[CLD] = sh.Li;
    // two-slot rings (rows 0..3 and 4..7) of the pending tile row: its four rows of W and of
    // L^-1 before the updates of their own quad step
    TF (*PW)[CLD] = reinterpret_cast<TF (*)[CLD]>(sh.Sf);
    TI (*PL)[CLD] = reinterpret_cast<TI (*)[CLD]>(reinterpret_cast<TF*>(sh.Sf) + 8 * CLD);
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
    // initial state: tile row 0 pending in slot 0
    if (wown) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (wi == wj) sh.diag0[4 * wi + r] = w[r][r];
            if (wi == 0) st4(&PW[r][4 * wj], w[r]);
        }
    }
    if (lown && lr == 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) st4(&PL[r][4 * lc], l[r]);
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
    const TF tau_dmax = TF(tau_rel) * dmax;
    const TF weak_t = TF(weak_rel);
    // the pivot used for a diagonal value d: d, or the floor when d does not exceed tau_rel * dmax
    auto piv_value = [&](TF d) { return d > tau_dmax ? d : floor_piv; };
    // quad step t: the four pivots of tile row t per block barrier.  Every thread factors the
    // pending 4 x 4 diagonal block itself and applies the block rows to the entries it needs, in
    // the arithmetic of the one-pivot-per-step elimination (the same operations in the same
    // order, so the result is bit-identical to it):
    //   W'[a][c] -= W'[p][a] (W'[p][c] / d_p),   L^-1[a][c] -= (W'[p][a] / d_p) L^-1[p][c],
    // for the pivots p = 4t .. 4t + 3 in turn (a > p).
    for (int t = 0; 4 * t < bi; ++t) {
        const int j = 4 * t, slot = (t & 1) * 4, nslot = 4 - slot;
        TF bl[4][4];                  // the diagonal block; row p final once p pivots are applied
#pragma unroll
        for (int i = 0; i < 4; ++i) ld4(&PW[slot + i][j], bl[i]);
        TF inv[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            inv[p] = rcp_rn(piv_value(bl[p][p]));
#pragma unroll
            for (int i = p + 1; i < 4; ++i)
#pragma unroll
                for (int i2 = i; i2 < 4; ++i2) bl[i][i2] = fma(-bl[p][i], bl[p][i2] * inv[p], bl[i][i2]);
        }
        if (tid == 0) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                if (j + p < bi) {
                    const TF d = bl[p][p];
                    if (!(d >= weak_t * sh.diag0[j + p])) sh.weak[0] = 1;
                    if (!(d > tau_dmax)) {
                        sh.weak[0] = 1;
                        if (flags) atomicOr(flags + 1, 1);
                    }
                    sh.dpiv[j + p] = piv_value(d);
                }
            }
        }
        if (wown && wi > t) {
            // the block rows at this tile's rows (vr: W'[j+p][4 wi + r]) and columns
            // (vc: W'[j+p][4 wj + q] / d_p), from their pending values
            TF vr[4][4], vc[4][4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                ld4(&PW[slot + p][4 * wi], vr[p]);
                ld4(&PW[slot + p][4 * wj], vc[p]);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                TF tr[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) tr[r] = vr[p][r] * inv[p];
#pragma unroll
                for (int q = 0; q < 4; ++q) vc[p][q] *= inv[p];
#pragma unroll
                for (int i = p + 1; i < 4; ++i) {
#pragma unroll
                    for (int r = 0; r < 4; ++r) vr[i][r] = fma(-bl[p][i], tr[r], vr[i][r]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) vc[i][q] = fma(-bl[p][i], vc[p][q], vc[i][q]);
                }
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[r][q] = fma(-vr[p][r], vc[p][q], w[r][q]);
        } else if (wown && wi == t) {
            // this tile's rows are the block rows: their updates within the block
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                TF tq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) tq[q] = w[p][q] * inv[p];
#pragma unroll
                for (int i = p + 1; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[i][q] = fma(-bl[p][i], tq[q], w[i][q]);
            }
        }
        if (lown && lr > t && lc <= t) {
            // final L^-1 block rows at this tile's columns (lf) and the multipliers' W' values at
            // its rows (vr), from their pending values
            TI lf[4][4];
            TF vr[4][4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                ld4(&PL[slot + p][4 * lc], lf[p]);
                ld4(&PW[slot + p][4 * lr], vr[p]);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const TI mm0 = TI(inv[p]);
                TF tr[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) tr[r] = vr[p][r] * inv[p];
#pragma unroll
                for (int i = p + 1; i < 4; ++i) {
                    const TI mm = TI(bl[p][i]) * mm0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) lf[i][q] = fma(-mm, lf[p][q], lf[i][q]);
#pragma unroll
                    for (int r = 0; r < 4; ++r) vr[i][r] = fma(-bl[p][i], tr[r], vr[i][r]);
                }
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const TI ip = TI(inv[p]);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const TI m = TI(vr[p][r]) * ip;
#pragma unroll
                    for (int q = 0; q < 4; ++q) l[r][q] = fma(-m, lf[p][q], l[r][q]);
                }
            }
        } else if (lown && lr == t) {
            // this tile's rows are the block rows of L^-1: their updates within the block
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const TI mm0 = TI(inv[p]);
#pragma unroll
                for (int i = p + 1; i < 4; ++i) {
                    const TI mm = TI(bl[p][i]) * mm0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) l[i][q] = fma(-mm, l[p][q], l[i][q]);
                }
            }
        }
        // tile row t is final; tile row t + 1 waits in the other slot
        if (wown) {
            if (wi == t) {
#pragma unroll
                for (int r = 0; r < 4; ++r) st4(&S[j + r][4 * wj], w[r]);
            } else if (wi == t + 1) {
#pragma unroll
                for (int r = 0; r < 4; ++r) st4(&PW[nslot + r][4 * wj], w[r]);
            }
        }
        if (lown) {
            if (lr == t) {
#pragma unroll
                for (int r = 0; r < 4; ++r) st4(&Li[j + r][4 * lc], l[r]);
            } else if (lr == t + 1) {
#pragma unroll
                for (int r = 0; r < 4; ++r) st4(&PL[nslot + r][4 * lc], l[r]);
            }
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
// The panel slice is held column by column (rows contiguous, so the global loads and stores are
// coalesced and 8 consecutive rows are two float4 reads).  Column c starts at pcol(c) =
// c TLD + 4 (c / 4): TLD is a multiple of 32 words, so the start lies on bank 4 (c / 4) mod 32 and
// the float4 reads of eight consecutive column quadruples at one row hit distinct banks (the
// Gram's access pattern).  The skew only grows, so columns never overlap (TLD >= COOP_ROWS).
constexpr int TLD = 448;
constexpr int PT_FLOATS = MAXB * TLD + MAXB;
static_assert(TLD % 32 == 0 && TLD >= COOP_ROWS && COOP_ROWS % 8 == 0, "panel slice layout");
__device__ __forceinline__ int pcol(int c) { return c * TLD + 4 * (c >> 2); }
constexpr uint64_t COOP_WAIT_NS = 2000000000ull;
// dynamic shared memory: panel slice, then S (float64 size), Sf, Li, Rs, Pc
constexpr size_t COOP_SMEM = sizeof(float) * PT_FLOATS + sizeof(double) * MAXB * CLD +
                             4 * sizeof(float) * MAXB * CLD;

struct CoopArgs {
    float* P;
    int64_t ldp, rows, rows_per;
    int bi, passes;
    double tau;
    const double* rinv_prev;  // MAXB x MAXB or null (identity)
    double* rinv_out;   // rinv_prev R_1^-1 ... R_passes^-1 (MAXB x MAXB) or null
    float2* part;       // gridDim.x x (MAXB x MAXB) partial Grams (float32 pairs)
    float2* wred;       // MAXB x MAXB summed Gram (float32 pair)
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
// sum of two float32 pairs (hi + lo each), renormalised: a two-sum of the leading terms, the
// error and the trailing terms added, then a fast two-sum
__device__ __forceinline__ float2 fp_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = ((a.x - (s - bb)) + (b.x - bb)) + (a.y + b.y);
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
__device__ __forceinline__ void df_add_sum(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

// Rs = R^-1 (row-major, CLD stride) from the factor's L^-1 tiles: R^-1[c][a] = L^-1[a][c] / sqrt(d_a);
// strictly lower tiles are zero
template <class TF>
__device__ __forceinline__ void coop_write_rinv(int bi, const float (&l)[4][4], int lr, int lc,
                                                const TF* idiag, float (*Rs)[CLD]) {
    const int tid = threadIdx.x;
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
                const float id = float(idiag[a < MAXB ? a : 0]);
                Rs[c][a] = (a < bi && c < bi) ? l[r][q] * id : 0.f;
            }
    }
}

// the float64 refactor of an ill-conditioned panel; kept out of line so that the float32 path of
// the fused kernel keeps its registers
__device__ __noinline__ void coop_factor_f64(int bi, double tau, int* flags, const float2* wred,
                                             CholShared<double, float> sh, float (*Rs)[CLD]) {
    float l[4][4];
    int lr, lc;
    auto ldw = [&](int i, int j) {
        const float2 v = __ldcg(wred + i + j * MAXB);
        return double(v.x) + double(v.y);
    };
    chol_core<double, float>(bi, tau, 0.0, flags, ldw, sh, l, lr, lc);
    coop_write_rinv(bi, l, lr, lc, sh.idiag, Rs);
}

template <bool PRECISE>
__global__ void __launch_bounds__(COOP_THREADS, 1) k_cholqr_coop(CoopArgs p) {
    extern __shared__ __align__(16) unsigned char coop_smem[];
    float* Pt = reinterpret_cast<float*>(coop_smem);
    unsigned char* rest = coop_smem + sizeof(float) * PT_FLOATS;
    unsigned char* sreg = rest;                                           // S (float or double)
    float (*Sf)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + sizeof(double) * MAXB * CLD);
    float (*Li)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + (sizeof(double) + sizeof(float)) * MAXB * CLD);
    float (*Rs)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + (sizeof(double) + 2 * sizeof(float)) * MAXB * CLD);
    float (*Pc)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + (sizeof(double) + 3 * sizeof(float)) * MAXB * CLD);
    float2* scratch = reinterpret_cast<float2*>(rest);   // Gram combine space (S, Sf, Li regions)
    // CTA 0 keeps the running product rinv_prev R_1^-1 R_2^-1 ... of the passes, transposed
    // (Pc[j][i] holds entry (i, j)) so that the product reads it without bank conflicts
    const bool chain = blockIdx.x == 0 && p.rinv_out != nullptr;
    if (chain) {
        for (int e = threadIdx.x; e < MAXB * MAXB; e += COOP_THREADS) {
            const int i = e % MAXB, j = e / MAXB;
            Pc[j][i] = p.rinv_prev ? float(p.rinv_prev[e]) : (i == j ? 1.f : 0.f);
        }
    }
    __shared__ float fpiv[MAXB], finvd[MAXB], fidiag[MAXB], fdiag0[MAXB], fdmax;
    __shared__ double dpiv[MAXB], dinvd[MAXB], didiag[MAXB], ddiag0[MAXB], ddmax;
    __shared__ int weak_s;
    __shared__ float2 red[16][32];
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x, cta = blockIdx.x;
    const int bi = p.bi;
    const int64_t r0 = int64_t(cta) * p.rows_per;
    const int64_t r_end = p.rows < r0 + p.rows_per ? p.rows : r0 + p.rows_per;
    const int nr = r_end > r0 ? int(r_end - r0) : 0;
    // A slice taller than COOP_ROWS is streamed through shared memory in tiles of COOP_ROWS rows
    // (each phase re-reads it from global memory); a slice of one tile stays resident throughout.
    const int ntile = nr > 0 ? (nr + COOP_ROWS - 1) / COOP_ROWS : 1;
    auto tile_rows = [&](int t) { return min(COOP_ROWS, nr - t * COOP_ROWS); };
    // rows up to the next multiple of 8 (zeros past the tile and in the columns >= bi) are
    // written so that the float4 reads of the Gram and the row update see zeros there
    // (warp w takes columns w, w + 16, w + 32, w + 48; its lanes consecutive rows)
    auto load_tile = [&](int t) {
        const int tn = tile_rows(t), tn8 = (tn + 7) & ~7;
        const int64_t rb = r0 + int64_t(t) * COOP_ROWS;
#pragma unroll
        for (int cc = 0; cc < MAXB / 16; ++cc) {
            const int col = warp + 16 * cc;
            const bool cok = col < bi;
            const float* src = p.P + rb + int64_t(cok ? col : 0) * p.ldp;
            float* dst = Pt + pcol(col);
#pragma unroll 4
            for (int r = lane; r < tn8; r += 32) dst[r] = (cok && r < tn) ? src[r] : 0.f;
        }
    };
    // write the tile back; the final write also emits the optional bf16 shadow
    auto store_tile = [&](int t, bool final) {
        const int tn = tile_rows(t);
        const int64_t rb = r0 + int64_t(t) * COOP_ROWS;
        for (int col = warp; col < bi; col += COOP_THREADS / 32) {
            const float* src = Pt + pcol(col);
#pragma unroll 4
            for (int r = lane; r < tn; r += 32) {
                const float v = src[r];
                const int64_t g = rb + r;
                p.P[g + int64_t(col) * p.ldp] = v;
                if (final && p.out_hi) {
                    const bf16 h = __float2bfloat16_rn(v);
                    p.out_hi[g + int64_t(col) * p.ldo] = h;
                    if (p.out_lo)
                        p.out_lo[g + int64_t(col) * p.ldo] = __float2bfloat16_rn(v - __bfloat162float(h));
                }
            }
        }
    };
    if (ntile == 1) load_tile(0);
    // Gram: warp w < 12 computes the 16 x 32 block GB[w % 6] of the upper part of the 64 x 64 Gram
    // over one half of the slice's rows (w / 6); lane (ti, tj) = (lane / 8, lane % 8) owns the
    // 4 x 4 sub-block at rows 4 ti, columns 4 tj of it.  Per 4 rows a thread reads 8 float4 and
    // does 64 FMAs.
    const bool gw = warp < 12;
    const int gblk = warp % 6, ghalf = warp / 6;
    const int gi0 = 16 * (gblk < 2 ? gblk : gblk - 2) + 4 * (lane >> 3);
    const int gj0 = 32 * (gblk < 2 ? 0 : 1) + 4 * (lane & 7);
    // partial Gram of the slice into p.part[cta]; mode 0 float32, 1 two-level, 2 exact products
    auto gram = [&](auto mode_c) {
        constexpr int mode = decltype(mode_c)::value;
        __syncthreads();
        float hi[4][4], lo[4][4], ch[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = ch[a][b] = 0.f;
        for (int t = 0; t < ntile; ++t) {
            if (ntile > 1) {
                __syncthreads();
                load_tile(t);
                __syncthreads();
            }
            const int tn = ntile > 1 ? tile_rows(t) : nr;
            if (!gw) continue;
            const int nch = (tn + 3) >> 2, cmid = (nch + 1) >> 1;
            const int cb = ghalf == 0 ? 0 : cmid, ce = ghalf == 0 ? cmid : nch;
            for (int c4 = cb; c4 < ce; ++c4) {
                const int r = 4 * c4;
                float4 x[4], y[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    x[q] = *reinterpret_cast<const float4*>(Pt + pcol(gi0 + q) + r);
                    y[q] = *reinterpret_cast<const float4*>(Pt + pcol(gj0 + q) + r);
                }
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float xa = rr == 0 ? x[a].x : rr == 1 ? x[a].y : rr == 2 ? x[a].z : x[a].w;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const float yb = rr == 0 ? y[b].x : rr == 1 ? y[b].y : rr == 2 ? y[b].z : y[b].w;
                            if (mode == 2) df_add(hi[a][b], lo[a][b], xa, yb);
                            else ch[a][b] = fmaf(xa, yb, ch[a][b]);
                        }
                    }
                }
                if (mode == 1 && ((c4 - cb) & 1)) {   // fold every 8 rows into the float32 pair
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
        // the Gram scratch aliases S / Sf / Li, free here: the factor of the previous pass is done
        __syncthreads();
        if (gw) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float2 v = mode == 0 ? make_float2(ch[a][b], 0.f)
                                               : fp_add(make_float2(hi[a][b], lo[a][b]),
                                                        make_float2(ch[a][b], 0.f));
                    scratch[ghalf * MAXB * MAXB + (gi0 + a) + (gj0 + b) * MAXB] = v;
                }
        }
        __syncthreads();
        float2* out = p.part + int64_t(cta) * MAXB * MAXB;
        for (int e = tid; e < MAXB * MAXB; e += COOP_THREADS)
            if ((e & (MAXB - 1)) <= (e / MAXB)) out[e] = fp_add(scratch[e], scratch[MAXB * MAXB + e]);
    };
    // sum the partials: this CTA owns an equal share of the upper entries
    auto reduce = [&]() {
        const int per = (MAXB * MAXB + G - 1) / G;
        const int e0 = cta * per, e1 = min(MAXB * MAXB, e0 + per);
        const int lane = tid & 31, sub = tid >> 5;   // 16 subsets of the partials
        for (int eb = e0; eb < e1; eb += 32) {
            const int e = eb + lane;
            float2 v = make_float2(0.f, 0.f);
            if (e < e1 && e % MAXB <= e / MAXB) {
                // partials sub, sub + 16, ... in that order, four loads in flight
                const float2* src = p.part + e;
                int q = sub;
                for (; q + 48 < G; q += 64) {
                    const float2 a0 = __ldcg(src + int64_t(q) * MAXB * MAXB);
                    const float2 a1 = __ldcg(src + int64_t(q + 16) * MAXB * MAXB);
                    const float2 a2 = __ldcg(src + int64_t(q + 32) * MAXB * MAXB);
                    const float2 a3 = __ldcg(src + int64_t(q + 48) * MAXB * MAXB);
                    v = fp_add(v, a0);
                    v = fp_add(v, a1);
                    v = fp_add(v, a2);
                    v = fp_add(v, a3);
                }
                for (; q < G; q += 16) v = fp_add(v, __ldcg(src + int64_t(q) * MAXB * MAXB));
            }
            red[sub][lane] = v;
            __syncthreads();
            if (sub == 0 && e < e1) {
                float2 t = make_float2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 16; ++q) t = fp_add(t, red[q][lane]);
                p.wred[e] = t;
            }
            __syncthreads();
        }
    };
    auto ldw = [&](int i, int j) {
        const float2 v = __ldcg(p.wred + i + j * MAXB);
        return v.x + v.y;
    };
    for (int pass = 0; pass < p.passes; ++pass) {
        gram(std::integral_constant<int, PRECISE ? 1 : 0>{});
        if (!coop_sync(p.bar, p.err)) return;
        reduce();
        if (!coop_sync(p.bar, p.err)) return;
        // ---- every CTA factors the summed Gram
        {
            float l[4][4];
            int lr, lc;
            float (*Sfl)[CLD] = reinterpret_cast<float (*)[CLD]>(sreg);
            chol_core<float, float>(bi, p.tau, PRECISE ? CHOL_WEAK_REL : 0.0,
                                    (cta == 0 && !PRECISE) ? p.flags : nullptr, ldw,
                                    CholShared<float, float>{Sfl, Sf, Li, fpiv, finvd, fidiag,
                                                             fdiag0, &fdmax, &weak_s},
                                    l, lr, lc);
            coop_write_rinv(bi, l, lr, lc, fidiag, Rs);
        }
        if (PRECISE && weak_s) {
            // ill-conditioned panel: exact-product Gram, float64 factor (replaces Rs)
            gram(std::integral_constant<int, 2>{});
            if (!coop_sync(p.bar, p.err)) return;
            reduce();
            if (!coop_sync(p.bar, p.err)) return;
            coop_factor_f64(bi, p.tau, cta == 0 ? p.flags : nullptr, p.wred,
                            CholShared<double, float>{reinterpret_cast<double (*)[CLD]>(sreg), Sf,
                                                      Li, dpiv, dinvd, didiag, ddiag0, &ddmax,
                                                      &weak_s},
                            Rs);
        }
        __syncthreads();
        if (chain) {
            // Pc <- Pc R^-1 (thread: row i, 8 consecutive columns)
            const int i = tid & 63, c0 = (tid >> 6) * 8;
            float acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = 0.f;
            for (int l2 = 0; l2 < MAXB; ++l2) {
                const float v = Pc[l2][i];
                const float4 r0v = *reinterpret_cast<const float4*>(&Rs[l2][c0]);
                const float4 r1v = *reinterpret_cast<const float4*>(&Rs[l2][c0 + 4]);
                acc[0] = fmaf(v, r0v.x, acc[0]);
                acc[1] = fmaf(v, r0v.y, acc[1]);
                acc[2] = fmaf(v, r0v.z, acc[2]);
                acc[3] = fmaf(v, r0v.w, acc[3]);
                acc[4] = fmaf(v, r1v.x, acc[4]);
                acc[5] = fmaf(v, r1v.y, acc[5]);
                acc[6] = fmaf(v, r1v.z, acc[6]);
                acc[7] = fmaf(v, r1v.w, acc[7]);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 8; ++q) Pc[c0 + q][i] = acc[q];
        }
        // ---- rows <- rows * R^-1 (R^-1 upper triangular).  Warp block (RG, CG) = 32 rows x 32
        // columns; lane (lane / 8, lane % 8) computes rows 8 rg .. 8 rg + 7 and columns
        // 4 cg .. 4 cg + 3 with terms q2 < 32 (CG + 1) (the others are zero), in the order
        // q2 = 0, 1, ...  Every row of a round is read before any of it is written.
        const bool last = pass + 1 == p.passes;
        for (int t = 0; t < ntile; ++t) {
            if (ntile > 1) {
                __syncthreads();
                load_tile(t);
                __syncthreads();
            }
            const int tn = ntile > 1 ? tile_rows(t) : nr;
            const int nrg = (tn + 7) >> 3, nblk = ((nrg + 3) >> 2) * 2;
            for (int base = 0; base < nblk; base += COOP_THREADS / 32) {
                const int bw = base + warp, CG = bw & 1;
                const int rg = 4 * (bw >> 1) + (lane >> 3), cg = 8 * CG + (lane & 7);
                const bool act = bw < nblk && rg < nrg;
                // acc[rp][c] holds rows 8 rg + 2 rp and 8 rg + 2 rp + 1 of column 4 cg + c: packed
                // float32-pair FMAs (round-to-nearest per element, the same sums as scalar FMAs)
                float2 acc[4][4];
#pragma unroll
                for (int rp = 0; rp < 4; ++rp)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[rp][c] = make_float2(0.f, 0.f);
                if (act) {
                    const int qmax = min(bi, 32 * CG + 32);
                    for (int q2 = 0; q2 < qmax; ++q2) {
                        const float4 u0 = *reinterpret_cast<const float4*>(Pt + pcol(q2) + 8 * rg);
                        const float4 u1 = *reinterpret_cast<const float4*>(Pt + pcol(q2) + 8 * rg + 4);
                        const float4 rv = *reinterpret_cast<const float4*>(&Rs[q2][4 * cg]);
                        const float2 u[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w),
                                             make_float2(u1.x, u1.y), make_float2(u1.z, u1.w)};
                        const float2 w2[4] = {make_float2(rv.x, rv.x), make_float2(rv.y, rv.y),
                                              make_float2(rv.z, rv.z), make_float2(rv.w, rv.w)};
#pragma unroll
                        for (int rp = 0; rp < 4; ++rp)
#pragma unroll
                            for (int c = 0; c < 4; ++c) acc[rp][c] = __ffma2_rn(u[rp], w2[c], acc[rp][c]);
                    }
                }
                __syncthreads();
                if (act) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float* dst = Pt + pcol(4 * cg + c) + 8 * rg;
#pragma unroll
                        for (int rp = 0; rp < 4; ++rp) {
                            if (8 * rg + 2 * rp < tn) dst[2 * rp] = acc[rp][c].x;
                            if (8 * rg + 2 * rp + 1 < tn) dst[2 * rp + 1] = acc[rp][c].y;
                        }
                    }
                }
            }
            __syncthreads();
            if (ntile > 1) store_tile(t, last);
        }
    }
    __syncthreads();
    if (chain) {
        for (int e = tid; e < MAXB * MAXB; e += COOP_THREADS)
            p.rinv_out[e] = double(Pc[e / MAXB][e % MAXB]);
    }
    if (ntile == 1) store_tile(0, true);
}

__global__ void k_identity(double* R, int bi) {
    for (int e = threadIdx.x; e < MAXB * MAXB; e += blockDim.x) {
        const int i = e % MAXB, j = e / MAXB;
        R[e] = (i == j && i < bi) ? 1.0 : 0.0;
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

// Squared norm of a float32 row: exact products summed as float32 pairs (two-sum), ~n u32^2 of
// relative error; the float64 chain it replaces ran on GB300's slow float64 pipe.  The block's
// partial pairs are combined in a fixed order (lanes by shuffles, then warps in order).
__global__ void k_row_norm2_f32(const float* __restrict__ B, int64_t ldb, int64_t n, double* rn) {
    const int j = blockIdx.x;
    const float* row = B + int64_t(j) * ldb;
    float hi = 0.f, lo = 0.f;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
        const float v = row[c];
        df_add(hi, lo, v, v);
    }
    float2 s = make_float2(hi, lo);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float2 t = make_float2(__shfl_down_sync(0xffffffffu, s.x, o),
                                     __shfl_down_sync(0xffffffffu, s.y, o));
        s = fp_add(s, t);
    }
    __shared__ float2 sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = make_float2(0.f, 0.f);
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t = fp_add(t, sh[w]);
        rn[j] = double(t.x) + double(t.y);
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


void chol_rinv(cudaStream_t st, const double* W, int bi, double tau_rel, double* R, double* Rinv,
               double* R_acc, int* flags, CholPrec prec) {
    switch (prec) {
        case CHOL_F64: {
            constexpr size_t sm = chol_smem<double, double>();
            smem_limit_once<k_chol<double, double, false>>(sm);
            k_chol<double, double, false><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv,
                                                                       R_acc, flags);
            break;
        }
        case CHOL_F64_INV_F32: {
            constexpr size_t sm = chol_smem<double, float>();
            smem_limit_once<k_chol<double, float, false>>(sm);
            k_chol<double, float, false><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv,
                                                                      R_acc, flags);
            break;
        }
        case CHOL_ADAPTIVE: {
            constexpr size_t sm = chol_smem<double, float>();
            smem_limit_once<k_chol<double, float, true>>(sm);
            k_chol<double, float, true><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv,
                                                                     R_acc, flags);
            break;
        }
        default: {
            constexpr size_t sm = chol_smem<float, float>();
            smem_limit_once<k_chol<float, float, false>>(sm);
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
    a.part = reinterpret_cast<float2*>(scratch);
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

void apply_rinv(cudaStream_t st, bool f64, void* P, int64_t ldp, int64_t m, int bi,
                const double* Rinv) {
    if (m <= 0) return;
    const unsigned g = unsigned(cdiv(m, APPLY_ROWS));
    if (f64) {
        const size_t sm = sizeof(double) * (MAXB * MAXB + APPLY_ROWS * LDS);
        smem_limit_once<k_apply_rinv<double>>(sm);
        k_apply_rinv<double><<<g, 256, sm, st>>>(reinterpret_cast<double*>(P), ldp, m, bi, Rinv);
    } else {
        const size_t sm = sizeof(float) * (MAXB * MAXB + APPLY_ROWS * LDS);
        smem_limit_once<k_apply_rinv<float>>(sm);
        k_apply_rinv<float><<<g, 256, sm, st>>>(reinterpret_cast<float*>(P), ldp, m, bi, Rinv);
    }
    QB_LAUNCHED();
}

void row_norm2(cudaStream_t st, bool f64, const void* B, int64_t ldb, int rows, int64_t n,
               double* rn) {
    if (rows <= 0) return;
    if (f64) k_row_norm2<double><<<rows, 256, 0, st>>>(reinterpret_cast<const double*>(B), ldb, n, rn);
    else k_row_norm2_f32<<<rows, 512, 0, st>>>(reinterpret_cast<const float*>(B), ldb, n, rn);
    QB_LAUNCHED();
}

void indicator(cudaStream_t st, double* state, const double* rn, int rows, double eps2,
               int row_by_row, const double* Wq, const double* Gb) {
    k_indicator<<<1, 32, 0, st>>>(state, rn, rows, eps2, row_by_row, Wq, Gb);
    QB_LAUNCHED();
}

}  // namespace qb
