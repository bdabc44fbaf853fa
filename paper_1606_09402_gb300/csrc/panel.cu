// CholeskyQR panel pieces (b x b float64 Cholesky, triangular inverse, R accumulation, applying
// R^-1 to an m x b panel) and the Frobenius-norm indicator of Theorem 1 with the row-by-row
// stopping rule of Sect. 3.1.
#include "qb_internal.cuh"

namespace qb {
namespace {

constexpr int LDS = MAXB + 1;

// Cholesky of a bi x bi Gram W (bi <= 64) by one CTA of 512 threads: W = R^T R (upper R) factored
// in TF, R^-1 formed in TI.
// Breakdown: a pivot d <= tau_rel * max_diag(W) (or NaN) is replaced by tau_rel * max_diag (or
// the smallest normal number) and flags[1] is raised; the column it produces has norm <= 1.
//
// One elimination sweep gives both factors: W = L D L^T (L unit lower), R = D^1/2 L^T and
// R^-1 = L^-T D^-1/2.  Step j removes row j from the rows a > j of [W | I] (Gaussian elimination
// without pivoting, multipliers m_a = W[j][a] / d_j read from the symmetric upper part), so the
// trailing upper triangle becomes the Schur complement and the right half becomes L^-1.  Thread t
// owns column t % 64 of rows 8 (t / 64) .. 8 (t / 64) + 7 of both halves in registers; the finished
// row j + 1 of each half (and its pivot) is published to shared memory for the next step, one
// barrier per step.  Rows of a warp with no work in a step are skipped with warp-uniform branches.
constexpr int CLD = MAXB + 4;          // shared row stride: rows stay 16-byte aligned
constexpr int CHOL_THREADS = 512;

template <class TF, class TI>
struct CholShared {
    TF (*S)[CLD];    // rows of W, then the rows W'[j][.] of the elimination
    TI (*Li)[CLD];   // rows of L^-1 as they are finished
    TF* dpiv;        // [MAXB] pivots d_j
    TF* invd;        // [MAXB] 1 / d_j
    TF* idiag;       // [MAXB] 1 / sqrt(d_j)
    TF* dmax;        // [1]
};

// load(i, j) returns W[i][j] for i <= j < bi.  On return (after a barrier) S rows hold W'[j][.],
// dpiv / idiag the pivots, and l[k] = L^-1[8 (t / 64) + k][t % 64].
template <class TF, class TI, class Load>
__device__ void chol_core(int bi, double tau_rel, int* flags, Load load, CholShared<TF, TI> sh,
                          TI (&l)[8]) {
    TF (*S)[CLD] = sh.S;
    TI (*Li)[CLD] = sh.Li;
    const int tid = threadIdx.x;
    const int c = tid & (MAXB - 1);
    const int a0 = (tid >> 6) * 8;
    const int cmin = c & 32, cmax = cmin + 31;   // columns of this warp
    TF s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int a = a0 + k;
        s[k] = (a <= c && c < bi) ? TF(load(a, c)) : TF(0);
        l[k] = (a == c && a < bi) ? TI(1) : TI(0);
        S[a][c] = s[k];
        Li[a][c] = l[k];
    }
    __syncthreads();
    if (tid < 32) {
        TF m = TF(0);
        for (int i = tid; i < bi; i += 32) m = S[i][i] > m ? S[i][i] : m;
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
        if (!(d > TF(tau_rel) * dmax)) {
            d = floor_piv;
            if (flags) atomicOr(flags + 1, 1);
        }
        sh.dpiv[j] = d;
        sh.invd[j] = TF(1) / d;
    };
    if (tid == 0 && bi > 0) pivot(0, S[0][0]);
    __syncthreads();
    for (int j = 0; j < bi; ++j) {
        const TF inv = sh.invd[j];
        const TF t = S[j][c] * inv;
        const TI u = Li[j][c];
        const TI inv_i = TI(inv);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int a = a0 + k;
            if (a > j) {
                const TF w = S[j][a];
                if (a <= cmax && a <= c && c < bi) s[k] = fma(-w, t, s[k]);
                if (j >= cmin && c <= j) l[k] = fma(-(TI(w) * inv_i), u, l[k]);
                if (a == j + 1) {
                    S[a][c] = s[k];
                    Li[a][c] = l[k];
                    if (a == c && a < bi) pivot(a, s[k]);
                }
            }
        }
        __syncthreads();
    }
    if (tid < bi) sh.idiag[tid] = TF(1) / sqrt(sh.dpiv[tid]);
    __syncthreads();
}

// Standalone: Rinv = R^-1 (and R, R_acc <- R R_acc when given), all MAXB x MAXB column-major.
template <class TF, class TI>
__global__ void __launch_bounds__(CHOL_THREADS)
k_chol(const double* __restrict__ W, int bi, double tau_rel, double* __restrict__ Rout,
       double* __restrict__ Rinv, double* __restrict__ Racc, int* flags) {
    extern __shared__ __align__(16) unsigned char chol_smem[];
    TF (*S)[CLD] = reinterpret_cast<TF (*)[CLD]>(chol_smem);
    TF (*X)[CLD] = reinterpret_cast<TF (*)[CLD]>(chol_smem + sizeof(TF) * MAXB * CLD);
    TI (*Li)[CLD] = reinterpret_cast<TI (*)[CLD]>(chol_smem + 2 * sizeof(TF) * MAXB * CLD);
    __shared__ TF dpiv[MAXB];
    __shared__ TF invd[MAXB];
    __shared__ TF idiag[MAXB];
    __shared__ TF dmax_s;
    const int tid = threadIdx.x;
    const int c = tid & (MAXB - 1);
    const int a0 = (tid >> 6) * 8;
    TI l[8];
    chol_core<TF, TI>(bi, tau_rel, flags, [&](int i, int j) { return W[i + j * MAXB]; },
                      CholShared<TF, TI>{S, Li, dpiv, invd, idiag, &dmax_s}, l);
    if (Rinv) {
        // R^-1[c][a] = L^-1[a][c] / sqrt(d_a)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int a = a0 + k;
            Rinv[c + a * MAXB] = (a < bi && c < bi) ? double(l[k] * TI(idiag[a])) : 0.0;
        }
    }
    if (!Rout && !Racc) return;
    // R in place: R[j][j] = sqrt(d_j), R[j][c] = W'[j][c] / sqrt(d_j); the lower part is zero
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int a = a0 + k;
        if (a < bi && c < bi && a <= c) S[a][c] = a == c ? sqrt(dpiv[a]) : S[a][c] * idiag[a];
    }
    __syncthreads();
    if (Rout) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int a = a0 + k;
            Rout[a + c * MAXB] = (a <= c && c < bi) ? double(S[a][c]) : 0.0;
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

// ---------------------------------------------------------------- fused CholeskyQR (float32 panel)
// One cooperative launch runs `passes` CholeskyQR passes on a float32 rows x bi panel: every CTA
// keeps its slice of rows in shared memory for the whole call, forms the partial Gram of the slice,
// the CTAs sum the partials (each CTA an equal share of the entries, in CTA order), every CTA
// factors the 64 x 64 Gram itself (chol_core; the same arithmetic in every CTA, so the same R),
// and applies R^-1 to its rows.  The panel is read and written once.  Grid-wide barriers use a
// global arrive counter and generation word; every wait is bounded and a timeout sets err.
constexpr int COOP_THREADS = 512;
constexpr int COOP_ROWS = 512;      // rows per CTA held in shared memory
constexpr int COOP_MAX_CTAS = 256;
constexpr int PLD = MAXB + 1;       // shared row stride of the panel slice
constexpr uint64_t COOP_WAIT_NS = 2000000000ull;

struct CoopArgs {
    float* P;
    int64_t ldp, rows, rows_per;
    int bi, passes;
    double tau;
    double* rinv_out;   // passes x (MAXB x MAXB) or null
    float* part;        // gridDim.x x (MAXB x MAXB) partial Grams
    float* wred;        // MAXB x MAXB summed Gram
    unsigned* bar;      // [0] arrivals, [1] generation
    int* flags;         // flags[1]: breakdown
    int* err;           // set when a grid barrier wait timed out
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

__global__ void __launch_bounds__(COOP_THREADS, 1) k_cholqr_coop(CoopArgs p) {
    extern __shared__ __align__(16) unsigned char coop_smem[];
    float (*Ps)[PLD] = reinterpret_cast<float (*)[PLD]>(coop_smem);
    unsigned char* rest = coop_smem + sizeof(float) * COOP_ROWS * PLD;
    float (*S)[CLD] = reinterpret_cast<float (*)[CLD]>(rest);
    float (*Li)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + sizeof(float) * MAXB * CLD);
    float (*Rs)[CLD] = reinterpret_cast<float (*)[CLD]>(rest + 2 * sizeof(float) * MAXB * CLD);
    float* scratch = reinterpret_cast<float*>(rest);   // Gram combine space (S and Li, 2 x 17 KB)
    __shared__ float dpiv[MAXB], invd[MAXB], idiag[MAXB], dmax_s;
    __shared__ double red[16][32];
    const int tid = threadIdx.x;
    const int G = gridDim.x, cta = blockIdx.x;
    const int bi = p.bi;
    const int64_t r0 = int64_t(cta) * p.rows_per;
    const int64_t r_end = p.rows < r0 + p.rows_per ? p.rows : r0 + p.rows_per;
    const int nr = r_end > r0 ? int(r_end - r0) : 0;
    for (int e = tid; e < nr * MAXB; e += COOP_THREADS) {
        const int r = e % nr, col = e / nr;
        Ps[r][col] = col < bi ? p.P[r0 + r + int64_t(col) * p.ldp] : 0.f;
    }
    // Gram block of thread t < 3 * 136: the (t % 136)-th 4 x 4 block of the upper triangle over
    // rows t / 136, t / 136 + 3, ...
    const int blk = tid % 136, grp = tid / 136;
    int gi = 0, gj = 0;
    {
        int t = blk;
        while (t >= 16 - gi) { t -= 16 - gi; ++gi; }
        gj = gi + t;
    }
    for (int pass = 0; pass < p.passes; ++pass) {
        __syncthreads();
        // ---- partial Gram of this slice
        if (grp < 3) {
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
            for (int r = grp; r < nr; r += 3) {
                float x[4], y[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    x[q] = Ps[r][gi * 4 + q];
                    y[q] = Ps[r][gj * 4 + q];
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(x[a], y[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) scratch[(grp * 136 + blk) * 16 + a * 4 + b] = acc[a][b];
        }
        __syncthreads();
        if (tid < 136) {
            float* out = p.part + int64_t(cta) * MAXB * MAXB;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float v = scratch[blk * 16 + q] + scratch[(136 + blk) * 16 + q] +
                                scratch[(272 + blk) * 16 + q];
                out[(gi * 4 + q / 4) + (gj * 4 + q % 4) * MAXB] = v;
            }
        }
        if (!coop_sync(p.bar, p.err)) return;
        // ---- sum the partials: this CTA owns entries [e0, e0 + 32 * nchunk)
        {
            const int per = (MAXB * MAXB + G - 1) / G;
            const int e0 = cta * per, e1 = min(MAXB * MAXB, e0 + per);
            const int lane = tid & 31, sub = tid >> 5;   // 16 subsets of the partials
            for (int eb = e0; eb < e1; eb += 32) {
                const int e = eb + lane;
                double v = 0.0;
                if (e < e1 && e % MAXB <= e / MAXB)
                    for (int q = sub; q < G; q += 16)
                        v += double(__ldcg(p.part + int64_t(q) * MAXB * MAXB + e));
                red[sub][lane] = v;
                __syncthreads();
                if (sub == 0 && e < e1) {
                    double t = 0.0;
#pragma unroll
                    for (int q = 0; q < 16; ++q) t += red[q][lane];
                    p.wred[e] = float(t);
                }
                __syncthreads();
            }
        }
        if (!coop_sync(p.bar, p.err)) return;
        // ---- every CTA factors the summed Gram
        float l[8];
        chol_core<float, float>(bi, p.tau, cta == 0 ? p.flags : nullptr,
                                [&](int i, int j) { return __ldcg(p.wred + i + j * MAXB); },
                                CholShared<float, float>{S, Li, dpiv, invd, idiag, &dmax_s}, l);
        {
            const int c = tid & (MAXB - 1), a0 = (tid >> 6) * 8;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int a = a0 + k;
                const float v = (a < bi && c < bi) ? l[k] * idiag[a] : 0.f;
                Rs[c][a] = v;                                   // R^-1[c][a]
                if (cta == 0 && p.rinv_out) p.rinv_out[int64_t(pass) * MAXB * MAXB + c + a * MAXB] = v;
            }
        }
        __syncthreads();
        // ---- rows <- rows * R^-1, 128 rows at a time (thread: one row, 16 columns)
        {
            const int i = tid & 127, c0 = (tid >> 7) * 16;
            for (int rb = 0; rb < nr; rb += 128) {
                const int r = rb + i;
                float acc[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = 0.f;
                if (r < nr) {
                    for (int q2 = 0; q2 < bi; ++q2) {
                        const float v = Ps[r][q2];
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc[q] = fmaf(v, Rs[q2][c0 + q], acc[q]);
                    }
                }
                __syncthreads();
                if (r < nr) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) Ps[r][c0 + q] = acc[q];
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < nr * MAXB; e += COOP_THREADS) {
        const int r = e % nr, col = e / nr;
        if (col < bi) p.P[r0 + r + int64_t(col) * p.ldp] = Ps[r][col];
    }
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
__global__ void k_indicator(double* state, const double* rn, int rows, double eps2,
                            int row_by_row) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double E = state[0];
    state[3] = E;
    int keep = rows;
    int stop = 0;
    if (row_by_row) {
        for (int j = 0; j < rows; ++j) {
            E -= rn[j];
            if (E < eps2) { keep = j + 1; stop = 1; break; }
        }
    } else {
        double s = 0.0;
        for (int j = 0; j < rows; ++j) s += rn[j];
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
    return (2 * sizeof(TF) + sizeof(TI)) * MAXB * CLD;
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
            allow_smem(k_chol<double, double>, sm);
            k_chol<double, double><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv, R_acc, flags);
            break;
        }
        case CHOL_F64_INV_F32: {
            constexpr size_t sm = chol_smem<double, float>();
            allow_smem(k_chol<double, float>, sm);
            k_chol<double, float><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv, R_acc, flags);
            break;
        }
        default: {
            constexpr size_t sm = chol_smem<float, float>();
            allow_smem(k_chol<float, float>, sm);
            k_chol<float, float><<<1, CHOL_THREADS, sm, st>>>(W, bi, tau_rel, R, Rinv, R_acc, flags);
            break;
        }
    }
    QB_LAUNCHED();
}

size_t cholqr_coop_scratch_bytes() {
    return size_t(COOP_MAX_CTAS) * MAXB * MAXB * sizeof(float) + MAXB * MAXB * sizeof(float) + 256;
}

bool cholqr_coop(cudaStream_t st, float* P, int64_t ldp, int64_t rows, int bi, int passes,
                 double tau, double* rinv_out, void* scratch, size_t scratch_bytes, unsigned* bar,
                 int* flags, int* err) {
    static int max_ctas = -1;
    constexpr size_t sm = sizeof(float) * (COOP_ROWS * PLD + 3 * MAXB * CLD);
    if (max_ctas < 0) {
        int dev = 0, coop = 0, per_sm = 0;
        QB_CUDA(cudaGetDevice(&dev));
        QB_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        QB_CUDA(cudaFuncSetAttribute(k_cholqr_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(sm)));
        QB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cholqr_coop, COOP_THREADS,
                                                               sm));
        max_ctas = coop ? std::min(per_sm * num_sms(), COOP_MAX_CTAS) : 0;
    }
    if (max_ctas <= 0 || bi < 1 || bi > MAXB || rows <= 0 || passes < 1) return false;
    int G = int(std::min<int64_t>(max_ctas, cdiv(rows, 64)));
    const int64_t rows_per = cdiv(rows, G);
    if (rows_per > COOP_ROWS) return false;
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
    a.rinv_out = rinv_out;
    a.part = reinterpret_cast<float*>(scratch);
    a.wred = a.part + size_t(COOP_MAX_CTAS) * MAXB * MAXB;
    a.bar = bar;
    a.flags = flags;
    a.err = err;
    void* args[] = {&a};
    QB_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_cholqr_coop), dim3(G),
                                        dim3(COOP_THREADS), args, sm, st));
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
               int row_by_row) {
    k_indicator<<<1, 32, 0, st>>>(state, rn, rows, eps2, row_by_row);
    QB_LAUNCHED();
}

}  // namespace qb
