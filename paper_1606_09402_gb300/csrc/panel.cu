// CholeskyQR panel pieces (b x b float64 Cholesky, triangular inverse, R accumulation, applying
// R^-1 to an m x b panel) and the Frobenius-norm indicator of Theorem 1 with the row-by-row
// stopping rule of Sect. 3.1.
#include "qb_internal.cuh"

namespace qb {
namespace {

constexpr int LDS = MAXB + 1;

// One CTA of 256 threads: W = R^T R (upper R) factored in TF, Rinv = R^-1 formed in TI, optional
// R_acc <- R R_acc (in TF).
// Breakdown: a pivot d <= tau_rel * max_diag(W) (or NaN) is replaced by tau_rel * max_diag (or
// the smallest normal number) and flags[1] is raised; the column it produces has norm <= 1.
//
// Factorisation: right-looking, one barrier per step.  Thread t owns column c = t % 64 of rows
// 16 (t / 64) .. 16 (t / 64) + 15 of the trailing matrix in registers; step j subtracts
// W[j][a] W[j][c] / d_j (the unnormalised row j, d_j its pivot) and publishes the finished row
// j + 1 to shared memory, the owner of its diagonal also its pivot and 1 / pivot, for the next
// step.  Inverse: each warp solves R x = e_c for 8 columns by back substitution, rows spread over
// the lanes, x_l broadcast by shuffle (no barriers).
// Dynamic shared memory: two MAXB x LDS arrays of TF (S: rows of W, then R; X: old R_acc).
template <class TF, class TI>
__global__ void __launch_bounds__(256)
k_chol(const double* __restrict__ W, int bi, double tau_rel, double* __restrict__ Rout,
       double* __restrict__ Rinv, double* __restrict__ Racc, int* flags) {
    using T = TF;
    extern __shared__ double smem[];
    T (*S)[LDS] = reinterpret_cast<T (*)[LDS]>(smem);
    T (*X)[LDS] = reinterpret_cast<T (*)[LDS]>(reinterpret_cast<T*>(smem) + MAXB * LDS);
    __shared__ T dpiv[MAXB];
    __shared__ T invd[MAXB];
    __shared__ T idiag[MAXB];
    __shared__ T dmax_s;
    const int tid = threadIdx.x;
    const int c = tid & (MAXB - 1);
    const int a0 = (tid >> 6) * 16;
    T s[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int a = a0 + k;
        s[k] = (a <= c && c < bi) ? T(W[a + c * MAXB]) : T(0);
        S[a][c] = s[k];
    }
    __syncthreads();
    if (tid < 32) {
        T m = T(0);
        for (int i = tid; i < bi; i += 32) m = S[i][i] > m ? S[i][i] : m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T v = __shfl_xor_sync(0xffffffffu, m, o);
            m = v > m ? v : m;
        }
        if (tid == 0) dmax_s = m;
    }
    __syncthreads();
    const T dmax = dmax_s;
    const T tiny = sizeof(T) == 8 ? T(2.2250738585072014e-308) : T(1.1754943508222875e-38);
    const T floor_piv = T(tau_rel) * dmax > tiny ? T(tau_rel) * dmax : tiny;
    // pivot of row j from its (updated) diagonal value; called by one thread
    auto pivot = [&](int j, T d) {
        if (!(d > T(tau_rel) * dmax)) {
            d = floor_piv;
            atomicOr(flags + 1, 1);
        }
        dpiv[j] = d;
        invd[j] = T(1) / d;
    };
    if (tid == 0 && bi > 0) pivot(0, S[0][0]);
    __syncthreads();
    for (int j = 0; j < bi; ++j) {
        const T t = S[j][c] * invd[j];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int a = a0 + k;
            if (a > j && a <= c && c < bi) s[k] = fma(-S[j][a], t, s[k]);
            if (a == j + 1 && a <= c) {
                S[a][c] = s[k];
                if (a == c && a < bi) pivot(a, s[k]);
            }
        }
        __syncthreads();
    }
    // R in place: R[j][j] = sqrt(d_j), R[j][c] = W'[j][c] / sqrt(d_j)
    if (tid < bi) idiag[tid] = T(1) / sqrt(dpiv[tid]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int a = a0 + k;
        if (a < bi && c < bi && a <= c) S[a][c] = a == c ? sqrt(dpiv[a]) : S[a][c] * idiag[a];
    }
    __syncthreads();
    // inverse in TI: warp w takes columns 8w .. 8w + 7; lane holds rows lane, lane + 32
    {
        const int warp = tid >> 5, lane = tid & 31;
        TI b[8][2];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int col = warp * 8 + q;
            b[q][0] = (lane == col && col < bi) ? TI(1) : TI(0);
            b[q][1] = (lane + 32 == col && col < bi) ? TI(1) : TI(0);
        }
        const int lmax = min(bi - 1, warp * 8 + 7);   // x_l = 0 for l above the warp's columns
        for (int l = lmax; l >= 0; --l) {
            const TI r0 = TI(S[lane][l]), r1 = TI(S[lane + 32][l]);
            const TI il = TI(idiag[l]);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const TI x = __shfl_sync(0xffffffffu, l < 32 ? b[q][0] : b[q][1], l & 31) * il;
                b[q][0] = lane < l ? fma(-r0, x, b[q][0]) : (lane == l ? x : b[q][0]);
                if (l >= 32)
                    b[q][1] = lane + 32 < l ? fma(-r1, x, b[q][1]) : (lane + 32 == l ? x : b[q][1]);
            }
        }
        if (Rinv) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int col = warp * 8 + q;
                Rinv[lane + col * MAXB] = double(b[q][0]);
                Rinv[lane + 32 + col * MAXB] = double(b[q][1]);
            }
        }
    }
    if (Rout) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int a = a0 + k;
            Rout[a + c * MAXB] = (a <= c && c < bi) ? double(S[a][c]) : 0.0;
        }
    }
    if (Racc) {
        // Racc <- R * Racc (both upper triangular); X holds the old Racc
        for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
            const int i = e % MAXB, j = e / MAXB;
            X[i][j] = T(Racc[i + j * MAXB]);
        }
        __syncthreads();
        for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
            const int i = e % MAXB, j = e / MAXB;
            T acc = T(0);
            if (i < bi && j < bi)
                for (int l = i; l <= j; ++l) acc = fma(S[i][l], X[l][j], acc);
            Racc[i + j * MAXB] = double(acc);
        }
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

constexpr size_t CHOL_SMEM = sizeof(double) * 2 * MAXB * LDS;

template <class K>
void allow_smem(K kernel, size_t bytes) {
    // idempotent, cheap; called before every launch so each device gets it
    QB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
}

void chol_rinv(cudaStream_t st, const double* W, int bi, double tau_rel, double* R, double* Rinv,
               double* R_acc, int* flags, CholPrec prec) {
    switch (prec) {
        case CHOL_F64:
            allow_smem(k_chol<double, double>, CHOL_SMEM);
            k_chol<double, double><<<1, 256, CHOL_SMEM, st>>>(W, bi, tau_rel, R, Rinv, R_acc, flags);
            break;
        case CHOL_F64_INV_F32:
            allow_smem(k_chol<double, float>, CHOL_SMEM);
            k_chol<double, float><<<1, 256, CHOL_SMEM, st>>>(W, bi, tau_rel, R, Rinv, R_acc, flags);
            break;
        default:
            allow_smem(k_chol<float, float>, CHOL_SMEM);
            k_chol<float, float><<<1, 256, CHOL_SMEM, st>>>(W, bi, tau_rel, R, Rinv, R_acc, flags);
            break;
    }
    QB_LAUNCHED();
}

void set_identity(cudaStream_t st, double* R, int bi) {
    k_identity<<<1, 256, 0, st>>>(R, bi);
    QB_LAUNCHED();
}

void tri_inv(cudaStream_t st, const double* R, int bi, double* Rinv) {
    allow_smem(k_tri_inv, CHOL_SMEM);
    k_tri_inv<<<1, 64, CHOL_SMEM, st>>>(R, bi, Rinv);
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
