// CholeskyQR panel pieces (b x b float64 Cholesky, triangular inverse, R accumulation, applying
// R^-1 to an m x b panel) and the Frobenius-norm indicator of Theorem 1 with the row-by-row
// stopping rule of Sect. 3.1.
#include "qb_internal.cuh"

namespace qb {
namespace {

constexpr int LDS = MAXB + 1;

// One CTA: W = R^T R (upper R), Rinv = R^-1, optional R_acc <- R R_acc.
// Breakdown: a pivot d <= tau_rel * max_diag(W) (or NaN) is replaced by tau_rel * max_diag (or
// the smallest normal double) and flags[1] is raised; the column it produces has norm <= 1.
// Dynamic shared memory: two MAXB x LDS float64 arrays (S holds W and becomes R in place).
template <class T>
__global__ void __launch_bounds__(256)
k_chol(const double* __restrict__ W, int bi, double tau_rel, double* __restrict__ Rout,
       double* __restrict__ Rinv, double* __restrict__ Racc, int* flags) {
    extern __shared__ double smem[];
    T (*S)[LDS] = reinterpret_cast<T (*)[LDS]>(smem);
    T (*X)[LDS] = reinterpret_cast<T (*)[LDS]>(reinterpret_cast<T*>(smem) + MAXB * LDS);
    __shared__ T piv;
    __shared__ T ipiv;
    __shared__ T dmax;
    __shared__ T idiag[MAXB];
    const int tid = threadIdx.x;
    for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
        const int i = e % MAXB, j = e / MAXB;
        S[i][j] = (i < bi && j < bi && i <= j) ? T(W[i + j * MAXB]) : T(0);
        X[i][j] = T(0);
    }
    __syncthreads();
    if (tid == 0) {
        T m = T(0);
        for (int i = 0; i < bi; ++i) m = S[i][i] > m ? S[i][i] : m;
        dmax = m;
    }
    __syncthreads();
    const T tiny = sizeof(T) == 8 ? T(2.2250738585072014e-308) : T(1.1754943508222875e-38);
    const T floor_piv = T(tau_rel) * dmax > tiny ? T(tau_rel) * dmax : tiny;
    for (int j = 0; j < bi; ++j) {
        if (tid == 0) {
            T d = S[j][j];
            if (!(d > T(tau_rel) * dmax)) {
                d = floor_piv;
                atomicOr(flags + 1, 1);
            }
            piv = sqrt(d);
            ipiv = T(1) / piv;
            idiag[j] = ipiv;
            S[j][j] = piv;
        }
        __syncthreads();
        for (int c = j + 1 + tid; c < bi; c += blockDim.x) S[j][c] *= ipiv;
        __syncthreads();
        // trailing update of the upper triangle: S[a][c] -= R[j][a] R[j][c], j < a <= c
        const int t = bi - j - 1;
        for (int e = tid; e < t * t; e += blockDim.x) {
            const int a = j + 1 + e % t, c = j + 1 + e / t;
            if (a <= c) S[a][c] -= S[j][a] * S[j][c];
        }
        __syncthreads();
    }
    // inverse of the upper-triangular R by back substitution, all columns at once: X[i][c]
    // (i < l) accumulates sum_{l' > i} R[i][l'] X[l'][c] while l sweeps down
    __syncthreads();
    for (int l = bi - 1; l >= 0; --l) {
        for (int c = l + tid; c < bi; c += blockDim.x)
            X[l][c] = (c == l ? T(1) : -X[l][c]) * idiag[l];
        __syncthreads();
        const int rows = l, cols = bi - l;
        for (int e = tid; e < rows * cols; e += blockDim.x) {
            const int i = e % rows, c = l + e / rows;
            X[i][c] = fma(S[i][l], X[l][c], X[i][c]);
        }
        __syncthreads();
    }
    for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
        const int i = e % MAXB, j = e / MAXB;
        if (Rout) Rout[i + j * MAXB] = i <= j ? double(S[i][j]) : 0.0;
        if (Rinv) Rinv[i + j * MAXB] = double(X[i][j]);
    }
    if (Racc) {
        // Racc <- R * Racc (both upper triangular); X reused for the old Racc
        __syncthreads();
        for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
            const int i = e % MAXB, j = e / MAXB;
            X[i][j] = T(Racc[i + j * MAXB]);
        }
        __syncthreads();
        for (int e = tid; e < MAXB * MAXB; e += blockDim.x) {
            const int i = e % MAXB, j = e / MAXB;
            T s = T(0);
            if (i < bi && j < bi)
                for (int l = i; l <= j; ++l) s = fma(S[i][l], X[l][j], s);
            Racc[i + j * MAXB] = double(s);
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

// P (rows x bi) <- P * Rinv, 64 rows per CTA, in place (each CTA owns its rows).
template <class T>
__global__ void __launch_bounds__(256)
k_apply_rinv(T* __restrict__ P, int64_t ldp, int64_t m, int bi, const double* __restrict__ Rinv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*Ps)[LDS] = reinterpret_cast<T (*)[LDS]>(smem_raw);                   // [row][col]
    T (*Rs)[LDS] = reinterpret_cast<T (*)[LDS]>(smem_raw + sizeof(T) * MAXB * LDS);  // [l][c]
    const int64_t r0 = int64_t(blockIdx.x) * 64;
    for (int e = threadIdx.x; e < MAXB * MAXB; e += blockDim.x) {
        const int i = e % MAXB, j = e / MAXB;
        Rs[i][j] = (i < bi && j < bi) ? T(Rinv[i + j * MAXB]) : T(0);
        const int64_t gr = r0 + i;
        Ps[i][j] = (gr < m && j < bi) ? P[gr + int64_t(j) * ldp] : T(0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * bi; e += blockDim.x) {
        const int i = e % 64, c = e / 64;
        const int64_t gr = r0 + i;
        if (gr >= m) continue;
        T s = T(0);
        for (int l = 0; l <= c; ++l) s = fma(Ps[i][l], Rs[l][c], s);
        P[gr + int64_t(c) * ldp] = s;
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
               double* R_acc, int* flags, bool f32) {
    if (f32) {
        allow_smem(k_chol<float>, CHOL_SMEM);
        k_chol<float><<<1, 256, CHOL_SMEM, st>>>(W, bi, tau_rel, R, Rinv, R_acc, flags);
    } else {
        allow_smem(k_chol<double>, CHOL_SMEM);
        k_chol<double><<<1, 256, CHOL_SMEM, st>>>(W, bi, tau_rel, R, Rinv, R_acc, flags);
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
    const unsigned g = unsigned(cdiv(m, 64));
    if (f64) {
        const size_t sm = sizeof(double) * 2 * MAXB * LDS;
        allow_smem(k_apply_rinv<double>, sm);
        k_apply_rinv<double><<<g, 256, sm, st>>>(reinterpret_cast<double*>(P), ldp, m, bi, Rinv);
    } else {
        const size_t sm = sizeof(float) * 2 * MAXB * LDS;
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
