// Batched randQB_EI (Algorithm 2, P = 0) over many independent float32 matrices of uneven shapes
// and tolerances.  Each stage of one EI iteration is ONE launch over the tiles of every matrix
// still running (grid-stride over a flattened (matrix, tile) list; finished matrices fall through
// at once), and the whole iteration is captured in a CUDA graph whose conditional WHILE node
// repeats it until every matrix has met its tolerance or its rank cap, with no host round trip.
//
// Per iteration, for every active matrix t (b columns, current rank k_t; the new block is built
// in workspace and only its kept rows/columns are appended to the caller's Q and B):
//   Omega_t,i = Philox columns [k_t, k_t + b) of seed + t;  Y = A_t Omega;  Y -= Q_t (B_t Omega);
//   CholeskyQR2(Y);  Y -= Q_t (Q_t^T Y);  CholeskyQR2(Y);  B_i = Y^T A_t;
//   E_t -= ||B_i(j,:)||^2 row by row (float64), stop at the first row with E_t < eps_t^2.
// Storage float32 (A, Q, B); Grams accumulated as float32 pairs (exact products), Cholesky and the
// indicator in float64.  Q_t column-major (ld m_t), B_t row-major (ld n_t), both caller-owned.
#include "qb_internal.cuh"

#include <algorithm>
#include <vector>

namespace qb {
namespace {

constexpr int BB = 16;          // block size of the batched path (columns per iteration)
constexpr int ROWS = 64;        // rows per tile
constexpr int NT = 256;         // threads per CTA

struct BDesc {
    const float* A;
    float* Q;
    float* B;
    float* Om;        // n x b, ld n
    float* Y;         // m x b, ld m: the new block before it is appended to Q
    float* Bi;        // b x n, ld n: the new rows before they are appended to B
    float* T;         // cap x b, ld cap
    double* W;        // b x b Gram (ld BB)
    double* Rinv;     // b x b
    double* rn;       // b row norms
    int64_t m, n, lda, ldq, ldb, cap;
    double eps2;      // stop threshold for E
    double E;         // indicator
    int64_t k;        // current rank
    int64_t blocks;
    int done;         // 1 converged, 2 rank cap
    int pad;
};

// tiles of each stage are laid out matrix after matrix; prefix[t] = first tile of matrix t
struct Plan {
    const int64_t* prefix;   // count + 1 entries
    int count;
};

__device__ __forceinline__ int find_matrix(const Plan& p, int64_t item) {
    int lo = 0, hi = p.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Philox4x32-10 + Box-Muller, the float32 variant of the library's Omega generator.
__device__ __forceinline__ float omega_f32(uint64_t seed, int64_t j, int64_t c) {
    uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
    uint32_t x = uint32_t(j), y = uint32_t(c >> 1), z = 0u, w = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * x, hi0 = __umulhi(0xD2511F53u, x);
        const uint32_t lo1 = 0xCD9E8D57u * z, hi1 = __umulhi(0xCD9E8D57u, z);
        const uint32_t nx = hi1 ^ y ^ k0, ny = lo1, nz = hi0 ^ w ^ k1, nw = lo0;
        x = nx; y = ny; z = nz; w = nw;
    }
    const float u1 = (float(x >> 8) + 0.5f) * 0x1.0p-24f;
    const float u2 = (float(z >> 8) + 0.5f) * 0x1.0p-24f;
    const float rho = sqrtf(-2.0f * logf(u1));
    float s, cs;
    sincospif(2.0f * u2, &s, &cs);
    return (c & 1) ? rho * s : rho * cs;
}

#define FOR_ITEMS(plan)                                                             \
    for (int64_t item = blockIdx.x; item < (plan).prefix[(plan).count];           \
         item += gridDim.x)

// Omega_t (n x b) for global columns [k_t, k_t + b); tile = 256 rows
__global__ void __launch_bounds__(NT) k_b_omega(BDesc* D, Plan p, uint64_t seed) {
    FOR_ITEMS(p) {
        const int t = find_matrix(p, item);
        BDesc& d = D[t];
        if (d.done) continue;
        const int64_t r = (item - p.prefix[t]) * NT + threadIdx.x;
        if (r >= d.n) continue;
        const int bi = int(d.cap - d.k < BB ? d.cap - d.k : int64_t(BB));
        for (int c = 0; c < BB; ++c)
            d.Om[r + c * d.n] = c < bi ? omega_f32(seed + uint64_t(t), r, d.k + c) : 0.f;
    }
}

// Y (slot of Q at column k) = A Omega; tile = 64 rows x b, thread = (row, 4 columns)
__global__ void __launch_bounds__(NT) k_b_sketch(BDesc* D, Plan p) {
    __shared__ float As[ROWS][65];
    __shared__ float Os[64][BB];
    FOR_ITEMS(p) {
        const int t = find_matrix(p, item);
        BDesc& d = D[t];
        if (d.done) continue;
        const int64_t r0 = (item - p.prefix[t]) * ROWS;
        const int row = threadIdx.x >> 2, cq = (threadIdx.x & 3) * 4;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t k0 = 0; k0 < d.n; k0 += 64) {
            __syncthreads();
            for (int e = threadIdx.x; e < ROWS * 64; e += NT) {
                const int i = e / 64, j = e % 64;
                const int64_t gr = r0 + i, gc = k0 + j;
                As[i][j] = (gr < d.m && gc < d.n) ? d.A[gr * d.lda + gc] : 0.f;
            }
            for (int e = threadIdx.x; e < 64 * BB; e += NT) {
                const int j = e % 64, c = e / 64;
                const int64_t gc = k0 + j;
                Os[j][c] = gc < d.n ? d.Om[gc + c * d.n] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int j = 0; j < 64; ++j) {
                const float a = As[row][j];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(a, Os[j][cq + q], acc[q]);
            }
        }
        const int64_t gr = r0 + row;
        if (gr < d.m) {
#pragma unroll
            for (int q = 0; q < 4; ++q) d.Y[gr + (cq + q) * d.m] = acc[q];
        }
    }
}

// T (k x b) = B Omega  (mode 0)  or  T = Q^T Y (mode 1); tile = 64 rows of T; K = n or m
template <int MODE>
__global__ void __launch_bounds__(NT) k_b_coef(BDesc* D, Plan p) {
    __shared__ float Xs[ROWS][65];
    __shared__ float Vs[64][BB];
    FOR_ITEMS(p) {
        const int t = find_matrix(p, item);
        BDesc& d = D[t];
        if (d.done || d.k == 0) continue;
        const int64_t r0 = (item - p.prefix[t]) * ROWS;
        if (r0 >= d.k) continue;
        const int64_t K = MODE == 0 ? d.n : d.m;
        const float* Y = d.Y;
        const int row = threadIdx.x >> 2, cq = (threadIdx.x & 3) * 4;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t k0 = 0; k0 < K; k0 += 64) {
            __syncthreads();
            for (int e = threadIdx.x; e < ROWS * 64; e += NT) {
                int i, j;
                float v = 0.f;
                if (MODE == 0) {            // B row-major: row i contiguous along n
                    i = e / 64; j = e % 64;
                    const int64_t gr = r0 + i, gc = k0 + j;
                    if (gr < d.k && gc < K) v = d.B[gr * d.ldb + gc];
                } else {                    // Q column-major: column i contiguous along m
                    i = e / 64; j = e % 64;
                    const int64_t gr = r0 + i, gc = k0 + j;
                    if (gr < d.k && gc < K) v = d.Q[gc + gr * d.ldq];
                }
                Xs[i][j] = v;
            }
            for (int e = threadIdx.x; e < 64 * BB; e += NT) {
                const int j = e % 64, c = e / 64;
                const int64_t gc = k0 + j;
                float v = 0.f;
                if (gc < K) v = MODE == 0 ? d.Om[gc + c * d.n] : Y[gc + c * d.m];
                Vs[j][c] = v;
            }
            __syncthreads();
#pragma unroll 8
            for (int j = 0; j < 64; ++j) {
                const float a = Xs[row][j];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(a, Vs[j][cq + q], acc[q]);
            }
        }
        const int64_t gr = r0 + row;
        if (gr < d.k) {
#pragma unroll
            for (int q = 0; q < 4; ++q) d.T[gr + (cq + q) * d.cap] = acc[q];
        }
    }
}

// Y -= Q T ; tile = 64 rows of Y
__global__ void __launch_bounds__(NT) k_b_update(BDesc* D, Plan p) {
    __shared__ float Qs[ROWS][65];
    __shared__ float Ts[64][BB];
    FOR_ITEMS(p) {
        const int t = find_matrix(p, item);
        BDesc& d = D[t];
        if (d.done || d.k == 0) continue;
        const int64_t r0 = (item - p.prefix[t]) * ROWS;
        float* Y = d.Y;
        const int row = threadIdx.x >> 2, cq = (threadIdx.x & 3) * 4;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t l0 = 0; l0 < d.k; l0 += 64) {
            __syncthreads();
            for (int e = threadIdx.x; e < ROWS * 64; e += NT) {
                const int i = e % ROWS, l = e / ROWS;
                const int64_t gr = r0 + i, gl = l0 + l;
                Qs[i][l] = (gr < d.m && gl < d.k) ? d.Q[gr + gl * d.ldq] : 0.f;
            }
            for (int e = threadIdx.x; e < 64 * BB; e += NT) {
                const int l = e % 64, c = e / 64;
                const int64_t gl = l0 + l;
                Ts[l][c] = gl < d.k ? d.T[gl + c * d.cap] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int l = 0; l < 64; ++l) {
                const float q = Qs[row][l];
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] = fmaf(q, Ts[l][cq + c], acc[c]);
            }
        }
        const int64_t gr = r0 + row;
        if (gr < d.m) {
#pragma unroll
            for (int c = 0; c < 4; ++c) Y[gr + (cq + c) * d.m] -= acc[c];
        }
    }
}

// Gram W = Y^T Y (float32 pair accumulation: exact products, ~48-bit sums), one CTA per matrix
// (thread = one entry of the upper triangle), then the b x b Cholesky W = R^T R and R^-1 in
// float64 by the first warp.  A pivot below 1e-12 of the largest is clamped (rank-deficient
// block: its column comes out with norm <= 1 and adds ~0 to ||B||^2).
__global__ void __launch_bounds__(NT) k_b_gram_chol(BDesc* D, int count) {
    __shared__ double Ws[BB][BB + 1];
    __shared__ double Xs[BB][BB + 1];
    constexpr int PAIRS = BB * (BB + 1) / 2;
    for (int t = blockIdx.x; t < count; t += gridDim.x) {
        BDesc& d = D[t];
        if (d.done) continue;
        for (int e = threadIdx.x; e < BB * (BB + 1); e += NT) Ws[e / (BB + 1)][e % (BB + 1)] = 0.0;
        __syncthreads();
        if (threadIdx.x < PAIRS) {
            int q = threadIdx.x, a = 0, c = 0;
            for (a = 0; a < BB; ++a) {
                const int len = BB - a;
                if (q < len) { c = a + q; break; }
                q -= len;
            }
            float hi = 0.f, lo = 0.f;
            for (int64_t r = 0; r < d.m; ++r) {
                const float x = d.Y[r + a * d.m], y = d.Y[r + c * d.m];
                const float pr = x * y, e = fmaf(x, y, -pr);
                const float s2 = hi + pr, bb = s2 - hi;
                const float err = (hi - (s2 - bb)) + (pr - bb);
                hi = s2;
                lo += err + e;
            }
            Ws[a][c] = double(hi) + double(lo);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            double dmax = 0.0;
            for (int i = 0; i < BB; ++i) dmax = fmax(dmax, Ws[i][i]);
            for (int j = 0; j < BB; ++j) {
                double piv = Ws[j][j];
                if (!(piv > 1e-12 * dmax)) piv = fmax(1e-12 * dmax, 1e-300);
                piv = sqrt(piv);
                __syncwarp();
                if (lane == 0) Ws[j][j] = piv;
                __syncwarp();
                if (lane > j && lane < BB) Ws[j][lane] /= piv;
                __syncwarp();
                if (lane > j && lane < BB)
                    for (int a2 = j + 1; a2 <= lane; ++a2) Ws[a2][lane] -= Ws[j][a2] * Ws[j][lane];
                __syncwarp();
            }
            if (lane < BB) {
                const int cc = lane;
                for (int i = 0; i < BB; ++i) Xs[i][cc] = 0.0;
                Xs[cc][cc] = 1.0 / Ws[cc][cc];
                for (int i = cc - 1; i >= 0; --i) {
                    double s = 0.0;
                    for (int l = i + 1; l <= cc; ++l) s = fma(Ws[i][l], Xs[l][cc], s);
                    Xs[i][cc] = -s / Ws[i][i];
                }
            }
            __syncwarp();
            for (int e = lane; e < BB * BB; e += 32) d.Rinv[e] = Xs[e % BB][e / BB];
        }
        __syncthreads();
    }
}

// Y <- Y R^-1 ; tile = 64 rows; thread = (row, 4 columns)
__global__ void __launch_bounds__(NT) k_b_apply(BDesc* D, Plan p) {
    __shared__ float Rs[BB][BB];
    FOR_ITEMS(p) {
        const int t = find_matrix(p, item);
        BDesc& d = D[t];
        if (d.done) continue;
        __syncthreads();
        if (threadIdx.x < BB * BB) Rs[threadIdx.x % BB][threadIdx.x / BB] = float(d.Rinv[threadIdx.x]);
        __syncthreads();
        const int64_t r0 = (item - p.prefix[t]) * ROWS;
        const int row = threadIdx.x >> 2, cq = (threadIdx.x & 3) * 4;
        const int64_t gr = r0 + row;
        const bool valid = gr < d.m;
        float y[BB];
#pragma unroll
        for (int l = 0; l < BB; ++l) y[l] = valid ? d.Y[gr + l * d.m] : 0.f;
        float out[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float s = 0.f;
#pragma unroll
            for (int l = 0; l < BB; ++l) s = fmaf(y[l], Rs[l][cq + c], s);
            out[c] = s;
        }
        __syncthreads();   // every read of this tile's rows precedes any write
        if (valid) {
#pragma unroll
            for (int c = 0; c < 4; ++c) d.Y[gr + (cq + c) * d.m] = out[c];
        }
    }
}

// B_i (rows k..k+b of B) = Y^T A; tile = 64 columns of B; thread = (column, 4 rows)
__global__ void __launch_bounds__(NT) k_b_bpass(BDesc* D, Plan p) {
    __shared__ float As[64][65];
    __shared__ float Ys[64][BB];
    FOR_ITEMS(p) {
        const int t = find_matrix(p, item);
        BDesc& d = D[t];
        if (d.done) continue;
        const int64_t c0 = (item - p.prefix[t]) * 64;
        const float* Y = d.Y;
        const int col = threadIdx.x & 63, rq = (threadIdx.x >> 6) * 4;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t r0 = 0; r0 < d.m; r0 += 64) {
            __syncthreads();
            for (int e = threadIdx.x; e < 64 * 64; e += NT) {
                const int i = e / 64, j = e % 64;
                const int64_t gr = r0 + i, gc = c0 + j;
                As[i][j] = (gr < d.m && gc < d.n) ? d.A[gr * d.lda + gc] : 0.f;
            }
            for (int e = threadIdx.x; e < 64 * BB; e += NT) {
                const int i = e % 64, c = e / 64;
                const int64_t gr = r0 + i;
                Ys[i][c] = gr < d.m ? Y[gr + c * d.m] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int i = 0; i < 64; ++i) {
                const float a = As[i][col];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(a, Ys[i][rq + q], acc[q]);
            }
        }
        const int64_t gc = c0 + col;
        if (gc < d.n) {
#pragma unroll
            for (int q = 0; q < 4; ++q) d.Bi[(rq + q) * d.n + gc] = acc[q];
        }
    }
}

// Row norms of B_i (float64), row-by-row indicator (Sect. 3.1), append the kept columns of the
// new block to Q and rows to B, rank update; one CTA per matrix.
__global__ void __launch_bounds__(NT) k_b_indicator(BDesc* D, int count, int* active,
                                                    int row_by_row) {
    __shared__ double rn[BB];
    __shared__ int keep_s;
    for (int t = blockIdx.x; t < count; t += gridDim.x) {
        BDesc& d = D[t];
        if (d.done) continue;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int rr = warp; rr < BB; rr += NT / 32) {
            double s = 0.0;
            for (int64_t c = lane; c < d.n; c += 32) {
                const double v = d.Bi[rr * d.n + c];
                s = fma(v, v, s);
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) rn[rr] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int bi = int(d.cap - d.k < BB ? d.cap - d.k : int64_t(BB));
            double E = d.E;
            int keep = bi, stop = 0;
            if (row_by_row) {
                for (int j = 0; j < bi; ++j) {
                    E -= rn[j];
                    if (E < d.eps2) { keep = j + 1; stop = 1; break; }
                }
            } else {
                for (int j = 0; j < bi; ++j) E -= rn[j];
                stop = E < d.eps2;
            }
            d.E = E;
            keep_s = keep;
            if (stop) d.done = 1;
            else if (d.k + keep >= d.cap) d.done = 2;
            if (!d.done) atomicOr(active, 1);
        }
        __syncthreads();
        const int keep = keep_s;
        for (int64_t e = threadIdx.x; e < int64_t(keep) * d.m; e += NT) {
            const int64_t c = e / d.m, r = e % d.m;
            d.Q[r + (d.k + c) * d.ldq] = d.Y[r + c * d.m];
        }
        for (int64_t e = threadIdx.x; e < int64_t(keep) * d.n; e += NT) {
            const int64_t r = e / d.n, c = e % d.n;
            d.B[(d.k + r) * d.ldb + c] = d.Bi[r * d.n + c];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            d.k += keep;
            d.blocks += 1;
        }
        __syncthreads();
    }
}

__global__ void k_b_clear(int* active) { *active = 0; }

// Continue the WHILE node while any matrix is running and the iteration budget lasts.
__global__ void k_b_cond(cudaGraphConditionalHandle h, int* active, int* iter, int max_iter) {
    const int it = ++(*iter);
    cudaGraphSetConditional(h, (*active != 0 && it < max_iter) ? 1u : 0u);
}

}  // namespace

// ------------------------------------------------------------------------------------ host side
struct BatchedPlan {
    std::vector<int64_t> pre_omega, pre_rows, pre_coefB, pre_coefQ, pre_cols;
};

namespace {
void prefix(std::vector<int64_t>& v, const std::vector<int64_t>& tiles) {
    v.assign(tiles.size() + 1, 0);
    for (size_t i = 0; i < tiles.size(); ++i) v[i + 1] = v[i] + tiles[i];
}
}  // namespace

// Workspace layout (also used to measure it): descriptors, tile prefixes, flags, norm partials,
// then per matrix Omega (n x b), Y (m x b), B_i (b x n), T (cap x b), W / R^-1 / row norms.
struct BatchedWs {
    BDesc* D = nullptr;
    int64_t* pre[5] = {};
    int* flags = nullptr;
    double* part = nullptr;
    double* nrm = nullptr;
    int* nf = nullptr;
};

void batched_reserve(Arena& ar, int32_t count, const qb_dense* As, int64_t cap_opt, BatchedWs& w,
                     std::vector<BDesc>* h) {
    w.D = ar.get<BDesc>(count);
    for (int s = 0; s < 5; ++s) w.pre[s] = ar.get<int64_t>(count + 1);
    w.flags = ar.get<int>(16);
    w.part = ar.get<double>(1024);
    w.nrm = ar.get<double>(count);
    w.nf = ar.get<int>(4);
    for (int t = 0; t < count; ++t) {
        const int64_t m = As[t].m, n = As[t].n;
        int64_t cap = std::min(m, n);
        if (cap_opt > 0) cap = std::min(cap, cap_opt);
        float* Om = ar.get<float>(n * BB);
        float* Y = ar.get<float>(m * BB);
        float* Bi = ar.get<float>(n * BB);
        float* T = ar.get<float>(std::max<int64_t>(cap, 1) * BB);
        double* W = ar.get<double>(BB * BB * 2 + BB);
        if (h) {
            BDesc& d = (*h)[t];
            d.Om = Om; d.Y = Y; d.Bi = Bi; d.T = T;
            d.W = W; d.Rinv = W + BB * BB; d.rn = d.Rinv + BB * BB;
            d.cap = cap;
        }
    }
}

size_t batched_workspace(int32_t count, const qb_dense* As, int64_t cap_opt) {
    Arena ar;
    BatchedWs w;
    batched_reserve(ar, count, As, cap_opt, w, nullptr);
    return ar.used + 4096;
}

}  // namespace qb

using namespace qb;

extern "C" size_t qb_ei_batched_workspace(int32_t count, const qb_dense* As, const qb_opts* opts) {
    if (count <= 0 || !As || !opts) return 0;
    return batched_workspace(count, As, opts->rank_cap);
}

extern "C" int32_t qb_ei_batched(int32_t count, const qb_dense* As, const double* tols,
                                 const qb_opts* opts, void* const* Qs, const int64_t* ldqs,
                                 void* const* Bs, const int64_t* ldbs, void* ws, size_t ws_bytes,
                                 qb_info* infos, void* stream) {
    if (count <= 0 || !As || !tols || !opts || !Qs || !ldqs || !Bs || !ldbs || !ws)
        return QB_ERR_INVALID_ARG;
    if (opts->b != BB || opts->P != 0 || opts->prec != QB_PREC_MIXED) return QB_ERR_UNSUPPORTED;
    for (int t = 0; t < count; ++t) {
        const qb_dense& a = As[t];
        if (a.dtype != QB_F32 || !a.a || a.m < 1 || a.n < 1 || a.ld < a.n || !Qs[t] || !Bs[t] ||
            ldqs[t] < a.m || ldbs[t] < a.n || !std::isfinite(tols[t]) || tols[t] < 0)
            return QB_ERR_INVALID_ARG;
    }
    if (ws_bytes < batched_workspace(count, As, opts->rank_cap)) return QB_ERR_WORKSPACE;
    try {
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        const int64_t l0 = launches_total();
        Arena ar;
        ar.base = reinterpret_cast<char*>(ws);
        ar.cap = ws_bytes;
        std::vector<BDesc> h(count);
        BatchedWs w;
        batched_reserve(ar, count, As, opts->rank_cap, w, &h);
        BDesc* dD = w.D;
        int64_t** pre = w.pre;
        int* flags = w.flags;
        std::vector<int64_t> t_omega(count), t_rows(count), t_coefB(count), t_cols(count);
        int64_t max_iter = 0;
        QB_CUDA(cudaMemsetAsync(w.nf, 0, 4 * sizeof(int), st));
        std::vector<double> nrm(count);
        for (int t = 0; t < count; ++t) {
            const qb_dense& a = As[t];
            BDesc& d = h[t];
            d.A = reinterpret_cast<const float*>(a.a);
            d.Q = reinterpret_cast<float*>(Qs[t]);
            d.B = reinterpret_cast<float*>(Bs[t]);
            d.m = a.m; d.n = a.n; d.lda = a.ld; d.ldq = ldqs[t]; d.ldb = ldbs[t];
            d.k = 0; d.blocks = 0; d.done = 0; d.pad = 0;
            if (std::isnan(a.src_norm2))
                dense_norm2(st, XOp{X_F32, a.a, nullptr, a.ld}, a.m, a.n, w.part, w.nrm + t, w.nf);
            t_omega[t] = cdiv(a.n, NT);
            t_rows[t] = cdiv(a.m, ROWS);
            t_coefB[t] = cdiv(d.cap, ROWS);
            t_cols[t] = cdiv(a.n, 64);
            max_iter = std::max<int64_t>(max_iter, cdiv(d.cap, BB));
        }
        QB_CUDA(cudaMemcpyAsync(nrm.data(), w.nrm, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
        QB_CUDA(cudaStreamSynchronize(st));
        for (int t = 0; t < count; ++t)
            if (!std::isnan(As[t].src_norm2)) nrm[t] = As[t].src_norm2;
        int nfh = 0;
        QB_CUDA(cudaMemcpy(&nfh, w.nf, sizeof(int), cudaMemcpyDeviceToHost));
        if (nfh) return QB_ERR_NONFINITE;
        for (int t = 0; t < count; ++t) {
            const double eps = opts->relative ? tols[t] * std::sqrt(nrm[t]) : tols[t];
            h[t].E = nrm[t];
            // Theorem 3 margin for float32 B (as on the single-matrix mixed path)
            h[t].eps2 = eps * eps - 2.0 * 5.9604644775390625e-08 * nrm[t];
            if (nrm[t] == 0.0) h[t].done = 1;
        }
        std::vector<int64_t> P[5];
        prefix(P[0], t_omega);
        prefix(P[1], t_rows);
        prefix(P[2], t_coefB);
        prefix(P[3], t_coefB);
        prefix(P[4], t_cols);
        QB_CUDA(cudaMemcpyAsync(dD, h.data(), sizeof(BDesc) * count, cudaMemcpyHostToDevice, st));
        for (int s = 0; s < 5; ++s)
            QB_CUDA(cudaMemcpyAsync(pre[s], P[s].data(), sizeof(int64_t) * (count + 1),
                                    cudaMemcpyHostToDevice, st));
        int init[2] = {1, 0};
        QB_CUDA(cudaMemcpyAsync(flags, init, sizeof init, cudaMemcpyHostToDevice, st));
        QB_CUDA(cudaStreamSynchronize(st));   // host vectors above die with this scope

        const Plan pOm{pre[0], count}, pRows{pre[1], count}, pCoef{pre[2], count},
            pCols{pre[4], count};
        const int G = 2 * num_sms();
        auto grid_for = [&](const std::vector<int64_t>& pv) {
            return unsigned(std::max<int64_t>(1, std::min<int64_t>(pv.back(), 8LL * G)));
        };
        const unsigned gOm = grid_for(P[0]), gRows = grid_for(P[1]), gCoef = grid_for(P[2]),
                       gCols = grid_for(P[4]), gMat = unsigned(std::min(count, 4 * num_sms()));
        int kernels_per_iter = 0;
        auto body = [&](cudaStream_t s) {
            kernels_per_iter = 0;
            auto L = [&]() { ++kernels_per_iter; QB_LAUNCHED(); };
            k_b_clear<<<1, 1, 0, s>>>(flags); L();
            k_b_omega<<<gOm, NT, 0, s>>>(dD, pOm, opts->seed); L();
            k_b_sketch<<<gRows, NT, 0, s>>>(dD, pRows); L();
            k_b_coef<0><<<gCoef, NT, 0, s>>>(dD, pCoef); L();
            k_b_update<<<gRows, NT, 0, s>>>(dD, pRows); L();
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) {
                    k_b_coef<1><<<gCoef, NT, 0, s>>>(dD, pCoef); L();
                    k_b_update<<<gRows, NT, 0, s>>>(dD, pRows); L();
                }
                for (int q = 0; q < 2; ++q) {
                    k_b_gram_chol<<<gMat, NT, 0, s>>>(dD, count); L();
                    k_b_apply<<<gRows, NT, 0, s>>>(dD, pRows); L();
                }
            }
            k_b_bpass<<<gCols, NT, 0, s>>>(dD, pCols); L();
            k_b_indicator<<<gMat, NT, 0, s>>>(dD, count, flags, opts->row_by_row); L();
        };

        // one iteration body under a conditional WHILE node
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        QB_CUDA(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle handle;
        QB_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        QB_CUDA(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
        cudaStream_t cs = nullptr;
        QB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        QB_CUDA(cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
        body(cs);
        k_b_cond<<<1, 1, 0, cs>>>(handle, flags, flags + 1, int(max_iter));
        ++kernels_per_iter;
        QB_CUDA(cudaGetLastError());
        QB_CUDA(cudaStreamEndCapture(cs, &bodyg));
        QB_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        QB_CUDA(cudaGraphLaunch(exec, st));
        QB_CUDA(cudaStreamSynchronize(st));
        int iters = 0;
        QB_CUDA(cudaMemcpy(&iters, flags + 1, sizeof(int), cudaMemcpyDeviceToHost));
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        // the capture counted one pass of kernels; the graph ran it `iters` times
        for (int64_t i = 1; i < int64_t(iters); ++i)
            for (int q = 0; q < kernels_per_iter; ++q) count_launch();

        std::vector<BDesc> out(count);
        QB_CUDA(cudaMemcpy(out.data(), dD, sizeof(BDesc) * count, cudaMemcpyDeviceToHost));
        int32_t worst = QB_OK;
        for (int t = 0; t < count; ++t) {
            const BDesc& d = out[t];
            int32_t bits = 0, status = QB_OK;
            if (d.done != 1) { bits |= QB_BIT_NOT_CONVERGED; status = QB_NOT_CONVERGED; }
            const double eps = opts->relative ? tols[t] * std::sqrt(nrm[t]) : tols[t];
            if (status == QB_OK && eps <= std::sqrt(4.0 * 5.9604644775390625e-08 / 0.01) *
                                              std::sqrt(nrm[t])) {
                bits |= QB_BIT_TOL_FLOOR;
                status = QB_WARN_TOL_FLOOR;
            }
            if (infos) {
                infos[t].rank = d.k;
                infos[t].err2_est = d.E;
                infos[t].err_est = std::sqrt(std::max(d.E, 0.0));
                infos[t].normA2 = nrm[t];
                infos[t].passes = 2 * d.blocks;
                infos[t].omega_cols = d.k;
                infos[t].status_bits = bits;
                infos[t].blocks = int32_t(d.blocks);
                infos[t].launches = launches_total() - l0;
            }
            if (status == QB_NOT_CONVERGED) worst = QB_NOT_CONVERGED;
            else if (status == QB_WARN_TOL_FLOOR && worst == QB_OK) worst = QB_WARN_TOL_FLOOR;
        }
        return worst;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return QB_ERR_CUDA;
    }
}
