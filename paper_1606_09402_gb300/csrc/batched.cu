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
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
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

// Asynchronous 4-byte global -> shared copies (cp.async, any alignment): src_bytes 0 writes a
// zero (used outside the matrix; src must still be a valid address).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc, bool valid) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gsrc),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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

// Y (slot of Q at column k) = A Omega; tile = 64 RT rows x b, thread = (RT rows, 4 columns).
// RT is a tile shape the autotuner picks per batch shape (more rows per thread reuse each Omega
// value RT times from shared memory).  The k-tiles of A and Omega are staged with asynchronous
// copies into two shared buffers, the next tile in flight while the current one is used.
template <int RT>
struct SkSmem {
    alignas(16) float O[2][64][BB];    // first: its rows are read as float4
    float A[2][ROWS * RT][65];
};

template <int RT>
__global__ void __launch_bounds__(NT) k_b_sketch(BDesc* D, Plan p) {
    extern __shared__ __align__(16) unsigned char sk_raw[];
    SkSmem<RT>& sm = *reinterpret_cast<SkSmem<RT>*>(sk_raw);
    FOR_ITEMS(p) {
        const int t = find_matrix(p, item);
        BDesc& d = D[t];
        if (d.done) continue;
        const int64_t r0 = (item - p.prefix[t]) * (ROWS * RT);
        const int row = threadIdx.x >> 2, cq = (threadIdx.x & 3) * 4;
        // copies: a warp takes 32 consecutive columns of a row (coalesced); thread t walks the
        // rows t/64 + 4q of column t%64 of the A tile and the columns t/64 + 4q of row t%64 of
        // the Omega tile with a fixed pointer step
        const int cj = threadIdx.x & 63, ci = threadIdx.x >> 6;
        auto issue = [&](int buf, int64_t k0) {
            const bool cok = k0 + cj < d.n;
            const int64_t rleft = d.m - (r0 + ci);     // rows of this thread's walk inside A
            const float* src = d.A + (rleft > 0 ? (r0 + ci) * d.lda : 0) + k0 + cj;
            float* dst = &sm.A[buf][ci][cj];
#pragma unroll
            for (int q = 0; q < ROWS * RT / 4; ++q) {
                const bool v = cok && 4 * q < rleft;
                cp_async4(dst + q * 4 * 65, v ? src + q * 4 * d.lda : d.A, v);
            }
            const float* osrc = d.Om + int64_t(ci) * d.n + k0 + cj;
#pragma unroll
            for (int q = 0; q < BB / 4; ++q)
                cp_async4(&sm.O[buf][cj][ci + 4 * q], cok ? osrc + q * 4 * d.n : d.Om, cok);
            cp_async_commit();
        };
        float acc[RT][4];
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
        const int64_t nk = (d.n + 63) / 64;
        __syncthreads();            // the buffers are free (previous item done with them)
        issue(0, 0);
        for (int64_t kt = 0; kt < nk; ++kt) {
            const int buf = int(kt & 1);
            if (kt + 1 < nk) {
                issue(buf ^ 1, (kt + 1) * 64);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
#pragma unroll 8
            for (int j = 0; j < 64; ++j) {
                const float4 o4 = *reinterpret_cast<const float4*>(&sm.O[buf][j][cq]);
                const float o[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
                for (int r = 0; r < RT; ++r) {
                    const float a = sm.A[buf][row + ROWS * r][j];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a, o[q], acc[r][q]);
                }
            }
            __syncthreads();        // done reading buf before it is refilled
        }
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            const int64_t gr = r0 + row + ROWS * r;
            if (gr < d.m) {
#pragma unroll
                for (int q = 0; q < 4; ++q) d.Y[gr + (cq + q) * d.m] = acc[r][q];
            }
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
        float lo[4] = {0.f, 0.f, 0.f, 0.f};   // MODE 1: low parts of the float32-pair sums
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
            if (MODE == 0) {
#pragma unroll 8
                for (int j = 0; j < 64; ++j) {
                    const float a = Xs[row][j];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] = fmaf(a, Vs[j][cq + q], acc[q]);
                }
            } else {
                // the re-orthogonalisation coefficients Q^T Y: exact products (fma residual) and
                // two-sum accumulation, so the coefficients carry ~u, not ~sqrt(m) u, of error;
                // what they miss is left along Q and feeds ||Q^T Q - I|| into the indicator
#pragma unroll 4
                for (int j = 0; j < 64; ++j) {
                    const float a = Xs[row][j];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float b = Vs[j][cq + q];
                        const float p = a * b, pe = fmaf(a, b, -p);
                        const float s2 = acc[q] + p, bb = s2 - acc[q];
                        lo[q] += ((acc[q] - (s2 - bb)) + (p - bb)) + pe;
                        acc[q] = s2;
                    }
                }
            }
        }
        const int64_t gr = r0 + row;
        if (gr < d.k) {
#pragma unroll
            for (int q = 0; q < 4; ++q) d.T[gr + (cq + q) * d.cap] = acc[q] + lo[q];
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
// CHOL = false: only the Gram of the (final) block, stored symmetric in d.W for the indicator.
template <bool CHOL>
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
        if (!CHOL) {
            for (int e = threadIdx.x; e < BB * BB; e += NT) {
                const int i = e % BB, j = e / BB;
                d.W[e] = i <= j ? Ws[i][j] : Ws[j][i];
            }
            __syncthreads();
            continue;
        }
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

// B_i (rows k..k+b of B) = Y^T A; tile = 64 CT columns of B; thread = (CT columns, 4 rows).
// CT is the autotuned tile shape of this stage.  Row tiles of A and Y are staged with
// asynchronous copies into two shared buffers (the next one in flight).
template <int CT>
struct BpSmem {
    alignas(16) float Y[2][64][BB];    // first: its rows are read as float4
    float A[2][64][64 * CT + 1];
};

template <int CT>
__global__ void __launch_bounds__(NT) k_b_bpass(BDesc* D, Plan p) {
    extern __shared__ __align__(16) unsigned char bp_raw[];
    BpSmem<CT>& sm = *reinterpret_cast<BpSmem<CT>*>(bp_raw);
    FOR_ITEMS(p) {
        const int t = find_matrix(p, item);
        BDesc& d = D[t];
        if (d.done) continue;
        const int64_t c0 = (item - p.prefix[t]) * (64 * CT);
        const float* Y = d.Y;
        const int col = threadIdx.x & 63, rq = (threadIdx.x >> 6) * 4;
        // copies: a warp takes 32 consecutive columns of a row (coalesced); thread t walks the
        // rows t/64 + 4q of columns t%64 + 64c of the A tile and the columns t/64 + 4q of row t%64
        // of the Y tile with a fixed pointer step
        const int cj = threadIdx.x & 63, ci = threadIdx.x >> 6;
        auto issue = [&](int buf, int64_t r0) {
            const int64_t rleft = d.m - (r0 + ci);
            const float* src = d.A + (rleft > 0 ? (r0 + ci) * d.lda : 0) + c0 + cj;
            float* dst = &sm.A[buf][ci][cj];
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                const bool cok = c0 + cj + 64 * c < d.n;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const bool v = cok && 4 * q < rleft;
                    cp_async4(dst + q * 4 * (64 * CT + 1) + 64 * c,
                              v ? src + q * 4 * d.lda + 64 * c : d.A, v);
                }
            }
            const bool yok = r0 + cj < d.m;
            const float* ysrc = Y + int64_t(ci) * d.m + r0 + cj;
#pragma unroll
            for (int q = 0; q < BB / 4; ++q)
                cp_async4(&sm.Y[buf][cj][ci + 4 * q], yok ? ysrc + q * 4 * d.m : Y, yok);
            cp_async_commit();
        };
        // B_i feeds the indicator: E misses 2 <B, B - Q^T A> of the true error, so the sum over m
        // rows is two-level (float32 within a 64-row tile, the tile sums into a float32 pair):
        // ~u of error instead of the plain chain's ~sqrt(m) u
        float acc[CT][4], hi[CT][4], lo[CT][4];
#pragma unroll
        for (int c = 0; c < CT; ++c)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[c][q] = hi[c][q] = lo[c][q] = 0.f;
        const int64_t nr = (d.m + 63) / 64;
        __syncthreads();
        issue(0, 0);
        for (int64_t rt = 0; rt < nr; ++rt) {
            const int buf = int(rt & 1);
            if (rt + 1 < nr) {
                issue(buf ^ 1, (rt + 1) * 64);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
#pragma unroll 8
            for (int i = 0; i < 64; ++i) {
                const float4 y4 = *reinterpret_cast<const float4*>(&sm.Y[buf][i][rq]);
                const float y[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int c = 0; c < CT; ++c) {
                    const float a = sm.A[buf][i][col + 64 * c];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[c][q] = fmaf(a, y[q], acc[c][q]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < CT; ++c)
#pragma unroll
                for (int q = 0; q < 4; ++q) {      // two-sum of the tile's sum into (hi, lo)
                    const float v = acc[c][q];
                    const float s2 = hi[c][q] + v, bb = s2 - hi[c][q];
                    lo[c][q] += (hi[c][q] - (s2 - bb)) + (v - bb);
                    hi[c][q] = s2;
                    acc[c][q] = 0.f;
                }
        }
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            const int64_t gc = c0 + col + 64 * c;
            if (gc < d.n) {
#pragma unroll
                for (int q = 0; q < 4; ++q) d.Bi[(rq + q) * d.n + gc] = hi[c][q] + lo[c][q];
            }
        }
    }
}

// Row norms of B_i (float64), row-by-row indicator (Sect. 3.1), append the kept columns of the
// new block to Q and rows to B, rank update; one CTA per matrix.
__global__ void __launch_bounds__(NT) k_b_indicator(BDesc* D, int count, int* active,
                                                    int row_by_row) {
    __shared__ double G[BB][BB + 1];
    __shared__ int keep_s;
    for (int t = blockIdx.x; t < count; t += gridDim.x) {
        BDesc& d = D[t];
        if (d.done) continue;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        // G = B_i B_i^T (float64), one warp per entry of the upper triangle
        constexpr int PAIRS = BB * (BB + 1) / 2;
        for (int pr = warp; pr < PAIRS; pr += NT / 32) {
            int a = 0, q = pr;
            while (q >= BB - a) { q -= BB - a; ++a; }
            const int c = a + q;
            double s = 0.0;
            for (int64_t x = lane; x < d.n; x += 32)
                s = fma(double(d.Bi[a * d.n + x]), double(d.Bi[c * d.n + x]), s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) { G[a][c] = s; G[c][a] = s; }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // Theorem 1 with a float32 Q: ||A - Q B||^2 = E + tr(B^T (Q^T Q - I) B) for B = Q^T A,
            // so each kept row j of the block also adds (W_jj - 1) G_jj + 2 sum_{p<j} W_pj G_pj,
            // W = Q_i^T Q_i (the final Gram of the block, exact-product sums; the terms between
            // blocks are second order after the re-orthogonalisation)
            const int bi = int(d.cap - d.k < BB ? d.cap - d.k : int64_t(BB));
            double E = d.E;
            int keep = bi, stop = 0;
            for (int j = 0; j < bi; ++j) {
                double corr = (d.W[j + j * BB] - 1.0) * G[j][j];
                for (int pp = 0; pp < j; ++pp) corr += 2.0 * d.W[pp + j * BB] * G[pp][j];
                E -= G[j][j];
                E += corr;
                if (row_by_row && E < d.eps2) { keep = j + 1; stop = 1; break; }
            }
            if (!row_by_row) stop = E < d.eps2;
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
namespace {
void prefix(std::vector<int64_t>& v, const std::vector<int64_t>& tiles) {
    v.assign(tiles.size() + 1, 0);
    for (size_t i = 0; i < tiles.size(); ++i) v[i + 1] = v[i] + tiles[i];
}

// Tile prefixes kept in the workspace: Omega rows, 64-row tiles, coefficient tiles, 64-column
// tiles, 128-row tiles (sketch, RT = 2), 128-column tiles (B pass, CT = 2).
constexpr int NPRE = 6;
enum { PRE_OMEGA = 0, PRE_ROWS, PRE_COEF, PRE_COLS, PRE_ROWS2, PRE_COLS2 };

// Launch plan of the two stages that stream A (the sketch Y = A Omega and the B pass B_i = Y^T A):
// tile shape (rows / columns per thread) and grid size.  The rest of the stages are fixed.
struct BatchedCfg {
    int rt = 1, ct = 1;      // tile shape: 64 rt rows per sketch tile, 64 ct columns per B tile
    int gsk = 0, gbp = 0;    // CTAs of the two launches
};

// Autotuner: the first call that sees a batch shape bucket times every candidate of the two
// A-streaming stages on the call's own matrices (both stages are pure functions of their inputs,
// so running them extra times changes nothing) and keeps the fastest per stage; later calls of the
// same bucket reuse the choice.  Bucket: (log2 of the matrix count, log2 of the mean m, log2 of
// the mean n).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, BatchedCfg> g_tune_cache;
BatchedCfg g_pinned;            // rt == 0: autotune (set by qb_batched_set_plan)
bool g_pinned_on = false;
int32_t g_last_plan[8] = {0};   // rt, ct, gsk, gbp, tuned this call, graph reused, cache entries

int ilog2c(double x) {
    int e = 0;
    while ((1LL << e) < int64_t(std::ceil(x))) ++e;
    return e;
}

// Instantiated graphs of earlier calls, keyed by everything a graph bakes in (workspace address
// and layout, shapes, plan, seed, stop rule): a repeated batch shape relaunches its graph.
struct GraphEntry {
    std::vector<int64_t> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels_per_iter = 0;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;   // most recently used last
constexpr size_t MAX_GRAPHS = 4;

}  // namespace

// Workspace layout (also used to measure it): descriptors, tile prefixes, flags, norm partials,
// then per matrix Omega (n x b), Y (m x b), B_i (b x n), T (cap x b), W / R^-1 / row norms.
struct BatchedWs {
    BDesc* D = nullptr;
    int64_t* pre[NPRE] = {};
    int* flags = nullptr;
    double* part = nullptr;
    double* nrm = nullptr;
    int* nf = nullptr;
};

void batched_reserve(Arena& ar, int32_t count, const qb_dense* As, int64_t cap_opt, BatchedWs& w,
                     std::vector<BDesc>* h) {
    w.D = ar.get<BDesc>(count);
    for (int s = 0; s < NPRE; ++s) w.pre[s] = ar.get<int64_t>(count + 1);
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

namespace {
// Raise a kernel's dynamic shared-memory limit once (per kernel, per process).
template <int TAG>
void allow_dyn_smem(const void* kern, size_t bytes) {
    static std::once_flag once;
    std::call_once(once, [&] {
        QB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
    });
}
void launch_sketch(int rt, unsigned g, cudaStream_t s, BDesc* D, const Plan& p1, const Plan& p2) {
    if (rt == 2) {
        allow_dyn_smem<0>(reinterpret_cast<const void*>(k_b_sketch<2>), sizeof(SkSmem<2>));
        k_b_sketch<2><<<g, NT, sizeof(SkSmem<2>), s>>>(D, p2);
    } else {
        allow_dyn_smem<1>(reinterpret_cast<const void*>(k_b_sketch<1>), sizeof(SkSmem<1>));
        k_b_sketch<1><<<g, NT, sizeof(SkSmem<1>), s>>>(D, p1);
    }
}
void launch_bpass(int ct, unsigned g, cudaStream_t s, BDesc* D, const Plan& p1, const Plan& p2) {
    if (ct == 2) {
        allow_dyn_smem<2>(reinterpret_cast<const void*>(k_b_bpass<2>), sizeof(BpSmem<2>));
        k_b_bpass<2><<<g, NT, sizeof(BpSmem<2>), s>>>(D, p2);
    } else {
        allow_dyn_smem<3>(reinterpret_cast<const void*>(k_b_bpass<1>), sizeof(BpSmem<1>));
        k_b_bpass<1><<<g, NT, sizeof(BpSmem<1>), s>>>(D, p1);
    }
}

// Time `reps` launches of fn on st (CUDA events), after one untimed launch.
template <class F>
float time_launches(cudaStream_t st, F fn, int reps) {
    cudaEvent_t e0, e1;
    QB_CUDA(cudaEventCreate(&e0));
    QB_CUDA(cudaEventCreate(&e1));
    fn();
    QB_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) fn();
    QB_CUDA(cudaEventRecord(e1, st));
    QB_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    QB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}
}  // namespace

}  // namespace qb

using namespace qb;

extern "C" size_t qb_ei_batched_workspace(int32_t count, const qb_dense* As, const qb_opts* opts) {
    if (count <= 0 || !As || !opts) return 0;
    return batched_workspace(count, As, opts->rank_cap);
}

extern "C" int32_t qb_batched_set_plan(const int32_t* cfg) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!cfg) {
        g_pinned_on = false;
        return QB_OK;
    }
    if ((cfg[0] != 1 && cfg[0] != 2) || (cfg[1] != 1 && cfg[1] != 2) || cfg[2] < 1 || cfg[3] < 1)
        return QB_ERR_INVALID_ARG;
    g_pinned = BatchedCfg{cfg[0], cfg[1], cfg[2], cfg[3]};
    g_pinned_on = true;
    return QB_OK;
}

extern "C" int32_t qb_batched_last_plan(int32_t* out, int32_t n) {
    if (!out || n < 0) return QB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int i = 0; i < n && i < 8; ++i) out[i] = g_last_plan[i];
    return 7;
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
        std::vector<int64_t> tiles[NPRE];
        for (auto& v : tiles) v.resize(count);
        int64_t max_iter = 0;
        double sum_m = 0, sum_n = 0;
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
            tiles[PRE_OMEGA][t] = cdiv(a.n, NT);
            tiles[PRE_ROWS][t] = cdiv(a.m, ROWS);
            tiles[PRE_COEF][t] = cdiv(d.cap, ROWS);
            tiles[PRE_COLS][t] = cdiv(a.n, 64);
            tiles[PRE_ROWS2][t] = cdiv(a.m, 2 * ROWS);
            tiles[PRE_COLS2][t] = cdiv(a.n, 128);
            max_iter = std::max<int64_t>(max_iter, cdiv(d.cap, BB));
            sum_m += double(a.m);
            sum_n += double(a.n);
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
        std::vector<int64_t> P[NPRE];
        for (int s2 = 0; s2 < NPRE; ++s2) prefix(P[s2], tiles[s2]);
        QB_CUDA(cudaMemcpyAsync(dD, h.data(), sizeof(BDesc) * count, cudaMemcpyHostToDevice, st));
        for (int s2 = 0; s2 < NPRE; ++s2)
            QB_CUDA(cudaMemcpyAsync(pre[s2], P[s2].data(), sizeof(int64_t) * (count + 1),
                                    cudaMemcpyHostToDevice, st));
        int init[2] = {1, 0};
        QB_CUDA(cudaMemcpyAsync(flags, init, sizeof init, cudaMemcpyHostToDevice, st));
        QB_CUDA(cudaStreamSynchronize(st));   // host vectors above die with this scope

        const Plan pOm{pre[PRE_OMEGA], count}, pRows{pre[PRE_ROWS], count},
            pCoef{pre[PRE_COEF], count}, pCols{pre[PRE_COLS], count},
            pRows2{pre[PRE_ROWS2], count}, pCols2{pre[PRE_COLS2], count};
        const int S = num_sms();
        const int G = 2 * S;
        auto grid_cap = [&](int64_t tiles_total, int64_t want) {
            return unsigned(std::max<int64_t>(1, std::min<int64_t>(tiles_total, want)));
        };
        const unsigned gOm = grid_cap(P[PRE_OMEGA].back(), 8LL * G),
                       gRows = grid_cap(P[PRE_ROWS].back(), 8LL * G),
                       gCoef = grid_cap(P[PRE_COEF].back(), 8LL * G),
                       gMat = unsigned(std::min(count, 4 * S));

        // ---- plan of the A-streaming stages: pinned, cached, or tuned now
        BatchedCfg cfg;
        int tuned_now = 0;
        const auto bucket = std::make_tuple(ilog2c(count), ilog2c(sum_m / count),
                                            ilog2c(sum_n / count));
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            if (g_pinned_on) {
                cfg = g_pinned;
                cfg.gsk = int(grid_cap(P[cfg.rt == 2 ? PRE_ROWS2 : PRE_ROWS].back(),
                                       int64_t(g_pinned.gsk) * S));
                cfg.gbp = int(grid_cap(P[cfg.ct == 2 ? PRE_COLS2 : PRE_COLS].back(),
                                       int64_t(g_pinned.gbp) * S));
            } else {
                auto it = g_tune_cache.find(bucket);
                if (it != g_tune_cache.end()) cfg = it->second;
            }
        }
        if (cfg.gsk == 0) {
            // candidates: tile shape x {4, 8, 16} CTAs per SM, each timed over 2 launches on this
            // batch after Omega has been drawn (the sketch reads it, the B pass reads Y)
            k_b_omega<<<gOm, NT, 0, st>>>(dD, pOm, opts->seed);
            QB_LAUNCHED();
            float best_sk = 1e30f, best_bp = 1e30f;
            for (int shape = 1; shape <= 2; ++shape) {
                for (int per_sm : {4, 8, 16}) {
                    const unsigned gs = grid_cap(P[shape == 2 ? PRE_ROWS2 : PRE_ROWS].back(),
                                                 int64_t(per_sm) * S);
                    const float ts = time_launches(st, [&] {
                        launch_sketch(shape, gs, st, dD, pRows, pRows2);
                        QB_LAUNCHED();
                    }, 2);
                    if (ts < best_sk) { best_sk = ts; cfg.rt = shape; cfg.gsk = int(gs); }
                    const unsigned gb = grid_cap(P[shape == 2 ? PRE_COLS2 : PRE_COLS].back(),
                                                 int64_t(per_sm) * S);
                    const float tb = time_launches(st, [&] {
                        launch_bpass(shape, gb, st, dD, pCols, pCols2);
                        QB_LAUNCHED();
                    }, 2);
                    if (tb < best_bp) { best_bp = tb; cfg.ct = shape; cfg.gbp = int(gb); }
                }
            }
            tuned_now = 1;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[bucket] = cfg;
        }

        auto body = [&](cudaStream_t s, int& kernels_per_iter) {
            kernels_per_iter = 0;
            auto L = [&]() { ++kernels_per_iter; QB_LAUNCHED(); };
            k_b_clear<<<1, 1, 0, s>>>(flags); L();
            k_b_omega<<<gOm, NT, 0, s>>>(dD, pOm, opts->seed); L();
            launch_sketch(cfg.rt, unsigned(cfg.gsk), s, dD, pRows, pRows2); L();
            k_b_coef<0><<<gCoef, NT, 0, s>>>(dD, pCoef); L();
            k_b_update<<<gRows, NT, 0, s>>>(dD, pRows); L();
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) {
                    k_b_coef<1><<<gCoef, NT, 0, s>>>(dD, pCoef); L();
                    k_b_update<<<gRows, NT, 0, s>>>(dD, pRows); L();
                }
                for (int q = 0; q < 2; ++q) {
                    k_b_gram_chol<true><<<gMat, NT, 0, s>>>(dD, count); L();
                    k_b_apply<<<gRows, NT, 0, s>>>(dD, pRows); L();
                }
            }
            k_b_gram_chol<false><<<gMat, NT, 0, s>>>(dD, count); L();   // Q_i^T Q_i for E
            launch_bpass(cfg.ct, unsigned(cfg.gbp), s, dD, pCols, pCols2); L();
            k_b_indicator<<<gMat, NT, 0, s>>>(dD, count, flags, opts->row_by_row); L();
        };

        // ---- the iteration under a conditional WHILE node: reuse the graph of an earlier call
        // with the same key, else capture and instantiate one (kept for the next call)
        std::vector<int64_t> key = {int64_t(reinterpret_cast<uintptr_t>(ws)), count,
                                    int64_t(opts->seed), opts->row_by_row, max_iter, cfg.rt,
                                    cfg.ct, cfg.gsk, cfg.gbp, int64_t(gOm), int64_t(gRows),
                                    int64_t(gCoef), int64_t(gMat), S};
        for (int t = 0; t < count; ++t) {
            key.push_back(h[t].m);
            key.push_back(h[t].n);
            key.push_back(h[t].cap);
        }
        cudaGraphExec_t exec = nullptr;
        int kernels_per_iter = 0;
        int reused = 0;
        std::unique_lock<std::mutex> glk(g_graph_mu);
        for (size_t i = 0; i < g_graphs.size(); ++i) {
            if (g_graphs[i].key == key) {
                GraphEntry e = g_graphs[i];
                g_graphs.erase(g_graphs.begin() + int64_t(i));
                g_graphs.push_back(e);
                exec = e.exec;
                kernels_per_iter = e.kernels_per_iter;
                reused = 1;
                break;
            }
        }
        if (!exec) {
            cudaGraph_t graph = nullptr;
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
            body(cs, kernels_per_iter);
            k_b_cond<<<1, 1, 0, cs>>>(handle, flags, flags + 1, int(max_iter));
            ++kernels_per_iter;
            QB_CUDA(cudaGetLastError());
            QB_CUDA(cudaStreamEndCapture(cs, &bodyg));
            QB_CUDA(cudaGraphInstantiate(&exec, graph, 0));
            cudaStreamDestroy(cs);
            GraphEntry e{key, graph, exec, kernels_per_iter};
            g_graphs.push_back(e);
            if (g_graphs.size() > MAX_GRAPHS) {
                cudaGraphExecDestroy(g_graphs.front().exec);
                cudaGraphDestroy(g_graphs.front().graph);
                g_graphs.erase(g_graphs.begin());
            }
        }
        QB_CUDA(cudaGraphLaunch(exec, st));
        glk.unlock();
        QB_CUDA(cudaStreamSynchronize(st));
        int iters = 0;
        QB_CUDA(cudaMemcpy(&iters, flags + 1, sizeof(int), cudaMemcpyDeviceToHost));
        // the capture counted no launches; the graph ran the body `iters` times
        for (int64_t i = (reused ? 0 : 1); i < int64_t(iters); ++i)
            for (int q = 0; q < kernels_per_iter; ++q) count_launch();
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_last_plan[0] = cfg.rt;
            g_last_plan[1] = cfg.ct;
            g_last_plan[2] = cfg.gsk;
            g_last_plan[3] = cfg.gbp;
            g_last_plan[4] = tuned_now;
            g_last_plan[5] = reused;
            g_last_plan[6] = int32_t(g_tune_cache.size());
        }

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
