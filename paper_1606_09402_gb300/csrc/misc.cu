// Omega generation (Philox4x32-10 + Box-Muller), norms, quantisation, copies.
#include "qb_internal.cuh"

namespace qb {
namespace {

// Philox4x32-10 (Salmon et al., SC'11): two 32x32->64 multiplications per round, key bumped by
// the Weyl constants before every round but the first.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

// One thread per (row j, column pair): both Box-Muller outputs of one counter are written.
template <int KIND>  // 0 = f64, 1 = f32, 2 = bf16
__global__ void k_omega(int64_t n, int64_t col0, int64_t w, uint32_t k0, uint32_t k1, void* out,
                        int64_t ld) {
    const int64_t pairs = (col0 + w + 1) / 2 - col0 / 2;
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n * pairs) return;
    const int64_t j = idx % n;
    const int64_t pc = col0 / 2 + idx / n;  // counter word 1 = c / 2
    const U4 r = philox4x32_10(U4{uint32_t(j), uint32_t(pc), 0u, 0u}, k0, k1);
    double z0, z1;
    float f0, f1;
    if (KIND == 0) {
        const uint64_t a = ((uint64_t(r.x) << 32) | r.y) >> 11;
        const uint64_t b = ((uint64_t(r.z) << 32) | r.w) >> 11;
        const double u1 = (double(a) + 0.5) * 0x1.0p-53;
        const double u2 = (double(b) + 0.5) * 0x1.0p-53;
        const double rho = sqrt(-2.0 * log(u1));
        double s, c;
        sincospi(2.0 * u2, &s, &c);
        z0 = rho * c;
        z1 = rho * s;
    } else {
        const float u1 = (float(r.x >> 8) + 0.5f) * 0x1.0p-24f;
        const float u2 = (float(r.z >> 8) + 0.5f) * 0x1.0p-24f;
        const float rho = sqrtf(-2.0f * logf(u1));
        float s, c;
        sincospif(2.0f * u2, &s, &c);
        f0 = rho * c;
        f1 = rho * s;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t c = 2 * pc + h;
        if (c < col0 || c >= col0 + w) continue;
        const int64_t o = j + (c - col0) * ld;
        if (KIND == 0) reinterpret_cast<double*>(out)[o] = h ? z1 : z0;
        else if (KIND == 1) reinterpret_cast<float*>(out)[o] = h ? f1 : f0;
        else reinterpret_cast<bf16*>(out)[o] = __float2bfloat16_rn(h ? f1 : f0);
    }
}

__global__ void k_to_bf16(const float* X, int64_t ldx, int64_t rows, int64_t cols, bf16* Y,
                          int64_t ldy) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx % rows, j = idx / rows;
    Y[i + j * ldy] = __float2bfloat16_rn(X[i + j * ldx]);
}

template <class T>
__global__ void k_copy_cols(const T* X, int64_t ldx, int64_t rows, int64_t cols, T* Y,
                            int64_t ldy) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx % rows, j = idx / rows;
    Y[i + j * ldy] = X[i + j * ldx];
}

// Block-level float64 sum, result in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

constexpr int NPART = 1024;

template <int KIND>  // XKind
__global__ void k_dense_norm2(const void* p, const void* lo, int64_t ld, int64_t m, int64_t n,
                              double* part, int* flags) {
    double s = 0.0;
    bool bad = false;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            double v;
            const int64_t o = i * ld + j;
            if (KIND == X_F64) v = reinterpret_cast<const double*>(p)[o];
            else if (KIND == X_F32) v = reinterpret_cast<const float*>(p)[o];
            else if (KIND == X_BF16) v = __bfloat162float(reinterpret_cast<const bf16*>(p)[o]);
            else v = double(__bfloat162float(reinterpret_cast<const bf16*>(p)[o])) +
                     double(__bfloat162float(reinterpret_cast<const bf16*>(lo)[o]));
            bad |= !isfinite(v);
            s = fma(v, v, s);
        }
    }
    s = block_sum(s);
    if (bad) atomicOr(flags, 1);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <bool F64>
__global__ void k_vec_norm2(const void* v, int64_t count, double* part, int* flags) {
    double s = 0.0;
    bool bad = false;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x) {
        const double x = F64 ? reinterpret_cast<const double*>(v)[i]
                             : double(reinterpret_cast<const float*>(v)[i]);
        bad |= !isfinite(x);
        s = fma(x, x, s);
    }
    s = block_sum(s);
    if (bad) atomicOr(flags, 1);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double* part, int count, int stride, double* out, int nout) {
    for (int q = 0; q < nout; ++q) {
        double s = 0.0;
        for (int i = threadIdx.x; i < count; i += blockDim.x) s += part[q * stride + i];
        s = block_sum(s);
        if (threadIdx.x == 0) out[q] = s;
        __syncthreads();
    }
}

// A = hi + lo: hi = bf16(a), lo = bf16(a - hi); float64 partial sums of a^2, (a-hi-lo)^2, (a-hi)^2
__global__ void k_quant(const double* src, int64_t lds, int64_t m, int64_t n, bf16* hi, bf16* lo,
                        int64_t ld, double* part) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            const double a = src[i * lds + j];
            const bf16 h = __double2bfloat16(a);
            const double r = a - double(__bfloat162float(h));
            const bf16 l = __double2bfloat16(r);
            const double d = r - double(__bfloat162float(l));
            hi[i * ld + j] = h;
            lo[i * ld + j] = l;
            s0 = fma(a, a, s0);
            s1 = fma(d, d, s1);
            s2 = fma(r, r, s2);
        }
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    s2 = block_sum(s2);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s0;
        part[NPART + blockIdx.x] = s1;
        part[2 * NPART + blockIdx.x] = s2;
    }
}

}  // namespace

void omega_gen(cudaStream_t st, int64_t n, int64_t col0, int64_t w, uint64_t seed, int dtype,
               void* out, int64_t ld) {
    if (n <= 0 || w <= 0) return;
    const int64_t pairs = (col0 + w + 1) / 2 - col0 / 2;
    const int64_t tot = n * pairs;
    const uint32_t k0 = uint32_t(seed & 0xffffffffu), k1 = uint32_t(seed >> 32);
    const unsigned grid = unsigned(cdiv(tot, 256));
    if (dtype == QB_F64) k_omega<0><<<grid, 256, 0, st>>>(n, col0, w, k0, k1, out, ld);
    else if (dtype == QB_F32) k_omega<1><<<grid, 256, 0, st>>>(n, col0, w, k0, k1, out, ld);
    else k_omega<2><<<grid, 256, 0, st>>>(n, col0, w, k0, k1, out, ld);
    QB_LAUNCHED();
}

void to_bf16(cudaStream_t st, const float* X, int64_t ldx, int64_t rows, int64_t cols, bf16* Y,
             int64_t ldy) {
    if (rows <= 0 || cols <= 0) return;
    k_to_bf16<<<unsigned(cdiv(rows * cols, 256)), 256, 0, st>>>(X, ldx, rows, cols, Y, ldy);
    QB_LAUNCHED();
}

void copy_cols(cudaStream_t st, bool f64, const void* X, int64_t ldx, int64_t rows, int64_t cols,
               void* Y, int64_t ldy) {
    if (rows <= 0 || cols <= 0) return;
    const unsigned g = unsigned(cdiv(rows * cols, 256));
    if (f64)
        k_copy_cols<double><<<g, 256, 0, st>>>(reinterpret_cast<const double*>(X), ldx, rows,
                                               cols, reinterpret_cast<double*>(Y), ldy);
    else
        k_copy_cols<float><<<g, 256, 0, st>>>(reinterpret_cast<const float*>(X), ldx, rows, cols,
                                              reinterpret_cast<float*>(Y), ldy);
    QB_LAUNCHED();
}

void fill_zero(cudaStream_t st, void* p, size_t bytes) {
    if (bytes) QB_CUDA(cudaMemsetAsync(p, 0, bytes, st));
}

void dense_norm2(cudaStream_t st, XOp A, int64_t m, int64_t n, double* part, double* out,
                 int* flags) {
    const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(m, NPART)));
    switch (A.kind) {
        case X_F64: k_dense_norm2<X_F64><<<g, 256, 0, st>>>(A.p, A.lo, A.ld, m, n, part, flags); break;
        case X_F32: k_dense_norm2<X_F32><<<g, 256, 0, st>>>(A.p, A.lo, A.ld, m, n, part, flags); break;
        case X_BF16: k_dense_norm2<X_BF16><<<g, 256, 0, st>>>(A.p, A.lo, A.ld, m, n, part, flags); break;
        case X_BF16X2: k_dense_norm2<X_BF16X2><<<g, 256, 0, st>>>(A.p, A.lo, A.ld, m, n, part, flags); break;
    }
    QB_LAUNCHED();
    k_sum_parts<<<1, 256, 0, st>>>(part, int(g), 0, out, 1);
    QB_LAUNCHED();
}

void vec_norm2(cudaStream_t st, const void* v, bool f64, int64_t count, double* part,
               double* out, int* flags) {
    const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(cdiv(count, 256), NPART)));
    if (f64) k_vec_norm2<true><<<g, 256, 0, st>>>(v, count, part, flags);
    else k_vec_norm2<false><<<g, 256, 0, st>>>(v, count, part, flags);
    QB_LAUNCHED();
    k_sum_parts<<<1, 256, 0, st>>>(part, int(g), 0, out, 1);
    QB_LAUNCHED();
}

void quantize_bf16x2(cudaStream_t st, const double* src, int64_t m, int64_t n, int64_t lds,
                     bf16* hi, bf16* lo, int64_t ld, double* part, double* out3) {
    const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(m, NPART)));
    k_quant<<<g, 256, 0, st>>>(src, lds, m, n, hi, lo, ld, part);
    QB_LAUNCHED();
    k_sum_parts<<<1, 256, 0, st>>>(part, int(g), NPART, out3, 3);
    QB_LAUNCHED();
}

}  // namespace qb

// ============================================================================ small dense helpers
namespace qb {
namespace {
template <class T>
__global__ void k_transpose(const T* __restrict__ X, int64_t ldx, int64_t rows, int64_t cols,
                            T* __restrict__ Y, int64_t ldy) {
    __shared__ T tile[32][33];
    const int64_t r0 = int64_t(blockIdx.x) * 32, c0 = int64_t(blockIdx.y) * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + threadIdx.x, c = c0 + k;
        if (r < rows && c < cols) tile[k][threadIdx.x] = X[r + c * ldx];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + threadIdx.x, r = r0 + k;
        if (r < rows && c < cols) Y[c + r * ldy] = tile[threadIdx.x][k];
    }
}

// Row-major bf16 packing of a float32 column-major block X (rows x cols, ldx): hi[r, off + c] =
// bf16(X(r, c)) and lo[r, off + c] = bf16(X(r, c) - hi) (round to nearest even both times; either
// output may be null); a 32 x 32 tile through shared memory keeps both sides coalesced.
__global__ void k_pack_rows_bf16(const float* __restrict__ X, int64_t ldx, int64_t rows,
                                 int64_t cols, bf16* __restrict__ hi, bf16* __restrict__ lo,
                                 int64_t ldo, int64_t off) {
    __shared__ float tile[32][33];
    const int64_t r0 = int64_t(blockIdx.x) * 32, c0 = int64_t(blockIdx.y) * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + threadIdx.x, c = c0 + k;
        if (r < rows && c < cols) tile[k][threadIdx.x] = X[r + c * ldx];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + threadIdx.x, r = r0 + k;
        if (r < rows && c < cols) {
            const float v = tile[threadIdx.x][k];
            const bf16 h = __float2bfloat16_rn(v);
            if (hi) hi[r * ldo + off + c] = h;
            if (lo) lo[r * ldo + off + c] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// C = tril(M) + tril(M, -1)^T, k x k column-major (ld k)
template <class T>
__global__ void k_copyltu(const T* __restrict__ M, int64_t k, T* __restrict__ C) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= k * k) return;
    const int64_t i = idx % k, j = idx / k;
    C[i + j * k] = i >= j ? M[i + j * k] : M[j + i * k];
}

// Y[i + j ldy] = (T) X[i + j ldx] from float64
template <class T>
__global__ void k_from_f64(const double* __restrict__ X, int64_t ldx, int64_t rows, int64_t cols,
                           T* __restrict__ Y, int64_t ldy) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx % rows, j = idx / rows;
    Y[i + j * ldy] = T(X[i + j * ldx]);
}

template <class T>
__global__ void k_axpy(int64_t rows, int64_t cols, T alpha, const T* __restrict__ X, int64_t ldx,
                       T* __restrict__ Y, int64_t ldy) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t i = idx % rows, j = idx / rows;
    Y[i + j * ldy] += alpha * X[i + j * ldx];
}

// Inverse of an upper-triangular k x k R (column-major, ld), one column of X per thread, R read
// through the cache; any k.  Used only where k_tri_inv_cols' running sums do not fit in shared
// memory.
template <class T>
__global__ void k_tri_inv_big(const T* __restrict__ R, int64_t ldr, int64_t k, T* __restrict__ X,
                              int64_t ldx) {
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= k) return;
    for (int64_t i = c + 1; i < k; ++i) X[i + c * ldx] = T(0);
    X[c + c * ldx] = T(1) / R[c + c * ldr];
    for (int64_t i = c - 1; i >= 0; --i) {
        T s = T(0);
        for (int64_t l = i + 1; l <= c; ++l) s = fma(R[i + l * ldr], X[l + c * ldx], s);
        X[i + c * ldx] = -s / R[i + i * ldr];
    }
}

// Column c of X = R^-1 (R upper triangular, column-major) by one CTA: back substitution by
// columns of R.  With s = e_c, for l = c, c - 1, ..., 0: x_l = s_l / R[l][l], then
// s_i -= R[i][l] x_l for every i < l.  Row i's running sum lives in shared memory and is only
// ever touched by thread i mod blockDim, so the one cross-thread value of a step is x_l
// (double-buffered, one barrier per step); the reads of column l of R are coalesced.  Computed
// in TC; R is read as TI and X written as TO.
constexpr int64_t TRI_COLS_SMEM = 48 * 1024;
template <class TI, class TO, class TC>
__global__ void k_tri_inv_cols(const TI* __restrict__ R, int64_t ldr, int64_t k,
                               TO* __restrict__ X, int64_t ldx) {
    extern __shared__ __align__(16) unsigned char tri_smem[];
    TC* s = reinterpret_cast<TC*>(tri_smem);
    __shared__ TC xs[2];
    const int64_t c = blockIdx.x;
    const int t = threadIdx.x, nt = blockDim.x;
    for (int64_t i = t; i <= c; i += nt) s[i] = i == c ? TC(1) : TC(0);
    for (int64_t i = c + 1 + t; i < k; i += nt) X[i + c * ldx] = TO(0);
    for (int64_t l = c; l >= 0; --l) {
        if (t == int(l % nt)) {            // the owner of row l: s_l is final
            const TC x = s[l] / TC(R[l + l * ldr]);
            xs[l & 1] = x;
            X[l + c * ldx] = TO(x);
        }
        __syncthreads();
        const TC x = xs[l & 1];
        const TI* Rl = R + l * ldr;
        for (int64_t i = t; i < l; i += nt) s[i] = fma(-TC(Rl[i]), x, s[i]);
    }
}

// Columns TRI_WARPS * blockIdx.x + warp of X = R^-1, one warp per column, for k small enough that
// the upper triangle of R fits in shared memory: it is staged packed (column l at l (l + 1) / 2,
// rows 0..l; eight loads in flight per thread) with the reciprocals of the diagonal beside it,
// and lane j keeps the running sums of rows j, j + 32, ... in registers.  Step l
// (l = c, ..., 0): every lane takes s_l from its owner by a shuffle and forms
// x_l = s_l * (1 / R[l][l]) itself, then updates its rows i < l; after the staging there is no
// block barrier.
constexpr int TRI_WARPS = 8;
constexpr int TRI_RPL = 10;                  // rows per lane: k <= 320
constexpr int TRI_STAGE_UNROLL = 8;
constexpr int64_t TRI_WARP_SMEM = 208 * 1024;
template <class TI, class TO, class TC>
__global__ void __launch_bounds__(TRI_WARPS * 32)
k_tri_inv_warp(const TI* __restrict__ R, int64_t ldr, int k, TO* __restrict__ X, int64_t ldx) {
    extern __shared__ __align__(16) unsigned char tri_smem[];
    TC* rdiag = reinterpret_cast<TC*>(tri_smem);   // k reciprocals of the diagonal
    TC* Rs = rdiag + k;                            // packed upper triangle
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int last = min(k - 1, int(blockIdx.x + 1) * TRI_WARPS - 1);
    const int T = (last + 1) * (last + 2) / 2;
    const int nt = blockDim.x;
    for (int e0 = threadIdx.x; e0 < T; e0 += TRI_STAGE_UNROLL * nt) {
        TI v[TRI_STAGE_UNROLL];
#pragma unroll
        for (int u = 0; u < TRI_STAGE_UNROLL; ++u) {
            const int e = e0 + u * nt;
            if (e < T) {
                int l = int((sqrtf(8.f * float(e) + 1.f) - 1.f) * 0.5f);
                while (l > 0 && l * (l + 1) / 2 > e) --l;
                while ((l + 1) * (l + 2) / 2 <= e) ++l;
                v[u] = R[(e - l * (l + 1) / 2) + int64_t(l) * ldr];
            }
        }
#pragma unroll
        for (int u = 0; u < TRI_STAGE_UNROLL; ++u) {
            const int e = e0 + u * nt;
            if (e < T) Rs[e] = TC(v[u]);
        }
    }
    for (int l = threadIdx.x; l <= last; l += nt) rdiag[l] = TC(1) / TC(R[l + int64_t(l) * ldr]);
    __syncthreads();
    const int c = int(blockIdx.x) * TRI_WARPS + warp;
    if (c >= k) return;   // the whole warp
    TC s[TRI_RPL];
#pragma unroll
    for (int j = 0; j < TRI_RPL; ++j) s[j] = lane + 32 * j == c ? TC(1) : TC(0);
    for (int i = c + 1 + lane; i < k; i += 32) X[i + int64_t(c) * ldx] = TO(0);
    for (int l = c; l >= 0; --l) {
        const TC* col = Rs + l * (l + 1) / 2;
        const int jl = l >> 5;
        TC sl = TC(0);
#pragma unroll
        for (int j = 0; j < TRI_RPL; ++j)
            if (j == jl) sl = s[j];
        sl = __shfl_sync(0xffffffffu, sl, l & 31);
        const TC x = sl * rdiag[l];
        if (lane == (l & 31)) X[l + int64_t(c) * ldx] = TO(x);
#pragma unroll
        for (int j = 0; j < TRI_RPL; ++j)
            if (lane + 32 * j < l) s[j] = fma(-col[lane + 32 * j], x, s[j]);
    }
}

template <class TC>
bool tri_warp_fits(int64_t k) {
    return k <= 32 * TRI_RPL && (k * (k + 1) / 2 + k) * int64_t(sizeof(TC)) <= TRI_WARP_SMEM;
}

template <class TI, class TO, class TC>
void launch_tri_inv_warp(cudaStream_t st, const TI* R, int64_t ldr, int64_t k, TO* X, int64_t ldx) {
    smem_limit_once<k_tri_inv_warp<TI, TO, TC>>(size_t(TRI_WARP_SMEM));
    const size_t sm = size_t(k * (k + 1) / 2 + k) * sizeof(TC);
    k_tri_inv_warp<TI, TO, TC><<<unsigned(cdiv(k, TRI_WARPS)), TRI_WARPS * 32, sm, st>>>(
        R, ldr, int(k), X, ldx);
}

template <class TI, class TO, class TC>
void launch_tri_inv(cudaStream_t st, const TI* R, int64_t ldr, int64_t k, TO* X, int64_t ldx) {
    const int nt = k <= 64 ? 64 : (k <= 128 ? 128 : 256);
    k_tri_inv_cols<TI, TO, TC><<<unsigned(k), nt, size_t(k) * sizeof(TC), st>>>(R, ldr, k, X, ldx);
}
}  // namespace

void transpose(cudaStream_t st, bool f64, const void* X, int64_t ldx, int64_t rows, int64_t cols,
               void* Y, int64_t ldy) {
    if (rows <= 0 || cols <= 0) return;
    dim3 g(unsigned(cdiv(rows, 32)), unsigned(cdiv(cols, 32))), b(32, 8);
    if (f64) k_transpose<double><<<g, b, 0, st>>>(reinterpret_cast<const double*>(X), ldx, rows, cols, reinterpret_cast<double*>(Y), ldy);
    else k_transpose<float><<<g, b, 0, st>>>(reinterpret_cast<const float*>(X), ldx, rows, cols, reinterpret_cast<float*>(Y), ldy);
    QB_LAUNCHED();
}

void pack_rows_bf16(cudaStream_t st, const float* X, int64_t ldx, int64_t rows, int64_t cols,
                    bf16* hi, bf16* lo, int64_t ldo, int64_t off) {
    if (rows <= 0 || cols <= 0) return;
    dim3 g(unsigned(cdiv(rows, 32)), unsigned(cdiv(cols, 32))), b(32, 8);
    k_pack_rows_bf16<<<g, b, 0, st>>>(X, ldx, rows, cols, hi, lo, ldo, off);
    QB_LAUNCHED();
}

void copyltu(cudaStream_t st, bool f64, const void* M, int64_t k, void* C) {
    if (k <= 0) return;
    const unsigned g = unsigned(cdiv(k * k, 256));
    if (f64) k_copyltu<double><<<g, 256, 0, st>>>(reinterpret_cast<const double*>(M), k, reinterpret_cast<double*>(C));
    else k_copyltu<float><<<g, 256, 0, st>>>(reinterpret_cast<const float*>(M), k, reinterpret_cast<float*>(C));
    QB_LAUNCHED();
}

void from_f64(cudaStream_t st, bool f64, const double* X, int64_t ldx, int64_t rows, int64_t cols,
              void* Y, int64_t ldy) {
    if (rows <= 0 || cols <= 0) return;
    const unsigned g = unsigned(cdiv(rows * cols, 256));
    if (f64) k_from_f64<double><<<g, 256, 0, st>>>(X, ldx, rows, cols, reinterpret_cast<double*>(Y), ldy);
    else k_from_f64<float><<<g, 256, 0, st>>>(X, ldx, rows, cols, reinterpret_cast<float*>(Y), ldy);
    QB_LAUNCHED();
}

void axpy(cudaStream_t st, bool f64, int64_t rows, int64_t cols, double alpha, const void* X,
          int64_t ldx, void* Y, int64_t ldy) {
    if (rows <= 0 || cols <= 0) return;
    const unsigned g = unsigned(cdiv(rows * cols, 256));
    if (f64) k_axpy<double><<<g, 256, 0, st>>>(rows, cols, alpha, reinterpret_cast<const double*>(X), ldx, reinterpret_cast<double*>(Y), ldy);
    else k_axpy<float><<<g, 256, 0, st>>>(rows, cols, float(alpha), reinterpret_cast<const float*>(X), ldx, reinterpret_cast<float*>(Y), ldy);
    QB_LAUNCHED();
}

void tri_inv_big(cudaStream_t st, bool f64, const void* R, int64_t ldr, int64_t k, void* X,
                 int64_t ldx) {
    if (k <= 0) return;
    if (f64 ? tri_warp_fits<double>(k) : tri_warp_fits<float>(k)) {
        if (f64)
            launch_tri_inv_warp<double, double, double>(st, reinterpret_cast<const double*>(R), ldr,
                                                        k, reinterpret_cast<double*>(X), ldx);
        else
            launch_tri_inv_warp<float, float, float>(st, reinterpret_cast<const float*>(R), ldr, k,
                                                     reinterpret_cast<float*>(X), ldx);
    } else if (k * int64_t(f64 ? sizeof(double) : sizeof(float)) <= TRI_COLS_SMEM) {
        if (f64)
            launch_tri_inv<double, double, double>(st, reinterpret_cast<const double*>(R), ldr, k,
                                                   reinterpret_cast<double*>(X), ldx);
        else
            launch_tri_inv<float, float, float>(st, reinterpret_cast<const float*>(R), ldr, k,
                                                reinterpret_cast<float*>(X), ldx);
    } else {
        const unsigned g = unsigned(cdiv(k, 64));
        if (f64) k_tri_inv_big<double><<<g, 64, 0, st>>>(reinterpret_cast<const double*>(R), ldr, k, reinterpret_cast<double*>(X), ldx);
        else k_tri_inv_big<float><<<g, 64, 0, st>>>(reinterpret_cast<const float*>(R), ldr, k, reinterpret_cast<float*>(X), ldx);
    }
    QB_LAUNCHED();
}

void tri_inv_from_f64(cudaStream_t st, bool f64, const double* R, int64_t ldr, int64_t k, void* X,
                      int64_t ldx) {
    if (k <= 0) return;
    if (!tri_warp_fits<double>(k)) throw Error{QB_ERR_INVALID_ARG, "triangular inverse too large"};
    if (f64)
        launch_tri_inv_warp<double, double, double>(st, R, ldr, k, reinterpret_cast<double*>(X), ldx);
    else
        launch_tri_inv_warp<double, float, float>(st, R, ldr, k, reinterpret_cast<float*>(X), ldx);
    QB_LAUNCHED();
}
}  // namespace qb
