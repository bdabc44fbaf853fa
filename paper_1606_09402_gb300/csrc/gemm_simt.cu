// SIMT tiled GEMM for the tall-skinny products of the QB loop and for the float64 path.
//
// C (M x N, column-major) = alpha * op(X) * Y + beta * C
//   TN: op(X) = X^T, X column-major K x M  -> both operands contiguous along K
//   NN: op(X) = X,   X column-major M x K  -> X contiguous along M, Y along K
// Every product of Algorithms 2-4 is one of the two forms once dense row-major A is viewed as a
// column-major n x m matrix (A Omega is TN, A^T V is NN) and B (row-major k x n) as a
// column-major n x k matrix (B Omega_i is TN, B^T C is NN).
//
// 64 x 64 output tile per 256-thread block, 4 x 4 outputs per thread, K step 16.  Long K is split
// across blockIdx.z; split partials go to scratch and are summed in a fixed order (deterministic).
#include "qb_internal.cuh"

namespace qb {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// ---------------------------------------------------------------- loaders (value type V)
template <class V> struct LdF64 {
    const double* p;
    __device__ __forceinline__ V operator()(int64_t i) const { return V(p[i]); }
};
template <class V> struct LdF32 {
    const float* p;
    __device__ __forceinline__ V operator()(int64_t i) const { return V(p[i]); }
};
template <class V> struct LdBF16 {
    const bf16* p;
    __device__ __forceinline__ V operator()(int64_t i) const { return V(__bfloat162float(p[i])); }
};
template <class V> struct LdBF16x2 {
    const bf16* hi;
    const bf16* lo;
    __device__ __forceinline__ V operator()(int64_t i) const {
        return V(__bfloat162float(hi[i])) + V(__bfloat162float(lo[i]));
    }
};

// ---------------------------------------------------------------- accumulators
struct AccDv {
    using V = double;     // operand value type
    using P = double;     // partial / result type
    double v;
    __device__ __forceinline__ void init() { v = 0.0; }
    __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double get() const { return v; }
};
struct AccFv {
    using V = float;
    using P = float;
    float v;
    __device__ __forceinline__ void init() { v = 0.f; }
    __device__ __forceinline__ void add(float a, float b) { v = fmaf(a, b, v); }
    __device__ __forceinline__ float get() const { return v; }
};
// float32 pair: the product a*b is split exactly into p + e with one FMA, p is added to hi with
// Knuth's two-sum and every rounding error is carried in lo.  About 48 significant bits.
struct AccDFv {
    using V = float;
    using P = double;
    float hi, lo;
    __device__ __forceinline__ void init() { hi = 0.f; lo = 0.f; }
    __device__ __forceinline__ void add(float a, float b) {
        float p = a * b;
        float e = fmaf(a, b, -p);
        float s = hi + p;
        float bb = s - hi;
        float err = (hi - (s - bb)) + (p - bb);
        hi = s;
        lo += err + e;
    }
    __device__ __forceinline__ double get() const { return double(hi) + double(lo); }
};

template <class LX, class LY, class A, bool XT, class TC>
__global__ void __launch_bounds__(256)
k_gemm(int64_t M, int64_t N, int64_t K, int64_t kchunk, LX X, int64_t ldx, LY Y, int64_t ldy,
       TC* __restrict__ C, int64_t ldc, double alpha, double beta, typename A::P* __restrict__ part) {
    using V = typename A::V;
    __shared__ V Xs[BK][BM + 1];
    __shared__ V Ys[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = int64_t(blockIdx.x) * BM, n0 = int64_t(blockIdx.y) * BN;
    const int64_t kb = int64_t(blockIdx.z) * kchunk;
    const int64_t ke = min(K, kb + kchunk);
    A acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c].init();

    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int e = tid; e < BM * BK; e += 256) {
            int i, kk;
            if (XT) { kk = e % BK; i = e / BK; } else { i = e % BM; kk = e / BM; }
            const int64_t gi = m0 + i, gk = k0 + kk;
            V v = V(0);
            if (gi < M && gk < ke) v = X(XT ? gk + gi * ldx : gi + gk * ldx);
            Xs[kk][i] = v;
        }
#pragma unroll
        for (int e = tid; e < BN * BK; e += 256) {
            const int kk = e % BK, j = e / BK;
            const int64_t gj = n0 + j, gk = k0 + kk;
            V v = V(0);
            if (gj < N && gk < ke) v = Y(gk + gj * ldy);
            Ys[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            V a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = Xs[kk][tx + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Ys[kk][ty + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c].add(a[r], b[c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t gi = m0 + tx + 16 * r, gj = n0 + ty + 16 * c;
            if (gi >= M || gj >= N) continue;
            if (part) {
                part[(int64_t(blockIdx.z) * N + gj) * M + gi] = typename A::P(acc[r][c].get());
            } else {
                double v = alpha * double(acc[r][c].get());
                if (beta != 0.0) v += beta * double(C[gi + gj * ldc]);
                C[gi + gj * ldc] = TC(v);
            }
        }
    }
}

template <class P, class TC>
__global__ void k_splitk_reduce(int64_t M, int64_t N, int splits, const P* __restrict__ part,
                                TC* __restrict__ C, int64_t ldc, double alpha, double beta) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int64_t i = idx % M, j = idx / M;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += double(part[(int64_t(z) * N + j) * M + i]);
    double v = alpha * s;
    if (beta != 0.0) v += beta * double(C[i + j * ldc]);
    C[i + j * ldc] = TC(v);
}

constexpr int64_t MAX_SPLITS = 64;

template <class A, class LX, class LY, class TC>
void launch(cudaStream_t st, bool xt, int64_t M, int64_t N, int64_t K, double alpha, LX X,
            int64_t ldx, LY Y, int64_t ldy, double beta, TC* C, int64_t ldc,
            const GemmScratch& scr) {
    if (M <= 0 || N <= 0) return;
    const int64_t tiles = cdiv(M, BM) * cdiv(N, BN);
    const int64_t target = 2LL * num_sms();
    int64_t splits = 1;
    if (K > 0 && tiles < target) {
        splits = std::min<int64_t>(cdiv(target, tiles), cdiv(K, 512));
        splits = std::max<int64_t>(1, std::min<int64_t>(splits, MAX_SPLITS));
        while (splits > 1 && size_t(splits) * M * N * sizeof(typename A::P) > scr.part_bytes) --splits;
    }
    const int64_t kchunk = splits > 1 ? align_up(cdiv(K, splits), BK) : std::max<int64_t>(K, 1);
    splits = K > 0 ? cdiv(K, kchunk) : 1;
    dim3 grid(unsigned(cdiv(M, BM)), unsigned(cdiv(N, BN)), unsigned(splits));
    if (cdiv(N, BN) > 65535) throw Error{QB_ERR_INVALID_ARG, "gemm: N too large"};
    typename A::P* part = splits > 1 ? reinterpret_cast<typename A::P*>(scr.part) : nullptr;
    if (xt)
        k_gemm<LX, LY, A, true, TC><<<grid, 256, 0, st>>>(M, N, K, kchunk, X, ldx, Y, ldy, C, ldc,
                                                           alpha, beta, part);
    else
        k_gemm<LX, LY, A, false, TC><<<grid, 256, 0, st>>>(M, N, K, kchunk, X, ldx, Y, ldy, C, ldc,
                                                            alpha, beta, part);
    QB_LAUNCHED();
    if (part) {
        const int64_t tot = M * N;
        k_splitk_reduce<typename A::P, TC><<<unsigned(cdiv(tot, 256)), 256, 0, st>>>(
            M, N, int(splits), part, C, ldc, alpha, beta);
        QB_LAUNCHED();
    }
}

template <class A, class TY, class TC>
void dispatch_x(cudaStream_t st, bool xt, int64_t M, int64_t N, int64_t K, double alpha, XOp X,
                const void* Y, int64_t ldy, double beta, TC* C, int64_t ldc,
                const GemmScratch& scr) {
    using V = typename A::V;
    using LY = typename std::conditional<std::is_same<TY, double>::value, LdF64<V>, LdF32<V>>::type;
    LY ly{reinterpret_cast<const TY*>(Y)};
    switch (X.kind) {
        case X_F64:
            launch<A>(st, xt, M, N, K, alpha, LdF64<V>{reinterpret_cast<const double*>(X.p)}, X.ld,
                      ly, ldy, beta, C, ldc, scr);
            break;
        case X_F32:
            launch<A>(st, xt, M, N, K, alpha, LdF32<V>{reinterpret_cast<const float*>(X.p)}, X.ld,
                      ly, ldy, beta, C, ldc, scr);
            break;
        case X_BF16:
            launch<A>(st, xt, M, N, K, alpha, LdBF16<V>{reinterpret_cast<const bf16*>(X.p)}, X.ld,
                      ly, ldy, beta, C, ldc, scr);
            break;
        case X_BF16X2:
            launch<A>(st, xt, M, N, K, alpha,
                      LdBF16x2<V>{reinterpret_cast<const bf16*>(X.p),
                                  reinterpret_cast<const bf16*>(X.lo)},
                      X.ld, ly, ldy, beta, C, ldc, scr);
            break;
    }
}

}  // namespace

size_t gemm_scratch_bytes(int64_t mn_max) {
    // Split-K is used only while the tile count is below 2 x SMs, so splits x M x N stays below
    // (2 x SMs + tiles) x 64 x 64 elements; 32 MB covers 152 SMs with room to spare.
    const size_t full = size_t(MAX_SPLITS) * size_t(std::max<int64_t>(mn_max, 1)) * sizeof(double);
    return std::min<size_t>(full, size_t(32) << 20);
}

void gemm(cudaStream_t st, bool xt, int64_t M, int64_t N, int64_t K, double alpha, XOp X,
          const void* Y, bool y_f64, int64_t ldy, double beta, void* C, bool c_f64, int64_t ldc,
          Acc acc, const GemmScratch& scr) {
    if (acc == ACC_D) {
        if (!y_f64 || !c_f64) throw Error{QB_ERR_UNSUPPORTED, "ACC_D needs f64 operands"};
        dispatch_x<AccDv, double>(st, xt, M, N, K, alpha, X, Y, ldy, beta,
                                  reinterpret_cast<double*>(C), ldc, scr);
    } else if (y_f64) {
        throw Error{QB_ERR_UNSUPPORTED, "f64 Y needs ACC_D"};
    } else if (acc == ACC_DF) {
        if (c_f64)
            dispatch_x<AccDFv, float>(st, xt, M, N, K, alpha, X, Y, ldy, beta,
                                      reinterpret_cast<double*>(C), ldc, scr);
        else
            dispatch_x<AccDFv, float>(st, xt, M, N, K, alpha, X, Y, ldy, beta,
                                      reinterpret_cast<float*>(C), ldc, scr);
    } else {
        if (c_f64) throw Error{QB_ERR_UNSUPPORTED, "ACC_F writes f32"};
        dispatch_x<AccFv, float>(st, xt, M, N, K, alpha, X, Y, ldy, beta,
                                 reinterpret_cast<float*>(C), ldc, scr);
    }
}

}  // namespace qb
