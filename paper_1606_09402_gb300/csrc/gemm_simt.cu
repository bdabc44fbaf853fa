// SIMT tiled GEMM for the tall-skinny products of the QB loop and for the float64 path.
//
// C (M x N, column-major) = alpha * op(X) * Y + beta * C
//   TN: op(X) = X^T, X column-major K x M  -> both operands contiguous along K
//   NN: op(X) = X,   X column-major M x K  -> X contiguous along M, Y along K
// Every product of Algorithms 2-4 is one of the two forms once dense row-major A is viewed as a
// column-major n x m matrix (A Omega is TN, A^T V is NN) and B (row-major k x n) as a
// column-major n x k matrix (B Omega_i is TN, B^T C is NN).
//
// 128 x 64 output tile per 256-thread block, 8 x 4 outputs per thread, K step 16.  Long K is split
// across blockIdx.z; split partials go to scratch and are summed in a fixed order (deterministic).
#include "qb_internal.cuh"

namespace qb {
namespace {


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
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ double get() const { return v; }
};
struct AccFv {
    using V = float;
    using P = float;
    float v;
    __device__ __forceinline__ void init() { v = 0.f; }
    __device__ __forceinline__ void add(float a, float b) { v = fmaf(a, b, v); }
    __device__ __forceinline__ void flush() {}
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
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ double get() const { return double(hi) + double(lo); }
};
// Two levels: float32 FMAs over one shared-memory stage (16 k-steps), then the stage sum is added
// to a float32 pair with Knuth's two-sum.  The error is a few float32 roundings of the terms
// instead of growing with the reduction length, at about 1.4 instructions per FMA (the pair above
// costs 9).  For products of float32 data whose own representation error is one rounding.
struct AccF2v {
    using V = float;
    using P = double;
    float v, hi, lo;
    __device__ __forceinline__ void init() { v = 0.f; hi = 0.f; lo = 0.f; }
    __device__ __forceinline__ void add(float a, float b) { v = fmaf(a, b, v); }
    __device__ __forceinline__ void flush() {
        const float s = hi + v;
        const float bb = s - hi;
        lo += (hi - (s - bb)) + (v - bb);
        hi = s;
        v = 0.f;
    }
    __device__ __forceinline__ double get() const { return double(hi) + double(lo) + double(v); }
};

// 128 x 64 output tile, 8 x 4 outputs per thread (rows tx*4.. and 64+tx*4.., columns ty*4..),
// k step 16, double-buffered shared memory; operands converted to the accumulator's value type V
// on load.
constexpr int GM = 128, GN = 64, GK = 16, GPAD = 4;

template <class V> struct Vec4;
template <> struct Vec4<float> {
    __device__ __forceinline__ static void load(const float* p, float (&o)[4]) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <> struct Vec4<double> {
    __device__ __forceinline__ static void load(const double* p, double (&o)[4]) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
};

template <class LX, class LY, class A, bool XT, class TC>
__global__ void __launch_bounds__(256)
k_gemm2(int64_t M, int64_t N, int64_t K, int64_t kchunk, LX X, int64_t ldx, LY Y, int64_t ldy,
        TC* __restrict__ C, int64_t ldc, double alpha, double beta, typename A::P* __restrict__ part) {
    using V = typename A::V;
    // k step: 16 for float operands, 8 for double (static shared memory stays below 48 KB)
    constexpr int KS = sizeof(V) == 8 ? 8 : GK;
    constexpr int NXQ = GM * KS / 256, NYQ = GN * KS / 256;
    __shared__ __align__(16) V Xs[2][KS][GM + GPAD];
    __shared__ __align__(16) V Ys[2][KS][GN + GPAD];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = int64_t(blockIdx.x) * GM, n0 = int64_t(blockIdx.y) * GN;
    const int64_t kb = int64_t(blockIdx.z) * kchunk;
    const int64_t ke = min(K, kb + kchunk);
    A acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c].init();
    V rx[NXQ], ry[NYQ];
    auto gload = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < NXQ; ++q) {
            const int e = tid + 256 * q;
            int i, kk;
            if (XT) { kk = e % KS; i = e / KS; } else { i = e % GM; kk = e / GM; }
            const int64_t gi = m0 + i, gk = k0 + kk;
            rx[q] = (gi < M && gk < ke) ? X(XT ? gk + gi * ldx : gi + gk * ldx) : V(0);
        }
#pragma unroll
        for (int q = 0; q < NYQ; ++q) {
            const int e = tid + 256 * q, kk = e % KS, j = e / KS;
            const int64_t gj = n0 + j, gk = k0 + kk;
            ry[q] = (gj < N && gk < ke) ? Y(gk + gj * ldy) : V(0);
        }
    };
    auto sstore = [&](int b) {
#pragma unroll
        for (int q = 0; q < NXQ; ++q) {
            const int e = tid + 256 * q;
            if (XT) Xs[b][e % KS][e / KS] = rx[q];
            else Xs[b][e / GM][e % GM] = rx[q];
        }
#pragma unroll
        for (int q = 0; q < NYQ; ++q) {
            const int e = tid + 256 * q;
            Ys[b][e % KS][e / KS] = ry[q];
        }
    };
    int buf = 0;
    if (kb < ke) {
        gload(kb);
        sstore(0);
    }
    __syncthreads();
    for (int64_t k0 = kb; k0 < ke; k0 += KS) {
        const bool more = k0 + KS < ke;
        if (more) gload(k0 + KS);
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) {
            V a[8], bv[4];
            V t0[4], t1[4];
            Vec4<V>::load(&Xs[buf][kk][tx * 4], t0);
            Vec4<V>::load(&Xs[buf][kk][64 + tx * 4], t1);
            Vec4<V>::load(&Ys[buf][kk][ty * 4], bv);
#pragma unroll
            for (int r = 0; r < 4; ++r) { a[r] = t0[r]; a[4 + r] = t1[r]; }
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c].add(a[r], bv[c]);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c].flush();
        if (more) sstore(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t gi = m0 + (r < 4 ? tx * 4 + r : 64 + tx * 4 + (r - 4));
        if (gi >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t gj = n0 + ty * 4 + c;
            if (gj >= N) continue;
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
    const int64_t tiles = cdiv(M, GM) * cdiv(N, GN);
    const int64_t target = 2LL * num_sms();
    int64_t splits = 1;
    if (K > 0 && tiles < target) {
        splits = std::min<int64_t>(cdiv(target, tiles), cdiv(K, 512));
        splits = std::max<int64_t>(1, std::min<int64_t>(splits, MAX_SPLITS));
        while (splits > 1 && size_t(splits) * M * N * sizeof(typename A::P) > scr.part_bytes) --splits;
    }
    const int64_t kchunk = splits > 1 ? align_up(cdiv(K, splits), GK) : std::max<int64_t>(K, 1);
    splits = K > 0 ? cdiv(K, kchunk) : 1;
    dim3 grid(unsigned(cdiv(M, GM)), unsigned(cdiv(N, GN)), unsigned(splits));
    if (cdiv(N, GN) > 65535) throw Error{QB_ERR_INVALID_ARG, "gemm: N too large"};
    typename A::P* part = splits > 1 ? reinterpret_cast<typename A::P*>(scr.part) : nullptr;
    if (xt)
        k_gemm2<LX, LY, A, true, TC><<<grid, 256, 0, st>>>(M, N, K, kchunk, X, ldx, Y, ldy, C, ldc,
                                                            alpha, beta, part);
    else
        k_gemm2<LX, LY, A, false, TC><<<grid, 256, 0, st>>>(M, N, K, kchunk, X, ldx, Y, ldy, C,
                                                             ldc, alpha, beta, part);
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

// ---------------------------------------------------------------- precise A^T V pass
// Z (n x w, column-major) = (A_hi + A_lo)^T V, A row-major m x n as two bf16 arrays (A_lo may be
// null: a plain bf16 A), V float32 column-major m x w.  Float32 FMA with exact operands (A_hi + A_lo and V are float32 values):
// every product and partial sum is rounded to nearest, so the result carries no systematic drift
// (the pass that forms B_i = Q_i^T A and H = A^T G feeds the indicator of Theorem 1).
// 128 x 64 output tile, 8 x 4 per thread, k step 16, double-buffered shared memory.
constexpr int TM_ = 128, TN_ = 64, TK_ = 16;

__global__ void __launch_bounds__(256)
k_trans_prec(int64_t m, int64_t n, int64_t w, int64_t kchunk, const bf16* __restrict__ Ahi,
             const bf16* __restrict__ Alo, int64_t lda, const float* __restrict__ V, int64_t ldv,
             float* __restrict__ Z, int64_t ldz, float* __restrict__ part) {
    __shared__ __align__(16) float As[2][TK_][TM_];
    __shared__ __align__(16) float Vs[2][TK_][TN_];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t n0 = int64_t(blockIdx.x) * TM_, w0 = int64_t(blockIdx.y) * TN_;
    const int64_t kb = int64_t(blockIdx.z) * kchunk, ke = min(m, kb + kchunk);
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    float ra[8], rv[4];
    auto gload = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + 256 * q, r = e / TM_, c = e % TM_;
            const int64_t gk = k0 + r, gn = n0 + c;
            float v = 0.f;
            if (gk < ke && gn < n) {
                const int64_t o = gk * lda + gn;
                v = __bfloat162float(Ahi[o]);
                if (Alo) v += __bfloat162float(Alo[o]);
            }
            ra[q] = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q, r = e % TK_, c = e / TK_;
            const int64_t gk = k0 + r, gw = w0 + c;
            rv[q] = (gk < ke && gw < w) ? V[gk + gw * ldv] : 0.f;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = tid + 256 * q;
            As[buf][e / TM_][e % TM_] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            Vs[buf][e % TK_][e / TK_] = rv[q];
        }
    };
    int buf = 0;
    if (kb < ke) {
        gload(kb);
        sstore(0);
    }
    __syncthreads();
    for (int64_t k0 = kb; k0 < ke; k0 += TK_) {
        const bool more = k0 + TK_ < ke;
        if (more) gload(k0 + TK_);
#pragma unroll
        for (int kk = 0; kk < TK_; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tx * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tx * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Vs[buf][kk][ty * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) sstore(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gn = n0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
        if (gn >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gw = w0 + ty * 4 + j;
            if (gw >= w) continue;
            if (part) part[(int64_t(blockIdx.z) * w + gw) * n + gn] = acc[i][j];
            else Z[gn + gw * ldz] = acc[i][j];
        }
    }
}

// ---------------------------------------------------------------- panel Gram
// W = P^T P for a rows x bi panel (bi <= MAXB).  Rows are split evenly across CTAs; thread t < 136
// owns the t-th 4 x 4 block of the upper triangle of the 16 x 16 block grid (row-major order), so
// the upper triangle is formed once.  CTA partials go to scratch and k_gram_reduce sums them in
// CTA order (deterministic) into the symmetric W.
constexpr int GRAM_THREADS = 160, GRAM_BLOCKS = 136, GRAM_ROWS = 32, GRAM_LD = MAXB + 4;

template <class A, class T>
__global__ void __launch_bounds__(GRAM_THREADS)
k_gram(const T* __restrict__ P, int64_t ldp, int64_t rows, int bi, int64_t rows_per,
       typename A::P* __restrict__ part) {
    using V = typename A::V;
    __shared__ __align__(16) V Ps[GRAM_ROWS][GRAM_LD];
    const int tid = threadIdx.x;
    const bool active = tid < GRAM_BLOCKS;
    int gi = 0, gj = 0;
    {
        int t = active ? tid : 0;
        while (t >= 16 - gi) { t -= 16 - gi; ++gi; }
        gj = gi + t;
    }
    const int64_t r_beg = int64_t(blockIdx.x) * rows_per;
    const int64_t r_end = min(rows, r_beg + rows_per);
    A acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b].init();
    for (int64_t r0 = r_beg; r0 < r_end; r0 += GRAM_ROWS) {
        __syncthreads();
        for (int e = tid; e < GRAM_ROWS * MAXB; e += GRAM_THREADS) {
            const int rr = e % GRAM_ROWS, c = e / GRAM_ROWS;
            const int64_t gr = r0 + rr;
            Ps[rr][c] = (gr < r_end && c < bi) ? V(P[gr + int64_t(c) * ldp]) : V(0);
        }
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int rr = 0; rr < GRAM_ROWS; ++rr) {
                V x[4], y[4];
                Vec4<V>::load(&Ps[rr][gi * 4], x);
                Vec4<V>::load(&Ps[rr][gj * 4], y);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b].add(x[a], y[b]);
            }
        }
    }
    if (!active) return;
    typename A::P* out = part + int64_t(blockIdx.x) * MAXB * MAXB;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) out[(gi * 4 + a) + (gj * 4 + b) * MAXB] = acc[a][b].get();
}

// One CTA per 32 Gram entries: warp w sums the partials w, w + 8, ... of its 32 entries (lane =
// entry, coalesced), then the 8 warp sums are added in warp order (deterministic).
template <class P>
__global__ void __launch_bounds__(256) k_gram_reduce(const P* __restrict__ part, int G, int bi,
                                                     double* __restrict__ W) {
    __shared__ double sh[8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * 32 + lane;
    const int i = e % MAXB, j = e / MAXB;
    const bool need = i <= j && j < bi;
    double s = 0.0;
    if (need)
        for (int c = warp; c < G; c += 8) s += double(part[int64_t(c) * MAXB * MAXB + e]);
    sh[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && i <= j) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += sh[w][lane];
        W[i + j * MAXB] = t;
        W[j + i * MAXB] = t;
    }
}

template <class A, class T>
void launch_gram(cudaStream_t st, const T* P, int64_t ldp, int64_t rows, int bi, double* W,
                 const GemmScratch& scr) {
    using PT = typename A::P;
    const int64_t cap = int64_t(scr.part_bytes / (sizeof(PT) * MAXB * MAXB));
    int64_t G = std::min<int64_t>(std::min<int64_t>(2LL * num_sms(), cdiv(std::max<int64_t>(rows, 1), 64)), cap);
    G = std::max<int64_t>(G, 1);
    const int64_t rows_per = align_up(cdiv(std::max<int64_t>(rows, 1), G), GRAM_ROWS);
    G = cdiv(std::max<int64_t>(rows, 1), rows_per);
    if (cap < 1) throw Error{QB_ERR_WORKSPACE, "gram partials"};
    PT* part = reinterpret_cast<PT*>(scr.part);
    k_gram<A, T><<<unsigned(G), GRAM_THREADS, 0, st>>>(P, ldp, rows, bi, rows_per, part);
    QB_LAUNCHED();
    k_gram_reduce<PT><<<MAXB * MAXB / 32, 256, 0, st>>>(part, int(G), bi, W);
    QB_LAUNCHED();
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
    } else if (acc == ACC_F2) {
        if (c_f64)
            dispatch_x<AccF2v, float>(st, xt, M, N, K, alpha, X, Y, ldy, beta,
                                      reinterpret_cast<double*>(C), ldc, scr);
        else
            dispatch_x<AccF2v, float>(st, xt, M, N, K, alpha, X, Y, ldy, beta,
                                      reinterpret_cast<float*>(C), ldc, scr);
    } else {
        if (c_f64)
            dispatch_x<AccFv, float>(st, xt, M, N, K, alpha, X, Y, ldy, beta,
                                     reinterpret_cast<double*>(C), ldc, scr);
        else
            dispatch_x<AccFv, float>(st, xt, M, N, K, alpha, X, Y, ldy, beta,
                                     reinterpret_cast<float*>(C), ldc, scr);
    }
}

void gram(cudaStream_t st, const void* P, int64_t ldp, int64_t rows, int bi, bool f64, Acc acc,
          double* W, const GemmScratch& scr) {
    if (bi < 1 || bi > MAXB) throw Error{QB_ERR_INVALID_ARG, "gram width"};
    if (f64 || acc == ACC_D) {
        if (!f64) throw Error{QB_ERR_UNSUPPORTED, "ACC_D needs f64 operands"};
        launch_gram<AccDv>(st, reinterpret_cast<const double*>(P), ldp, rows, bi, W, scr);
    } else if (acc == ACC_DF) {
        launch_gram<AccDFv>(st, reinterpret_cast<const float*>(P), ldp, rows, bi, W, scr);
    } else {
        launch_gram<AccFv>(st, reinterpret_cast<const float*>(P), ldp, rows, bi, W, scr);
    }
}

void trans_precise(cudaStream_t st, const bf16* Ahi, const bf16* Alo, int64_t lda, int64_t m,
                   int64_t n, const float* V, int64_t ldv, int64_t w, float* Z, int64_t ldz,
                   const GemmScratch& scr) {
    if (n <= 0 || w <= 0) return;
    const int64_t tiles = cdiv(n, TM_) * cdiv(w, TN_);
    const int64_t target = 2LL * num_sms();
    int64_t splits = 1;
    if (tiles < target && m > 0) {
        splits = std::min<int64_t>(cdiv(target, tiles), cdiv(m, 1024));
        splits = std::max<int64_t>(1, std::min<int64_t>(splits, MAX_SPLITS));
        while (splits > 1 && size_t(splits) * n * w * sizeof(float) > scr.part_bytes) --splits;
    }
    const int64_t kchunk = splits > 1 ? align_up(cdiv(m, splits), TK_) : std::max<int64_t>(m, 1);
    splits = m > 0 ? cdiv(m, kchunk) : 1;
    float* part = splits > 1 ? reinterpret_cast<float*>(scr.part) : nullptr;
    dim3 grid(unsigned(cdiv(n, TM_)), unsigned(cdiv(w, TN_)), unsigned(splits));
    k_trans_prec<<<grid, 256, 0, st>>>(m, n, w, kchunk, Ahi, Alo, lda, V, ldv, Z, ldz, part);
    QB_LAUNCHED();
    if (part) {
        k_splitk_reduce<float, float><<<unsigned(cdiv(n * w, 256)), 256, 0, st>>>(
            n, w, int(splits), part, Z, ldz, 1.0, 0.0);
        QB_LAUNCHED();
    }
}

}  // namespace qb
