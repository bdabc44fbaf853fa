// Sparse CSR passes (Sect. 5.1, sparse experiments): Y = A X with one warp per row of A.
//
// The dense operands are column-major in the QB loop; a warp-per-row gather wants the w values of
// one row of X contiguous, so X is transposed into a row-major staging buffer, 128 columns at a
// time (the 128-column slice of X for n = 1e5 is 51 MB and stays in L2), and the row-major result
// is transposed back.  A^T X runs the same kernels on a CSC copy of A built once per call.
//
// Rows longer than CSR_SEG nonzeros (the Zipf-hot columns of A, in the CSC copy: the hottest of
// 1e5 columns holds about an eighth of all nonzeros) would serialise a whole pass behind one warp,
// so a per-call table cuts them into CSR_SEG-nonzero segments, one warp each, whose partial rows
// are added with atomics into the row that the warp-per-row kernel zeroed.  Rows up to CSR_SEG
// nonzeros keep a fixed summation order.
#include "qb_internal.cuh"

namespace qb {
namespace {

constexpr int WCH = 128;   // columns of X per staging slice

__global__ void k_hist(const int32_t* __restrict__ colind, int64_t nnz, int32_t* __restrict__ cnt) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nnz;
         i += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(cnt + colind[i], 1);
}

// Exclusive scan of cnt[0..n) into ptr[0..n], single CTA of 1024 threads; cursor = copy of ptr.
__global__ void __launch_bounds__(1024)
k_scan(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ ptr, int32_t* __restrict__ cursor) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t b = t * chunk, e = min(n, b + chunk);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = t > 0 ? part[t - 1] : 0;
    for (int64_t i = b; i < e; ++i) {
        ptr[i] = int32_t(run);
        cursor[i] = int32_t(run);
        run += cnt[i];
    }
    if (t == 1023) ptr[n] = int32_t(part[1023]);
}

template <class T>
__global__ void k_scatter(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                          const T* __restrict__ val, int64_t m, int32_t* __restrict__ cursor,
                          int32_t* __restrict__ rowind, T* __restrict__ cval) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= m) return;
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; ++p) {
        const int32_t pos = atomicAdd(cursor + colind[p], 1);
        rowind[pos] = int32_t(r);
        cval[pos] = val[p];
    }
}

template <class T, int NQ> struct Vec;
template <> struct Vec<float, 1> {
    static __device__ __forceinline__ void ld(const float* p, float* o) { o[0] = __ldg(p); }
    static __device__ __forceinline__ void st(float* p, const float* v) { p[0] = v[0]; }
};
template <> struct Vec<float, 2> {
    static __device__ __forceinline__ void ld(const float* p, float* o) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void st(float* p, const float* v) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    }
};
template <> struct Vec<float, 4> {
    static __device__ __forceinline__ void ld(const float* p, float* o) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void st(float* p, const float* v) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec<double, 1> {
    static __device__ __forceinline__ void ld(const double* p, double* o) { o[0] = __ldg(p); }
    static __device__ __forceinline__ void st(double* p, const double* v) { p[0] = v[0]; }
};
template <> struct Vec<double, 2> {
    static __device__ __forceinline__ void ld(const double* p, double* o) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void st(double* p, const double* v) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
};
template <> struct Vec<double, 4> {
    static __device__ __forceinline__ void ld(const double* p, double* o) {
        Vec<double, 2>::ld(p, o);
        Vec<double, 2>::ld(p + 2, o + 2);
    }
    static __device__ __forceinline__ void st(double* p, const double* v) {
        Vec<double, 2>::st(p, v);
        Vec<double, 2>::st(p + 2, v + 2);
    }
};

// acc += sum over p in [b, e) of val[p] * X[idx[p], lane*NQ .. lane*NQ+NQ).  The 32 (index, value)
// pairs of a chunk are loaded once by the warp and broadcast; full chunks are unrolled so that
// 32 / NQ row gathers are in flight per warp (32 registers of gathered X per lane).
// Positions are int64 so that p0 + 32 cannot wrap for nnz near INT32_MAX.
template <class T, int NQ>
__device__ __forceinline__ void row_acc(const int32_t* __restrict__ idx, const T* __restrict__ val,
                                        int64_t b, int64_t e, const T* __restrict__ X, int64_t ldx,
                                        int lane, T (&acc)[NQ]) {
    const T* xl = X + lane * NQ;
    for (int64_t p0 = b; p0 < e; p0 += 32) {
        const int64_t p = p0 + lane;
        int32_t c = 0;
        T v = T(0);
        if (p < e) { c = idx[p]; v = val[p]; }
        const int cnt = int(e - p0 < 32 ? e - p0 : 32);
        auto step = [&](int t) {
            const int32_t cc = __shfl_sync(0xffffffffu, c, t);
            const T vv = __shfl_sync(0xffffffffu, v, t);
            T x[NQ];
            Vec<T, NQ>::ld(xl + int64_t(cc) * ldx, x);
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = fma(vv, x[q], acc[q]);
        };
        if (cnt == 32) {
            constexpr int UNR = 32 / NQ;
#pragma unroll UNR
            for (int t = 0; t < 32; ++t) step(t);
        } else {
            for (int t = 0; t < cnt; ++t) step(t);
        }
    }
}

// Y_rm (rows x 32 NQ, ld ldy) = A * X_rm (cols x 32 NQ, ld ldx), one warp per row; lane l owns
// columns [l NQ, l NQ + NQ).  Rows longer than long_len are written as zeros here: their segments
// are added by k_spmm_seg, which runs after this kernel on the same stream.
template <class T, int NQ>
__global__ void __launch_bounds__(256)
k_spmm_rm(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, const T* __restrict__ val,
          int64_t rows, const T* __restrict__ X, int64_t ldx, T* __restrict__ Y, int64_t ldy,
          int32_t long_len) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    T acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = T(0);
    const int32_t b = ptr[r], e = ptr[r + 1];
    if (e - b <= long_len) row_acc<T, NQ>(idx, val, b, e, X, ldx, lane, acc);
    Vec<T, NQ>::st(Y + r * ldy + lane * NQ, acc);
}

// One warp per segment of a long row: the CSR_SEG-nonzero piece [beg, beg + CSR_SEG) of row
// seg_row[s], added into Y with atomics (grid-stride over the *count segments).
template <class T, int NQ>
__global__ void __launch_bounds__(256)
k_spmm_seg(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, const T* __restrict__ val,
           const int32_t* __restrict__ seg_row, const int32_t* __restrict__ seg_beg,
           const int32_t* __restrict__ count, const T* __restrict__ X, int64_t ldx, int wc,
           T* __restrict__ Y, int64_t ldy) {
    const int lane = threadIdx.x & 31;
    const int64_t S = *count;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t s = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < S; s += nw) {
        const int32_t r = seg_row[s];
        const int64_t b = seg_beg[s];
        const int64_t e = b + CSR_SEG < int64_t(ptr[r + 1]) ? b + CSR_SEG : int64_t(ptr[r + 1]);
        T acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = T(0);
        row_acc<T, NQ>(idx, val, b, e, X, ldx, lane, acc);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int j = lane * NQ + q;
            if (j < wc) atomicAdd(Y + int64_t(r) * ldy + j, acc[q]);
        }
    }
}

__global__ void k_seg_count(const int32_t* __restrict__ ptr, int64_t rows, int32_t* __restrict__ cnt) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows;
         r += int64_t(gridDim.x) * blockDim.x) {
        const int32_t len = ptr[r + 1] - ptr[r];
        cnt[r] = len > CSR_SEG ? len / CSR_SEG + (len % CSR_SEG != 0) : 0;
    }
}

__global__ void k_seg_fill(const int32_t* __restrict__ ptr, int64_t rows, const int32_t* __restrict__ off,
                           int32_t* __restrict__ seg_row, int32_t* __restrict__ seg_beg) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < rows;
         r += int64_t(gridDim.x) * blockDim.x) {
        const int32_t b = ptr[r], len = ptr[r + 1] - b;
        if (len <= CSR_SEG) continue;
        const int32_t o = off[r];
        const int32_t nk = len / CSR_SEG + (len % CSR_SEG != 0);   // b + k CSR_SEG < b + len
        for (int32_t k = 0; k < nk; ++k) {
            seg_row[o + k] = int32_t(r);
            seg_beg[o + k] = b + k * CSR_SEG;
        }
    }
}

// col-major (rows x cols, ld) slice [c0, c0+wc) -> row-major (rows x wc, ld wp)
template <class T>
__global__ void k_cm_to_rm(const T* __restrict__ X, int64_t ldx, int64_t rows, int64_t c0, int wc,
                           T* __restrict__ Xr, int wp) {
    __shared__ T tile[32][33];
    const int64_t r0 = int64_t(blockIdx.x) * 32;
    const int j0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int j = j0 + k;
        const int64_t r = r0 + threadIdx.x;
        if (r < rows && j < wc) tile[k][threadIdx.x] = X[r + (c0 + j) * ldx];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k;
        const int j = j0 + threadIdx.x;
        if (r < rows && j < wc) Xr[r * wp + j] = tile[threadIdx.x][k];
    }
}

template <class T>
__global__ void k_rm_to_cm(const T* __restrict__ Yr, int wp, int64_t rows, int wc, T* __restrict__ Y,
                           int64_t ldy, int64_t c0) {
    __shared__ T tile[32][33];
    const int64_t r0 = int64_t(blockIdx.x) * 32;
    const int j0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k;
        const int j = j0 + threadIdx.x;
        if (r < rows && j < wc) tile[k][threadIdx.x] = Yr[r * wp + j];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int j = j0 + k;
        const int64_t r = r0 + threadIdx.x;
        if (r < rows && j < wc) Y[r + (c0 + j) * ldy] = tile[threadIdx.x][k];
    }
}

template <class T, int NQ>
void spmm_slice(cudaStream_t st, const int32_t* ptr, const int32_t* idx, const T* val, int64_t rows,
                const CsrSegs* segs, const T* Xr, int wc, T* Yr) {
    constexpr int wp = 32 * NQ;
    k_spmm_rm<T, NQ><<<unsigned(cdiv(rows * 32, 256)), 256, 0, st>>>(
        ptr, idx, val, rows, Xr, wp, Yr, wp, segs ? int32_t(CSR_SEG) : INT32_MAX);
    QB_LAUNCHED();
    if (segs && segs->cap > 0) {
        const unsigned g = unsigned(std::min<int64_t>(cdiv(segs->cap, 8), 152 * 16));
        k_spmm_seg<T, NQ><<<g, 256, 0, st>>>(ptr, idx, val, segs->row, segs->beg, segs->count, Xr,
                                             wp, wc, Yr, wp);
        QB_LAUNCHED();
    }
}

template <class T>
void spmm_t(cudaStream_t st, const int32_t* ptr, const int32_t* idx, const T* val, int64_t rows,
            int64_t cols, const CsrSegs* segs, const T* X, int64_t ldx, int64_t w, T* Y,
            int64_t ldy, T* stage) {
    T* Xr = stage;
    T* Yr = stage + cols * WCH;
    for (int64_t c0 = 0; c0 < w; c0 += WCH) {
        const int wc = int(std::min<int64_t>(WCH, w - c0));
        const int nq = wc <= 32 ? 1 : wc <= 64 ? 2 : 4;
        const int wp = 32 * nq;
        dim3 blk(32, 8);
        k_cm_to_rm<T><<<dim3(unsigned(cdiv(cols, 32)), unsigned(cdiv(wc, 32))), blk, 0, st>>>(
            X, ldx, cols, c0, wc, Xr, wp);
        QB_LAUNCHED();
        if (nq == 1)
            spmm_slice<T, 1>(st, ptr, idx, val, rows, segs, Xr, wc, Yr);
        else if (nq == 2)
            spmm_slice<T, 2>(st, ptr, idx, val, rows, segs, Xr, wc, Yr);
        else
            spmm_slice<T, 4>(st, ptr, idx, val, rows, segs, Xr, wc, Yr);
        k_rm_to_cm<T><<<dim3(unsigned(cdiv(rows, 32)), unsigned(cdiv(wc, 32))), blk, 0, st>>>(
            Yr, wp, rows, wc, Y, ldy, c0);
        QB_LAUNCHED();
    }
}

// ---------------------------------------------------------------- COO (coordinate) passes
// Y_rm (rows x 32 NQ) += A X_rm for A given as nnz (key, idx, val) triplets: Y(key) += val X(idx).
// Nonzero-balanced: warp w takes the COO_SEG triplets [w COO_SEG, (w + 1) COO_SEG) in storage
// order whatever rows they belong to, sums val X(idx, :) in registers while the key stays the
// same and adds the sum into row `key` of the zeroed Y with atomics when the key changes and at the
// chunk's end.  Correct for any order; with triplets sorted by key most rows lie inside one chunk
// (a single addition into zero, so their sums have a fixed order), and a row spread over two
// chunks gets two additions (commutative, also exact in order); only rows over three or more
// chunks sum in a run-dependent order.
constexpr int COO_SEG = 256;

template <class T, int NQ>
__global__ void __launch_bounds__(256)
k_coo_spmm(const int32_t* __restrict__ key, const int32_t* __restrict__ idx,
           const T* __restrict__ val, int64_t nnz, const T* __restrict__ X, int64_t ldx, int wc,
           T* __restrict__ Y, int64_t ldy) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const T* xl = X + lane * NQ;
    for (int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w * COO_SEG < nnz;
         w += nw) {
        const int64_t b = w * COO_SEG;
        const int64_t e = b + COO_SEG < nnz ? b + COO_SEG : nnz;
        T acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = T(0);
        int32_t cur = -1;
        auto flush = [&]() {
            if (cur < 0) return;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int j = lane * NQ + q;
                if (j < wc) atomicAdd(Y + int64_t(cur) * ldy + j, acc[q]);
                acc[q] = T(0);
            }
        };
        for (int64_t p0 = b; p0 < e; p0 += 32) {
            const int64_t p = p0 + lane;
            int32_t kk = 0, c = 0;
            T v = T(0);
            if (p < e) { kk = key[p]; c = idx[p]; v = val[p]; }
            const int cnt = int(e - p0 < 32 ? e - p0 : 32);
            for (int t = 0; t < cnt; ++t) {
                const int32_t kt = __shfl_sync(0xffffffffu, kk, t);
                const int32_t ct = __shfl_sync(0xffffffffu, c, t);
                const T vt = __shfl_sync(0xffffffffu, v, t);
                if (kt != cur) {
                    flush();
                    cur = kt;
                }
                T x[NQ];
                Vec<T, NQ>::ld(xl + int64_t(ct) * ldx, x);
#pragma unroll
                for (int q = 0; q < NQ; ++q) acc[q] = fma(vt, x[q], acc[q]);
            }
        }
        flush();
    }
}

// Column-sorted copy of COO triplets: position = cursor[col]++ (counting sort by column).
template <class T>
__global__ void k_coo_scatter(const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                              const T* __restrict__ val, int64_t nnz, int32_t* __restrict__ cursor,
                              int32_t* __restrict__ ocol, int32_t* __restrict__ orow,
                              T* __restrict__ oval) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int32_t c = col[e];
        const int32_t pos = atomicAdd(cursor + c, 1);
        ocol[pos] = c;
        orow[pos] = row[e];
        oval[pos] = val[e];
    }
}

template <class T>
void coo_spmm_t(cudaStream_t st, const int32_t* key, const int32_t* idx, const T* val, int64_t nnz,
                int64_t rows, int64_t cols, const T* X, int64_t ldx, int64_t w, T* Y, int64_t ldy,
                T* stage) {
    T* Xr = stage;
    T* Yr = stage + cols * WCH;
    const int64_t chunks = cdiv(std::max<int64_t>(nnz, 1), COO_SEG);
    const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(cdiv(chunks, 8), 1 << 20)));
    for (int64_t c0 = 0; c0 < w; c0 += WCH) {
        const int wc = int(std::min<int64_t>(WCH, w - c0));
        const int nq = wc <= 32 ? 1 : wc <= 64 ? 2 : 4;
        const int wp = 32 * nq;
        dim3 blk(32, 8);
        k_cm_to_rm<T><<<dim3(unsigned(cdiv(cols, 32)), unsigned(cdiv(wc, 32))), blk, 0, st>>>(
            X, ldx, cols, c0, wc, Xr, wp);
        QB_LAUNCHED();
        QB_CUDA(cudaMemsetAsync(Yr, 0, sizeof(T) * size_t(rows) * size_t(wp), st));
        if (nnz > 0) {
            if (nq == 1)
                k_coo_spmm<T, 1><<<g, 256, 0, st>>>(key, idx, val, nnz, Xr, wp, wc, Yr, wp);
            else if (nq == 2)
                k_coo_spmm<T, 2><<<g, 256, 0, st>>>(key, idx, val, nnz, Xr, wp, wc, Yr, wp);
            else
                k_coo_spmm<T, 4><<<g, 256, 0, st>>>(key, idx, val, nnz, Xr, wp, wc, Yr, wp);
            QB_LAUNCHED();
        }
        k_rm_to_cm<T><<<dim3(unsigned(cdiv(rows, 32)), unsigned(cdiv(wc, 32))), blk, 0, st>>>(
            Yr, wp, rows, wc, Y, ldy, c0);
        QB_LAUNCHED();
    }
}

}  // namespace

size_t csr_stage_bytes(int64_t m, int64_t n, bool f64) {
    return size_t(m + n) * WCH * (f64 ? 8 : 4);
}

void csr_to_csc(cudaStream_t st, const CsrDev& A, int32_t* colptr, int32_t* rowind, void* cval,
                int32_t* cnt) {
    QB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * size_t(A.n), st));
    if (A.nnz > 0) {
        k_hist<<<unsigned(std::min<int64_t>(cdiv(A.nnz, 256), 4096)), 256, 0, st>>>(A.colind, A.nnz, cnt);
        QB_LAUNCHED();
    }
    // cursor reuses cnt after the scan has read it: scan writes ptr then cursor, reading cnt
    // first in each thread's chunk, so use a second region for the cursor.
    int32_t* cursor = cnt + A.n;
    k_scan<<<1, 1024, 0, st>>>(cnt, A.n, colptr, cursor);
    QB_LAUNCHED();
    if (A.m > 0) {
        if (A.f64)
            k_scatter<double><<<unsigned(cdiv(A.m, 256)), 256, 0, st>>>(
                A.rowptr, A.colind, reinterpret_cast<const double*>(A.val), A.m, cursor, rowind,
                reinterpret_cast<double*>(cval));
        else
            k_scatter<float><<<unsigned(cdiv(A.m, 256)), 256, 0, st>>>(
                A.rowptr, A.colind, reinterpret_cast<const float*>(A.val), A.m, cursor, rowind,
                reinterpret_cast<float*>(cval));
        QB_LAUNCHED();
    }
}

int64_t csr_seg_cap(int64_t nnz) { return 2 * nnz / CSR_SEG + 1; }

void csr_segments(cudaStream_t st, const int32_t* ptr, int64_t rows, int32_t* off, int32_t* tmp,
                  CsrSegs& segs) {
    segs.count = off + rows;
    if (rows <= 0) {
        QB_CUDA(cudaMemsetAsync(segs.count, 0, sizeof(int32_t), st));
        return;
    }
    const unsigned g = unsigned(std::min<int64_t>(cdiv(rows, 256), 4096));
    k_seg_count<<<g, 256, 0, st>>>(ptr, rows, tmp);
    QB_LAUNCHED();
    k_scan<<<1, 1024, 0, st>>>(tmp, rows, off, tmp + rows);
    QB_LAUNCHED();
    k_seg_fill<<<g, 256, 0, st>>>(ptr, rows, off, segs.row, segs.beg);
    QB_LAUNCHED();
}

void csr_spmm(cudaStream_t st, bool f64, const int32_t* ptr, const int32_t* idx, const void* val,
              int64_t rows, int64_t cols, const CsrSegs* segs, const void* X, int64_t ldx,
              int64_t w, void* Y, int64_t ldy, void* stage) {
    if (rows <= 0 || w <= 0) return;
    if (f64)
        spmm_t<double>(st, ptr, idx, reinterpret_cast<const double*>(val), rows, cols, segs,
                       reinterpret_cast<const double*>(X), ldx, w, reinterpret_cast<double*>(Y),
                       ldy, reinterpret_cast<double*>(stage));
    else
        spmm_t<float>(st, ptr, idx, reinterpret_cast<const float*>(val), rows, cols, segs,
                      reinterpret_cast<const float*>(X), ldx, w, reinterpret_cast<float*>(Y), ldy,
                      reinterpret_cast<float*>(stage));
}

}  // namespace qb

namespace qb {

void coo_by_column(cudaStream_t st, const CooDev& A, int32_t* ocol, int32_t* orow, void* oval,
                   int32_t* colptr, int32_t* cnt) {
    QB_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * size_t(A.n), st));
    const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(cdiv(A.nnz, 256), 4096)));
    if (A.nnz > 0) {
        k_hist<<<g, 256, 0, st>>>(A.col, A.nnz, cnt);
        QB_LAUNCHED();
    }
    int32_t* cursor = cnt + A.n;
    k_scan<<<1, 1024, 0, st>>>(cnt, A.n, colptr, cursor);
    QB_LAUNCHED();
    if (A.nnz > 0) {
        if (A.f64)
            k_coo_scatter<double><<<g, 256, 0, st>>>(A.row, A.col,
                                                    reinterpret_cast<const double*>(A.val), A.nnz,
                                                    cursor, ocol, orow,
                                                    reinterpret_cast<double*>(oval));
        else
            k_coo_scatter<float><<<g, 256, 0, st>>>(A.row, A.col,
                                                   reinterpret_cast<const float*>(A.val), A.nnz,
                                                   cursor, ocol, orow,
                                                   reinterpret_cast<float*>(oval));
        QB_LAUNCHED();
    }
}

void coo_spmm(cudaStream_t st, bool f64, const int32_t* key, const int32_t* idx, const void* val,
              int64_t nnz, int64_t rows, int64_t cols, const void* X, int64_t ldx, int64_t w,
              void* Y, int64_t ldy, void* stage) {
    if (rows <= 0 || w <= 0) return;
    if (f64)
        coo_spmm_t<double>(st, key, idx, reinterpret_cast<const double*>(val), nnz, rows, cols,
                           reinterpret_cast<const double*>(X), ldx, w,
                           reinterpret_cast<double*>(Y), ldy, reinterpret_cast<double*>(stage));
    else
        coo_spmm_t<float>(st, key, idx, reinterpret_cast<const float*>(val), nnz, rows, cols,
                          reinterpret_cast<const float*>(X), ldx, w, reinterpret_cast<float*>(Y),
                          ldy, reinterpret_cast<float*>(stage));
}

}  // namespace qb
