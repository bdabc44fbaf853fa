// Sparse CSR passes (Sect. 5.1, sparse experiments): Y = A X with one warp per row of A.
//
// The dense operands are column-major in the QB loop; a warp-per-row gather wants the w values of
// one row of X contiguous, so X is transposed into a row-major staging buffer, 128 columns at a
// time (the 128-column slice of X for n = 1e5 is 51 MB and stays in L2), and the row-major result
// is transposed back.  A^T X runs the same kernel on a CSC copy of A built once per call, so no
// atomics touch the Zipf-hot columns.
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

// Y_rm (rows x wc, ld ldy) = A * X_rm (cols x wc, ld ldx), one warp per row, up to 128 columns.
template <class T>
__global__ void __launch_bounds__(256)
k_spmm_rm(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, const T* __restrict__ val,
          int64_t rows, const T* __restrict__ X, int64_t ldx, int wc, T* __restrict__ Y, int64_t ldy) {
    const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    T acc[WCH / 32];
#pragma unroll
    for (int q = 0; q < WCH / 32; ++q) acc[q] = T(0);
    const int32_t b = ptr[r], e = ptr[r + 1];
    for (int32_t p0 = b; p0 < e; p0 += 32) {
        const int32_t p = p0 + lane;
        int32_t c = 0;
        T v = T(0);
        if (p < e) { c = idx[p]; v = val[p]; }
        const int cnt = min(32, e - p0);
        for (int t = 0; t < cnt; ++t) {
            const int32_t cc = __shfl_sync(0xffffffffu, c, t);
            const T vv = __shfl_sync(0xffffffffu, v, t);
            const T* xr = X + int64_t(cc) * ldx;
#pragma unroll
            for (int q = 0; q < WCH / 32; ++q) {
                const int j = lane + 32 * q;
                if (j < wc) acc[q] = fma(vv, xr[j], acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < WCH / 32; ++q) {
        const int j = lane + 32 * q;
        if (j < wc) Y[r * ldy + j] = acc[q];
    }
}

// col-major (rows x cols, ld) slice [c0, c0+wc) -> row-major (rows x wc)
template <class T>
__global__ void k_cm_to_rm(const T* __restrict__ X, int64_t ldx, int64_t rows, int64_t c0, int wc,
                           T* __restrict__ Xr) {
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
        if (r < rows && j < wc) Xr[r * wc + j] = tile[threadIdx.x][k];
    }
}

template <class T>
__global__ void k_rm_to_cm(const T* __restrict__ Yr, int64_t rows, int wc, T* __restrict__ Y,
                           int64_t ldy, int64_t c0) {
    __shared__ T tile[32][33];
    const int64_t r0 = int64_t(blockIdx.x) * 32;
    const int j0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k;
        const int j = j0 + threadIdx.x;
        if (r < rows && j < wc) tile[k][threadIdx.x] = Yr[r * wc + j];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int j = j0 + k;
        const int64_t r = r0 + threadIdx.x;
        if (r < rows && j < wc) Y[r + (c0 + j) * ldy] = tile[threadIdx.x][k];
    }
}

template <class T>
void spmm_t(cudaStream_t st, const int32_t* ptr, const int32_t* idx, const T* val, int64_t rows,
            int64_t cols, const T* X, int64_t ldx, int64_t w, T* Y, int64_t ldy, T* stage) {
    T* Xr = stage;
    T* Yr = stage + cols * WCH;
    for (int64_t c0 = 0; c0 < w; c0 += WCH) {
        const int wc = int(std::min<int64_t>(WCH, w - c0));
        dim3 blk(32, 8);
        k_cm_to_rm<T><<<dim3(unsigned(cdiv(cols, 32)), unsigned(cdiv(wc, 32))), blk, 0, st>>>(
            X, ldx, cols, c0, wc, Xr);
        QB_LAUNCHED();
        k_spmm_rm<T><<<unsigned(cdiv(rows * 32, 256)), 256, 0, st>>>(ptr, idx, val, rows, Xr, wc,
                                                                     wc, Yr, wc);
        QB_LAUNCHED();
        k_rm_to_cm<T><<<dim3(unsigned(cdiv(rows, 32)), unsigned(cdiv(wc, 32))), blk, 0, st>>>(
            Yr, rows, wc, Y, ldy, c0);
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

void csr_spmm(cudaStream_t st, bool f64, const int32_t* ptr, const int32_t* idx, const void* val,
              int64_t rows, int64_t cols, const void* X, int64_t ldx, int64_t w, void* Y,
              int64_t ldy, void* stage) {
    if (rows <= 0 || w <= 0) return;
    if (f64)
        spmm_t<double>(st, ptr, idx, reinterpret_cast<const double*>(val), rows, cols,
                       reinterpret_cast<const double*>(X), ldx, w, reinterpret_cast<double*>(Y),
                       ldy, reinterpret_cast<double*>(stage));
    else
        spmm_t<float>(st, ptr, idx, reinterpret_cast<const float*>(val), rows, cols,
                      reinterpret_cast<const float*>(X), ldx, w, reinterpret_cast<float*>(Y), ldy,
                      reinterpret_cast<float*>(stage));
}

}  // namespace qb
