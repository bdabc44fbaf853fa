// SVD from a QB factorisation (Sect. 2): with B = U~ S V~^T, A ~ Q B = (Q U~) S V~^T, so the
// first columns of Q U~ and V~ and the leading entries of S approximate A's singular triplets.
//
// B is k x n with k small (the rank), so its SVD goes through the k x k Gram W = B B^T:
//   W = U~ diag(lambda) U~^T (symmetric eigendecomposition), S = sqrt(lambda), V~ = B^T U~ S^-1.
// The eigendecomposition is the cyclic Jacobi method in float64: in each step a round-robin
// tournament pairs all indices, every pair (p, q) gets the plane rotation that zeroes W(p, q)
// (Golub & Van Loan, symmetric Schur 2x2), and W <- J^T W J, V <- V J for the product J of the
// step's rotations (disjoint planes, so they commute).  One cooperative launch runs all sweeps:
// every CTA derives all rotations of a step from W itself (the same arithmetic in every CTA, so
// no exchange is needed), applies its share of the 2 x 2 blocks of W and of the rows of V, and
// the grid meets once per step at a barrier whose wait is bounded.  The sweeps stop when a whole
// sweep applies no rotation (every |W(p, q)| <= 1e-15 sqrt(W(p, p) W(q, q))).
//
// Singular values carry the Gram's squaring: sigma_j is accurate to about u (sigma_1 / sigma_j)^2
// relative, which is ample for the leading triplets the QB approximation is used for.
#include "qb_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace qb {
namespace {

constexpr int JAC_THREADS = 512;
constexpr int SVD_MAX_K = 4096;
constexpr int JAC_MAX_SWEEPS = 40;
constexpr uint64_t JAC_WAIT_NS = 2000000000ull;   // bounded grid-barrier waits: 2 s
constexpr double JAC_TOL = 1e-15;

struct JacArgs {
    double* W;        // k x k, column-major, ld k (symmetric, both triangles kept)
    double* V;        // k x k, column-major, ld k (starts as the identity)
    double* snap;     // 2 x (kk + kk / 2): per step, diag(W) and W(p, q) of the step's pairs
    int k;            // order
    int kk;           // tournament size: k rounded up to even (index k, if present, is empty)
    unsigned* bar;    // [0] arrivals, [1] generation (zero on entry)
    int* err;         // set when a barrier wait ran out
    int* info;        // [0] sweeps run, [1] 1 when converged
};

__device__ __forceinline__ uint64_t jac_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier; false when a wait ran out (err set) or another CTA reported one.
__device__ bool jac_sync(unsigned* bar, int* err) {
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
                const uint64_t t0 = jac_timer();
                while (*gen == g) {
                    if (jac_timer() - t0 > JAC_WAIT_NS ||
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

// Round-robin tournament (circle method) over kk players: player 0 keeps seat 0, players
// 1..kk-1 turn one seat per step; seat i meets seat kk-1-i (pair i, i < kk / 2).  Over kk - 1
// steps every pair of players meets once.
struct Tour {
    int kk;
    __device__ int player(int seat, int step) const {
        return seat == 0 ? 0 : 1 + (seat - 1 + step) % (kk - 1);
    }
    __device__ int seat(int pl, int step) const {
        if (pl == 0) return 0;
        const int m = kk - 1;
        return 1 + ((pl - 1 - step) % m + m) % m;
    }
    __device__ int pair_of(int pl, int step) const {
        const int st = seat(pl, step);
        return min(st, kk - 1 - st);
    }
    __device__ int partner(int pl, int step) const { return player(kk - 1 - seat(pl, step), step); }
};

struct Rot {
    double c, s;  // J = [[c, s], [-s, c]] on the plane (p, q)
    int p, q;     // the pair, p < q; q == k is the empty index of an odd order
    int on;       // 0: identity (converged pair or the empty index)
};

// Records W(r, c) in the next step's snapshot when (r, c) is one of that step's pairs.
__device__ __forceinline__ void snap_pair(const Tour& T, int nstep, int k, double* nopq, int r,
                                          int c, double v) {
    if (r < k && c < k && r != c && T.partner(r, nstep) == c) nopq[T.pair_of(r, nstep)] = v;
}

__global__ void __launch_bounds__(JAC_THREADS, 1) k_jacobi(JacArgs a) {
    extern __shared__ __align__(16) unsigned char jac_smem[];
    Rot* rot = reinterpret_cast<Rot*>(jac_smem);
    __shared__ int any_s;
    const int k = a.k, kk = a.kk, P = kk / 2, steps = kk - 1;
    const Tour T{kk};
    const int64_t ld = k;
    const int64_t nblk = int64_t(P) * (P + 1) / 2;         // pair blocks (x, y), x <= y
    const int64_t nv = int64_t(k) * P;                      // rows of V times pairs
    const int64_t items = nblk + nv;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
    const int64_t sn = kk + P;
    // snapshot of step 0: diag(W) and W(p, q) of step 0's pairs
    for (int64_t i = tid; i < kk; i += nthr) a.snap[i] = i < k ? a.W[i + i * ld] : 0.0;
    for (int64_t i = tid; i < P; i += nthr) {
        const int p = T.player(int(i), 0), q = T.player(kk - 1 - int(i), 0);
        a.snap[kk + i] = (p < k && q < k) ? a.W[p + int64_t(q) * ld] : 0.0;
    }
    if (!jac_sync(a.bar, a.err)) return;
    int sweep = 0;
    bool converged = false;
    int64_t g = 0;    // global step counter: snapshot g % 2 holds this step's inputs
    for (; sweep < JAC_MAX_SWEEPS && !converged; ++sweep) {
        bool rotated = false;
        for (int step = 0; step < steps; ++step, ++g) {
            const double* diag = a.snap + (g & 1) * sn;
            const double* opq = diag + kk;
            double* ndiag = a.snap + ((g + 1) & 1) * sn;
            double* nopq = ndiag + kk;
            const int nstep = step + 1 < steps ? step + 1 : 0;
            // every CTA computes all rotations of the step from the snapshot (the same values
            // and arithmetic in every CTA; nobody writes this snapshot during the step)
            if (threadIdx.x == 0) any_s = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int p = T.player(i, step), q = T.player(kk - 1 - i, step);
                if (p > q) { const int t = p; p = q; q = t; }
                Rot r{1.0, 0.0, p, q, 0};
                if (q < k) {
                    const double app = diag[p], aqq = diag[q], apq = opq[i];
                    if (fabs(apq) > JAC_TOL * sqrt(fabs(app * aqq)) && fabs(apq) > 1e-300) {
                        // symmetric Schur 2 x 2: J^T [[app, apq], [apq, aqq]] J is diagonal
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double t =
                            (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        r.c = 1.0 / sqrt(1.0 + t * t);
                        r.s = t * r.c;
                        r.on = 1;
                        any_s = 1;
                    }
                }
                rot[i] = r;
            }
            __syncthreads();
            const bool any = any_s != 0;       // the same in every CTA
            rotated |= any;
            for (int64_t it = tid; it < (any ? items : nblk); it += nthr) {
                if (it < nblk) {
                    // pair block index it -> (x, y), x <= y, it = y (y + 1) / 2 + x
                    int64_t y = int64_t((sqrt(8.0 * double(it) + 1.0) - 1.0) * 0.5);
                    while (y * (y + 1) / 2 > it) --y;
                    while ((y + 1) * (y + 2) / 2 <= it) ++y;
                    const int64_t x = it - y * (y + 1) / 2;
                    const Rot rx = rot[x], ry = rot[y];
                    if (x == y) {
                        const int p = rx.p, q = rx.q;
                        double app = p < k ? diag[p] : 0.0, aqq = q < k ? diag[q] : 0.0;
                        double apq = q < k ? opq[x] : 0.0;
                        if (rx.on) {
                            // J^T [[a, c], [c, b]] J = diag(a - t c, b + t c), t = s / c
                            const double t = rx.s / rx.c;
                            app = app - t * apq;
                            aqq = aqq + t * apq;
                            apq = 0.0;
                            a.W[p + p * ld] = app;
                            a.W[q + q * ld] = aqq;
                            a.W[p + q * ld] = 0.0;
                            a.W[q + p * ld] = 0.0;
                        }
                        if (p < k) ndiag[p] = app;
                        if (q < k) ndiag[q] = aqq;
                        snap_pair(T, nstep, k, nopq, p, q, apq);
                        continue;
                    }
                    // rows {x.p, x.q}, columns {y.p, y.q}: W <- J_x^T W J_y, mirrored
                    const int r[2] = {rx.p, rx.q}, c[2] = {ry.p, ry.q};
                    if (!rx.on && !ry.on) {
                        for (int i = 0; i < 2; ++i)
                            for (int j = 0; j < 2; ++j)
                                if (r[i] < k && c[j] < k && T.partner(r[i], nstep) == c[j])
                                    nopq[T.pair_of(r[i], nstep)] = a.W[r[i] + int64_t(c[j]) * ld];
                        continue;
                    }
                    double X[2][2];
                    for (int i = 0; i < 2; ++i)
                        for (int j = 0; j < 2; ++j)
                            X[i][j] = (r[i] < k && c[j] < k) ? a.W[r[i] + int64_t(c[j]) * ld] : 0.0;
                    if (rx.on) {
                        for (int j = 0; j < 2; ++j) {
                            const double a0 = X[0][j], a1 = X[1][j];
                            X[0][j] = rx.c * a0 - rx.s * a1;
                            X[1][j] = rx.s * a0 + rx.c * a1;
                        }
                    }
                    if (ry.on) {
                        for (int i = 0; i < 2; ++i) {
                            const double a0 = X[i][0], a1 = X[i][1];
                            X[i][0] = ry.c * a0 - ry.s * a1;
                            X[i][1] = ry.s * a0 + ry.c * a1;
                        }
                    }
                    for (int i = 0; i < 2; ++i)
                        for (int j = 0; j < 2; ++j)
                            if (r[i] < k && c[j] < k) {
                                a.W[r[i] + int64_t(c[j]) * ld] = X[i][j];
                                a.W[c[j] + int64_t(r[i]) * ld] = X[i][j];
                                snap_pair(T, nstep, k, nopq, r[i], c[j], X[i][j]);
                            }
                } else {
                    // V <- V J: row r of V, plane of pair x
                    const int64_t v = it - nblk;
                    const int x = int(v / k);
                    const int64_t r = v - int64_t(x) * k;
                    const Rot rx = rot[x];
                    if (!rx.on) continue;
                    double* vp = a.V + r + int64_t(rx.p) * ld;
                    double* vq = a.V + r + int64_t(rx.q) * ld;
                    const double xp = *vp, xq = *vq;
                    *vp = rx.c * xp - rx.s * xq;
                    *vq = rx.s * xp + rx.c * xq;
                }
            }
            if (!jac_sync(a.bar, a.err)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) { a.info[0] = sweep + 1; a.info[1] = 0; }
                return;
            }
        }
        if (!rotated) converged = true;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.info[0] = sweep;
        a.info[1] = converged ? 1 : 0;
    }
}


__global__ void k_identity_k(double* V, int k) {
    const int64_t n = int64_t(k) * k;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        V[i] = (i % k == i / k) ? 1.0 : 0.0;
}

// Eigenvalues (diag of the rotated W) in descending order: entry i goes to position
// #{j : lambda_j > lambda_i, or lambda_j == lambda_i and j < i}.  S = sqrt(max(lambda, 0)).
__global__ void k_eig_sort(const double* W, int k, int* pos, double* S) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double li = W[i + int64_t(i) * k];
        int r = 0;
        for (int j = 0; j < k; ++j) {
            const double lj = W[j + int64_t(j) * k];
            r += (lj > li || (lj == li && j < i)) ? 1 : 0;
        }
        pos[i] = r;
        S[r] = sqrt(fmax(li, 0.0));
    }
}

// U~ (column pos[i] = V column i) and U~ S^-1 (zero where S == 0); float64 and, when Uf != null,
// float32 copies for the float32 products.
__global__ void k_eig_gather(const double* V, int k, const int* pos, const double* S, double* U,
                             double* Us, float* Uf, float* Usf) {
    const int64_t n = int64_t(k) * k;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = e / k, r = e - i * k;
        const int c = pos[i];
        const double v = V[e];
        const double sc = S[c] > 0.0 ? v / S[c] : 0.0;
        U[r + int64_t(c) * k] = v;
        Us[r + int64_t(c) * k] = sc;
        if (Uf) {
            Uf[r + int64_t(c) * k] = float(v);
            Usf[r + int64_t(c) * k] = float(sc);
        }
    }
}

struct SvdBufs {
    double *W, *V, *U, *Us, *snap;
    float *Uf, *Usf;
    int* pos;
    unsigned* bar;
    int* err;
    int* info;
    GemmScratch scr;
};

void svd_reserve(Arena& ar, int64_t m, int64_t n, int64_t k, bool f64, SvdBufs& b) {
    const int64_t kk = k + (k & 1);
    b.W = ar.get<double>(k * k);
    b.V = ar.get<double>(k * k);
    b.U = ar.get<double>(k * k);
    b.Us = ar.get<double>(k * k);
    b.snap = ar.get<double>(2 * (kk + kk / 2));
    b.Uf = f64 ? nullptr : ar.get<float>(k * k);
    b.Usf = f64 ? nullptr : ar.get<float>(k * k);
    b.pos = ar.get<int>(k);
    b.bar = ar.get<unsigned>(64);
    b.err = reinterpret_cast<int*>(b.bar + 2);
    b.info = reinterpret_cast<int*>(b.bar + 4);
    b.scr.part_bytes = gemm_scratch_bytes(std::max({m, n, k}) * k);
    b.scr.part = ar.get<char>(int64_t(b.scr.part_bytes));
}

size_t jac_smem_bytes(int k) {
    const int kk = k + (k & 1);
    return sizeof(Rot) * size_t(std::max(kk / 2, 1));
}

}  // namespace
}  // namespace qb

extern "C" size_t qb_svd_workspace(int64_t m, int64_t n, int64_t k, int32_t prec) {
    using namespace qb;
    if (m < 1 || n < 1 || k < 1 || k > SVD_MAX_K || k > std::min(m, n)) return 0;
    if (prec != QB_PREC_FP64 && prec != QB_PREC_MIXED) return 0;
    Arena ar;
    SvdBufs b;
    svd_reserve(ar, m, n, k, prec == QB_PREC_FP64, b);
    return ar.used + 4096;
}

extern "C" int32_t qb_svd_from_qb(int64_t m, int64_t n, int64_t k, int32_t prec, const void* Q,
                                  int64_t ldq, const void* B, int64_t ldb, double* S, void* U,
                                  int64_t ldu, void* V, int64_t ldv, void* ws, size_t ws_bytes,
                                  int32_t* sweeps, void* stream) {
    using namespace qb;
    if (m < 1 || n < 1 || k < 1 || k > SVD_MAX_K || k > std::min(m, n)) return QB_ERR_INVALID_ARG;
    if (prec != QB_PREC_FP64 && prec != QB_PREC_MIXED) return QB_ERR_INVALID_ARG;
    if (!Q || !B || !S || ldq < m || ldb < n || (U && ldu < m) || (V && ldv < n))
        return QB_ERR_INVALID_ARG;
    const size_t need = qb_svd_workspace(m, n, k, prec);
    if (!ws || ws_bytes < need) return QB_ERR_WORKSPACE;
    try {
        const bool f64 = prec == QB_PREC_FP64;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        Arena ar;
        ar.base = reinterpret_cast<char*>(ws);
        ar.cap = ws_bytes;
        SvdBufs b;
        svd_reserve(ar, m, n, k, f64, b);
        QB_CUDA(cudaMemsetAsync(b.bar, 0, 64 * sizeof(unsigned), st));
        // W = B B^T: B row-major k x n is column-major n x k, so W = (B^T)^T (B^T) (float64
        // sums; the float32 B of the mixed path with exact products summed in float32 pairs)
        gemm(st, true, k, k, n, 1.0, XOp{f64 ? X_F64 : X_F32, B, nullptr, ldb}, B, f64, ldb, 0.0,
             b.W, true, k, f64 ? ACC_D : ACC_DF, b.scr);
        const unsigned g1 = unsigned(std::min<int64_t>(cdiv(k * k, 256), 4096));
        k_identity_k<<<g1, 256, 0, st>>>(b.V, int(k));
        QB_LAUNCHED();
        // eigendecomposition of W (cooperative launch, one CTA per SM at most)
        static int max_ctas = -1;
        const size_t smem = jac_smem_bytes(SVD_MAX_K);
        if (max_ctas < 0) {
            int dev = 0, coop = 0, per_sm = 0;
            QB_CUDA(cudaGetDevice(&dev));
            QB_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
            QB_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem)));
            QB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, JAC_THREADS,
                                                                   smem));
            max_ctas = coop ? std::min(per_sm, 1) * num_sms() : 0;
        }
        if (max_ctas <= 0) return QB_ERR_UNSUPPORTED;
        const int kk = int(k + (k & 1));
        const int64_t work = int64_t(kk / 2) * (kk / 2 + 1) / 2 + k * (kk / 2);
        const int G = int(std::max<int64_t>(1, std::min<int64_t>(max_ctas, cdiv(work, JAC_THREADS))));
        JacArgs a{b.W, b.V, b.snap, int(k), kk, b.bar, b.err, b.info};
        void* args[] = {&a};
        QB_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_jacobi), dim3(G),
                                            dim3(JAC_THREADS), args, smem, st));
        QB_LAUNCHED();
        k_eig_sort<<<1, 1024, 0, st>>>(b.W, int(k), b.pos, S);
        QB_LAUNCHED();
        k_eig_gather<<<g1, 256, 0, st>>>(b.V, int(k), b.pos, S, b.U, b.Us, b.Uf, b.Usf);
        QB_LAUNCHED();
        // U = Q U~ (m x k), V = B^T U~ S^-1 (n x k)
        if (U)
            gemm(st, false, m, k, k, 1.0, XOp{f64 ? X_F64 : X_F32, Q, nullptr, ldq},
                 f64 ? static_cast<const void*>(b.U) : static_cast<const void*>(b.Uf), f64, k, 0.0,
                 U, f64, ldu, f64 ? ACC_D : ACC_F2, b.scr);
        if (V)
            gemm(st, false, n, k, k, 1.0, XOp{f64 ? X_F64 : X_F32, B, nullptr, ldb},
                 f64 ? static_cast<const void*>(b.Us) : static_cast<const void*>(b.Usf), f64, k,
                 0.0, V, f64, ldv, f64 ? ACC_D : ACC_F2, b.scr);
        int h[4] = {0, 0, 0, 0};   // err, (pad), sweeps, converged
        QB_CUDA(cudaMemcpyAsync(h, b.err, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        QB_CUDA(cudaStreamSynchronize(st));
        if (sweeps) *sweeps = h[2];
        if (h[0]) return QB_ERR_TIMEOUT;
        return h[3] ? QB_OK : QB_NOT_CONVERGED;
    } catch (const Error& e) {
        return e.code;
    } catch (...) {
        return QB_ERR_CUDA;
    }
}
