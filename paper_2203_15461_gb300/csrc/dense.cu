// Dense FP64 linear algebra of the one-time setup: Cholesky factorisation A = L L^T,
// the inverse A^-1 = L^-T L^-1, and the charge-neutral capacitance matrix of
// Eq. (S), Sec. II.A:  S = A^-1 - d d^T / (e^T d),  d = A^-1 e.
// Also the electrode response SG = S G (Sec. II.B) and the neutraliser u = d / (e^T d).
#include "common.cuh"

namespace cpm {

// ----------------------------------------------------------------------------- DGEMM
// C = alpha op(A) op(B) + beta C, row-major, 64 x 64 tiles, 256 threads (4 x 4 each).
// lower: skip tiles strictly above the diagonal of C.  tri & 1: op(A)[i][k] = 0 for k < i;
// tri & 2: op(B)[k][j] = 0 for k < j (triangular operands; the K loop starts past the zeros).
// status: when non-null and nonzero the kernel returns without touching C.
constexpr int DG_BM = 64, DG_BK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, double alpha, const double* A,
                                               int64_t lda, const double* B, int64_t ldb, double beta,
                                               double* C, int64_t ldc, int lower, int tri, const unsigned* status) {
    if (status && *status) return;
    const int r0 = blockIdx.y * DG_BM, c0 = blockIdx.x * DG_BM;
    if (lower && c0 > r0 + DG_BM - 1) return;
    __shared__ double As[DG_BK][DG_BM + 1];
    __shared__ double Bs[DG_BK][DG_BM + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
    int kbeg = 0;
    if (tri & 1) kbeg = max(kbeg, r0);
    if (tri & 2) kbeg = max(kbeg, c0);
    kbeg = (kbeg / DG_BK) * DG_BK;
    for (int k0 = kbeg; k0 < K; k0 += DG_BK) {
        for (int e = threadIdx.x; e < DG_BK * DG_BM; e += 256) {
            int m, kk;
            if (TA) { m = e % DG_BM; kk = e / DG_BM; } else { kk = e % DG_BK; m = e / DG_BK; }
            int gi = r0 + m, gk = k0 + kk;
            double v = 0.0;
            if (gi < M && gk < K) v = TA ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk];
            As[kk][m] = v;
            int nn;
            if (TB) { kk = e % DG_BK; nn = e / DG_BK; } else { nn = e % DG_BM; kk = e / DG_BM; }
            int gj = c0 + nn;
            gk = k0 + kk;
            v = 0.0;
            if (gj < N && gk < K) v = TB ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < DG_BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) a[p] = As[kk][ty + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int i = r0 + ty + 16 * p;
        if (i >= M) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int j = c0 + tx + 16 * q;
            if (j >= N) continue;
            double* cp = C + (int64_t)i * ldc + j;
            *cp = beta == 0.0 ? alpha * acc[p][q] : fma(beta, *cp, alpha * acc[p][q]);
        }
    }
}

cpm_status launch_dgemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int lower,
                        int tri, const unsigned* status) {
    if (M <= 0 || N <= 0) return CPM_OK;
    dim3 grid((N + DG_BM - 1) / DG_BM, (M + DG_BM - 1) / DG_BM);
    if (ta && tb) k_dgemm<true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, tri, status);
    else if (ta) k_dgemm<true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, tri, status);
    else if (tb) k_dgemm<false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, tri, status);
    else k_dgemm<false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, tri, status);
    return cudaGetLastError() == cudaSuccess ? CPM_OK : CPM_E_CUDA;
}

// ----------------------------------------------------------------------------- diagonal blocks
constexpr int NB = 64;

// Unblocked Cholesky of one kb x kb diagonal block (in place, lower), and the inverse of
// its factor written to Linv (NB x NB, zero above the diagonal).  A pivot that is not
// positive and finite sets ST_NOT_SPD and stops the factorisation.
__global__ void __launch_bounds__(256) k_potrf(double* Ab, int64_t lda, int kb, double* Linv, unsigned* status) {
    if (*status) return;
    __shared__ double L[NB][NB + 1];
    __shared__ int bad;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        int i = e / NB, j = e % NB;
        L[i][j] = (i < kb && j <= i) ? Ab[(int64_t)i * lda + j] : 0.0;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (threadIdx.x == 0) {
            double pv = L[j][j];
            if (!(pv > 0.0) || !isfinite(pv)) bad = 1;
            else L[j][j] = sqrt(pv);
        }
        __syncthreads();
        if (bad) break;
        for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) L[i][j] /= L[j][j];
        __syncthreads();
        const int rem = kb - j - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            int i = j + 1 + e / rem, k = j + 1 + e % rem;
            if (k <= i) L[i][k] -= L[i][j] * L[k][j];
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) atomicOr(status, ST_NOT_SPD);
        return;
    }
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
        int i = e / kb, j = e % kb;
        Ab[(int64_t)i * lda + j] = j <= i ? L[i][j] : 0.0;
    }
    // inverse of the lower-triangular factor, one column per thread
    for (int col = threadIdx.x; col < NB; col += blockDim.x) {
        for (int i = 0; i < NB; ++i) {
            double x = 0.0;
            if (col < kb && i < kb && i >= col) {
                if (i == col) x = 1.0 / L[i][i];
                else {
                    double s = 0.0;
                    for (int k = col; k < i; ++k) s += L[i][k] * Linv[k * NB + col];
                    x = -s / L[i][i];
                }
            }
            Linv[i * NB + col] = x;
        }
    }
}

// Inverse of a kb x kb lower-triangular diagonal block, in place (the factor is staged in
// shared memory; each thread writes one column of the inverse straight to the block).
__global__ void __launch_bounds__(64) k_trtri(double* Ab, int64_t lda, int kb, const unsigned* status) {
    if (*status) return;
    __shared__ double L[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        int i = e / NB, j = e % NB;
        L[i][j] = (i < kb && j <= i) ? Ab[(int64_t)i * lda + j] : 0.0;
    }
    __syncthreads();
    const int col = threadIdx.x;
    if (col < kb) {
        for (int i = 0; i < kb; ++i) {
            double x = 0.0;
            if (i == col) x = 1.0 / L[i][i];
            else if (i > col) {
                double s = 0.0;
                for (int k = col; k < i; ++k) s += L[i][k] * Ab[(int64_t)k * lda + col];
                x = -s / L[i][i];
            }
            Ab[(int64_t)i * lda + col] = x;
        }
    }
}

// ----------------------------------------------------------------------------- projection
__global__ void k_mirror_lower(double* S, int64_t n) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
        if (j < i) S[j * n + i] = S[i * n + j];
}

// d_i = sum_j S_ij, one warp per row (fixed order).
__global__ void k_rowsum(const double* S, int64_t n, double* d) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += S[row * n + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) d[row] = s;
}

// out[0] = sum_i v_i, single block, fixed order.
__global__ void k_sum1(const double* v, int64_t n, double* out) {
    __shared__ double sh[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

__global__ void k_project(double* S, float* S32, const double* d, const double* dsum, int64_t n, int symm,
                          double* u) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double s = *dsum;
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
        double v = S[i * n + j];
        if (symm) v -= d[i] * d[j] / s;
        S[i * n + j] = v;
        S32[i * n + j] = (float)v;
        if (i == 0 && u) u[j] = symm ? d[j] / s : 0.0;
    }
}

// SG[i][g] = sum_{j in electrode g} S_ij, one warp per row; at most 16 electrodes.
__global__ void k_sg(const double* S, const int* group, int64_t n, int ng, double* SG) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double acc[16];
#pragma unroll
    for (int g = 0; g < 16; ++g) acc[g] = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
        int g = group[j];
        double v = S[row * n + j];
#pragma unroll
        for (int h = 0; h < 16; ++h)
            if (h == g) acc[h] += v;
    }
    for (int g = 0; g < ng; ++g) {
        double s = acc[g < 16 ? g : 0];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) SG[row * ng + g] = s;
    }
}

cpm_status invert_and_project(cpm_ctx* c) {
    const int64_t n = c->n;
    cudaStream_t st = c->stream;
    double* W = c->W;
    double* Linv = c->red + 64;   // NB x NB scratch follows the scalars
    CPM_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), st));
    CPM_CUDA(c, cudaMemcpyAsync(W, c->A, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // blocked right-looking Cholesky, lower triangle
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        const int kb = (int)std::min<int64_t>(NB, n - k0);
        k_potrf<<<1, 256, 0, st>>>(W + k0 * n + k0, n, kb, Linv, c->status);
        CPM_LAUNCH(c, "k_potrf");
        const int rows = (int)(n - k0 - kb);
        if (rows > 0) {
            double* P = W + (k0 + kb) * n + k0;
            // panel: P <- P L_kk^-T (in place; one 64-wide tile column, so every block owns its rows)
            CPM_TRY(launch_dgemm(st, false, true, rows, kb, kb, 1.0, P, n, Linv, NB, 0.0, P, n, 0, 0, c->status));
            // trailing update, lower triangle: A22 <- A22 - P P^T
            CPM_TRY(launch_dgemm(st, false, true, rows, rows, kb, -1.0, P, n, P, n, 1.0, W + (k0 + kb) * (n + 1), n, 1,
                                 0, c->status));
        }
    }
    unsigned hst = 0;
    CPM_CUDA(c, cudaMemcpyAsync(&hst, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CPM_CUDA(c, cudaStreamSynchronize(st));
    if (hst & ST_NOT_SPD) return set_err(c, CPM_E_NOT_SPD, "elastance matrix is not positive definite");
    // W <- L^-1, block row by block row; R is an NB x n scratch held in S
    double* R = c->S;
    for (int64_t i0 = 0; i0 < n; i0 += NB) {
        const int kb = (int)std::min<int64_t>(NB, n - i0);
        k_trtri<<<1, 64, 0, st>>>(W + i0 * n + i0, n, kb, c->status);
        CPM_LAUNCH(c, "k_trtri");
        if (i0 > 0) {
            CPM_TRY(launch_dgemm(st, false, false, kb, (int)i0, (int)i0, 1.0, W + i0 * n, n, W, n, 0.0, R, n, 0, 2,
                                 c->status));
            CPM_TRY(launch_dgemm(st, false, false, kb, (int)i0, kb, -1.0, W + i0 * n + i0, n, R, n, 0.0, W + i0 * n, n,
                                 0, 0, c->status));
        }
    }
    // A^-1 = W^T W, lower tiles, then mirrored
    CPM_TRY(launch_dgemm(st, true, false, (int)n, (int)n, (int)n, 1.0, W, n, W, n, 0.0, c->S, n, 1, 3, c->status));
    dim3 g2((unsigned)((n + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
    k_mirror_lower<<<g2, 256, 0, st>>>(c->S, n);
    CPM_LAUNCH(c, "k_mirror_lower");
    return project_inverse(c);
}

// Row sums of the single-precision S in FP64 (one warp per row, a fixed order), into dvec.  The
// single-precision products centre b per output, sum_j S_ij (b_j - b_i); without the projection
// (symm = 0) the rows of A^-1 do not sum to zero, and the update adds b_i times these sums back.
__global__ void k_rowsum32(const float* S32, int64_t n, double* out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += (double)S32[row * n + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[row] = s;
}

cpm_status fp32_rowsums(cpm_ctx* c) {
    if (c->p.symm) return CPM_OK;
    k_rowsum32<<<(unsigned)((c->n * 32 + 255) / 256), 256, 0, c->stream>>>(c->S32, c->n, c->dvec);
    CPM_LAUNCH(c, "k_rowsum32");
    return CPM_OK;
}

// With A^-1 in S: d = A^-1 e, e^T d, the projection of Eq. (S) (symm = 1), the FP32 copy of S, u and
// SG = S G; synchronises.
cpm_status project_inverse(cpm_ctx* c) {
    const int64_t n = c->n;
    cudaStream_t st = c->stream;
    dim3 g2((unsigned)((n + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
    k_rowsum<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(c->S, n, c->dvec);
    CPM_LAUNCH(c, "k_rowsum");
    k_sum1<<<1, 1024, 0, st>>>(c->dvec, n, c->red);
    CPM_LAUNCH(c, "k_sum1");
    k_project<<<g2, 256, 0, st>>>(c->S, c->S32, c->dvec, c->red, n, c->p.symm, c->u);
    CPM_LAUNCH(c, "k_project");
    k_sg<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(c->S, c->group, n, c->ng, c->SG);
    CPM_LAUNCH(c, "k_sg");
    CPM_TRY(fp32_rowsums(c));
    CPM_CUDA(c, cudaMemcpyAsync(&c->etd, c->red, sizeof(double), cudaMemcpyDeviceToHost, st));
    CPM_CUDA(c, cudaStreamSynchronize(st));
    ccm_invalidate(c);
    return CPM_OK;
}

}  // namespace cpm
