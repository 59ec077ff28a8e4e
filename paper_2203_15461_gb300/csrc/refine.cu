// Electrode-wise capacitance from a single-precision Cholesky factor and FP64 iterative refinement.
//
// C~ = G^T S G (Sec. II.C; Sec. III.B reads the vacuum capacitance C0 from it) needs only
// A^-1 e and A^-1 g_h, not the whole inverse: solve A X = [e, g_1 .. g_Ng] with the factor
// A ~ L L^T computed in FP32, and refine X <- X + (L L^T)^-1 (B - A X) with the residual
// formed in FP64 against the FP64 elastance until it stops shrinking.  Then, with d = A^-1 e
// and s = e^T d (Eq. S):  C~_gh = g_g^T A^-1 g_h - (g_g^T d)(g_h^T d) / s.
#include "common.cuh"

namespace cpm {

constexpr int RB = 64;   // block size of the factorisation

// ----------------------------------------------------------------------------- FP32 GEMM
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, float alpha, const float* A, int64_t lda,
                                               const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                                               int lower, const unsigned* status) {
    if (status && *status) return;
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    if (lower && c0 > r0 + 63) return;
    __shared__ float As[16][65];
    __shared__ float Bs[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int m, kk;
            if (TA) { m = e % 64; kk = e / 64; } else { kk = e % 16; m = e / 16; }
            int gi = r0 + m, gk = k0 + kk;
            As[kk][m] = (gi < M && gk < K) ? (TA ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk]) : 0.f;
            int nn;
            if (TB) { kk = e % 16; nn = e / 16; } else { nn = e % 64; kk = e / 64; }
            int gj = c0 + nn;
            gk = k0 + kk;
            Bs[kk][nn] = (gj < N && gk < K) ? (TB ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) a[p] = As[kk][ty + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
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
            float* cp = C + (int64_t)i * ldc + j;
            *cp = beta == 0.f ? alpha * acc[p][q] : beta * *cp + alpha * acc[p][q];
        }
    }
}

static cpm_status sgemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, float alpha, const float* A,
                        int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc, int lower,
                        const unsigned* status) {
    if (M <= 0 || N <= 0) return CPM_OK;
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    if (ta && tb) k_sgemm<true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status);
    else if (ta) k_sgemm<true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status);
    else if (tb) k_sgemm<false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status);
    else k_sgemm<false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower, status);
    return cudaGetLastError() == cudaSuccess ? CPM_OK : CPM_E_CUDA;
}

// Unblocked FP32 Cholesky of one diagonal block (in place, lower) and the inverse of its factor
// (RB x RB, zero above the diagonal) in Linv.  A pivot that is not positive sets ST_NOT_SPD.
__global__ void __launch_bounds__(256) k_spotrf(float* Ab, int64_t lda, int kb, float* Linv, unsigned* status) {
    if (*status) return;
    __shared__ float L[RB][RB + 1];
    __shared__ int bad;
    for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) {
        int i = e / RB, j = e % RB;
        L[i][j] = (i < kb && j <= i) ? Ab[(int64_t)i * lda + j] : 0.f;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (threadIdx.x == 0) {
            float pv = L[j][j];
            if (!(pv > 0.f) || !isfinite(pv)) bad = 1;
            else L[j][j] = sqrtf(pv);
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
        Ab[(int64_t)i * lda + j] = j <= i ? L[i][j] : 0.f;
    }
    for (int col = threadIdx.x; col < RB; col += blockDim.x) {
        for (int i = 0; i < RB; ++i) {
            float x = 0.f;
            if (col < kb && i < kb && i >= col) {
                if (i == col) x = 1.f / L[i][i];
                else {
                    float s = 0.f;
                    for (int k = col; k < i; ++k) s += L[i][k] * Linv[k * RB + col];
                    x = -s / L[i][i];
                }
            }
            Linv[i * RB + col] = x;
        }
    }
}

__global__ void k_d2f(const double* a, float* b, int64_t cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) b[i] = (float)a[i];
}
__global__ void k_axpy_f2d(const float* d, double* x, int64_t cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) x[i] += (double)d[i];
}
// B = [e, g_1 .. g_Ng] (n x (1 + Ng), row-major)
__global__ void k_rhs(const int* group, int64_t n, int ng, double* B) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    B[i * (ng + 1)] = 1.0;
    for (int g = 0; g < ng; ++g) B[i * (ng + 1) + 1 + g] = group[i] == g ? 1.0 : 0.0;
}
// out[0] = max_i,c |R[i][c]| / max(1, max |B|) per call (single block)
__global__ void k_maxabs(const double* R, int64_t cnt, double* out) {
    __shared__ double sh[1024];
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) m = fmax(m, fabs(R[i]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}
// GX[g][c] = sum over sites i of electrode g of X[i][c] (fixed order)
__global__ void k_gsum(const double* X, const int* group, int64_t n, int ng, int nr, double* GX) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ng * nr) return;
    const int g = t / nr, cc = t % nr;
    double a = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (group[i] == g) a += X[i * nr + cc];
    GX[t] = a;
}

__global__ void k_add_identity(double* R, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) R[i * n + i] += 1.0;
}
// X <- (X + X^T) / 2 (A^-1 is symmetric; the refined columns agree with it to the refinement residual)
__global__ void k_symmetrize(double* X, int64_t n) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = blockIdx.y; i < j && j < n; i += gridDim.y) {
        const double v = 0.5 * (X[i * n + j] + X[j * n + i]);
        X[i * n + j] = v;
        X[j * n + i] = v;
    }
}

// FP32 blocked Cholesky of A into L (lower, in place) with the inverses of its diagonal blocks
static cpm_status factor32(cpm_ctx* c, float* L, float* Linv) {
    const int64_t n = c->n;
    const int nb = (int)((n + RB - 1) / RB);
    cudaStream_t st = c->stream;
    CPM_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), st));
    k_d2f<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(c->A, L, n * n);
    for (int kb0 = 0; kb0 < nb; ++kb0) {
        const int64_t k0 = (int64_t)kb0 * RB;
        const int kb = (int)std::min<int64_t>(RB, n - k0);
        k_spotrf<<<1, 256, 0, st>>>(L + k0 * n + k0, n, kb, Linv + (int64_t)kb0 * RB * RB, c->status);
        const int rows = (int)(n - k0 - kb);
        if (rows > 0) {
            float* P = L + (k0 + kb) * n + k0;
            CPM_TRY(sgemm(st, false, true, rows, kb, kb, 1.f, P, n, Linv + (int64_t)kb0 * RB * RB, RB, 0.f, P, n, 0,
                          c->status));
            CPM_TRY(sgemm(st, false, true, rows, rows, kb, -1.f, P, n, P, n, 1.f, L + (k0 + kb) * (n + 1), n, 1,
                          c->status));
        }
    }
    unsigned hst = 0;
    CPM_CUDA(c, cudaMemcpyAsync(&hst, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CPM_CUDA(c, cudaStreamSynchronize(st));
    if (hst & ST_NOT_SPD) return set_err(c, CPM_E_NOT_SPD, "elastance matrix is not positive definite (FP32 factor)");
    return CPM_OK;
}

// Y <- (L L^T)^-1 Y for nr right-hand sides in FP32: forward then backward block substitution
static cpm_status solve32(cpm_ctx* c, const float* L, const float* Linv, float* Y, int nr) {
    const int64_t n = c->n;
    const int nb = (int)((n + RB - 1) / RB);
    cudaStream_t st = c->stream;
    for (int ib = 0; ib < nb; ++ib) {
        const int64_t i0 = (int64_t)ib * RB;
        const int kb = (int)std::min<int64_t>(RB, n - i0);
        CPM_TRY(sgemm(st, false, false, kb, nr, kb, 1.f, Linv + (int64_t)ib * RB * RB, RB, Y + i0 * nr, nr, 0.f,
                      Y + i0 * nr, nr, 0, nullptr));
        const int below = (int)(n - i0 - kb);
        if (below > 0)
            CPM_TRY(sgemm(st, false, false, below, nr, kb, -1.f, L + (i0 + kb) * n + i0, n, Y + i0 * nr, nr, 1.f,
                          Y + (i0 + kb) * nr, nr, 0, nullptr));
    }
    for (int ib = nb - 1; ib >= 0; --ib) {
        const int64_t i0 = (int64_t)ib * RB;
        const int kb = (int)std::min<int64_t>(RB, n - i0);
        CPM_TRY(sgemm(st, true, false, kb, nr, kb, 1.f, Linv + (int64_t)ib * RB * RB, RB, Y + i0 * nr, nr, 0.f,
                      Y + i0 * nr, nr, 0, nullptr));
        if (i0 > 0)
            CPM_TRY(sgemm(st, true, false, (int)i0, nr, kb, -1.f, L + i0 * n, n, Y + i0 * nr, nr, 1.f, Y, nr, 0, nullptr));
    }
    return CPM_OK;
}

// A^-1 from the FP32 factor, refined in FP64 (X <- X + (L L^T)^-1 (I - A X), residual against the FP64
// A) until the residual stops shrinking; X is kept in S and the residual in the factor workspace W.
cpm_status invert_ir(cpm_ctx* c) {
    const int64_t n = c->n;
    const int nb = (int)((n + RB - 1) / RB);
    cudaStream_t st = c->stream;
    float *L = nullptr, *Linv = nullptr, *Y = nullptr;
    double* red = nullptr;
    auto cleanup = [&]() { dev_free(c, L); dev_free(c, Linv); dev_free(c, Y); dev_free(c, red); };
    cpm_status s = CPM_OK;
#define IR_TRY(expr)       \
    do {                   \
        s = (expr);        \
        if (s != CPM_OK) { \
            cleanup();     \
            return s;      \
        }                  \
    } while (0)
    IR_TRY(dev_alloc(c, (void**)&L, sizeof(float) * n * n));
    IR_TRY(dev_alloc(c, (void**)&Linv, sizeof(float) * RB * RB * nb));
    IR_TRY(dev_alloc(c, (void**)&Y, sizeof(float) * n * n));
    IR_TRY(dev_alloc(c, (void**)&red, sizeof(double) * 8));
    IR_TRY(factor32(c, L, Linv));
    double* X = c->S;
    double* R = c->W;
    IR_TRY(cuda_check(c, cudaMemsetAsync(X, 0, sizeof(double) * n * n, st), "memset"));
    double resid = 1.0, prev = 1e300;
    int it = 0;
    for (; it < 30; ++it) {
        // R = I - A X (FP64)
        IR_TRY(launch_dgemm(st, false, false, (int)n, (int)n, (int)n, -1.0, c->A, n, X, n, 0.0, R, n, 0, 0, nullptr));
        k_add_identity<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(R, n);
        k_maxabs<<<1, 1024, 0, st>>>(R, n * n, red);
        double rmax = 0.0;
        IR_TRY(cuda_check(c, cudaMemcpyAsync(&rmax, red, sizeof(double), cudaMemcpyDeviceToHost, st), "copy"));
        IR_TRY(cuda_check(c, cudaStreamSynchronize(st), "sync"));
        resid = rmax;
        if (!(resid < prev * 0.9) && it > 0) break;   // no longer shrinking
        prev = resid;
        if (resid < 1e-15) break;
        k_d2f<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(R, Y, n * n);
        IR_TRY(solve32(c, L, Linv, Y, (int)n));
        k_axpy_f2d<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(Y, X, n * n);
    }
    c->ir_sweeps = it;
    c->ir_resid = resid;
    dim3 g2((unsigned)((n + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
    k_symmetrize<<<g2, 256, 0, st>>>(X, n);
    IR_TRY(cuda_check(c, cudaGetLastError(), "k_symmetrize"));
    cleanup();
#undef IR_TRY
    return project_inverse(c);
}

}  // namespace cpm

using namespace cpm;

extern "C" cpm_status cpm_capacitance_ir(cpm_ctx* c, double* C_out, int32_t* iters_out, double* resid_out) {
    if (!c || !C_out) return CPM_E_ARG;
    if (!c->assembled) return set_err(c, CPM_E_STATE, "cpm_capacitance_ir before cpm_assemble");
    if (!c->has_A) return set_err(c, CPM_E_STATE, "cpm_capacitance_ir: A is not held (cpm_prepare or cpm_release_assembly)");
    const int64_t n = c->n;
    const int ng = c->ng, nr = ng + 1;
    cudaStream_t st = c->stream;
    float *L = nullptr, *Linv = nullptr, *Y = nullptr;
    double *B = nullptr, *X = nullptr, *R = nullptr, *red = nullptr;
    const int nb = (int)((n + RB - 1) / RB);
    auto cleanup = [&]() {
        dev_free(c, L); dev_free(c, Linv); dev_free(c, Y); dev_free(c, B); dev_free(c, X); dev_free(c, R);
        dev_free(c, red);
    };
    cpm_status s = CPM_OK;
#define IR_TRY(expr)                  \
    do {                              \
        s = (expr);                   \
        if (s != CPM_OK) {            \
            cleanup();                \
            return s;                 \
        }                             \
    } while (0)
    IR_TRY(dev_alloc(c, (void**)&L, sizeof(float) * n * n));
    IR_TRY(dev_alloc(c, (void**)&Linv, sizeof(float) * RB * RB * nb));
    IR_TRY(dev_alloc(c, (void**)&Y, sizeof(float) * n * nr));
    IR_TRY(dev_alloc(c, (void**)&B, sizeof(double) * n * nr));
    IR_TRY(dev_alloc(c, (void**)&X, sizeof(double) * n * nr));
    IR_TRY(dev_alloc(c, (void**)&R, sizeof(double) * n * nr));
    IR_TRY(dev_alloc(c, (void**)&red, sizeof(double) * (8 + ng * nr)));
    IR_TRY(cuda_check(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), st), "memset"));
    k_d2f<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(c->A, L, n * n);
    // FP32 blocked Cholesky, right-looking, lower
    for (int kb0 = 0; kb0 < nb; ++kb0) {
        const int64_t k0 = (int64_t)kb0 * RB;
        const int kb = (int)std::min<int64_t>(RB, n - k0);
        k_spotrf<<<1, 256, 0, st>>>(L + k0 * n + k0, n, kb, Linv + (int64_t)kb0 * RB * RB, c->status);
        const int rows = (int)(n - k0 - kb);
        if (rows > 0) {
            float* P = L + (k0 + kb) * n + k0;
            IR_TRY(sgemm(st, false, true, rows, kb, kb, 1.f, P, n, Linv + (int64_t)kb0 * RB * RB, RB, 0.f, P, n, 0,
                         c->status));
            IR_TRY(sgemm(st, false, true, rows, rows, kb, -1.f, P, n, P, n, 1.f, L + (k0 + kb) * (n + 1), n, 1,
                         c->status));
        }
    }
    unsigned hst = 0;
    IR_TRY(cuda_check(c, cudaMemcpyAsync(&hst, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "copy"));
    IR_TRY(cuda_check(c, cudaStreamSynchronize(st), "sync"));
    if (hst & ST_NOT_SPD) {
        cleanup();
        return set_err(c, CPM_E_NOT_SPD, "elastance matrix is not positive definite (FP32 factor)");
    }
    k_rhs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c->group, n, ng, B);
    IR_TRY(cuda_check(c, cudaMemsetAsync(X, 0, sizeof(double) * n * nr, st), "memset"));
    double bmax = 1.0, resid = 1.0, prev = 1e300;
    int it = 0;
    for (; it < 30; ++it) {
        // R = B - A X  (FP64)
        IR_TRY(cuda_check(c, cudaMemcpyAsync(R, B, sizeof(double) * n * nr, cudaMemcpyDeviceToDevice, st), "copy"));
        IR_TRY(launch_dgemm(st, false, false, (int)n, nr, (int)n, -1.0, c->A, n, X, nr, 1.0, R, nr, 0, 0, nullptr));
        k_maxabs<<<1, 1024, 0, st>>>(R, n * nr, red);
        double rmax = 0.0;
        IR_TRY(cuda_check(c, cudaMemcpyAsync(&rmax, red, sizeof(double), cudaMemcpyDeviceToHost, st), "copy"));
        IR_TRY(cuda_check(c, cudaStreamSynchronize(st), "sync"));
        resid = rmax / bmax;
        if (!(resid < prev * 0.9) && it > 0) break;   // no longer shrinking
        prev = resid;
        if (resid < 1e-15) break;
        // Y = (L L^T)^-1 R in FP32: forward then backward block substitution, right-looking
        k_d2f<<<(unsigned)((n * nr + 255) / 256), 256, 0, st>>>(R, Y, n * nr);
        for (int ib = 0; ib < nb; ++ib) {
            const int64_t i0 = (int64_t)ib * RB;
            const int kb = (int)std::min<int64_t>(RB, n - i0);
            IR_TRY(sgemm(st, false, false, kb, nr, kb, 1.f, Linv + (int64_t)ib * RB * RB, RB, Y + i0 * nr, nr, 0.f,
                         Y + i0 * nr, nr, 0, nullptr));
            const int below = (int)(n - i0 - kb);
            if (below > 0)
                IR_TRY(sgemm(st, false, false, below, nr, kb, -1.f, L + (i0 + kb) * n + i0, n, Y + i0 * nr, nr, 1.f,
                             Y + (i0 + kb) * nr, nr, 0, nullptr));
        }
        for (int ib = nb - 1; ib >= 0; --ib) {
            const int64_t i0 = (int64_t)ib * RB;
            const int kb = (int)std::min<int64_t>(RB, n - i0);
            IR_TRY(sgemm(st, true, false, kb, nr, kb, 1.f, Linv + (int64_t)ib * RB * RB, RB, Y + i0 * nr, nr, 0.f,
                         Y + i0 * nr, nr, 0, nullptr));
            if (i0 > 0)
                IR_TRY(sgemm(st, true, false, (int)i0, nr, kb, -1.f, L + i0 * n, n, Y + i0 * nr, nr, 1.f, Y, nr, 0,
                             nullptr));
        }
        k_axpy_f2d<<<(unsigned)((n * nr + 255) / 256), 256, 0, st>>>(Y, X, n * nr);
    }
    k_gsum<<<(ng * nr + 63) / 64, 64, 0, st>>>(X, c->group, n, ng, nr, red + 8);
    std::vector<double> GX((size_t)ng * nr);
    IR_TRY(cuda_check(c, cudaMemcpyAsync(GX.data(), red + 8, sizeof(double) * ng * nr, cudaMemcpyDeviceToHost, st),
                      "copy"));
    IR_TRY(cuda_check(c, cudaStreamSynchronize(st), "sync"));
    double ssum = 0.0;
    for (int g = 0; g < ng; ++g) ssum += GX[(size_t)g * nr];
    for (int g = 0; g < ng; ++g)
        for (int h = 0; h < ng; ++h) {
            double v = GX[(size_t)g * nr + 1 + h];
            if (c->p.symm) v -= GX[(size_t)g * nr] * GX[(size_t)h * nr] / ssum;
            C_out[g * ng + h] = v;
        }
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = resid;
    cleanup();
#undef IR_TRY
    return CPM_OK;
}
