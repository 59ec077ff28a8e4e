// Charge update q = S (G psi - b) (Eq. electrode-wise, Sec. II.B, in the library's sign of b),
// followed by the FP64 neutrality fix q <- q - u (e^T q), u = A^-1 e / (e^T A^-1 e), and the
// total charge e^T q.  In exact arithmetic S e = 0 already (Eq. S); the fix removes the
// rounding left by a single-precision S.
#include "common.cuh"

namespace cpm {

constexpr int GV_ROWS = 16;   // rows per block
constexpr int GV_M = 4;       // right-hand sides per pass

template <typename TS> struct Acc;
template <> struct Acc<float> { using t = float; };
template <> struct Acc<double> { using t = double; };

// q[r][i] = sum_g SG[i][g] psi[r][g] - sum_j S[i][j] b[r][j]; a warp per row, GV_M replicas per pass.
template <typename TS>
__global__ void __launch_bounds__(256) k_gemv(const TS* __restrict__ S, const double* __restrict__ SG, int ng,
                                              const double* __restrict__ psi, const double* __restrict__ b,
                                              int64_t n, int m, double* __restrict__ q) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r0 = 0; r0 < m; r0 += GV_M) {
        const int mm = min(GV_M, m - r0);
        for (int64_t row = (int64_t)blockIdx.x * GV_ROWS + warp; row < min(n, (int64_t)(blockIdx.x + 1) * GV_ROWS);
             row += 8) {
            const TS* Sr = S + row * n;
            TS acc[GV_M];
#pragma unroll
            for (int t = 0; t < GV_M; ++t) acc[t] = 0;
            for (int64_t j = lane; j < n; j += 32) {
                TS s = Sr[j];
#pragma unroll
                for (int t = 0; t < GV_M; ++t)
                    if (t < mm) acc[t] += s * (TS)b[(int64_t)(r0 + t) * n + j];
            }
#pragma unroll
            for (int t = 0; t < GV_M; ++t) {
                double v = (double)acc[t];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0 && t < mm) {
                    double sv = 0.0;
                    for (int g = 0; g < ng; ++g) sv += SG[row * ng + g] * psi[(int64_t)(r0 + t) * ng + g];
                    q[(int64_t)(r0 + t) * n + row] = sv - v;
                }
            }
        }
    }
}

// One block per replica: s = e^T q; q <- q - u s (symm); qtot = e^T q with Neumaier compensation.
__global__ void k_neutral(double* q, const double* u, int64_t n, int symm, double* qtot) {
    __shared__ double sh[1024];
    __shared__ double shc[1024];
    const int r = blockIdx.x;
    double* qr = q + (int64_t)r * n;
    double s = 0.0;
    if (symm) {
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += qr[i];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        s = sh[0];
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) qr[i] -= u[i] * s;
    }
    double a = 0.0, comp = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double v = qr[i];
        double t = a + v;
        comp += fabs(a) >= fabs(v) ? (a - t) + v : (v - t) + a;
        a = t;
    }
    sh[threadIdx.x] = a;
    shc[threadIdx.x] = comp;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            double x = sh[threadIdx.x], y = sh[threadIdx.x + o];
            double t = x + y;
            double e = fabs(x) >= fabs(y) ? (x - t) + y : (y - t) + x;
            sh[threadIdx.x] = t;
            shc[threadIdx.x] += shc[threadIdx.x + o] + e;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && qtot) qtot[r] = sh[0] + shc[0];
}

cpm_status update(cpm_ctx* c, int m, const double* psi, const double* b, double* q, double* qtot) {
    const int64_t n = c->n;
    cudaStream_t st = c->stream;
    const unsigned blocks = (unsigned)((n + GV_ROWS - 1) / GV_ROWS);
    c->launches += 2;
    prof_begin(c, CPM_K_GEMV);
    if (c->p.s_prec == CPM_PREC_FP32)
        k_gemv<float><<<blocks, 256, 0, st>>>(c->S32, c->SG, c->ng, psi, b, n, m, q);
    else
        k_gemv<double><<<blocks, 256, 0, st>>>(c->S, c->SG, c->ng, psi, b, n, m, q);
    prof_end(c, CPM_K_GEMV);
    CPM_LAUNCH(c, "k_gemv");
    prof_begin(c, CPM_K_NEUTRAL);
    k_neutral<<<m, 1024, 0, st>>>(q, c->u, n, c->p.symm, qtot);
    prof_end(c, CPM_K_NEUTRAL);
    CPM_LAUNCH(c, "k_neutral");
    return CPM_OK;
}

}  // namespace cpm
