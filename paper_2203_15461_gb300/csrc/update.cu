// Charge update q = S (G psi - b) (Eq. electrode-wise, Sec. II.B, in the library's sign of b),
// followed by the FP64 neutrality fix q <- q - u (e^T q), u = A^-1 e / (e^T A^-1 e), and the
// total charge e^T q.  In exact arithmetic S e = 0 already (Eq. S); the fix removes the
// rounding left by a single-precision S.
#include "common.cuh"

namespace cpm {

// S is symmetric, so q_i = sum_j S_ji b_j: one thread per output i reads column i of S (row
// j = column j, coalesced across the block), the b_j are broadcast from shared memory, and the
// rows j are split over blocks (partial sums reduced in FP64 in a fixed order).
//
// Single precision: the sum is centred per output, sum_j S_ij (b_j - b_i), which equals S b
// because the rows of S sum to zero (Eq. S); without the projection (symm = 0, S = A^-1) the
// reduction adds b_i sum_j S_ij back, from the FP64 row sums of the stored single-precision S.  S rounded to FP32 then only perturbs the
// products where b_j differs from b_i, i.e. mostly far sites where S_ij is small; b enters as
// an FP32 hi + lo pair so the differences are formed to about 2^-24 of themselves, and each
// thread's partial sum is Kahan-compensated.
constexpr int GT_COLS = 128;   // outputs (threads) per block
constexpr int GT_JT = 64;      // rows of S staged per iteration
constexpr int GT_MR = 8;       // replicas per block

template <typename TS> struct LaneSum {
    TS s = 0;
    __device__ __forceinline__ void add(TS x) { s += x; }
    __device__ __forceinline__ double value() const { return (double)s; }
};
template <> struct LaneSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// bhl[t] = (hi, lo) with hi = float(b[t]) and lo = float(b[t] - hi)
__global__ void k_split_b(const double* __restrict__ b, int64_t cnt, float2* __restrict__ bhl) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    double v = b[t];
    float hi = (float)v;
    bhl[t] = make_float2(hi, (float)(v - (double)hi));
}

template <typename TS> struct BVal;
template <> struct BVal<float> { using t = float2; };
template <> struct BVal<double> { using t = double; };

__device__ __forceinline__ float centred(float2 bj, float2 bi) { return (bj.x - bi.x) + (bj.y - bi.y); }
__device__ __forceinline__ double centred(double bj, double) { return bj; }

// part[split][r][i] = sum over this split's rows j of S_ji x_j (x_j = b_j - b_i in FP32, b_j in FP64)
template <typename TS>
__global__ void __launch_bounds__(GT_COLS) k_gemv_t(const TS* __restrict__ S, const typename BVal<TS>::t* __restrict__ bv,
                                                     int64_t n, int m, int64_t jchunk, double* __restrict__ part) {
    typedef typename BVal<TS>::t B;
    __shared__ B bs[GT_MR][GT_JT];
    const int64_t i = (int64_t)blockIdx.x * GT_COLS + threadIdx.x;
    const int split = blockIdx.y;
    const int r0 = blockIdx.z * GT_MR;
    const int mm = min(GT_MR, m - r0);
    const int64_t jb = (int64_t)split * jchunk, je = min(n, jb + jchunk);
    B bi[GT_MR];
    LaneSum<TS> acc[GT_MR];
#pragma unroll
    for (int t = 0; t < GT_MR; ++t) bi[t] = (t < mm && i < n) ? bv[(int64_t)(r0 + t) * n + i] : B{};
    for (int64_t j0 = jb; j0 < je; j0 += GT_JT) {
        for (int e = threadIdx.x; e < GT_MR * GT_JT; e += GT_COLS) {
            int t = e / GT_JT, jj = e % GT_JT;
            int64_t j = j0 + jj;
            bs[t][jj] = (t < mm && j < je) ? bv[(int64_t)(r0 + t) * n + j] : B{};
        }
        __syncthreads();
        const int jn = (int)min((int64_t)GT_JT, je - j0);
        if (i < n) {
            // eight loads of S in flight before they are used
            int jj = 0;
            for (; jj + 8 <= jn; jj += 8) {
                TS sv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) sv[u] = S[(j0 + jj + u) * n + i];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int t = 0; t < GT_MR; ++t)
                        if (t < mm) acc[t].add(sv[u] * (TS)centred(bs[t][jj + u], bi[t]));
            }
            for (; jj < jn; ++jj) {
                const TS sv = S[(j0 + jj) * n + i];
#pragma unroll
                for (int t = 0; t < GT_MR; ++t)
                    if (t < mm) acc[t].add(sv * (TS)centred(bs[t][jj], bi[t]));
            }
        }
        __syncthreads();
    }
    if (i < n) {
#pragma unroll
        for (int t = 0; t < GT_MR; ++t)
            if (t < mm) part[((int64_t)split * m + r0 + t) * n + i] = acc[t].value();
    }
}

// Single-precision variant of k_gemv_t: the hi/lo pairs of b are staged jj-major in shared memory so
// one 16-byte load serves two replicas, and eight loads of S are in flight before use.  Each tile
// of GT_JT terms is summed plainly in FP32 as S_ij (hi_j - hi_i) + S_ij lo_j (the hi difference
// is exact; centring the tiny lo part would change nothing), and the tile sums are added with
// compensation.
__global__ void __launch_bounds__(GT_COLS) k_gemv32(const float* __restrict__ S, const float2* __restrict__ bv,
                                                   int64_t n, int m, int64_t jchunk, double* __restrict__ part) {
    __shared__ __align__(16) float2 bs[GT_JT][GT_MR];
    const int64_t i = (int64_t)blockIdx.x * GT_COLS + threadIdx.x;
    const int split = blockIdx.y;
    const int r0 = blockIdx.z * GT_MR;
    const int mm = min(GT_MR, m - r0);
    const int64_t jb = (int64_t)split * jchunk, je = min(n, jb + jchunk);
    float2 bi[GT_MR];
    LaneSum<float> acc[GT_MR];
#pragma unroll
    for (int t = 0; t < GT_MR; ++t) bi[t] = (t < mm && i < n) ? bv[(int64_t)(r0 + t) * n + i] : make_float2(0.f, 0.f);
    for (int64_t j0 = jb; j0 < je; j0 += GT_JT) {
        for (int e = threadIdx.x; e < GT_MR * GT_JT; e += GT_COLS) {
            const int t = e / GT_JT, jj = e % GT_JT;
            const int64_t j = j0 + jj;
            bs[jj][t] = (t < mm && j < je) ? bv[(int64_t)(r0 + t) * n + j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int jn = (int)min((int64_t)GT_JT, je - j0);
        if (i < n) {
            float tile[GT_MR];
#pragma unroll
            for (int t = 0; t < GT_MR; ++t) tile[t] = 0.f;
            int jj = 0;
            for (; jj + 8 <= jn; jj += 8) {
                float sv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) sv[u] = S[(j0 + jj + u) * n + i];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4* row = reinterpret_cast<const float4*>(bs[jj + u]);
#pragma unroll
                    for (int tp = 0; tp < GT_MR / 2; ++tp) {
                        const float4 v = row[tp];
                        tile[2 * tp] = fmaf(sv[u], v.x - bi[2 * tp].x, tile[2 * tp]);
                        tile[2 * tp] = fmaf(sv[u], v.y, tile[2 * tp]);
                        tile[2 * tp + 1] = fmaf(sv[u], v.z - bi[2 * tp + 1].x, tile[2 * tp + 1]);
                        tile[2 * tp + 1] = fmaf(sv[u], v.w, tile[2 * tp + 1]);
                    }
                }
            }
            for (; jj < jn; ++jj) {
                const float sv = S[(j0 + jj) * n + i];
#pragma unroll
                for (int t = 0; t < GT_MR; ++t) {
                    tile[t] = fmaf(sv, bs[jj][t].x - bi[t].x, tile[t]);
                    tile[t] = fmaf(sv, bs[jj][t].y, tile[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < GT_MR; ++t) acc[t].add(tile[t]);
        }
        __syncthreads();
    }
    if (i < n) {
#pragma unroll
        for (int t = 0; t < GT_MR; ++t)
            if (t < mm) part[((int64_t)split * m + r0 + t) * n + i] = acc[t].value();
    }
}

// k_gemv32 with two output columns per thread (8-byte loads of S, n even) and sixteen rows of S
// in flight, so that enough bytes are outstanding to stream S at HBM speed.
constexpr int G2_T = 256;
__global__ void __launch_bounds__(G2_T, 2) k_gemv32x2(const float* __restrict__ S, const float2* __restrict__ bv,
                                                      int64_t n, int m, int64_t jchunk, double* __restrict__ part) {
    __shared__ __align__(16) float2 bs[GT_JT][GT_MR];
    const int64_t i0 = ((int64_t)blockIdx.x * G2_T + threadIdx.x) * 2;
    const int split = blockIdx.y;
    const int r0 = blockIdx.z * GT_MR;
    const int mm = min(GT_MR, m - r0);
    const int64_t jb = (int64_t)split * jchunk, je = min(n, jb + jchunk);
    const bool live = i0 < n;
    float bh[2][GT_MR];
    LaneSum<float> acc[2][GT_MR];
#pragma unroll
    for (int t = 0; t < GT_MR; ++t) {
        bh[0][t] = (t < mm && live) ? bv[(int64_t)(r0 + t) * n + i0].x : 0.f;
        bh[1][t] = (t < mm && live) ? bv[(int64_t)(r0 + t) * n + i0 + 1].x : 0.f;
    }
    for (int64_t j0 = jb; j0 < je; j0 += GT_JT) {
        for (int e = threadIdx.x; e < GT_MR * GT_JT; e += G2_T) {
            const int t = e / GT_JT, jj = e % GT_JT;
            const int64_t j = j0 + jj;
            bs[jj][t] = (t < mm && j < je) ? bv[(int64_t)(r0 + t) * n + j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int jn = (int)min((int64_t)GT_JT, je - j0);
        if (live) {
            float tile[2][GT_MR];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int t = 0; t < GT_MR; ++t) tile[c][t] = 0.f;
            int jj = 0;
            for (; jj + 16 <= jn; jj += 16) {
                float2 sv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) sv[u] = *reinterpret_cast<const float2*>(S + (j0 + jj + u) * n + i0);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float4* row = reinterpret_cast<const float4*>(bs[jj + u]);
#pragma unroll
                    for (int tp = 0; tp < GT_MR / 2; ++tp) {
                        const float4 v = row[tp];   // (hi, lo) of replicas 2 tp and 2 tp + 1
                        tile[0][2 * tp] = fmaf(sv[u].x, v.x - bh[0][2 * tp], tile[0][2 * tp]);
                        tile[0][2 * tp] = fmaf(sv[u].x, v.y, tile[0][2 * tp]);
                        tile[1][2 * tp] = fmaf(sv[u].y, v.x - bh[1][2 * tp], tile[1][2 * tp]);
                        tile[1][2 * tp] = fmaf(sv[u].y, v.y, tile[1][2 * tp]);
                        tile[0][2 * tp + 1] = fmaf(sv[u].x, v.z - bh[0][2 * tp + 1], tile[0][2 * tp + 1]);
                        tile[0][2 * tp + 1] = fmaf(sv[u].x, v.w, tile[0][2 * tp + 1]);
                        tile[1][2 * tp + 1] = fmaf(sv[u].y, v.z - bh[1][2 * tp + 1], tile[1][2 * tp + 1]);
                        tile[1][2 * tp + 1] = fmaf(sv[u].y, v.w, tile[1][2 * tp + 1]);
                    }
                }
            }
            for (; jj < jn; ++jj) {
                const float2 sv = *reinterpret_cast<const float2*>(S + (j0 + jj) * n + i0);
#pragma unroll
                for (int t = 0; t < GT_MR; ++t) {
                    tile[0][t] = fmaf(sv.x, bs[jj][t].x - bh[0][t], tile[0][t]);
                    tile[0][t] = fmaf(sv.x, bs[jj][t].y, tile[0][t]);
                    tile[1][t] = fmaf(sv.y, bs[jj][t].x - bh[1][t], tile[1][t]);
                    tile[1][t] = fmaf(sv.y, bs[jj][t].y, tile[1][t]);
                }
            }
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int t = 0; t < GT_MR; ++t) acc[c][t].add(tile[c][t]);
        }
        __syncthreads();
    }
    if (live) {
#pragma unroll
        for (int t = 0; t < GT_MR; ++t)
            if (t < mm) {
                part[((int64_t)split * m + r0 + t) * n + i0] = acc[0][t].value();
                part[((int64_t)split * m + r0 + t) * n + i0 + 1] = acc[1][t].value();
            }
    }
}

// q[r][i] = sum_g SG[i][g] psi[r][g] - sum_split part[split][r][i]; grid (sites / NB_T, m); with p1,
// each block also writes the sum of its q values (the first pass of the neutrality fix)
constexpr int NB_T = 256;
template <typename P> struct PartSum;
template <> struct PartSum<double> { using type = PartSumD; };
template <> struct PartSum<float2> { using type = PartSumF2; };

// q = SG psi - sum of the split partials, then the neutrality fix of Sec. II.B in the last block of
// each replica: every block writes its slice of q and the slice's sum p1[r][b]; the replica's last
// block (ticket) adds the p1 in block order, applies q <- q - u (e^T q) with symm, and writes
// qtot[r] = e^T q of the result (plain FP64 sums in a fixed order: the rounding, about n eps max|q|,
// is far below the 1e-12 e the total is held to)
template <typename P>
__global__ void __launch_bounds__(NB_T) k_gemv_reduce(const P* __restrict__ part, int splits,
                                                      const double* __restrict__ SG, int ng,
                                                      const double* __restrict__ psi, int64_t n, int m,
                                                      double* __restrict__ q, double* __restrict__ p1,
                                                      const double* __restrict__ u, int symm,
                                                      int* __restrict__ tickets, double* __restrict__ qtot,
                                                      const double* __restrict__ b, const double* __restrict__ srow) {
    __shared__ double sh[NB_T / 32];
    __shared__ double buf[NB_T];
    __shared__ double s_sum;
    const int r = blockIdx.y, nb = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * NB_T + threadIdx.x;
    double* qr = q + (int64_t)r * n;
    double qi = 0.0;
    if (i < n) {
        typename PartSum<P>::type v;
        const P* pi = part + (int64_t)r * n + i;
        const int64_t stride = (int64_t)m * n;
        for (int sp = 0; sp < splits; sp += 16) {   // sixteen loads in flight, added in split order
            P x[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) x[k] = sp + k < splits ? pi[(int64_t)(sp + k) * stride] : P{};
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (sp + k < splits) v.add(x[k]);
        }
        double sv = 0.0;
        for (int g = 0; g < ng; ++g) sv += SG[i * ng + g] * psi[(int64_t)r * ng + g];
        // the centred products give sum_j S_ij (b_j - b_i): add b_i sum_j S_ij back where rows do not sum to zero
        qi = sv - (srow ? v.value() + b[(int64_t)r * n + i] * srow[i] : v.value());
        qr[i] = qi;
        __threadfence();   // this slice of q is visible device-wide before the block takes its ticket
    }
    auto block_sum = [&](double a) {   // fixed order: warp trees, then warps in order
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[warp] = a;
        __syncthreads();
        double t = 0.0;
        if (threadIdx.x == 0) {
            t = sh[0];
            for (int w = 1; w < NB_T / 32; ++w) t += sh[w];
        }
        __syncthreads();
        return t;   // valid in thread 0
    };
    const double bsum = block_sum(qi);
    if (threadIdx.x == 0) p1[(int64_t)r * nb + blockIdx.x] = bsum;
    if (!last_block_of(&tickets[r], nb)) return;
    double s = 0.0;
    if (symm) {
        const volatile double* pv = p1 + (int64_t)r * nb;
        for (int k0 = 0; k0 < nb; k0 += NB_T) {
            if (k0 + (int)threadIdx.x < nb) buf[threadIdx.x] = pv[k0 + threadIdx.x];
            __syncthreads();
            if (threadIdx.x == 0)
                for (int k = 0; k < min(NB_T, nb - k0); ++k) s += buf[k];
            __syncthreads();
        }
        if (threadIdx.x == 0) s_sum = s;
        __syncthreads();
        s = s_sum;
    }
    // the replica's q, written by the other blocks: loaded past L1 (__ldcg), eight per thread in
    // flight, fixed and summed in index order per thread
    double a = 0.0;
    for (int64_t k0 = 0; k0 < n; k0 += 8 * NB_T) {
        double v[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int64_t k = k0 + (int64_t)w * NB_T + threadIdx.x;
            v[w] = k < n ? __ldcg(qr + k) : 0.0;
        }
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int64_t k = k0 + (int64_t)w * NB_T + threadIdx.x;
            if (k < n) {
                if (symm) {
                    v[w] -= u[k] * s;
                    qr[k] = v[w];
                }
                a += v[w];
            }
        }
    }
    const double tot = block_sum(a);
    if (threadIdx.x == 0 && qtot) qtot[r] = tot;
}

__device__ __forceinline__ void neumaier_add(double& a, double& comp, double v) {
    const double t = a + v;
    comp += fabs(a) >= fabs(v) ? (a - t) + v : (v - t) + a;
    a = t;
}

// Neutrality fix and total charge, Sec. II.B (q <- q - u e^T q with u = A^-1 e / (e^T A^-1 e), then
// the FP64 total): grid (slices of the sites, m); two passes because the fix needs the replica's
// whole sum first (the first pass is k_qsum, or the GEMV reduction when it writes p1).

// p1[r][b] = sum of q[r][i] over slice b
__global__ void __launch_bounds__(NB_T) k_qsum(const double* __restrict__ q, int64_t n, double* __restrict__ p1) {
    __shared__ double sh[NB_T / 32];
    const int b = blockIdx.x, nb = gridDim.x, r = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t chunk = (n + nb - 1) / nb, ib = (int64_t)b * chunk, ie = min(n, ib + chunk);
    double s = 0.0;
    for (int64_t i = ib + threadIdx.x; i < ie; i += NB_T) s += q[(int64_t)r * n + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = sh[0];
        for (int w = 1; w < NB_T / 32; ++w) t += sh[w];
        p1[(int64_t)r * nb + b] = t;
    }
}

// with symm: q[r][i] -= u[i] * sum_b p1[r][b] (np1 block sums); then p2[r][b] = sum of the new q over
// slice b, and the replica's last block writes qtot[r] = sum of p2 in slice order (plain FP64 sums in
// a fixed order: the rounding, about n eps max|q|, is far below the 1e-12 e the total is held to)
__global__ void __launch_bounds__(NB_T) k_neutral_fix(double* __restrict__ q, const double* __restrict__ u, int64_t n,
                                                      int symm, const double* __restrict__ p1, int np1,
                                                      double* __restrict__ p2, int* __restrict__ tickets,
                                                      double* __restrict__ qtot) {
    __shared__ double sh[NB_T / 32];
    __shared__ double buf[NB_T];
    __shared__ double s_sum;
    const int b = blockIdx.x, nb = gridDim.x, r = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t chunk = (n + nb - 1) / nb, ib = (int64_t)b * chunk, ie = min(n, ib + chunk);
    double* qr = q + (int64_t)r * n;
    double s = 0.0;
    if (symm) {
        // sum of the np1 block sums in order: loaded by all threads at once, added by thread 0
        for (int k0 = 0; k0 < np1; k0 += NB_T) {
            if (k0 + (int)threadIdx.x < np1) buf[threadIdx.x] = p1[(int64_t)r * np1 + k0 + threadIdx.x];
            __syncthreads();
            if (threadIdx.x == 0)
                for (int k = 0; k < min(NB_T, np1 - k0); ++k) s += buf[k];
            __syncthreads();
        }
        if (threadIdx.x == 0) s_sum = s;
        __syncthreads();
        s = s_sum;
    }
    double a = 0.0;
    for (int64_t i = ib + threadIdx.x; i < ie; i += NB_T) {
        double v = qr[i];
        if (symm) {
            v -= u[i] * s;
            qr[i] = v;
        }
        a += v;
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = sh[0];
        for (int w = 1; w < NB_T / 32; ++w) t += sh[w];
        p2[(int64_t)r * nb + b] = t;
    }
    if (!last_block_of(&tickets[r], nb)) return;
    if (!qtot) return;
    const volatile double* pv = p2 + (int64_t)r * nb;
    if ((int)threadIdx.x < nb) buf[threadIdx.x] = pv[threadIdx.x];   // nb <= 64 slices
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < nb; ++k) t += buf[k];
        qtot[r] = t;
    }
}

static int neutral_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, (n + 1023) / 1024)); }
static int reduce_blocks(int64_t n) { return (int)((n + NB_T - 1) / NB_T); }

static cpm_status reserve_neutral(cpm_ctx* c, int m) {
    CPM_TRY(ensure_tickets(c, m));
    const size_t need = sizeof(double) * (size_t)m * (reduce_blocks(c->n) + neutral_blocks(c->n));
    if (c->nbuf_bytes >= need) return CPM_OK;
    c->graph_valid = false;
    dev_free(c, c->nbuf);
    c->nbuf = nullptr;
    c->nbuf_bytes = 0;
    CPM_TRY(dev_alloc(c, (void**)&c->nbuf, need));
    c->nbuf_bytes = need;
    return CPM_OK;
}

// have_p1: the block sums p1 were written by the GEMV reduction; else k_qsum writes them
static cpm_status launch_neutral(cpm_ctx* c, int m, double* q, double* qtot, bool have_p1) {
    CPM_TRY(reserve_neutral(c, m));
    const int nb = neutral_blocks(c->n);
    const int np1 = have_p1 ? reduce_blocks(c->n) : nb;
    double* p1 = c->nbuf;
    double* p2 = c->nbuf + (size_t)m * reduce_blocks(c->n);
    prof_begin(c, CPM_K_NEUTRAL);
    if (c->p.symm && !have_p1) {
        k_qsum<<<dim3(nb, m), NB_T, 0, c->stream>>>(q, c->n, p1);
        c->launches += 1;
    }
    k_neutral_fix<<<dim3(nb, m), NB_T, 0, c->stream>>>(q, c->u, c->n, c->p.symm, p1, np1, p2, c->tickets, qtot);
    prof_end(c, CPM_K_NEUTRAL);
    CPM_LAUNCH(c, "k_neutral_fix");
    c->launches += 1;
    return CPM_OK;
}

// split count and row chunk of the centred product; grows the scratch when needed
static bool gemv_pairs(const cpm_ctx* c) { return c->p.s_prec == CPM_PREC_FP32 && c->n % 2 == 0; }
static int64_t gemv_colblocks(const cpm_ctx* c) {
    return gemv_pairs(c) ? (c->n + 2 * G2_T - 1) / (2 * G2_T) : (c->n + GT_COLS - 1) / GT_COLS;
}

static cpm_status reserve_update_plan(cpm_ctx* c, int m, int64_t* splits_out, int64_t* jchunk_out) {
    const int64_t n = c->n;
    const int64_t colblocks = gemv_colblocks(c);
    const int rchunks = (m + GT_MR - 1) / GT_MR;
    const int64_t want = gemv_pairs(c) ? 2 * 152 : 4 * 152;   // resident blocks: about one wave
    int64_t splits = (want + colblocks * rchunks - 1) / (colblocks * rchunks);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, (n + GT_JT - 1) / GT_JT));
    int64_t jchunk = (((n + splits - 1) / splits + GT_JT - 1) / GT_JT) * GT_JT;
    splits = (n + jchunk - 1) / jchunk;
    if (gemv_tma_supported(c)) {
        int64_t cb;
        gemv_tma_plan(n, m, &cb, &splits, &jchunk);
    }
    const size_t need = ((sizeof(double) * splits * m * n + 255) & ~(size_t)255) + sizeof(float2) * m * n;
    if (c->ubuf_bytes < need) {
        dev_free(c, c->ubuf);
        c->ubuf = nullptr;
        c->ubuf_bytes = 0;
        c->graph_valid = false;
        CPM_TRY(dev_alloc(c, &c->ubuf, need));
        c->ubuf_bytes = need;
    }
    *splits_out = splits;
    *jchunk_out = jchunk;
    return CPM_OK;
}

cpm_status reserve_update(cpm_ctx* c, int m) {
    CPM_TRY(reserve_neutral(c, m));
    if (c->p.s_prec == CPM_PREC_BF16X3) return tc_reserve(c, m);
    int64_t s, j;
    return reserve_update_plan(c, m, &s, &j);
}

float2* update_bhl(cpm_ctx* c, int m) {
    if (c->p.s_prec != CPM_PREC_FP32) return nullptr;
    int64_t splits = 0, jchunk = 0;
    if (reserve_update_plan(c, m, &splits, &jchunk) != CPM_OK) return nullptr;
    return (float2*)((char*)c->ubuf + ((sizeof(double) * splits * m * c->n + 255) & ~(size_t)255));
}

cpm_status update(cpm_ctx* c, int m, const double* psi, const double* b, double* q, double* qtot, bool bhl_ready) {
    const int64_t n = c->n;
    cudaStream_t st = c->stream;
    if (c->p.s_prec == CPM_PREC_BF16X3) {
        prof_begin(c, CPM_K_GEMV);
        CPM_TRY(tc_update(c, m, psi, b, q));
        prof_end(c, CPM_K_GEMV);
        return launch_neutral(c, m, q, qtot, false);
    }
    const bool f32 = c->p.s_prec == CPM_PREC_FP32;
    int64_t splits = 0, jchunk = 0;
    CPM_TRY(reserve_update_plan(c, m, &splits, &jchunk));
    const int64_t colblocks = gemv_colblocks(c);
    const int rchunks = (m + GT_MR - 1) / GT_MR;
    double* part = (double*)c->ubuf;
    float2* bhl = (float2*)((char*)c->ubuf + ((sizeof(double) * splits * m * n + 255) & ~(size_t)255));
    bhl_ready = bhl_ready && f32;
    c->launches += (f32 && !bhl_ready) ? 3 : 2;
    // profiled stages: the split of b with the combination of b, the S stream alone, the reduction
    // of the split partial sums with the neutrality fix
    dim3 grid((unsigned)colblocks, (unsigned)splits, (unsigned)rchunks);
    if (f32) {
        if (!bhl_ready) {
            prof_begin(c, CPM_K_COMBINE);
            k_split_b<<<(unsigned)((m * n + 255) / 256), 256, 0, st>>>(b, (int64_t)m * n, bhl);
            prof_end(c, CPM_K_COMBINE);
        }
        prof_begin(c, CPM_K_GEMV);
        if (gemv_tma_supported(c)) CPM_TRY(gemv_tma(c, m, bhl, (float2*)part, splits, jchunk));
        else if (gemv_pairs(c)) k_gemv32x2<<<grid, G2_T, 0, st>>>(c->S32, bhl, n, m, jchunk, part);
        else k_gemv32<<<grid, GT_COLS, 0, st>>>(c->S32, bhl, n, m, jchunk, part);
    } else {
        prof_begin(c, CPM_K_GEMV);
        k_gemv_t<double><<<grid, GT_COLS, 0, st>>>(c->S, b, n, m, jchunk, part);
    }
    prof_end(c, CPM_K_GEMV);
    CPM_TRY(reserve_neutral(c, m));
    prof_begin(c, CPM_K_NEUTRAL);
    const dim3 rgrid((unsigned)reduce_blocks(n), m);
    const double* srow = (f32 && !c->p.symm) ? c->dvec : nullptr;
    if (f32 && gemv_tma_supported(c))
        k_gemv_reduce<float2><<<rgrid, NB_T, 0, st>>>((const float2*)part, (int)splits, upd_sg(c), upd_ng(c), psi, n, m, q,
                                                      c->nbuf, c->u, c->p.symm, c->tickets, qtot, b, srow);
    else
        k_gemv_reduce<double><<<rgrid, NB_T, 0, st>>>(part, (int)splits, upd_sg(c), upd_ng(c), psi, n, m, q, c->nbuf, c->u,
                                                      c->p.symm, c->tickets, qtot, b, srow);
    prof_end(c, CPM_K_NEUTRAL);
    CPM_LAUNCH(c, "k_gemv");
    return CPM_OK;
}

}  // namespace cpm
