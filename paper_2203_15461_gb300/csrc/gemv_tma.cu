// Charge update q = S G psi - S b for m replicas with the single-precision capacitance matrix
// (Sec. II.B), streaming S once per eight replicas:
//
//   part[split][r][i] = sum over the split's rows j of S_ij ((bh_j - bh_i) + bl_j)
//
// with b = bh + bl split into two floats (the centred form is exact because the rows of S sum to
// zero, Eq. S; it keeps the large common part of b out of the single-precision sums).
//
// A block owns 512 consecutive columns i and a range of rows j.  One producer thread streams S
// through a two-stage shared-memory ring with TMA (16 rows x 512 columns per stage, 32 KB; two blocks
// per SM); the
// 256 consumer threads take two columns each and evaluate the eight replicas as four packed pairs
// (fma.rn.f32x2), summing each stage plainly in FP32 and adding the stage sums with compensation.
// Every mbarrier wait is bounded by wall time; on expiry the block records ST_TIMEOUT, lets its
// copies in flight land and returns.
#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpm {

constexpr int GV_T = 256;                      // consumer threads (two columns each)
constexpr int GV_BC = 2 * GV_T;                // columns per block
constexpr int GV_RJ = 16;                      // rows of S per stage
constexpr int GV_STAGES = 2;                   // per block; two blocks per SM
constexpr int GV_STAGE_BYTES = GV_RJ * GV_BC * 4;
constexpr int GV_JMAX = 256;                   // rows of b staged per block
constexpr int GV_MR = 8;                       // replicas per block
constexpr int GV_SMEM = 1024 + GV_STAGES * GV_STAGE_BYTES + GV_JMAX * 2 * GV_MR * 4 + 256;
constexpr uint64_t GV_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up2(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c, t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// grid (column blocks, splits, replica chunks of eight)
__global__ void __launch_bounds__(GV_T + 32, 2)
    k_gemv_tma(const __grid_constant__ CUtensorMap smap, const float2* __restrict__ bv, int64_t n, int m,
               int64_t jchunk, double* __restrict__ part, unsigned* __restrict__ status, uint64_t wait_ns) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float* shi = (float*)(smem + GV_STAGES * GV_STAGE_BYTES);   // [jj][8] high parts of b
    float* slo = shi + GV_JMAX * GV_MR;                          // [jj][8] low parts
    uint64_t* full = (uint64_t*)(slo + GV_JMAX * GV_MR);
    uint64_t* empty = full + GV_STAGES;
    volatile int* abort = (volatile int*)(empty + GV_STAGES);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t i0 = (int64_t)blockIdx.x * GV_BC;
    const int split = blockIdx.y, r0 = blockIdx.z * GV_MR;
    const int mm = min(GV_MR, m - r0);
    const int64_t jb = (int64_t)split * jchunk, je = min(n, jb + jchunk);
    const int nrow = (int)max((int64_t)0, je - jb);
    const int nst = (nrow + GV_RJ - 1) / GV_RJ;

    if (tid == 0) {
        for (int s = 0; s < GV_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], GV_T / 32); }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (warp == GV_T / 32) {
        // producer
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nst; ++t) {
                const int s = t % GV_STAGES;
                if (t >= GV_STAGES && !mbar_wait(&empty[s], ((t / GV_STAGES) - 1) & 1, abort, wait_ns)) break;
                uint8_t* st = smem + s * GV_STAGE_BYTES;
                mbar_expect_tx(&full[s], GV_STAGE_BYTES);
                const int y = (int)(jb + (int64_t)t * GV_RJ);
                tma_load_2d(st, &smap, (int)i0, y, &full[s]);
                tma_load_2d(st + GV_STAGE_BYTES / 2, &smap, (int)i0 + GV_BC / 2, y, &full[s]);
                ++issued;
            }
            if (*abort) {
                for (int t = 0; t < issued; ++t) {   // let the copies already issued land (bounded)
                    const int s = t % GV_STAGES;
                    const uint64_t ts = gtimer_ns();
                    while (!mbar_try(&full[s], (t / GV_STAGES) & 1) && gtimer_ns() - ts < wait_ns) {}
                }
            }
        }
        return;
    }

    // consumers: stage b of the block's rows, replica-minor, high and low parts apart
    for (int e = tid; e < nrow * GV_MR; e += GV_T) {
        const int jj = e / GV_MR, t = e % GV_MR;
        const float2 v = t < mm ? bv[(int64_t)(r0 + t) * n + jb + jj] : make_float2(0.f, 0.f);
        shi[e] = v.x;
        slo[e] = v.y;
    }
    const int64_t ic = i0 + 2 * tid;
    const bool live0 = ic < n, live1 = ic + 1 < n;
    uint64_t bh[2][GV_MR / 2];
#pragma unroll
    for (int tp = 0; tp < GV_MR / 2; ++tp) {
        const int ta = 2 * tp, tb = 2 * tp + 1;
        bh[0][tp] = pk2((ta < mm && live0) ? bv[(int64_t)(r0 + ta) * n + ic].x : 0.f,
                        (tb < mm && live0) ? bv[(int64_t)(r0 + tb) * n + ic].x : 0.f);
        bh[1][tp] = pk2((ta < mm && live1) ? bv[(int64_t)(r0 + ta) * n + ic + 1].x : 0.f,
                        (tb < mm && live1) ? bv[(int64_t)(r0 + tb) * n + ic + 1].x : 0.f);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(GV_T) : "memory");
    Kahan acc[2][GV_MR];
    const uint32_t col_off = (uint32_t)((tid / (GV_T / 2)) * (GV_STAGE_BYTES / 2) + (2 * tid % (GV_BC / 2)) * 4);
    bool ok = true;
    for (int t = 0; t < nst; ++t) {
        const int s = t % GV_STAGES;
        if (!mbar_wait(&full[s], (t / GV_STAGES) & 1, abort, wait_ns)) { ok = false; break; }
        const uint8_t* st = smem + s * GV_STAGE_BYTES + col_off;
        const int rows = min(GV_RJ, nrow - t * GV_RJ);
        uint64_t tile[2][GV_MR / 2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int tp = 0; tp < GV_MR / 2; ++tp) tile[c][tp] = 0ull;
#pragma unroll 4
        for (int u = 0; u < rows; ++u) {
            const float2 sv = *reinterpret_cast<const float2*>(st + u * (GV_BC / 2) * 4);
            const int jj = t * GV_RJ + u;
            const float4 h0 = *reinterpret_cast<const float4*>(shi + jj * GV_MR);
            const float4 h1 = *reinterpret_cast<const float4*>(shi + jj * GV_MR + 4);
            const float4 l0 = *reinterpret_cast<const float4*>(slo + jj * GV_MR);
            const float4 l1 = *reinterpret_cast<const float4*>(slo + jj * GV_MR + 4);
            const uint64_t hp[4] = {pk2(h0.x, h0.y), pk2(h0.z, h0.w), pk2(h1.x, h1.y), pk2(h1.z, h1.w)};
            const uint64_t lp[4] = {pk2(l0.x, l0.y), pk2(l0.z, l0.w), pk2(l1.x, l1.y), pk2(l1.z, l1.w)};
            const uint64_t s0 = pk2(sv.x, sv.x), s1 = pk2(sv.y, sv.y);
#pragma unroll
            for (int tp = 0; tp < GV_MR / 2; ++tp) {
                tile[0][tp] = fma2(s0, sub2(hp[tp], bh[0][tp]), tile[0][tp]);
                tile[0][tp] = fma2(s0, lp[tp], tile[0][tp]);
                tile[1][tp] = fma2(s1, sub2(hp[tp], bh[1][tp]), tile[1][tp]);
                tile[1][tp] = fma2(s1, lp[tp], tile[1][tp]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int tp = 0; tp < GV_MR / 2; ++tp) {
                const float2 v = up2(tile[c][tp]);
                acc[c][2 * tp].add(v.x);
                acc[c][2 * tp + 1].add(v.y);
            }
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, ST_TIMEOUT);
        return;
    }
#pragma unroll
    for (int t = 0; t < GV_MR; ++t) {
        if (t >= mm) continue;
        double* pr = part + ((int64_t)split * m + r0 + t) * n;
        if (live0) pr[ic] = (double)acc[0][t].s - (double)acc[0][t].c;
        if (live1) pr[ic + 1] = (double)acc[1][t].s - (double)acc[1][t].c;
    }
}

bool gemv_tma_supported(const cpm_ctx* c) { return c->p.s_prec == CPM_PREC_FP32 && c->n % 4 == 0 && c->n >= 256; }

void gemv_tma_plan(int64_t n, int m, int64_t* colblocks, int64_t* splits, int64_t* jchunk) {
    *colblocks = (n + GV_BC - 1) / GV_BC;
    const int64_t rchunks = (m + GV_MR - 1) / GV_MR;
    // one wave: two blocks per SM
    int64_t sp = std::max<int64_t>(1, 2 * 152 / (*colblocks * rchunks));
    sp = std::max<int64_t>(sp, (n + GV_JMAX - 1) / GV_JMAX);
    int64_t jc = (n + sp - 1) / sp;
    jc = ((jc + GV_RJ - 1) / GV_RJ) * GV_RJ;
    *jchunk = std::min<int64_t>(jc, GV_JMAX);
    *splits = (n + *jchunk - 1) / *jchunk;
}

cpm_status gemv_tma(cpm_ctx* c, int m, const float2* bhl, double* part, int64_t splits, int64_t jchunk) {
    const int64_t n = c->n;
    auto enc = encode_fn();
    if (!enc) return set_err(c, CPM_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    CUtensorMap smap;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(n * 4)};
    cuuint32_t box[2] = {(cuuint32_t)(GV_BC / 2), (cuuint32_t)GV_RJ};
    cuuint32_t estr[2] = {1, 1};
    if (enc(&smap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)c->S32, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_err(c, CPM_E_CUDA, "cuTensorMapEncodeTiled failed");
    int64_t colblocks, sp, jc;
    gemv_tma_plan(n, m, &colblocks, &sp, &jc);
    if (sp != splits || jc != jchunk) return set_err(c, CPM_E_STATE, "gemv_tma: plan mismatch");
    CPM_CUDA(c, cudaFuncSetAttribute(k_gemv_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, GV_SMEM));
    const dim3 grid((unsigned)colblocks, (unsigned)splits, (unsigned)((m + GV_MR - 1) / GV_MR));
    k_gemv_tma<<<grid, GV_T + 32, GV_SMEM, c->stream>>>(smap, bhl, n, m, jchunk, part, c->status, GV_WAIT_NS);
    CPM_LAUNCH(c, "k_gemv_tma");
    return CPM_OK;
}

}  // namespace cpm
