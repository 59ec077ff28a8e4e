// Charge update q = S G psi - S b for m replicas with the single-precision capacitance matrix
// (Sec. II.B), streaming S once per eight replicas.  A block owns 512 consecutive columns i and a
// range of rows j (a split); every consumer thread owns four adjacent columns i0 .. i0 + 3 and
// centres b on beta = bh_i0 (b = bh + bl split into two floats):
//
//   part[split][r][i] = sum_j S_ij d_j  -  (b_i - beta) sum_j S_ij,   d_j = (bh_j - beta) + bl_j,
//
// over the split's rows j.  This equals sum_j S_ij (b_j - b_i) for any matrix, and the rows of the
// exact S sum to zero (Eq. S), so the result is the S b of the method; centring on a site next to
// i keeps the large common part of b out of the single-precision sums, and the row sums are taken
// over the stored single-precision S so the identity holds for the stored values too.  d_j is formed
// once per row and replica and serves the thread's four columns: 1.5 FP32 operations per (i, j, r)
// plus one row-sum addition per (i, j).
//
// One producer thread streams S through a three-stage shared-memory ring with TMA (16 rows x 512
// columns per stage, 32 KB; two blocks per SM); 128 consumer threads read their four columns of a
// row with one 16-byte shared load and evaluate the eight replicas as four packed pairs
// (fma.rn.f32x2), summing each stage plainly in FP32 and adding the stage sums with compensation
// (packed Kahan).  The (b_i - beta) row-sum term is applied in double-float arithmetic, and the
// result leaves as an FP32 pair (high, low) per replica and column that the reduction over the
// splits adds in double-float arithmetic, so no FP64 instruction runs in this kernel.
// Every mbarrier wait is bounded by wall time; on expiry the block records ST_TIMEOUT, lets its
// copies in flight land and returns.
#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpm {

constexpr int GV_T = 128;                      // consumer threads
constexpr int GV_CPT = 4;                      // adjacent columns per consumer thread
constexpr int GV_BC = GV_CPT * GV_T;           // columns per block (two TMA boxes of 256)
constexpr int GV_RJ = 16;                      // rows of S per stage
constexpr int GV_STAGES = 3;                   // per block; two blocks per SM
constexpr int GV_STAGE_BYTES = GV_RJ * GV_BC * 4;
constexpr int GV_JMAX = 192;                   // rows of b staged per block
constexpr int GV_MR = 8;                       // replicas per block
constexpr int GV_SPT = (GV_JMAX * GV_MR + GV_T - 1) / GV_T;   // staged entries per consumer thread
constexpr int GV_SMEM = 1024 + GV_STAGES * GV_STAGE_BYTES + GV_JMAX * 2 * GV_MR * 4 + 256;
constexpr uint64_t GV_WAIT_NS = 2000000000ull;

// compensated sum of packed pairs (Kahan): the sum is s - c; every step is one rounding
struct Kahan2 {
    uint64_t s = 0ull, c = 0ull;
    __device__ __forceinline__ void add(uint64_t x) {
        const uint64_t y = sub2(x, c), t = add2(s, y);
        c = sub2(sub2(t, s), y);
        s = t;
    }
};

// double-float helpers (value = hi + lo): exact sum and difference (Knuth's two-sum) and a product
// with the rounding error of the leading term recovered by an FMA
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_norm(float hi, float lo) {
    const float s = __fadd_rn(hi, lo);
    return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);
    return df_norm(p, __fadd_rn(e, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi))));
}
__device__ __forceinline__ DF df_sub(DF a, DF b) {
    const DF s = two_sum(a.hi, -b.hi);
    return df_norm(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}

// grid (column blocks, splits, replica chunks of eight)
__global__ void __launch_bounds__(GV_T + 32, 2)
    k_gemv_tma(const __grid_constant__ CUtensorMap smap, const float2* __restrict__ bv, int64_t n, int m,
               int64_t jchunk, float2* __restrict__ part, unsigned* __restrict__ status, uint64_t wait_ns) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
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

    // consumers: stage b of the block's rows, replica-minor, high and low parts apart (coalesced
    // loads along the rows, all in flight before the first store)
    const int64_t ic = i0 + GV_CPT * tid;
    const bool live = ic < n;   // n is a multiple of 4: a thread's columns are all in range or all out
    {
        float2 v[GV_SPT];
#pragma unroll
        for (int k = 0; k < GV_SPT; ++k) {
            const int e = tid + GV_T * k, t = e / GV_JMAX, jj = e % GV_JMAX;
            v[k] = (t < mm && jj < nrow) ? bv[(int64_t)(r0 + t) * n + jb + jj] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < GV_SPT; ++k) {
            const int e = tid + GV_T * k, t = e / GV_JMAX, jj = e % GV_JMAX;
            if (t < GV_MR) {
                shi[jj * GV_MR + t] = v[k].x;
                slo[jj * GV_MR + t] = v[k].y;
            }
        }
    }
    // beta_r = bh of this thread's first column, as replica pairs
    uint64_t beta[GV_MR / 2];
#pragma unroll
    for (int h = 0; h < GV_MR / 2; ++h) {
        const int ta = 2 * h, tb = 2 * h + 1;
        beta[h] = pk2((ta < mm && live) ? bv[(int64_t)(r0 + ta) * n + ic].x : 0.f,
                      (tb < mm && live) ? bv[(int64_t)(r0 + tb) * n + ic].x : 0.f);
    }
    asm volatile("bar.sync 1, %0;" ::"n"(GV_T) : "memory");
    Kahan2 acc[GV_CPT][GV_MR / 2], rsum[GV_CPT / 2];
    // this thread's 16-byte run of a staged row: box (4 tid) / 256, offset (4 tid) % 256
    const uint32_t col_off = (uint32_t)((GV_CPT * tid / 256) * (GV_STAGE_BYTES / 2) + (GV_CPT * tid % 256) * 4);
    bool ok = true;
    for (int t = 0; t < nst; ++t) {
        const int s = t % GV_STAGES;
        if (!mbar_wait(&full[s], (t / GV_STAGES) & 1, abort, wait_ns)) { ok = false; break; }
        const uint8_t* st = smem + s * GV_STAGE_BYTES + col_off;
        const int rows = min(GV_RJ, nrow - t * GV_RJ);
        uint64_t tile[GV_CPT][GV_MR / 2], rs[GV_CPT / 2] = {0ull, 0ull};
#pragma unroll
        for (int c = 0; c < GV_CPT; ++c)
#pragma unroll
            for (int h = 0; h < GV_MR / 2; ++h) tile[c][h] = 0ull;
#pragma unroll 2
        for (int u = 0; u < rows; ++u) {
            const float4 s4 = *reinterpret_cast<const float4*>(st + u * 256 * 4);   // S_j,i0 .. S_j,i0+3
            const int jj = t * GV_RJ + u;
            const float4 h0 = *reinterpret_cast<const float4*>(shi + jj * GV_MR);
            const float4 h1 = *reinterpret_cast<const float4*>(shi + jj * GV_MR + 4);
            const float4 l0 = *reinterpret_cast<const float4*>(slo + jj * GV_MR);
            const float4 l1 = *reinterpret_cast<const float4*>(slo + jj * GV_MR + 4);
            const uint64_t hp[4] = {pk2(h0.x, h0.y), pk2(h0.z, h0.w), pk2(h1.x, h1.y), pk2(h1.z, h1.w)};
            const uint64_t lp[4] = {pk2(l0.x, l0.y), pk2(l0.z, l0.w), pk2(l1.x, l1.y), pk2(l1.z, l1.w)};
            uint64_t d[GV_MR / 2];
#pragma unroll
            for (int h = 0; h < GV_MR / 2; ++h) d[h] = add2(sub2(hp[h], beta[h]), lp[h]);
            const float sc[GV_CPT] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int c = 0; c < GV_CPT; ++c) {
                const uint64_t sp = pk2(sc[c], sc[c]);
#pragma unroll
                for (int h = 0; h < GV_MR / 2; ++h) tile[c][h] = fma2(sp, d[h], tile[c][h]);
            }
            rs[0] = add2(rs[0], pk2(s4.x, s4.y));
            rs[1] = add2(rs[1], pk2(s4.z, s4.w));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
        for (int c = 0; c < GV_CPT; ++c)
#pragma unroll
            for (int h = 0; h < GV_MR / 2; ++h) acc[c][h].add(tile[c][h]);
        rsum[0].add(rs[0]);
        rsum[1].add(rs[1]);
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, ST_TIMEOUT);
        return;
    }
    if (!live) return;
    // row sums of the four columns and the sums of the products, as double-float values
    DF rsc[GV_CPT];
    {
        const float2 s01 = up2(rsum[0].s), c01 = up2(rsum[0].c), s23 = up2(rsum[1].s), c23 = up2(rsum[1].c);
        rsc[0] = df_norm(s01.x, -c01.x);
        rsc[1] = df_norm(s01.y, -c01.y);
        rsc[2] = df_norm(s23.x, -c23.x);
        rsc[3] = df_norm(s23.y, -c23.y);
    }
#pragma unroll
    for (int t = 0; t < GV_MR; ++t) {
        if (t >= mm) continue;
        const float2* br = bv + (int64_t)(r0 + t) * n + ic;
        const float bt = br[0].x;   // beta_t
        float2 o[GV_CPT];
#pragma unroll
        for (int c = 0; c < GV_CPT; ++c) {
            const float2 as = up2(acc[c][t / 2].s), ac = up2(acc[c][t / 2].c);
            const DF a = df_norm((t & 1) ? as.y : as.x, -((t & 1) ? ac.y : ac.x));
            const float2 bi = br[c];
            const DF e0 = two_sum(bi.x, -bt);                          // bh_i - beta, exactly
            const DF e = df_norm(e0.hi, __fadd_rn(e0.lo, bi.y));      // (b_i - beta)
            const DF r = df_sub(a, df_mul(e, rsc[c]));
            o[c] = make_float2(r.hi, r.lo);
        }
        float4* pr = reinterpret_cast<float4*>(part + ((int64_t)split * m + r0 + t) * n + ic);   // 32-byte aligned
        pr[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        pr[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
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

cpm_status gemv_tma(cpm_ctx* c, int m, const float2* bhl, float2* part, int64_t splits, int64_t jchunk) {
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
