// Batched charge update on the 5th-generation tensor cores:
//
//   D[i][r] = sum_j S[i][j] b[r][j]       (q_r = S G psi_r - D[:, r], Eq. electrode-wise, Sec. II.B)
//
// for m replicas sharing one capacitance matrix S.  Both operands are split into three bf16
// terms, S = S0 + S1 + S2 and b = B0 + B1 + B2 (24 significant bits each), and the six
// products of combined order <= 2 (S0B0, S0B1, S1B0, S0B2, S1B1, S2B0) are accumulated in
// FP32 in tensor memory, which keeps the single-precision accuracy of S.
//
// One CTA computes a 128-row x BN-replica tile over one K range: TMA loads the six operand
// tiles of a 64-wide K step into 128-byte-swizzled shared memory, one thread issues the
// tcgen05.mma instructions, the accumulator lives in TMEM and four warps read it back with
// tcgen05.ld.  Partial sums of the K ranges are added in FP64 by the reduction kernel.
// Every mbarrier wait is bounded: on expiry the CTA records a timeout in the status word,
// lets its copies in flight land, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpm {

constexpr int TC_BM = 128;          // rows of S per CTA (MMA M)
constexpr int TC_BK = 64;           // K elements per stage (128 bytes of bf16 per row)
constexpr int TC_THREADS = 128;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;   // bound on any single mbarrier wait: 2 s

template <int BN> struct TcCfg {
    static constexpr int A_BYTES = TC_BM * 128;            // one bf16 split of the S tile
    static constexpr int B_BYTES = BN * 128;               // one bf16 split of the b tile
    static constexpr int STAGE = 3 * A_BYTES + 3 * B_BYTES;
    static constexpr int STAGES = (220 * 1024) / STAGE >= 4 ? 4 : (220 * 1024) / STAGE;
    static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
    static constexpr int SMEM = 1024 + STAGES * STAGE + 256;
};

struct TcMaps {
    CUtensorMap a[3];
    CUtensorMap b[3];
};

template <int BN>
// skip_loads = 1 issues no TMA copies at all: every wait must then run out (the failure-detection
// self test); it is never set on the compute path.
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_sb(const __grid_constant__ TcMaps maps, int n, int m,
                                                         int kchunk, float* __restrict__ part,
                                                         unsigned* __restrict__ status, int skip_loads,
                                                         uint64_t wait_ns) {
    typedef TcCfg<BN> C;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE);
    uint64_t* empty = full + C::STAGES;
    uint64_t* done = empty + C::STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * TC_BM, r0 = blockIdx.y * BN;
    const int kb = blockIdx.z * kchunk;
    const int nsteps = kchunk / TC_BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(done, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: six TMA tiles per K step
        int issued = 0, waited_free = 0;
        for (int t = 0; t < nsteps; ++t) {
            const int s = t % C::STAGES;
            if (skip_loads) break;
            if (t >= C::STAGES) {
                if (!mbar_wait(&empty[s], ((t / C::STAGES) - 1) & 1, abort, wait_ns)) break;
                ++waited_free;
            }
            uint8_t* st = smem + s * C::STAGE;
            mbar_expect_tx(&full[s], C::STAGE);
            const int kx = kb + t * TC_BK;
            for (int q = 0; q < 3; ++q) tma_load_2d(st + q * C::A_BYTES, &maps.a[q], kx, i0, &full[s]);
            for (int q = 0; q < 3; ++q) tma_load_2d(st + 3 * C::A_BYTES + q * C::B_BYTES, &maps.b[q], kx, r0, &full[s]);
            ++issued;
        }
        if (*abort) {
            // let the copies already issued land before the CTA exits (bounded)
            for (int t = 0; t < issued; ++t) {
                const int s = t % C::STAGES;
                const uint64_t t0 = gtimer_ns();
                while (!mbar_try(&full[s], (t / C::STAGES) & 1) && gtimer_ns() - t0 < wait_ns) {}
            }
        }
        (void)waited_free;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_bf16(TC_BM, BN);
        const int pa[6] = {0, 0, 1, 0, 1, 2};
        const int pb[6] = {0, 1, 0, 2, 1, 0};
        bool ok = true;
        for (int t = 0; t < nsteps; ++t) {
            const int s = t % C::STAGES;
            if (!mbar_wait(&full[s], (t / C::STAGES) & 1, abort, wait_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = su32(smem + s * C::STAGE);
            const uint32_t sb = sa + 3 * C::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint64_t ad = sdesc_sw128(sa + pa[p] * C::A_BYTES + kk * 32);
                    const uint64_t bd = sdesc_sw128(sb + pb[p] * C::B_BYTES + kk * 32);
                    umma_f16(tmem, ad, bd, idesc, (t > 0 || kk > 0 || p > 0) ? 1u : 0u);
                }
            }
            umma_commit(&empty[s]);
        }
        if (ok) umma_commit(done);
    }
    // epilogue: every thread owns one row of the 128-row tile
    __syncwarp();
    const bool have = __all_sync(0xffffffffu, mbar_wait(done, 0, abort, wait_ns) ? 1 : 0) != 0;
    tc_fence_after();
    if (have) {
        const int i = i0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(trow + c0, v);
            if (i < n) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int r = r0 + c0 + k;
                    if (r < m) part[((int64_t)blockIdx.z * m + r) * n + i] = v[k];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(status, ST_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
}

// ----------------------------------------------------------------------------- operand splits
// x = x0 + x1 + x2 with bf16 terms: x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1).
// With `gmean`, row r is first centred by its group means: x[r][c] - gmean[r][gid[c]].
__global__ void k_split3(const double* __restrict__ x, int64_t rows, int64_t cols, int64_t ld,
                         __nv_bfloat16* __restrict__ out, const double* __restrict__ gmean = nullptr,
                         const int* __restrict__ gid = nullptr, int ngrp = 0) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * ld) return;
    const int64_t r = t / ld, c = t % ld;
    double v = c < cols ? x[r * cols + c] : 0.0;
    if (gmean && c < cols) v -= gmean[r * ngrp + gid[c]];
    __nv_bfloat16 h0 = __double2bfloat16(v);
    double r1 = v - (double)__bfloat162float(h0);
    __nv_bfloat16 h1 = __double2bfloat16(r1);
    double r2 = r1 - (double)__bfloat162float(h1);
    __nv_bfloat16 h2 = __double2bfloat16(r2);
    const int64_t plane = rows * ld;
    out[t] = h0;
    out[plane + t] = h1;
    out[2 * plane + t] = h2;
}

// ----------------------------------------------------------------------------- host side
int64_t tc_ld(int64_t n) { return ((n + TC_BK - 1) / TC_BK) * TC_BK; }

// S (FP64, n x n) -> three bf16 planes [3][n][ld] in c->Sb
cpm_status tc_prepare_s(cpm_ctx* c) {
    const int64_t n = c->n, ld = tc_ld(n);
    dev_free(c, c->Sb);
    c->Sb = nullptr;
    CPM_TRY(dev_alloc(c, (void**)&c->Sb, sizeof(__nv_bfloat16) * 3 * n * ld));
    k_split3<<<(unsigned)((n * ld + 255) / 256), 256, 0, c->stream>>>(c->S, n, n, ld, (__nv_bfloat16*)c->Sb);
    CPM_LAUNCH(c, "k_split3(S)");
    return CPM_OK;
}

template <int BN>
static cpm_status launch_tc(cpm_ctx* c, const TcMaps& maps, int n, int m, int64_t ld, float* part, int* splits_out,
                           int skip_loads = 0, uint64_t wait_ns = TC_WAIT_NS) {
    typedef TcCfg<BN> C;
    const int mt = (n + TC_BM - 1) / TC_BM, nt = (m + BN - 1) / BN;
    const int ksteps = (int)(ld / TC_BK);
    // about one wave of CTAs (one per SM): longer K ranges per CTA keep the TMA/MMA pipeline full
    int splits = std::max(1, std::min(ksteps, 152 / (mt * nt)));
    const int kchunk_steps = (ksteps + splits - 1) / splits;
    splits = (ksteps + kchunk_steps - 1) / kchunk_steps;
    CPM_CUDA(c, cudaFuncSetAttribute(k_tc_sb<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    k_tc_sb<BN><<<dim3(mt, nt, splits), TC_THREADS, C::SMEM, c->stream>>>(maps, n, m, kchunk_steps * TC_BK, part,
                                                                          c->status, skip_loads, wait_ns);
    CPM_LAUNCH(c, "k_tc_sb");
    *splits_out = splits;
    return CPM_OK;
}

// part[split][r][i] = sum over the split's K range of S[i][j] b[r][j]; returns the split count
cpm_status tc_sb(cpm_ctx* c, int m, const double* b, float* part, int* splits, void* bsplit, const double* gmean,
                 const int* gid, int ngrp) {
    const int64_t n = c->n, ld = tc_ld(n);
    k_split3<<<(unsigned)((m * ld + 255) / 256), 256, 0, c->stream>>>(b, m, n, ld, (__nv_bfloat16*)bsplit, gmean, gid,
                                                                      ngrp);
    CPM_LAUNCH(c, "k_split3(b)");
    const int BN = m <= 32 ? 32 : (m <= 64 ? 64 : 128);
    TcMaps maps;
    const __nv_bfloat16* Sb = (const __nv_bfloat16*)c->Sb;
    const __nv_bfloat16* Bb = (const __nv_bfloat16*)bsplit;
    for (int q = 0; q < 3; ++q) {
        if (!make_map(&maps.a[q], Sb + (size_t)q * n * ld, n, ld, TC_BM) ||
            !make_map(&maps.b[q], Bb + (size_t)q * m * ld, m, ld, BN))
            return set_err(c, CPM_E_CUDA, "cuTensorMapEncodeTiled failed");
    }
    if (BN == 32) return launch_tc<32>(c, maps, (int)n, m, ld, part, splits);
    if (BN == 64) return launch_tc<64>(c, maps, (int)n, m, ld, part, splits);
    return launch_tc<128>(c, maps, (int)n, m, ld, part, splits);
}

size_t tc_part_bytes(int64_t n, int m);
size_t tc_bsplit_bytes(int64_t n, int m);
cpm_status tc_sb(cpm_ctx* c, int m, const double* b, float* part, int* splits, void* bsplit, const double* gmean,
                 const int* gid, int ngrp);

// Layer groups for centring: the distinct site heights when there are at most 64 of them
// (layered electrodes), else the electrodes themselves.
// SZ[i][g] = sum over sites j of group g of S[i][j] (FP64), one thread per (i, g).
__global__ void k_sgroups(const double* __restrict__ S, const int* __restrict__ gid, int64_t n, int ngrp,
                          double* __restrict__ SZ) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * ngrp) return;
    const int64_t i = t / ngrp;
    const int g = (int)(t % ngrp);
    double a = 0.0;
    for (int64_t j = 0; j < n; ++j)
        if (gid[j] == g) a += S[i * n + j];
    SZ[t] = a;
}

// gmean[r][g] = mean of b[r][i] over the sites of group g; one warp per (r, g), fixed order
__global__ void k_gmeans(const double* __restrict__ b, const int* __restrict__ gid, int64_t n, int m, int ngrp,
                         double* __restrict__ gmean) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)m * ngrp) return;
    const int r = (int)(w / ngrp), g = (int)(w % ngrp);
    double a = 0.0;
    int cnt = 0;
    for (int64_t i = lane; i < n; i += 32)
        if (gid[i] == g) { a += b[(int64_t)r * n + i]; ++cnt; }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) gmean[w] = cnt ? a / cnt : 0.0;
}

// q[r][i] = sum_g SG[i][g] psi[r][g] - sum_g' SZ[i][g'] gmean[r][g'] - sum_split part[split][r][i]
__global__ void k_tc_reduce(const float* __restrict__ part, int splits, const double* __restrict__ SG, int ng,
                            const double* __restrict__ psi, const double* __restrict__ SZ,
                            const double* __restrict__ gmean, int ngrp, int64_t n, int m, double* __restrict__ q) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * n) return;
    const int r = (int)(t / n);
    const int64_t i = t % n;
    double v = 0.0;
    for (int sp = 0; sp < splits; ++sp) v += (double)part[((int64_t)sp * m + r) * n + i];
    for (int g = 0; g < ngrp; ++g) v += SZ[i * ngrp + g] * gmean[(int64_t)r * ngrp + g];
    double sv = 0.0;
    for (int g = 0; g < ng; ++g) sv += SG[i * ng + g] * psi[(int64_t)r * ng + g];
    q[t] = sv - v;
}

cpm_status tc_reserve(cpm_ctx* c, int m) {
    const int64_t n = c->n;
    if (!c->Sb) {
        c->graph_valid = false;
        CPM_TRY(tc_prepare_s(c));
        // centring groups and their responses S G_z
        c->tc_use_z = c->nzu <= 64;
        c->tc_ngrp = c->tc_use_z ? c->nzu : c->ng;
        dev_free(c, c->SZ);
        c->SZ = nullptr;
        CPM_TRY(dev_alloc(c, (void**)&c->SZ, sizeof(double) * n * c->tc_ngrp));
        const int* gid = c->tc_use_z ? c->zmap : c->group;
        k_sgroups<<<(unsigned)((n * c->tc_ngrp + 255) / 256), 256, 0, c->stream>>>(c->S, gid, n, c->tc_ngrp, c->SZ);
        CPM_LAUNCH(c, "k_sgroups");
    }
    const size_t pb = (tc_part_bytes(n, m) + 255) & ~(size_t)255;
    const size_t need = pb + tc_bsplit_bytes(n, m) + 256 + sizeof(double) * (size_t)m * c->tc_ngrp;
    if (c->tbuf_bytes < need) {
        dev_free(c, c->tbuf);
        c->tbuf = nullptr;
        c->tbuf_bytes = 0;
        c->graph_valid = false;
        CPM_TRY(dev_alloc(c, &c->tbuf, need));
        c->tbuf_bytes = need;
    }
    return CPM_OK;
}

cpm_status tc_update(cpm_ctx* c, int m, const double* psi, const double* b, double* q) {
    const int64_t n = c->n;
    CPM_TRY(tc_reserve(c, m));
    const size_t pb = (tc_part_bytes(n, m) + 255) & ~(size_t)255;
    float* part = (float*)c->tbuf;
    void* bsplit = (char*)c->tbuf + pb;
    double* gmean = (double*)((char*)bsplit + ((tc_bsplit_bytes(n, m) + 255) & ~(size_t)255));
    const int* gid = c->tc_use_z ? c->zmap : c->group;
    k_gmeans<<<(unsigned)(((int64_t)m * c->tc_ngrp * 32 + 255) / 256), 256, 0, c->stream>>>(b, gid, n, m, c->tc_ngrp,
                                                                                              gmean);
    CPM_LAUNCH(c, "k_gmeans");
    int splits = 0;
    CPM_TRY(tc_sb(c, m, b, part, &splits, bsplit, gmean, gid, c->tc_ngrp));
    k_tc_reduce<<<(unsigned)((m * n + 255) / 256), 256, 0, c->stream>>>(part, splits, c->SG, c->ng, psi, c->SZ, gmean,
                                                                        c->tc_ngrp, n, m, q);
    CPM_LAUNCH(c, "k_tc_reduce");
    c->launches += 4;
    return CPM_OK;
}

// Failure-detection self test: one tensor-core launch that issues no loads, so its first wait
// runs out after wait_ms; the CTA must record ST_TIMEOUT, free its TMEM and return.
cpm_status tc_selftest_timeout(cpm_ctx* c, double wait_ms) {
    const int m = 32;
    CPM_TRY(tc_reserve(c, m));
    const int64_t n = c->n, ld = tc_ld(n);
    TcMaps maps;
    const __nv_bfloat16* Sb = (const __nv_bfloat16*)c->Sb;
    const size_t pb = (tc_part_bytes(n, m) + 255) & ~(size_t)255;
    const __nv_bfloat16* Bb = (const __nv_bfloat16*)((char*)c->tbuf + pb);
    for (int q = 0; q < 3; ++q) {
        if (!make_map(&maps.a[q], Sb + (size_t)q * n * ld, n, ld, TC_BM) ||
            !make_map(&maps.b[q], Bb + (size_t)q * m * ld, m, ld, 32))
            return set_err(c, CPM_E_CUDA, "cuTensorMapEncodeTiled failed");
    }
    int splits = 0;
    return launch_tc<32>(c, maps, (int)n, m, ld, (float*)c->tbuf, &splits, 1, (uint64_t)(wait_ms * 1e6));
}

size_t tc_part_bytes(int64_t n, int m) {
    const int64_t ksteps = tc_ld(n) / TC_BK;
    return sizeof(float) * (size_t)std::min<int64_t>(ksteps, 2 * 152) * m * n;
}
size_t tc_bsplit_bytes(int64_t n, int m) { return sizeof(__nv_bfloat16) * 3 * (size_t)m * tc_ld(n); }

}  // namespace cpm
