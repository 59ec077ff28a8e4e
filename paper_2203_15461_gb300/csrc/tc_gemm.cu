// Batched charge update on the 5th-generation tensor cores:
//
//   D[i][r] = sum_j S[i][j] b[r][j]       (q_r = S G psi_r - D[:, r], Eq. electrode-wise, Sec. II.B)
//
// for m replicas sharing one capacitance matrix S.  Both operands are split into three bf16
// terms, S = S0 + S1 + S2 and b = B0 + B1 + B2 (24 significant bits each), and the six
// products of combined order <= 2 (S0B0, S0B1, S1B0, S0B2, S1B1, S2B0) are accumulated in
// FP32 in tensor memory, which keeps the single-precision accuracy of S.
//
// The product runs as a persistent kernel: a grid of at most one CTA per SM walks a static list
// of work items (row tile of 128 sites, replica tile of BN, K split), the replica tile varying
// fastest so that CTAs running at the same time read the same tile of S (the second read is an
// L2 hit).  Per CTA one thread streams the six operand tiles of each 64-wide K step into a
// STAGES-deep ring of 128-byte-swizzled shared memory with TMA, one thread issues the
// tcgen05.mma instructions into one of two TMEM accumulators, and four epilogue warps read the
// other accumulator back (tcgen05.ld) and store the tile's FP32 partial sums, so the epilogue of
// one item overlaps the products of the next.  Partial sums of the K splits are added in FP64 by
// the reduction kernel.  BN, STAGES and the split count are chosen per (n, m) by timing the
// candidates on the device (tc_tune).  Every mbarrier wait is bounded: on expiry the CTA records
// a timeout in the status word, lets its copies in flight land, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpm {

constexpr int TC_BM = 128;          // rows of S per item (MMA M)
constexpr int TC_BK = 64;           // K elements per stage (128 bytes of bf16 per row)
constexpr int TC_THREADS = 192;     // warp 0: TMA, warp 1: MMA, warps 2-5: epilogue
constexpr uint64_t TC_WAIT_NS = 2000000000ull;   // bound on any single mbarrier wait: 2 s
constexpr int TC_SMS = 152;

template <int BN, int STAGES> struct TcCfg {
    static constexpr int A_BYTES = TC_BM * 128;            // one bf16 split of the S tile
    static constexpr int B_BYTES = BN * 128;               // one bf16 split of the b tile
    static constexpr int STAGE = 3 * A_BYTES + 3 * B_BYTES;
    static constexpr int TMEM_COLS = 2 * BN;               // two accumulators
    static constexpr int SMEM = 1024 + STAGES * STAGE + 256;
    static_assert(SMEM <= 227 * 1024, "stage ring exceeds shared memory");
};

struct TcMaps {
    CUtensorMap a[3];
    CUtensorMap b[3];
};

// item -> (row tile, replica tile, split), replica tile fastest
struct TcItems {
    int mt, nt, splits, ksteps, kchunk;   // kchunk: K steps per split
    __device__ __forceinline__ void get(int it, int& row, int& rep, int& split, int& kb, int& ke) const {
        rep = it % nt;
        const int rest = it / nt;
        split = rest % splits;
        row = rest / splits;
        kb = split * kchunk;
        ke = min(ksteps, kb + kchunk);
    }
};

// skip_loads = 1 issues no TMA copies at all: every wait must then run out (the failure-detection
// self test); it is never set on the compute path.
template <int BN, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_sb(const __grid_constant__ TcMaps maps, TcItems W, int n, int m,
                                                         float* __restrict__ part, unsigned* __restrict__ status,
                                                         int skip_loads, uint64_t wait_ns) {
    typedef TcCfg<BN, STAGES> C;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint64_t* full = (uint64_t*)(smem + STAGES * C::STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;      // [2] accumulator written (MMA -> epilogue)
    uint64_t* acce = accf + 2;            // [2] accumulator read back (epilogue -> MMA)
    uint32_t* tmem_slot = (uint32_t*)(acce + 2);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int items = W.mt * W.nt * W.splits;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(&accf[a], 1); mbar_init(&acce[a], 4); }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0 && !skip_loads) {
            // producer: six TMA tiles per K step, continuing across items without a break
            uint32_t g = 0, issued = 0;
            for (int it = blockIdx.x; it < items && !*abort; it += gridDim.x) {
                int row, rep, split, kb, ke;
                W.get(it, row, rep, split, kb, ke);
                for (int t = kb; t < ke; ++t, ++g) {
                    const int s = (int)(g % STAGES);
                    if (g >= (uint32_t)STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1, abort, wait_ns)) break;
                    uint8_t* st = smem + s * C::STAGE;
                    mbar_expect_tx(&full[s], C::STAGE);
                    const int kx = t * TC_BK;
                    for (int q = 0; q < 3; ++q) tma_load_2d(st + q * C::A_BYTES, &maps.a[q], kx, row * TC_BM, &full[s]);
                    for (int q = 0; q < 3; ++q)
                        tma_load_2d(st + 3 * C::A_BYTES + q * C::B_BYTES, &maps.b[q], kx, rep * BN, &full[s]);
                    ++issued;
                }
            }
            if (*abort) {
                // let the copies already issued land before the CTA exits (bounded)
                for (uint32_t t = (issued > (uint32_t)STAGES ? issued - STAGES : 0); t < issued; ++t) {
                    const int s = (int)(t % STAGES);
                    const uint64_t t0 = gtimer_ns();
                    while (!mbar_try(&full[s], (t / STAGES) & 1) && gtimer_ns() - t0 < wait_ns) {}
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: item li accumulates into TMEM columns (li & 1) * BN
            const uint32_t idesc = idesc_bf16(TC_BM, BN);
            const int pa[6] = {0, 0, 1, 0, 1, 2};
            const int pb[6] = {0, 1, 0, 2, 1, 0};
            uint32_t g = 0, li = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < items && ok; it += gridDim.x, ++li) {
                int row, rep, split, kb, ke;
                W.get(it, row, rep, split, kb, ke);
                const uint32_t acc = li & 1;
                if (li >= 2 && !mbar_wait(&acce[acc], ((li >> 1) - 1) & 1, abort, wait_ns)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dt = tmem + acc * BN;
                for (int t = kb; t < ke; ++t, ++g) {
                    const int s = (int)(g % STAGES);
                    if (!mbar_wait(&full[s], (g / STAGES) & 1, abort, wait_ns)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = su32(smem + s * C::STAGE);
                    const uint32_t sb = sa + 3 * C::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
                        for (int p = 0; p < 6; ++p) {
                            const uint64_t ad = sdesc_sw128(sa + pa[p] * C::A_BYTES + kk * 32);
                            const uint64_t bd = sdesc_sw128(sb + pb[p] * C::B_BYTES + kk * 32);
                            umma_f16(dt, ad, bd, idesc, (t > kb || kk > 0 || p > 0) ? 1u : 0u);
                        }
                    }
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&accf[acc]);
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. rows 32 (w % 4) .. of the item's tile
        const int quarter = warp & 3;
        uint32_t li = 0;
        for (int it = blockIdx.x; it < items; it += gridDim.x, ++li) {
            int row, rep, split, kb, ke;
            W.get(it, row, rep, split, kb, ke);
            const uint32_t acc = li & 1;
            const bool have = __all_sync(0xffffffffu, mbar_wait(&accf[acc], (li >> 1) & 1, abort, wait_ns) ? 1 : 0) != 0;
            if (!have) break;
            tc_fence_after();
            const int i = row * TC_BM + quarter * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + acc * BN;
            float* pout = part + (int64_t)split * m * n;
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(trow + c0, v);
                if (i < n) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int r = rep * BN + c0 + k;
                        if (r < m) pout[(int64_t)r * n + i] = v[k];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    if (warp == 1) {
        __syncwarp();   // lane 0 ran the MMA loop alone: reconverge before the warp-wide dealloc
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

// ----------------------------------------------------------------------------- tile plans
// A plan fixes the replica tile BN, the ring depth, the K split count (after rounding the K range
// of a split to whole 64-wide steps) and the grid.  The (BN, STAGES) pairs below are the ones
// whose stage ring fits in shared memory next to the barriers.
struct TcPlan {
    int bn = 0, stages = 0, splits = 0, grid = 0;
    float ms = -1.f;          // measured time per product (ms); negative: chosen without timing
    int candidates = 0;       // plans timed to choose it
};

static bool tc_valid(int bn, int stages) {
    return (bn == 32 && (stages == 2 || stages == 3)) || (bn == 64 && (stages == 2 || stages == 3)) ||
           (bn == 128 && stages == 2);
}

static TcItems tc_items(int64_t n, int m, int bn, int splits) {
    TcItems W;
    W.mt = (int)((n + TC_BM - 1) / TC_BM);
    W.nt = (m + bn - 1) / bn;
    W.ksteps = (int)(tc_ld(n) / TC_BK);
    W.kchunk = (W.ksteps + splits - 1) / splits;
    W.splits = (W.ksteps + W.kchunk - 1) / W.kchunk;   // every split holds at least one K step
    return W;
}

template <int BN, int STAGES>
static cpm_status launch_tc_t(cpm_ctx* c, const TcMaps& maps, const TcItems& W, int grid, int n, int m, float* part,
                             int skip_loads, uint64_t wait_ns) {
    typedef TcCfg<BN, STAGES> C;
    CPM_CUDA(c, cudaFuncSetAttribute(k_tc_sb<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    k_tc_sb<BN, STAGES><<<grid, TC_THREADS, C::SMEM, c->stream>>>(maps, W, n, m, part, c->status, skip_loads, wait_ns);
    CPM_LAUNCH(c, "k_tc_sb");
    return CPM_OK;
}

static cpm_status launch_plan(cpm_ctx* c, const TcPlan& p, const TcMaps& maps, int n, int m, float* part,
                              int skip_loads = 0, uint64_t wait_ns = TC_WAIT_NS) {
    const TcItems W = tc_items(n, m, p.bn, p.splits);
    const int grid = std::max(1, std::min(p.grid, W.mt * W.nt * W.splits));
    if (p.bn == 32 && p.stages == 2) return launch_tc_t<32, 2>(c, maps, W, grid, n, m, part, skip_loads, wait_ns);
    if (p.bn == 32 && p.stages == 3) return launch_tc_t<32, 3>(c, maps, W, grid, n, m, part, skip_loads, wait_ns);
    if (p.bn == 64 && p.stages == 2) return launch_tc_t<64, 2>(c, maps, W, grid, n, m, part, skip_loads, wait_ns);
    if (p.bn == 64 && p.stages == 3) return launch_tc_t<64, 3>(c, maps, W, grid, n, m, part, skip_loads, wait_ns);
    if (p.bn == 128 && p.stages == 2) return launch_tc_t<128, 2>(c, maps, W, grid, n, m, part, skip_loads, wait_ns);
    return set_err(c, CPM_E_ARG, "tensor-core plan (BN %d, %d stages) not built", p.bn, p.stages);
}

// bytes of the split partial sums a plan with `splits` needs
static size_t tc_plan_part_bytes(int64_t n, int m, int splits) { return sizeof(float) * (size_t)splits * m * n; }
// the part buffer of the tuning candidates is capped here
constexpr size_t TC_PART_CAP = (size_t)256 << 20;

// The plan without timing: the largest replica tile up to m, the deepest ring, and about two
// items per SM.
static TcPlan tc_default_plan(int64_t n, int m) {
    TcPlan p;
    p.bn = m <= 32 ? 32 : (m <= 64 ? 64 : 128);
    p.stages = p.bn == 128 ? 2 : 3;
    const TcItems W0 = tc_items(n, m, p.bn, 1);
    const int base = W0.mt * W0.nt;
    int sp = std::max(1, std::min(W0.ksteps, (2 * TC_SMS + base - 1) / base));
    while (sp > 1 && tc_plan_part_bytes(n, m, sp) > TC_PART_CAP) --sp;
    p.splits = tc_items(n, m, p.bn, sp).splits;
    p.grid = std::min(TC_SMS, base * p.splits);
    return p;
}

// Candidate plans for (n, m): every built (BN, STAGES) with BN no larger than needed, and split
// counts that make the item count close to whole multiples of the SM count (1 to 8 waves).
static std::vector<TcPlan> tc_candidates(int64_t n, int m) {
    std::vector<TcPlan> out;
    const int bns[3] = {32, 64, 128};
    for (int bn : bns) {
        if (bn > 32 && bn / 2 >= m) continue;   // a smaller tile already covers all replicas
        for (int stages = 2; stages <= 3; ++stages) {
            if (!tc_valid(bn, stages)) continue;
            const TcItems W0 = tc_items(n, m, bn, 1);
            const int base = W0.mt * W0.nt;
            std::vector<int> sps = {1};
            for (int w = 1; w <= 8; ++w) {
                sps.push_back(std::max(1, (w * TC_SMS) / base));
                sps.push_back(std::max(1, (w * TC_SMS + base - 1) / base));
            }
            std::vector<int> seen;
            for (int sp : sps) {
                sp = std::min(sp, W0.ksteps);
                if (tc_plan_part_bytes(n, m, sp) > TC_PART_CAP) continue;
                const int eff = tc_items(n, m, bn, sp).splits;
                if (std::find(seen.begin(), seen.end(), eff) != seen.end()) continue;
                seen.push_back(eff);
                TcPlan p;
                p.bn = bn;
                p.stages = stages;
                p.splits = eff;
                p.grid = std::min(TC_SMS, base * eff);
                out.push_back(p);
            }
        }
    }
    return out;
}

static std::mutex g_tc_mutex;
static std::map<std::tuple<int, int64_t, int>, TcPlan> g_tc_plans;   // (device, n, m) -> tuned plan

static cpm_status tc_maps(cpm_ctx* c, int m, int bn, const void* bsplit, TcMaps* maps) {
    const int64_t n = c->n, ld = tc_ld(n);
    const __nv_bfloat16* Sb = (const __nv_bfloat16*)c->Sb;
    const __nv_bfloat16* Bb = (const __nv_bfloat16*)bsplit;
    for (int q = 0; q < 3; ++q) {
        if (!make_map(&maps->a[q], Sb + (size_t)q * n * ld, n, ld, TC_BM) ||
            !make_map(&maps->b[q], Bb + (size_t)q * m * ld, m, ld, bn))
            return set_err(c, CPM_E_CUDA, "cuTensorMapEncodeTiled failed");
    }
    return CPM_OK;
}

size_t tc_bsplit_bytes(int64_t n, int m);

// Times every candidate plan for (n, m) on the context stream (CUDA events; one launch to warm up,
// then the best of three) with the context's operand buffers, and keeps the fastest per
// (device, n, m).  Not during stream capture (the caller checks).
static cpm_status tc_tune(cpm_ctx* c, int m, float* part, void* bsplit, TcPlan* out) {
    const int64_t n = c->n;
    std::vector<TcPlan> cands = tc_candidates(n, m);
    if (cands.empty()) { *out = tc_default_plan(n, m); return CPM_OK; }
    CPM_CUDA(c, cudaMemsetAsync(bsplit, 0, tc_bsplit_bytes(n, m), c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CPM_CUDA(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return set_err(c, CPM_E_CUDA, "cudaEventCreate"); }
    TcPlan best;
    best.ms = 1e30f;
    cpm_status st = CPM_OK;
    for (TcPlan& p : cands) {
        TcMaps maps;
        if ((st = tc_maps(c, m, p.bn, bsplit, &maps)) != CPM_OK) break;
        if ((st = launch_plan(c, p, maps, (int)n, m, part)) != CPM_OK) break;
        float t = 1e30f;
        for (int rep = 0; rep < 3 && st == CPM_OK; ++rep) {
            cudaEventRecord(e0, c->stream);
            st = launch_plan(c, p, maps, (int)n, m, part);
            cudaEventRecord(e1, c->stream);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = set_err(c, CPM_E_CUDA, "tensor-core tuning: event timing failed");
                break;
            }
            t = std::min(t, ms);
        }
        if (st != CPM_OK) break;
        p.ms = t;
        if (t < best.ms) best = p;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CPM_TRY(st);
    best.candidates = (int)cands.size();
    *out = best;
    return CPM_OK;
}

// The plan in use for m replicas: the tuned one when there is one; otherwise tuned now (outside
// capture), or the untimed default while the stream is being captured.
static cpm_status tc_plan_for(cpm_ctx* c, int m, float* part, void* bsplit, TcPlan* out) {
    const auto key = std::make_tuple(c->device, (int64_t)c->n, m);
    {
        std::lock_guard<std::mutex> lock(g_tc_mutex);
        auto it = g_tc_plans.find(key);
        if (it != g_tc_plans.end()) { *out = it->second; return CPM_OK; }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CPM_CUDA(c, cudaStreamIsCapturing(c->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone || !c->tc_autotune) { *out = tc_default_plan(c->n, m); return CPM_OK; }
    TcPlan p;
    CPM_TRY(tc_tune(c, m, part, bsplit, &p));
    std::lock_guard<std::mutex> lock(g_tc_mutex);
    g_tc_plans[key] = p;
    *out = p;
    return CPM_OK;
}

// largest part buffer any candidate, the default plan or the kept plan for (n, m) can need
static size_t tc_part_need(int device, int64_t n, int m) {
    size_t b = tc_plan_part_bytes(n, m, tc_default_plan(n, m).splits);
    for (const TcPlan& p : tc_candidates(n, m)) b = std::max(b, tc_plan_part_bytes(n, m, p.splits));
    {
        std::lock_guard<std::mutex> lock(g_tc_mutex);
        auto it = g_tc_plans.find(std::make_tuple(device, n, m));
        if (it != g_tc_plans.end()) b = std::max(b, tc_plan_part_bytes(n, m, it->second.splits));
    }
    return (b + 255) & ~(size_t)255;
}

// part[split][r][i] = sum over the split's K range of S[i][j] b[r][j]; returns the split count
cpm_status tc_sb(cpm_ctx* c, int m, const double* b, float* part, int* splits, void* bsplit, const double* gmean,
                 const int* gid, int ngrp) {
    const int64_t n = c->n, ld = tc_ld(n);
    TcPlan p;
    CPM_TRY(tc_plan_for(c, m, part, bsplit, &p));
    k_split3<<<(unsigned)((m * ld + 255) / 256), 256, 0, c->stream>>>(b, m, n, ld, (__nv_bfloat16*)bsplit, gmean, gid,
                                                                      ngrp);
    CPM_LAUNCH(c, "k_split3(b)");
    TcMaps maps;
    CPM_TRY(tc_maps(c, m, p.bn, bsplit, &maps));
    prof_begin(c, CPM_K_TCGEMM);
    CPM_TRY(launch_plan(c, p, maps, (int)n, m, part));
    prof_end(c, CPM_K_TCGEMM);
    *splits = p.splits;
    return CPM_OK;
}


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
    const size_t pb = std::max(tc_part_need(c->device, n, m), c->tc_pbytes);
    const size_t need = pb + ((tc_bsplit_bytes(n, m) + 255) & ~(size_t)255) + sizeof(double) * (size_t)m * c->tc_ngrp;
    if (c->tbuf_bytes < need || c->tc_pbytes != pb) {
        dev_free(c, c->tbuf);
        c->tbuf = nullptr;
        c->tbuf_bytes = 0;
        c->tc_pbytes = 0;
        c->graph_valid = false;
        CPM_TRY(dev_alloc(c, &c->tbuf, need));
        c->tbuf_bytes = need;
        c->tc_pbytes = pb;
    }
    // choose (or tune) the tile plan now, before any capture of the step
    TcPlan p;
    return tc_plan_for(c, m, (float*)c->tbuf, (char*)c->tbuf + c->tc_pbytes, &p);
}

cpm_status tc_update(cpm_ctx* c, int m, const double* psi, const double* b, double* q) {
    const int64_t n = c->n;
    CPM_TRY(tc_reserve(c, m));
    float* part = (float*)c->tbuf;
    void* bsplit = (char*)c->tbuf + c->tc_pbytes;
    double* gmean = (double*)((char*)bsplit + ((tc_bsplit_bytes(n, m) + 255) & ~(size_t)255));
    const int* gid = c->tc_use_z ? c->zmap : c->group;
    k_gmeans<<<(unsigned)(((int64_t)m * c->tc_ngrp * 32 + 255) / 256), 256, 0, c->stream>>>(b, gid, n, m, c->tc_ngrp,
                                                                                              gmean);
    CPM_LAUNCH(c, "k_gmeans");
    int splits = 0;
    CPM_TRY(tc_sb(c, m, b, part, &splits, bsplit, gmean, gid, c->tc_ngrp));
    k_tc_reduce<<<(unsigned)((m * n + 255) / 256), 256, 0, c->stream>>>(part, splits, upd_sg(c), upd_ng(c), psi, c->SZ, gmean,
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
    TcMaps maps;
    CPM_TRY(tc_maps(c, m, 32, (char*)c->tbuf + c->tc_pbytes, &maps));
    TcPlan p;
    p.bn = 32;
    p.stages = 2;
    p.splits = 1;
    p.grid = 1;
    return launch_plan(c, p, maps, (int)c->n, m, (float*)c->tbuf, 1, (uint64_t)(wait_ms * 1e6));
}

cpm_status tc_plan_set(cpm_ctx* c, int m, const int32_t* plan) {
    if (!tc_valid(plan[0], plan[1]) || plan[2] < 1 || plan[3] < 1)
        return set_err(c, CPM_E_ARG, "tensor-core plan: (BN %d, %d stages) not built, or splits / CTAs < 1", plan[0],
                       plan[1]);
    const TcItems W0 = tc_items(c->n, m, plan[0], 1);
    TcPlan p;
    p.bn = plan[0];
    p.stages = plan[1];
    p.splits = tc_items(c->n, m, p.bn, std::min(plan[2], W0.ksteps)).splits;
    p.grid = std::min(plan[3], TC_SMS);
    if (tc_plan_part_bytes(c->n, m, p.splits) > TC_PART_CAP)
        return set_err(c, CPM_E_ARG, "tensor-core plan: %d splits need more than %zu bytes of partial sums", p.splits,
                       TC_PART_CAP);
    {
        std::lock_guard<std::mutex> lock(g_tc_mutex);
        g_tc_plans[std::make_tuple(c->device, (int64_t)c->n, m)] = p;
    }
    c->graph_valid = false;
    return tc_reserve(c, m);
}

cpm_status tc_plan_query(cpm_ctx* c, int m, int32_t* plan, double* ms) {
    CPM_TRY(tc_reserve(c, m));
    TcPlan p;
    CPM_TRY(tc_plan_for(c, m, (float*)c->tbuf, (char*)c->tbuf + c->tc_pbytes, &p));
    if (plan) {
        plan[0] = p.bn;
        plan[1] = p.stages;
        plan[2] = p.splits;
        plan[3] = p.grid;
        plan[4] = p.candidates;
    }
    if (ms) *ms = p.ms;
    return CPM_OK;
}

size_t tc_bsplit_bytes(int64_t n, int m) { return sizeof(__nv_bfloat16) * 3 * (size_t)m * tc_ld(n); }

}  // namespace cpm
