// Real-space part of b in single precision from gathered candidate lists (Sec. II.A: the erfc terms
// of the Ewald sum between the electrolyte charges and the electrode Gaussians, Eq. (b)).
//
// b_i(real) = sum_j Q_j f_i(r_ij) over the pairs within r_c, f_i(r) = (erfc(alpha r) - erfc(eta_i r)) / r.
// The site term erfc(eta r) / r is below 5e-11 eta once eta r >= 4.5; the rare pairs closer than
// r_eta = 4.5 / eta take the tabulated pair function (cubic Hermite, FP64-built) instead, in a
// branch taken per warp.  Outside the cores, with erfcx(x) = e^{x^2} erfc(x),
//     erfc(alpha r) / r = e^{-alpha^2 r^2} erfcx(alpha r) / r,
// and erfcx(alpha r), smooth and slowly varying, is replaced on [r_lo, r_c] (r_lo the smallest core
// radius) by its Chebyshev interpolant, fitted here in FP64 (degree 12, or 14 where 12 does not
// reach 1e-7 alpha in f): a pair costs a reciprocal square root, an exponential and a Horner chain,
// run for two charges at a time with packed FP32 instructions, and every factor of f is accurate
// relative to f itself.
//
// Work: persistent blocks of four warps take (chunk, replica) items from a queue, a chunk being at
// most 32 sites of one real-space cell.  A block works on one item at a time, in three phases
// separated by block barriers, so that the memory latency of one item is spread over 128 threads
// and the blocks sharing an SM overlap one another's phases:
//   1. every stencil row of the cell list, trimmed to the bounding box of the chunk's sites grown by
//      r_c, is one contiguous range of the cell-sorted charges per image shift along x (a "run"); the
//      runs of each chunk are fixed by the geometry and listed once on the host (read together with the
//      chunk's sites), so per item a thread per run reads its two cell starts and a block scan numbers
//      the charges of all runs;
//   2. the charges are read in rounds of up to 1,536, up to twelve loads in flight per thread (each
//      charge finds its run in a shared-memory map), shifted to their image, and those within r_c of
//      the box are kept in a structure-of-arrays list, in the order (warp, slot, lane);
//   3. the list is evaluated against the chunk's sites in groups of four: the (group, 64-charge
//      batch) work is cut into four equal contiguous ranges, one per warp, every lane two candidates
//      (one packed pair) against the four sites of a group, the lane sums reduced by a fixed
//      butterfly; a group's sums from the warps are added in warp order and the rounds in round order.
// The list order and the work split depend only on the item, so the result does not depend on
// scheduling.

#include <cmath>

#include "common.cuh"

namespace cpm {

constexpr int RB_T = 128;                       // threads per block
constexpr int RB_W = RB_T / 32;
constexpr int RB_K = 12;                        // charges per thread and round, all loads in flight
constexpr int RB_CAP = RB_T * RB_K;             // charges read per round (the kept ones fit the list)
constexpr int RB_RUNS = 256;                    // runs of one chunk, at most
constexpr int RB_G = 8;                         // groups of four sites of a chunk, at most
constexpr float RP_XETA = 4.5f;                 // eta r past which erfc(eta r) / r is dropped
constexpr float RP_BIG = 1099511627776.0f;      // 2^40: turns a sign into a 0/1 weight (saturated product)
constexpr float RP_TINY = 1e-30f;               // keeps 1 / sqrt(r^2) finite at r = 0

// ----------------------------------------------------------------------------- the fit (host, FP64)
// erfcx(x) = e^{x^2} erfc(x), for 0 <= x <= 7 (e^{49} erfc(7) stays well inside FP64)
static double erfcx_d(double x) { return std::exp(x * x) * std::erfc(x); }

RealPoly fit_real_poly(double alpha, double rcut, double rlo) {
    RealPoly rp{};
    const float rc2 = (float)(rcut * rcut);
    // the kernel takes pairs with r^2 < rc2 in FP32 and, outside the cores, r > rlo; the interval
    // covers them with a margin
    const double hi = rcut * (1.0 + 1e-6), lo = rlo * (1.0 - 1e-6);
    if (!(lo > 0.0 && lo < hi) || alpha * hi > 7.0) return rp;
    for (int d : {12, 14}) {
        const int N = d + 1;
        // Chebyshev interpolation of erfcx(alpha r) at the N Chebyshev points of [lo, hi]
        std::vector<double> gk(N), ch(N);
        for (int k = 0; k < N; ++k) gk[k] = erfcx_d(alpha * (0.5 * (lo + hi) + 0.5 * (hi - lo) * std::cos(PI * (k + 0.5) / N)));
        for (int j = 0; j < N; ++j) {
            double sum = 0.0;
            for (int k = 0; k < N; ++k) sum += gk[k] * std::cos(PI * j * (k + 0.5) / N);
            ch[j] = (j == 0 ? 1.0 : 2.0) * sum / N;
        }
        // to monomials in v: T_0 = 1, T_1 = v, T_{j+1} = 2 v T_j - T_{j-1}
        std::vector<double> mono(N, 0.0), t0(N, 0.0), t1(N, 0.0), tn(N, 0.0);
        t0[0] = 1.0;
        t1[1] = 1.0;
        mono[0] = ch[0];
        mono[1] = ch[1];
        for (int j = 2; j < N; ++j) {
            for (int k = 0; k < N; ++k) tn[k] = (k > 0 ? 2.0 * t1[k - 1] : 0.0) - t0[k];
            for (int k = 0; k < N; ++k) mono[k] += ch[j] * tn[k];
            t0.swap(t1);
            t1.swap(tn);
        }
        for (int k = 0; k <= RP_DEG_MAX; ++k) rp.c[k] = k < N ? (float)mono[k] : 0.f;
        // the pair function from the FP32 coefficients against erfc(alpha r) / r on a fine grid
        double err = 0.0;
        for (int i = 0; i <= 8192; ++i) {
            const double r = lo + (hi - lo) * i / 8192.0, v = (2.0 * r - lo - hi) / (hi - lo);
            double p = rp.c[d];
            for (int k = d - 1; k >= 0; --k) p = p * v + rp.c[k];
            err = std::max(err, std::fabs(std::exp(-alpha * alpha * r * r) * p / r - std::erfc(alpha * r) / r));
        }
        if (err <= 1e-7 * alpha) {
            rp.deg = d;
            rp.s1 = (float)(2.0 / (hi - lo));
            rp.s0 = (float)(-(hi + lo) / (hi - lo));
            rp.ke = (float)(-alpha * alpha / std::log(2.0));
            rp.rc2 = rc2;
            return rp;
        }
    }
    return RealPoly{};
}

// ----------------------------------------------------------------------------- chunk site slots
__global__ void k_real_sites(const int4* __restrict__ chunks, int nchunks, const int* __restrict__ perm,
                             const float* __restrict__ s32, int64_t n, const int* __restrict__ tabid,
                             float4* __restrict__ rsite, int* __restrict__ rsite_tab, int* __restrict__ rsite_idx) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nchunks * 32) return;
    const int4 ci = chunks[t >> 5];
    const int l = t & 31;
    const int i = perm[ci.x + (l < ci.y ? l : 0)];
    const float rl = RP_XETA / s32[3 * n + i];
    rsite[t] = make_float4(s32[i], s32[n + i], s32[2 * n + i], fmaxf(rl * rl, 1e-6f));
    rsite_tab[t] = tabid[i] * RT_S;
    rsite_idx[t] = i;
}

// ----------------------------------------------------------------------------- the kernel
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mul_sat(float a, float b) {
    float y;
    asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two (site, charge) pairs in the two halves of packed registers (here one site, its coordinates in
// both halves, against two charges): acc += Q w f for the pairs with r_eta^2 < r^2 < r_c^2 (w is 1
// there and 0 elsewhere), f = 2^(ke r^2) P(r s1 + s0) / r; det <= 0 marks a pair inside a Gaussian
// core.  Every factor of f carries a relative rounding error, so f is accurate relative to itself
// also where it is small (no difference of two terms of size 1/r).
template <int DEG>
__device__ __forceinline__ void rp_pair2(uint64_t SX, uint64_t SY, uint64_t SZ, uint64_t NL, uint64_t QX,
                                         uint64_t QY, uint64_t QZ, uint64_t QW, const uint64_t (&C)[DEG + 1],
                                         uint64_t S1, uint64_t S0, uint64_t KE, uint64_t RC2, uint64_t BIG2,
                                         uint64_t TINY2, uint64_t& acc, float& det) {
    const uint64_t dx = sub2(SX, QX), dy = sub2(SY, QY), dz = sub2(SZ, QZ);
    uint64_t r2 = fma2(dx, dx, TINY2);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    const float2 r2s = up2(r2);
    const uint64_t rs = pk2(rsqrt_approx(r2s.x), rsqrt_approx(r2s.y));   // 1 / r
    const uint64_t v = fma2(mul2(r2, rs), S1, S0);
    uint64_t p = fma2(C[DEG], v, C[DEG - 1]);
#pragma unroll
    for (int k = DEG - 2; k >= 0; --k) p = fma2(p, v, C[k]);
    const float2 y = up2(mul2(r2, KE));
    const uint64_t f = mul2(mul2(pk2(ex2_approx(y.x), ex2_approx(y.y)), p), rs);
    const float2 a = up2(sub2(RC2, r2)), bq = up2(fma2(r2, BIG2, NL));
    const uint64_t w = mul2(pk2(mul_sat(a.x, bq.x), mul_sat(a.y, bq.y)), QW);
    acc = fma2(w, f, acc);
    det = fminf(bq.x, bq.y);
}


// Single-precision constants of the launch (made on the host).
struct RbGrid {
    float inv_h;      // RT_N / r_c: table rows per unit distance
};

// cp.async copies into shared memory (completion per thread by cp.async.wait_all, visibility to
// the block by the barrier after it)
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The inputs of one item, copied into shared memory at its start.
struct RbItem {
    float4 site[32];          // the chunk's sites (x, y, z, r_eta^2), slots past the count repeat the first
    float4 box[2];            // their bounding box: lo, hi
    int4 chunk;               // (first site, site count, run count, 0)
    int sidx[32];             // site index of each slot
    int toff[32];             // pair-table offset of each slot
    int2 rcell[RB_RUNS];      // runs: first cell and one past the last (one replica's cell list)
    float4 rsh[RB_RUNS];      // their image shifts
    int rb[RB_RUNS];          // per run, the first charge in the sorted order ...
    int re[RB_RUNS];          // ... and one past its last
    int item;
};

// Block shared memory.
struct RbShared {
    float2 cx[RB_CAP / 2], cy[RB_CAP / 2], cz[RB_CAP / 2], cq[RB_CAP / 2];   // kept charges, in list order
    RbItem it;                // the current item's inputs
    int rpre[RB_RUNS + 1];    // exclusive prefix of the run lengths
    short erun[RB_CAP];       // the run of each charge of the round
    int wsum[RB_W + 1];       // block scan of the run lengths: warp totals
    int wkept[RB_W];          // kept charges per warp
    float part[RB_W * RB_G][4];   // per (warp, group): the warp's sums of the group's four sites
    float acc[32];            // per site: the sums of the rounds so far
    int next;                 // the next item (taken from the queue one item ahead)
};

// One (group, list part) unit: the four sites of group gi against the list's 64-charge batches
// [b0, b1); the four sums go to part[u].
template <int DEG>
__device__ __forceinline__ void rb_unit(RbShared& sm, const RbItem& I, int gi, int b0, int b1, int u,
                                        const uint64_t (&C)[DEG + 1], const RealPoly& rp,
                                        const float4* __restrict__ tab, float inv_h) {
    const int lane = threadIdx.x & 31;
    const uint64_t S1 = pk2(rp.s1, rp.s1), S0 = pk2(rp.s0, rp.s0), KE = pk2(rp.ke, rp.ke), RC2 = pk2(rp.rc2, rp.rc2);
    const uint64_t BIG2 = pk2(RP_BIG, RP_BIG), TINY2 = pk2(RP_TINY, RP_TINY);
    uint64_t SX[4], SY[4], SZ[4], NL[4], acc[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float4 a = I.site[4 * gi + s];
        SX[s] = pk2(a.x, a.x);
        SY[s] = pk2(a.y, a.y);
        SZ[s] = pk2(a.z, a.z);
        NL[s] = pk2(-a.w * RP_BIG, -a.w * RP_BIG);
        acc[s] = 0ull;   // +0.0f in both halves
    }
    for (int b = b0; b < b1; ++b) {
        const int idx = (b << 5) + lane;
        const float2 qx = sm.cx[idx], qy = sm.cy[idx], qz = sm.cz[idx], qq = sm.cq[idx];
        const uint64_t QX = pk2(qx.x, qx.y), QY = pk2(qy.x, qy.y), QZ = pk2(qz.x, qz.y), QW = pk2(qq.x, qq.y);
        float d[4];
#pragma unroll
        for (int s = 0; s < 4; ++s)
            rp_pair2<DEG>(SX[s], SY[s], SZ[s], NL[s], QX, QY, QZ, QW, C, S1, S0, KE, RC2, BIG2, TINY2, acc[s], d[s]);
        if (__any_sync(0xffffffffu, fminf(fminf(d[0], d[1]), fminf(d[2], d[3])) <= 0.f)) {
            // pairs inside a Gaussian core: the tabulated pair function, with r^2 and the core test
            // computed exactly as above (same operations, same roundings)
            const float hx[2] = {qx.x, qx.y}, hy[2] = {qy.x, qy.y}, hz[2] = {qz.x, qz.y}, hq[2] = {qq.x, qq.y};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const float4 st = I.site[4 * gi + s];
                const float2 A = up2(acc[s]);
                float av[2] = {A.x, A.y};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float ex = __fsub_rn(st.x, hx[h]), ey = __fsub_rn(st.y, hy[h]), ez = __fsub_rn(st.z, hz[h]);
                    float rr = __fmaf_rn(ex, ex, RP_TINY);
                    rr = __fmaf_rn(ey, ey, rr);
                    rr = __fmaf_rn(ez, ez, rr);
                    if (hq[h] != 0.f && __fmaf_rn(rr, RP_BIG, -st.w * RP_BIG) <= 0.f) {
                        const float uu = sqrtf(rr) * inv_h;
                        const int k = min((int)uu, RT_N);
                        const float t = uu - (float)k;
                        const float4 cf = tab[I.toff[4 * gi + s] + k];
                        av[h] = fmaf(hq[h], cf.x + t * (cf.y + t * (cf.z + t * cf.w)), av[h]);
                    }
                }
                acc[s] = pk2(av[0], av[1]);
            }
        }
    }
    // both halves of each site's sum, then a fixed butterfly over the lanes: lanes 8 s .. 8 s + 7
    // end with the sum of site s
    const float2 a0 = up2(acc[0]), a1 = up2(acc[1]), a2 = up2(acc[2]), a3 = up2(acc[3]);
    const float Ax = a0.x + a0.y, Ay = a1.x + a1.y, Bx = a2.x + a2.y, By = a3.x + a3.y;
    const bool h16 = lane & 16, h8 = lane & 8;
    float k0 = h16 ? Bx : Ax, k1 = h16 ? By : Ay;
    const float s0 = h16 ? Ax : Bx, s1 = h16 ? Ay : By;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    float kk = h8 ? k1 : k0;
    kk += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    kk += __shfl_xor_sync(0xffffffffu, kk, 4);
    kk += __shfl_xor_sync(0xffffffffu, kk, 2);
    kk += __shfl_xor_sync(0xffffffffu, kk, 1);
    if ((lane & 7) == 0) sm.part[u][lane >> 3] = kk;
}

struct RbInputs {
    const float4* site;       // [nchunks * 32] sites of each chunk slot
    const int* sidx;          // [nchunks * 32] their site indices
    const int* toff;          // [nchunks * 32] their pair-table offsets
    const float4* box;        // [nchunks * 2] bounding box of each chunk
    const int4* chunk;        // [nchunks] (first site, site count, run count, 0)
    const int2* rcell;        // [nchunks * stride] runs of each chunk
    const float4* rsh;        // [nchunks * stride] their image shifts
    int stride;
    int nchunks;
};

// Copies the fixed inputs of item `item` (chunk item / m) into I; one commit group per thread.
__device__ __forceinline__ void rb_fetch_static(RbItem& I, const RbInputs& in, int item, int m) {
    const int tid = threadIdx.x, ch = item / m;
    if (tid < 32) {
        cpa16(&I.site[tid], &in.site[(int64_t)ch * 32 + tid]);
        cpa4(&I.sidx[tid], &in.sidx[(int64_t)ch * 32 + tid]);
        cpa4(&I.toff[tid], &in.toff[(int64_t)ch * 32 + tid]);
    } else if (tid < 34) {
        cpa16(&I.box[tid - 32], &in.box[2 * (int64_t)ch + tid - 32]);
    } else if (tid == 34) {
        cpa16(&I.chunk, &in.chunk[ch]);
    }
    for (int j = tid; j < in.stride; j += RB_T) {
        cpa8(&I.rcell[j], &in.rcell[(int64_t)ch * in.stride + j]);
        cpa16(&I.rsh[j], &in.rsh[(int64_t)ch * in.stride + j]);
    }
    cpa_commit();
}

// Copies the charge ranges of the runs of I (whose fixed inputs have landed) from the cell list.
__device__ __forceinline__ void rb_fetch_starts(RbItem& I, const int* __restrict__ start, int ncells, int m) {
    const int r = I.item % m, nr = I.chunk.z;
    for (int j = threadIdx.x; j < nr; j += RB_T) {
        const int2 ce = I.rcell[j];
        cpa4(&I.rb[j], &start[(int64_t)r * ncells + ce.x]);
        cpa4(&I.re[j], &start[(int64_t)r * ncells + ce.y]);
    }
    cpa_commit();
}

template <int DEG>
__global__ void __launch_bounds__(RB_T, 4)
    k_real_blk(RbInputs in, RbGrid gr, int ncells, const int* __restrict__ start, const float4* __restrict__ sorted,
               const float4* __restrict__ tab, RealPoly rp, int m, int64_t n, int* __restrict__ rqueue,
               double* __restrict__ out) {
    __shared__ RbShared sm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float rc2 = rp.rc2;
    const float inv_h = gr.inv_h;
    const int nitems = in.nchunks * m;
    uint64_t C[DEG + 1];
#pragma unroll
    for (int k = 0; k <= DEG; ++k) C[k] = pk2(rp.c[k], rp.c[k]);
    float* fx = (float*)sm.cx;
    float* fy = (float*)sm.cy;
    float* fz = (float*)sm.cz;
    float* fq = (float*)sm.cq;
    if (tid == 0) sm.next = atomicAdd(&rqueue[0], 1);
    __syncthreads();
    RbItem& I = sm.it;
    for (;;) {
        const int item = sm.next;
        if (item >= nitems) break;   // uniform
        __syncthreads();             // every thread has read the item before the next one is taken
        if (tid == 0) {
            sm.next = atomicAdd(&rqueue[0], 1);
            I.item = item;
        }
        // the item's fixed inputs, then the charge ranges of its runs
        rb_fetch_static(I, in, item, m);
        cpa_wait_all();
        __syncthreads();
        rb_fetch_starts(I, start, ncells, m);
        cpa_wait_all();
        __syncthreads();
        const int r = item % m;
        const int4 ci = I.chunk;
        const float bx0 = I.box[0].x, by0 = I.box[0].y, bz0 = I.box[0].z;
        const float bx1 = I.box[1].x, by1 = I.box[1].y, bz1 = I.box[1].z;
        if (tid < 32) sm.acc[tid] = 0.f;
        // phase 1: exclusive block scan of the run lengths, two runs per thread
        const int nslots = ci.z;
        {
            const int i0 = 2 * tid, i1 = i0 + 1;
            const int l0 = i0 < nslots ? I.re[i0] - I.rb[i0] : 0, l1 = i1 < nslots ? I.re[i1] - I.rb[i1] : 0;
            int v = l0 + l1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            if (lane == 31) sm.wsum[warp] = v;
            __syncthreads();
            int wb = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < RB_W; ++w) {
                const int c = sm.wsum[w];
                wb += w < warp ? c : 0;
                tot += c;
            }
            const int ex = wb + v - l0 - l1;
            if (i0 < nslots) sm.rpre[i0] = ex;
            if (i1 < nslots) sm.rpre[i1] = ex + l0;
            if (tid == 0) sm.rpre[nslots] = tot;
        }
        __syncthreads();
        const int total = sm.rpre[nslots];
        for (int v0 = 0; v0 < total; v0 += RB_CAP) {
            // the run of every charge of this round
            const int vend = min(total, v0 + RB_CAP);
            for (int j = tid; j < nslots; j += RB_T) {
                const int vb = max(sm.rpre[j], v0), ve = min(sm.rpre[j + 1], vend);
                for (int v = vb; v < ve; ++v) sm.erun[v - v0] = (short)j;
            }
            __syncthreads();
            // phase 2: charge v0 + k RB_T + tid of the concatenated runs, all loads in flight
            const int kk = (vend - v0 + RB_T - 1) / RB_T;
            int e[RB_K];
            float4 q[RB_K];
#pragma unroll
            for (int k = 0; k < RB_K; ++k) {
                const int v = v0 + k * RB_T + tid;
                e[k] = -1;
                q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < kk && v < vend) {
                    e[k] = sm.erun[v - v0];
                    q[k] = sorted[I.rb[e[k]] + (v - sm.rpre[e[k]])];
                }
            }
            int rk[RB_K];
            unsigned keepbits = 0u;
            int wk = 0;   // kept by this warp in the slots before k
#pragma unroll
            for (int k = 0; k < RB_K; ++k) {
                if (k >= kk) break;   // uniform
                bool keep = false;
                if (e[k] >= 0) {
                    const float4 sh = I.rsh[e[k]];
                    q[k].x += sh.x;
                    q[k].y += sh.y;
                    q[k].z += sh.z;
                    // only charges within r_c of the sites' box can reach a site
                    const float ex = fmaxf(0.f, fmaxf(bx0 - q[k].x, q[k].x - bx1));
                    const float ey = fmaxf(0.f, fmaxf(by0 - q[k].y, q[k].y - by1));
                    const float ez = fmaxf(0.f, fmaxf(bz0 - q[k].z, q[k].z - bz1));
                    keep = ex * ex + ey * ey + ez * ez < rc2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                rk[k] = wk + __popc(bal & ((1u << lane) - 1u));
                wk += __popc(bal);
                keepbits |= keep ? 1u << k : 0u;
            }
            if (lane == 0) sm.wkept[warp] = wk;
            __syncthreads();
            int before = 0, nk = 0;
#pragma unroll
            for (int w = 0; w < RB_W; ++w) {
                const int c = sm.wkept[w];
                before += w < warp ? c : 0;
                nk += c;
            }
#pragma unroll
            for (int k = 0; k < RB_K; ++k) {
                if (k >= kk) break;   // uniform
                if (keepbits & (1u << k)) {
                    const int pos = before + rk[k];
                    fx[pos] = q[k].x;
                    fy[pos] = q[k].y;
                    fz[pos] = q[k].z;
                    fq[pos] = q[k].w;
                }
            }
            __syncthreads();
            if (nk > 0) {   // uniform
                // pad the list to whole 64-charge batches with zero charges at its last position
                const int nb = (nk + 63) >> 6;
                const float px = fx[nk - 1], py = fy[nk - 1], pz = fz[nk - 1];
                for (int k = nk + tid; k < (nb << 6); k += RB_T) {
                    fx[k] = px;
                    fy[k] = py;
                    fz[k] = pz;
                    fq[k] = 0.f;
                }
                __syncthreads();
                // phase 3: the (group, batch) work split into four equal contiguous ranges, one per
                // warp; a warp evaluates the part of each group its range covers and keeps the sums
                // in its own slot of that group (slots it does not reach stay zero)
                const int ngrp = (ci.y + 3) >> 2;
                const int work = ngrp * nb;
                sm.part[warp * RB_G + (lane >> 2)][lane & 3] = 0.f;
                __syncwarp();
                for (int f = warp * work / RB_W, f1 = (warp + 1) * work / RB_W; f < f1;) {
                    const int gi = f / nb, b0 = f - gi * nb, b1 = min(nb, b0 + (f1 - f));
                    rb_unit<DEG>(sm, I, gi, b0, b1, warp * RB_G + gi, C, rp, tab, inv_h);
                    f += b1 - b0;
                }
                __syncthreads();
                if (tid < ci.y) {
                    const int gi = tid >> 2, s = tid & 3;
                    float t = 0.f;
                    for (int w = 0; w < RB_W; ++w) t += sm.part[w * RB_G + gi][s];   // warp order
                    sm.acc[tid] += t;
                }
            }
            __syncthreads();   // the next round rewrites the list and the counts
        }
        if (tid < ci.y) out[(int64_t)r * n + I.sidx[tid]] = (double)sm.acc[tid];
    }
    // every take of this block is done; the last block to finish puts the queue back to zero for the
    // next launch (launches on one context are stream-ordered)
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&rqueue[1], 1) == (int)gridDim.x - 1) {
            atomicExch(&rqueue[0], 0);
            atomicExch(&rqueue[1], 0);
        }
    }
}

// ----------------------------------------------------------------------------- host
// The runs of every chunk: each stencil row (dy, dz) of the chunk's cell, trimmed to the sites' box
// grown by r_c (with a small margin, so no charge within r_c of the box is left out), split where it
// crosses the periodic boundary in x; empty rows are left out.  Arithmetic in FP32 on the FP32 box.
static cpm_status chunk_runs(cpm_ctx* c, const std::vector<int4>& chunks, const std::vector<float4>& sites,
                             float rc2, std::vector<int2>& cells, std::vector<float4>& shifts,
                             std::vector<int>& off) {
    const CellGrid cg = make_grid(c->g);
    const float hx = (float)cg.h[0], hy = (float)cg.h[1], hz = (float)cg.h[2];
    const float lx = (float)c->g.boxL[0], ly = (float)c->g.boxL[1], lz = (float)c->g.boxL[2];
    const int wy = 2 * cg.S[1] + 1, nrows = wy * (2 * cg.S[2] + 1);
    auto fdiv = [](int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    off.assign(1, 0);
    for (size_t ch = 0; ch < chunks.size(); ++ch) {
        float bx0 = sites[ch * 32].x, by0 = sites[ch * 32].y, bz0 = sites[ch * 32].z;
        float bx1 = bx0, by1 = by0, bz1 = bz0;
        for (int l = 1; l < 32; ++l) {
            const float4 v = sites[ch * 32 + l];
            bx0 = std::min(bx0, v.x); by0 = std::min(by0, v.y); bz0 = std::min(bz0, v.z);
            bx1 = std::max(bx1, v.x); by1 = std::max(by1, v.y); bz1 = std::max(bz1, v.z);
        }
        const int cell = chunks[ch].z;
        const int cx = cell % cg.nc[0], cy = (cell / cg.nc[0]) % cg.nc[1], cz = cell / (cg.nc[0] * cg.nc[1]);
        for (int row = 0; row < nrows; ++row) {
            const int dy = row % wy - cg.S[1], dz = row / wy - cg.S[2];
            const int uz = cz + dz, uy = cy + dy;
            const float dyd = std::max(0.f, std::max((float)uy * hy - by1, by0 - (float)(uy + 1) * hy));
            const float dzd = std::max(0.f, std::max((float)uz * hz - bz1, bz0 - (float)(uz + 1) * hz));
            const float rx2 = rc2 - dyd * dyd - dzd * dzd;
            if (!(rx2 > 0.f)) continue;
            const float rx = std::sqrt(rx2) * 1.0001f + 1e-3f;
            const int ux = std::max(cx - cg.S[0], (int)std::floor((bx0 - rx) / hx));
            const int uxe = std::min(cx + cg.S[0], (int)std::floor((bx1 + rx) / hx));
            if (ux > uxe) continue;
            const int fzz = fdiv(uz, cg.nc[2]), wz = uz - fzz * cg.nc[2];
            const int fyy = fdiv(uy, cg.nc[1]), wyy = uy - fyy * cg.nc[1];
            const int rowcell = (wz * cg.nc[1] + wyy) * cg.nc[0];
            for (int f = fdiv(ux, cg.nc[0]); f <= fdiv(uxe, cg.nc[0]); ++f) {
                const int a = std::max(ux, f * cg.nc[0]), e = std::min(uxe, f * cg.nc[0] + cg.nc[0] - 1);
                cells.push_back(make_int2(rowcell + a - f * cg.nc[0], rowcell + e - f * cg.nc[0] + 1));
                shifts.push_back(make_float4((float)f * lx, (float)fyy * ly, (float)fzz * lz, 0.f));
            }
        }
        if ((int)cells.size() - off.back() > RB_RUNS) return CPM_E_BUDGET;   // caller keeps the tabulated kernel
        off.push_back((int)cells.size());
    }
    return CPM_OK;
}

cpm_status build_real_poly(cpm_ctx* c, const std::vector<double>& etas) {
    void* old[] = {c->rsite, c->rsite_tab, c->rsite_idx, c->rbox, c->rrun_cell, c->rrun_sh, c->rchunk};
    for (void* p : old) dev_free(c, p);
    c->rsite = nullptr;
    c->rsite_tab = nullptr;
    c->rsite_idx = nullptr;
    c->rbox = nullptr;
    c->rrun_cell = nullptr;
    c->rrun_sh = nullptr;
    c->rchunk = nullptr;
    c->rrun_stride = 0;
    c->rpoly = RealPoly{};
    if (!c->schunks || !c->rtab || !c->rtab_id || c->nschunk == 0 || etas.empty()) return CPM_OK;
    // with Gaussian cores wider than half the cut-off most pairs would take the table: keep the
    // tabulated kernel for such electrodes
    const double emin = *std::min_element(etas.begin(), etas.end());
    if (!(RP_XETA / emin < 0.5 * c->g.rcut)) return CPM_OK;
    const double emax = *std::max_element(etas.begin(), etas.end());
    const RealPoly rp = fit_real_poly(c->g.alpha, c->g.rcut, RP_XETA / emax);
    if (rp.deg == 0) return CPM_OK;
    const size_t slots = (size_t)c->nschunk * 32;
    CPM_TRY(dev_alloc(c, (void**)&c->rsite, sizeof(float4) * slots));
    CPM_TRY(dev_alloc(c, (void**)&c->rsite_tab, sizeof(int) * slots));
    CPM_TRY(dev_alloc(c, (void**)&c->rsite_idx, sizeof(int) * slots));
    k_real_sites<<<(unsigned)((slots + 255) / 256), 256, 0, c->stream>>>(
        (const int4*)c->schunks, c->nschunk, c->sperm, c->s32, c->n, c->rtab_id, c->rsite, c->rsite_tab, c->rsite_idx);
    CPM_LAUNCH(c, "k_real_sites");
    // the runs from the same single-precision sites the kernel reads
    std::vector<float4> hs(slots);
    std::vector<int4> hch(c->nschunk);
    CPM_CUDA(c, cudaMemcpyAsync(hs.data(), c->rsite, sizeof(float4) * slots, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(hch.data(), c->schunks, sizeof(int4) * c->nschunk, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<int2> cells;
    std::vector<float4> shifts;
    std::vector<int> off;
    if (chunk_runs(c, hch, hs, rp.rc2, cells, shifts, off) != CPM_OK || cells.empty()) {
        dev_free(c, c->rsite);
        dev_free(c, c->rsite_tab);
        dev_free(c, c->rsite_idx);
        c->rsite = nullptr;
        c->rsite_tab = nullptr;
        c->rsite_idx = nullptr;
        return CPM_OK;   // a chunk with more runs than a block holds: the tabulated kernel runs
    }
    // runs at a fixed stride per chunk (empty runs past each chunk's count) and the chunk records
    int stride = 0;
    for (int ch = 0; ch < c->nschunk; ++ch) stride = std::max(stride, off[ch + 1] - off[ch]);
    std::vector<int2> pc((size_t)c->nschunk * stride, make_int2(0, 0));
    std::vector<float4> ps((size_t)c->nschunk * stride, make_float4(0.f, 0.f, 0.f, 0.f));
    std::vector<int4> rch(c->nschunk);
    std::vector<float4> box(2 * (size_t)c->nschunk);
    for (int ch = 0; ch < c->nschunk; ++ch) {
        float4 lo = hs[(size_t)ch * 32], hi = lo;
        for (int l = 1; l < 32; ++l) {
            const float4 v = hs[(size_t)ch * 32 + l];
            lo.x = std::min(lo.x, v.x); lo.y = std::min(lo.y, v.y); lo.z = std::min(lo.z, v.z);
            hi.x = std::max(hi.x, v.x); hi.y = std::max(hi.y, v.y); hi.z = std::max(hi.z, v.z);
        }
        lo.w = hi.w = 0.f;
        box[2 * (size_t)ch] = lo;
        box[2 * (size_t)ch + 1] = hi;
        for (int j = off[ch]; j < off[ch + 1]; ++j) {
            pc[(size_t)ch * stride + j - off[ch]] = cells[j];
            ps[(size_t)ch * stride + j - off[ch]] = shifts[j];
        }
        rch[ch] = make_int4(hch[ch].x, hch[ch].y, off[ch + 1] - off[ch], 0);
    }
    CPM_TRY(dev_alloc(c, (void**)&c->rrun_cell, sizeof(int2) * pc.size()));
    CPM_TRY(dev_alloc(c, (void**)&c->rrun_sh, sizeof(float4) * ps.size()));
    CPM_TRY(dev_alloc(c, (void**)&c->rchunk, sizeof(int4) * rch.size()));
    CPM_TRY(dev_alloc(c, (void**)&c->rbox, sizeof(float4) * box.size()));
    CPM_CUDA(c, cudaMemcpyAsync(c->rbox, box.data(), sizeof(float4) * box.size(), cudaMemcpyHostToDevice, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(c->rrun_cell, pc.data(), sizeof(int2) * pc.size(), cudaMemcpyHostToDevice, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(c->rrun_sh, ps.data(), sizeof(float4) * ps.size(), cudaMemcpyHostToDevice, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(c->rchunk, rch.data(), sizeof(int4) * rch.size(), cudaMemcpyHostToDevice, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->rrun_stride = stride;
    int dev = 0, nsm = 0, occ = 0;
    CPM_CUDA(c, cudaGetDevice(&dev));
    CPM_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (rp.deg == 12)
        CPM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_real_blk<12>, RB_T, 0));
    else
        CPM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_real_blk<14>, RB_T, 0));
    c->rpoly = rp;
    c->rpoly_blocks = std::max(1, occ) * std::max(1, nsm);
    return CPM_OK;
}

cpm_status real_poly_run(cpm_ctx* c, cudaStream_t st, int m, const CellGrid& cg, const int* start,
                         const float4* sorted, double* out) {
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->nschunk * m, c->rpoly_blocks));
    const float4* tab = (const float4*)c->rtab;
    RbGrid gr;
    gr.inv_h = (float)(RT_N / c->g.rcut);
    RbInputs in;
    in.site = c->rsite;
    in.sidx = c->rsite_idx;
    in.toff = c->rsite_tab;
    in.box = c->rbox;
    in.chunk = c->rchunk;
    in.rcell = c->rrun_cell;
    in.rsh = c->rrun_sh;
    in.stride = c->rrun_stride;
    in.nchunks = c->nschunk;
    if (c->rpoly.deg == 12)
        k_real_blk<12><<<grid, RB_T, 0, st>>>(in, gr, cg.ncells, start, sorted, tab, c->rpoly, m, c->n, c->rqueue, out);
    else
        k_real_blk<14><<<grid, RB_T, 0, st>>>(in, gr, cg.ncells, start, sorted, tab, c->rpoly, m, c->n, c->rqueue, out);
    CPM_LAUNCH(c, "k_real_blk");
    return CPM_OK;
}

}  // namespace cpm
