// Reciprocal-space part of the electrolyte vector b on the 5th-generation tensor cores.
//
// The Ewald sum of b over the half-space k set (Sec. II.E, Gaussian electrode charges of
// Sec. III.B) factorises over the column layout of the k grid (column c = (nx, ny), harmonic
// nz, phase tables X, Y, Z of the Cartesian components):
//
//   stage 1  rho_r[c][nz] = sum_j P_r[c][j] Z_j[nz],        P_r[c][j] = Q_j X_j[nx_c] Y_j[ny_c]
//   stage 2  T_r[c][i]    = sum_nz conj(Z_i[nz]) W_r[c][nz],  W_r = w rho_r
//            b_r[i]      += sum_c Re[ conj(X_i[nx_c] Y_i[ny_c]) T_r[c][i] ]
//
// Both stages are dense complex contractions (over the charges j, then over the harmonics nz),
// so they run as real matrix products with (re, im) interleaved along K and N:
//   stage 1: A = P (rows c, K = (j, re/im)), B rows (nz, re) = (Zr, -Zi), (nz, im) = (Zi, Zr)
//   stage 2: A = site phases (rows i, K = (nz, re/im)), B rows (c, r, re) = (Wr, Wi),
//            (c, r, im) = (Wi, -Wr); the epilogue contracts over c with conj(X_i Y_i).
//
// Operand precision: every operand x is scaled by a power of two s (|s x| < 2^14) and split as
// x0 = fp16(s x), x1 = fp16(s x - x0) (22 significant bits); the products x0 y0 + x0 y1 + x1 y0
// are accumulated in FP32 in tensor memory and the scales are removed exactly afterwards.  The
// k_perp = 0 column keeps its double-float treatment (its single-precision weight is zero here).
//
// Stage 1 builds both operand tiles in shared memory from the phase tables (128 columns x 32
// charges of P, 2 x 128 harmonic rows x 32 charges of Z per K step, 128-byte swizzle); stage 2
// streams its operands with TMA.  One thread issues the tcgen05.mma instructions; every
// mbarrier wait is bounded by wall time and on expiry the CTA records ST_TIMEOUT, frees its
// tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tc_common.cuh"

namespace cpm {

constexpr uint64_t RT_WAIT_NS = 2000000000ull;   // bound on any single mbarrier wait: 2 s

// stage 1 (structure factor)
constexpr int RF_BM = 128;                     // columns per tile (MMA M)
constexpr int RF_ZT = 128;                     // harmonics per tile (MMA N = 2 x 128)
constexpr int RF_KC = 32;                      // charges per K step (64 fp16 = 128 bytes per row)
constexpr int RF_GEN = 512;                    // operand-building threads (warps 0-15)
constexpr int RF_THREADS = RF_GEN + 32;        // + the MMA warp
constexpr int RF_ROWSTEP = RF_GEN / 8;         // tile rows covered by one pass of the builders
constexpr int RF_PK = RF_BM / RF_ROWSTEP;      // P rows per builder
constexpr int RF_ZK = RF_ZT / RF_ROWSTEP;      // Z row pairs per builder
constexpr int RF_A = RF_BM * 128;              // one fp16 term of the P tile (16 KB)
constexpr int RF_B = 2 * RF_ZT * 128;          // one fp16 term of the Z tile (32 KB)
constexpr int RF_STAGE = 2 * RF_A + 2 * RF_B;  // 96 KB
constexpr int RF_STAGES = 2;
constexpr int RF_XYROWS = 60;                 // staged phase-table rows: (NX + 1) + (2 NY + 1) at most
constexpr int RF_STAGE_XY = (RF_XYROWS + 1) * RF_KC * 8;   // X, Y rows and Q of one K step
constexpr int RF_PX = ((RF_XYROWS + 1) * RF_KC + RF_GEN - 1) / RF_GEN;   // staging entries per builder
constexpr int RF_QSLOT = 1 << 16;              // staging slots at or above this are charges
constexpr int RF_SMEM = 1024 + RF_STAGES * RF_STAGE + 2048 + RF_STAGE_XY;
constexpr float RF_ZSCALE = TC_ZSCALE;         // charge phases scaled by 2^14 (in the table)

// stage 2 (site potentials)
constexpr int RS_BM = 128;                     // sites per tile (MMA M)
constexpr int RS_EPI = 8;                      // epilogue warps (two per TMEM lane quarter)
constexpr int RS_THREADS = 32 * (RS_EPI + 2);   // warps 0-7 epilogue, warp 8 TMA, warp 9 MMA
constexpr int RS_TMA_WARP = RS_EPI, RS_MMA_WARP = RS_EPI + 1;
constexpr int RS_A = RS_BM * 128;              // one fp16 term of the site-phase tile (16 KB)
constexpr int RS_BMAX = 256 * 128;             // one fp16 term of the W tile, N <= 256 (32 KB)
constexpr int RS_STAGE = 2 * RS_A + 2 * RS_BMAX;
constexpr int RS_STAGES = 2;
constexpr int RS_SMEM = 1024 + RS_STAGES * RS_STAGE + 256;
constexpr int RS_ZEXP = 14;                    // site phases scaled by 2^14
constexpr int RS_CT = 16;                      // columns per group (N = 2 x 16 x replicas of the group)
constexpr int RS_MR = 8;                       // replicas per group

// 2^e with bound * 2^e < 2^top; 1 for a zero or non-finite bound
__device__ __forceinline__ float pow2_below(float bound, int top) {
    if (!(bound > 0.f) || !isfinite(bound)) return 1.f;
    int e;
    frexpf(bound, &e);   // bound = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, top - e);
}

// (re, im) -> two packed fp16 pairs: hi = fp16(v), lo = fp16(v - hi); low half = re
__device__ __forceinline__ void split2(float2 v, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(v.x, v.y);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(v.x - f.x, v.y - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}
__device__ __forceinline__ uint32_t neg_hi(uint32_t h) { return h ^ 0x80000000u; }            // (a, b) -> (a, -b)
__device__ __forceinline__ uint32_t swap_h(uint32_t h) { return __byte_perm(h, 0u, 0x1032); }  // (a, b) -> (b, a)

// barrier 1 over the RF_GEN operand-building threads; returns the AND of every thread's flag
__device__ __forceinline__ bool gen_bar_and(bool flag) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(out)
        : "r"((uint32_t)flag), "n"(RF_GEN)
        : "memory");
    return out != 0;
}
__device__ __forceinline__ void gen_bar() { asm volatile("bar.sync 1, %0;" ::"n"(RF_GEN) : "memory"); }

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
// byte offset of 16-byte chunk ch of row r in a K-major tile of 128-byte rows, 128-byte swizzle
__device__ __forceinline__ uint32_t sw128(int r, int ch) { return (uint32_t)(r * 128 + ((ch ^ (r & 7)) << 4)); }

// ----------------------------------------------------------------------------- stage 1
// part[s][r][zi][c] = 2^14 sA_r sum over the charges of split s of P_r[c][j] Z_j[zi]   (zi = nz + NZ)
// grid (column tiles, harmonic tiles, m * splits); sA_r = 2^e with |Q| sA_r < 2^14.
// largest harmonic extent of each 128-column tile, known on the host (fixed with the k set)
struct TileMx {
    int n;          // number of tiles given; 0: the kernel finds the extents itself
    int mx[32];
};

__global__ void __launch_bounds__(RF_THREADS, 1)
    k_tc_sf(const int2* __restrict__ cols, const int* __restrict__ colext, int ncols, int NX, int NY, int NZ, int nzw,
            const float2* __restrict__ EX, const float2* __restrict__ EY, const float2* __restrict__ EZ,
            const float* __restrict__ Qv, const float2* __restrict__ qabs, int64_t ptot, int64_t ne, int splits,
            int64_t chunk, int m, int cpad, const __grid_constant__ TileMx tmx, float2* __restrict__ part,
            unsigned* __restrict__ status, uint64_t wait_ns) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint8_t* aux = smem + RF_STAGES * RF_STAGE;
    uint64_t* full = (uint64_t*)aux;
    uint64_t* empty = full + RF_STAGES;
    uint64_t* done = empty + RF_STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort = (volatile int*)(tmem_slot + 1);
    int* s_mx = (int*)(tmem_slot + 2);
    int2* s_cols = (int2*)(aux + 64);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * RF_BM;
    const int r = blockIdx.z / splits, sp = blockIdx.z % splits;

    int mx;
    if ((int)blockIdx.x < tmx.n) {
        mx = tmx.mx[blockIdx.x];
    } else {
        if (warp == 0) {
            int v = -1;
            for (int t = lane; t < RF_BM; t += 32)
                if (c0 + t < ncols) v = max(v, colext[c0 + t]);
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) *s_mx = v;
        }
        __syncthreads();
        mx = *s_mx;
    }
    const int zoff = blockIdx.y * RF_ZT;
    const int zcount = min(RF_ZT, 2 * mx + 1 - zoff);
    if (mx < 0 || zcount <= 0) return;   // block-uniform; nothing allocated yet
    const int z_lo = NZ - mx + zoff;     // grid index of the tile's first harmonic
    const int nused = ((2 * zcount + 15) / 16) * 16;
    const int64_t jb = (int64_t)r * ne + (int64_t)sp * chunk;
    const int64_t je = min((int64_t)r * ne + ne, jb + chunk);
    const int nsteps = je > jb ? (int)((je - jb + RF_KC - 1) / RF_KC) : 0;
    const int rem0 = (int)max((int64_t)0, je - jb);   // charges of this split

    // Operand builders.  Thread g owns 16-byte chunk ch = g % 8 (charges 4 ch .. 4 ch + 3 of the step)
    // of P rows g / 8 + 64 k and of Z row pairs g / 8 + 64 k.  The X and Y table rows and the charges
    // of a step are staged in shared memory; the loads of step t + 1 (staging entries and Z values)
    // are issued before the tiles of step t are built.  Within a staged table row, charge 4 ch + u sits
    // at 16 (u / 2) + 2 ch + u % 2, so that the eight threads of a quarter warp (one P row) read two
    // 128-byte runs with two 16-byte loads each; the charges are a row of 32 floats in natural order.
    // Every source address and staging slot of a thread is fixed for the split and advances by one
    // step (32 charges) at a time, so it is computed once here.
    const int g = threadIdx.x, ch = g & 7, rbase = g >> 3;
    const int xyrows = (NX + 1) + (2 * NY + 1);
    const int nst = (xyrows + 1) * RF_KC;
    float2* sxy = (float2*)(aux + 2048);
    float* sqf = (float*)(sxy + xyrows * RF_KC);
    const bool vec = (ne & 1) == 0;   // then every Z run of a thread starts on a 16-byte boundary
    // entry k of this thread is charge jj = g % 32 of staged row (g + RF_GEN k) / 32; xdst: its slot
    // in the staged table rows, or RF_QSLOT + jj for the charge row, or -1 past the last row
    const int xjj = g & 31;
    const float2* xsrc[RF_PX];
    int xdst[RF_PX];
    const float2* zsrc[RF_ZK];
    bool zlive[RF_ZK];
    float sA = 1.f;
    float2 px[RF_PX], pz[RF_ZK][4];
    auto prefetch = [&](int t) {
        const int o = t * RF_KC;
#pragma unroll
        for (int k = 0; k < RF_PX; ++k) {
            float2 v = make_float2(0.f, 0.f);
            if (xdst[k] >= 0 && xjj + o < rem0)
                v = xdst[k] < RF_QSLOT ? xsrc[k][o] : make_float2(reinterpret_cast<const float*>(xsrc[k])[o] * sA, 0.f);
            px[k] = v;
        }
        const int jt = o + 4 * ch;   // first charge of this thread's run, relative to the split
#pragma unroll
        for (int k = 0; k < RF_ZK; ++k) {
            if (!zlive[k]) {
#pragma unroll
                for (int u = 0; u < 4; ++u) pz[k][u] = make_float2(0.f, 0.f);
            } else if (vec && jt + 3 < rem0) {
                const float4 a01 = *reinterpret_cast<const float4*>(zsrc[k] + o);
                const float4 a23 = *reinterpret_cast<const float4*>(zsrc[k] + o + 2);
                pz[k][0] = make_float2(a01.x, a01.y);
                pz[k][1] = make_float2(a01.z, a01.w);
                pz[k][2] = make_float2(a23.x, a23.y);
                pz[k][3] = make_float2(a23.z, a23.w);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) pz[k][u] = jt + u < rem0 ? zsrc[k][o + u] : make_float2(0.f, 0.f);
            }
        }
    };
    if (warp < RF_GEN / 32) {
        sA = pow2_below(qabs[r].x, 14);
#pragma unroll
        for (int k = 0; k < RF_PX; ++k) {
            const int e = g + RF_GEN * k, row = e >> 5, jj = xjj;
            xdst[k] = e >= nst ? -1
                    : row < xyrows ? row * RF_KC + (((jj & 2) << 3) | ((jj >> 2) << 1) | (jj & 1)) : RF_QSLOT + jj;
            xsrc[k] = row <= NX ? EX + (int64_t)row * ptot + jb + jj
                    : row < xyrows ? EY + (int64_t)(row - NX - 1) * ptot + jb + jj
                                   : reinterpret_cast<const float2*>(Qv + jb + jj);
        }
#pragma unroll
        for (int k = 0; k < RF_ZK; ++k) {
            const int zr = rbase + RF_ROWSTEP * k;
            zlive[k] = zr < zcount;
            zsrc[k] = EZ + (int64_t)(z_lo + min(zr, zcount - 1)) * ptot + jb + 4 * ch;
        }
        if (nsteps > 0) prefetch(0);   // in flight during the set-up below
    }

    if (threadIdx.x < RF_BM) s_cols[threadIdx.x] = c0 + (int)threadIdx.x < ncols ? cols[c0 + threadIdx.x] : make_int2(0, 0);
    if (threadIdx.x == 0) {
        for (int s = 0; s < RF_STAGES; ++s) { mbar_init(&full[s], RF_GEN); mbar_init(&empty[s], 1); }
        mbar_init(done, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == RF_GEN / 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < RF_GEN / 32) {
        for (int t = 0; t < nsteps; ++t) {
            const int s = t % RF_STAGES;
            bool ok = true;
            if (t >= RF_STAGES) ok = mbar_wait(&empty[s], ((t / RF_STAGES) - 1) & 1, abort, wait_ns);
            if (!gen_bar_and(ok)) break;   // uniform; also: everyone is done reading the staged step t - 1
#pragma unroll
            for (int k = 0; k < RF_PX; ++k) {
                if (xdst[k] >= RF_QSLOT) sqf[xdst[k] - RF_QSLOT] = px[k].x;
                else if (xdst[k] >= 0) sxy[xdst[k]] = px[k];
            }
            const uint32_t sa = su32(smem + s * RF_STAGE);
            const uint32_t sb = sa + 2 * RF_A;
            // the Z tile needs nothing staged: built from registers before they take the next step
#pragma unroll
            for (int k = 0; k < RF_ZK; ++k) {
                const int zr = rbase + RF_ROWSTEP * k;
                if (zr >= zcount) continue;
                uint32_t h[4], l[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    split2(pz[k][u], h[u], l[u]);   // the table holds 2^14 Z
                const uint32_t o0 = sw128(2 * zr, ch), o1 = sw128(2 * zr + 1, ch);
                sts128(sb + o0, neg_hi(h[0]), neg_hi(h[1]), neg_hi(h[2]), neg_hi(h[3]));
                sts128(sb + o1, swap_h(h[0]), swap_h(h[1]), swap_h(h[2]), swap_h(h[3]));
                sts128(sb + RF_B + o0, neg_hi(l[0]), neg_hi(l[1]), neg_hi(l[2]), neg_hi(l[3]));
                sts128(sb + RF_B + o1, swap_h(l[0]), swap_h(l[1]), swap_h(l[2]), swap_h(l[3]));
            }
            gen_bar();   // the staged rows of step t are complete
            if (t + 1 < nsteps) prefetch(t + 1);
            const float4 q4 = reinterpret_cast<const float4*>(sqf)[ch];
            const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
            for (int k = 0; k < RF_PK; ++k) {
                const int row = rbase + RF_ROWSTEP * k;
                const int2 cn = s_cols[row];
                const bool live = c0 + row < ncols;
                float2 x[4], y[4];
                if (live) {
                    const float4* xr = reinterpret_cast<const float4*>(sxy + cn.x * RF_KC);
                    const float4* yr = reinterpret_cast<const float4*>(sxy + (NX + 1 + cn.y + NY) * RF_KC);
                    const float4 x01 = xr[ch], x23 = xr[8 + ch], y01 = yr[ch], y23 = yr[8 + ch];
                    x[0] = make_float2(x01.x, x01.y); x[1] = make_float2(x01.z, x01.w);
                    x[2] = make_float2(x23.x, x23.y); x[3] = make_float2(x23.z, x23.w);
                    y[0] = make_float2(y01.x, y01.y); y[1] = make_float2(y01.z, y01.w);
                    y[2] = make_float2(y23.x, y23.y); y[3] = make_float2(y23.z, y23.w);
                }
                uint32_t h[4], l[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float2 p = make_float2(0.f, 0.f);
                    if (live)
                        p = make_float2((x[u].x * y[u].x - x[u].y * y[u].y) * qv[u],
                                        (x[u].x * y[u].y + x[u].y * y[u].x) * qv[u]);
                    split2(p, h[u], l[u]);
                }
                const uint32_t off = sw128(row, ch);
                sts128(sa + off, h[0], h[1], h[2], h[3]);
                sts128(sa + RF_A + off, l[0], l[1], l[2], l[3]);
            }
            fence_async_smem();
            mbar_arrive(&full[s]);
        }
    } else if (lane == 0) {
        // MMA issuer: per 16-wide K slice the products P0 Z0 + P0 Z1 + P1 Z0
        const uint32_t idesc = idesc_f16(RF_BM, nused);
        for (int t = 0; t < nsteps; ++t) {
            const int s = t % RF_STAGES;
            if (!mbar_wait(&full[s], (t / RF_STAGES) & 1, abort, wait_ns)) break;
            tc_fence_after();
            const uint32_t sa = su32(smem + s * RF_STAGE), sb = sa + 2 * RF_A;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t a0 = sdesc_sw128(sa + kk * 32), a1 = sdesc_sw128(sa + RF_A + kk * 32);
                const uint64_t b0 = sdesc_sw128(sb + kk * 32), b1 = sdesc_sw128(sb + RF_B + kk * 32);
                umma_f16(tmem, a0, b0, idesc, (t > 0 || kk > 0) ? 1u : 0u);
                umma_f16(tmem, a0, b1, idesc, 1u);
                umma_f16(tmem, a1, b0, idesc, 1u);
            }
            umma_commit(&empty[s]);
        }
        umma_commit(done);   // also after an abort: the epilogue then waits for the MMAs in flight
    }
    if (warp < RF_GEN / 32) {
        // epilogue on all builder warps: warp w reads accumulator lanes 32 (w % 4) .. + 31 (its columns)
        // and accumulator columns 16 (w / 4) + 64 i (eight harmonics each)
        const bool ok = mbar_wait(done, 0, abort, wait_ns);
        tc_fence_after();
        const bool good = __all_sync(0xffffffffu, ok && !*abort) != 0;
        if (good) {
            const int lq = warp & 3, cg = warp >> 2;
            const int c = c0 + lq * 32 + lane;
            float2* out = part + ((int64_t)sp * m + r) * nzw * cpad + c;
            const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16);
            for (int q0 = 16 * cg; q0 < nused; q0 += 64) {
                float v[16];
                if (nsteps > 0) {
                    tmem_ld16(trow + q0, v);
                } else {
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] = 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int zz = q0 / 2 + u;
                    if (zz < zcount) out[(int64_t)(z_lo + zz) * cpad] = make_float2(v[2 * u], v[2 * u + 1]);
                }
            }
        } else if (lane == 0) {
            atomicOr(status, ST_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == RF_GEN / 32) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
    }
}

// ----------------------------------------------------------------------------- between the stages
// W planes (two fp16 terms) of the site stage from the split structure factors:
//   W_r[c][zi] = sW_r w[c][zi] (sum_s part[s][r][zi][c]) / (2^14 sA_r)   (zero outside the k set)
// row (group g, pair p, re) = (Wr, Wi) and row (.., im) = (Wi, -Wr) at K = 2 zi, 2 zi + 1.
// Groups hold CT columns x mr replicas: g = (r / mr) ncb + c / CT, p = (r % mr) CT + c % CT.
// One block transposes a 32-harmonic x 32-column tile of one replica slot.
__global__ void __launch_bounds__(1024)
    k_tc_wsplit(const float2* __restrict__ part, int splits, int m, int cpad, int nzw, int NZ,
                const int* __restrict__ colext, const float* __restrict__ w32, int ncols,
                const float2* __restrict__ qabs, float wmax, int CT, int mr, int ncb, int NB, int KZ,
                uint32_t* __restrict__ w16, int64_t plane_words) {
    __shared__ float2 tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int zb = blockIdx.x * 32, cb0 = blockIdx.y * 32, rp = blockIdx.z;
    const bool rlive = rp < m;
    {
        const int zi = zb + ty, c = cb0 + tx;
        float2 W = make_float2(0.f, 0.f);
        if (rlive && c < ncols && zi < nzw) {
            const int ext = colext[c], nz = zi - NZ;
            const float wt = w32[(int64_t)c * nzw + zi];
            if (nz >= -ext && nz <= ext && wt != 0.f) {
                const float2 qa = qabs[rp];
                const float f = pow2_below(wmax * qa.y, 14) / (pow2_below(qa.x, 14) * RF_ZSCALE);
                float sx = 0.f, sy = 0.f;
                const float2* pp = part + ((int64_t)rp * nzw + zi) * cpad + c;
                const int64_t sstride = (int64_t)m * nzw * cpad;
                int s = 0;
                for (; s + 8 <= splits; s += 8) {   // eight loads in flight, added in split order
                    float2 v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = pp[(s + k) * sstride];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        sx += v[k].x;
                        sy += v[k].y;
                    }
                }
                for (; s < splits; ++s) {
                    const float2 v = pp[s * sstride];
                    sx += v.x;
                    sy += v.y;
                }
                W = make_float2(sx * wt * f, sy * wt * f);
            }
        }
        tile[ty][tx] = W;
    }
    __syncthreads();
    const int rb = rp / mr, rr = rp % mr;
    const int kw = KZ / 2;
    const int c = cb0 + ty, zi = zb + tx;
    if (c >= ncb * CT || zi >= kw) return;
    const int64_t row = (int64_t)(rb * ncb + c / CT) * NB + 2 * (rr * CT + c % CT);
    uint32_t h, l;
    split2(tile[tx][ty], h, l);
    const int64_t w0 = row * kw + zi;
    w16[w0] = h;
    w16[w0 + kw] = neg_hi(swap_h(h));
    w16[plane_words + w0] = l;
    w16[plane_words + w0 + kw] = neg_hi(swap_h(l));
}

// ----------------------------------------------------------------------------- stage 2
struct SiteMaps {
    CUtensorMap a[2];
    CUtensorMap b[2];
};

// K steps (64 wide) covering the harmonics zi in [NZ - mx, NZ + mx] of column group g (two K entries
// per harmonic), mx = the largest harmonic extent of the group's columns; nsteps = 0 for no column
__device__ __forceinline__ void site_group_steps(const int* __restrict__ colext, int ncols, int NZ, int g, int ncb,
                                                 int& t0, int& nsteps) {
    const int cb = g % ncb;
    const int cfirst = cb * RS_CT, clast = min(ncols, cfirst + RS_CT);
    int mx = -1;
    for (int c = cfirst; c < clast; ++c) mx = max(mx, colext[c]);
    t0 = mx >= 0 ? (2 * (NZ - mx)) / 64 : 0;
    nsteps = mx >= 0 ? (2 * (NZ + mx + 1) + 63) / 64 - t0 : 0;
}

// partial[r][cb][i] = sum over the 16 columns of block cb of Re[conj(X_i Y_i) T_r[c][i]]
// Persistent: CTA b takes the tiles tau = b, b + gridDim.x, ... of the (site tile, group) grid, in
// group-major order (groups of low |k_perp| have the most harmonics and come first); group g holds
// mr <= 8 replicas x 16 columns.  Two accumulators in tensor memory (columns 256 buf + 32 rr + 2 cc
// + {re, im}): the epilogue warps read tile k from one while the MMA thread fills the other with
// tile k + 1; tfull[buf] / tempty[buf] hand the buffers over.
__global__ void __launch_bounds__(RS_THREADS, 1)
    k_tc_site(const __grid_constant__ SiteMaps maps, const int* __restrict__ colext, int ncols, int NZ,
              int mr, int ncb, int NB, int m, int ntx, int ntiles, const float2* __restrict__ XY, int64_t n,
              const float2* __restrict__ qabs, float wmax, float* __restrict__ partial,
              unsigned* __restrict__ status, uint64_t wait_ns) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = align1024(smem_raw);
    uint64_t* full = (uint64_t*)(smem + RS_STAGES * RS_STAGE);
    uint64_t* empty = full + RS_STAGES;
    uint64_t* tfull = empty + RS_STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* done = tempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < RS_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], RS_EPI); }
        mbar_init(done, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == RS_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t stage_bytes = 2 * RS_A + 2 * NB * 128;

    if (warp == RS_TMA_WARP && lane == 0) {
        // TMA producer: one ring over the K steps of all this CTA's tiles
        int it = 0;
        for (int tau = blockIdx.x; tau < ntiles && !*abort; tau += gridDim.x) {
            const int g = tau / ntx, tx = tau % ntx;
            int t0, nsteps;
            site_group_steps(colext, ncols, NZ, g, ncb, t0, nsteps);
            for (int t = 0; t < nsteps; ++t, ++it) {
                const int s = it % RS_STAGES;
                if (it >= RS_STAGES && !mbar_wait(&empty[s], ((it / RS_STAGES) - 1) & 1, abort, wait_ns)) break;
                uint8_t* st = smem + s * RS_STAGE;
                mbar_expect_tx(&full[s], stage_bytes);
                const int kx = (t0 + t) * 64;
                tma_load_2d(st, &maps.a[0], kx, tx * RS_BM, &full[s]);
                tma_load_2d(st + RS_A, &maps.a[1], kx, tx * RS_BM, &full[s]);
                tma_load_2d(st + 2 * RS_A, &maps.b[0], kx, g * NB, &full[s]);
                tma_load_2d(st + 2 * RS_A + RS_BMAX, &maps.b[1], kx, g * NB, &full[s]);
            }
        }
        if (*abort) {
            // let the copies still in flight land (bounded): only the last RS_STAGES issued steps can be
            for (int t = max(0, it - RS_STAGES); t < it; ++t) {
                const int s = t % RS_STAGES;
                const uint64_t ts = gtimer_ns();
                while (!mbar_try(&full[s], (t / RS_STAGES) & 1) && gtimer_ns() - ts < wait_ns) {}
            }
        }
    } else if (warp == RS_MMA_WARP && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_f16(RS_BM, NB);
        int it = 0, k = 0;
        for (int tau = blockIdx.x; tau < ntiles; tau += gridDim.x, ++k) {
            const int g = tau / ntx;
            int t0, nsteps;
            site_group_steps(colext, ncols, NZ, g, ncb, t0, nsteps);
            const int buf = k & 1;
            if (k >= 2 && !mbar_wait(&tempty[buf], ((k >> 1) - 1) & 1, abort, wait_ns)) break;
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)(256 * buf);
            bool ok = true;
            for (int t = 0; t < nsteps; ++t, ++it) {
                const int s = it % RS_STAGES;
                if (!mbar_wait(&full[s], (it / RS_STAGES) & 1, abort, wait_ns)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = su32(smem + s * RS_STAGE), sb = sa + 2 * RS_A;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t a0 = sdesc_sw128(sa + kk * 32), a1 = sdesc_sw128(sa + RS_A + kk * 32);
                    const uint64_t b0 = sdesc_sw128(sb + kk * 32), b1 = sdesc_sw128(sb + RS_BMAX + kk * 32);
                    umma_f16(acc, a0, b0, idesc, (t > 0 || kk > 0) ? 1u : 0u);
                    umma_f16(acc, a0, b1, idesc, 1u);
                    umma_f16(acc, a1, b0, idesc, 1u);
                }
                umma_commit(&empty[s]);
            }
            if (!ok) break;
            umma_commit(&tfull[buf]);
        }
        umma_commit(done);   // also after an abort: the MMAs in flight complete before the dealloc
        const uint64_t ts = gtimer_ns();
        while (!mbar_try(done, 0) && gtimer_ns() - ts < wait_ns) {}
    } else if (warp < RS_EPI) {
        // epilogue: thread = site i of the tile, accumulator lane (warp % 4) * 32 + lane; warp w takes
        // the replicas of parity w / 4 of the group
        const int lq = warp & 3, rpar = warp >> 2;
        const uint32_t trow = (uint32_t)(lq * 32) << 16;
        const float zinv = ldexpf(1.f, -RS_ZEXP);
        int k = 0;
        for (int tau = blockIdx.x; tau < ntiles; tau += gridDim.x, ++k) {
            const int g = tau / ntx, tx = tau % ntx;
            const int rb = g / ncb, cb = g % ncb;
            const int cfirst = cb * RS_CT, clast = min(ncols, cfirst + RS_CT);
            int t0, nsteps;
            site_group_steps(colext, ncols, NZ, g, ncb, t0, nsteps);
            const int64_t i = (int64_t)tx * RS_BM + lq * 32 + lane;
            float2 xy[RS_CT];   // the column factors of this thread's site, loaded while the products run
#pragma unroll
            for (int u = 0; u < RS_CT; ++u) {
                const int c = cfirst + u;
                xy[u] = (c < clast && i < n) ? XY[(int64_t)c * n + i] : make_float2(0.f, 0.f);
            }
            const int buf = k & 1;
            const bool ok = mbar_wait(&tfull[buf], (k >> 1) & 1, abort, wait_ns);
            tc_fence_after();
            if (__any_sync(0xffffffffu, !ok || *abort)) break;
            for (int rr = rpar; rr < mr; rr += RS_EPI / 4) {
                float v[2 * RS_CT];
                if (nsteps > 0) {
                    tmem_ld32(tmem + trow + (uint32_t)(256 * buf + 2 * RS_CT * rr), v);
                } else {
#pragma unroll
                    for (int q = 0; q < 2 * RS_CT; ++q) v[q] = 0.f;
                }
                float sacc = 0.f;
#pragma unroll
                for (int u = 0; u < RS_CT; ++u) {
                    sacc = fmaf(xy[u].x, v[2 * u], sacc);
                    sacc = fmaf(xy[u].y, v[2 * u + 1], sacc);
                }
                const int r = rb * mr + rr;
                if (r < m && i < n)
                    partial[((int64_t)r * ncb + cb) * n + i] = sacc * (zinv / pow2_below(wmax * qabs[r].y, 14));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        if (*abort && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (*abort && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    if (warp == RS_MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

// ----------------------------------------------------------------------------- fixed site operands
// a[q][i][2 zi + {0,1}] = term q of 2^14 (Re, Im) Z_i[zi], split in FP64; zero padding rows/columns
__global__ void k_tc_site_a(const double2* __restrict__ Zs, int64_t n, int64_t npad, int nzw, int KZ,
                            uint32_t* __restrict__ a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int kw = KZ / 2;
    if (t >= npad * kw) return;
    const int64_t i = t / kw;
    const int zi = (int)(t % kw);
    const double2 z = (i < n && zi < nzw) ? Zs[(int64_t)zi * n + i] : make_double2(0.0, 0.0);
    const double zr = ldexp(z.x, RS_ZEXP), zm = ldexp(z.y, RS_ZEXP);
    const __half hr = __double2half(zr), hm = __double2half(zm);
    const __half lr = __double2half(zr - (double)__half2float(hr)), lm = __double2half(zm - (double)__half2float(hm));
    const __half2 h = __halves2half2(hr, hm), l = __halves2half2(lr, lm);
    a[t] = *reinterpret_cast<const uint32_t*>(&h);
    a[npad * kw + t] = *reinterpret_cast<const uint32_t*>(&l);
}

// xy[c][i] = X_i[nx_c] Y_i[ny_c] (FP64 product, rounded once)
__global__ void k_tc_site_xy(const double2* __restrict__ SX, const double2* __restrict__ SY,
                             const int2* __restrict__ cols, int ncols, int NY, int64_t n, float2* __restrict__ xy) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)ncols * n) return;
    const int c = (int)(t / n);
    const int64_t i = t % n;
    const int2 cn = cols[c];
    const double2 x = SX[(int64_t)cn.x * n + i], y = SY[(int64_t)(cn.y + NY) * n + i];
    xy[t] = make_float2((float)(x.x * y.x - x.y * y.y), (float)(x.x * y.y + x.y * y.x));
}

// ----------------------------------------------------------------------------- host side
bool tc_recip_supported(const KTable& k) { return k.nk > 0 && (k.NX + 1) + (2 * k.NY + 1) <= RF_XYROWS; }

TcRecipDims tc_recip_dims(const cpm_ctx* c, int m, int64_t ne) {
    const KTable& k = c->kt;
    TcRecipDims d;
    d.mtiles = (k.ncols + RF_BM - 1) / RF_BM;
    d.cpad = d.mtiles * RF_BM;
    d.ntiles = (k.nzw + RF_ZT - 1) / RF_ZT;
    const int base = std::max(1, d.mtiles * d.ntiles * m);
    const int64_t maxs = std::max<int64_t>(1, (ne + 4 * RF_KC - 1) / (4 * RF_KC));   // >= 4 K steps per CTA
    d.splits = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(1, 152 / base), maxs));
    d.chunk = (ne + d.splits - 1) / d.splits;
    d.chunk = ((d.chunk + RF_KC - 1) / RF_KC) * RF_KC;
    d.mr = std::min(m, RS_MR);
    d.nrb = (m + d.mr - 1) / d.mr;
    d.CT = RS_CT;
    d.ncb = (k.ncols + d.CT - 1) / d.CT;
    d.NB = 2 * d.CT * d.mr;
    d.ngroups = d.nrb * d.ncb;
    d.KZ = ((2 * k.nzw + 63) / 64) * 64;
    d.npad = ((c->n + RS_BM - 1) / RS_BM) * RS_BM;
    return d;
}

size_t tc_recip_part_bytes(const TcRecipDims& d, int m, int nzw) {
    return sizeof(float2) * (size_t)d.splits * m * nzw * d.cpad;
}
size_t tc_recip_w16_bytes(const TcRecipDims& d) { return 2 * sizeof(uint16_t) * (size_t)d.ngroups * d.NB * d.KZ; }

// site operands that stay fixed with the geometry: phase planes and column factors X_i Y_i
cpm_status tc_recip_prepare(cpm_ctx* c) {
    const KTable& k = c->kt;
    dev_free(c, c->tcz);
    dev_free(c, c->tcxy);
    c->tcz = nullptr;
    c->tcxy = nullptr;
    if (!tc_recip_supported(k)) return CPM_OK;
    const TcRecipDims d = tc_recip_dims(c, 1, 0);
    const int64_t n = c->n;
    CPM_TRY(dev_alloc(c, &c->tcz, sizeof(uint16_t) * 2 * (size_t)d.npad * d.KZ));
    CPM_TRY(dev_alloc(c, (void**)&c->tcxy, sizeof(float2) * (size_t)k.ncols * n));
    const int64_t ta = d.npad * (d.KZ / 2);
    k_tc_site_a<<<(unsigned)((ta + 255) / 256), 256, 0, c->stream>>>(c->site64.Z, n, d.npad, k.nzw, d.KZ,
                                                                    (uint32_t*)c->tcz);
    CPM_LAUNCH(c, "k_tc_site_a");
    const int64_t tx = (int64_t)k.ncols * n;
    k_tc_site_xy<<<(unsigned)((tx + 255) / 256), 256, 0, c->stream>>>(c->site64.X, c->site64.Y, k.cols, k.ncols, k.NY,
                                                                     n, c->tcxy);
    CPM_LAUNCH(c, "k_tc_site_xy");
    // bound on the weights: w_k <= (8 pi / V) / |k|^2 <= (8 pi / V) / k_min^2
    double kmin2 = 1e300;
    for (int a = 0; a < 3; ++a) {
        const double kk = 2.0 * PI * c->g.inv[a];
        kmin2 = std::min(kmin2, kk * kk);
    }
    c->tc_wmax = (float)(1.01 * 8.0 * PI / c->g.V / kmin2);
    // largest harmonic extent of each 128-column tile of the structure-factor stage
    c->tc_nmx = 0;
    if (d.mtiles <= 32) {
        std::vector<int> ext(k.ncols);
        CPM_CUDA(c, cudaMemcpyAsync(ext.data(), k.colext, sizeof(int) * k.ncols, cudaMemcpyDeviceToHost, c->stream));
        CPM_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int t = 0; t < d.mtiles; ++t) {
            int mx = -1;
            for (int cc = t * RF_BM; cc < std::min(k.ncols, (t + 1) * RF_BM); ++cc) mx = std::max(mx, ext[cc]);
            c->tc_mx[t] = mx;
        }
        c->tc_nmx = d.mtiles;
    }
    return CPM_OK;
}

cpm_status tc_recip_run(cpm_ctx* c, int m, int64_t ne, const float2* EX, const float2* EY, const float2* EZ,
                        const float* Qv, const float2* qabs, void* part, void* w16, float* site_partial) {
    const KTable& k = c->kt;
    const TcRecipDims d = tc_recip_dims(c, m, ne);
    cudaStream_t st = c->stream;
    const int64_t n = c->n, ptot = (int64_t)m * ne;
    if (!c->tcz || !c->tcxy) return set_err(c, CPM_E_STATE, "tensor-core reciprocal operands not prepared");

    prof_begin(c, CPM_K_SF);
    CPM_CUDA(c, cudaFuncSetAttribute(k_tc_sf, cudaFuncAttributeMaxDynamicSharedMemorySize, RF_SMEM));
    TileMx tmx;
    tmx.n = c->tc_nmx;
    for (int t = 0; t < 32; ++t) tmx.mx[t] = c->tc_mx[t];
    k_tc_sf<<<dim3(d.mtiles, d.ntiles, m * d.splits), RF_THREADS, RF_SMEM, st>>>(
        k.cols, k.colext, k.ncols, k.NX, k.NY, k.NZ, k.nzw, EX, EY, EZ, Qv, qabs, ptot, ne, d.splits, d.chunk, m, d.cpad,
        tmx, (float2*)part, c->status, RT_WAIT_NS);
    prof_end(c, CPM_K_SF);
    CPM_LAUNCH(c, "k_tc_sf");

    prof_begin(c, CPM_K_SFRED);
    const int64_t plane_words = (int64_t)d.ngroups * d.NB * (d.KZ / 2);
    if (d.NB != 2 * d.CT * d.mr) CPM_CUDA(c, cudaMemsetAsync(w16, 0, tc_recip_w16_bytes(d), st));
    dim3 gw((unsigned)((d.KZ / 2 + 31) / 32), (unsigned)((d.ncb * d.CT + 31) / 32), (unsigned)(d.nrb * d.mr));
    k_tc_wsplit<<<gw, 1024, 0, st>>>((const float2*)part, d.splits, m, d.cpad, k.nzw, k.NZ, k.colext, k.w32, k.ncols,
                                    qabs, c->tc_wmax, d.CT, d.mr, d.ncb, d.NB, d.KZ, (uint32_t*)w16, plane_words);
    prof_end(c, CPM_K_SFRED);
    CPM_LAUNCH(c, "k_tc_wsplit");

    prof_begin(c, CPM_K_SITE);
    SiteMaps maps;
    const uint16_t* za = (const uint16_t*)c->tcz;
    const uint16_t* wb = (const uint16_t*)w16;
    for (int q = 0; q < 2; ++q) {
        if (!make_map(&maps.a[q], za + (size_t)q * d.npad * d.KZ, d.npad, d.KZ, RS_BM, CU_TENSOR_MAP_DATA_TYPE_FLOAT16) ||
            !make_map(&maps.b[q], wb + (size_t)q * d.ngroups * d.NB * d.KZ, (int64_t)d.ngroups * d.NB, d.KZ, d.NB,
                      CU_TENSOR_MAP_DATA_TYPE_FLOAT16))
            return set_err(c, CPM_E_CUDA, "cuTensorMapEncodeTiled failed");
    }
    CPM_CUDA(c, cudaFuncSetAttribute(k_tc_site, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM));
    const int ntx = (int)(d.npad / RS_BM), ntiles = ntx * d.ngroups;
    k_tc_site<<<(unsigned)std::min(ntiles, 152), RS_THREADS, RS_SMEM, st>>>(
        maps, k.colext, k.ncols, k.NZ, d.mr, d.ncb, d.NB, m, ntx, ntiles, c->tcxy, n, qabs, c->tc_wmax, site_partial,
        c->status, RT_WAIT_NS);
    prof_end(c, CPM_K_SITE);
    CPM_LAUNCH(c, "k_tc_site");
    return CPM_OK;
}

}  // namespace cpm
