// Electrolyte vector b: the potential of the electrolyte point charges at every electrode
// site (Sec. II.A: the dominant cost of each MD step), for m electrolyte configurations at once.
//
//   b_i = K_E [ sum_j Q_j sum'_n (erfc(alpha r) - erfc(eta_i r)) / r     real space, cell list
//             + sum_k w_k Re[exp(-i k.R_i) rho(k)]                      reciprocal space
//             - pi Q_tot / (V alpha^2) + B_i ]                          background, Sec. II.E
//
// Reciprocal space in two contractions over the column layout of the k set
// (column c = (nx, ny), harmonic nz):
//   structure factor  rho[c][nz] = sum_j (Q_j X_j[nx_c] Y_j[ny_c]) Z_j[nz]
//   site potential    b_i      += sum_c Re[ conj(X_i[nx_c] Y_i[ny_c]) sum_nz w[c][nz] rho[c][nz] conj(Z_i[nz]) ]
// register-tiled on the CUDA cores here (k_prec FP64 and FP32), or as tensor-core products
// (k_prec F16X2, tc_recip.cu).
#include <algorithm>

#include "common.cuh"

namespace cpm {


template <typename T> struct V4;
template <> struct V4<float> { using t = float4; };
template <> struct V4<double> { using t = double4_32a; };

CellGrid make_grid(const Geometry& g) {
    CellGrid cg;
    for (int d = 0; d < 3; ++d) {
        int nc = (int)floor(g.boxL[d] / (g.rcut / 3.0));
        nc = std::max(1, std::min(nc, 256));
        cg.nc[d] = nc;
        cg.h[d] = g.boxL[d] / nc;
        cg.S[d] = (int)ceil(g.rcut / cg.h[d]);
    }
    cg.ncells = cg.nc[0] * cg.nc[1] * cg.nc[2];
    return cg;
}


// ----------------------------------------------------------------------------- per-replica totals
constexpr int ST_THREADS = 256;

// ----------------------------------------------------------------------------- cell list
// Binning and the per-replica totals in one pass: grid (charge blocks, m), one thread per charge.
// Each charge gets its wrapped position and its cell (cells of the real-space grid); each block sums
// (Q, Q x, Q y, Q z) over its charges into part[r][b][4], and the replica's last block adds the
// block sums in order (stats[r]).  Charges with Q = 0 (padding) get no cell (key -1) and are not
// counted: nzc[r] counts the replica's others, and the cell list holds only those.
constexpr int ST_Q = 4;   // totals per replica
template <typename T>
__global__ void __launch_bounds__(ST_THREADS) k_bin(const double* __restrict__ xyz, const double* __restrict__ Q,
                                                  int64_t ne, Geometry g, CellGrid cg, float3 inv_h, int* key,
                                                  int* count, typename V4<T>::t* wpos, double* part,
                                                  int* tickets, double* stats, int* nzc) {
    const int b = blockIdx.x, nb = gridDim.x, r = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j = (int64_t)b * ST_THREADS + threadIdx.x;
    double a[ST_Q] = {0, 0, 0, 0};
    if (j < ne) {
        const int64_t p = (int64_t)r * ne + j;
        const double q = Q[p];
        double w[3];
        int ci[3];
        const float ih[3] = {inv_h.x, inv_h.y, inv_h.z};
        for (int d = 0; d < 3; ++d) {
            const double x = xyz[3 * p + d];
            a[1 + d] = q * x;
            w[d] = x - g.boxL[d] * floor(x * g.inv[d]);
            if (w[d] >= g.boxL[d]) w[d] -= g.boxL[d];
            if (w[d] < 0) w[d] = 0;
            ci[d] = min(cg.nc[d] - 1, (int)((float)w[d] * ih[d]));
        }
        a[0] = q;
        const int k = r * cg.ncells + (ci[2] * cg.nc[1] + ci[1]) * cg.nc[0] + ci[0];
        key[p] = q != 0.0 ? k : -1;
        if (q != 0.0) atomicAdd(&count[k], 1);
        typename V4<T>::t v;
        v.x = (T)w[0]; v.y = (T)w[1]; v.z = (T)w[2]; v.w = (T)q;
        wpos[p] = v;
    }
    {   // nonzero charges of the replica, one atomic per warp
        const bool nz = j < ne && Q[(int64_t)r * ne + j] != 0.0;
        const unsigned bal = __ballot_sync(0xffffffffu, nz);
        if (lane == 0 && bal) atomicAdd(&nzc[r], __popc(bal));
    }
    // block sums in a fixed order: the thread values through shared memory, warp t of the first four
    // takes quantity t (each lane adds eight threads' values, then a shuffle tree)
    __shared__ double sv[ST_Q][ST_THREADS];
    for (int t = 0; t < ST_Q; ++t) sv[t][threadIdx.x] = a[t];
    __syncthreads();
    double* pr = part + ((int64_t)r * nb + b) * ST_Q;
    if (warp < ST_Q) {
        const int t = warp;
        double v = sv[t][lane];
        for (int k = 1; k < ST_THREADS / 32; ++k) v += sv[t][lane + 32 * k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) pr[t] = v;
    }
    if (!last_block_of(&tickets[r], nb)) return;
    // the block sums, ST_THREADS blocks at a time, loaded by all threads at once and added by
    // threads 0..3 in block order
    __shared__ double buf[ST_Q][ST_THREADS];
    const volatile double* pv = part + (int64_t)r * nb * ST_Q;
    double v = 0.0;
    for (int k0 = 0; k0 < nb; k0 += ST_THREADS) {
        const int k = k0 + threadIdx.x;
        if (k < nb)
            for (int t = 0; t < ST_Q; ++t) buf[t][threadIdx.x] = pv[k * ST_Q + t];
        __syncthreads();
        if (threadIdx.x < ST_Q) {
            const int t = threadIdx.x, cnt = min(ST_THREADS, nb - k0);
            for (int kk = 0; kk < cnt; ++kk) {
                const double x = buf[t][kk];
                v = (k0 == 0 && kk == 0) ? x : v + x;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < ST_Q) stats[4 * r + threadIdx.x] = v;
}

// Per-replica exclusive scan of cell counts into global start offsets (replica r starts after the
// nonzero charges of the replicas before it, so the cells of all replicas are contiguous):
// one block per replica; each thread takes CS_PER consecutive cells of a tile of CS_THREADS x CS_PER.
// The block is small enough to run beside a structure-factor CTA on its SM.
constexpr int CS_THREADS = 256, CS_PER = 8;
__global__ void __launch_bounds__(CS_THREADS) k_cellscan(const int* count, int* start, int ncells, int64_t ne, int m,
                                                         const int* nzc) {
    __shared__ int warp_tot[CS_THREADS / 32];
    __shared__ int carry;
    const int r = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int c0 = 0;
        for (int q = 0; q < r; ++q) c0 += nzc[q];
        carry = c0;
    }
    __syncthreads();
    for (int base = 0; base < ncells; base += CS_THREADS * CS_PER) {
        const int i0 = base + (int)threadIdx.x * CS_PER;
        int v[CS_PER];
#pragma unroll
        for (int k = 0; k < CS_PER; ++k) v[k] = i0 + k < ncells ? count[r * ncells + i0 + k] : 0;
        int tsum = 0;
#pragma unroll
        for (int k = 0; k < CS_PER; ++k) tsum += v[k];
        int x = tsum;   // inclusive scan of the thread totals within the warp
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int t = lane < CS_THREADS / 32 ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < CS_THREADS / 32) warp_tot[lane] = t;
        }
        __syncthreads();
        int run = carry + (wid > 0 ? warp_tot[wid - 1] : 0) + x - tsum;
#pragma unroll
        for (int k = 0; k < CS_PER; ++k) {
            if (i0 + k < ncells) start[r * ncells + i0 + k] = run;
            run += v[k];
        }
        __syncthreads();   // carry has been read by every thread
        if (threadIdx.x == CS_THREADS - 1) carry = run;
        __syncthreads();
    }
    if (r == m - 1 && threadIdx.x == 0) start[m * ncells] = carry;
}

__global__ void k_scatter(const int* key, const int* start, int* cursor, int64_t ptot, int* order) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ptot) return;
    int k = key[p];
    if (k < 0) return;   // a zero charge: in no cell
    order[start[k] + atomicAdd(&cursor[k], 1)] = (int)p;
}

// One warp per cell: every charge's rank in the cell is the number of the cell's charges with a
// smaller input index, so the sorted order (and every sum over a cell) is the same on every
// call, whatever order the atomic scatter produced.
template <typename T>
__global__ void k_cellsort(const int* start, int ncells_total, const int* order, const typename V4<T>::t* wpos,
                           typename V4<T>::t* sorted) {
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= ncells_total) return;
    const int b = start[c], e = start[c + 1];
    for (int i = b + lane; i < e; i += 32) {
        const int v = order[i];
        int rank = 0;
        for (int j = b; j < e; ++j) rank += order[j] < v ? 1 : 0;
        sorted[b + rank] = wpos[v];
    }
}

template <typename T> __device__ __forceinline__ T erfc_t(T x);
template <> __device__ __forceinline__ float erfc_t<float>(float x) { return erfcf(x); }
template <> __device__ __forceinline__ double erfc_t<double>(double x) { return erfc(x); }

// Pair-function tables (RT_N, RT_S): cubic Hermite pieces on RT_N equal intervals of [0, rcut], built
// in FP64 from f and f' (f is even and smooth, f(0) = 2 (eta - alpha) / sqrt(pi)); the
// interpolation error is below 1e-8 of f(0) for the widths and cut-offs used here.

__device__ inline void pair_f_df(double r, double a, double e, double* f, double* df) {
    if (r == 0.0) {
        *f = 2.0 * (e - a) / sqrt(PI);
        *df = 0.0;
        return;
    }
    const double v = (erf(e * r) - erf(a * r)) / r;
    *f = v;
    *df = (2.0 / sqrt(PI)) * (e * exp(-e * e * r * r) - a * exp(-a * a * r * r)) / r - v / r;
}

__global__ void k_pair_tables(const double* __restrict__ etas, int ntab, double alpha, double rcut,
                              float4* __restrict__ tab) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntab * RT_S) return;
    const int id = t / RT_S, k = t % RT_S;
    if (k == RT_N) {
        tab[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const double h = rcut / RT_N, e = etas[id];
    double f0, d0, f1, d1;
    pair_f_df(k * h, alpha, e, &f0, &d0);
    pair_f_df((k + 1) * h, alpha, e, &f1, &d1);
    d0 *= h;
    d1 *= h;
    tab[t] = make_float4((float)f0, (float)d0, (float)(3.0 * (f1 - f0) - 2.0 * d0 - d1), (float)(2.0 * (f0 - f1) + d0 + d1));
}

// Real-space part: one warp per (replica, site); lanes split the stencil cells, skipping cells whose
// nearest point is beyond rcut.  Single precision reads the tabulated pair function when tables exist.
template <typename T>
__global__ void __launch_bounds__(256) k_real_b(const double* __restrict__ sx, int64_t n, int m, Geometry g,
                                                CellGrid cg, const int* __restrict__ start,
                                                const typename V4<T>::t* __restrict__ sorted,
                                                const float4* __restrict__ tab, const int* __restrict__ tabid,
                                                double* out) {
    int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)m * n) return;
    const int r = (int)(wid / n);
    const int64_t i = wid % n;
    double sw[3];
    int ci[3];
    for (int d = 0; d < 3; ++d) {
        double x = sx[d * n + i];
        sw[d] = x - g.boxL[d] * floor(x * g.inv[d]);
        if (sw[d] >= g.boxL[d]) sw[d] -= g.boxL[d];
        if (sw[d] < 0) sw[d] = 0;
        ci[d] = min(cg.nc[d] - 1, (int)(sw[d] / cg.h[d]));
    }
    const T ex = (T)sx[3 * n + i];
    const T a = (T)g.alpha;
    const T rc2 = (T)(g.rcut * g.rcut);
    const T px = (T)sw[0], py = (T)sw[1], pz = (T)sw[2];
    const float4* tb = (tab && tabid) ? tab + (int64_t)tabid[i] * RT_S : nullptr;
    const float inv_h = (float)(RT_N / g.rcut);
    const float hf[3] = {(float)cg.h[0], (float)cg.h[1], (float)cg.h[2]};
    const float swf[3] = {(float)sw[0], (float)sw[1], (float)sw[2]};
    const float rcf2 = (float)(g.rcut * g.rcut);
    const int wx = 2 * cg.S[0] + 1, wy = 2 * cg.S[1] + 1, wz = 2 * cg.S[2] + 1;
    const int nst = wx * wy * wz;
    T acc = 0;
    for (int s = lane; s < nst; s += 32) {
        int dx = s % wx - cg.S[0], dy = (s / wx) % wy - cg.S[1], dz = s / (wx * wy) - cg.S[2];
        int ux = ci[0] + dx, uy = ci[1] + dy, uz = ci[2] + dz;
        // distance from the site to the (unwrapped) cell box
        const float gx = fmaxf(0.f, fmaxf(ux * hf[0] - swf[0], swf[0] - (ux + 1) * hf[0]));
        const float gy = fmaxf(0.f, fmaxf(uy * hf[1] - swf[1], swf[1] - (uy + 1) * hf[1]));
        const float gz = fmaxf(0.f, fmaxf(uz * hf[2] - swf[2], swf[2] - (uz + 1) * hf[2]));
        if (gx * gx + gy * gy + gz * gz >= rcf2 * 1.0001f) continue;
        int fx = floordiv(ux, cg.nc[0]), fy = floordiv(uy, cg.nc[1]), fz = floordiv(uz, cg.nc[2]);
        int cx = ux - fx * cg.nc[0], cy = uy - fy * cg.nc[1], cz = uz - fz * cg.nc[2];
        const T shx = (T)(fx * g.boxL[0]), shy = (T)(fy * g.boxL[1]), shz = (T)(fz * g.boxL[2]);
        int cell = r * cg.ncells + (cz * cg.nc[1] + cy) * cg.nc[0] + cx;
        int p1 = start[cell + 1];
        for (int p = start[cell]; p < p1; ++p) {
            typename V4<T>::t q = sorted[p];
            if (q.w == (T)0) continue;
            T ddx = px - (q.x + shx), ddy = py - (q.y + shy), ddz = pz - (q.z + shz);
            T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (r2 < rc2) {
                T rr = sqrt(r2);
                if (std::is_same<T, float>::value && tb) {
                    const float u = (float)rr * inv_h;
                    const int k = min((int)u, RT_N - 1);
                    const float t = u - (float)k;
                    const float4 cf = tb[k];
                    acc += q.w * (T)(cf.x + t * (cf.y + t * (cf.z + t * cf.w)));
                } else {
                    acc += q.w * (erfc_t<T>(a * rr) - erfc_t<T>(ex * rr)) / rr;
                }
            }
        }
    }
    double acc64 = (double)acc;
    for (int o = 16; o > 0; o >>= 1) acc64 += __shfl_down_sync(0xffffffffu, acc64, o);
    if (lane == 0) out[(int64_t)r * n + i] = acc64;
}

// Real space, single precision, cell pairs: the sites are grouped by real-space cell into chunks
// of at most 32 (assembled once).  A block of RC_WARPS warps takes one chunk; its warps split the
// rows (dy, dz) of the cell's stencil.  Rows whose cells lie farther than r_c from the bounding box
// of the chunk's sites are skipped and the x range of each row is trimmed the same way; since the
// cells of a row are consecutive in the sorted charge array, a row is one contiguous range per
// image shift.  The lanes of a warp read 32 charges of its concatenated ranges at a time; those
// within r_c of the sites' box are compacted into a per-warp ring, and whenever 32 are there every
// lane takes one and runs over all sites of the chunk, keeping one partial sum per site; the
// partial sums of all lanes and warps are added per site in a fixed order at the end.  The pair-function tables of up to two widths
// are staged in shared memory.
constexpr int RC_WARPS = 4;
constexpr int RC_SMEM_TABS = 2;
constexpr int RC_LIST = 64;                         // charge ranges listed per warp at a time
constexpr int RC_RING = 64;                         // per-warp ring of charges that passed the box test

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float4 lds128(const float4* p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
    return v;
}

template <bool SMEM_TAB, bool ONE_TAB>
__global__ void __launch_bounds__(32 * RC_WARPS, 4)
    k_real_cells(const float* __restrict__ s32, const int* __restrict__ perm, const int4* __restrict__ chunks,
                 int nchunks, int64_t n, Geometry g, CellGrid cg, const int* __restrict__ start,
                 const float4* __restrict__ sorted, const float4* __restrict__ tab, int ntab,
                 const int* __restrict__ tabid, int m, int* __restrict__ rqueue, double* __restrict__ out) {
    __shared__ float4 stab[RC_SMEM_TABS * RT_S];
    __shared__ float4 ssite[32];                    // (x, y, z, table offset as int bits)
    __shared__ float ssite_x[32], ssite_y[32], ssite_z[32];   // the same coordinates, one array each
    __shared__ float sbox[6];
    // per warp while streaming: the charge ranges of a group of rows and the ring of charges that
    // passed the box test; at the end the same bytes hold the per-site partial sums
    struct Lists {
        int beg[RC_WARPS][RC_LIST];
        int pre[RC_WARPS][RC_LIST + 1];
        float4 sh[RC_WARPS][RC_LIST];
        float4 ring[RC_WARPS][RC_RING];
    };
    union Shared {
        Lists l;
        float red[RC_WARPS][32][33];   // [warp][site][lane]
    };
    __shared__ Shared u_;
    auto& lbeg = u_.l.beg;
    auto& lpre = u_.l.pre;
    auto& lsh = u_.l.sh;
    auto& red = u_.red;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // persistent, items from a queue: item k is chunk k / m (chunks are stored with the most sites
    // first) of replica k % m; thread 0 takes the next item while the block works on the current one
    __shared__ int s_item;
    const int nitems = nchunks * m;
    int nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(&rqueue[0], 1);
    if (SMEM_TAB) {   // staged once per block, eight loads per thread in flight
        const int tot = ntab * RT_S;
        for (int e0 = 0; e0 < tot; e0 += 8 * (int)blockDim.x) {
            float4 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = e0 + k * (int)blockDim.x + (int)threadIdx.x;
                if (e < tot) v[k] = tab[e];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = e0 + k * (int)blockDim.x + (int)threadIdx.x;
                if (e < tot) stab[e] = v[k];
            }
        }
    }
    for (;;) {
    __syncthreads();   // the previous item's partial sums and s_item have been read
    if (threadIdx.x == 0) s_item = nxt;
    __syncthreads();
    const int item = s_item;
    if (item >= nitems) break;
    if (threadIdx.x == 0) nxt = atomicAdd(&rqueue[0], 1);   // used at the next item
    const int ch = item / m, r = item % m;
    const int4 cinfo = chunks[ch];   // (first, count, cell, 0)
    const int nsites = cinfo.y;
    if (warp == 0) {
        float px = 0.f, py = 0.f, pz = 0.f;
        int toff = 0;
        if (lane < nsites) {
            const int i = perm[cinfo.x + lane];
            px = s32[i]; py = s32[n + i]; pz = s32[2 * n + i];
            toff = tabid[i] * RT_S;
        }
        if (lane >= nsites) px = py = pz = 1.0e6f;   // dummy sites, beyond any cutoff
        ssite[lane] = make_float4(px, py, pz, __int_as_float(toff));
        ssite_x[lane] = px;
        ssite_y[lane] = py;
        ssite_z[lane] = pz;
        float lo[3] = {px, py, pz}, hi[3] = {px, py, pz};   // (dummies excluded below)
        if (lane >= nsites) {
            lo[0] = lo[1] = lo[2] = 3.0e38f;
            hi[0] = hi[1] = hi[2] = -3.0e38f;
        }
        for (int o = 16; o > 0; o >>= 1)
            for (int d = 0; d < 3; ++d) {
                lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
            }
        if (lane == 0) {
            sbox[0] = lo[0]; sbox[1] = lo[1]; sbox[2] = lo[2];
            sbox[3] = hi[0]; sbox[4] = hi[1]; sbox[5] = hi[2];
        }
    }
    __syncthreads();
    const float4* tb = SMEM_TAB ? stab : tab;
    const int cx = cinfo.z % cg.nc[0], cy = (cinfo.z / cg.nc[0]) % cg.nc[1], cz = cinfo.z / (cg.nc[0] * cg.nc[1]);
    const float rc2 = (float)(g.rcut * g.rcut);
    const float inv_h = (float)(RT_N / g.rcut);
    const float hx = (float)cg.h[0], hy = (float)cg.h[1], hz = (float)cg.h[2];
    const float lx = (float)g.boxL[0], ly = (float)g.boxL[1], lz = (float)g.boxL[2];
    const float bx0 = sbox[0], by0 = sbox[1], bz0 = sbox[2], bx1 = sbox[3], by1 = sbox[4], bz1 = sbox[5];
    float acc[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) acc[s] = 0.f;
    // every lane holds one charge (weight qw, zero for an empty lane) and runs over the chunk's sites
    auto pair_term = [&](const float4 st, const float4 q) {
        // branch-free pair term: the table index is clamped and the weight is zero outside the
        // cutoff, so the sites of a group interleave
        const float ddx = st.x - q.x, ddy = st.y - q.y, ddz = st.z - q.z;
        const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        const float u = sqrt_approx(r2) * inv_h;
        // floor(u) from the bits of u + 1.5 * 2^23 rounded toward zero (u >= 0); at and past the
        // cutoff the index clamps to the table's zero row
        const float ur = __fadd_rz(u, 12582912.0f);
        const int kk = min(__float_as_int(ur) - 0x4B400000, RT_N);
        const float t = u - (ur - 12582912.0f);
        const float4 cf = tb[__float_as_int(st.w) + kk];
        return cf.x + t * (cf.y + t * (cf.z + t * cf.w));
    };
    auto eval_sites = [&](const float4 q, const float qw) {
#pragma unroll
        for (int sg = 0; sg < 32; sg += 8) {
            if (sg >= nsites) break;   // uniform; sites past nsites are far-away dummies
#pragma unroll
            for (int s = sg; s < sg + 8; ++s) {
                // re-read: keeps 32 sites out of registers; with one table the offset is zero and
                // three 4-byte broadcasts cost fewer wavefronts than one 16-byte broadcast
                const float4 st = ONE_TAB ? make_float4(ssite_x[s], ssite_y[s], ssite_z[s], 0.f) : lds128(&ssite[s]);
                acc[s] = fmaf(qw, pair_term(st, q), acc[s]);
            }
        }
    };
    // charges that pass the box test wait in a per-warp ring until 32 are there
    float4* ring = u_.l.ring[warp];
    int rhead = 0, rcount = 0;   // warp-uniform
    // The warp's rows are taken in groups; the charge ranges (runs of cells with one image shift)
    // of a group are listed in shared memory and streamed as one concatenated sequence, 32 charges
    // per step, so that the lanes stay busy across the ends of the ranges.
    int* rbeg = lbeg[warp];
    int* rpre = lpre[warp];
    float4* rsh = lsh[warp];
    const int wy = 2 * cg.S[1] + 1, nrows = wy * (2 * cg.S[2] + 1);
    const int maxruns = (2 * cg.S[0] + 1 + cg.nc[0] - 1) / cg.nc[0] + 1;
    const int group = max(1, min(32, RC_LIST / maxruns));
    for (int g0 = warp; g0 < nrows; g0 += RC_WARPS * group) {
        // lane l takes row g0 + RC_WARPS l of the group
        const int row = g0 + RC_WARPS * lane;
        int nrun = 0, ux = 0, uxe = -1, fx0 = 0, rowbase = 0;
        float shy = 0.f, shz = 0.f;
        if (lane < group && row < nrows) {
            const int dy = row % wy - cg.S[1], dz = row / wy - cg.S[2];
            const int uz = cz + dz, uy = cy + dy;
            const float dyd = fmaxf(0.f, fmaxf((float)uy * hy - by1, by0 - (float)(uy + 1) * hy));
            const float dzd = fmaxf(0.f, fmaxf((float)uz * hz - bz1, bz0 - (float)(uz + 1) * hz));
            const float rx2 = rc2 - dyd * dyd - dzd * dzd;
            if (rx2 > 0.f) {
                const float rx = sqrtf(rx2) * 1.0001f + 1e-3f;
                ux = max(cx - cg.S[0], (int)floorf((bx0 - rx) / hx));
                uxe = min(cx + cg.S[0], (int)floorf((bx1 + rx) / hx));
                if (ux <= uxe) {
                    fx0 = floordiv(ux, cg.nc[0]);
                    nrun = floordiv(uxe, cg.nc[0]) - fx0 + 1;
                    const int fz = floordiv(uz, cg.nc[2]), wz = uz - fz * cg.nc[2];
                    const int fy = floordiv(uy, cg.nc[1]), wyy = uy - fy * cg.nc[1];
                    shz = (float)fz * lz;
                    shy = (float)fy * ly;
                    rowbase = r * cg.ncells + (wz * cg.nc[1] + wyy) * cg.nc[0];
                }
            }
        }
        // place this lane's runs after those of the lanes before it
        int off = nrun;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, off, o);
            if (lane >= o) off += v;
        }
        const int nent = __shfl_sync(0xffffffffu, off, 31);
        off -= nrun;
        for (int k = 0; k < nrun; ++k) {
            const int fx = fx0 + k;
            const int a = max(ux, fx * cg.nc[0]), bnd = min(uxe, fx * cg.nc[0] + cg.nc[0] - 1);
            const int wx0 = a - fx * cg.nc[0], wx1 = bnd - fx * cg.nc[0];
            const int b = start[rowbase + wx0], e = start[rowbase + wx1 + 1];
            rbeg[off + k] = b;
            rpre[off + k] = e - b;
            rsh[off + k] = make_float4((float)fx * lx, shy, shz, 0.f);
        }
        __syncwarp();
        // exclusive prefix of the range lengths (nent <= RC_LIST)
        int total = 0;
        for (int e0 = 0; e0 < nent; e0 += 32) {
            const int e = e0 + lane;
            int len = e < nent ? rpre[e] : 0, inc = len;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            __syncwarp();
            if (e < nent) rpre[e] = total + inc - len;
            total += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) rpre[nent] = total;
        __syncwarp();
        // charge v of the concatenated ranges (its image shift applied later), loaded one batch ahead;
        // each lane keeps the index of the range its next charge falls in and moves it forward (the
        // charges a lane takes only increase)
        int ec = 0;
        {
            int lo = 0, hi = nent - 1;   // last entry with rpre[e] <= lane
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (rpre[mid] <= lane) lo = mid; else hi = mid - 1;
            }
            ec = lo;
        }
        auto fetch = [&](int v, float4& q, float4& sh) {
            while (ec + 1 < nent && rpre[ec + 1] <= v) ++ec;
            q = sorted[rbeg[ec] + (v - rpre[ec])];
            sh = rsh[ec];
        };
        float4 qn = make_float4(0.f, 0.f, 0.f, 0.f), shn = qn;
        if (lane < total) fetch(lane, qn, shn);
        for (int base = 0; base < total; base += 32) {
            const int v = base + lane;
            bool keep = v < total;
            float4 q = qn;
            const float4 sh = shn;
            if (v + 32 < total) fetch(v + 32, qn, shn);
            if (keep) {
                q.x += sh.x; q.y += sh.y; q.z += sh.z;
                // only charges within r_c of the sites' box can reach a site
                const float ex = fmaxf(0.f, fmaxf(bx0 - q.x, q.x - bx1));
                const float ey = fmaxf(0.f, fmaxf(by0 - q.y, q.y - by1));
                const float ez = fmaxf(0.f, fmaxf(bz0 - q.z, q.z - bz1));
                keep = ex * ex + ey * ey + ez * ez < rc2;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) ring[(rhead + rcount + __popc(bal & ((1u << lane) - 1u))) & (RC_RING - 1)] = q;
            rcount += __popc(bal);
            __syncwarp();
            if (rcount >= 32) {
                const float4 qq = ring[(rhead + lane) & (RC_RING - 1)];
                __syncwarp();
                rhead = (rhead + 32) & (RC_RING - 1);
                rcount -= 32;
                eval_sites(qq, qq.w);
            }
        }
        __syncwarp();
    }
    if (rcount > 0) {   // the rest of the ring
        const float4 qq = lane < rcount ? ring[(rhead + lane) & (RC_RING - 1)] : make_float4(0.f, 0.f, 0.f, 0.f);
        eval_sites(qq, lane < rcount ? qq.w : 0.f);
    }
    __syncthreads();   // the lists and rings are done: their bytes now take the partial sums
#pragma unroll
    for (int s = 0; s < 32; ++s) red[warp][s][lane] = acc[s];
    __syncthreads();
    if (warp == 0 && lane < nsites) {
        double a = 0.0;
        for (int w = 0; w < RC_WARPS; ++w) {
            float fs = 0.f;
            for (int l = 0; l < 32; ++l) fs += red[w][lane][l];
            a += (double)fs;
        }
        out[(int64_t)r * n + perm[cinfo.x + lane]] = a;
    }
    }
    // every take of this block is done; the last block to finish puts the queue back to zero for
    // the next launch (launches on one context are stream-ordered)
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&rqueue[1], 1) == (int)gridDim.x - 1) {
            atomicExch(&rqueue[0], 0);
            atomicExch(&rqueue[1], 0);
        }
    }
}

// one wave of the persistent real-space kernel: four blocks per SM (its launch bound)
static unsigned real_grid(int nchunks, int m) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)nchunks * m, 4 * 152));
}

cpm_status build_pair_tables(cpm_ctx* c, const std::vector<double>& etas) {
    dev_free(c, c->rtab);
    c->rtab = nullptr;
    CPM_TRY(dev_alloc(c, (void**)&c->rtab, sizeof(float4) * RT_S * etas.size()));
    double* de = nullptr;
    CPM_TRY(dev_alloc(c, (void**)&de, sizeof(double) * etas.size()));
    CPM_CUDA(c, cudaMemcpyAsync(de, etas.data(), sizeof(double) * etas.size(), cudaMemcpyHostToDevice, c->stream));
    const int tot = (int)etas.size() * RT_S;
    k_pair_tables<<<(tot + 127) / 128, 128, 0, c->stream>>>(de, (int)etas.size(), c->g.alpha, c->g.rcut,
                                                             (float4*)c->rtab);
    CPM_LAUNCH(c, "k_pair_tables");
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, de);
    return CPM_OK;
}

// ----------------------------------------------------------------------------- reciprocal space
constexpr int SF_BM = 64, SF_BN = 64, SF_BK = 16;

template <typename T>
__device__ __forceinline__ int tile_maxext(const int* colext, int c0, int ncols) {
    __shared__ int mx;
    if (threadIdx.x == 0) mx = -1;
    __syncthreads();
    if (threadIdx.x < SF_BM && c0 + (int)threadIdx.x < ncols) atomicMax(&mx, colext[c0 + threadIdx.x]);
    __syncthreads();
    return mx;
}

// rho_part[s][r][c][nz] = sum over the s-th particle chunk of replica r of Q_j X_j Y_j Z_j.
template <typename T>
__global__ void __launch_bounds__(256) k_sf(const int2* __restrict__ cols, const int* __restrict__ colext, int ncols,
                                            int NY, int NZ, int nzw, const c2<T>* __restrict__ EX,
                                            const c2<T>* __restrict__ EY, const c2<T>* __restrict__ EZ,
                                            const T* __restrict__ Qv, int64_t ptot, int64_t ne, int splits,
                                            int64_t chunk, int m, c2<T>* __restrict__ rho_part) {
    __shared__ c2<T> Ps[SF_BK][SF_BM + 1];
    __shared__ c2<T> Zs[SF_BK][SF_BN + 1];
    // z tiles are centred on nz = 0: tile t covers grid indices zbase + t*BN ... + BN - 1
    const int zbase = NZ - SF_BN / 2 - SF_BN * ((int)gridDim.y / 2);
    const int c0 = blockIdx.x * SF_BM, z0 = zbase + blockIdx.y * SF_BN;
    const int r = blockIdx.z / splits, s = blockIdx.z % splits;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    c2<T>* outp = rho_part + ((int64_t)s * m + r) * ncols * nzw;
    const int mx = tile_maxext<T>(colext, c0, ncols);
    const bool skip = (z0 - NZ > mx) || (z0 + SF_BN - 1 - NZ < -mx);
    typedef c2<T> V;
    V acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = cmake<T>(0, 0);
    const int64_t jb = (int64_t)r * ne + (int64_t)s * chunk;
    const int64_t je = min((int64_t)r * ne + ne, jb + chunk);
    if (!skip) {
        for (int64_t j0 = jb; j0 < je; j0 += SF_BK) {
            for (int e = threadIdx.x; e < SF_BK * SF_BM; e += 256) {
                int kk = e % SF_BK, mm = e / SF_BK;
                int64_t j = j0 + kk;
                int c = c0 + mm;
                V v = cmake<T>(0, 0);
                if (j < je && c < ncols) {
                    int2 cn = cols[c];
                    V xy = cmul(EX[(int64_t)cn.x * ptot + j], EY[(int64_t)(cn.y + NY) * ptot + j]);
                    T qj = Qv[j];
                    v.x = qj * xy.x; v.y = qj * xy.y;
                }
                Ps[kk][mm] = v;
                int z = z0 + mm;
                V zv = cmake<T>(0, 0);
                if (j < je && z >= 0 && z < nzw) zv = EZ[(int64_t)z * ptot + j];
                Zs[kk][mm] = zv;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < SF_BK; ++kk) {
                V av[4], bv[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) av[p] = Ps[kk][ty + 16 * p];
#pragma unroll
                for (int q = 0; q < 4; ++q) bv[q] = Zs[kk][tx + 16 * q];
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        acc[p][q].x += av[p].x * bv[q].x - av[p].y * bv[q].y;
                        acc[p][q].y += av[p].x * bv[q].y + av[p].y * bv[q].x;
                    }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int c = c0 + ty + 16 * p;
        if (c >= ncols) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int z = z0 + tx + 16 * q;
            if (z >= 0 && z < nzw) outp[(int64_t)c * nzw + z] = acc[p][q];
        }
    }
}

// Single-precision structure factor with a 64-column x 128-harmonic accumulator tile per block:
// warp w owns harmonics [16w, 16w + 16) of the tile's z range and skips the contraction when that
// slab lies outside the largest |nz| of the tile's columns (columns are sorted by k_perp, so the
// slab test removes most of the padding of the dense grid); the charge operand Q_j X_j Y_j of the
// tile's columns is formed once per chunk of charges and shared by all 128 harmonics.
constexpr int S2_BM = 64, S2_BZ = 128, S2_BK = 16;

__global__ void __launch_bounds__(256, 2) k_sf32(const int2* __restrict__ cols, const int* __restrict__ colext,
                                                 int ncols, int NY, int NZ, int nzw, const float2* __restrict__ EX,
                                                 const float2* __restrict__ EY, const float2* __restrict__ EZ,
                                                 const float* __restrict__ Qv, int64_t ptot, int64_t ne, int splits,
                                                 int64_t chunk, int m, int nsup, float2* __restrict__ rho_part) {
    __shared__ float2 Ps[S2_BK][S2_BM + 1];
    __shared__ float2 Zs[S2_BK][S2_BZ + 1];
    const int c0 = blockIdx.x * S2_BM;
    const int zbase = NZ - S2_BZ / 2 - S2_BZ * (nsup / 2) + S2_BZ * (int)blockIdx.y;   // grid index of row 0
    const int r = blockIdx.z / splits, s = blockIdx.z % splits;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cg = lane & 15, zh = lane >> 4;
    float2* outp = rho_part + ((int64_t)s * m + r) * ncols * nzw;
    const int mx = tile_maxext<float>(colext, c0, ncols);
    // harmonics of this warp: zbase + 16 warp + zh + 2 q, q = 0..7  (nz = index - NZ)
    const int wz0 = zbase + 16 * warp - NZ, wz1 = wz0 + 15;
    const bool active = mx >= 0 && !(wz0 > mx || wz1 < -mx);
    const bool block_any = mx >= 0 && !(zbase - NZ > mx || zbase + S2_BZ - 1 - NZ < -mx);
    float2 acc[4][8];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = make_float2(0.f, 0.f);
    const int64_t jb = (int64_t)r * ne + (int64_t)s * chunk;
    const int64_t je = min((int64_t)r * ne + ne, jb + chunk);
    if (block_any) {
        for (int64_t j0 = jb; j0 < je; j0 += S2_BK) {
            for (int e = threadIdx.x; e < S2_BK * S2_BM; e += 256) {
                const int kk = e % S2_BK, mm = e / S2_BK;
                const int64_t j = j0 + kk;
                const int c = c0 + mm;
                float2 v = make_float2(0.f, 0.f);
                if (j < je && c < ncols) {
                    const int2 cn = cols[c];
                    const float2 xy = cmul(EX[(int64_t)cn.x * ptot + j], EY[(int64_t)(cn.y + NY) * ptot + j]);
                    const float qj = Qv[j];
                    v = make_float2(qj * xy.x, qj * xy.y);
                }
                Ps[kk][mm] = v;
            }
            for (int e = threadIdx.x; e < S2_BK * S2_BZ; e += 256) {
                const int kk = e % S2_BK, zz = e / S2_BK;
                const int64_t j = j0 + kk;
                const int z = zbase + zz;
                Zs[kk][zz] = (j < je && z >= 0 && z < nzw) ? EZ[(int64_t)z * ptot + j] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            if (active) {
#pragma unroll 2
                for (int kk = 0; kk < S2_BK; ++kk) {
                    float2 av[4], bv[8];
#pragma unroll
                    for (int p = 0; p < 4; ++p) av[p] = Ps[kk][cg + 16 * p];
#pragma unroll
                    for (int q = 0; q < 8; ++q) bv[q] = Zs[kk][16 * warp + zh + 2 * q];
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            acc[p][q].x += av[p].x * bv[q].x - av[p].y * bv[q].y;
                            acc[p][q].y += av[p].x * bv[q].y + av[p].y * bv[q].x;
                        }
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int c = c0 + cg + 16 * p;
        if (c >= ncols) continue;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int z = zbase + 16 * warp + zh + 2 * q;
            if (z >= 0 && z < nzw) outp[(int64_t)c * nzw + z] = acc[p][q];
        }
    }
}

// wrho[r][c][nz] = w[c][nz] * sum_s rho_part[s][r][c][nz]  (Neumaier-compensated over the splits)
template <typename T>
__global__ void k_sf_reduce(const c2<T>* rho_part, const T* w, int64_t per_rep, int m, int splits, c2<T>* wrho) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= per_rep * m) return;
    T sx = 0, sy = 0, cx = 0, cy = 0;
    for (int s = 0; s < splits; ++s) {
        c2<T> v = rho_part[(int64_t)s * per_rep * m + t];
        T tx = sx + v.x;
        cx += fabs(sx) >= fabs(v.x) ? (sx - tx) + v.x : (v.x - tx) + sx;
        sx = tx;
        T ty = sy + v.y;
        cy += fabs(sy) >= fabs(v.y) ? (sy - ty) + v.y : (v.y - ty) + sy;
        sy = ty;
    }
    T wt = w[t % per_rep];
    wrho[t] = cmake<T>(wt * (sx + cx), wt * (sy + cy));
}

// partial[r][tile][i] = sum over the tile's columns c of Re[conj(X_i Y_i) sum_nz wrho[c][nz] conj(Z_i[nz])]
template <typename T>
__global__ void __launch_bounds__(256) k_site(const int2* __restrict__ cols, const int* __restrict__ colext,
                                              int ncols, int NY, int NZ, int nzw, const c2<T>* __restrict__ wrho,
                                              const c2<T>* __restrict__ SX, const c2<T>* __restrict__ SY,
                                              const c2<T>* __restrict__ SZ, int64_t n, int nctiles,
                                              T* __restrict__ partial) {
    __shared__ c2<T> As[SF_BK][SF_BM + 1];
    __shared__ c2<T> Bs[SF_BK][SF_BN + 1];
    __shared__ T red[16][SF_BN + 1];
    const int64_t i0 = (int64_t)blockIdx.x * SF_BN;
    const int c0 = blockIdx.y * SF_BM;
    const int r = blockIdx.z;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const c2<T>* rho = wrho + (int64_t)r * ncols * nzw;
    const int mx = tile_maxext<T>(colext, c0, ncols);
    typedef c2<T> V;
    V acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = cmake<T>(0, 0);
    if (mx >= 0) {
        const int zb = NZ - mx, ze = NZ + mx + 1;
        for (int z0 = zb; z0 < ze; z0 += SF_BK) {
            for (int e = threadIdx.x; e < SF_BK * SF_BM; e += 256) {
                int kk = e % SF_BK, mm = e / SF_BK;
                int z = z0 + kk, c = c0 + mm;
                As[kk][mm] = (z < ze && c < ncols) ? rho[(int64_t)c * nzw + z] : cmake<T>(0, 0);
                int nn = e % SF_BN;
                kk = e / SF_BN;
                z = z0 + kk;
                int64_t i = i0 + nn;
                Bs[kk][nn] = (z < ze && i < n) ? SZ[(int64_t)z * n + i] : cmake<T>(0, 0);
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < SF_BK; ++kk) {
                V av[4], bv[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) av[p] = As[kk][ty + 16 * p];
#pragma unroll
                for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {   // a * conj(b)
                        acc[p][q].x += av[p].x * bv[q].x + av[p].y * bv[q].y;
                        acc[p][q].y += av[p].y * bv[q].x - av[p].x * bv[q].y;
                    }
            }
            __syncthreads();
        }
    }
    // epilogue: multiply by conj(X_i Y_i) per column, sum the columns of this thread, then over ty
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int64_t i = i0 + tx + 16 * q;
        T s = 0;
        if (i < n) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                int c = c0 + ty + 16 * p;
                if (c < ncols) {
                    int2 cn = cols[c];
                    V xy = cmul(SX[(int64_t)cn.x * n + i], SY[(int64_t)(cn.y + NY) * n + i]);
                    s += xy.x * acc[p][q].x + xy.y * acc[p][q].y;
                }
            }
        }
        red[ty][tx + 16 * q] = s;
    }
    __syncthreads();
    if (threadIdx.x < SF_BN) {
        T s = 0;
        for (int t = 0; t < 16; ++t) s += red[t][threadIdx.x];
        int64_t i = i0 + threadIdx.x;
        if (i < n) partial[((int64_t)r * nctiles + blockIdx.y) * n + i] = s;
    }
}

// ----------------------------------------------------------------------------- k_perp = 0 column, double-float
// The single-precision paths sum the first harmonics of the column (0, 0, nz), nz = 1..COL0_NZ,
// in double-float: their weights are the largest of the whole set (they carry the laterally
// averaged charge profile), so their terms would dominate the rounding of a single-precision sum.
// Phases by a double-float recurrence in nz from an exactly reduced first harmonic.
__device__ __forceinline__ double2 z_phase_n(double z, double invLz, int nz) {
    double s = z * invLz;
    s -= floor(s);
    double t = s * 18446744073709551616.0;
    uint64_t u = t >= 18446744073709551616.0 ? 0ull : (uint64_t)t;
    u *= (uint64_t)nz;   // fraction of nz z / Lz, reduced exactly (mod 2^64)
    double sn, cs;
    sincospi((double)(int64_t)u * 0x1p-63, &sn, &cs);
    return make_double2(cs, sn);
}
__device__ __forceinline__ double2 z_phase1(double z, double invLz) { return z_phase_n(z, invLz, 1); }

// Double-float arithmetic (pairs of floats, about 48 significant bits; Dekker 1971, Knuth TAOCP
// vol. 2): the k_perp = 0 column needs better than FP32 accuracy, and FP32 pairs run far faster
// than FP64 on this GPU.
struct dfl { float hi, lo; };
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl df_fast(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    dfl s = df_two_sum(a.hi, b.hi), t = df_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = df_fast(s.hi, s.lo);
    s.lo += t.lo;
    return df_fast(s.hi, s.lo);
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast(p, e);
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_of(double x) {
    float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}
struct dcx { dfl re, im; };
__device__ __forceinline__ dcx dcx_mul(dcx a, dcx b) {
    return {df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}

// part[r][chunk][nz - 1] for nz in one block of C0_NB harmonics: each thread takes 2 charges of the
// chunk (256 charges per block), raises exp(i theta) of both to the block's first harmonic and steps
// through the block by a double-float recurrence (the two charges' chains interleaved); the block
// sums its threads in a fixed order.
constexpr int C0_THREADS = 128, C0_PER_THREAD = 2, C0_NB = 6;

__device__ __forceinline__ dcx dcx_pow(dcx e1, int pw) {   // e1^pw by binary powering, pw >= 1
    dcx e = {{1.f, 0.f}, {0.f, 0.f}}, base = e1;
    for (; pw > 0; pw >>= 1) {
        if (pw & 1) e = dcx_mul(e, base);
        base = dcx_mul(base, base);
    }
    return e;
}

__global__ void __launch_bounds__(C0_THREADS) k_col0_rho(const float4* __restrict__ e1s, const float2* __restrict__ Qd,
                                                       int64_t ne, int nz0, double2* __restrict__ part) {
    __shared__ double2 red[C0_THREADS / 32][C0_NB];
    const int chunk = blockIdx.x, nb = blockIdx.y, r = blockIdx.z;
    const int nzs = nb * C0_NB + 1;   // first harmonic of this block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    dcx acc[C0_NB];
#pragma unroll
    for (int k = 0; k < C0_NB; ++k) acc[k] = {{0.f, 0.f}, {0.f, 0.f}};
    // the thread's two charges (a zero charge, also past the end, contributes exact zeros)
    dfl q[C0_PER_THREAD];
    dcx e1[C0_PER_THREAD], e[C0_PER_THREAD];
#pragma unroll
    for (int t = 0; t < C0_PER_THREAD; ++t) {
        const int64_t j = (int64_t)chunk * C0_THREADS * C0_PER_THREAD + (int64_t)t * C0_THREADS + threadIdx.x;
        float2 qf = make_float2(0.f, 0.f);
        float4 f = make_float4(1.f, 0.f, 0.f, 0.f);
        if (j < ne) {
            const int64_t p = (int64_t)r * ne + j;
            qf = Qd[p];
            f = e1s[p];
        }
        q[t] = {qf.x, qf.y};
        e1[t] = {{f.x, f.y}, {f.z, f.w}};
        e[t] = dcx_pow(e1[t], nzs);
    }
#pragma unroll
    for (int k = 0; k < C0_NB; ++k) {
#pragma unroll
        for (int t = 0; t < C0_PER_THREAD; ++t) {
            acc[k].re = df_add(acc[k].re, df_mul(q[t], e[t].re));
            acc[k].im = df_add(acc[k].im, df_mul(q[t], e[t].im));
            e[t] = dcx_mul(e[t], e1[t]);
        }
    }
#pragma unroll
    for (int k = 0; k < C0_NB; ++k) {   // warp sums in double-float, one FP64 value per warp
        dfl re = acc[k].re, im = acc[k].im;
        for (int o = 16; o > 0; o >>= 1) {
            const dfl ore = {__shfl_down_sync(0xffffffffu, re.hi, o), __shfl_down_sync(0xffffffffu, re.lo, o)};
            const dfl oim = {__shfl_down_sync(0xffffffffu, im.hi, o), __shfl_down_sync(0xffffffffu, im.lo, o)};
            re = df_add(re, ore);
            im = df_add(im, oim);
        }
        if (lane == 0) red[warp][k] = make_double2((double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo);
    }
    __syncthreads();
    if (threadIdx.x < C0_NB) {
        const int k = threadIdx.x, nz = nzs + k;
        if (nz <= nz0) {
            double2 tt = red[0][k];
            for (int w = 1; w < C0_THREADS / 32; ++w) { tt.x += red[w][k].x; tt.y += red[w][k].y; }
            part[((int64_t)r * gridDim.x + chunk) * nz0 + nz - 1] = tt;
        }
    }
}

// wrho0[r][nz - 1] = w(0, 0, nz) * sum over chunks of part: one warp per (r, nz), lanes over the
// chunks, combined in a fixed order
__global__ void k_col0_reduce(const double2* __restrict__ part, int nchunks, int nz0, const double* __restrict__ w,
                              int NZ, int m, double2* __restrict__ wrho0) {
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (t >= m * nz0) return;
    const int r = t / nz0, k = t % nz0;
    double2 a = make_double2(0.0, 0.0);
    for (int ch = lane; ch < nchunks; ch += 32) {
        const double2 v = part[((int64_t)r * nchunks + ch) * nz0 + k];
        a.x += v.x;
        a.y += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_down_sync(0xffffffffu, a.x, o);
        a.y += __shfl_down_sync(0xffffffffu, a.y, o);
    }
    if (lane == 0) {
        const double wt = w[NZ + k + 1];   // column 0 occupies the first row of the dense grid
        wrho0[t] = make_double2(wt * a.x, wt * a.y);
    }
}

// e0[u][nz - 1] = exp(i kz z_u) for each distinct site height z_u and nz = 1 .. COL0_NZ (fixed with
// the geometry), one exactly reduced FP64 sincospi per entry
__global__ void k_col0_e0(const double* __restrict__ zu, int nzu, double invLz, int nz0, double2* __restrict__ e0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nzu * nz0) return;
    const int iu = t / nz0, nz = t % nz0 + 1;
    e0[t] = z_phase_n(zu[iu], invLz, nz);
}

// b0[r][u] = sum_nz Re[conj(e0[u][nz]) wrho0[r][nz]]: one warp per (r, u), lanes over nz
__global__ void k_col0_site(const double2* __restrict__ e0, int nzu, int m, int nz0, const double2* __restrict__ wrho0,
                            double* __restrict__ b0) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= m * nzu) return;
    const int r = w / nzu, iu = w % nzu;
    double acc = 0.0;
    for (int k = lane; k < nz0; k += 32) {
        const double2 e = e0[(int64_t)iu * nz0 + k], v = wrho0[(int64_t)r * nz0 + k];
        acc += e.x * v.x + e.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) b0[w] = acc;
}

// Single-precision site potential with a 64-column x 128-site tile per block (4 columns x 8 sites
// per thread): warp w owns sites [16w, 16w + 16) of the tile; the contraction over nz runs only
// over the tile's nz range; the epilogue weights each column by conj(X_i Y_i) and reduces the
// 16 column groups of a half warp with shuffles.
constexpr int T2_BC = 64, T2_BS = 128, T2_BK = 16;

__global__ void __launch_bounds__(256, 2) k_site32(const int2* __restrict__ cols, const int* __restrict__ colext,
                                                   int ncols, int NY, int NZ, int nzw, const float2* __restrict__ wrho,
                                                   const float2* __restrict__ SX, const float2* __restrict__ SY,
                                                   const float2* __restrict__ SZ, int64_t n, int nctiles,
                                                   float* __restrict__ partial) {
    __shared__ float2 As[T2_BK][T2_BC + 1];
    __shared__ float2 Bs[T2_BK][T2_BS + 1];
    const int64_t i0 = (int64_t)blockIdx.x * T2_BS;
    const int c0 = blockIdx.y * T2_BC;
    const int r = blockIdx.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cg = lane & 15, sh = lane >> 4;
    const float2* rho = wrho + (int64_t)r * ncols * nzw;
    const int mx = tile_maxext<float>(colext, c0, ncols);
    float2 acc[4][8];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = make_float2(0.f, 0.f);
    if (mx >= 0) {
        const int zb = NZ - mx, ze = NZ + mx + 1;
        for (int z0 = zb; z0 < ze; z0 += T2_BK) {
            for (int e = threadIdx.x; e < T2_BK * T2_BC; e += 256) {
                const int kk = e % T2_BK, cc = e / T2_BK;
                const int z = z0 + kk, c = c0 + cc;
                As[kk][cc] = (z < ze && c < ncols) ? rho[(int64_t)c * nzw + z] : make_float2(0.f, 0.f);
            }
            for (int e = threadIdx.x; e < T2_BK * T2_BS; e += 256) {
                const int ss = e % T2_BS, kk = e / T2_BS;
                const int z = z0 + kk;
                const int64_t i = i0 + ss;
                Bs[kk][ss] = (z < ze && i < n) ? SZ[(int64_t)z * n + i] : make_float2(0.f, 0.f);
            }
            __syncthreads();
#pragma unroll 2
            for (int kk = 0; kk < T2_BK; ++kk) {
                float2 av[4], bv[8];
#pragma unroll
                for (int p = 0; p < 4; ++p) av[p] = As[kk][cg + 16 * p];
#pragma unroll
                for (int q = 0; q < 8; ++q) bv[q] = Bs[kk][16 * warp + sh + 2 * q];
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 8; ++q) {   // a * conj(b)
                        acc[p][q].x += av[p].x * bv[q].x + av[p].y * bv[q].y;
                        acc[p][q].y += av[p].y * bv[q].x - av[p].x * bv[q].y;
                    }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t i = i0 + 16 * warp + sh + 2 * q;
        float v = 0.f;
        if (i < n) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int c = c0 + cg + 16 * p;
                if (c < ncols) {
                    const int2 cn = cols[c];
                    const float2 xy = cmul(SX[(int64_t)cn.x * n + i], SY[(int64_t)(cn.y + NY) * n + i]);
                    v += xy.x * acc[p][q].x + xy.y * acc[p][q].y;
                }
            }
        }
        // reduce over the 16 column groups of this half warp
        for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (cg == 0 && i < n) partial[((int64_t)r * nctiles + blockIdx.y) * n + i] = v;
    }
}

// b[r][i] = K_E (recip + real - pi Q_tot / (V alpha^2) + boundary)
// with bhl also the two-float split of b for the single-precision S product (the same arithmetic as
// k_split_b, so the update gives bit-identical results either way)
template <typename T>
__global__ void k_combine(const T* partial, int nctiles, const double* real, const double* b0, const int* zmap,
                          int nzu, const double* stats, const double* sx, int64_t n, int m, Geometry g, double* b,
                          float2* bhl, const double* ew, const double* pm) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * n) return;
    const int r = (int)(t / n);
    const int64_t i = t % n;
    const double rl = real[t];   // issued with the tile loads below
    const double bz = b0 ? b0[(int64_t)r * nzu + zmap[i]] : 0.0;
    double s = 0.0;
    const T* pp = partial + (int64_t)r * nctiles * n + i;
    int k = 0;
    for (; k + 16 <= nctiles; k += 16) {   // sixteen loads in flight, added in tile order
        T x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = pp[(int64_t)(k + u) * n];
#pragma unroll
        for (int u = 0; u < 16; ++u) s += (double)x[u];
    }
    if (k + 8 <= nctiles) {
        T x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = pp[(int64_t)(k + u) * n];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)x[u];
        k += 8;
    }
    for (; k < nctiles; ++k) s += (double)pp[(int64_t)k * n];
    s += rl;
    if (b0) s += bz;
    if (pm) s += pm[t];   // P3M: the mesh potential in place of the Ewald tiles
    const double* st = stats + 4 * r;
    if (ew) s += ew[t];   // EW2D: the 2D long-range sum with its constant, no background or dipole term
    else s += -PI * st[0] / (g.V * g.alpha * g.alpha);
    if (g.bc == CPM_BC_SLAB) s += (4.0 * PI / g.V) * sx[2 * n + i] * st[3];
    else if (g.bc == CPM_BC_WIRE) s += (2.0 * PI / g.V) * (sx[i] * st[1] + sx[n + i] * st[2]);
    const double v = KE * s;
    b[t] = v;
    if (bhl) {
        const float hi = (float)v;
        bhl[t] = make_float2(hi, (float)(v - (double)hi));
    }
}

// ----------------------------------------------------------------------------- driver
static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
struct BvecPlan {
    CellGrid cg;
    int splits, nctiles, ctiles, ztiles;
    int64_t chunk;
    size_t off_EX, off_EY, off_EZ, off_Q, off_rp, off_wr, off_part, off_real, off_stats, off_key, off_cnt, off_cur,
        off_nzc, off_start, off_wpos, off_sorted, off_order, off_c0part, off_c0w, off_b0, off_u, off_c0e1, off_ew,
        off_ewT, off_pm, off_p3m, total;
    int c0chunks;
    bool p3m;                           // reciprocal part of b by P3M (p3m.cu)
    bool tc;                            // reciprocal sums on the tensor cores (tc_recip.cu)
    size_t off_qabs, off_tcpart, off_w16, off_spart, off_qpart, off_c0q;
};

template <typename T>
static BvecPlan<T> plan_bvec(const cpm_ctx* c, int m, int64_t ne) {
    BvecPlan<T> p;
    const KTable& k = c->kt;
    p.cg = make_grid(c->g);
    p.ctiles = (k.ncols + SF_BM - 1) / SF_BM;
    // odd number 2h + 1 of BN-wide z tiles centred on nz = 0, covering -NZ..NZ
    const int zh = k.NZ + 1 - SF_BN / 2 > 0 ? (k.NZ + 1 - SF_BN / 2 + SF_BN - 1) / SF_BN : 0;
    p.ztiles = 2 * zh + 1;
    p.p3m = c->p.kspace == CPM_KSPACE_P3M;
    p.nctiles = p.p3m ? 0 : p.ctiles;
    p.tc = !p.p3m && std::is_same<T, float>::value && c->p.k_prec == CPM_PREC_F16X2 && tc_recip_supported(k);
    TcRecipDims td{};
    if (p.tc) {
        td = tc_recip_dims(c, m, ne);
        p.nctiles = td.ncb;
    }
    // the single-precision structure factor uses 128-harmonic super-tiles (k_sf32)
    const int zh2 = k.NZ + 1 - S2_BZ / 2 > 0 ? (k.NZ + 1 - S2_BZ / 2 + S2_BZ - 1) / S2_BZ : 0;
    const int yt = std::is_same<T, float>::value ? 2 * zh2 + 1 : p.ztiles;
    const int64_t base = (int64_t)p.ctiles * yt * m;
    int64_t want = (4 * 152 + base - 1) / std::max<int64_t>(base, 1);
    int64_t maxs = std::max<int64_t>(1, (ne + 127) / 128);
    p.splits = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min<int64_t>(maxs, 64)));
    p.chunk = (ne + p.splits - 1) / p.splits;
    p.chunk = ((p.chunk + SF_BK - 1) / SF_BK) * SF_BK;
    const int64_t ptot = (int64_t)m * ne;
    const int64_t pph = p.p3m ? 0 : ptot;   // points with electrolyte phase tables (none with P3M)
    const size_t pe = phase_elems(k, pph);
    const size_t grid = (size_t)k.ncols * k.nzw;
    size_t o = 0;
    const int64_t tabX = (int64_t)(k.NX + 1) * pph, tabY = (int64_t)(2 * k.NY + 1) * pph;
    p.off_EX = o; o += al(sizeof(c2<T>) * tabX);
    p.off_EY = o; o += al(sizeof(c2<T>) * tabY);
    p.off_EZ = o; o += al(sizeof(c2<T>) * (pe - tabX - tabY));
    p.off_Q = o; o += al(sizeof(T) * ptot);
    if (p.tc || p.p3m) {   // the CUDA-core structure-factor buffers are not used
        p.off_rp = p.off_wr = o;
    } else {
        p.off_rp = o; o += al(sizeof(c2<T>) * grid * m * p.splits);
        p.off_wr = o; o += al(sizeof(c2<T>) * grid * m);
    }
    p.off_part = o; o += al(sizeof(T) * (size_t)m * p.nctiles * c->n);
    p.off_real = o; o += al(sizeof(double) * (size_t)m * c->n);
    p.off_stats = o; o += al(sizeof(double) * 4 * m);
    p.off_key = o; o += al(sizeof(int) * ptot);
    p.off_cnt = o; o += al(sizeof(int) * ((size_t)m * p.cg.ncells + 1));
    p.off_cur = o; o += al(sizeof(int) * ((size_t)m * p.cg.ncells + 1));
    p.off_nzc = o; o += al(sizeof(int) * (size_t)m);
    p.off_start = o; o += al(sizeof(int) * ((size_t)m * p.cg.ncells + 1));
    p.off_wpos = o; o += al(sizeof(typename V4<T>::t) * ptot);
    p.off_sorted = o; o += al(sizeof(typename V4<T>::t) * ptot);
    p.off_order = o; o += al(sizeof(int) * ptot);
    p.c0chunks = (int)std::max<int64_t>(1, (ne + C0_THREADS * C0_PER_THREAD - 1) / (C0_THREADS * C0_PER_THREAD));
    const int nz0 = std::max(std::min(k.ext0, COL0_NZ), 1);
    p.off_c0part = o; o += al(sizeof(double2) * (size_t)m * p.c0chunks * nz0);
    p.off_c0w = o; o += al(sizeof(double2) * (size_t)m * nz0);
    p.off_b0 = o; o += al(sizeof(double) * (size_t)m * std::max(c->nzu, 1));
    p.off_u = o; o += al(sizeof(uint64_t) * 3 * pph);
    p.off_c0e1 = o; o += al(sizeof(float4) * pph);
    p.off_c0q = o; o += al(sizeof(float2) * pph);
    p.off_qabs = o; o += al(sizeof(float2) * m);
    p.off_spart = o; o += al(sizeof(double) * ST_Q * (size_t)std::max<int64_t>(1, (ne + ST_THREADS - 1) / ST_THREADS) * m);
    p.off_qpart = o; o += al(sizeof(double) * 2 * (size_t)std::max<int64_t>(1, (ne + FR_THREADS - 1) / FR_THREADS) * m);
    p.off_ew = p.off_ewT = o;
    if (c->g.bc == CPM_BC_EW2D) {
        p.off_ew = o; o += al(sizeof(double) * (size_t)m * c->n);
        p.off_ewT = o; o += al(ew2d_T_bytes(c, m));
    }
    p.off_pm = p.off_p3m = o;
    if (p.p3m) {
        p.off_pm = o; o += al(sizeof(double) * (size_t)m * c->n);
        p.off_p3m = o; o += al(p3m_scratch_bytes<T>(c, m, ne));
    }
    p.off_tcpart = p.off_w16 = o;
    if (p.tc) {
        p.off_tcpart = o; o += al(tc_recip_part_bytes(td, m, k.nzw));
        p.off_w16 = o; o += al(tc_recip_w16_bytes(td));
    }
    p.total = o;
    return p;
}

template <typename T>
size_t bvec_scratch_bytes(const cpm_ctx* c, int m, int64_t ne) { return plan_bvec<T>(c, m, ne).total; }

template <typename T> static const Phases<T>& site_tables(const cpm_ctx* c);
template <> const Phases<double>& site_tables<double>(const cpm_ctx* c) { return c->site64; }
template <> const Phases<float>& site_tables<float>(const cpm_ctx* c) { return c->site32; }

template <typename T>
cpm_status bvec_run(cpm_ctx* c, int m, int64_t ne, const double* xyz, const double* Q, double* b_out, float2* bhl,
                    char* scr) {
    const BvecPlan<T> p = plan_bvec<T>(c, m, ne);
    const KTable& k = c->kt;
    cudaStream_t st = c->stream;
    const int64_t n = c->n, ptot = (int64_t)m * ne;
    c2<T>* EX = (c2<T>*)(scr + p.off_EX);
    c2<T>* EY = (c2<T>*)(scr + p.off_EY);
    c2<T>* EZ = (c2<T>*)(scr + p.off_EZ);
    T* Qv = (T*)(scr + p.off_Q);
    c2<T>* rp = (c2<T>*)(scr + p.off_rp);
    c2<T>* wr = (c2<T>*)(scr + p.off_wr);
    T* part = (T*)(scr + p.off_part);
    double* real = (double*)(scr + p.off_real);
    double* stats = (double*)(scr + p.off_stats);
    int* key = (int*)(scr + p.off_key);
    int* cnt = (int*)(scr + p.off_cnt);
    int* cur = (int*)(scr + p.off_cur);
    int* start = (int*)(scr + p.off_start);
    typedef typename V4<T>::t V4T;
    V4T* wpos = (V4T*)(scr + p.off_wpos);
    V4T* sorted = (V4T*)(scr + p.off_sorted);
    int* order = (int*)(scr + p.off_order);
    const int nc = m * p.cg.ncells;
    c->launches += 4 + (ptot > 0 ? 2 : 0) + ((k.nk > 0 && ptot > 0 && !p.p3m) ? 5 : 0);

    // Three chains: the origin stream bins the charges (per-replica totals) and runs the cell list and
    // the real-space sum; side stream 1 takes the fractions, the charges in the working precision and
    // their scales in one pass, then the phase tables and the reciprocal sums; side stream 2 sums the
    // k_perp = 0 column once the fractions are written.  k_combine joins them.  With per-kernel
    // profiling on, everything runs on the origin stream in the same order.
    const bool recip = k.nk > 0 && ptot > 0 && !p.p3m;
    const bool fork = !c->prof_on;
    cudaStream_t s0 = st, s1 = st, s2 = st;
    if (fork) {
        CPM_TRY(ensure_aux(c));
        s1 = c->aux[0];
        s2 = c->aux[1];
        CPM_CUDA(c, cudaEventRecord(c->fev[0], s0));
        CPM_CUDA(c, cudaStreamWaitEvent(s1, c->fev[0], 0));
    }
    if (recip) {
        prof_begin(c, CPM_K_PHASES);
        // the k_perp = 0 chain needs only the fractions: it starts after k_fracs
        CPM_TRY(launch_phases_u<T>(s1, c->g, k, xyz, Q, ne, m, (uint64_t*)(scr + p.off_u), Qv,
                                   (double*)(scr + p.off_qpart), c->tickets + m,
                                   p.tc ? (float2*)(scr + p.off_qabs) : nullptr, EX, EY, EZ,
                                   fork ? c->fev[1] : nullptr, p.tc ? TC_ZSCALE : 1.f));
        prof_end(c, CPM_K_PHASES);
    } else if (fork) {
        CPM_CUDA(c, cudaEventRecord(c->fev[1], s1));
    }
    if (fork) CPM_CUDA(c, cudaStreamWaitEvent(s2, c->fev[1], 0));
    double* b0 = nullptr;
    if (std::is_same<T, float>::value && k.ext0 > 0 && ptot > 0 && !p.p3m) {
        // the k_perp = 0 column in FP64 (its single-precision weights are zero)
        double2* c0part = (double2*)(scr + p.off_c0part);
        double2* c0w = (double2*)(scr + p.off_c0w);
        b0 = (double*)(scr + p.off_b0);
        prof_begin(c, CPM_K_COL0);
        const int nz0 = std::min(k.ext0, COL0_NZ);
        const int nblk = (nz0 + C0_NB - 1) / C0_NB;
        float4* e1s = (float4*)(scr + p.off_c0e1);
        float2* q0 = (float2*)(scr + p.off_c0q);
        CPM_TRY(launch_col0_inputs(s2, (const uint64_t*)(scr + p.off_u), Q, ptot, e1s, q0));
        k_col0_rho<<<dim3(p.c0chunks, nblk, m), C0_THREADS, 0, s2>>>(e1s, q0, ne, nz0, c0part);
        CPM_LAUNCH(c, "k_col0_rho");
        k_col0_reduce<<<(m * nz0 * 32 + 255) / 256, 256, 0, s2>>>(c0part, p.c0chunks, nz0, k.w, k.NZ, m, c0w);
        CPM_LAUNCH(c, "k_col0_reduce");
        k_col0_site<<<(m * c->nzu * 32 + 255) / 256, 256, 0, s2>>>(c->c0e, c->nzu, m, nz0, c0w, b0);
        CPM_LAUNCH(c, "k_col0_site");
        prof_end(c, CPM_K_COL0);
        c->launches += 4;
    }
    // binning and the per-replica totals (one pass over the charges)
    prof_begin(c, CPM_K_CELLS);
    float2* qabs = (float2*)(scr + p.off_qabs);
    CPM_CUDA(c, cudaMemsetAsync(cnt, 0, p.off_start - p.off_cnt, st));   // counts, cursors, nonzero counts
    int* nzc = (int*)(scr + p.off_nzc);
    {
        const float3 inv_h = make_float3((float)(1.0 / p.cg.h[0]), (float)(1.0 / p.cg.h[1]), (float)(1.0 / p.cg.h[2]));
        const unsigned nbx = (unsigned)std::max<int64_t>(1, (ne + ST_THREADS - 1) / ST_THREADS);
        k_bin<T><<<dim3(nbx, m), ST_THREADS, 0, st>>>(xyz, Q, ne, c->g, p.cg, inv_h, key, cnt, wpos,
                                                     (double*)(scr + p.off_spart), c->tickets, stats, nzc);
        CPM_LAUNCH(c, "k_bin");
    }
    prof_end(c, CPM_K_CELLS);
    if (recip) {
        if (p.tc) {
            c->stream = s1;   // tc_recip_run launches on the context stream
            const cpm_status rs = tc_recip_run(c, m, ne, (const float2*)EX, (const float2*)EY, (const float2*)EZ,
                                               (const float*)Qv, qabs, scr + p.off_tcpart, scr + p.off_w16,
                                               (float*)part);
            c->stream = s0;
            CPM_TRY(rs);
        } else {
        prof_begin(c, CPM_K_SF);
        if (std::is_same<T, float>::value) {
            const int zh2 = k.NZ + 1 - S2_BZ / 2 > 0 ? (k.NZ + 1 - S2_BZ / 2 + S2_BZ - 1) / S2_BZ : 0;
            const int nsup = 2 * zh2 + 1;
            dim3 gsf(p.ctiles, nsup, m * p.splits);
            k_sf32<<<gsf, 256, 0, s1>>>(k.cols, k.colext, k.ncols, k.NY, k.NZ, k.nzw, (const float2*)EX,
                                        (const float2*)EY, (const float2*)EZ, (const float*)Qv, ptot, ne, p.splits,
                                        p.chunk, m, nsup, (float2*)rp);
        } else {
            dim3 gsf(p.ctiles, p.ztiles, m * p.splits);
            k_sf<T><<<gsf, 256, 0, s1>>>(k.cols, k.colext, k.ncols, k.NY, k.NZ, k.nzw, EX, EY, EZ, Qv, ptot, ne,
                                         p.splits, p.chunk, m, rp);
        }
        prof_end(c, CPM_K_SF);
        CPM_LAUNCH(c, "k_sf");
        prof_begin(c, CPM_K_SFRED);
        const int64_t per_rep = (int64_t)k.ncols * k.nzw;
        const T* w = std::is_same<T, float>::value ? (const T*)k.w32 : (const T*)k.w;
        k_sf_reduce<T><<<(unsigned)((per_rep * m + 255) / 256), 256, 0, s1>>>(rp, w, per_rep, m, p.splits, wr);
        prof_end(c, CPM_K_SFRED);
        CPM_LAUNCH(c, "k_sf_reduce");
        prof_begin(c, CPM_K_SITE);
        const Phases<T>& sp = site_tables<T>(c);
        if (std::is_same<T, float>::value) {
            dim3 gs((unsigned)((n + T2_BS - 1) / T2_BS), p.ctiles, m);
            k_site32<<<gs, 256, 0, s1>>>(k.cols, k.colext, k.ncols, k.NY, k.NZ, k.nzw, (const float2*)wr,
                                         (const float2*)sp.X, (const float2*)sp.Y, (const float2*)sp.Z, n, p.nctiles,
                                         (float*)part);
        } else {
            dim3 gs((unsigned)((n + SF_BN - 1) / SF_BN), p.ctiles, m);
            k_site<T><<<gs, 256, 0, s1>>>(k.cols, k.colext, k.ncols, k.NY, k.NZ, k.nzw, wr, sp.X, sp.Y, sp.Z, n,
                                          p.nctiles, part);
        }
        prof_end(c, CPM_K_SITE);
        CPM_LAUNCH(c, "k_site");
        }
    } else if (p.nctiles > 0) {
        CPM_CUDA(c, cudaMemsetAsync(part, 0, sizeof(T) * (size_t)m * p.nctiles * n, s1));
    }
    double* pm = nullptr;
    if (p.p3m && ptot > 0) {
        pm = (double*)(scr + p.off_pm);
        prof_begin(c, CPM_K_P3M);
        CPM_TRY(p3m_run<T>(c, s1, m, ne, xyz, Q, scr + p.off_p3m, pm));
        prof_end(c, CPM_K_P3M);
    }
    double* ew = nullptr;
    if (c->g.bc == CPM_BC_EW2D) {
        ew = (double*)(scr + p.off_ew);
        prof_begin(c, CPM_K_SF);
        CPM_TRY(ew2d_run<T>(c, s1, m, ne, xyz, Q, scr + p.off_ewT, ew));
        prof_end(c, CPM_K_SF);
    }
    prof_begin(c, CPM_K_CELLS);
    k_cellscan<<<m, CS_THREADS, 0, st>>>(cnt, start, p.cg.ncells, ne, m, nzc);
    CPM_LAUNCH(c, "k_cellscan");
    if (ptot > 0) {
        k_scatter<<<(unsigned)((ptot + 255) / 256), 256, 0, st>>>(key, start, cur, ptot, order);
        CPM_LAUNCH(c, "k_scatter");
        k_cellsort<T><<<(unsigned)(((int64_t)nc * 32 + 255) / 256), 256, 0, st>>>(start, nc, order, wpos, sorted);
        CPM_LAUNCH(c, "k_cellsort");
    }
    prof_end(c, CPM_K_CELLS);
    prof_begin(c, CPM_K_REAL);
    if (std::is_same<T, float>::value && c->rpoly.deg) {
        CPM_TRY(real_poly_run(c, st, m, p.cg, start, (const float4*)sorted, real));
    } else if (std::is_same<T, float>::value && c->rtab && c->schunks) {
        const int4* ch4 = (const int4*)c->schunks;
        const float4* tab4 = (const float4*)c->rtab;
        const unsigned rg = real_grid(c->nschunk, m);
        if (c->nrtab == 1)
            k_real_cells<true, true><<<rg, 32 * RC_WARPS, 0, st>>>(c->s32, c->sperm, ch4, c->nschunk, n, c->g, p.cg,
                                                                  start, (const float4*)sorted, tab4, c->nrtab,
                                                                  c->rtab_id, m, c->rqueue, real);
        else if (c->nrtab <= RC_SMEM_TABS)
            k_real_cells<true, false><<<rg, 32 * RC_WARPS, 0, st>>>(c->s32, c->sperm, ch4, c->nschunk, n, c->g, p.cg,
                                                                   start, (const float4*)sorted, tab4, c->nrtab,
                                                                   c->rtab_id, m, c->rqueue, real);
        else
            k_real_cells<false, false><<<rg, 32 * RC_WARPS, 0, st>>>(c->s32, c->sperm, ch4, c->nschunk, n, c->g,
                                                                    p.cg, start, (const float4*)sorted, tab4,
                                                                    c->nrtab, c->rtab_id, m, c->rqueue, real);
    } else {
        k_real_b<T><<<(unsigned)(((int64_t)m * n * 32 + 255) / 256), 256, 0, st>>>(c->sx, n, m, c->g, p.cg, start,
                                                                                    sorted, (const float4*)c->rtab,
                                                                                    c->rtab_id, real);
    }
    prof_end(c, CPM_K_REAL);
    CPM_LAUNCH(c, "k_real_b");
    if (fork) {
        CPM_CUDA(c, cudaEventRecord(c->fev[3], s1));
        CPM_CUDA(c, cudaEventRecord(c->fev[4], s2));
        CPM_CUDA(c, cudaStreamWaitEvent(s0, c->fev[3], 0));
        CPM_CUDA(c, cudaStreamWaitEvent(s0, c->fev[4], 0));
    }
    prof_begin(c, CPM_K_COMBINE);
    k_combine<T><<<(unsigned)(((int64_t)m * n + 255) / 256), 256, 0, st>>>(part, p.nctiles, real, b0, c->zmap, c->nzu,
                                                                          stats, c->sx, n, m, c->g, b_out, bhl, ew,
                                                                          pm);
    prof_end(c, CPM_K_COMBINE);
    CPM_LAUNCH(c, "k_combine");
    return CPM_OK;
}

// phase factors of the k_perp = 0 column at the distinct site heights (after the k table)
cpm_status build_col0_sites(cpm_ctx* c) {
    dev_free(c, c->c0e);
    c->c0e = nullptr;
    const int nz0 = std::min(c->kt.ext0, COL0_NZ);
    if (nz0 <= 0 || c->nzu == 0) return CPM_OK;
    CPM_TRY(dev_alloc(c, (void**)&c->c0e, sizeof(double2) * (size_t)c->nzu * nz0));
    k_col0_e0<<<(c->nzu * nz0 + 255) / 256, 256, 0, c->stream>>>(c->zuniq, c->nzu, c->g.inv[2], nz0, c->c0e);
    CPM_LAUNCH(c, "k_col0_e0");
    return CPM_OK;
}

cpm_status ensure_aux(cpm_ctx* c) {
    for (cudaStream_t& s : c->aux)
        if (!s) CPM_CUDA(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (cudaEvent_t& e : c->fev)
        if (!e) CPM_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return CPM_OK;
}

cpm_status reserve_bvec(cpm_ctx* c, int m, int64_t ne) {
    const bool f32 = c->p.k_prec != CPM_PREC_FP64;
    CPM_TRY(ensure_aux(c));
    CPM_TRY(ensure_tickets(c, 2 * m));   // k_bin takes [0, m), k_fracs [m, 2m)
    return ensure_scratch(c, f32 ? bvec_scratch_bytes<float>(c, m, ne) : bvec_scratch_bytes<double>(c, m, ne));
}

cpm_status bvec(cpm_ctx* c, int m, int64_t ne, const double* xyz, const double* Q, double* b_out, float2* bhl) {
    const bool f32 = c->p.k_prec != CPM_PREC_FP64;
    const size_t need = f32 ? bvec_scratch_bytes<float>(c, m, ne) : bvec_scratch_bytes<double>(c, m, ne);
    CPM_TRY(ensure_scratch(c, need));
    CPM_TRY(ensure_tickets(c, 2 * m));   // k_bin takes [0, m), k_fracs [m, 2m)
    char* scr = (char*)c->scratch;
    return f32 ? bvec_run<float>(c, m, ne, xyz, Q, b_out, bhl, scr) : bvec_run<double>(c, m, ne, xyz, Q, b_out, bhl, scr);
}

}  // namespace cpm
