// Reciprocal-space tables (the k-vector set and Ewald weights) and per-point phase tables.
//
// The k-vector set is the half space of k = 2 pi (nx/Lx, ny/Ly, nz/Lz) with
// 0 < |k| <= kcut; each vector carries the weight 2 (4 pi / V) exp(-k^2/4 alpha^2)/k^2
// of the Ewald reciprocal sum (ELECTRODE's ewald/electrode solver, SI Sec. 1.A),
// the factor 2 standing for the mirror vector -k.  Membership is decided with
// correctly rounded multiplies and adds in a fixed order so that the set does
// not depend on FMA contraction.
#include <type_traits>

#include "common.cuh"

namespace cpm {

__device__ __forceinline__ double k2_of(double tx, double ty, double tz, int nx, int ny, int nz) {
    double kx = __dmul_rn(tx, (double)nx), ky = __dmul_rn(ty, (double)ny), kz = __dmul_rn(tz, (double)nz);
    return __dadd_rn(__dadd_rn(__dmul_rn(kx, kx), __dmul_rn(ky, ky)), __dmul_rn(kz, kz));
}

// Single-block exclusive scan of `cnt` (int64) into `off` (cnt + 1 entries), deterministic.
__device__ void block_exclusive_scan(const int64_t* in, int64_t* off, int64_t cnt) {
    __shared__ int64_t s[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < cnt; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < cnt ? in[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < (int)blockDim.x; d <<= 1) {
            int64_t t = threadIdx.x >= (unsigned)d ? s[threadIdx.x - d] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < cnt) off[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[cnt] = carry;
}

// Columns (nx, ny) of the half plane whose transverse |k| is within kcut, sorted by the
// transverse |k|^2 (ties by (nx, ny)), so that the first column is k_perp = 0 and columns
// with similar nz extents share tiles.
__global__ void k_columns(int NX, int NY, double tx, double ty, double kc2, int64_t* flags, int64_t* off,
                          int2* cols, int* ncols) {
    const int64_t ncand = (int64_t)(NX + 1) * (2 * NY + 1);
    for (int64_t i = threadIdx.x; i < ncand; i += blockDim.x) {
        int nx = (int)(i / (2 * NY + 1)), ny = (int)(i % (2 * NY + 1)) - NY;
        bool half = nx > 0 || ny >= 0;
        flags[i] = (half && k2_of(tx, ty, 0.0, nx, ny, 0) <= kc2) ? 1 : 0;
    }
    __syncthreads();
    block_exclusive_scan(flags, off, ncand);
    __syncthreads();
    for (int64_t i = threadIdx.x; i < ncand; i += blockDim.x) {
        if (flags[i]) {
            int nx = (int)(i / (2 * NY + 1)), ny = (int)(i % (2 * NY + 1)) - NY;
            cols[off[i]] = make_int2(nx, ny);
        }
    }
    __syncthreads();
    const int nc = (int)off[ncand];
    int2* tmp = reinterpret_cast<int2*>(flags);   // flags are no longer needed
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        int2 a = cols[c];
        double ka = k2_of(tx, ty, 0.0, a.x, a.y, 0);
        int rank = 0;
        for (int d = 0; d < nc; ++d) {
            int2 b = cols[d];
            double kb = k2_of(tx, ty, 0.0, b.x, b.y, 0);
            rank += (kb < ka || (kb == ka && d < c)) ? 1 : 0;
        }
        tmp[rank] = a;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x) cols[c] = tmp[c];
    if (threadIdx.x == 0) *ncols = nc;
}

__global__ void k_weights(const int2* cols, int ncols, int NZ, double tx, double ty, double tz, double kc2,
                          double pref, double inv4a2, double* w, float* w32, int* colext) {
    const int nzw = 2 * NZ + 1;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ncols * nzw) return;
    int c = (int)(i / nzw), nz = (int)(i % nzw) - NZ;
    int2 cn = cols[c];
    bool half = cn.x > 0 || cn.y > 0 || nz > 0;
    double k2 = k2_of(tx, ty, tz, cn.x, cn.y, nz);
    double wt = 0.0;
    if (half && k2 <= kc2) {
        wt = pref * exp(-k2 * inv4a2) / k2;
        atomicMax(&colext[c], nz < 0 ? -nz : nz);
    }
    w[i] = wt;
    // The k_perp = 0 column carries the largest weights (the laterally averaged charge
    // profile); the single-precision path leaves its first COL0_NZ harmonics to a double-float
    // kernel.
    w32[i] = (cn.x == 0 && cn.y == 0 && nz <= COL0_NZ) ? 0.0f : (float)wt;
}

__global__ void k_colcounts(const int2* cols, const int* colext, int ncols, int64_t* cnt) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    int e = colext[c];
    bool origin = cols[c].x == 0 && cols[c].y == 0;
    cnt[c] = e < 0 ? 0 : (origin ? e : 2 * e + 1);
}

__global__ void k_scan1(const int64_t* cnt, int64_t* off, int64_t n) { block_exclusive_scan(cnt, off, n); }

__global__ void k_compact(const int2* cols, const int* colext, const int64_t* coloff, const double* w, int ncols,
                          int NZ, int4* klist, double* kw) {
    const int nzw = 2 * NZ + 1;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ncols * nzw) return;
    int c = (int)(i / nzw), nz = (int)(i % nzw) - NZ;
    double wt = w[i];
    if (wt == 0.0) return;
    int2 cn = cols[c];
    int lo = (cn.x == 0 && cn.y == 0) ? 1 : -colext[c];
    int64_t o = coloff[c] + (nz - lo);
    klist[o] = make_int4(c, nz, cn.x, cn.y);
    kw[o] = wt;
}

void free_ktable(cpm_ctx* c) {
    KTable& k = c->kt;
    dev_free(c, k.cols); dev_free(c, k.colext); dev_free(c, k.coloff); dev_free(c, k.w);
    dev_free(c, k.w32); dev_free(c, k.klist); dev_free(c, k.kw);
    k = KTable{};
}

cpm_status build_ktable(cpm_ctx* c) {
    free_ktable(c);
    KTable& k = c->kt;
    const Geometry& g = c->g;
    const double tx = (2.0 * PI) / g.boxL[0], ty = (2.0 * PI) / g.boxL[1], tz = (2.0 * PI) / g.boxL[2];
    // EW2D: no 3D reciprocal set (the 2D sum of ew2d.cu replaces it); the harmonic ranges, and with
    // them the site phase tables, still follow kcut
    const double kc2 = g.bc == CPM_BC_EW2D ? 0.0 : g.kcut * g.kcut;
    k.NX = (int)(g.kcut / tx) + 1;
    k.NY = (int)(g.kcut / ty) + 1;
    k.NZ = (int)(g.kcut / tz) + 1;
    k.nzw = 2 * k.NZ + 1;
    const int64_t ncand = (int64_t)(k.NX + 1) * (2 * k.NY + 1);
    int64_t *flags = nullptr, *off = nullptr;
    int* dn = nullptr;
    CPM_TRY(dev_alloc(c, (void**)&flags, ncand * sizeof(int64_t)));
    CPM_TRY(dev_alloc(c, (void**)&off, (ncand + 1) * sizeof(int64_t)));
    CPM_TRY(dev_alloc(c, (void**)&dn, sizeof(int)));
    CPM_TRY(dev_alloc(c, (void**)&k.cols, ncand * sizeof(int2)));
    k_columns<<<1, 1024, 0, c->stream>>>(k.NX, k.NY, tx, ty, kc2, flags, off, k.cols, dn);
    CPM_LAUNCH(c, "k_columns");
    CPM_CUDA(c, cudaMemcpyAsync(&k.ncols, dn, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, flags); dev_free(c, off); dev_free(c, dn);

    const int64_t grid = (int64_t)k.ncols * k.nzw;
    CPM_TRY(dev_alloc(c, (void**)&k.w, grid * sizeof(double)));
    CPM_TRY(dev_alloc(c, (void**)&k.w32, grid * sizeof(float)));
    CPM_TRY(dev_alloc(c, (void**)&k.colext, k.ncols * sizeof(int)));
    CPM_TRY(dev_alloc(c, (void**)&k.coloff, (k.ncols + 1) * sizeof(int64_t)));
    CPM_CUDA(c, cudaMemsetAsync(k.colext, 0xff, k.ncols * sizeof(int), c->stream));   // -1
    const double pref = 8.0 * PI / g.V, inv4a2 = 1.0 / (4.0 * g.alpha * g.alpha);
    k_weights<<<(unsigned)((grid + 255) / 256), 256, 0, c->stream>>>(k.cols, k.ncols, k.NZ, tx, ty, tz, kc2, pref,
                                                                    inv4a2, k.w, k.w32, k.colext);
    CPM_LAUNCH(c, "k_weights");
    CPM_CUDA(c, cudaMemcpyAsync(&k.ext0, k.colext, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    int64_t* cnt = nullptr;
    CPM_TRY(dev_alloc(c, (void**)&cnt, k.ncols * sizeof(int64_t)));
    k_colcounts<<<(k.ncols + 255) / 256, 256, 0, c->stream>>>(k.cols, k.colext, k.ncols, cnt);
    CPM_LAUNCH(c, "k_colcounts");
    k_scan1<<<1, 1024, 0, c->stream>>>(cnt, k.coloff, k.ncols);
    CPM_LAUNCH(c, "k_scan1");
    CPM_CUDA(c, cudaMemcpyAsync(&k.nk, k.coloff + k.ncols, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, cnt);
    CPM_TRY(dev_alloc(c, (void**)&k.klist, (k.nk > 0 ? k.nk : 1) * sizeof(int4)));
    CPM_TRY(dev_alloc(c, (void**)&k.kw, (k.nk > 0 ? k.nk : 1) * sizeof(double)));
    k_compact<<<(unsigned)((grid + 255) / 256), 256, 0, c->stream>>>(k.cols, k.colext, k.coloff, k.w, k.ncols,
                                                                     k.NZ, k.klist, k.kw);
    CPM_LAUNCH(c, "k_compact");
    return CPM_OK;
}

// ----------------------------------------------------------------------------- phase tables
// The phase 2 pi h x / L is reduced exactly: the fractional coordinate x / L mod 1
// is held as a 64-bit fixed-point number, so h times it modulo one turn is an
// exact integer product; only the final conversion to a half-turn count in
// [-1, 1) for sincospi rounds.
__device__ __forceinline__ uint64_t frac_fixed(double x, double invL) {
    double s = x * invL;
    s -= floor(s);
    double t = s * 18446744073709551616.0;   // 2^64
    return t >= 18446744073709551616.0 ? 0ull : (uint64_t)t;
}

template <typename T> __device__ __forceinline__ c2<T> phase_of(uint64_t u, int h);
template <> __device__ __forceinline__ double2 phase_of<double>(uint64_t u, int h) {
    int64_t p = (int64_t)(u * (uint64_t)(int64_t)h);
    double s, co;
    sincospi((double)p * 0x1p-63, &s, &co);
    return make_double2(co, s);
}
// single precision: bits 32..63 of h u (mod 2^64) are a signed 32-bit turn fraction (resolution
// 2^-31 turn, far below the sincospif error); two 32-bit multiplies and an int32 conversion
template <> __device__ __forceinline__ float2 phase_of<float>(uint64_t u, int h) {
    const uint32_t lo = (uint32_t)u, hi = (uint32_t)(u >> 32), hl = (uint32_t)h;
    uint32_t top = __umulhi(lo, hl) + hi * hl;   // (u * h) >> 32 mod 2^32 for h >= 0
    if (h < 0) top -= lo;                         // the sign extension of h contributes -lo * 2^32
    float s, co;
    sincospif((float)(int32_t)top * 0x1p-31f, &s, &co);
    return make_float2(co, s);
}

template <typename T>
__global__ void k_phases(const double* __restrict__ xyz, int64_t P, double ix, double iy, double iz, int NX,
                         int NY, int NZ, c2<T>* X, c2<T>* Y, c2<T>* Z) {
    const int nslot = (NX + 1) + (2 * NY + 1) + (2 * NZ + 1);
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * nslot) return;
    int slot = (int)(t / P);
    int64_t p = t % P;
    if (slot <= NX) {
        X[(int64_t)slot * P + p] = phase_of<T>(frac_fixed(xyz[3 * p + 0], ix), slot);
    } else if (slot <= NX + 2 * NY + 1) {
        int r = slot - (NX + 1);
        Y[(int64_t)r * P + p] = phase_of<T>(frac_fixed(xyz[3 * p + 1], iy), r - NY);
    } else {
        int r = slot - (NX + 1) - (2 * NY + 1);
        Z[(int64_t)r * P + p] = phase_of<T>(frac_fixed(xyz[3 * p + 2], iz), r - NZ);
    }
}

// The fixed-point fractions of each point once per axis (u[d][p]), then the tables from them:
// the table kernel then needs no FP64 arithmetic at all.  The same pass writes the charges in the
// working precision (Qv) and, when qabs is given, max |Q| and sum |Q| of each replica (the scales
// of the tensor-core reciprocal sums), so that the reciprocal chain needs nothing from the binning
// of the real-space chain: each block reduces its charges into part[r][b][2] (lane l takes threads
// l, l + 32, ..., then a shuffle tree) and the replica's last block adds the block values in block
// order.  grid (charge blocks, m); point p = r ne + j.
template <typename T>
__global__ void __launch_bounds__(FR_THREADS) k_fracs(const double* __restrict__ xyz, const double* __restrict__ Q,
                                                    int64_t ne, double ix, double iy, double iz,
                                                    uint64_t* __restrict__ u, T* __restrict__ Qv,
                                                    double* __restrict__ part, int* __restrict__ tickets,
                                                    float2* __restrict__ qabs) {
    const int b = blockIdx.x, nb = gridDim.x, r = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j = (int64_t)b * FR_THREADS + threadIdx.x;
    const int64_t P = (int64_t)gridDim.y * ne;
    double aq = 0.0;
    if (j < ne) {
        const int64_t p = (int64_t)r * ne + j;
        u[p] = frac_fixed(xyz[3 * p + 0], ix);
        u[P + p] = frac_fixed(xyz[3 * p + 1], iy);
        u[2 * P + p] = frac_fixed(xyz[3 * p + 2], iz);
        const double q = Q[p];
        Qv[p] = (T)q;
        aq = fabs(q);
    }
    if (!qabs) return;   // uniform
    __shared__ double sv[FR_THREADS];
    sv[threadIdx.x] = aq;
    __syncthreads();
    if (warp < 2) {   // warp 0: max |Q|, warp 1: sum |Q|
        double v = sv[lane];
        for (int k = 1; k < FR_THREADS / 32; ++k) v = warp == 0 ? fmax(v, sv[lane + 32 * k]) : v + sv[lane + 32 * k];
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = warp == 0 ? fmax(v, w) : v + w;
        }
        if (lane == 0) part[((int64_t)r * nb + b) * 2 + warp] = v;
    }
    if (!last_block_of(&tickets[r], nb)) return;
    __shared__ double buf[2][FR_THREADS];
    const volatile double* pv = part + (int64_t)r * nb * 2;
    double v = 0.0;
    for (int k0 = 0; k0 < nb; k0 += FR_THREADS) {
        const int k = k0 + threadIdx.x;
        if (k < nb) {
            buf[0][threadIdx.x] = pv[2 * k];
            buf[1][threadIdx.x] = pv[2 * k + 1];
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            const int t = threadIdx.x, cnt = min(FR_THREADS, nb - k0);
            for (int kk = 0; kk < cnt; ++kk) {
                const double x = buf[t][kk];
                v = (k0 == 0 && kk == 0) ? x : (t == 0 ? fmax(v, x) : v + x);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) qabs[r].x = (float)v;
    if (threadIdx.x == 1) qabs[r].y = (float)v;
}

// For the double-float k_perp = 0 column of the single-precision paths: the first z harmonic
// exp(2 pi i z / Lz) as a double-float pair (from the exactly reduced fraction, one FP64 sincospi)
// and the charge as a double-float pair.
__global__ void k_col0_inputs(const uint64_t* __restrict__ uz, const double* __restrict__ Q, int64_t P,
                              float4* __restrict__ e1, float2* __restrict__ q2) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double2 e = phase_of<double>(uz[p], 1);
    const float rh = (float)e.x, ih = (float)e.y;
    e1[p] = make_float4(rh, (float)(e.x - (double)rh), ih, (float)(e.y - (double)ih));
    const double qd = Q[p];
    const float qh = (float)qd;
    q2[p] = make_float2(qh, (float)(qd - (double)qh));
}

// grid (points / 256, slots): no index division per entry
template <typename T>
__global__ void k_phases_u(const uint64_t* __restrict__ u, int64_t P, int NX, int NY, int NZ, c2<T>* X, c2<T>* Y,
                           c2<T>* Z) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int slot = blockIdx.y;
    if (slot <= NX) {
        X[(int64_t)slot * P + p] = phase_of<T>(u[p], slot);
    } else if (slot <= NX + 2 * NY + 1) {
        int r = slot - (NX + 1);
        Y[(int64_t)r * P + p] = phase_of<T>(u[P + p], r - NY);
    } else {
        int r = slot - (NX + 1) - (2 * NY + 1);
        Z[(int64_t)r * P + p] = phase_of<T>(u[2 * P + p], r - NZ);
    }
}

// Single precision, one thread per (point, axis): the harmonics h = 8a + k >= 0 of the axis are
// products e^{2 pi i 8a f} e^{2 pi i k f} of sixteen exactly reduced phases at most (k = 0..7 and the
// multiples of 8, each from the fixed-point fraction f), one rounding more than a direct evaluation
// (below the precision the single-precision sums keep); h < 0 is the conjugate of -h.  The z table
// is multiplied by zscale (a power of two: exact).
// grid (points / 128, 3 axes)
__global__ void __launch_bounds__(128) k_phases_rows(const uint64_t* __restrict__ u, int64_t P, int NX, int NY,
                                                     int NZ, float2* __restrict__ X, float2* __restrict__ Y,
                                                     float2* __restrict__ Z, float zscale) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int axis = blockIdx.y;
    const int H = axis == 0 ? NX : axis == 1 ? NY : NZ;   // largest |h|
    float2* T = axis == 0 ? X : axis == 1 ? Y : Z;
    const int64_t h0row = axis == 0 ? 0 : H;              // row of h = 0
    const uint64_t f = u[(int64_t)axis * P + p];
    const float sc = axis == 2 ? zscale : 1.f;
    float2 base[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) base[k] = k <= H ? phase_of<float>(f, k) : make_float2(1.f, 0.f);
    for (int a = 0; 8 * a <= H; ++a) {
        const float2 g = a == 0 ? make_float2(1.f, 0.f) : phase_of<float>(f, 8 * a);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int h = 8 * a + k;
            if (h > H) break;
            const float2 b = base[k];
            float2 v = a == 0 ? b : make_float2(g.x * b.x - g.y * b.y, g.x * b.y + g.y * b.x);
            v.x *= sc;
            v.y *= sc;
            T[(h0row + h) * P + p] = v;
            if (axis != 0 && h > 0) T[(h0row - h) * P + p] = make_float2(v.x, -v.y);
        }
    }
}

cpm_status launch_col0_inputs(cudaStream_t st, const uint64_t* u, const double* Q, int64_t P, float4* e1,
                              float2* q2) {
    if (P == 0) return CPM_OK;
    k_col0_inputs<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(u + 2 * P, Q, P, e1, q2);
    return cudaGetLastError() == cudaSuccess ? CPM_OK : CPM_E_CUDA;
}

template <typename T>
cpm_status launch_phases_u(cudaStream_t st, const Geometry& g, const KTable& k, const double* xyz, const double* Q,
                           int64_t ne, int m, uint64_t* u, T* Qv, double* qpart, int* tickets, float2* qabs,
                           c2<T>* X, c2<T>* Y, c2<T>* Z, cudaEvent_t after_fracs, float zscale) {
    const int64_t P = (int64_t)m * ne;
    if (P == 0) return CPM_OK;
    k_fracs<T><<<dim3((unsigned)((ne + FR_THREADS - 1) / FR_THREADS), (unsigned)m), FR_THREADS, 0, st>>>(
        xyz, Q, ne, g.inv[0], g.inv[1], g.inv[2], u, Qv, qpart, tickets, qabs);
    if (after_fracs && cudaEventRecord(after_fracs, st) != cudaSuccess) return CPM_E_CUDA;
    if (std::is_same<T, float>::value) {
        k_phases_rows<<<dim3((unsigned)((P + 127) / 128), 3), 128, 0, st>>>(u, P, k.NX, k.NY, k.NZ, (float2*)X,
                                                                            (float2*)Y, (float2*)Z, zscale);
    } else {
        const int nslot = (k.NX + 1) + (2 * k.NY + 1) + (2 * k.NZ + 1);
        k_phases_u<T><<<dim3((unsigned)((P + 255) / 256), (unsigned)nslot), 256, 0, st>>>(u, P, k.NX, k.NY, k.NZ, X,
                                                                                          Y, Z);
    }
    return cudaGetLastError() == cudaSuccess ? CPM_OK : CPM_E_CUDA;
}
template cpm_status launch_phases_u<float>(cudaStream_t, const Geometry&, const KTable&, const double*, const double*,
                                           int64_t, int, uint64_t*, float*, double*, int*, float2*, float2*, float2*,
                                           float2*, cudaEvent_t, float);
template cpm_status launch_phases_u<double>(cudaStream_t, const Geometry&, const KTable&, const double*,
                                            const double*, int64_t, int, uint64_t*, double*, double*, int*, float2*,
                                            double2*, double2*, double2*, cudaEvent_t, float);

template <typename T>
cpm_status launch_phases(cudaStream_t st, const Geometry& g, const KTable& k, const double* xyz, int64_t P,
                         c2<T>* X, c2<T>* Y, c2<T>* Z) {
    const int nslot = (k.NX + 1) + (2 * k.NY + 1) + (2 * k.NZ + 1);
    const int64_t tot = P * nslot;
    if (tot == 0) return CPM_OK;
    k_phases<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(xyz, P, g.inv[0], g.inv[1], g.inv[2], k.NX, k.NY,
                                                               k.NZ, X, Y, Z);
    return cudaGetLastError() == cudaSuccess ? CPM_OK : CPM_E_CUDA;
}
template cpm_status launch_phases<float>(cudaStream_t, const Geometry&, const KTable&, const double*, int64_t,
                                         float2*, float2*, float2*);
template cpm_status launch_phases<double>(cudaStream_t, const Geometry&, const KTable&, const double*, int64_t,
                                          double2*, double2*, double2*);

size_t phase_elems(const KTable& k, int64_t P) {
    return (size_t)P * ((k.NX + 1) + (2 * k.NY + 1) + (2 * k.NZ + 1));
}

}  // namespace cpm
