// Exact 2D-periodic slab sum (EW2D, Sec. II.E; Parry's and Heyes' 2D Ewald sum) in place of the
// 3D reciprocal sum, its neutralising background and the dipole term of Eq. (ew3dc_slab).
//
// The long-range erf(alpha r) / r part of every pair, summed over the in-plane lattice, with rho
// the in-plane and z the normal displacement and A = Lx Ly:
//   (2 pi / A) sum_{h in the half plane} cos(h . rho) / |h| F(|h|, z)
//     - (2 pi / A) [z erf(alpha z) + exp(-alpha^2 z^2) / (alpha sqrt(pi))],
//   F(h, z) = e^{h z} erfc(h / 2 alpha + alpha z) + e^{-h z} erfc(h / 2 alpha - alpha z).
// A net charge per cell has no defined energy in 2D, so A is fixed up to c e e^T (S and every
// neutral result do not depend on c): c = (2 pi / A) L_z with L_z the cell height given by the
// caller, and b carries the matching c Q_tot.
//
// F does not factor into site and charge parts, but the electrode sites sit on few layers: per
// step, for every 2D vector h and layer height z_u,
//   T(h, u) = (2 pi / (A |h|)) sum_j Q_j exp(-i h . rho_j) F(|h|, z_u - z_j)
// (one block per (h, replica), threads over the charges, the layers in chunks), then
//   b_i += sum_h Re[exp(i h . rho_i) T(h, u_i)] + H0(u_i) + c Q_tot.
// The work is N_h x layers x N_e instead of N_h x n x N_e.  The phases come from exact 64-bit
// fixed-point fractions of x / Lx and y / Ly.
#include "common.cuh"

namespace cpm {

constexpr int EW_T = 256;
constexpr int EW_LC = 8;   // layers per pass of a block

__device__ __forceinline__ uint64_t ew_frac(double x, double invL) {
    double s = x * invL;
    s -= floor(s);
    const double t = s * 18446744073709551616.0;
    return t >= 18446744073709551616.0 ? 0ull : (uint64_t)t;
}

template <typename T> __device__ __forceinline__ T ew_zf(T h, T z, T a);
template <> __device__ __forceinline__ double ew_zf<double>(double h, double z, double a) {
    double out = 0.0;
    const double h2a = h / (2.0 * a), g = -h2a * h2a - (a * z) * (a * z);
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
        const double s = sg ? -1.0 : 1.0;
        const double x = h2a + s * a * z;
        out += x >= 0.0 ? erfcx(x) * exp(g) : exp(s * h * z) * erfc(x);
    }
    return out;
}
template <> __device__ __forceinline__ float ew_zf<float>(float h, float z, float a) {
    float out = 0.f;
    const float h2a = h / (2.f * a), g = -h2a * h2a - (a * z) * (a * z);
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
        const float s = sg ? -1.f : 1.f;
        const float x = h2a + s * a * z;
        out += x >= 0.f ? erfcxf(x) * expf(g) : expf(s * h * z) * erfcf(x);
    }
    return out;
}

__device__ __forceinline__ double ew_h0(double z, double a) {
    return z * erf(a * z) + exp(-(a * z) * (a * z)) / (a * 1.7724538509055160273);
}

// A_ij += K_E [(2 pi / A) sum_h cos(h . rho_ij) F(|h|, z_ij) / |h| - (2 pi / A) h0(z_ij) + c], i >= j, mirrored
__global__ void k_A_ew2d(const double* __restrict__ sx, int64_t n, Geometry g, const int2* __restrict__ hidx,
                         const double* __restrict__ hn, int nh, double* __restrict__ A) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double pre = 2.0 * PI / (g.boxL[0] * g.boxL[1]);
    const uint64_t uxj = ew_frac(sx[j], g.inv[0]), uyj = ew_frac(sx[n + j], g.inv[1]);
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
        if (i < j) continue;
        const uint64_t dux = ew_frac(sx[i], g.inv[0]) - uxj, duy = ew_frac(sx[n + i], g.inv[1]) - uyj;
        const double z = sx[2 * n + i] - sx[2 * n + j];
        double acc = 0.0;
        for (int k = 0; k < nh; ++k) {
            const int2 h = hidx[k];
            const uint64_t u = dux * (uint64_t)(int64_t)h.x + duy * (uint64_t)(int64_t)h.y;
            const double c = cospi((double)(int64_t)u * 0x1p-63);
            acc += c * ew_zf<double>(hn[k], z, g.alpha) / hn[k];
        }
        const double v = KE * pre * (acc - ew_h0(z, g.alpha) + g.boxL[2]);
        A[i * n + j] += v;
        if (i != j) A[j * n + i] += v;
    }
}

// T[r][k][u] (k = 0: the h = 0 term H0 in .x; k >= 1: vector k - 1) and Qtot[r]; block (k, r)
template <typename T>
__global__ void __launch_bounds__(EW_T) k_ew2d_T(const double* __restrict__ xyz, const double* __restrict__ Q,
                                                 int64_t ne, Geometry g, const int2* __restrict__ hidx,
                                                 const double* __restrict__ hn, int nh, const double* __restrict__ zu,
                                                 int nzu, double2* __restrict__ Tout, double* __restrict__ qtot) {
    __shared__ double2 sh[EW_T / 32][EW_LC];
    __shared__ double shq[EW_T / 32];
    const int k = blockIdx.x, r = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double* xr = xyz + (int64_t)r * ne * 3;
    const double* qr = Q + (int64_t)r * ne;
    const double pre = 2.0 * PI / (g.boxL[0] * g.boxL[1]);
    const T a = (T)g.alpha;
    const int2 h = k > 0 ? hidx[k - 1] : make_int2(0, 0);
    const T hh = k > 0 ? (T)hn[k - 1] : (T)0;
    double2* out = Tout + ((int64_t)r * (nh + 1) + k) * nzu;
    if (k == 0) {   // the replica's total charge, for the constant term
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < ne; j += EW_T) s += qr[j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) shq[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < EW_T / 32; ++w) t += shq[w];
            qtot[r] = t;
        }
        __syncthreads();
    }
    for (int u0 = 0; u0 < nzu; u0 += EW_LC) {
        const int nl = min(EW_LC, nzu - u0);
        T acc_re[EW_LC], acc_im[EW_LC];
#pragma unroll
        for (int l = 0; l < EW_LC; ++l) { acc_re[l] = (T)0; acc_im[l] = (T)0; }
        for (int64_t j = threadIdx.x; j < ne; j += EW_T) {
            const double q = qr[j];
            if (q == 0.0) continue;
            const double zj = xr[3 * j + 2];
            if (k == 0) {
#pragma unroll
                for (int l = 0; l < EW_LC; ++l)
                    if (l < nl) acc_re[l] += (T)(q * ew_h0(zu[u0 + l] - zj, g.alpha));
            } else {
                const uint64_t u = ew_frac(xr[3 * j], g.inv[0]) * (uint64_t)(int64_t)h.x +
                                   ew_frac(xr[3 * j + 1], g.inv[1]) * (uint64_t)(int64_t)h.y;
                T s, c;
                if (std::is_same<T, double>::value) {
                    double sd, cd;
                    sincospi((double)(int64_t)u * 0x1p-63, &sd, &cd);
                    s = (T)sd; c = (T)cd;
                } else {
                    float sf, cf;
                    sincospif((float)(int)(uint32_t)(u >> 32) * 0x1p-31f, &sf, &cf);
                    s = (T)sf; c = (T)cf;
                }
#pragma unroll
                for (int l = 0; l < EW_LC; ++l) {
                    if (l < nl) {
                        const T f = (T)q * ew_zf<T>(hh, (T)(zu[u0 + l] - zj), a);
                        acc_re[l] += f * c;      // Q exp(-i h.rho) F: (c, -s)
                        acc_im[l] -= f * s;
                    }
                }
            }
        }
#pragma unroll
        for (int l = 0; l < EW_LC; ++l) {
            double re = (double)acc_re[l], im = (double)acc_im[l];
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_down_sync(0xffffffffu, re, o);
                im += __shfl_down_sync(0xffffffffu, im, o);
            }
            if (lane == 0) sh[warp][l] = make_double2(re, im);
        }
        __syncthreads();
        if ((int)threadIdx.x < nl) {
            const int l = threadIdx.x;
            double re = 0.0, im = 0.0;
            for (int w = 0; w < EW_T / 32; ++w) { re += sh[w][l].x; im += sh[w][l].y; }
            const double f = k == 0 ? -pre : pre / (double)hn[k - 1];
            out[u0 + l] = make_double2(f * re, f * im);
        }
        __syncthreads();
    }
}

// ew[r][i] = sum_k Re[exp(i h.rho_i) T[r][k][u_i]] + H0[r][u_i] + c Q_tot[r]  (before K_E)
__global__ void k_ew2d_site(const double2* __restrict__ Tin, const double* __restrict__ qtot, int nh, int nzu,
                            const int* __restrict__ zmap, const int2* __restrict__ hidx,
                            const double2* __restrict__ PX, const double2* __restrict__ PY, int NY, int64_t n, int m,
                            Geometry g, double* __restrict__ ew) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * n) return;
    const int r = (int)(t / n);
    const int64_t i = t % n;
    const int u = zmap[i];
    const double2* Tr = Tin + (int64_t)r * (nh + 1) * nzu;
    double s = Tr[u].x;
    for (int k = 0; k < nh; ++k) {
        const int2 h = hidx[k];
        const double2 e = cmul(PX[(int64_t)h.x * n + i], PY[(int64_t)(h.y + NY) * n + i]);   // exp(i h.rho_i)
        const double2 v = Tr[(int64_t)(k + 1) * nzu + u];
        s += e.x * v.x - e.y * v.y;
    }
    s += 2.0 * PI / (g.boxL[0] * g.boxL[1]) * g.boxL[2] * qtot[r];
    ew[t] = s;
}

cpm_status build_ew2d(cpm_ctx* c) {
    dev_free(c, c->h2d_idx);
    dev_free(c, c->h2d_norm);
    c->h2d_idx = nullptr;
    c->h2d_norm = nullptr;
    c->nh2d = 0;
    if (c->g.bc != CPM_BC_EW2D) return CPM_OK;
    const Geometry& g = c->g;
    const double tx = (2.0 * PI) / g.boxL[0], ty = (2.0 * PI) / g.boxL[1];
    const int NX = (int)(g.kcut / tx) + 1, NY = (int)(g.kcut / ty) + 1;
    std::vector<int2> idx;
    std::vector<double> nrm;
    for (int nx = 0; nx <= NX; ++nx)
        for (int ny = -NY; ny <= NY; ++ny) {
            if (!(nx > 0 || (nx == 0 && ny > 0))) continue;
            const double kx = (double)nx * tx, ky = (double)ny * ty;
            const double h2 = kx * kx + ky * ky;
            if (h2 <= g.kcut * g.kcut) {
                idx.push_back(make_int2(nx, ny));
                nrm.push_back(std::sqrt(h2));
            }
        }
    if (NY > c->kt.NY || NX > c->kt.NX) return set_err(c, CPM_E_STATE, "EW2D: site phase tables too short");
    c->nh2d = (int)idx.size();
    CPM_TRY(dev_alloc(c, (void**)&c->h2d_idx, sizeof(int2) * std::max<size_t>(1, idx.size())));
    CPM_TRY(dev_alloc(c, (void**)&c->h2d_norm, sizeof(double) * std::max<size_t>(1, nrm.size())));
    if (!idx.empty()) {
        CPM_CUDA(c, cudaMemcpyAsync(c->h2d_idx, idx.data(), sizeof(int2) * idx.size(), cudaMemcpyHostToDevice, c->stream));
        CPM_CUDA(c, cudaMemcpyAsync(c->h2d_norm, nrm.data(), sizeof(double) * nrm.size(), cudaMemcpyHostToDevice, c->stream));
    }
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return CPM_OK;
}

cpm_status assemble_ew2d(cpm_ctx* c) {
    const int64_t n = c->n;
    dim3 g1((unsigned)((n + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
    k_A_ew2d<<<g1, 256, 0, c->stream>>>(c->sx, n, c->g, c->h2d_idx, c->h2d_norm, c->nh2d, c->A);
    CPM_LAUNCH(c, "k_A_ew2d");
    return CPM_OK;
}

size_t ew2d_T_bytes(const cpm_ctx* c, int m) {
    return sizeof(double2) * (size_t)m * (c->nh2d + 1) * std::max(c->nzu, 1) + sizeof(double) * (size_t)m;
}

template <typename T>
cpm_status ew2d_run(cpm_ctx* c, cudaStream_t st, int m, int64_t ne, const double* xyz, const double* Q, void* Tbuf,
                    double* ew) {
    double2* Tv = (double2*)Tbuf;
    double* qt = (double*)((char*)Tbuf + sizeof(double2) * (size_t)m * (c->nh2d + 1) * c->nzu);
    k_ew2d_T<T><<<dim3(c->nh2d + 1, m), EW_T, 0, st>>>(xyz, Q, ne, c->g, c->h2d_idx, c->h2d_norm, c->nh2d, c->zuniq,
                                                       c->nzu, Tv, qt);
    CPM_LAUNCH(c, "k_ew2d_T");
    k_ew2d_site<<<(unsigned)(((int64_t)m * c->n + 255) / 256), 256, 0, st>>>(Tv, qt, c->nh2d, c->nzu, c->zmap,
                                                                            c->h2d_idx, c->site64.X, c->site64.Y,
                                                                            c->kt.NY, c->n, m, c->g, ew);
    CPM_LAUNCH(c, "k_ew2d_site");
    c->launches += 2;
    return CPM_OK;
}

template cpm_status ew2d_run<float>(cpm_ctx*, cudaStream_t, int, int64_t, const double*, const double*, void*, double*);
template cpm_status ew2d_run<double>(cpm_ctx*, cudaStream_t, int, int64_t, const double*, const double*, void*, double*);

}  // namespace cpm
