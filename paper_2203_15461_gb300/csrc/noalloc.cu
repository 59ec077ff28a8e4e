// cpm_bvec_noalloc: the electrolyte potential b for one configuration without any device
// allocation, for callers that cannot allocate device memory (see include/cpm.h).
//
// Its only scratch is the structure-factor grid below, a file-scope device array that
// every GPU loading this library holds until the process exits.  Host code must not pass
// the array's name to a kernel (on the host it is only a stand-in symbol); it passes the
// device address that cudaGetSymbolAddress returns, looked up on every call made outside stream
// capture.
#include <mutex>

#include "common.cuh"

namespace cpm {

// Dense (nx, ny, nz) grid of weighted structure factors w_k rho(k), at most this many entries.
constexpr int64_t NOALLOC_MAX_KGRID = (int64_t)1 << 18;   // 262,144 double2 = 4 MiB

static __device__ __align__(256) double2 g_noalloc_rho[NOALLOC_MAX_KGRID];

constexpr int NOALLOC_MAX_DEVICES = 64;
static double2* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_noalloc_mutex;

__device__ __forceinline__ uint64_t na_frac_fixed(double x, double invL) {
    double s = x * invL;
    s -= floor(s);
    double t = s * 18446744073709551616.0;
    return t >= 18446744073709551616.0 ? 0ull : (uint64_t)t;
}

// One thread per grid entry: writes w_k rho(k) for k in the half-space ball and zero elsewhere,
// so every entry the second kernel reads is written by this call.
__global__ void k_noalloc_rho(Geometry g, int NX, int NY, int NZ, const double* __restrict__ xyz,
                              const double* __restrict__ Q, int64_t ne, double2* __restrict__ rho) {
    const int64_t G = (int64_t)(NX + 1) * (2 * NY + 1) * (2 * NZ + 1);
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G) return;
    const int nz = (int)(t % (2 * NZ + 1)) - NZ;
    const int ny = (int)((t / (2 * NZ + 1)) % (2 * NY + 1)) - NY;
    const int nx = (int)(t / ((int64_t)(2 * NZ + 1) * (2 * NY + 1)));
    const double tx = (2.0 * PI) / g.boxL[0], ty = (2.0 * PI) / g.boxL[1], tz = (2.0 * PI) / g.boxL[2];
    double kx = __dmul_rn(tx, (double)nx), ky = __dmul_rn(ty, (double)ny), kz = __dmul_rn(tz, (double)nz);
    double k2 = __dadd_rn(__dadd_rn(__dmul_rn(kx, kx), __dmul_rn(ky, ky)), __dmul_rn(kz, kz));
    bool half = nx > 0 || (nx == 0 && ny > 0) || (nx == 0 && ny == 0 && nz > 0);
    double2 out = make_double2(0.0, 0.0);
    if (half && k2 <= __dmul_rn(g.kcut, g.kcut)) {
        double re = 0.0, im = 0.0;
        for (int64_t j = 0; j < ne; ++j) {
            double q = Q[j];
            if (q == 0.0) continue;
            uint64_t u = na_frac_fixed(xyz[3 * j], g.inv[0]) * (uint64_t)(int64_t)nx +
                         na_frac_fixed(xyz[3 * j + 1], g.inv[1]) * (uint64_t)(int64_t)ny +
                         na_frac_fixed(xyz[3 * j + 2], g.inv[2]) * (uint64_t)(int64_t)nz;
            double s, c;
            sincospi((double)(int64_t)u * 0x1p-63, &s, &c);
            re += q * c;
            im += q * s;
        }
        double w = (8.0 * PI / g.V) * exp(-k2 / (4.0 * g.alpha * g.alpha)) / k2;
        out = make_double2(w * re, w * im);
    }
    rho[t] = out;
}

// One thread per site: reciprocal sum over the grid, direct real-space sum over all charges and
// their images within rcut, background and boundary terms.
__global__ void k_noalloc_site(Geometry g, int NX, int NY, int NZ, const double* __restrict__ sxyz,
                               const double* __restrict__ seta, int64_t n, const double* __restrict__ xyz,
                               const double* __restrict__ Q, int64_t ne, const double2* __restrict__ rho,
                               double* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double Ri[3] = {sxyz[3 * i], sxyz[3 * i + 1], sxyz[3 * i + 2]};
    const double eta = seta[i], a = g.alpha, rc = g.rcut, rc2 = rc * rc;
    const uint64_t ux = na_frac_fixed(Ri[0], g.inv[0]), uy = na_frac_fixed(Ri[1], g.inv[1]),
                   uz = na_frac_fixed(Ri[2], g.inv[2]);
    double acc = 0.0;
    int64_t t = 0;
    for (int nx = 0; nx <= NX; ++nx)
        for (int ny = -NY; ny <= NY; ++ny)
            for (int nz = -NZ; nz <= NZ; ++nz, ++t) {
                double2 r = rho[t];
                if (r.x == 0.0 && r.y == 0.0) continue;
                uint64_t u = ux * (uint64_t)(int64_t)nx + uy * (uint64_t)(int64_t)ny + uz * (uint64_t)(int64_t)nz;
                double s, c;
                sincospi((double)(int64_t)u * 0x1p-63, &s, &c);
                acc += c * r.x + s * r.y;   // Re[exp(-i k.R) w rho]
            }
    double qt = 0.0, M[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < ne; ++j) {
        const double q = Q[j];
        if (q == 0.0) continue;
        double d[3];
        int lo[3], hi[3];
        for (int k = 0; k < 3; ++k) {
            d[k] = Ri[k] - xyz[3 * j + k];
            M[k] += q * xyz[3 * j + k];
            lo[k] = (int)floor((-rc - d[k]) / g.boxL[k]);
            hi[k] = (int)ceil((rc - d[k]) / g.boxL[k]);
        }
        qt += q;
        for (int ix = lo[0]; ix <= hi[0]; ++ix)
            for (int iy = lo[1]; iy <= hi[1]; ++iy)
                for (int iz = lo[2]; iz <= hi[2]; ++iz) {
                    double dx = d[0] + ix * g.boxL[0], dy = d[1] + iy * g.boxL[1], dz = d[2] + iz * g.boxL[2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < rc2) {
                        double r = sqrt(r2);
                        acc += q * (erfc(a * r) - erfc(eta * r)) / r;
                    }
                }
    }
    acc += -PI * qt / (g.V * a * a);
    if (g.bc == CPM_BC_SLAB) acc += (4.0 * PI / g.V) * Ri[2] * M[2];
    else if (g.bc == CPM_BC_WIRE) acc += (2.0 * PI / g.V) * (Ri[0] * M[0] + Ri[1] * M[1]);
    b[i] = KE * acc;
}

}  // namespace cpm

using namespace cpm;

extern "C" cpm_status cpm_bvec_noalloc(const cpm_params* p, int64_t n, const double* site_xyz,
                                       const double* site_eta, int64_t n_e, const double* xyz, const double* Q,
                                       double* b_out, void* cuda_stream) {
    if (!p || n < 1 || n_e < 0 || !site_xyz || !site_eta || !b_out || (n_e > 0 && (!xyz || !Q))) return CPM_E_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(p->box[d] > 0.0)) return CPM_E_ARG;
    if (!(p->alpha > 0.0) || !(p->rcut > 0.0) || !(p->kcut > 0.0)) return CPM_E_ARG;
    if (p->boundary < CPM_BC_3D || p->boundary > CPM_BC_WIRE) return CPM_E_ARG;   // EW2D: not here
    if (p->kspace != CPM_KSPACE_EWALD) return CPM_E_ARG;                           // P3M: not here
    Geometry g;
    for (int d = 0; d < 3; ++d) { g.boxL[d] = p->box[d]; g.inv[d] = 1.0 / p->box[d]; }
    g.V = p->box[0] * p->box[1] * p->box[2];
    g.alpha = p->alpha; g.rcut = p->rcut; g.kcut = p->kcut; g.bc = p->boundary;
    // harmonics per axis, checked in floating point before any conversion to int: a grid that
    // cannot fit the scratch is refused without forming (and overflowing) its size
    double hd[3];
    for (int d = 0; d < 3; ++d) {
        hd[d] = g.kcut / ((2.0 * PI) / g.boxL[d]);
        if (!(hd[d] >= 0.0) || hd[d] > (double)NOALLOC_MAX_KGRID) return CPM_E_BUDGET;
    }
    const int NX = (int)hd[0] + 1, NY = (int)hd[1] + 1, NZ = (int)hd[2] + 1;
    const double Gd = (double)(NX + 1) * (double)(2 * NY + 1) * (double)(2 * NZ + 1);
    if (!(Gd >= 1.0) || Gd > (double)NOALLOC_MAX_KGRID) return CPM_E_BUDGET;   // larger than the fixed scratch
    const int64_t G = (int64_t)Gd;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return CPM_E_CUDA; }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return CPM_E_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // The array's device address is looked up again on every call made outside stream capture, so
    // a device reset or a new primary context between calls leaves no stale address behind; while
    // the stream is being captured only the address of an earlier call on this device is used.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) { cudaGetLastError(); return CPM_E_CUDA; }
    double2* rho = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (cap == cudaStreamCaptureStatusNone) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_rho) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return CPM_E_CUDA;
            }
            g_noalloc_addr[dev] = (double2*)ptr;
        } else if (!g_noalloc_addr[dev]) {
            return CPM_E_STATE;   // first call on this device inside a capture: no address yet
        }
        rho = g_noalloc_addr[dev];
    }
    k_noalloc_rho<<<(unsigned)((G + 127) / 128), 128, 0, st>>>(g, NX, NY, NZ, xyz, Q, n_e, rho);
    if (cudaGetLastError() != cudaSuccess) return CPM_E_CUDA;
    k_noalloc_site<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, NX, NY, NZ, site_xyz, site_eta, n, xyz, Q, n_e,
                                                               rho, b_out);
    if (cudaGetLastError() != cudaSuccess) return CPM_E_CUDA;
    return CPM_OK;
}
