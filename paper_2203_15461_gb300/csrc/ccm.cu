// Electrodes at prescribed total charge (constant charge method, Sec. II.C, Eq. ewise-conq), the
// thermo-potentiostat step (Sec. II.D, Eq. deissenbeck) and the finite-field site potentials
// (Sec. II.F, Eq. cpm-ffield), all on top of the CPM update q = S (v - b).
//
// Constant charge: with the capacitance matrix A^-1 the electrode totals are
//   q~ = G^T A^-1 (G v~ - b) = C~_A v~ - G^T A^-1 b,   C~_A = G^T A^-1 G,
// solved per replica for the electrode potentials v~, which the CPM then applies.  The context
// holds S = A^-1 - d d^T / (e^T d) (d = A^-1 e), SG = S G and u = d / (e^T d), so
//   G^T A^-1 b = (SG)^T b + (G^T u)(u^T b)(e^T d),   C~_A = G^T S G + (G^T u)(G^T u)^T (e^T d),
// and q = A^-1 (G v~ - b) = S (G v~ - b) + u Q with Q = sum q~ (e^T q = Q).  With symm = 0 the
// context's S is A^-1 itself and u = 0.  One block per replica forms the n-long dot products
// (FP64, fixed order), one thread solves the N_g x N_g system with the precomputed inverse of
// C~_A, and the potentials go to the ordinary update.
//
// Thermo-potentiostat (two electrodes): the present capacitor charge q (electrode 1 at +q,
// electrode 0 at -q) gives Delta v = v~_1 - v~_0 by the same relation; the new charge is
//   q' = q - C0 (Delta v - Delta v0)(1 - a) + X sqrt(k_B T C0 (1 - a^2)),  a = exp(-dt/tau),
// with C0 = g_1^T S g_1 and X the caller's standard normal number, and is applied by the constant
// charge relation.
//
// Finite field: the site potentials -Delta v0 zeta (zeta_i = z_i / L_z, plus one on the bottom
// electrode) enter the update through S zeta, kept as one more column next to SG.
#include "common.cuh"

namespace cpm {

constexpr int CC_T = 256;
constexpr double K_B_EV = 8.617333262e-5;   // Boltzmann constant, eV / K

// psi[r][g] (and for the thermo-potentiostat qcap_out, dv_out) from the replica's b
__global__ void __launch_bounds__(CC_T) k_ccm_solve(const double* __restrict__ b, int64_t n, const double* __restrict__ SG,
                                                    const double* __restrict__ u, int ng, const double* __restrict__ Cinv,
                                                    const double* __restrict__ gu, double etd, int symm, int mode,
                                                    const double* __restrict__ qtilde, const double* __restrict__ qcap,
                                                    const double* __restrict__ X, double dt, double tau, double T,
                                                    double dv0, double C0, double* __restrict__ psi,
                                                    double* __restrict__ qtot_target, double* __restrict__ qcap_out,
                                                    double* __restrict__ dv_out) {
    __shared__ double sh[CC_T / 32][17];
    const int r = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double* br = b + (int64_t)r * n;
    double acc[17];
#pragma unroll
    for (int g = 0; g < 17; ++g) acc[g] = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += CC_T) {
        const double bi = br[i];
        for (int g = 0; g < ng; ++g) acc[g] += SG[i * ng + g] * bi;
        if (symm) acc[16] += u[i] * bi;
    }
#pragma unroll
    for (int g = 0; g < 17; ++g) {
        double a = acc[g];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[warp][g] = a;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double base[16], rhs[16], v[16];
    double tu = 0.0;
    for (int w = 0; w < CC_T / 32; ++w) tu += sh[w][16];
    for (int g = 0; g < ng; ++g) {
        double t = 0.0;
        for (int w = 0; w < CC_T / 32; ++w) t += sh[w][g];
        base[g] = t + (symm ? gu[g] * tu * etd : 0.0);   // (G^T A^-1 b)_g
    }
    auto solve = [&](const double* qt) {
        for (int g = 0; g < ng; ++g) rhs[g] = qt[g] + base[g];
        for (int g = 0; g < ng; ++g) {
            double s = 0.0;
            for (int h = 0; h < ng; ++h) s += Cinv[g * ng + h] * rhs[h];
            v[g] = s;
        }
    };
    double qt[16];
    double Q = 0.0;
    if (mode == 0) {
        for (int g = 0; g < ng; ++g) { qt[g] = qtilde[(int64_t)r * ng + g]; Q += qt[g]; }
        solve(qt);
    } else {
        const double q = qcap[r];
        qt[0] = -q; qt[1] = q;
        solve(qt);
        const double dv = v[1] - v[0];
        const double a = exp(-dt / tau);
        const double qn = q - C0 * (dv - dv0) * (1.0 - a) + X[r] * sqrt(K_B_EV * T * C0 * (1.0 - a * a));
        qt[0] = -qn; qt[1] = qn;
        solve(qt);
        qcap_out[r] = qn;
        if (dv_out) dv_out[r] = dv;
    }
    for (int g = 0; g < ng; ++g) psi[(int64_t)r * ng + g] = v[g];
    if (qtot_target) qtot_target[r] = Q;
}

// q[r][i] += u_i Q_r and qtot[r] = the replica's sum (fixed order: strided partial sums, warp trees,
// warps in order); one block per replica
__global__ void __launch_bounds__(CC_T) k_ccm_total(double* __restrict__ q, const double* __restrict__ u, int64_t n,
                                                    const double* __restrict__ Qt, double* __restrict__ qtot) {
    __shared__ double sh[CC_T / 32];
    const int r = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double Q = Qt[r];
    double* qr = q + (int64_t)r * n;
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += CC_T) {
        const double v = qr[i] + u[i] * Q;
        qr[i] = v;
        a += v;
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) sh[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0 && qtot) {
        double t = 0.0;
        for (int w = 0; w < CC_T / 32; ++w) t += sh[w];
        qtot[r] = t;
    }
}

// zeta_i = z_i / L_z + [site i on the bottom electrode]
__global__ void k_zeta(const double* __restrict__ sx, const int* __restrict__ group, int64_t n, double invLz, int bottom,
                       double* __restrict__ zeta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) zeta[i] = sx[2 * n + i] * invLz + (group[i] == bottom ? 1.0 : 0.0);
}

// SGx[i][0..ng) = SG[i][:], SGx[i][ng] = sum_j S_ij zeta_j; one warp per row, fixed order
__global__ void k_sgx(const double* __restrict__ S, const double* __restrict__ zeta, const double* __restrict__ SG,
                      int64_t n, int ng, double* __restrict__ SGx) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double a = 0.0;
    for (int64_t j = lane; j < n; j += 32) a += S[i * n + j] * zeta[j];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) {
        for (int g = 0; g < ng; ++g) SGx[i * (ng + 1) + g] = SG[i * ng + g];
        SGx[i * (ng + 1) + ng] = a;
    }
}

// psi'[r] = (0, .., 0, -dv0[r])
__global__ void k_ff_psi(const double* __restrict__ dv0, int m, int ng, double* __restrict__ psi) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * (ng + 1)) return;
    const int r = t / (ng + 1), g = t % (ng + 1);
    psi[t] = g == ng ? -dv0[r] : 0.0;
}

// small dense inverse on the host (Gauss-Jordan with partial pivoting); false if singular
static bool invert_small(std::vector<double> a, int k, std::vector<double>& inv) {
    inv.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) inv[i * k + i] = 1.0;
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (std::fabs(a[r * k + c]) > std::fabs(a[p * k + c])) p = r;
        if (!(std::fabs(a[p * k + c]) > 0.0)) return false;
        if (p != c)
            for (int j = 0; j < k; ++j) { std::swap(a[p * k + j], a[c * k + j]); std::swap(inv[p * k + j], inv[c * k + j]); }
        const double d = a[c * k + c];
        for (int j = 0; j < k; ++j) { a[c * k + j] /= d; inv[c * k + j] /= d; }
        for (int r = 0; r < k; ++r) {
            if (r == c) continue;
            const double f = a[r * k + c];
            if (f == 0.0) continue;
            for (int j = 0; j < k; ++j) { a[r * k + j] -= f * a[c * k + j]; inv[r * k + j] -= f * inv[c * k + j]; }
        }
    }
    return true;
}

// Cinv, G^T u (device) and C0 (host) for the present S; built once per inversion / import
static cpm_status ccm_prepare(cpm_ctx* c) {
    if (c->ccm_ready) return CPM_OK;
    const int64_t n = c->n;
    const int ng = c->ng;
    std::vector<double> sg((size_t)n * ng), u(n);
    std::vector<int> gr(n);
    CPM_CUDA(c, cudaMemcpyAsync(sg.data(), c->SG, sizeof(double) * sg.size(), cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(u.data(), c->u, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(gr.data(), c->group, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<double> C((size_t)ng * ng, 0.0), gu(ng, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        for (int h = 0; h < ng; ++h) C[gr[i] * ng + h] += sg[(size_t)i * ng + h];
        gu[gr[i]] += u[i];
    }
    c->ccm_C0 = ng >= 2 ? C[1 * ng + 1] : 0.0;
    if (c->p.symm)
        for (int g = 0; g < ng; ++g)
            for (int h = 0; h < ng; ++h) C[g * ng + h] += gu[g] * gu[h] * c->etd;
    std::vector<double> inv;
    if (!invert_small(C, ng, inv)) return set_err(c, CPM_E_NOT_SPD, "electrode-wise capacitance matrix is singular");
    if (!c->ccm_buf) CPM_TRY(dev_alloc(c, (void**)&c->ccm_buf, sizeof(double) * (16 * 16 + 16 + 4 * 1024)));
    std::vector<double> up(inv);
    up.insert(up.end(), gu.begin(), gu.end());
    CPM_CUDA(c, cudaMemcpyAsync(c->ccm_buf, up.data(), sizeof(double) * up.size(), cudaMemcpyHostToDevice, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->ccm_ready = true;
    return CPM_OK;
}

static cpm_status ccm_scratch(cpm_ctx* c, int m, int width, double** psi, double** qt) {
    const size_t need = sizeof(double) * (size_t)m * (width + 1);
    if (c->ccm_scr_bytes < need) {
        dev_free(c, c->ccm_scr);
        c->ccm_scr = nullptr;
        c->ccm_scr_bytes = 0;
        CPM_TRY(dev_alloc(c, &c->ccm_scr, need));
        c->ccm_scr_bytes = need;
    }
    *psi = (double*)c->ccm_scr;
    *qt = *psi + (size_t)m * width;
    return CPM_OK;
}

cpm_status ccm_update(cpm_ctx* c, int m, int mode, const double* qtilde, const cpm_tp_params* tp, const double* qcap,
                      const double* X, const double* b, double* q, double* qtot, double* psi_out, double* qcap_out,
                      double* dv_out) {
    CPM_TRY(ccm_prepare(c));
    const int ng = c->ng;
    double *psi = nullptr, *Qt = nullptr;
    CPM_TRY(ccm_scratch(c, m, ng, &psi, &Qt));
    if (psi_out) psi = psi_out;
    const double* Cinv = c->ccm_buf;
    const double* gu = c->ccm_buf + ng * ng;
    k_ccm_solve<<<m, CC_T, 0, c->stream>>>(b, c->n, c->SG, c->u, ng, Cinv, gu, c->etd, c->p.symm, mode, qtilde, qcap, X,
                                           tp ? tp->dt : 0.0, tp ? tp->tau : 1.0, tp ? tp->T : 0.0,
                                           tp ? tp->dv0 : 0.0, c->ccm_C0, psi, mode == 0 ? Qt : nullptr, qcap_out,
                                           dv_out);
    CPM_LAUNCH(c, "k_ccm_solve");
    c->launches += 1;
    CPM_TRY(update(c, m, psi, b, q, qtot));
    if (mode == 0 && c->p.symm) {
        k_ccm_total<<<m, CC_T, 0, c->stream>>>(q, c->u, c->n, Qt, qtot);
        CPM_LAUNCH(c, "k_ccm_total");
        c->launches += 1;
    }
    return CPM_OK;
}

cpm_status ffield_update(cpm_ctx* c, int m, const double* dv0, const double* b, double* q, double* qtot) {
    const int64_t n = c->n;
    const int ng = c->ng;
    if (!c->SGx) {
        std::vector<double> z(n);
        std::vector<int> gr(n);
        CPM_CUDA(c, cudaMemcpyAsync(z.data(), c->sx + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
        CPM_CUDA(c, cudaMemcpyAsync(gr.data(), c->group, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
        CPM_CUDA(c, cudaStreamSynchronize(c->stream));
        double zs[2] = {0.0, 0.0};
        int64_t cnt[2] = {0, 0};
        for (int64_t i = 0; i < n; ++i) { zs[gr[i]] += z[i]; cnt[gr[i]] += 1; }
        if (!cnt[0] || !cnt[1]) return set_err(c, CPM_E_ARG, "finite field: both electrodes need sites");
        const int bottom = zs[0] / cnt[0] < zs[1] / cnt[1] ? 0 : 1;
        double* zeta = nullptr;
        CPM_TRY(dev_alloc(c, (void**)&zeta, sizeof(double) * n));
        CPM_TRY(dev_alloc(c, (void**)&c->SGx, sizeof(double) * n * (ng + 1)));
        k_zeta<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->sx, c->group, n, 1.0 / c->g.boxL[2], bottom, zeta);
        k_sgx<<<(unsigned)((n * 32 + 255) / 256), 256, 0, c->stream>>>(c->S, zeta, c->SG, n, ng, c->SGx);
        CPM_LAUNCH(c, "k_sgx");
        CPM_CUDA(c, cudaStreamSynchronize(c->stream));
        dev_free(c, zeta);
    }
    double *psi = nullptr, *Qt = nullptr;
    CPM_TRY(ccm_scratch(c, m, ng + 1, &psi, &Qt));
    k_ff_psi<<<(unsigned)((m * (ng + 1) + 255) / 256), 256, 0, c->stream>>>(dv0, m, ng, psi);
    CPM_LAUNCH(c, "k_ff_psi");
    c->launches += 1;
    c->sg_over = c->SGx;
    c->ng_over = ng + 1;
    cpm_status st = update(c, m, psi, b, q, qtot);
    c->sg_over = nullptr;
    c->ng_over = 0;
    return st;
}

void ccm_invalidate(cpm_ctx* c) {
    c->ccm_ready = false;
    dev_free(c, c->SGx);
    c->SGx = nullptr;
}

}  // namespace cpm

using namespace cpm;

extern "C" {

cpm_status cpm_update_ccm(cpm_ctx* c, int32_t m, const double* qtilde, const double* b, double* q_out,
                          double* qtot_out, double* vtilde_out) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_update_ccm before cpm_invert");
    if (m < 1 || !qtilde || !b || !q_out) return set_err(c, CPM_E_ARG, "cpm_update_ccm: need m >= 1 and non-null buffers");
    return ccm_update(c, m, 0, qtilde, nullptr, nullptr, nullptr, b, q_out, qtot_out, vtilde_out, nullptr, nullptr);
}

cpm_status cpm_update_tp(cpm_ctx* c, int32_t m, const cpm_tp_params* tp, const double* qcap, const double* X,
                         const double* b, double* q_out, double* qcap_out, double* dv_out) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_update_tp before cpm_invert");
    if (c->ng != 2) return set_err(c, CPM_E_ARG, "cpm_update_tp: the thermo-potentiostat takes two electrodes");
    if (m < 1 || !tp || !qcap || !X || !b || !q_out || !qcap_out)
        return set_err(c, CPM_E_ARG, "cpm_update_tp: need m >= 1 and non-null buffers");
    if (!(tp->dt > 0.0) || !(tp->tau > 0.0) || !(tp->T >= 0.0) || !std::isfinite(tp->dv0))
        return set_err(c, CPM_E_ARG, "cpm_update_tp: need dt > 0, tau > 0, T >= 0 and a finite dv0");
    return ccm_update(c, m, 1, nullptr, tp, qcap, X, b, q_out, nullptr, nullptr, qcap_out, dv_out);
}

cpm_status cpm_update_ffield(cpm_ctx* c, int32_t m, const double* dv0, const double* b, double* q_out,
                             double* qtot_out) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_update_ffield before cpm_invert");
    if (c->ng != 2) return set_err(c, CPM_E_ARG, "cpm_update_ffield: the finite-field method takes two electrodes");
    if (c->p.boundary != CPM_BC_3D)
        return set_err(c, CPM_E_ARG, "cpm_update_ffield: the finite-field method needs a fully periodic cell (CPM_BC_3D)");
    if (m < 1 || !dv0 || !b || !q_out) return set_err(c, CPM_E_ARG, "cpm_update_ffield: need m >= 1 and non-null buffers");
    return ffield_update(c, m, dv0, b, q_out, qtot_out);
}

}  // extern "C"
