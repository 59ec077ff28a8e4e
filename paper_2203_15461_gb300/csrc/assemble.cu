// Elastance matrix A of Eq. (coulomb), Sec. II.A, for Gaussian electrode charges (Sec. III.B).
//
//   A_ij = K_E [ sum'_n (erfc(alpha r) - erfc(eta_ij r)) / r                      (real space)
//              + delta_ij (sqrt(2) eta_i - 2 alpha) / sqrt(pi) - pi / (V alpha^2)  (self, background)
//              + B_ij                                                              (Sec. II.E)
//              + sum_{k in half space} w_k Re[E_i(k) conj(E_j(k))] ]               (reciprocal space)
//
// with E_i(k) = exp(i k.R_i) = X_i[nx] Y_i[ny] Z_i[nz] from the site phase tables.
// The reciprocal part is a dense, symmetric contraction over the k-vector list;
// only lower-triangular 64 x 64 tiles are computed and mirrored.
#include "common.cuh"

namespace cpm {

// One thread per (i, j).  Writes the real-space, self, background and boundary terms.
__global__ void k_A_real(const double* __restrict__ sx, int64_t n, Geometry g, double* __restrict__ A) {
    const double* X = sx;
    const double* Y = sx + n;
    const double* Z = sx + 2 * n;
    const double* E = sx + 3 * n;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double rc = g.rcut, rc2 = __dmul_rn(rc, rc), a = g.alpha;
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
        double d[3] = {X[i] - X[j], Y[i] - Y[j], Z[i] - Z[j]};
        double ei = E[i], ej = E[j];
        double eij = ei * ej / sqrt(ei * ei + ej * ej);
        int lo[3], hi[3];
        for (int q = 0; q < 3; ++q) {
            lo[q] = (int)floor((-rc - d[q]) / g.boxL[q]);
            hi[q] = (int)ceil((rc - d[q]) / g.boxL[q]);
        }
        double acc = 0.0;
        for (int ix = lo[0]; ix <= hi[0]; ++ix) {
            double dx = __dadd_rn(d[0], __dmul_rn((double)ix, g.boxL[0]));
            for (int iy = lo[1]; iy <= hi[1]; ++iy) {
                double dy = __dadd_rn(d[1], __dmul_rn((double)iy, g.boxL[1]));
                double r2xy = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                for (int iz = lo[2]; iz <= hi[2]; ++iz) {
                    double dz = __dadd_rn(d[2], __dmul_rn((double)iz, g.boxL[2]));
                    double r2 = __dadd_rn(r2xy, __dmul_rn(dz, dz));
                    if (!(r2 < rc2)) continue;
                    if (i == j && ix == 0 && iy == 0 && iz == 0) continue;
                    double r = sqrt(r2);
                    acc += (erfc(a * r) - erfc(eij * r)) / r;
                }
            }
        }
        if (i == j) acc += (sqrt(2.0) * ei - 2.0 * a) / sqrt(PI);
        if (g.bc != CPM_BC_EW2D) acc += -PI / (g.V * a * a);
        if (g.bc == CPM_BC_SLAB) acc += (4.0 * PI / g.V) * (Z[i] * Z[j]);
        else if (g.bc == CPM_BC_WIRE) acc += (2.0 * PI / g.V) * (X[i] * X[j] + Y[i] * Y[j]);
        A[i * n + j] = KE * acc;
    }
}

// Reciprocal-space part, added to A.  Block (ti, tj) with ti >= tj; 256 threads, each a
// 4 x 4 strided sub-tile; operands generated on the fly from the phase tables.
constexpr int KA_BM = 64, KA_BK = 16;

__global__ void __launch_bounds__(256) k_A_recip(const double2* __restrict__ PX, const double2* __restrict__ PY,
                                                 const double2* __restrict__ PZ, int64_t n, int NY, int NZ,
                                                 const int4* __restrict__ klist, const double* __restrict__ kw,
                                                 int64_t nk, double* __restrict__ A) {
    __shared__ double2 Ea[KA_BK][KA_BM];
    __shared__ double2 Eb[KA_BK][KA_BM];
    // lower-triangular tile index
    int64_t b = blockIdx.x;
    int ti = (int)floor((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((int64_t)(ti + 1) * (ti + 2) / 2 <= b) ++ti;
    while ((int64_t)ti * (ti + 1) / 2 > b) --ti;
    int tj = (int)(b - (int64_t)ti * (ti + 1) / 2);
    const int64_t i0 = (int64_t)ti * KA_BM, j0 = (int64_t)tj * KA_BM;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;

    for (int64_t k0 = 0; k0 < nk; k0 += KA_BK) {
        for (int e = threadIdx.x; e < KA_BK * KA_BM * 2; e += 256) {
            int side = e / (KA_BK * KA_BM);
            int r = e % (KA_BK * KA_BM);
            int m = r % KA_BM, kk = r / KA_BM;
            int64_t k = k0 + kk;
            int64_t p = (side ? j0 : i0) + m;
            double2 v = make_double2(0.0, 0.0);
            if (k < nk && p < n) {
                int4 kv = klist[k];
                double2 ex = PX[(int64_t)kv.z * n + p];
                double2 ey = PY[(int64_t)(kv.w + NY) * n + p];
                double2 ez = PZ[(int64_t)(kv.y + NZ) * n + p];
                v = cmul(cmul(ex, ey), ez);
                if (!side) { double wk = kw[k]; v.x *= wk; v.y *= wk; }
            }
            if (side) Eb[kk][m] = v; else Ea[kk][m] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KA_BK; ++kk) {
            double2 av[4], bv[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) av[p] = Ea[kk][ty + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q] = Eb[kk][tx + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += av[p].x * bv[q].x + av[p].y * bv[q].y;
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int64_t i = i0 + ty + 16 * p;
        if (i >= n) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int64_t j = j0 + tx + 16 * q;
            if (j >= n) continue;
            if (ti == tj && j > i) continue;   // diagonal tile: lower half, mirrored below
            double v = KE * acc[p][q];
            A[i * n + j] += v;
            if (i != j) A[j * n + i] += v;
        }
    }
}

cpm_status assemble_A(cpm_ctx* c) {
    const int64_t n = c->n;
    dim3 g1((unsigned)((n + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
    k_A_real<<<g1, 256, 0, c->stream>>>(c->sx, n, c->g, c->A);
    CPM_LAUNCH(c, "k_A_real");
    if (c->g.bc == CPM_BC_EW2D) return assemble_ew2d(c);
    if (c->p.kspace == CPM_KSPACE_P3M && c->p.p3m_matrix) return p3m_assemble_recip(c);
    if (c->kt.nk > 0) {
        const int64_t nt = (n + KA_BM - 1) / KA_BM;
        const int64_t blocks = nt * (nt + 1) / 2;
        k_A_recip<<<(unsigned)blocks, 256, 0, c->stream>>>(c->site64.X, c->site64.Y, c->site64.Z, n, c->kt.NY,
                                                           c->kt.NZ, c->kt.klist, c->kt.kw, c->kt.nk, c->A);
        CPM_LAUNCH(c, "k_A_recip");
    }
    return CPM_OK;
}

}  // namespace cpm
