// P3M (particle-particle particle-mesh) reciprocal part of the electrolyte vector b: the k-space
// solver the paper's package offers beside the Ewald sum (Introduction; SI Sec. 1.A-B), written
// after the textbook method of Hockney and Eastwood:
//   1. every charge is assigned to the p^3 nearest mesh points with the order-p cardinal B-spline
//      W(s) = M_p(s + p/2) per axis,
//   2. the mesh is Fourier transformed, multiplied by the optimal influence function for potentials
//        G(k) = sum_m U^2(k_m) R(k_m) / (sum_m U^2(k_m))^2,  k_m = k + 2 pi m / h,  m in [-2, 2]^3,
//        U(k) = prod_d sinc(k_d h_d / 2)^p,  R(k) = 4 pi exp(-k^2 / 4 alpha^2) / k^2,  G(0) = 0,
//      and transformed back,
//   3. the mesh potential is interpolated at the electrode sites with the same weights:
//        phi_i = (1/V) sum_mesh W_i(x) IFFT[G FFT[rho]](x).
// The elastance matrix A keeps the Ewald sum; only the per-step b takes this path.
//
// GPU design (one GPU, m replicas per launch):
// * Two replicas share one complex mesh (real part, imaginary part).  G is real and even on the
//   mesh, so IFFT(G FFT(rho_a + i rho_b)) = phi_a + i phi_b exactly: one complex transform serves
//   two replicas.
// * Charge assignment: one CTA per (mesh brick, replica pair) owns the brick's points in shared
//   memory and takes every charge whose stencil reaches into the brick, adding only the points it
//   owns.  Every mesh point is written by exactly one CTA, with a plain store: no halo exchange and
//   no global atomics.  Inside the brick the contributions are added as exact fixed-point integers
//   with 32-bit shared-memory atomics, so the mesh charge does not depend on the order of the
//   atomics and the whole path is deterministic.
// * Transforms: radix-2 decimation in time in shared memory with twiddles tabulated in FP64 on the
//   host.  The forward and inverse xy transforms take a whole plane per CTA; the z pass loads
//   16 z lines per CTA, transforms them forward, multiplies by G, transforms back and stores, so
//   the reciprocal-space product never leaves shared memory.
// * Interpolation: one warp per (site, replica pair); lanes take the p^2 (x, y) columns, each runs
//   over the p z points; the warp sum is a fixed butterfly.
// Arithmetic in T = double (k_prec = FP64) or float (the single-precision paths); the influence
// function is computed in FP64 and stored in T.
#include "common.cuh"

namespace cpm {

constexpr int P3M_THREADS = 256;
constexpr int P3M_ZTX = 16;                       // z lines per CTA of the z pass

__host__ __device__ inline int ilog2i(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

bool p3m_mesh_ok(const cpm_params* p) {
    if (p->p3m_order < 2 || p->p3m_order > 7) return false;
    for (int d = 0; d < 3; ++d) {
        const int K = p->p3m_mesh[d];
        if (K < 8 || K > P3M_MAX_MESH || (K & (K - 1))) return false;
    }
    const size_t cs = (p->k_prec == CPM_PREC_FP64 || p->p3m_matrix) ? 16 : 8;
    return (size_t)p->p3m_mesh[0] * p->p3m_mesh[1] * cs <= P3M_PLANE_BYTES;
}

// ----------------------------------------------------------------------------- influence function
// One thread per mesh point (x fastest); frequency index n_d = i_d for i_d < K_d / 2, else i_d - K_d
// (the ordering of a discrete Fourier transform).  Stores G / V in T.
template <typename T>
__global__ void k_p3m_green(int Kx, int Ky, int Kz, int P, double Lx, double Ly, double Lz, double alpha, double V,
                            T* __restrict__ G) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = (int64_t)Kx * Ky * Kz;
    if (t >= N) return;
    const int ix = (int)(t % Kx), iy = (int)((t / Kx) % Ky), iz = (int)(t / ((int64_t)Kx * Ky));
    const int K[3] = {Kx, Ky, Kz};
    const int I[3] = {ix, iy, iz};
    const double L[3] = {Lx, Ly, Lz};
    double u2[3][5], kk[3][5], den[3];
    for (int d = 0; d < 3; ++d) {
        const int nd = I[d] < K[d] / 2 ? I[d] : I[d] - K[d];
        den[d] = 0.0;
        for (int m = -2; m <= 2; ++m) {
            const double s = (double)nd / K[d] + m;
            const double sc = s == 0.0 ? 1.0 : sinpi(s) / (PI * s);
            double pw = 1.0;
            for (int e = 0; e < 2 * P; ++e) pw *= sc;
            u2[d][m + 2] = pw;
            den[d] += pw;
            kk[d][m + 2] = 2.0 * PI * (nd + (double)m * K[d]) / L[d];
        }
    }
    double num = 0.0;
    const double q = 1.0 / (4.0 * alpha * alpha);
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            for (int c = 0; c < 5; ++c) {
                const double k2 = kk[0][a] * kk[0][a] + kk[1][b] * kk[1][b] + kk[2][c] * kk[2][c];
                if (k2 > 0.0) num += u2[0][a] * u2[1][b] * u2[2][c] * (4.0 * PI * exp(-k2 * q) / k2);
            }
    const double dd = den[0] * den[1] * den[2];
    const double g = (ix == 0 && iy == 0 && iz == 0) ? 0.0 : num / (dd * dd);
    G[t] = (T)(g / V);
}

// ----------------------------------------------------------------------------- charge preparation
// Per charge: the first mesh index of its stencil per axis, packed as bx | by << 10 | bz << 20 (-1 for
// Q = 0), and (fx, fy, fz, Q) with f the offset of the point from that stencil's assignment origin:
// u = x K / L (wrapped into the cell), t = u - p/2, base = floor(t) + 1, f = t - floor(t).  The weight of
// mesh point base + a is then M_p(f + p - 1 - a).
template <typename T> struct P3mV4;
template <> struct P3mV4<float> { using t = float4; };
template <> struct P3mV4<double> { using t = double4_32a; };

template <typename T>
__global__ void k_p3m_prep(const double* __restrict__ xyz, const double* __restrict__ Q, int64_t ptot, Geometry g,
                           int Kx, int Ky, int Kz, int P, int* __restrict__ key, typename P3mV4<T>::t* __restrict__ fq) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ptot) return;
    const double q = Q[t];
    const int K[3] = {Kx, Ky, Kz};
    double f[3];
    int b[3];
    for (int d = 0; d < 3; ++d) {
        double s = xyz[3 * t + d] * g.inv[d];
        s -= floor(s);
        const double u = s * K[d] - 0.5 * P;
        const double fl = floor(u);
        f[d] = u - fl;
        int bi = ((int)fl + 1) % K[d];
        if (bi < 0) bi += K[d];
        b[d] = bi;
    }
    key[t] = q == 0.0 ? -1 : (b[0] | (b[1] << 10) | (b[2] << 20));
    typename P3mV4<T>::t v;
    v.x = (T)f[0]; v.y = (T)f[1]; v.z = (T)f[2]; v.w = (T)q;
    fq[t] = v;
}

// The p weights M_p(f + p - 1 - a), a = 0..p-1, of offset f in [0, 1), by the B-spline recursion
// M_1 = 1 on [0, 1), M_n(x) = (x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)) / (n - 1) evaluated at x = f + j.
template <typename T, int P>
__device__ __forceinline__ void bspline_weights(T f, T* w) {
    T m[P];   // m[j] = M_n(f + j), j = 0..n-1
    m[0] = (T)1;
#pragma unroll
    for (int j = 1; j < P; ++j) m[j] = (T)0;
#pragma unroll
    for (int n = 2; n <= P; ++n) {
        const T inv = (T)1 / (T)(n - 1);
#pragma unroll
        for (int j = n - 1; j >= 0; --j) {
            const T x = f + (T)j;
            const T lo = j > 0 ? m[j - 1] : (T)0;   // M_{n-1}(x - 1)
            m[j] = (x * m[j] + ((T)n - x) * lo) * inv;
        }
    }
#pragma unroll
    for (int a = 0; a < P; ++a) w[a] = m[P - 1 - a];
}

// ----------------------------------------------------------------------------- charge assignment
// grid (bricks, replica pairs, charge splits); a brick is BX x BY x BZ mesh points (x fastest), brick
// index bx fastest; split sp takes the chunks [sp cps, (sp + 1) cps) of NT charges of each replica.
// Those whose stencil reaches into the brick are compacted (warp ballots, then warp offsets) into
// shared memory with their 3 p weights and their stencil origin relative to the brick; then the
// chunk's (charge, z offset, y offset) items are spread over the threads, each adding its p x
// contributions that land in the brick.
// Every contribution is rounded to 2^-40 e (FP64: 2^-60 e) and added as exact integers split over
// 32-bit words, a = floor(v 2^20), then the next 20 bits (FP64: and 20 more), with native 32-bit
// shared-memory atomics; integer addition is associative, so the brick's charge does not depend on
// the order of the atomics.  The low words carry into the next after every chunk (a chunk adds at
// most 1,024 x 2^20 to a low word), and a wraps modulo 2^32, exact while the final charge of a mesh
// point stays below 2,048 e.  Brick
// rows are padded to BX + 1 words so that the x offsets of one charge fall in distinct banks.  The
// split's brick goes to its own partial mesh; the first transform sums the splits in split order.
template <typename T> struct P3mWords { static constexpr int n = std::is_same<T, double>::value ? 3 : 2; };
template <typename T> struct P3mSpreadThreads { static constexpr int n = std::is_same<T, double>::value ? 512 : 1024; };

template <typename T, int P>
__global__ void __launch_bounds__(P3mSpreadThreads<T>::n) k_p3m_spread(const int* __restrict__ key,
                                                                      const typename P3mV4<T>::t* __restrict__ fq,
                                                                      int64_t ne, int m, int Kx, int Ky, int Kz, int BX,
                                                                      int BY, int BZ, int cps,
                                                                      c2<T>* __restrict__ part) {
    constexpr int NW = P3mWords<T>::n;
    constexpr int NT = P3mSpreadThreads<T>::n;
    extern __shared__ __align__(16) unsigned char p3m_smem[];
    const int RX = BX + 1;                              // padded row
    const int NB = RX * BY * BZ;
    int* acc = (int*)p3m_smem;                          // [2 replicas][NW words][NB]
    T* sw = (T*)(acc + ((2 * NW * NB + 3) & ~3));       // [NT][3 p + 1]: weights x | y | z, then Q
    int* so = (int*)(sw + NT * (3 * P + 1));            // [NT]: origin sx | sy << 10 | sz << 20
    __shared__ int wcount[NT / 32];
    const int nbx = Kx / BX, nby = Ky / BY;
    const int bi = blockIdx.x;
    const int b0x = (bi % nbx) * BX, b0y = ((bi / nbx) % nby) * BY, b0z = (bi / (nbx * nby)) * BZ;
    const int pair = blockIdx.y;
    const int nrep = min(2, m - 2 * pair);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t jbeg = (int64_t)blockIdx.z * cps * NT;
    const int64_t jend = min(ne, jbeg + (int64_t)cps * NT);
    for (int i = threadIdx.x; i < 2 * NW * NB; i += NT) acc[i] = 0;
    for (int rep = 0; rep < nrep; ++rep) {
        const int64_t base = (int64_t)(2 * pair + rep) * ne;
        int* A = acc + rep * NW * NB;
        for (int64_t j0 = jbeg; j0 < jend; j0 += NT) {
            const int64_t j = j0 + threadIdx.x;
            bool sel = false;
            int sx = 0, sy = 0, sz = 0;
            if (j < jend) {
                const int kv = key[base + j];
                if (kv >= 0) {
                    sx = ((kv & 1023) - b0x + Kx) & (Kx - 1);
                    sy = (((kv >> 10) & 1023) - b0y + Ky) & (Ky - 1);
                    sz = ((kv >> 20) - b0z + Kz) & (Kz - 1);
                    sel = (sx < BX || sx + P - 1 >= Kx) && (sy < BY || sy + P - 1 >= Ky) &&
                          (sz < BZ || sz + P - 1 >= Kz);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, sel);
            if (lane == 0) wcount[wid] = __popc(bal);
            __syncthreads();   // also orders the previous chunk's reads of sw / so before the writes below
            int off = 0, L = 0;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) {
                const int cw = wcount[w];
                off += w < wid ? cw : 0;
                L += cw;
            }
            if (sel) {
                const int slot = off + __popc(bal & ((1u << lane) - 1u));
                const typename P3mV4<T>::t v = fq[base + j];
                T* w = sw + slot * (3 * P + 1);
                bspline_weights<T, P>(v.x, w);
                bspline_weights<T, P>(v.y, w + P);
                bspline_weights<T, P>(v.z, w + 2 * P);
                w[3 * P] = v.w;
                so[slot] = sx | (sy << 10) | (sz << 20);
            }
            __syncthreads();
            // items (charge, z offset c, y offset b): the y and z rows inside the brick, then p x points
            for (int it = threadIdx.x; it < L * P * P; it += NT) {
                const int sl = it / (P * P), cb = it - sl * (P * P);
                const int c = cb / P, b = cb - c * P;
                const int o = so[sl];
                int gy = ((o >> 10) & 1023) + b;
                if (gy >= Ky) gy -= Ky;
                int gz = (o >> 20) + c;
                if (gz >= Kz) gz -= Kz;
                if (gy >= BY || gz >= BZ) continue;
                const T* w = sw + sl * (3 * P + 1);
                const T wyz = w[3 * P] * w[P + b] * w[2 * P + c];
                const int ox = o & 1023;
                int* row = A + (gz * BY + gy) * RX;
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    int gx = ox + a;
                    if (gx >= Kx) gx -= Kx;
                    if (gx < BX) {
                        // v = hi 2^-20 + lo 2^-40 (+ lo2 2^-60): exact splits of the scaled contribution
                        if (std::is_same<T, double>::value) {
                            const double x = (double)(wyz * w[a]) * 1048576.0;   // 2^20
                            const double h = floor(x);
                            const double y = (x - h) * 1048576.0;
                            const double l = floor(y);
                            atomicAdd(&row[gx], (int)h);
                            atomicAdd(&row[NB + gx], (int)l);
                            atomicAdd(&row[2 * NB + gx], __double2int_rn((y - l) * 1048576.0));
                        } else {
                            const float x = (float)(wyz * w[a]) * 1048576.0f;
                            const float h = floorf(x);
                            atomicAdd(&row[gx], (int)h);
                            atomicAdd(&row[NB + gx], __float2int_rn((x - h) * 1048576.0f));
                        }
                    }
                }
            }
            {   // carry the low words (every point's words belong to one thread here)
                __syncthreads();
                for (int i = threadIdx.x; i < NB; i += NT) {
                    int lo = A[NB + i];
                    if (NW == 3) {
                        const int c = A[2 * NB + i];
                        lo += c >> 20;
                        A[2 * NB + i] = c & 0xFFFFF;
                    }
                    A[i] += lo >> 20;
                    A[NB + i] = lo & 0xFFFFF;
                }
            }
        }
    }
    __syncthreads();
    const int64_t N = (int64_t)Kx * Ky * Kz;
    c2<T>* out = part + ((int64_t)blockIdx.z * gridDim.y + pair) * N;
    for (int i = threadIdx.x; i < BX * BY * BZ; i += NT) {
        const int lx = i % BX, ly = (i / BX) % BY, lz = i / (BX * BY);
        const int at = (lz * BY + ly) * RX + lx;
        double v[2] = {0.0, 0.0};
        for (int r = 0; r < nrep; ++r) {
            const int* W = acc + r * NW * NB;
            v[r] = (double)W[at] * 0x1p-20 + (double)W[NB + at] * 0x1p-40;
            if (NW == 3) v[r] += (double)W[2 * NB + at] * 0x1p-60;
        }
        out[((int64_t)(b0z + lz) * Ky + (b0y + ly)) * Kx + (b0x + lx)] = cmake<T>((T)v[0], (T)v[1]);
    }
}

// ----------------------------------------------------------------------------- transforms
__device__ __forceinline__ int bitrev(int v, int lg) { return lg ? (int)(__brev((unsigned)v) >> (32 - lg)) : 0; }

// radix-2 decimation-in-time stages over `lines` transforms of length K = 2^lg held in shared memory
// at x[line * ls + i * es] (input in bit-reversed order, output natural); tw[j] = exp(-+ 2 pi i j / K)
template <typename T>
__device__ __forceinline__ void dit_stages(c2<T>* x, int K, int lg, int lines, int ls, int es, const c2<T>* tw) {
    const int half = K >> 1;
    for (int s = 1; s <= lg; ++s) {
        const int hs = 1 << (s - 1);
        for (int t = threadIdx.x; t < lines * half; t += blockDim.x) {
            int line, q;
            if (ls == 1) { line = t % lines; q = t / lines; }   // lines adjacent in memory: line fastest
            else { line = t / half; q = t - line * half; }
            const int j = q & (hs - 1);
            const int i0 = ((q >> (s - 1)) << s) + j, i1 = i0 + hs;
            const c2<T> w = tw[j << (lg - s)];
            c2<T>* p0 = x + line * ls + i0 * es;
            c2<T>* p1 = x + line * ls + i1 * es;
            const c2<T> a = *p0, b = cmul(*p1, w);
            *p0 = cmake<T>(a.x + b.x, a.y + b.y);
            *p1 = cmake<T>(a.x - b.x, a.y - b.y);
        }
        __syncthreads();
    }
}

// 2D transform of every (z plane, replica pair) over x and y; INV: exp(+i ...) (unnormalised).  The
// forward transform first sums the nsplit partial meshes of the charge assignment (split_stride
// elements apart) in split order.  Dynamic shared memory: the plane [Ky][Kx], then Kx/2 + Ky/2 twiddles.
template <typename T, bool INV>
__global__ void __launch_bounds__(P3M_THREADS) k_p3m_plane(c2<T>* __restrict__ mesh, int Kx, int Ky, int Kz,
                                                          const c2<T>* __restrict__ twx, const c2<T>* __restrict__ twy,
                                                          int nsplit, int64_t split_stride) {
    extern __shared__ __align__(16) unsigned char p3m_smem[];
    c2<T>* pl = (c2<T>*)p3m_smem;
    c2<T>* tx = pl + Kx * Ky;
    c2<T>* ty = tx + Kx / 2;
    const int lx = ilog2i(Kx), ly = ilog2i(Ky);
    for (int j = threadIdx.x; j < Kx / 2; j += P3M_THREADS) { c2<T> w = twx[j]; if (INV) w.y = -w.y; tx[j] = w; }
    for (int j = threadIdx.x; j < Ky / 2; j += P3M_THREADS) { c2<T> w = twy[j]; if (INV) w.y = -w.y; ty[j] = w; }
    c2<T>* g = mesh + ((int64_t)blockIdx.y * Kz + blockIdx.x) * Kx * Ky;
    for (int i = threadIdx.x; i < Kx * Ky; i += P3M_THREADS) {
        const int x = i & (Kx - 1), y = i >> lx;
        c2<T> v = g[i];
        for (int sp = 1; sp < nsplit; ++sp) {   // the charge splits of the assignment, in split order
            const c2<T> u = g[sp * split_stride + i];
            v.x += u.x;
            v.y += u.y;
        }
        pl[bitrev(y, ly) * Kx + bitrev(x, lx)] = v;
    }
    __syncthreads();
    dit_stages<T>(pl, Kx, lx, Ky, Kx, 1, tx);    // rows: line = y (stride Kx), element stride 1
    dit_stages<T>(pl, Ky, ly, Kx, 1, Kx, ty);    // columns: line = x (stride 1), element stride Kx
    for (int i = threadIdx.x; i < Kx * Ky; i += P3M_THREADS) g[i] = pl[i];
}

// z pass: for P3M_ZTX adjacent x at one (y, replica pair): forward transform along z, times G / V,
// inverse transform along z.  Dynamic shared memory: [Kz][tx] lines, then Kz/2 twiddles.
template <typename T>
__global__ void __launch_bounds__(P3M_THREADS) k_p3m_zline(c2<T>* __restrict__ mesh, int Kx, int Ky, int Kz, int tx,
                                                          const T* __restrict__ G, const c2<T>* __restrict__ twz) {
    extern __shared__ __align__(16) unsigned char p3m_smem[];
    c2<T>* ln = (c2<T>*)p3m_smem;
    c2<T>* tw = ln + Kz * tx;
    const int lz = ilog2i(Kz);
    const int x0 = blockIdx.x * tx, y = blockIdx.y;
    const int64_t plane = (int64_t)Kx * Ky;
    c2<T>* g = mesh + (int64_t)blockIdx.z * plane * Kz + (int64_t)y * Kx + x0;
    for (int j = threadIdx.x; j < Kz / 2; j += P3M_THREADS) tw[j] = twz[j];
    for (int i = threadIdx.x; i < Kz * tx; i += P3M_THREADS) {
        const int z = i / tx, x = i - z * tx;
        ln[bitrev(z, lz) * tx + x] = g[z * plane + x];
    }
    __syncthreads();
    dit_stages<T>(ln, Kz, lz, tx, 1, tx, tw);
    for (int i = threadIdx.x; i < Kz * tx; i += P3M_THREADS) {
        const int z = i / tx, x = i - z * tx;
        const T gv = G[z * plane + (int64_t)y * Kx + x0 + x];
        ln[i] = cmake<T>(ln[i].x * gv, ln[i].y * gv);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < Kz * tx; i += P3M_THREADS) {   // natural -> bit-reversed order
        const int z = i / tx, x = i - z * tx;
        const int rz = bitrev(z, lz);
        if (z < rz) {
            const c2<T> a = ln[i];
            ln[i] = ln[rz * tx + x];
            ln[rz * tx + x] = a;
        }
    }
    for (int j = threadIdx.x; j < Kz / 2; j += P3M_THREADS) { c2<T> w = tw[j]; w.y = -w.y; tw[j] = w; }
    __syncthreads();
    dit_stages<T>(ln, Kz, lz, tx, 1, tx, tw);
    for (int i = threadIdx.x; i < Kz * tx; i += P3M_THREADS) {
        const int z = i / tx, x = i - z * tx;
        g[z * plane + x] = ln[i];
    }
}

// ----------------------------------------------------------------------------- interpolation
// One warp per (site, replica pair), warps site-fastest.  pm[r][i] = sum_stencil W phi (e/Angstrom).
template <typename T, int P>
__global__ void __launch_bounds__(P3M_THREADS) k_p3m_interp(const double* __restrict__ sx, int64_t n, int m,
                                                           Geometry g, int Kx, int Ky, int Kz,
                                                           const c2<T>* __restrict__ mesh, double* __restrict__ pm) {
    __shared__ T sw[P3M_THREADS / 32][3][8];
    __shared__ int sb[P3M_THREADS / 32][3];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (P3M_THREADS / 32) + wid;
    const int npairs = (m + 1) / 2;
    const bool live = w < n * npairs;
    const int64_t i = live ? w % n : 0;
    const int pair = live ? (int)(w / n) : 0;
    if (live && lane < 3) {
        const int K = lane == 0 ? Kx : (lane == 1 ? Ky : Kz);
        const double inv = lane == 0 ? g.inv[0] : (lane == 1 ? g.inv[1] : g.inv[2]);
        double s = sx[lane * n + i] * inv;
        s -= floor(s);
        const double u = s * K - 0.5 * P;
        const double fl = floor(u);
        int bi = ((int)fl + 1) % K;
        if (bi < 0) bi += K;
        sb[wid][lane] = bi;
        T wt[P];
        bspline_weights<T, P>((T)(u - fl), wt);
#pragma unroll
        for (int a = 0; a < P; ++a) sw[wid][lane][a] = wt[a];
    }
    __syncwarp();
    if (!live) return;
    const c2<T>* ph = mesh + (int64_t)pair * Kx * Ky * Kz;
    T re = (T)0, im = (T)0;
    for (int col = lane; col < P * P; col += 32) {
        const int a = col % P, b = col / P;
        const int gx = (sb[wid][0] + a) & (Kx - 1), gy = (sb[wid][1] + b) & (Ky - 1);
        const T wxy = sw[wid][0][a] * sw[wid][1][b];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const int gz = (sb[wid][2] + c) & (Kz - 1);
            const c2<T> v = ph[((int64_t)gz * Ky + gy) * Kx + gx];
            const T ww = wxy * sw[wid][2][c];
            re += ww * v.x;
            im += ww * v.y;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        pm[(int64_t)(2 * pair) * n + i] = (double)re;
        if (2 * pair + 1 < m) pm[(int64_t)(2 * pair + 1) * n + i] = (double)im;
    }
}

// ----------------------------------------------------------------------------- host side
static size_t p3m_al(size_t b) { return (b + 255) & ~(size_t)255; }

static int64_t mesh_pts(const cpm_ctx* c) {
    return (int64_t)c->p.p3m_mesh[0] * c->p.p3m_mesh[1] * c->p.p3m_mesh[2];
}

// Assignment bricks (32 x 16 x 8 points at most: 2 x 3 words of 33 x 16 x 8 points and the staged
// weights of a chunk fit in 227 KiB of shared memory) and charge splits: enough CTAs for four per SM of
// 152, no split without a chunk of charges, at most 8 partial meshes.
struct P3mSpread { int BX, BY, BZ, nbricks, nsplit, cps; };
template <typename T>
static P3mSpread p3m_spread_plan(const cpm_ctx* c, int m, int64_t ne) {
    P3mSpread sp;
    const int Kx = c->p.p3m_mesh[0], Ky = c->p.p3m_mesh[1], Kz = c->p.p3m_mesh[2];
    sp.BX = std::min(Kx, 32);
    sp.BY = std::min(Ky, 16);
    sp.BZ = std::min(Kz, 8);
    sp.nbricks = (Kx / sp.BX) * (Ky / sp.BY) * (Kz / sp.BZ);
    const int64_t ctas = (int64_t)sp.nbricks * ((m + 1) / 2);
    const int64_t nchunks = std::max<int64_t>(1, (ne + P3mSpreadThreads<T>::n - 1) / P3mSpreadThreads<T>::n);
    int64_t ns = std::max<int64_t>(1, (4 * 152 + ctas - 1) / ctas);
    ns = std::min<int64_t>(std::min<int64_t>(ns, 8), nchunks);
    sp.cps = (int)((nchunks + ns - 1) / ns);
    sp.nsplit = (int)((nchunks + sp.cps - 1) / sp.cps);
    return sp;
}

template <typename T>
size_t p3m_scratch_bytes(const cpm_ctx* c, int m, int64_t ne) {
    const int64_t ptot = (int64_t)m * ne;
    const P3mSpread sp = p3m_spread_plan<T>(c, m, ne);
    return p3m_al(sizeof(int) * ptot) + p3m_al(sizeof(typename P3mV4<T>::t) * ptot) +
           p3m_al(sizeof(c2<T>) * (size_t)sp.nsplit * ((m + 1) / 2) * mesh_pts(c));
}
template size_t p3m_scratch_bytes<float>(const cpm_ctx*, int, int64_t);
template size_t p3m_scratch_bytes<double>(const cpm_ctx*, int, int64_t);

template <typename T>
static cpm_status p3m_prepare_t(cpm_ctx* c, void** Gp, void** twp) {
    const int Kx = c->p.p3m_mesh[0], Ky = c->p.p3m_mesh[1], Kz = c->p.p3m_mesh[2];
    const int64_t N = mesh_pts(c);
    CPM_TRY(dev_alloc(c, Gp, sizeof(T) * N));
    CPM_TRY(dev_alloc(c, twp, sizeof(c2<T>) * (Kx + Ky + Kz) / 2));
    std::vector<c2<T>> tw((Kx + Ky + Kz) / 2);
    size_t o = 0;
    for (int K : {Kx, Ky, Kz})
        for (int j = 0; j < K / 2; ++j) {
            const double a = 2.0 * PI * j / K;
            tw[o++] = cmake<T>((T)std::cos(a), (T)-std::sin(a));
        }
    CPM_CUDA(c, cudaMemcpyAsync(*twp, tw.data(), sizeof(c2<T>) * tw.size(), cudaMemcpyHostToDevice, c->stream));
    k_p3m_green<T><<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(Kx, Ky, Kz, c->p.p3m_order, c->g.boxL[0],
                                                                     c->g.boxL[1], c->g.boxL[2], c->g.alpha, c->g.V,
                                                                     (T*)*Gp);
    CPM_LAUNCH(c, "k_p3m_green");
    // the twiddles are copied from pageable host memory: wait before the vector goes out of scope
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return CPM_OK;
}

cpm_status p3m_prepare(cpm_ctx* c) {
    if (c->p3m_G) return CPM_OK;   // depends on the cell and the parameters only
    if (c->p.k_prec == CPM_PREC_FP64) return p3m_prepare_t<double>(c, &c->p3m_G, &c->p3m_tw);
    CPM_TRY(p3m_prepare_t<float>(c, &c->p3m_G, &c->p3m_tw));
    if (c->p.p3m_matrix) CPM_TRY(p3m_prepare_t<double>(c, &c->p3m_G64, &c->p3m_tw64));   // the elastance: FP64
    return CPM_OK;
}

// the influence function and twiddles in T (the FP64 copies of a single-precision context for T = double)
template <typename T> static const T* p3m_green(const cpm_ctx* c) {
    return (const T*)((std::is_same<T, double>::value && c->p.k_prec != CPM_PREC_FP64) ? c->p3m_G64 : c->p3m_G);
}
template <typename T> static const c2<T>* p3m_twiddles(const cpm_ctx* c) {
    return (const c2<T>*)((std::is_same<T, double>::value && c->p.k_prec != CPM_PREC_FP64) ? c->p3m_tw64 : c->p3m_tw);
}

template <typename T, int P>
static cpm_status launch_p3m_pp(cudaStream_t st, cpm_ctx* c, int m, int64_t ne, const int* key,
                          const typename P3mV4<T>::t* fq, c2<T>* mesh, double* pm) {
    const int Kx = c->p.p3m_mesh[0], Ky = c->p.p3m_mesh[1], Kz = c->p.p3m_mesh[2];
    const P3mSpread sp = p3m_spread_plan<T>(c, m, ne);
    const int npairs = (m + 1) / 2;
    constexpr int NT = P3mSpreadThreads<T>::n;
    const size_t ssm = sizeof(int) * ((2 * P3mWords<T>::n * (sp.BX + 1) * sp.BY * sp.BZ + 3) & ~3) +
                       sizeof(T) * NT * (3 * P + 1) + sizeof(int) * NT;
    CPM_CUDA(c, cudaFuncSetAttribute(k_p3m_spread<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
    k_p3m_spread<T, P><<<dim3(sp.nbricks, npairs, sp.nsplit), NT, ssm, st>>>(key, fq, ne, m, Kx, Ky, Kz, sp.BX, sp.BY,
                                                                             sp.BZ, sp.cps, mesh);
    const int64_t sstride = (int64_t)npairs * Kx * Ky * Kz;
    const c2<T>* tw = p3m_twiddles<T>(c);
    const size_t psm = sizeof(c2<T>) * ((size_t)Kx * Ky + Kx / 2 + Ky / 2);
    CPM_CUDA(c, cudaFuncSetAttribute(k_p3m_plane<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
    CPM_CUDA(c, cudaFuncSetAttribute(k_p3m_plane<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
    k_p3m_plane<T, false><<<dim3(Kz, npairs), P3M_THREADS, psm, st>>>(mesh, Kx, Ky, Kz, tw, tw + Kx / 2, sp.nsplit,
                                                                      sstride);
    const int tx = std::min(Kx, P3M_ZTX);
    const size_t zsm = sizeof(c2<T>) * ((size_t)Kz * tx + Kz / 2);
    CPM_CUDA(c, cudaFuncSetAttribute(k_p3m_zline<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm));
    k_p3m_zline<T><<<dim3(Kx / tx, Ky, npairs), P3M_THREADS, zsm, st>>>(mesh, Kx, Ky, Kz, tx, p3m_green<T>(c),
                                                                        tw + Kx / 2 + Ky / 2);
    k_p3m_plane<T, true><<<dim3(Kz, npairs), P3M_THREADS, psm, st>>>(mesh, Kx, Ky, Kz, tw, tw + Kx / 2, 1, 0);
    const int64_t warps = c->n * npairs;
    k_p3m_interp<T, P><<<(unsigned)((warps + P3M_THREADS / 32 - 1) / (P3M_THREADS / 32)), P3M_THREADS, 0, st>>>(
        c->sx, c->n, m, c->g, Kx, Ky, Kz, mesh, pm);
    CPM_LAUNCH(c, "k_p3m (spread, transforms, interpolation)");
    return CPM_OK;
}

template <typename T>
cpm_status p3m_run(cpm_ctx* c, cudaStream_t st, int m, int64_t ne, const double* xyz, const double* Q, char* scr,
                   double* pm) {
    const int64_t ptot = (int64_t)m * ne;
    int* key = (int*)scr;
    typedef typename P3mV4<T>::t V4T;
    V4T* fq = (V4T*)(scr + p3m_al(sizeof(int) * ptot));
    c2<T>* mesh = (c2<T>*)(scr + p3m_al(sizeof(int) * ptot) + p3m_al(sizeof(V4T) * ptot));
    const int P = c->p.p3m_order;
    const int Kx = c->p.p3m_mesh[0], Ky = c->p.p3m_mesh[1], Kz = c->p.p3m_mesh[2];
    k_p3m_prep<T><<<(unsigned)((ptot + 255) / 256), 256, 0, st>>>(xyz, Q, ptot, c->g, Kx, Ky, Kz, P, key, fq);
    CPM_LAUNCH(c, "k_p3m_prep");
    c->launches += 6;
    switch (P) {
        case 2: return launch_p3m_pp<T, 2>(st, c, m, ne, key, fq, mesh, pm);
        case 3: return launch_p3m_pp<T, 3>(st, c, m, ne, key, fq, mesh, pm);
        case 4: return launch_p3m_pp<T, 4>(st, c, m, ne, key, fq, mesh, pm);
        case 5: return launch_p3m_pp<T, 5>(st, c, m, ne, key, fq, mesh, pm);
        case 6: return launch_p3m_pp<T, 6>(st, c, m, ne, key, fq, mesh, pm);
        default: return launch_p3m_pp<T, 7>(st, c, m, ne, key, fq, mesh, pm);
    }
}
// ----------------------------------------------------------------------------- the P3M elastance
__global__ void k_p3m_add_rows(double* __restrict__ A, const double* __restrict__ pm, int64_t cnt, double s) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) A[t] += s * pm[t];
}

// A <- (A + A^T) / 2 (the mesh operator is symmetric up to rounding): one thread per lower entry
__global__ void k_p3m_sym(double* __restrict__ A, int64_t n) {
    const int64_t i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= i || i >= n) return;
    const double v = 0.5 * (A[i * n + j] + A[j * n + i]);
    A[i * n + j] = v;
    A[j * n + i] = v;
}

__global__ void k_p3m_ones(double* __restrict__ q, int64_t cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) q[t] = 1.0;
}

cpm_status p3m_assemble_recip(cpm_ctx* c) {
    const int64_t n = c->n;
    const int B = (int)std::min<int64_t>(n, 512);   // sites per batch: every site one replica of one unit charge
    const size_t sbytes = p3m_scratch_bytes<double>(c, B, 1);
    char* scr = nullptr;
    double* pm = nullptr;
    double* ones = nullptr;
    cpm_status st = dev_alloc(c, (void**)&scr, sbytes);
    if (st == CPM_OK) st = dev_alloc(c, (void**)&pm, sizeof(double) * B * n);
    if (st == CPM_OK) st = dev_alloc(c, (void**)&ones, sizeof(double) * B);
    const int64_t l0 = c->launches;   // assembly work is not counted with the per-step launches
    if (st == CPM_OK) {
        k_p3m_ones<<<(B + 255) / 256, 256, 0, c->stream>>>(ones, B);
        for (int64_t r0 = 0; r0 < n && st == CPM_OK; r0 += B) {
            const int mb = (int)std::min<int64_t>(B, n - r0);
            st = p3m_run<double>(c, c->stream, mb, 1, c->sxyz + 3 * r0, ones, scr, pm);
            if (st == CPM_OK) {
                const int64_t cnt = (int64_t)mb * n;
                k_p3m_add_rows<<<(unsigned)((cnt + 255) / 256), 256, 0, c->stream>>>(c->A + r0 * n, pm, cnt, KE);
            }
        }
        if (st == CPM_OK) {
            k_p3m_sym<<<dim3((unsigned)((n + 255) / 256), (unsigned)n), 256, 0, c->stream>>>(c->A, n);
            st = cuda_check(c, cudaGetLastError(), "k_p3m (elastance)");
        }
    }
    c->launches = l0;
    if (scr || pm || ones) cudaStreamSynchronize(c->stream);   // the buffers are in use until the stream has passed
    dev_free(c, scr);
    dev_free(c, pm);
    dev_free(c, ones);
    return st;
}

template cpm_status p3m_run<float>(cpm_ctx*, cudaStream_t, int, int64_t, const double*, const double*, char*, double*);
template cpm_status p3m_run<double>(cpm_ctx*, cudaStream_t, int, int64_t, const double*, const double*, char*,
                                    double*);

}  // namespace cpm
