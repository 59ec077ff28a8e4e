// Internal declarations shared by the CPM CUDA translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <type_traits>
#include <string>
#include <vector>

#include "cpm.h"

namespace cpm {

// Coulomb constant e / (4 pi eps0 Angstrom) in volts.
constexpr double KE = 14.399645;
constexpr double PI = 3.141592653589793;

// ----------------------------------------------------------------------------- complex helpers
template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };
template <typename T> using c2 = typename C2<T>::t;

template <typename T> __host__ __device__ __forceinline__ c2<T> cmake(T a, T b) { c2<T> r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
    V r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}

// ----------------------------------------------------------------------------- packed FP32 pairs
// Two FP32 values in one 64-bit register for the packed (f32x2) arithmetic of sm_100 and later;
// each lane of an operation rounds once, exactly like the scalar instruction.
__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up2(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// sum of the split partials of one output: FP64 partials added in FP64; FP32 pairs (sum, low part)
// added in double-float arithmetic (the exact error of each high-part addition, by the two-sum of
// Knuth, is carried in the low part) and converted to FP64 once
struct PartSumD {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double value() const { return v; }
};
struct PartSumF2 {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float2 x) {
        const float s = __fadd_rn(hi, x.x);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x.x, bb));
        lo = __fadd_rn(lo, __fadd_rn(e, x.y));
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
// ----------------------------------------------------------------------------- device status word
// Kernels never trap: they set one of these bits and return.  The host reads the
// word when it synchronises.
enum : unsigned { ST_NOT_SPD = 1u, ST_NONFINITE = 2u, ST_TIMEOUT = 4u };

// ----------------------------------------------------------------------------- reciprocal-space table
// Half-space reciprocal vectors organised as "columns" (nx, ny) with nx >= 0 and
// (nx > 0 or ny >= 0), each with the nz harmonics -NZ..NZ on a dense grid of
// width nzw = 2 NZ + 1.  The Ewald weight of an entry is zero outside the
// half-space ball 0 < |k| <= kcut, so the dense grid and the compact list hold
// the same set of vectors.
// Harmonics of the k_perp = 0 column that the single-precision paths sum in double-float; its
// higher harmonics (weights below ~1e-3 of the first for the usual splittings) go through the
// single-precision sums with the rest of the k set.
// charge phases of the tensor-core structure factor are written scaled by 2^14 (exact)
constexpr float TC_ZSCALE = 16384.f;
constexpr int COL0_NZ = 12;

struct KTable {
    int NX = 0, NY = 0, NZ = 0;
    int ncols = 0, nzw = 0;
    int ext0 = -1;                  // largest nz of the k_perp = 0 column (column 0), -1 if empty
    int64_t nk = 0;                 // number of vectors with nonzero weight
    int2* cols = nullptr;           // [ncols] (nx, ny)
    int* colext = nullptr;          // [ncols] largest |nz| with nonzero weight, -1 if none
    int64_t* coloff = nullptr;      // [ncols + 1] offsets of each column in the compact list
    double* w = nullptr;            // [ncols * nzw] dense weights (8 pi / V) e^{-k^2/4a^2} / k^2
    float* w32 = nullptr;
    int4* klist = nullptr;          // [nk] compact list: (column, nz, nx, ny)
    double* kw = nullptr;           // [nk] weight of each compact entry
};

// Phase tables of a point set: X[h][p] = exp(2 pi i h x_p / Lx) for h = 0..NX,
// Y[h + NY][p] for h = -NY..NY, Z[h + NZ][p] for h = -NZ..NZ (point-minor layout).
template <typename T> struct Phases {
    c2<T>* X = nullptr;
    c2<T>* Y = nullptr;
    c2<T>* Z = nullptr;
    int64_t P = 0;       // points per set (ld of the tables)
};

struct CellGrid {
    int nc[3];
    int S[3];        // stencil half-widths (cells)
    double h[3];     // cell edges
    int ncells;
};

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Single-precision pair function f(r) = (erfc(alpha r) - erfc(eta r)) / r of a site's Gaussian width
// eta, tabulated as RT_N cubic Hermite pieces on [0, rcut] plus an all-zero row (index RT_N) for
// distances at or past the cut-off; one table per distinct eta.
constexpr int RT_N = 1024;
constexpr int RT_S = RT_N + 1;   // rows per table

// Outside the Gaussian cores the same pair function as e^{-alpha^2 r^2} P(r) / r, P a polynomial in
// v = r s1 + s0 replacing erfcx(alpha r) on [r_lo, r_c] (real_poly.cu), r_lo the smallest core radius.
constexpr int RP_DEG_MAX = 14;
struct RealPoly {
    float c[RP_DEG_MAX + 1];   // monomial coefficients of P in v
    float s1, s0;              // v = r s1 + s0 maps [r_lo, r_c] onto [-1, 1]
    float ke;                  // -alpha^2 log2(e): e^{-alpha^2 r^2} = 2^(ke r^2)
    float rc2;                 // r_c^2 in FP32
    int deg;                   // 0: not available (the tabulated kernel runs)
};

struct Geometry {
    double boxL[3];
    double inv[3];       // 1 / L
    double V;
    double alpha, rcut, kcut;
    int bc;
};

}  // namespace cpm

// ----------------------------------------------------------------------------- context
struct cpm_ctx {
    cpm_params p{};
    cudaStream_t stream = nullptr;
    // two side streams and fork/join events: the reciprocal-space and k_perp = 0 chains of b run beside
    // the real-space chain (in an eager call and inside a captured graph alike)
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t fev[5] = {};
    int device = 0;
    std::string err;
    size_t bytes = 0;
    std::vector<void*> owned;
    cpm::Geometry g{};

    // electrode geometry (SoA)
    int64_t n = 0;
    int ng = 0;
    double* sx = nullptr;        // [4 * n]: x | y | z | eta
    double* sxyz = nullptr;      // [n * 3] row-major copy of the site coordinates
    int* group = nullptr;
    int* zmap = nullptr;         // [n] index of each site's height in zuniq
    double* zuniq = nullptr;     // distinct site heights (exact values)
    int nzu = 0;
    int* sperm = nullptr;        // sites ordered by real-space cell
    void* schunks = nullptr;     // int4 (first, count, cell, 0): chunks of at most 32 sites of one cell,
                                 // the most sites first
    int* rqueue = nullptr;       // real-space work queue: next item, blocks done (both zero between launches)
    int nschunk = 0;
    void* rtab = nullptr;        // single-precision pair-function tables, one per distinct eta
    int* rtab_id = nullptr;      // [n] table of each site
    int nrtab = 0;
    float* s32 = nullptr;        // [4 * n] wrapped single-precision x | y | z | eta
    float4* rsite = nullptr;     // [nschunk * 32] sites of each chunk (x, y, z, r_eta^2), slots past the
                                 // chunk's count repeat its first site
    int* rsite_tab = nullptr;    // [nschunk * 32] pair-table offset of each slot
    int* rsite_idx = nullptr;    // [nschunk * 32] site index of each slot
    float4* rbox = nullptr;      // [nschunk * 2] bounding box of each chunk's single-precision sites
    int4* rchunk = nullptr;      // [nschunk] per chunk: first site in sperm, site count, run count
    int2* rrun_cell = nullptr;   // [nschunk * rrun_stride] runs of each chunk: first cell and one past
                                 // the last (cell indices within one replica's cell list)
    float4* rrun_sh = nullptr;   // the image shift of each run
    int rrun_stride = 0;         // run slots per chunk
    cpm::RealPoly rpoly{};       // fitted pair function of the gathered real-space kernel
    int rpoly_blocks = 0;        // its persistent grid (resident blocks per SM x SMs)
    cpm::KTable kt;
    int2* h2d_idx = nullptr;     // EW2D: half-plane 2D vectors (nx, ny), 0 < |h| <= kcut
    double* h2d_norm = nullptr;  // their |h|
    int nh2d = 0;
    cpm::Phases<double> site64;
    cpm::Phases<float> site32;
    uint64_t geom_hash = 0;

    // dense matrices
    double* A = nullptr;
    double* W = nullptr;         // Cholesky factor, then its inverse, then A^-1
    double* S = nullptr;
    float* S32 = nullptr;
    double* SG = nullptr;        // [n * ng]
    double* u = nullptr;         // [n]
    double* dvec = nullptr;      // [n] scratch; with symm = 0 the row sums of the single-precision S
    double* red = nullptr;       // [64] scratch scalars
    unsigned* status = nullptr;  // device status word
    int* tickets = nullptr;      // [tickets_n] per-replica arrival counters, zero between launches
    int tickets_n = 0;
    double2* c0e = nullptr;      // [nzu][min(ext0, COL0_NZ)] exp(i kz z_u) of the k_perp = 0 column at the sites
    double* nbuf = nullptr;      // neutrality fix: per-block partial sums of q
    size_t nbuf_bytes = 0;
    bool assembled = false, inverted = false;
    bool has_A = false;          // A (and the factor workspace W) allocated and valid
    double etd = 0.0;            // e^T A^-1 e (FP64), kept with S
    int ir_sweeps = 0;           // refinement sweeps of the last FP32-factor inversion
    double ir_resid = 0.0;       // its final max-norm residual of A X = I
    // constant charge / thermo-potentiostat / finite field (ccm.cu), rebuilt after every inversion
    bool ccm_ready = false;
    double* ccm_buf = nullptr;   // inverse of G^T A^-1 G (N_g x N_g), then G^T u (N_g)
    double ccm_C0 = 0.0;         // g_1^T S g_1
    void* ccm_scr = nullptr;     // per-call electrode potentials and totals
    size_t ccm_scr_bytes = 0;
    double* SGx = nullptr;       // [n][N_g + 1]: SG and S zeta (finite field)
    const double* sg_over = nullptr;   // when set, the update reads these responses and columns
    int ng_over = 0;

    // per-step scratch, grown on demand
    int cap_m = 0;
    int64_t cap_ne = 0;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // host staging for cpm_step_host
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
    void* dstage = nullptr;
    size_t dstage_bytes = 0;
    void* ubuf = nullptr;        // cpm_update scratch (split partial sums, b hi/lo)
    size_t ubuf_bytes = 0;
    // cpm_step_graph: captured bvec + update sequences, one per (m, n_e, buffer addresses), at most
    // CPM_MAX_GRAPHS (24), least recently used replaced first; graph_valid = false (set when a scratch
    // buffer is reallocated) drops them all at the next step
    struct StepGraph {
        int m = 0;
        int64_t ne = 0;
        const void* ptrs[11] = {};   // device buffers, then the pinned host buffers of cpm_step_host (or null)
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
        uint64_t used = 0;
    };
    std::vector<StepGraph> graphs;
    uint64_t graph_clock = 0;
    bool graph_valid = false;
    void* Sb = nullptr;          // S as three bf16 planes [3][n][ld] for the tensor-core update
    double* SZ = nullptr;        // [n][tc_ngrp] S times the centring-group indicators
    int tc_ngrp = 0;
    bool tc_use_z = false;
    void* tbuf = nullptr;        // tensor-core update scratch (K-split partials, b planes)
    size_t tbuf_bytes = 0;
    size_t tc_pbytes = 0;        // bytes of tbuf holding the K-split partial sums
    bool tc_autotune = true;     // time the tile plans of the tensor-core product per (n, m)
    void* tcz = nullptr;         // tensor-core reciprocal space: site phase planes [2][npad][KZ] (fp16)
    float2* tcxy = nullptr;      // [ncols][n] column factors X_i Y_i of the sites
    float tc_wmax = 0.f;         // bound on the k-space weights
    int tc_mx[32] = {};          // largest harmonic extent of each 128-column structure-factor tile
    int tc_nmx = 0;              // tiles in tc_mx (0: the kernel finds them)
    void* p3m_G = nullptr;       // P3M (kspace = CPM_KSPACE_P3M): influence function / V on the mesh (k_prec's T)
    void* p3m_tw = nullptr;      // its FFT twiddles exp(-2 pi i j / K), j < K / 2, for K = Kx, Ky, Kz
    void* p3m_G64 = nullptr;     // the same in FP64 for the P3M elastance when k_prec is single precision
    void* p3m_tw64 = nullptr;

    int64_t launches = 0;        // kernels launched by cpm_bvec / cpm_update / cpm_step_host

    // tracing (cpm_profile)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending[CPM_K_COUNT];
    cudaEvent_t prof_open[CPM_K_COUNT] = {};
    double prof_ms[CPM_K_COUNT] = {};
    int64_t prof_cnt[CPM_K_COUNT] = {};
};

namespace cpm {

constexpr int CPM_MAX_GRAPHS = 24;

// error helpers (api.cu)
cpm_status set_err(cpm_ctx* c, cpm_status s, const char* fmt, ...);
cpm_status cuda_check(cpm_ctx* c, cudaError_t e, const char* what);
cpm_status dev_alloc(cpm_ctx* c, void** ptr, size_t bytes);
void dev_free(cpm_ctx* c, void* ptr);

#define CPM_CUDA(ctx, call)                                                     \
    do {                                                                        \
        cudaError_t e__ = (call);                                               \
        if (e__ != cudaSuccess) return ::cpm::cuda_check((ctx), e__, #call);    \
    } while (0)
#define CPM_LAUNCH(ctx, what)                                                   \
    do {                                                                        \
        cudaError_t e__ = cudaGetLastError();                                   \
        if (e__ != cudaSuccess) return ::cpm::cuda_check((ctx), e__, what);     \
    } while (0)
#define CPM_TRY(expr)                                                           \
    do {                                                                        \
        cpm_status s__ = (expr);                                                \
        if (s__ != CPM_OK) return s__;                                          \
    } while (0)

// api.cu: bracket one kernel launch with events when tracing is on
void prof_begin(cpm_ctx* c, int k);
void prof_end(cpm_ctx* c, int k);

// ktables.cu
cpm_status build_ktable(cpm_ctx* c);
void free_ktable(cpm_ctx* c);
template <typename T>
cpm_status launch_phases(cudaStream_t st, const Geometry& g, const KTable& k, const double* xyz, int64_t P,
                         c2<T>* X, c2<T>* Y, c2<T>* Z);
size_t phase_elems(const KTable& k, int64_t P);
constexpr int FR_THREADS = 256;   // threads per block of the fractions kernel (k_fracs)
// fractions u, charges Qv in T and (qabs non-null) the per-replica max |Q|, sum |Q| (qpart: m x blocks
// x 2 doubles, tickets: m counters), then the phase tables; after_fracs is recorded after the first kernel
template <typename T>
cpm_status launch_phases_u(cudaStream_t st, const Geometry& g, const KTable& k, const double* xyz, const double* Q,
                           int64_t ne, int m, uint64_t* u, T* Qv, double* qpart, int* tickets, float2* qabs,
                           c2<T>* X, c2<T>* Y, c2<T>* Z, cudaEvent_t after_fracs = nullptr, float zscale = 1.f);
// inputs of the double-float k_perp = 0 column from the z fractions (u as written by the phase kernels)
cpm_status launch_col0_inputs(cudaStream_t st, const uint64_t* u, const double* Q, int64_t P, float4* e1,
                              float2* q2);

// api.cu
cpm_status ensure_scratch(cpm_ctx* c, size_t bytes);
cpm_status ensure_tickets(cpm_ctx* c, int m);

// Last-block reduction: every block of a replica stores its partial, then takes a ticket; the
// block that draws the last ticket sums the partials in block order (a fixed order, so the result
// does not depend on scheduling) and resets the counter for the next launch.
__device__ __forceinline__ bool last_block_of(int* ticket, int nblocks) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1) == nblocks - 1;
        if (s_last) atomicExch(ticket, 0);
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// assemble.cu
cpm_status assemble_A(cpm_ctx* c);

// ew2d.cu: the exact 2D-periodic slab sum
cpm_status build_ew2d(cpm_ctx* c);
cpm_status assemble_ew2d(cpm_ctx* c);
size_t ew2d_T_bytes(const cpm_ctx* c, int m);
template <typename T>
cpm_status ew2d_run(cpm_ctx* c, cudaStream_t st, int m, int64_t ne, const double* xyz, const double* Q, void* Tbuf,
                    double* ew);

// dense.cu
cpm_status invert_and_project(cpm_ctx* c);
// the projection tail once S holds A^-1 (dense.cu)
cpm_status project_inverse(cpm_ctx* c);
// symm = 0: the FP64 row sums of the single-precision S into dvec (the centred products add b_i times them)
cpm_status fp32_rowsums(cpm_ctx* c);
// A^-1 by an FP32 Cholesky factor and FP64 iterative refinement of A X = I, then the projection (refine.cu)
cpm_status invert_ir(cpm_ctx* c);
cpm_status launch_dgemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
                        int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, int lower,
                        int tri, const unsigned* status);

// bvec.cu
struct Geometry;
CellGrid make_grid(const Geometry& g);
// bhl (optional): also write the two-float split of b that the single-precision update reads
cpm_status bvec(cpm_ctx* c, int m, int64_t ne, const double* xyz, const double* Q, double* b_out,
                float2* bhl = nullptr);
cpm_status reserve_bvec(cpm_ctx* c, int m, int64_t ne);
cpm_status ensure_aux(cpm_ctx* c);
cpm_status build_col0_sites(cpm_ctx* c);
cpm_status build_pair_tables(cpm_ctx* c, const std::vector<double>& etas);

// real_poly.cu: real-space b from per-chunk candidate lists and the fitted pair function
// fit of g for this splitting (deg = 0 when no supported degree reaches the accuracy)
RealPoly fit_real_poly(double alpha, double rcut, double rlo);
// after the site chunks and pair tables: the chunk site slots and the fit (rpoly.deg = 0 if the
// geometry cannot take the kernel)
cpm_status build_real_poly(cpm_ctx* c, const std::vector<double>& etas);
cpm_status real_poly_run(cpm_ctx* c, cudaStream_t st, int m, const CellGrid& cg, const int* start,
                         const float4* sorted, double* out);

// update.cu
// bhl_ready: the split of b is already in update_bhl(c, m) (written by bvec in the same step)
cpm_status update(cpm_ctx* c, int m, const double* psi, const double* b, double* q, double* qtot,
                  bool bhl_ready = false);
// where the single-precision update keeps the two-float split of b (nullptr for other S precisions)
float2* update_bhl(cpm_ctx* c, int m);

cpm_status reserve_update(cpm_ctx* c, int m);
// the electrode responses and their count the update uses (SG, or the override of the finite field)
inline const double* upd_sg(const cpm_ctx* c) { return c->sg_over ? c->sg_over : c->SG; }
inline int upd_ng(const cpm_ctx* c) { return c->sg_over ? c->ng_over : c->ng; }
// after S changes (cpm_invert, cpm_import): the constant-charge tables are stale
void ccm_invalidate(cpm_ctx* c);

// tc_gemm.cu
cpm_status tc_update(cpm_ctx* c, int m, const double* psi, const double* b, double* q);
cpm_status tc_reserve(cpm_ctx* c, int m);
cpm_status tc_selftest_timeout(cpm_ctx* c, double wait_ms);
// tile plan of the tensor-core product for m replicas: BN, stages, splits, CTAs, candidates timed
cpm_status tc_plan_query(cpm_ctx* c, int m, int32_t* plan, double* ms);
cpm_status tc_plan_set(cpm_ctx* c, int m, const int32_t* plan);

// gemv_tma.cu: single-precision S streaming with TMA (n a multiple of 4)
bool gemv_tma_supported(const cpm_ctx* c);
void gemv_tma_plan(int64_t n, int m, int64_t* colblocks, int64_t* splits, int64_t* jchunk);
cpm_status gemv_tma(cpm_ctx* c, int m, const float2* bhl, float2* part, int64_t splits, int64_t jchunk);

// tc_recip.cu: reciprocal-space sums of b on the tensor cores (k_prec = CPM_PREC_F16X2)
struct TcRecipDims {
    int mtiles, ntiles, cpad, splits;   // stage 1: column tiles, harmonic tiles, padded columns, charge splits
    int64_t chunk;                      // charges per split
    int mr, nrb, CT, ncb, NB, ngroups;  // stage 2: replicas per block, blocks, columns per group, ...
    int KZ;                             // padded K extent (2 x harmonics)
    int64_t npad;                       // padded site count
};
bool tc_recip_supported(const KTable& k);   // phase-table rows fit the staging buffer
TcRecipDims tc_recip_dims(const cpm_ctx* c, int m, int64_t ne);
size_t tc_recip_part_bytes(const TcRecipDims& d, int m, int nzw);
size_t tc_recip_w16_bytes(const TcRecipDims& d);
cpm_status tc_recip_prepare(cpm_ctx* c);
cpm_status tc_recip_run(cpm_ctx* c, int m, int64_t ne, const float2* EX, const float2* EY, const float2* EZ,
                        const float* Qv, const float2* qabs, void* part, void* w16, float* site_partial);

// p3m.cu: the reciprocal part of b by P3M (cpm_params.kspace = CPM_KSPACE_P3M)
constexpr int P3M_MAX_MESH = 512;                 // mesh points per axis (powers of two, at least 8)
constexpr size_t P3M_PLANE_BYTES = 128 * 1024;    // one complex xy plane must fit in shared memory
bool p3m_mesh_ok(const cpm_params* p);
cpm_status p3m_prepare(cpm_ctx* c);
template <typename T>
size_t p3m_scratch_bytes(const cpm_ctx* c, int m, int64_t ne);
// pm: m x n doubles, the mesh potential at every site (e / Angstrom, before K_E)
template <typename T>
cpm_status p3m_run(cpm_ctx* c, cudaStream_t st, int m, int64_t ne, const double* xyz, const double* Q, char* scr,
                   double* pm);
// p3m_matrix: A += K_E x the P3M reciprocal part (rows of unit charges at the sites, FP64), symmetrised
cpm_status p3m_assemble_recip(cpm_ctx* c);

}  // namespace cpm
