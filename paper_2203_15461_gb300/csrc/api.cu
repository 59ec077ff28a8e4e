// C ABI of the CPM library: argument checks, device-memory ownership, call ordering and the
// host-buffer entry point.  All arithmetic runs in the kernels of the other translation units.
#include <cstdarg>
#include <cstring>

#include "common.cuh"

namespace cpm {

cpm_status set_err(cpm_ctx* c, cpm_status s, const char* fmt, ...) {
    if (!c) return s;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    return s;
}

cpm_status cuda_check(cpm_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return CPM_OK;
    if (e == cudaErrorMemoryAllocation) return set_err(c, CPM_E_OOM, "%s: %s", what, cudaGetErrorString(e));
    return set_err(c, CPM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cpm_status dev_alloc(cpm_ctx* c, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->p.hbm_budget && c->bytes + bytes > c->p.hbm_budget)
        return set_err(c, CPM_E_BUDGET, "device budget of %zu bytes exceeded (%zu held, %zu requested)",
                       c->p.hbm_budget, c->bytes, bytes);
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return set_err(c, CPM_E_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->bytes += bytes;
    c->owned.push_back(*ptr);
    c->owned.push_back((void*)bytes);
    return CPM_OK;
}

void dev_free(cpm_ctx* c, void* ptr) {
    if (!ptr) return;
    for (size_t i = 0; i < c->owned.size(); i += 2) {
        if (c->owned[i] == ptr) {
            c->bytes -= (size_t)c->owned[i + 1];
            c->owned.erase(c->owned.begin() + i, c->owned.begin() + i + 2);
            break;
        }
    }
    cudaFree(ptr);
}

static cudaEvent_t take_event(cpm_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

void prof_begin(cpm_ctx* c, int k) {
    if (!c->prof_on) return;
    cudaEvent_t e = take_event(c);
    if (!e) return;
    cudaEventRecord(e, c->stream);
    c->prof_open[k] = e;
}

void prof_end(cpm_ctx* c, int k) {
    if (!c->prof_on || !c->prof_open[k]) return;
    cudaEvent_t e = take_event(c);
    if (!e) return;
    cudaEventRecord(e, c->stream);
    c->prof_pending[k].push_back({c->prof_open[k], e});
    c->prof_open[k] = nullptr;
}

cpm_status ensure_tickets(cpm_ctx* c, int m) {
    if (c->tickets_n >= m) return CPM_OK;
    c->graph_valid = false;
    dev_free(c, c->tickets);
    c->tickets = nullptr;
    c->tickets_n = 0;
    const int cap = ((m + 255) / 256) * 256;
    CPM_TRY(dev_alloc(c, (void**)&c->tickets, sizeof(int) * cap));
    CPM_CUDA(c, cudaMemsetAsync(c->tickets, 0, sizeof(int) * cap, c->stream));
    c->tickets_n = cap;
    return CPM_OK;
}

cpm_status ensure_scratch(cpm_ctx* c, size_t bytes) {
    if (c->scratch_bytes >= bytes) return CPM_OK;
    c->graph_valid = false;
    dev_free(c, c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    CPM_TRY(dev_alloc(c, &c->scratch, bytes));
    c->scratch_bytes = bytes;
    return CPM_OK;
}


__global__ void k_soa(const double* xyz, const double* eta, const int32_t* grp, int64_t n, int ng, Geometry g,
                      double* sx, float* s32, int* group, unsigned* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int d = 0; d < 3; ++d) {
        double x = xyz[3 * i + d];
        sx[d * n + i] = x;
        double w = x - g.boxL[d] * floor(x * g.inv[d]);
        s32[d * n + i] = (float)w;
        if (!isfinite(x)) atomicOr(status, ST_NONFINITE);
    }
    double e = eta[i];
    if (!(e > 0.0) || !isfinite(e)) atomicOr(status, ST_NONFINITE);
    sx[3 * n + i] = e;
    s32[3 * n + i] = (float)e;
    int gg = grp[i];
    if (gg < 0 || gg >= ng) atomicOr(status, ST_NONFINITE);
    group[i] = gg;
}

static void drop_graph(cpm_ctx* c) {
    for (auto& gr : c->graphs)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    c->graphs.clear();
    c->graph_valid = false;
}

static void free_geometry(cpm_ctx* c) {
    drop_graph(c);
    free_ktable(c);
    void* ptrs[] = {c->sx, c->group, c->s32, c->site64.X, c->site64.Y, c->site64.Z, c->site32.X, c->site32.Y,
                    c->site32.Z, c->A, c->W, c->S, c->S32, c->SG, c->u, c->dvec, c->sxyz, c->zmap, c->zuniq, c->Sb, c->SZ, c->rtab, c->rtab_id,
                    c->sperm, c->schunks, c->rqueue, c->tcz, c->tcxy, c->c0e, c->ccm_buf, c->ccm_scr, c->SGx,
                    c->h2d_idx, c->h2d_norm, c->rsite, c->rsite_tab, c->rrun_cell, c->rrun_sh,
                    c->rchunk, c->rsite_idx, c->rbox};
    for (void* p : ptrs) dev_free(c, p);
    c->sx = nullptr; c->group = nullptr; c->s32 = nullptr; c->sxyz = nullptr;
    c->zmap = nullptr; c->zuniq = nullptr; c->nzu = 0;
    c->Sb = nullptr; c->SZ = nullptr;
    c->rtab = nullptr; c->rtab_id = nullptr; c->nrtab = 0;
    c->sperm = nullptr; c->schunks = nullptr; c->rqueue = nullptr; c->nschunk = 0;
    c->tcz = nullptr; c->tcxy = nullptr; c->c0e = nullptr;
    c->ccm_buf = nullptr; c->ccm_scr = nullptr; c->SGx = nullptr; c->ccm_scr_bytes = 0; c->ccm_ready = false;
    c->h2d_idx = nullptr; c->h2d_norm = nullptr; c->nh2d = 0;
    c->rsite = nullptr; c->rsite_tab = nullptr; c->rpoly = cpm::RealPoly{}; c->rpoly_blocks = 0;
    c->rrun_cell = nullptr; c->rrun_sh = nullptr; c->rchunk = nullptr; c->rrun_stride = 0;
    c->rsite_idx = nullptr; c->rbox = nullptr;
    c->site64 = Phases<double>{}; c->site32 = Phases<float>{};
    c->A = c->W = c->S = c->SG = c->u = c->dvec = nullptr;
    c->S32 = nullptr;
    c->n = 0;
    c->assembled = c->inverted = false;
    c->has_A = false;
}

static uint64_t fnv1a(uint64_t h, const void* data, size_t bytes) {
    const unsigned char* p = (const unsigned char*)data;
    for (size_t i = 0; i < bytes; ++i) { h ^= p[i]; h *= 1099511628211ull; }
    return h;
}

// cpm_bvec followed by cpm_update as one CUDA graph on the context stream: captured and
// instantiated on the first call for given (m, n_e, buffer addresses), replayed afterwards.
// Pinned host buffers of cpm_step_host whose copies go into the captured graph (null: device only).
struct HostIO {
    const double *xyz, *Q, *psi;
    double *q, *qtot;
};

static cpm_status step_graph(cpm_ctx* c, int32_t m, int64_t n_e, const double* xyz, const double* Q,
                             const double* psi, double* b_out, double* q_out, double* qtot_out,
                             const HostIO* hio = nullptr) {
    const void* ptrs[11] = {xyz, Q, psi, b_out, q_out, qtot_out, hio ? hio->xyz : nullptr, hio ? hio->Q : nullptr,
                            hio ? hio->psi : nullptr, hio ? hio->q : nullptr, hio ? hio->qtot : nullptr};
    CPM_TRY(reserve_bvec(c, m, n_e));
    CPM_TRY(reserve_update(c, m));
    if (!c->graph_valid) drop_graph(c);   // a scratch buffer moved: every captured graph is stale
    cpm_ctx::StepGraph* hit = nullptr;
    for (auto& gr : c->graphs) {
        bool same = gr.m == m && gr.ne == n_e;
        for (int k = 0; k < 11 && same; ++k) same = gr.ptrs[k] == ptrs[k];
        if (same) { hit = &gr; break; }
    }
    if (!hit) {
        if ((int)c->graphs.size() >= CPM_MAX_GRAPHS) {
            auto lru = std::min_element(c->graphs.begin(), c->graphs.end(),
                                        [](const cpm_ctx::StepGraph& a, const cpm_ctx::StepGraph& b) { return a.used < b.used; });
            if (lru->exec) cudaGraphExecDestroy(lru->exec);
            c->graphs.erase(lru);
        }
        const bool prof = c->prof_on;
        c->prof_on = false;
        const int64_t l0 = c->launches;
        CPM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        float2* bhl = update_bhl(c, m);
        cpm_status s1 = CPM_OK;
        if (hio) {   // the host-to-device copies as graph nodes (pinned buffers)
            const size_t pt = (size_t)m * n_e;
            cudaError_t ce = cudaSuccess;
            if (pt) ce = cudaMemcpyAsync((void*)xyz, hio->xyz, sizeof(double) * 3 * pt, cudaMemcpyHostToDevice, c->stream);
            if (pt && ce == cudaSuccess)
                ce = cudaMemcpyAsync((void*)Q, hio->Q, sizeof(double) * pt, cudaMemcpyHostToDevice, c->stream);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync((void*)psi, hio->psi, sizeof(double) * m * c->ng, cudaMemcpyHostToDevice,
                                     c->stream);
            if (ce != cudaSuccess) s1 = cuda_check(c, ce, "cudaMemcpyAsync (captured)");
        }
        if (s1 == CPM_OK) s1 = bvec(c, m, n_e, xyz, Q, b_out, bhl);
        cpm_status s2 = s1 == CPM_OK ? update(c, m, psi, b_out, q_out, qtot_out, bhl != nullptr) : s1;
        if (s2 == CPM_OK && hio) {   // and the results back
            cudaError_t ce = cudaMemcpyAsync(hio->q, q_out, sizeof(double) * m * c->n, cudaMemcpyDeviceToHost, c->stream);
            if (ce == cudaSuccess && hio->qtot)
                ce = cudaMemcpyAsync(hio->qtot, qtot_out, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream);
            if (ce != cudaSuccess) s2 = cuda_check(c, ce, "cudaMemcpyAsync (captured)");
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->prof_on = prof;
        if (s2 != CPM_OK) { if (g) cudaGraphDestroy(g); return s2; }
        if (e != cudaSuccess) return cuda_check(c, e, "cudaStreamEndCapture");
        cpm_ctx::StepGraph gr;
        gr.m = m;
        gr.ne = n_e;
        for (int k = 0; k < 11; ++k) gr.ptrs[k] = ptrs[k];
        e = cudaGraphInstantiate(&gr.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_check(c, e, "cudaGraphInstantiate");
        gr.launches = c->launches - l0;
        c->launches = l0;
        c->graphs.push_back(gr);
        hit = &c->graphs.back();
        c->graph_valid = true;
    }
    hit->used = ++c->graph_clock;
    CPM_CUDA(c, cudaGraphLaunch(hit->exec, c->stream));
    c->launches += hit->launches;
    return CPM_OK;
}

}  // namespace cpm

using namespace cpm;

extern "C" {

cpm_status cpm_create(const cpm_params* p, void* cuda_stream, cpm_ctx** out) {
    if (!p || !out) return CPM_E_ARG;
    *out = nullptr;
    for (int d = 0; d < 3; ++d)
        if (!(p->box[d] > 0.0)) return CPM_E_ARG;
    if (!(p->alpha > 0.0) || !(p->rcut > 0.0) || !(p->kcut > 0.0)) return CPM_E_ARG;
    if (p->boundary < CPM_BC_3D || p->boundary > CPM_BC_EW2D) return CPM_E_ARG;
    if (p->boundary == CPM_BC_EW2D && p->k_prec == CPM_PREC_F16X2) return CPM_E_ARG;
    if (p->chol != CPM_CHOL_FP64 && p->chol != CPM_CHOL_FP32_IR) return CPM_E_ARG;
    if (p->kspace != CPM_KSPACE_EWALD && p->kspace != CPM_KSPACE_P3M) return CPM_E_ARG;
    if (p->kspace == CPM_KSPACE_P3M && (p->boundary == CPM_BC_EW2D || !p3m_mesh_ok(p))) return CPM_E_ARG;
    if (p->p3m_matrix != 0 && (p->p3m_matrix != 1 || p->kspace != CPM_KSPACE_P3M)) return CPM_E_ARG;
    if ((p->s_prec != CPM_PREC_FP64 && p->s_prec != CPM_PREC_FP32 && p->s_prec != CPM_PREC_BF16X3) ||
        (p->k_prec != CPM_PREC_FP64 && p->k_prec != CPM_PREC_FP32 && p->k_prec != CPM_PREC_F16X2))
        return CPM_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return CPM_E_CUDA;
    }
    cpm_ctx* c = new cpm_ctx();
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    Geometry& g = c->g;
    for (int d = 0; d < 3; ++d) { g.boxL[d] = p->box[d]; g.inv[d] = 1.0 / p->box[d]; }
    g.V = p->box[0] * p->box[1] * p->box[2];
    g.alpha = p->alpha; g.rcut = p->rcut; g.kcut = p->kcut; g.bc = p->boundary;
    cpm_status s = dev_alloc(c, (void**)&c->status, 256);
    if (s == CPM_OK) s = dev_alloc(c, (void**)&c->red, sizeof(double) * (64 + 64 * 64));
    if (s != CPM_OK) { cpm_destroy(c); return s; }
    cudaMemsetAsync(c->status, 0, 256, c->stream);
    *out = c;
    return CPM_OK;
}

void cpm_destroy(cpm_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    drop_graph(c);
    for (size_t i = 0; i < c->owned.size(); i += 2) cudaFree(c->owned[i]);
    for (int k = 0; k < CPM_K_COUNT; ++k)
        for (auto& pr : c->prof_pending[k]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaStream_t s : c->aux)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : c->fev)
        if (e) cudaEventDestroy(e);
    delete c;
}

const char* cpm_last_error(const cpm_ctx* c) { return c ? c->err.c_str() : "null context"; }

size_t cpm_device_bytes(const cpm_ctx* c) { return c ? c->bytes : 0; }

int64_t cpm_launch_count(const cpm_ctx* c) { return c ? c->launches : 0; }

// The geometry part of cpm_assemble (sites, k table, phase tables, real-space chunks, dense buffers
// for S); with_A also allocates A and the factor workspace and assembles A.
static cpm_status assemble_impl(cpm_ctx* c, int64_t n, const double* xyz, const double* eta, const int32_t* group,
                                int32_t n_groups, bool with_A) {
    if (!c) return CPM_E_ARG;
    c->err.clear();
    if (n < 1 || n_groups < 1 || n_groups > 16 || !xyz || !eta || !group)
        return set_err(c, CPM_E_ARG, "cpm_assemble: need n >= 1, 1 <= n_groups <= 16 and non-null inputs");
    if (n > (int64_t)46000) return set_err(c, CPM_E_ARG, "cpm_assemble: n = %lld exceeds 46000", (long long)n);
    free_geometry(c);
    c->n = n;
    c->ng = n_groups;
    cudaStream_t st = c->stream;
    CPM_TRY(dev_alloc(c, (void**)&c->sx, sizeof(double) * 4 * n));
    CPM_TRY(dev_alloc(c, (void**)&c->sxyz, sizeof(double) * 3 * n));
    CPM_TRY(dev_alloc(c, (void**)&c->s32, sizeof(float) * 4 * n));
    CPM_TRY(dev_alloc(c, (void**)&c->group, sizeof(int) * n));
    CPM_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), st));
    CPM_CUDA(c, cudaMemcpyAsync(c->sxyz, xyz, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    k_soa<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xyz, eta, group, n, n_groups, c->g, c->sx, c->s32, c->group,
                                                       c->status);
    CPM_LAUNCH(c, "k_soa");
    // geometry hash for cpm_save / cpm_load
    {
        std::vector<double> hx(4 * n);
        std::vector<int> hg(n);
        unsigned hst = 0;
        CPM_CUDA(c, cudaMemcpyAsync(hx.data(), c->sx, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, st));
        CPM_CUDA(c, cudaMemcpyAsync(hg.data(), c->group, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
        CPM_CUDA(c, cudaMemcpyAsync(&hst, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CPM_CUDA(c, cudaStreamSynchronize(st));
        if (hst) {
            free_geometry(c);
            return set_err(c, CPM_E_NONFINITE, "cpm_assemble: non-finite coordinate, eta <= 0 or group out of range");
        }
        // distinct site heights: the k_perp = 0 column of b depends on z only
        std::vector<double> zs(hx.begin() + 2 * n, hx.begin() + 3 * n);
        std::vector<double> zu = zs;
        std::sort(zu.begin(), zu.end());
        zu.erase(std::unique(zu.begin(), zu.end()), zu.end());
        std::vector<int> zm(n);
        for (int64_t i = 0; i < n; ++i) zm[i] = (int)(std::lower_bound(zu.begin(), zu.end(), zs[i]) - zu.begin());
        c->nzu = (int)zu.size();
        // distinct Gaussian widths: one real-space pair-function table each (at most 16)
        std::vector<double> es(hx.begin() + 3 * n, hx.begin() + 4 * n);
        std::vector<double> eu = es;
        std::sort(eu.begin(), eu.end());
        eu.erase(std::unique(eu.begin(), eu.end()), eu.end());
        // sites grouped by real-space cell, in chunks of at most 32 (one warp each)
        {
            const CellGrid cg = make_grid(c->g);
            std::vector<int> cell(n);
            for (int64_t i = 0; i < n; ++i) {
                int cc[3];
                for (int d = 0; d < 3; ++d) {
                    const double x = hx[d * n + i];
                    double w = x - c->g.boxL[d] * std::floor(x * c->g.inv[d]);
                    if (w >= c->g.boxL[d]) w -= c->g.boxL[d];
                    if (w < 0) w = 0;
                    cc[d] = std::min(cg.nc[d] - 1, (int)((float)w / (float)cg.h[d]));
                }
                cell[i] = (cc[2] * cg.nc[1] + cc[1]) * cg.nc[0] + cc[0];
            }
            std::vector<int> perm(n);
            for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
            std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return cell[a] < cell[b]; });
            std::vector<int4> chunks;
            for (int64_t k = 0; k < n;) {
                int64_t e = k;
                while (e < n && cell[perm[e]] == cell[perm[k]]) ++e;
                for (int64_t f = k; f < e; f += 32)
                    chunks.push_back(make_int4((int)f, (int)std::min<int64_t>(32, e - f), cell[perm[k]], 0));
                k = e;
            }
            // most sites first (padded to the kernel's groups of eight): the real-space kernel takes
            // chunks from a queue in this order, so the long items start early and the short ones fill in
            std::stable_sort(chunks.begin(), chunks.end(),
                             [](const int4& a, const int4& b) { return (a.y + 7) / 8 > (b.y + 7) / 8; });
            c->nschunk = (int)chunks.size();
            CPM_TRY(dev_alloc(c, (void**)&c->sperm, sizeof(int) * n));
            CPM_TRY(dev_alloc(c, &c->schunks, sizeof(int4) * chunks.size()));
            CPM_TRY(dev_alloc(c, (void**)&c->rqueue, 2 * sizeof(int)));
            CPM_CUDA(c, cudaMemsetAsync(c->rqueue, 0, 2 * sizeof(int), st));
            CPM_CUDA(c, cudaMemcpyAsync(c->sperm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
            CPM_CUDA(c, cudaMemcpyAsync(c->schunks, chunks.data(), sizeof(int4) * chunks.size(),
                                        cudaMemcpyHostToDevice, st));
            CPM_CUDA(c, cudaStreamSynchronize(st));
        }
        if (eu.size() <= 16) {
            std::vector<int> em(n);
            for (int64_t i = 0; i < n; ++i) em[i] = (int)(std::lower_bound(eu.begin(), eu.end(), es[i]) - eu.begin());
            CPM_TRY(dev_alloc(c, (void**)&c->rtab_id, sizeof(int) * n));
            CPM_CUDA(c, cudaMemcpyAsync(c->rtab_id, em.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
            CPM_TRY(build_pair_tables(c, eu));
            c->nrtab = (int)eu.size();
            CPM_TRY(build_real_poly(c, eu));
        }
        CPM_TRY(dev_alloc(c, (void**)&c->zmap, sizeof(int) * n));
        CPM_TRY(dev_alloc(c, (void**)&c->zuniq, sizeof(double) * zu.size()));
        CPM_CUDA(c, cudaMemcpyAsync(c->zmap, zm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        CPM_CUDA(c, cudaMemcpyAsync(c->zuniq, zu.data(), sizeof(double) * zu.size(), cudaMemcpyHostToDevice, st));
        CPM_CUDA(c, cudaStreamSynchronize(st));
        uint64_t h = 1469598103934665603ull;
        h = fnv1a(h, hx.data(), hx.size() * sizeof(double));
        h = fnv1a(h, hg.data(), hg.size() * sizeof(int));
        h = fnv1a(h, &c->p, sizeof(double) * 3);
        c->geom_hash = h;
    }
    CPM_TRY(build_ktable(c));
    if (c->g.bc == CPM_BC_EW2D) {
        // z is not periodic: every real-space pair must stay within one period of the cell height
        double zmin = 1e300, zmax = -1e300;
        {
            std::vector<double> zz(n);
            CPM_CUDA(c, cudaMemcpyAsync(zz.data(), c->sx + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
            CPM_CUDA(c, cudaStreamSynchronize(st));
            for (double z : zz) { zmin = std::min(zmin, z); zmax = std::max(zmax, z); }
        }
        if (!(zmax - zmin + c->g.rcut < c->g.boxL[2])) {
            free_geometry(c);
            return set_err(c, CPM_E_ARG, "EW2D: box[2] must exceed the sites' z range (%g) by rcut", zmax - zmin);
        }
        CPM_TRY(build_ew2d(c));
    }
    const KTable& k = c->kt;
    const size_t pe = phase_elems(k, n);
    const int64_t tX = (int64_t)(k.NX + 1) * n, tY = (int64_t)(2 * k.NY + 1) * n, tZ = (int64_t)pe - tX - tY;
    CPM_TRY(dev_alloc(c, (void**)&c->site64.X, sizeof(double2) * tX));
    CPM_TRY(dev_alloc(c, (void**)&c->site64.Y, sizeof(double2) * tY));
    CPM_TRY(dev_alloc(c, (void**)&c->site64.Z, sizeof(double2) * tZ));
    CPM_TRY(dev_alloc(c, (void**)&c->site32.X, sizeof(float2) * tX));
    CPM_TRY(dev_alloc(c, (void**)&c->site32.Y, sizeof(float2) * tY));
    CPM_TRY(dev_alloc(c, (void**)&c->site32.Z, sizeof(float2) * tZ));
    c->site64.P = c->site32.P = n;
    CPM_TRY(launch_phases<double>(st, c->g, k, c->sxyz, n, c->site64.X, c->site64.Y, c->site64.Z));
    CPM_TRY(launch_phases<float>(st, c->g, k, c->sxyz, n, c->site32.X, c->site32.Y, c->site32.Z));
    CPM_LAUNCH(c, "k_phases(sites)");
    if (c->p.k_prec == CPM_PREC_F16X2) CPM_TRY(tc_recip_prepare(c));
    CPM_TRY(build_col0_sites(c));
    if (c->p.kspace == CPM_KSPACE_P3M) CPM_TRY(p3m_prepare(c));
    const size_t nn = (size_t)n * n;
    if (with_A) {
        CPM_TRY(dev_alloc(c, (void**)&c->A, sizeof(double) * nn));
        CPM_TRY(dev_alloc(c, (void**)&c->W, sizeof(double) * nn));
    }
    CPM_TRY(dev_alloc(c, (void**)&c->S, sizeof(double) * nn));
    CPM_TRY(dev_alloc(c, (void**)&c->S32, sizeof(float) * nn));
    CPM_TRY(dev_alloc(c, (void**)&c->SG, sizeof(double) * n * n_groups));
    CPM_TRY(dev_alloc(c, (void**)&c->u, sizeof(double) * n));
    CPM_TRY(dev_alloc(c, (void**)&c->dvec, sizeof(double) * n));
    if (with_A) CPM_TRY(assemble_A(c));
    CPM_CUDA(c, cudaStreamSynchronize(st));
    c->has_A = with_A;
    c->assembled = true;
    return CPM_OK;
}

cpm_status cpm_assemble(cpm_ctx* c, int64_t n, const double* xyz, const double* eta, const int32_t* group,
                        int32_t n_groups) {
    return assemble_impl(c, n, xyz, eta, group, n_groups, true);
}

cpm_status cpm_prepare(cpm_ctx* c, int64_t n, const double* xyz, const double* eta, const int32_t* group,
                       int32_t n_groups) {
    return assemble_impl(c, n, xyz, eta, group, n_groups, false);
}

cpm_status cpm_release_assembly(cpm_ctx* c) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_release_assembly before cpm_invert");
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, c->A);
    dev_free(c, c->W);
    c->A = c->W = nullptr;
    c->has_A = false;
    return CPM_OK;
}

cpm_status cpm_invert(cpm_ctx* c) {
    if (!c) return CPM_E_ARG;
    c->err.clear();
    if (!c->assembled) return set_err(c, CPM_E_STATE, "cpm_invert before cpm_assemble");
    if (!c->has_A) return set_err(c, CPM_E_STATE, "cpm_invert: A is not held (cpm_prepare or cpm_release_assembly)");
    c->inverted = false;
    dev_free(c, c->Sb);
    c->Sb = nullptr;
    drop_graph(c);
    CPM_TRY(c->p.chol == CPM_CHOL_FP32_IR ? invert_ir(c) : invert_and_project(c));
    c->inverted = true;
    return CPM_OK;
}

cpm_status cpm_bvec(cpm_ctx* c, int32_t m, int64_t n_e, const double* xyz, const double* Q, double* b_out) {
    if (!c) return CPM_E_ARG;
    if (!c->assembled) return set_err(c, CPM_E_STATE, "cpm_bvec before cpm_assemble");
    if (m < 1 || n_e < 0 || !b_out || (n_e > 0 && (!xyz || !Q)))
        return set_err(c, CPM_E_ARG, "cpm_bvec: need m >= 1, n_e >= 0 and non-null buffers");
    if ((int64_t)m * n_e > (int64_t)1 << 30) return set_err(c, CPM_E_ARG, "cpm_bvec: m * n_e too large");
    return bvec(c, m, n_e, xyz, Q, b_out);
}

cpm_status cpm_update(cpm_ctx* c, int32_t m, const double* psi, const double* b, double* q_out, double* qtot_out) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_update before cpm_invert");
    if (m < 1 || !psi || !b || !q_out) return set_err(c, CPM_E_ARG, "cpm_update: need m >= 1 and non-null buffers");
    return update(c, m, psi, b, q_out, qtot_out);
}

// page-locked host memory (cudaHostAlloc / cudaHostRegister): copies from it can be graph nodes
static bool pinned_host(const void* p) {
    if (!p) return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

cpm_status cpm_step_host(cpm_ctx* c, int32_t m, int64_t n_e, const double* xyz, const double* Q, const double* psi,
                         double* q_out, double* qtot_out) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_step_host before cpm_invert");
    if (m < 1 || n_e < 0 || !psi || !q_out || (n_e > 0 && (!xyz || !Q)))
        return set_err(c, CPM_E_ARG, "cpm_step_host: need m >= 1, n_e >= 0 and non-null buffers");
    const size_t pt = (size_t)m * n_e;
    const size_t need = sizeof(double) * (4 * pt + (size_t)m * c->ng + 2 * (size_t)m * c->n + m) + 8 * 256;
    if (c->dstage_bytes < need) {
        dev_free(c, c->dstage);
        c->dstage = nullptr;
        c->dstage_bytes = 0;
        CPM_TRY(dev_alloc(c, &c->dstage, need));
        c->dstage_bytes = need;
    }
    char* base = (char*)c->dstage;
    auto take = [&](size_t bytes) { char* p = base; base += (bytes + 255) & ~(size_t)255; return (double*)p; };
    double* dxyz = take(sizeof(double) * 3 * pt);
    double* dQ = take(sizeof(double) * pt);
    double* dpsi = take(sizeof(double) * m * c->ng);
    double* db = take(sizeof(double) * m * c->n);
    double* dq = take(sizeof(double) * m * c->n);
    double* dqt = take(sizeof(double) * m);
    cudaStream_t st = c->stream;
    if (c->stream && !c->prof_on && pinned_host(xyz) && pinned_host(Q) && pinned_host(psi) && pinned_host(q_out) &&
        (!qtot_out || pinned_host(qtot_out))) {
        // pinned buffers: the copies are nodes of the captured step, one graph launch per call
        const HostIO hio{xyz, Q, psi, q_out, qtot_out};
        CPM_TRY(step_graph(c, m, n_e, dxyz, dQ, dpsi, db, dq, dqt, &hio));
        CPM_CUDA(c, cudaStreamSynchronize(st));
        return CPM_OK;
    }
    if (pt) {
        CPM_CUDA(c, cudaMemcpyAsync(dxyz, xyz, sizeof(double) * 3 * pt, cudaMemcpyHostToDevice, st));
        CPM_CUDA(c, cudaMemcpyAsync(dQ, Q, sizeof(double) * pt, cudaMemcpyHostToDevice, st));
    }
    CPM_CUDA(c, cudaMemcpyAsync(dpsi, psi, sizeof(double) * m * c->ng, cudaMemcpyHostToDevice, st));
    if (c->stream && !c->prof_on) {
        // the captured step, replayed on the staging buffers (addresses stable while dstage is)
        CPM_TRY(step_graph(c, m, n_e, dxyz, dQ, dpsi, db, dq, dqt));
    } else {
        float2* bhl = update_bhl(c, m);   // b's two-float split written by bvec: no separate split pass
        CPM_TRY(bvec(c, m, n_e, dxyz, dQ, db, bhl));
        CPM_TRY(update(c, m, dpsi, db, dq, dqt, bhl != nullptr));
    }
    CPM_CUDA(c, cudaMemcpyAsync(q_out, dq, sizeof(double) * m * c->n, cudaMemcpyDeviceToHost, st));
    if (qtot_out) CPM_CUDA(c, cudaMemcpyAsync(qtot_out, dqt, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    CPM_CUDA(c, cudaStreamSynchronize(st));
    return CPM_OK;
}

cpm_status cpm_step_graph(cpm_ctx* c, int32_t m, int64_t n_e, const double* xyz, const double* Q, const double* psi,
                          double* b_out, double* q_out, double* qtot_out) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_step_graph before cpm_invert");
    if (m < 1 || n_e < 0 || !psi || !b_out || !q_out || (n_e > 0 && (!xyz || !Q)))
        return set_err(c, CPM_E_ARG, "cpm_step_graph: need m >= 1, n_e >= 0 and non-null buffers");
    if (!c->stream) return set_err(c, CPM_E_ARG, "cpm_step_graph: needs a context created on a non-default stream");
    return step_graph(c, m, n_e, xyz, Q, psi, b_out, q_out, qtot_out);
}

cpm_status cpm_selftest_timeout(cpm_ctx* c, double wait_ms) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_selftest_timeout before cpm_invert");
    if (!(wait_ms > 0.0) || wait_ms > 10000.0) return set_err(c, CPM_E_ARG, "wait_ms must be in (0, 10000]");
    CPM_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    CPM_TRY(tc_selftest_timeout(c, wait_ms));
    cpm_status s = cpm_sync(c);
    CPM_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return s;
}

cpm_status cpm_gemm_plan(cpm_ctx* c, int32_t m, int32_t* plan_out, double* ms_out) {
    if (!c || m < 1) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_gemm_plan before cpm_invert");
    if (c->p.s_prec != CPM_PREC_BF16X3) return set_err(c, CPM_E_ARG, "cpm_gemm_plan: s_prec is not CPM_PREC_BF16X3");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CPM_CUDA(c, cudaStreamIsCapturing(c->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) return set_err(c, CPM_E_STATE, "cpm_gemm_plan during stream capture");
    CPM_TRY(tc_plan_query(c, m, plan_out, ms_out));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return CPM_OK;
}

cpm_status cpm_set_s_prec(cpm_ctx* c, int32_t s_prec) {
    if (!c) return CPM_E_ARG;
    if (s_prec != CPM_PREC_FP64 && s_prec != CPM_PREC_FP32 && s_prec != CPM_PREC_BF16X3)
        return set_err(c, CPM_E_ARG, "cpm_set_s_prec: %d is not an S precision", s_prec);
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_set_s_prec before cpm_invert");
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->p.s_prec != s_prec) {
        c->p.s_prec = s_prec;
        drop_graph(c);
    }
    return CPM_OK;
}

cpm_status cpm_inversion_info(cpm_ctx* c, int32_t* sweeps, double* resid) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_inversion_info before cpm_invert");
    if (sweeps) *sweeps = c->p.chol == CPM_CHOL_FP32_IR ? c->ir_sweeps : 0;
    if (resid) *resid = c->p.chol == CPM_CHOL_FP32_IR ? c->ir_resid : 0.0;
    return CPM_OK;
}

cpm_status cpm_gemm_set_plan(cpm_ctx* c, int32_t m, const int32_t* plan) {
    if (!c || m < 1 || !plan) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_gemm_set_plan before cpm_invert");
    if (c->p.s_prec != CPM_PREC_BF16X3) return set_err(c, CPM_E_ARG, "cpm_gemm_set_plan: s_prec is not CPM_PREC_BF16X3");
    CPM_TRY(tc_plan_set(c, m, plan));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return CPM_OK;
}

cpm_status cpm_sync(cpm_ctx* c) {
    if (!c) return CPM_E_ARG;
    unsigned hst = 0;
    CPM_CUDA(c, cudaMemcpyAsync(&hst, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hst & ST_NOT_SPD) return set_err(c, CPM_E_NOT_SPD, "elastance matrix is not positive definite");
    if (hst & ST_NONFINITE) return set_err(c, CPM_E_NONFINITE, "non-finite input");
    if (hst & ST_TIMEOUT) return set_err(c, CPM_E_TIMEOUT, "bounded device wait expired");
    return CPM_OK;
}

cpm_status cpm_get_matrix(cpm_ctx* c, int32_t which, double* out) {
    if (!c || !out) return CPM_E_ARG;
    const double* src = nullptr;
    size_t cnt = 0;
    const size_t n = (size_t)c->n;
    switch (which) {
        case CPM_MAT_A: if (!c->assembled || !c->has_A) return CPM_E_STATE; src = c->A; cnt = n * n; break;
        case CPM_MAT_S: if (!c->inverted) return CPM_E_STATE; src = c->S; cnt = n * n; break;
        case CPM_MAT_SG: if (!c->inverted) return CPM_E_STATE; src = c->SG; cnt = n * c->ng; break;
        case CPM_MAT_U: if (!c->inverted) return CPM_E_STATE; src = c->u; cnt = n; break;
        default: return CPM_E_ARG;
    }
    CPM_CUDA(c, cudaMemcpyAsync(out, src, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return CPM_OK;
}

cpm_status cpm_capacitance(cpm_ctx* c, double* C) {
    if (!c || !C) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_capacitance before cpm_invert");
    const int64_t n = c->n;
    const int ng = c->ng;
    std::vector<double> sg((size_t)n * ng);
    std::vector<int> gr(n);
    CPM_CUDA(c, cudaMemcpyAsync(sg.data(), c->SG, sizeof(double) * sg.size(), cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(gr.data(), c->group, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int a = 0; a < ng * ng; ++a) C[a] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int h = 0; h < ng; ++h) C[gr[i] * ng + h] += sg[(size_t)i * ng + h];
    return CPM_OK;
}

cpm_status cpm_kvectors(cpm_ctx* c, int32_t* nidx, int64_t cap, int64_t* nk) {
    if (!c || !nk) return CPM_E_ARG;
    if (!c->assembled) return set_err(c, CPM_E_STATE, "cpm_kvectors before cpm_assemble");
    *nk = c->kt.nk;
    const int64_t cnt = std::min<int64_t>(cap, c->kt.nk);
    if (cnt <= 0 || !nidx) return CPM_OK;
    std::vector<int4> kl(cnt);
    CPM_CUDA(c, cudaMemcpyAsync(kl.data(), c->kt.klist, sizeof(int4) * cnt, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int64_t i = 0; i < cnt; ++i) {
        nidx[3 * i] = kl[i].z;
        nidx[3 * i + 1] = kl[i].w;
        nidx[3 * i + 2] = kl[i].y;
    }
    return CPM_OK;
}

struct FileHeader {
    char magic[8];
    int32_t version, ng;
    int64_t n;
    uint64_t hash;
    double alpha, rcut, kcut;
    int32_t boundary, symm;
    double etd;          // e^T A^-1 e
};

static size_t export_bytes(const cpm_ctx* c) {
    const size_t n = (size_t)c->n;
    return sizeof(FileHeader) + sizeof(double) * (n * n + n * c->ng + n);
}

cpm_status cpm_export(cpm_ctx* c, void* buf, size_t cap, size_t* bytes) {
    if (!c) return CPM_E_ARG;
    if (!c->inverted) return set_err(c, CPM_E_STATE, "cpm_export before cpm_invert");
    const size_t need = export_bytes(c);
    if (bytes) *bytes = need;
    if (!buf) return CPM_OK;
    if (cap < need) return set_err(c, CPM_E_ARG, "cpm_export: %zu bytes needed, %zu given", need, cap);
    const size_t n = (size_t)c->n;
    FileHeader h{};
    memcpy(h.magic, "CPMSMAT", 8);
    h.version = 2; h.ng = c->ng; h.n = c->n; h.hash = c->geom_hash;
    h.alpha = c->p.alpha; h.rcut = c->p.rcut; h.kcut = c->p.kcut; h.boundary = c->p.boundary; h.symm = c->p.symm;
    h.etd = c->etd;
    memcpy(buf, &h, sizeof h);
    double* d = (double*)((char*)buf + sizeof h);
    CPM_CUDA(c, cudaMemcpyAsync(d, c->S, sizeof(double) * n * n, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(d + n * n, c->SG, sizeof(double) * n * c->ng, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(d + n * n + n * c->ng, c->u, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return CPM_OK;
}

__global__ void k_tofloat(const double* a, float* b, int64_t cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) b[i] = (float)a[i];
}

cpm_status cpm_import(cpm_ctx* c, const void* buf, size_t bytes) {
    if (!c || !buf) return CPM_E_ARG;
    if (!c->assembled) return set_err(c, CPM_E_STATE, "cpm_import before cpm_assemble or cpm_prepare");
    const size_t n = (size_t)c->n;
    FileHeader h{};
    if (bytes < sizeof h) return set_err(c, CPM_E_ARG, "cpm_import: %zu bytes is shorter than the header", bytes);
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, "CPMSMAT", 8) != 0 || h.version != 2 || h.n != c->n || h.ng != c->ng ||
        h.hash != c->geom_hash || h.alpha != c->p.alpha || h.rcut != c->p.rcut || h.kcut != c->p.kcut ||
        h.boundary != c->p.boundary || h.symm != c->p.symm)
        return set_err(c, CPM_E_ARG, "cpm_import: the checkpoint does not match this geometry and parameters");
    if (bytes < export_bytes(c)) return set_err(c, CPM_E_ARG, "cpm_import: short checkpoint (%zu bytes)", bytes);
    const double* d = (const double*)((const char*)buf + sizeof h);
    CPM_CUDA(c, cudaMemcpyAsync(c->S, d, sizeof(double) * n * n, cudaMemcpyHostToDevice, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(c->SG, d + n * n, sizeof(double) * n * c->ng, cudaMemcpyHostToDevice, c->stream));
    CPM_CUDA(c, cudaMemcpyAsync(c->u, d + n * n + n * c->ng, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    dev_free(c, c->Sb);
    c->Sb = nullptr;
    drop_graph(c);
    k_tofloat<<<(unsigned)((n * n + 255) / 256), 256, 0, c->stream>>>(c->S, c->S32, (int64_t)(n * n));
    CPM_LAUNCH(c, "k_tofloat");
    CPM_TRY(fp32_rowsums(c));
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->etd = h.etd;
    ccm_invalidate(c);
    c->inverted = true;
    return CPM_OK;
}

cpm_status cpm_save(cpm_ctx* c, const char* path) {
    if (!c || !path) return CPM_E_ARG;
    size_t need = 0;
    CPM_TRY(cpm_export(c, nullptr, 0, &need));
    std::vector<char> buf(need);
    CPM_TRY(cpm_export(c, buf.data(), need, &need));
    FILE* f = fopen(path, "wb");
    if (!f) return set_err(c, CPM_E_ARG, "cpm_save: cannot open %s", path);
    bool ok = fwrite(buf.data(), 1, need, f) == need;
    ok = (fclose(f) == 0) && ok;
    return ok ? CPM_OK : set_err(c, CPM_E_ARG, "cpm_save: write failed for %s", path);
}

cpm_status cpm_load(cpm_ctx* c, const char* path) {
    if (!c || !path) return CPM_E_ARG;
    if (!c->assembled) return set_err(c, CPM_E_STATE, "cpm_load before cpm_assemble");
    FILE* f = fopen(path, "rb");
    if (!f) return set_err(c, CPM_E_ARG, "cpm_load: cannot open %s", path);
    std::vector<char> buf(export_bytes(c));
    const size_t got = fread(buf.data(), 1, buf.size(), f);
    fclose(f);
    if (got < sizeof(FileHeader)) return set_err(c, CPM_E_ARG, "cpm_load: %s does not match this geometry and parameters", path);
    cpm_status st = cpm_import(c, buf.data(), got);
    if (st == CPM_E_ARG) return set_err(c, CPM_E_ARG, "cpm_load: %s does not match this geometry and parameters", path);
    return st;
}

cpm_status cpm_profile(cpm_ctx* c, int32_t enable) {
    if (!c) return CPM_E_ARG;
    c->prof_on = enable != 0;
    return CPM_OK;
}

cpm_status cpm_profile_read(cpm_ctx* c, int32_t k, double* total_ms, int64_t* launches, int32_t reset) {
    if (!c || k < 0 || k >= CPM_K_COUNT) return CPM_E_ARG;
    CPM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int j = 0; j < CPM_K_COUNT; ++j) {
        for (auto& pr : c->prof_pending[j]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
                c->prof_ms[j] += ms;
                c->prof_cnt[j] += 1;
            } else {
                cudaGetLastError();
            }
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        c->prof_pending[j].clear();
    }
    if (total_ms) *total_ms = c->prof_ms[k];
    if (launches) *launches = c->prof_cnt[k];
    if (reset)
        for (int j = 0; j < CPM_K_COUNT; ++j) { c->prof_ms[j] = 0; c->prof_cnt[j] = 0; }
    return CPM_OK;
}

}  // extern "C"
