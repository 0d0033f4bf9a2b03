// C ABI of libf3r and the host driver of the nest.
//
// The outer fp64 FGMRES(m1) runs on the host loop (Sec. 4.2: convergence is
// checked only there; the whole nest restarts after m1 iterations).  One
// outer iteration -- the inner call F_{m2}(F_{m3}(R_{m4}(M))) plus the outer
// SpMV, CGS2 and Givens step -- has no data-dependent control flow on the
// host, so it is captured once as a CUDA graph and replayed; the host reads
// one small status record per outer iteration.  The Richardson update calls
// (every c-th call, Algorithm 1) fall at positions fixed by c_ntr mod c, so
// graphs are cached per residue.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "ctx.h"
#include "kernels.cuh"

using namespace f3r;

struct f3r_ctx {
    Ctx c;
    cudaStream_t cs = nullptr;  // internal stream (graph capture needs a non-legacy stream)
    bool owns_stream = false;
    Readback *rb_dev = nullptr;
};

namespace {

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device allocation, zero-filled in the context's stream (so the fill is
// ordered before every later use in that stream, unlike a legacy-stream memset)
void *dalloc(Ctx &c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = pool_alloc(c.dev, bytes, c.zstream);
    if (!p) return nullptr;
    c.allocs.push_back(p);
    c.bytes += (long long)bytes;
    cudaMemsetAsync(p, 0, bytes, c.zstream);
    return p;
}

f3r_status check_params(const f3r_params &p) {
    if (p.nlevels < 1 || p.nlevels > 4) return F3R_ERR_ARG;
    if (p.m[0] < 1 || p.m[0] > kMaxOuterM) return F3R_ERR_ARG;
    if (p.a_prec[0] != F3R_F64 || p.v_prec[0] != F3R_F64) return F3R_ERR_ARG;
    for (int d = 1; d < p.nlevels; ++d) {
        if (p.m[d] < 1 || p.m[d] > kMaxLongM) return F3R_ERR_ARG;
        if (p.v_prec[d] == F3R_F64) {
            if (p.a_prec[d] != F3R_F64) return F3R_ERR_UNSUPPORTED;
        } else if (p.v_prec[d] == F3R_F32) {
            if (p.a_prec[d] != F3R_F32 && p.a_prec[d] != F3R_F16 && p.a_prec[d] != F3R_BF16) return F3R_ERR_UNSUPPORTED;
        } else if (p.v_prec[d] == F3R_F16 || p.v_prec[d] == F3R_BF16) {
            // 16-bit stored vectors (Table 4): the innermost level, applying M itself
            if (d != p.nlevels - 1 || p.rich_m != 0) return F3R_ERR_UNSUPPORTED;
            if (p.a_prec[d] != F3R_F32 && p.a_prec[d] != F3R_F16 && p.a_prec[d] != F3R_BF16) return F3R_ERR_UNSUPPORTED;
        } else {
            return F3R_ERR_UNSUPPORTED;
        }
    }
    if (p.rich_m < 0 || p.rich_m > kMaxRich) return F3R_ERR_ARG;
    if (p.m_prec < 0 || p.m_prec > 3) return F3R_ERR_ARG;
    const int pv = p.v_prec[p.nlevels - 1];
    if (p.rich_m > 0) {
        const int a = p.rich_a_prec, v = p.rich_v_prec;
        const bool ok = (a == v) && (a >= 0 && a <= 3);
        if (!ok) return F3R_ERR_UNSUPPORTED;
        if ((v == F3R_F64) != (pv == F3R_F64)) return F3R_ERR_UNSUPPORTED;
        if (p.m_prec != v) return F3R_ERR_UNSUPPORTED;
    }
    if (p.c < 1 || p.max_outer < 1 || !(p.tol >= 0.0)) return F3R_ERR_ARG;
    if (p.cgs_passes != 1 && p.cgs_passes != 2) return F3R_ERR_ARG;
    if (!(p.inner_rtol >= 0.0f && p.inner_rtol < 1.0f)) return F3R_ERR_ARG;
    if (p.precond != F3R_PC_IDENTITY && p.precond != F3R_PC_JACOBI && p.precond != F3R_PC_LEARNED &&
        p.precond != F3R_PC_AINV)
        return F3R_ERR_ARG;
    if (p.precond == F3R_PC_AINV &&
        (p.rich_m < 1 || p.rich_v_prec != F3R_F16 || p.rich_a_prec != F3R_F16 || p.m_prec != F3R_F16 ||
         p.row_scale || !(p.ainv_alpha > 0.0f)))
        return F3R_ERR_UNSUPPORTED;
    if (p.precond == F3R_PC_LEARNED &&
        (p.rich_m < 1 || p.rich_v_prec != F3R_F16 || p.rich_a_prec != F3R_F16 || p.row_scale))
        return F3R_ERR_UNSUPPORTED;
    return F3R_OK;
}

bool rich_is_double(const Ctx &c) { return c.prm.rich_v_prec == F3R_F64; }

void upload_omega(Ctx &c, cudaStream_t s) {
    if (c.prm.rich_m <= 0) return;
    if (rich_is_double(c)) {
        cudaMemcpyAsync(c.omega, c.omega_host, sizeof(double) * kMaxRich, cudaMemcpyHostToDevice, s);
    } else {
        float tmp[kMaxRich];
        for (int k = 0; k < kMaxRich; ++k) tmp[k] = (float)c.omega_host[k];
        cudaMemcpyAsync(c.omega, tmp, sizeof(tmp), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);  // tmp lives on this stack frame
    }
}

void download_omega(Ctx &c, cudaStream_t s) {
    if (c.prm.rich_m <= 0) return;
    if (rich_is_double(c)) {
        cudaMemcpyAsync(c.omega_host, c.omega, sizeof(double) * kMaxRich, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
    } else {
        float tmp[kMaxRich];
        cudaMemcpyAsync(tmp, c.omega, sizeof(tmp), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        for (int k = 0; k < kMaxRich; ++k) c.omega_host[k] = tmp[k];
    }
}

void upload_cntr(Ctx &c, cudaStream_t s) {
    *c.hostval = 0.0;
    long long v = c.c_ntr;
    cudaMemcpyAsync(c.c_ntr_base, &v, sizeof(long long), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
}

bool is_update(const Ctx &c, long long pos) {
    if (c.prm.rich_m <= 0 || c.prm.omega_fixed > 0.0) return false;
    return ((c.c_ntr + pos) % c.prm.c) == 0;
}

// number of Richardson calls made by one call of level d (d >= 1), or by one
// outer iteration (d = 0)
long long calls_per_call(const Ctx &c, int d) {
    if (c.prm.rich_m <= 0) return 0;
    long long k = 1;
    for (int l = std::max(d, 1); l < c.prm.nlevels; ++l) k *= c.prm.m[l];
    return k;
}

void *zslot(Ctx &c, int d, int j) {
    return (char *)c.L[d].Z + (size_t)j * c.ld * level_vec_bytes(c, d);
}
void *vslot(Ctx &c, int d, int j) {
    return (char *)c.L[d].V + (size_t)j * c.ld * level_vec_bytes(c, d);
}
void *misc_of(Ctx &c, int d) {
    return (char *)c.L[d].scal + (size_t)scal_misc(c.L[d].m) * level_vec_bytes(c, d);
}

// One call of inner FGMRES level d (x0 = 0, m_d iterations, no convergence
// test), whose normalised input sits in V[0] / its scalars; result to `out`.
void run_level(Ctx &c, int d, const OutSlot &out, long long &pos, cudaStream_t s) {
    LevelHost &L = c.L[d];
    const bool lng = L.m > kMaxInnerM;  // Table 4's F2: CGS2 over the basis in chunks
    launch_normalize(c, d, false, 0, s);
    for (int j = 0; j < L.m; ++j) {
        if (L.child == CHILD_F) {
            OutSlot o;
            o.ptr = zslot(c, d, j);
            o.prec = L.v_prec;
            run_level(c, d + 1, o, pos, s);
        } else if (L.child == CHILD_R) {
            // the whole iteration in one cooperative launch when it applies
            if (!lng && launch_f3_step(c, d, j, j == L.m - 1, is_update(c, pos), s)) {
                ++pos;
                continue;
            }
            launch_rich_call(c, is_update(c, pos), (int)pos, zslot(c, d, j), misc_of(c, d), s);
            ++pos;
        } else {
            launch_M(c, d, j, vslot(c, d, j), zslot(c, d, j), d, false, s, vround_of(c, d));
        }
        if (lng) {
            launch_long_step(c, d, j, j == L.m - 1, s);
            if (j < L.m - 1) launch_normalize(c, d, true, j + 1, s);
            continue;
        }
        launch_spmv_dots(c, d, j, s);
        if (launch_cgs_fused(c, d, j, j == L.m - 1, j < L.m - 1, s)) continue;
        if (c.prm.cgs_passes == 2) launch_cgs_pass(c, d, j, s);
        launch_cgs_final(c, d, j, j == L.m - 1, s);
        if (j < L.m - 1) launch_normalize(c, d, true, j + 1, s);
    }
    launch_combine(c, d, out, s);
}

__global__ void k_pack_readback(const double *misc0, const int *flags, const unsigned long long *counters,
                                const int *err, Readback *rb) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        rb->err = *err;
        rb->est = misc0[MS_EST];
        rb->rel = misc0[MS_REL];
        rb->nb = misc0[MS_NB];
        for (int k = 0; k < 16; ++k) rb->flags[k] = flags[k];
        for (int k = 0; k < 4; ++k) rb->counters[k] = counters[k];
    }
}

void pack_readback(f3r_ctx *h, cudaStream_t s) {
    Ctx &c = h->c;
    launch_pdl(k_pack_readback, dim3(1), dim3(32), 0, s, (const double *)misc_of(c, 0), c.flags, c.counters, c.err, h->rb_dev);
    c.launches++;
    cudaMemcpyAsync(c.rb, h->rb_dev, sizeof(Readback), cudaMemcpyDeviceToHost, s);
}

// the device work of one outer iteration j (j itself lives on the device)
void outer_iteration_body(f3r_ctx *h, cudaStream_t s) {
    Ctx &c = h->c;
    long long pos = 0;
    LevelHost &L0 = c.L[0];
    if (L0.child == CHILD_F) {
        OutSlot o;
        o.ptr = c.zst;
        o.prec = F3R_F64;
        o.dscale = c.prm.diag_scale != 0;
        run_level(c, 1, o, pos, s);
    } else if (L0.child == CHILD_R) {
        launch_rich_call(c, is_update(c, pos), (int)pos, c.zst, misc_of(c, 0), s);
        ++pos;
    } else {
        launch_M(c, 0, 0, c.L[0].V, c.zst, 0, true, s);
    }
    if (!launch_outer_step(c, s)) launch_normalize(c, 0, true, 1, s);
    if (c.calls_per_outer) launch_advance(c, c.calls_per_outer, s);
    pack_readback(h, s);
}

cudaError_t run_outer_iteration(f3r_ctx *h, cudaStream_t s) {
    Ctx &c = h->c;
    if (!c.prm.use_graphs || c.prof) {
        outer_iteration_body(h, s);
        return cudaGetLastError();
    }
    const long long key = (c.prm.rich_m > 0 && c.prm.omega_fixed <= 0.0) ? (c.c_ntr % c.prm.c) : 0;
    auto it = c.graphs.find(key);
    if (it == c.graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        const long long before = c.launches;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        outer_iteration_body(h, s);
        e = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        c.launches_per_graph_iter = c.launches - before;
        c.launches = before;
        it = c.graphs.emplace(key, ge).first;
    }
    c.launches += c.launches_per_graph_iter;
    c.graph_launches++;
    return cudaGraphLaunch(it->second, s);
}

void push(double *arr, int cap, int &len, double v) {
    if (arr && len < cap) arr[len] = v;
    ++len;
}

}  // namespace

extern "C" {

f3r_status f3r_default_params(f3r_params *p) {
    if (!p) return F3R_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->nlevels = 3;
    p->m[0] = 100;
    p->m[1] = 8;
    p->m[2] = 4;
    p->a_prec[0] = F3R_F64;
    p->a_prec[1] = F3R_F32;
    p->a_prec[2] = F3R_F16;
    p->a_prec[3] = F3R_F16;
    p->v_prec[0] = F3R_F64;
    p->v_prec[1] = F3R_F32;
    p->v_prec[2] = F3R_F32;
    p->v_prec[3] = F3R_F32;
    p->rich_m = 2;
    p->rich_a_prec = F3R_F16;
    p->rich_v_prec = F3R_F16;
    p->m_prec = F3R_F16;
    p->precond = F3R_PC_JACOBI;
    p->c = 64;
    p->omega_fixed = 0.0;
    p->diag_scale = 1;
    p->row_scale = 0;
    p->scale_cast = 1;
    p->cgs_passes = 2;
    p->tol = 1e-9;
    p->max_outer = 300;
    p->use_graphs = 1;
    p->keep_omega = 0;
    p->fuse_cgs = 1;
    p->fuse_step = 0;
    p->ainv_alpha = 1.0f;
    return F3R_OK;
}

const char *f3r_status_str(f3r_status s) {
    switch (s) {
        case F3R_OK: return "ok";
        case F3R_ERR_ARG: return "invalid argument";
        case F3R_ERR_CUDA: return "CUDA error";
        case F3R_ERR_NOMEM: return "out of memory";
        case F3R_NOT_CONVERGED: return "not converged";
        case F3R_ERR_BREAKDOWN: return "breakdown";
        case F3R_ERR_NONFINITE: return "non-finite value";
        case F3R_ERR_TIMEOUT: return "device wait timed out";
        case F3R_ERR_UNSUPPORTED: return "unsupported parameter combination";
    }
    return "unknown";
}

void f3r_destroy(f3r_ctx *h) {
    if (!h) return;
    Ctx &c = h->c;
    for (auto &kv : c.graphs) cudaGraphExecDestroy(kv.second);
    learned_free(c);
    krylov_free(c);
    for (auto &r : c.prec) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (void *p : c.allocs) pool_free(p, c.zstream);
    if (c.zstream) cudaStreamSynchronize(c.zstream);
    if (c.rb) cudaFreeHost(c.rb);
    if (c.hostval) cudaFreeHost(c.hostval);
    if (c.ev0) cudaEventDestroy(c.ev0);
    if (c.ev1) cudaEventDestroy(c.ev1);
    if (h->owns_stream && h->cs) cudaStreamDestroy(h->cs);
    delete h;
}

int64_t f3r_device_bytes(const f3r_ctx *h) { return h ? h->c.bytes : 0; }

f3r_status f3r_setup(f3r_ctx **out, int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                     const double *val, const f3r_params *params, void *stream) {
    if (!out || n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!colidx || !val))) return F3R_ERR_ARG;
    *out = nullptr;
    f3r_params prm;
    if (params) prm = *params;
    else f3r_default_params(&prm);
    f3r_status st = check_params(prm);
    if (st != F3R_OK) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return F3R_ERR_CUDA;
    }
    f3r_ctx *h = new (std::nothrow) f3r_ctx;
    if (!h) return F3R_ERR_NOMEM;
    Ctx &c = h->c;
    c.dev = dev;
    cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev);
    if (c.nsm <= 0) c.nsm = 1;
    c.prm = prm;
    c.n = n;
    c.nnz = nnz;
    c.ld = (int)(((long long)n + kTileRows - 1) / kTileRows * kTileRows);  // whole tiles
    if (cudaStreamCreateWithFlags(&h->cs, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return F3R_ERR_CUDA;
    }
    h->owns_stream = true;
    cudaStream_t s = h->cs;
    c.zstream = s;
    cudaStream_t us = (cudaStream_t)stream;
    cudaEventCreate(&c.ev0);
    cudaEventCreate(&c.ev1);
    // order after the caller's pending work (us = 0 is the legacy default stream)
    cudaEventRecord(c.ev0, us);
    cudaStreamWaitEvent(s, c.ev0, 0);
    // the CSR arrays on the device
    const int *rp = rowptr, *ci = colidx;
    const double *va = val;
    void *tmp[3] = {nullptr, nullptr, nullptr};
    auto up = [&](const void *src, size_t bytes, int slot) -> const void * {
        if (is_device_ptr(src)) return src;
        tmp[slot] = pool_alloc(dev, bytes, s);
        if (!tmp[slot]) return nullptr;
        cudaMemcpyAsync(tmp[slot], src, bytes, cudaMemcpyHostToDevice, s);
        return tmp[slot];
    };
    rp = (const int *)up(rowptr, sizeof(int) * ((size_t)n + 1), 0);
    ci = (const int *)up(colidx, sizeof(int) * (size_t)nnz, 1);
    va = (const double *)up(val, sizeof(double) * (size_t)nnz, 2);
    auto fail = [&](f3r_status e) {
        for (void *p : tmp)
            if (p) pool_free(p, s);
        f3r_destroy(h);
        return e;
    };
    if (!rp || (nnz > 0 && (!ci || !va))) return fail(F3R_ERR_NOMEM);
    st = build_matrix(c, rp, ci, va, s);
    if (st != F3R_OK) return fail(st);
    for (void *p : tmp)
        if (p) pool_free(p, s);
    tmp[0] = tmp[1] = tmp[2] = nullptr;

    // grid shapes: a few resident blocks per SM, never more blocks than work
    c.G = std::max(1, std::min(ceil_div(n, kBlock), c.nsm * 4));
    c.Gs = std::max(1, std::min(ceil_div(c.nslices, kWarps), c.nsm * 4));
    c.G1 = std::max(1, std::min(ceil_div(n, 512), c.nsm));
    c.Gv = std::max(1, std::min(ceil_div(n, 512 * 16), c.nsm * 2));

    // levels (Table 1)
    for (int d = 0; d < prm.nlevels; ++d) {
        LevelHost &L = c.L[d];
        L.m = prm.m[d];
        L.a_prec = prm.a_prec[d];
        L.v_prec = prm.v_prec[d];
        L.child = (d + 1 < prm.nlevels) ? CHILD_F : (prm.rich_m > 0 ? CHILD_R : CHILD_M);
        const size_t eb = (size_t)level_vec_bytes(c, d);
        L.V = dalloc(c, eb * c.ld * (L.m + 1));
        L.Z = dalloc(c, eb * c.ld * L.m);
        L.w = dalloc(c, eb * c.ld);
        L.scal = dalloc(c, eb * scal_size(L.m));
        if (!L.V || !L.Z || !L.w || !L.scal) return fail(F3R_ERR_NOMEM);
    }
    if (prm.rich_m > 0) {
        const size_t vb = (size_t)prec_bytes(prm.rich_v_prec) * c.ld;
        c.rin = dalloc(c, vb);
        c.rz[0] = dalloc(c, vb);
        c.rz[1] = dalloc(c, vb);
        c.rr = dalloc(c, vb);
        if (!c.rin || !c.rz[0] || !c.rz[1] || !c.rr) return fail(F3R_ERR_NOMEM);
    }
    c.omega = dalloc(c, sizeof(double) * kMaxRich);
    c.wcur = dalloc(c, sizeof(double) * 2);
    c.counters = (unsigned long long *)dalloc(c, sizeof(unsigned long long) * 4);
    c.c_ntr_base = (long long *)dalloc(c, sizeof(long long));
    c.zst = dalloc(c, sizeof(double) * c.ld);
    c.apply_misc = dalloc(c, sizeof(double) * MS_COUNT);
    // partial sums: grid reductions, the outer CGS, and the fused kernels'
    // [vector][block] regions (two of kMaxOuterM + 1 rows, one more row; <= 2 blocks per SM)
    const size_t pbytes = std::max({(size_t)c.nsm * kMaxStagedBlocksPerSM * kMaxDots * sizeof(double),
                                    (size_t)(kMaxOuterM + 2) * c.G1 * sizeof(double),
                                    (size_t)(2 * (kMaxOuterM + 1) + 2) * c.nsm * 2 * sizeof(double),
                                    (size_t)(kMaxLongM + 1) * c.nsm * 2 * sizeof(double)});
    c.partials = dalloc(c, pbytes);
    c.hpart = dalloc(c, (size_t)c.nsm * kMaxStagedBlocksPerSM * kMaxDots * sizeof(double));
    c.ticket = (unsigned *)dalloc(c, sizeof(unsigned) * 4);
    c.coop = (unsigned *)dalloc(c, sizeof(unsigned) * 4);
    c.err = (int *)dalloc(c, sizeof(int) * 4);
    c.flags = (int *)dalloc(c, sizeof(int) * 16);
    c.jdev = (int *)dalloc(c, sizeof(int) * 4);
    h->rb_dev = (Readback *)dalloc(c, sizeof(Readback));
    if (!c.omega || !c.wcur || !c.counters || !c.c_ntr_base || !c.zst || !c.apply_misc || !c.partials ||
        !c.hpart || !c.ticket || !c.coop || !c.err || !c.flags || !c.jdev || !h->rb_dev)
        return fail(F3R_ERR_NOMEM);
    plan_cgs_fused(c);
    if (cudaHostAlloc((void **)&c.rb, sizeof(Readback), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&c.hostval, sizeof(double) * 8, cudaHostAllocDefault) != cudaSuccess)
        return fail(F3R_ERR_NOMEM);
    c.calls_per_outer = (int)calls_per_call(c, 0);
    for (int k = 0; k < kMaxRich; ++k) c.omega_host[k] = (prm.omega_fixed > 0.0) ? prm.omega_fixed : 1.0;
    c.c_ntr = 1;
    upload_omega(c, s);
    upload_cntr(c, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(F3R_ERR_CUDA);
    *out = h;
    return F3R_OK;
}

f3r_status f3r_solve(f3r_ctx *h, const double *b, double *x, f3r_stats *stats, void *stream) {
    if (!h || !b || !x) return F3R_ERR_ARG;
    Ctx &c = h->c;
    cudaStream_t s = h->cs;
    cudaStream_t us = (cudaStream_t)stream;
    const int n = c.n;
    cudaEventRecord(c.ev0, us);
    cudaStreamWaitEvent(s, c.ev0, 0);
    const bool bdevp = is_device_ptr(b), xdevp = is_device_ptr(x);
    const double *bd = b;
    double *xd = x;
    if (!bdevp || !xdevp) {
        if (!c.bdev) {
            c.bdev = (double *)dalloc(c, sizeof(double) * n);
            c.xdev = (double *)dalloc(c, sizeof(double) * n);
            if (!c.bdev || !c.xdev) return F3R_ERR_NOMEM;
        }
        if (!bdevp) {
            cudaMemcpyAsync(c.bdev, b, sizeof(double) * n, cudaMemcpyHostToDevice, s);
            bd = c.bdev;
        }
        if (!xdevp) {
            cudaMemcpyAsync(c.xdev, x, sizeof(double) * n, cudaMemcpyHostToDevice, s);
            xd = c.xdev;
        }
    }
    cudaEventRecord(c.ev0, s);
    // Algorithm 1: weights start at 1 on the first call of a solve
    if (!c.prm.keep_omega) {
        c.c_ntr = 1;
        for (int k = 0; k < kMaxRich; ++k) c.omega_host[k] = (c.prm.omega_fixed > 0.0) ? c.prm.omega_fixed : 1.0;
        upload_omega(c, s);
    }
    upload_cntr(c, s);
    cudaMemsetAsync(c.counters, 0, sizeof(unsigned long long) * 4, s);
    cudaMemsetAsync(c.flags, 0, sizeof(int) * 16, s);
    cudaMemsetAsync(c.err, 0, sizeof(int) * 4, s);
    // reduction tickets and barrier counters: zero unless an earlier solve gave up inside a kernel
    cudaMemsetAsync(c.ticket, 0, sizeof(unsigned) * 4, s);
    cudaMemsetAsync(c.coop, 0, sizeof(unsigned) * 4, s);
    const long long launches0 = c.launches, glaunch0 = c.graph_launches;

    int hist_len = 0, true_len = 0;
    int total = 0, cycles = 0;
    f3r_status status = F3R_NOT_CONVERGED;
    double rel = 0.0;
    bool first = true;
    const int m1 = c.prm.m[0];
    for (;;) {
        launch_outer_residual(c, bd, xd, first, s);
        first = false;
        pack_readback(h, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
        rel = c.rb->rel;
        push(stats ? stats->true_hist : nullptr, stats ? stats->true_cap : 0, true_len, rel);
        if (c.rb->nb == 0.0) {
            // ||b|| = 0: x = 0 solves the system
            cudaMemsetAsync(xd, 0, sizeof(double) * n, s);
            rel = 0.0;
            true_len = 0;
            push(stats ? stats->true_hist : nullptr, stats ? stats->true_cap : 0, true_len, rel);
            status = F3R_OK;
            break;
        }
        if (!std::isfinite(rel)) {
            status = F3R_ERR_NONFINITE;
            break;
        }
        if (rel < c.prm.tol) {
            status = F3R_OK;
            break;
        }
        if (total >= c.prm.max_outer) {
            status = F3R_NOT_CONVERGED;
            break;
        }
        ++cycles;
        launch_normalize(c, 0, true, 0, s);
        bool nonfinite = false;
        for (int j = 0; j < m1; ++j) {
            cudaError_t e = run_outer_iteration(h, s);
            if (e != cudaSuccess) return F3R_ERR_CUDA;
            if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
            prof_collect(c);
            ++total;
            c.c_ntr += c.calls_per_outer;
            const Readback &rb = *c.rb;
            if (rb.err) return F3R_ERR_TIMEOUT;
            const int *fl0 = rb.flags;  // outer level flags
            if (fl0[IF_NONFINITE]) {
                nonfinite = true;
                break;
            }
            if (fl0[IF_KDIM] == j + 1)
                push(stats ? stats->hist : nullptr, stats ? stats->hist_cap : 0, hist_len, rb.est);
            if (fl0[IF_STOP]) break;
            if (rb.est < c.prm.tol || total >= c.prm.max_outer) break;
        }
        launch_outer_finish(c, xd, s);
        if (nonfinite) {
            launch_outer_residual(c, bd, xd, false, s);
            pack_readback(h, s);
            cudaStreamSynchronize(s);
            rel = c.rb->rel;
            push(stats ? stats->true_hist : nullptr, stats ? stats->true_cap : 0, true_len, rel);
            status = F3R_ERR_NONFINITE;
            break;
        }
    }
    cudaEventRecord(c.ev1, s);
    if (!xdevp) cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
    prof_collect(c);
    download_omega(c, s);
    if (stats) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, c.ev0, c.ev1);
        stats->status = status;
        stats->outer_iters = total;
        stats->restarts = cycles > 0 ? cycles - 1 : 0;
        stats->rel_res_true = rel;
        stats->m_applies = (int64_t)c.rb->counters[0];
        stats->r_calls = (int64_t)c.rb->counters[1];
        stats->r_update_calls = (int64_t)c.rb->counters[2];
        for (int k = 0; k < 8; ++k) stats->omega[k] = c.omega_host[k];
        stats->hist_len = hist_len;
        stats->true_len = true_len;
        stats->t_solve_ms = ms;
        stats->kernel_launches = c.launches - launches0;
        stats->graph_launches = c.graph_launches - glaunch0;
    }
    cudaEventRecord(c.ev1, s);
    cudaStreamWaitEvent(us, c.ev1, 0);
    if (cudaGetLastError() != cudaSuccess) return F3R_ERR_CUDA;
    return status;
}

f3r_status f3r_solve_krylov(f3r_ctx *h, int method, const double *b, double *x, int max_iters, f3r_stats *stats,
                            void *stream) {
    if (!h || !b || !x || (method != F3R_KRYLOV_CG && method != F3R_KRYLOV_BICGSTAB) || max_iters < 0)
        return F3R_ERR_ARG;
    Ctx &c = h->c;
    cudaStream_t s = h->cs;
    cudaStream_t us = (cudaStream_t)stream;
    const int n = c.n;
    cudaEventRecord(c.ev0, us);
    cudaStreamWaitEvent(s, c.ev0, 0);
    const bool bdevp = is_device_ptr(b), xdevp = is_device_ptr(x);
    const double *bd = b;
    double *xd = x;
    if (!bdevp || !xdevp) {
        if (!c.bdev) {
            c.bdev = (double *)dalloc(c, sizeof(double) * n);
            c.xdev = (double *)dalloc(c, sizeof(double) * n);
            if (!c.bdev || !c.xdev) return F3R_ERR_NOMEM;
        }
        if (!bdevp) {
            cudaMemcpyAsync(c.bdev, b, sizeof(double) * n, cudaMemcpyHostToDevice, s);
            bd = c.bdev;
        }
        if (!xdevp) {
            cudaMemcpyAsync(c.xdev, x, sizeof(double) * n, cudaMemcpyHostToDevice, s);
            xd = c.xdev;
        }
    }
    cudaEventRecord(c.ev0, s);
    f3r_status st = krylov_solve(c, s, method == F3R_KRYLOV_CG ? 1 : 2, bd, xd, max_iters, stats);
    cudaEventRecord(c.ev1, s);
    if (!xdevp) cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
    if (stats) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, c.ev0, c.ev1);
        stats->t_solve_ms = ms;
    }
    cudaEventRecord(c.ev1, s);
    cudaStreamWaitEvent(us, c.ev1, 0);
    return st;
}

f3r_status f3r_spmv(f3r_ctx *h, int p, int vp, const void *x, void *y, void *stream) {
    if (!h || !x || !y) return F3R_ERR_ARG;
    f3r_status st = launch_spmv(h->c, p, vp, x, y, (cudaStream_t)stream);
    if (st != F3R_OK) return st;
    return cudaGetLastError() == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

f3r_status f3r_apply(f3r_ctx *h, int level, const void *x, void *z, void *stream) {
    if (!h || !x || !z) return F3R_ERR_ARG;
    Ctx &c = h->c;
    const int nl = c.prm.nlevels;
    if (level < 1 || level > nl) return F3R_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    upload_cntr(c, s);
    cudaMemsetAsync(c.flags, 0, sizeof(int) * 16, s);
    if (level < nl) {
        launch_level_start(c, level, x, s);
        OutSlot o;
        o.ptr = z;
        o.prec = c.L[level].v_prec;
        long long pos = 0;
        run_level(c, level, o, pos, s);
        c.c_ntr += pos;
    } else if (c.prm.rich_m > 0) {
        launch_rich_prep(c, x, s);
        launch_rich_call(c, is_update(c, 0), 0, z, c.apply_misc, s);
        c.c_ntr += 1;
    } else {
        launch_M(c, nl - 1, 0, x, z, 0, false, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
    download_omega(c, s);
    return cudaGetLastError() == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

f3r_status f3r_get_basis(f3r_ctx *h, int level, int k, void *out, void *stream) {
    if (!h || !out) return F3R_ERR_ARG;
    Ctx &c = h->c;
    if (level < 0 || level >= c.prm.nlevels || k < 0 || k > c.L[level].m) return F3R_ERR_ARG;
    const size_t eb = (size_t)level_vec_bytes(c, level);
    const char *src = (const char *)c.L[level].V + (size_t)k * c.ld * eb;
    cudaStream_t s = (cudaStream_t)stream;
    // ordered after the context's own work (the solve that left the basis)
    cudaEventRecord(c.ev1, h->cs);
    cudaStreamWaitEvent(s, c.ev1, 0);
    if (cudaMemcpyAsync(out, src, eb * (size_t)c.n, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return F3R_ERR_CUDA;
    }
    return F3R_OK;
}

f3r_status f3r_get_rich_state(f3r_ctx *h, double *omega8, int64_t *c_ntr) {
    if (!h) return F3R_ERR_ARG;
    if (omega8)
        for (int k = 0; k < 8; ++k) omega8[k] = h->c.omega_host[k];
    if (c_ntr) *c_ntr = h->c.c_ntr;
    return F3R_OK;
}

f3r_status f3r_set_rich_state(f3r_ctx *h, const double *omega8, int64_t c_ntr) {
    if (!h || c_ntr < 1) return F3R_ERR_ARG;
    Ctx &c = h->c;
    if (omega8)
        for (int k = 0; k < 8; ++k) c.omega_host[k] = omega8[k];
    c.c_ntr = c_ntr;
    upload_omega(c, h->cs);
    upload_cntr(c, h->cs);
    return cudaStreamSynchronize(h->cs) == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

f3r_status f3r_profile_enable(f3r_ctx *h, int enable) {
    if (!h) return F3R_ERR_ARG;
    Ctx &c = h->c;
    if (cudaDeviceSynchronize() != cudaSuccess) return F3R_ERR_CUDA;
    prof_collect(c);
    c.prof = enable != 0;
    if (c.prof)
        for (int k = 0; k < kProfSlots; ++k) {
            c.prof_ms[k] = 0.0;
            c.prof_cnt[k] = 0;
        }
    return F3R_OK;
}

f3r_status f3r_profile_get(f3r_ctx *h, int slot, int64_t *launches, double *total_ms) {
    if (!h || slot < 0 || slot >= kProfSlots) return F3R_ERR_ARG;
    Ctx &c = h->c;
    if (cudaDeviceSynchronize() != cudaSuccess) return F3R_ERR_CUDA;
    prof_collect(c);
    if (launches) *launches = c.prof_cnt[slot];
    if (total_ms) *total_ms = c.prof_ms[slot];
    return F3R_OK;
}

int f3r_profile_slots(void) { return kProfSlots; }

const char *f3r_profile_slot_name(int slot) {
    static const char *names[PK_KINDS] = {"spmv_dots", "cgs_pass", "cgs_final", "normalize", "combine",
                                          "level_start", "apply_M", "rich_fused2", "rich_step", "rich_update",
                                          "outer_spmv", "outer_cgs", "outer_other", "spmv", "cgs_fused", "f3_step"};
    if (slot < 0 || slot >= kProfSlots) return "";
    return names[slot / 4];
}

f3r_status f3r_learned_set_loss(f3r_ctx *h, int kind) {
    if (!h) return F3R_ERR_ARG;
    return learned_set_loss(h->c, kind);
}

f3r_status f3r_learned_load(f3r_ctx *h, const float *params, int train) {
    if (!h || !params) return F3R_ERR_ARG;
    return learned_enable(h->c, params, train != 0);
}

f3r_status f3r_learned_get(f3r_ctx *h, float *out) {
    if (!h || !out || !h->c.learned) return F3R_ERR_ARG;
    return cudaMemcpy(out, learned_theta(h->c), sizeof(float) * F3R_LEARNED_NPARAMS, cudaMemcpyDeviceToHost) ==
                   cudaSuccess
               ? F3R_OK
               : F3R_ERR_CUDA;
}

f3r_status f3r_learned_apply(f3r_ctx *h, const float *r, float *z, void *stream) {
    if (!h || !r || !z || !h->c.learned) return F3R_ERR_ARG;
    learned_forward(h->c, r, z, false, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

f3r_status f3r_learned_loss_grad(f3r_ctx *h, const float *R, const float *E, int P, float *loss, float *grad,
                                 void *stream) {
    if (!h || !R || P < 1 || !h->c.learned) return F3R_ERR_ARG;
    if (!E && learned_loss_kind(h->c) == 0) return F3R_ERR_ARG;
    f3r_status st = learned_enable(h->c, nullptr, true);
    if (st != F3R_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = learned_loss_grad(h->c, R, E, P, s);
    if (st != F3R_OK) return st;
    if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
    if (loss) cudaMemcpy(loss, learned_loss(h->c), sizeof(float), cudaMemcpyDeviceToHost);
    if (grad) cudaMemcpy(grad, learned_grad(h->c), sizeof(float) * F3R_LEARNED_NPARAMS, cudaMemcpyDeviceToHost);
    return cudaGetLastError() == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

f3r_status f3r_learned_train(f3r_ctx *h, const float *R, const float *E, int P, int steps, int batch, float lr,
                             float *loss_hist, void *stream) {
    if (!h || !R || P < 1 || steps < 0 || batch < 1 || batch > P || !h->c.learned) return F3R_ERR_ARG;
    if (!E && learned_loss_kind(h->c) == 0) return F3R_ERR_ARG;
    f3r_status st = learned_enable(h->c, nullptr, true);
    if (st != F3R_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = h->c.n;
    int p0 = 0;
    for (int k = 0; k < steps; ++k) {
        const int b = std::min(batch, P - p0);
        st = learned_loss_grad(h->c, R + (size_t)p0 * n, E ? E + (size_t)p0 * n : nullptr, b, s);
        if (st != F3R_OK) return st;
        learned_adam(h->c, lr, s);
        if (loss_hist) {
            if (cudaMemcpyAsync(loss_hist + k, learned_loss(h->c), sizeof(float), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
                return F3R_ERR_CUDA;
        }
        p0 = (p0 + b) % P;
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

f3r_status f3r_export(f3r_ctx *h, int which, void *out) {
    if (!h || !out) return F3R_ERR_ARG;
    return export_array(h->c, which, out, h->cs);
}

f3r_status f3r_matrix_info(f3r_ctx *h, int64_t *out) {
    if (!h || !out) return F3R_ERR_ARG;
    const Ctx &c = h->c;
    out[0] = c.win ? 1 : 0;
    out[1] = c.win_max;
    out[2] = c.nsell;
    out[3] = c.wmax;
    out[4] = c.nslices;
    out[5] = c.win ? 2 : 4;
    out[6] = kWinChunk;
    out[7] = c.m_unit ? 1 : 0;
    return F3R_OK;
}

}  // extern "C"
