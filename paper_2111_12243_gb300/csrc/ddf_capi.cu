// C ABI of libddf.so (declared in include/ddf.h): argument checks, plan
// ownership, host/device staging and the execute entry points.
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ddf_internal.cuh"

static std::atomic<int64_t> g_launches{0};
void ddf_count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ddf_debug_fail_alloc: allocations still to succeed before one fails (-1: off)
static std::atomic<int64_t> g_alloc_countdown{-1};

bool ddf_alloc_injected_failure() {
    int64_t c = g_alloc_countdown.load(std::memory_order_relaxed);
    while (c >= 0) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1, std::memory_order_relaxed)) return c == 0;
    }
    return false;
}

ddf_nvtx_range::ddf_nvtx_range(const char* name) { nvtxRangePushA(name); }
ddf_nvtx_range::~ddf_nvtx_range() { nvtxRangePop(); }

namespace {

void init_pool_once(int dev) {
    static std::atomic<bool> done[64];
    if (dev < 0 || dev >= 64 || done[dev].load()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        // keep freed plan memory in the process-local pool between inspections
        uint64_t thr = ~0ull;
        (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    (void)cudaGetLastError();
    done[dev].store(true);
}

void release(ddf_plan_s* p) {
    cudaStream_t s = p->stream;
    ddf_free(p->starts, s);
    ddf_free(p->col, s);
    ddf_free(p->val, s);
    ddf_free(p->seq, s);
    ddf_free(p->part_ptr, s);
    ddf_free(p->dinv, s);
    ddf_free(p->orig_rowptr, s);
    ddf_free(p->orig_rowend, s);
    ddf_free(p->cod, s);
    for (int k = 0; k < 3; ++k) ddf_free(p->units[k], s);
    for (int k = 0; k < 2; ++k) ddf_free(p->tiles[k], s);
    ddf_free(p->unit_q, s);
    ddf_free(p->mrhs_order, s);
    ddf_free(p->mrhs_q, s);
    ddf_free(p->mrhs_seg, s);
    ddf_free(p->mrhs_part, s);
    ddf_free(p->mrhs_cnt, s);
    ddf_free(p->mrhs_moff, s);
    ddf_free(p->long_q, s);
    ddf_free(p->status, s);
    ddf_free(p->ticket, s);
    if (p->val_lp) (void)cudaFreeAsync(p->val_lp, s);
    p->val_lp = nullptr;
    ddf_free(p->dinv_lp, s);
    ddf_free(p->diag, s);
    ddf_free(p->r64, s);
    ddf_free(p->rlp, s);
    ddf_free(p->xlp, s);
    ddf_free(p->nrm, s);
    ddf_free(p->blk_ptr, s);
    ddf_free(p->esplit, s);
    ddf_free(p->qcod, s);
    ddf_free(p->chunk_q0, s);
    ddf_free(p->chunk_meta, s);
    ddf_free(p->blk_chunk, s);
}

ddf_status check_opts(const ddf_opts* o) {
    if (o->window_t < 1 || o->window_t > DDF_MAX_T) return DDF_ERR_ARG;
    if (!(o->allowed_types & DDF_ALLOW_PSC2) || (o->allowed_types & ~DDF_ALLOW_ALL)) return DDF_ERR_ARG;
    if (o->w_op < 0 || o->w_codelet < 0 || o->w_index < 0) return DDF_ERR_ARG;
    if (o->spin_cap_ns <= 0 || o->unit_nnz < 1) return DDF_ERR_ARG;
    if (o->store_dtype != DDF_F64 && o->store_dtype != DDF_F32 && o->store_dtype != DDF_BF16) return DDF_ERR_ARG;
    if (o->coarsen_rows < 0 || o->coarsen_rows > DDF_COARSEN_MAX_ROWS) return DDF_ERR_ARG;
    if (o->lower_of_input != 0 && o->lower_of_input != 1) return DDF_ERR_ARG;
    return DDF_OK;
}

template <typename T>
ddf_status stage(T** dst, const T* src, int64_t n, int on_device, cudaStream_t s) {
    *dst = nullptr;
    if (n <= 0) return DDF_OK;
    ddf_status st = ddf_alloc(dst, n, s);
    if (st) return st;
    DDF_CUDA_TRY(cudaMemcpyAsync(*dst, src, (size_t)n * sizeof(T),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return DDF_OK;
}

// re[r]: end of row r of L (its diagonal is the entry before it)
__global__ void k_check_diag(int32_t n, const int32_t* __restrict__ re, const double* __restrict__ v,
                             int32_t* __restrict__ bad) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n && v[re[r] - 1] == 0.0) atomicExch(bad, 1);
}

}  // namespace

// A plan shell: options checked, status words allocated, nothing inspected.
ddf_status ddf_new_plan(ddf_kind kind, const ddf_opts* o, cudaStream_t s, int32_t n, int32_t n_cols, int64_t nnz,
                        ddf_plan_s** out) {
    *out = nullptr;
    ddf_opts opts;
    if (o) opts = *o;
    else ddf_opts_default(&opts);
    ddf_status st = check_opts(&opts);
    if (st) return st;
    if (kind == DDF_SPMV && opts.lower_of_input) return DDF_ERR_ARG;
    ddf_plan_s* p = new (std::nothrow) ddf_plan_s();
    if (!p) return DDF_ERR_OOM;
    memset(p, 0, sizeof(*p));
    p->kind = kind;
    p->opts = opts;
    p->stream = s;
    p->n = n;
    p->n_cols = n_cols;
    p->nnz = nnz;
    p->mrhs_units_per_ticket = 1;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        (void)cudaGetLastError();
        delete p;
        return DDF_ERR_CUDA;
    }
    (void)cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    init_pool_once(p->device);
    st = ddf_alloc(&p->status, 1, s);
    if (!st) st = ddf_alloc(&p->ticket, 2, s);
    if (!st && (cudaMemsetAsync(p->status, 0, sizeof(int32_t), s) != cudaSuccess ||
                cudaMemsetAsync(p->ticket, 0, 2 * sizeof(uint32_t), s) != cudaSuccess)) {
        (void)cudaGetLastError();
        st = DDF_ERR_CUDA;
    }
    if (st) {
        release(p);
        delete p;
        return st;
    }
    *out = p;
    return DDF_OK;
}

// Inspect device CSR arrays the plan takes over (rp, ci and, when present, v);
// on error everything is released and *out stays NULL.
ddf_status ddf_finish_plan(ddf_plan_s* p, int32_t* rp, int32_t* ci, double* v, cudaStream_t s, ddf_plan_t* out,
                           bool borrowed) {
    const ddf_kind kind = p->kind;
    ddf_status st = DDF_OK;
    if (kind == DDF_SPMV) {
        // The pattern is inspected first; the plan's own value array is then
        // filled from v in the executor's layout (tiles point-major).  Without
        // values it is reserved for ddf_update_values.
        st = ddf_build_plan(p, rp, ci, nullptr, s);
        p->val = nullptr;
        if (!st) st = ddf_alloc(&p->val, p->nnz, s);
        if (!st && v != nullptr) st = ddf_gather_values(p, v, s);
        // on success the plan adopted rp / ci as its own arrays; v is released
        // unless it is borrowed (the caller's device values)
        if (st) {
            p->starts = nullptr;
            p->col = nullptr;
            ddf_free(rp, s);
            ddf_free(ci, s);
        }
        if (!borrowed) ddf_free(v, s);
    } else {
        st = ddf_build_plan(p, rp, ci, v, s);
        // SpTRSV keeps rowptr (as orig_rowptr) and drops the CSR copies
        if (p->orig_rowptr != rp) ddf_free(rp, s);
        if (!borrowed) {
            ddf_free(ci, s);
            ddf_free(v, s);
        }
    }
    if (!st) st = ddf_make_lowp(p, s);
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (st) {
        release(p);
        (void)cudaStreamSynchronize(s);
        (void)cudaGetLastError();
        delete p;
        return st;
    }
    *out = p;
    return DDF_OK;
}

extern "C" {

void ddf_opts_default(ddf_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->window_t = 256;
    o->allowed_types = DDF_ALLOW_ALL;
    o->w_op = 8;
    o->w_codelet = 32;
    o->w_index = 4;
    o->spin_cap_ns = 2000000000ll;
    o->unit_nnz = 256;
    o->coarsen_rows = DDF_COARSEN_DEFAULT_ROWS;
}

const char* ddf_status_string(ddf_status st) {
    switch (st) {
        case DDF_OK: return "ok";
        case DDF_ERR_ARG: return "invalid argument";
        case DDF_ERR_NOT_SQUARE: return "matrix is not square";
        case DDF_ERR_UNSORTED: return "rowptr not monotone or columns not strictly increasing";
        case DDF_ERR_OUT_OF_RANGE: return "column index out of range";
        case DDF_ERR_NOT_LOWER: return "entry above the diagonal";
        case DDF_ERR_MISSING_DIAG: return "diagonal entry missing or not last in its row";
        case DDF_ERR_ZERO_DIAG: return "zero diagonal entry";
        case DDF_ERR_WRONG_KIND: return "plan kind does not match the call";
        case DDF_ERR_OOM: return "device out of memory";
        case DDF_ERR_CUDA: return "CUDA runtime error";
        case DDF_ERR_TIMEOUT: return "dependency wait timed out";
        case DDF_ERR_NOT_CONVERGED: return "not converged";
        case DDF_ERR_TOO_LARGE: return "size beyond the supported maximum";
    }
    return "unknown status";
}

ddf_status ddf_inspect(const ddf_csr* A, ddf_kind kind, const ddf_opts* o, ddf_stream_t stream,
                       ddf_plan_t* out) {
    ddf_nvtx_range nvtx_("ddf_inspect");
    if (!out) return DDF_ERR_ARG;
    *out = nullptr;
    if (!A || (kind != DDF_SPMV && kind != DDF_SPTRSV)) return DDF_ERR_ARG;
    if (A->n_rows < 0 || A->n_cols < 0 || A->nnz < 0 || A->nnz > 0x7fffffffll) return DDF_ERR_ARG;
    if (!A->rowptr || (A->nnz > 0 && !A->colidx)) return DDF_ERR_ARG;
    if (kind == DDF_SPTRSV && A->n_rows != A->n_cols) return DDF_ERR_NOT_SQUARE;
    {
        ddf_opts opts;
        if (o) opts = *o;
        else ddf_opts_default(&opts);
        ddf_status sto = check_opts(&opts);
        if (sto) return sto;
    }
    if (!A->on_device) {
        // host CSR: cheap structural checks before any device work
        if (A->rowptr[0] != 0 || (int64_t)A->rowptr[A->n_rows] != A->nnz) return DDF_ERR_UNSORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    ddf_plan_s* p = nullptr;
    ddf_status st = ddf_new_plan(kind, o, s, A->n_rows, A->n_cols, A->nnz, &p);
    if (st) return st;
    int32_t* rp = nullptr;
    int32_t* ci = nullptr;
    double* v = nullptr;
    // A SpTRSV plan keeps only rowptr of the input (its columns and values are
    // re-laid in level order), so device-resident columns and values are read
    // in place during inspection instead of being copied first.  A SpMV plan
    // keeps copies of rowptr and the columns; its values are written once, in
    // the executor's layout, from the caller's device array.
    const bool borrow = A->on_device && (kind == DDF_SPTRSV || kind == DDF_SPMV);
    st = stage(&rp, A->rowptr, (int64_t)A->n_rows + 1, A->on_device, s);
    if (borrow && kind == DDF_SPTRSV) {
        ci = const_cast<int32_t*>(A->colidx);
        v = const_cast<double*>(A->values);
    } else if (borrow) {
        if (!st) st = stage(&ci, A->colidx, A->nnz, A->on_device, s);
        v = const_cast<double*>(A->values);
    } else {
        if (!st) st = stage(&ci, A->colidx, A->nnz, A->on_device, s);
        if (!st && A->values) st = stage(&v, A->values, A->nnz, A->on_device, s);
    }
    if (st) {
        ddf_free(rp, s);
        if (!borrow || kind == DDF_SPMV) ddf_free(ci, s);
        if (!borrow) ddf_free(v, s);
        ddf_plan_destroy(p);
        return st;
    }
    return ddf_finish_plan(p, rp, ci, v, s, out, borrow);
}

ddf_status ddf_update_values(ddf_plan_t p, const double* values, int32_t on_device, ddf_stream_t stream) {
    ddf_nvtx_range nvtx_("ddf_update_values");
    if (!p || (!values && p->nnz > 0)) return DDF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double* v = nullptr;
    const double* src = values;
    if (!on_device && p->nnz > 0) {
        ddf_status st = stage(&v, values, p->nnz, 0, s);
        if (st) return st;
        src = v;
    }
    ddf_status st = DDF_OK;
    if (p->kind == DDF_SPTRSV && p->n > 0) {
        int32_t* bad = nullptr;
        st = ddf_alloc(&bad, 1, s);
        if (!st) {
            int32_t hb = 0;
            cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
            const int32_t* re = p->orig_rowend ? p->orig_rowend : p->orig_rowptr + 1;
            k_check_diag<<<ddf_grid(p->n, 256), 256, 0, s>>>(p->n, re, src, bad);
            ddf_count_launch();
            cudaMemcpyAsync(&hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) st = DDF_ERR_CUDA;
            else if (hb) st = DDF_ERR_ZERO_DIAG;
            ddf_free(bad, s);
        }
    }
    if (!st) st = ddf_gather_values(p, src, s);
    if (!st) st = ddf_make_lowp(p, s);
    ddf_free(v, s);
    return st;
}

ddf_status ddf_spmv(ddf_plan_t p, const double* x, double* y, ddf_stream_t stream) {
    ddf_nvtx_range nvtx_("ddf_spmv");
    if (!p) return DDF_ERR_ARG;
    if (p->kind != DDF_SPMV) return DDF_ERR_WRONG_KIND;
    if ((p->n > 0 && !y) || (p->n_cols > 0 && !x) || (p->nnz > 0 && !p->has_values)) return DDF_ERR_ARG;
    if (p->n == 0) {
        p->last_launches = 0;
        return DDF_OK;
    }
    return ddf_launch_spmv(p, x, y, (cudaStream_t)stream);
}

ddf_status ddf_sptrsv(ddf_plan_t p, const double* b, double* x, ddf_stream_t stream) {
    ddf_nvtx_range nvtx_("ddf_sptrsv");
    if (!p) return DDF_ERR_ARG;
    if (p->kind != DDF_SPTRSV) return DDF_ERR_WRONG_KIND;
    if (p->n > 0 && (!b || !x || !p->has_values)) return DDF_ERR_ARG;
    if (p->n > 0 && (const void*)b < (const void*)(x + p->n) && (const void*)x < (const void*)(b + p->n))
        return DDF_ERR_ARG;   // b and x overlap
    if (p->n == 0) {
        p->last_launches = 0;
        return DDF_OK;
    }
    return ddf_launch_sptrsv(p, b, x, (cudaStream_t)stream);
}

ddf_status ddf_spmv_lowp(ddf_plan_t p, const void* x, void* y, ddf_dtype vec_dtype, ddf_stream_t stream) {
    ddf_nvtx_range nvtx_("ddf_spmv_lowp");
    if (!p) return DDF_ERR_ARG;
    if (p->kind != DDF_SPMV) return DDF_ERR_WRONG_KIND;
    if (p->vdtype != DDF_F32 && p->vdtype != DDF_BF16) return DDF_ERR_ARG;
    if (vec_dtype != DDF_F32 && vec_dtype != DDF_BF16) return DDF_ERR_ARG;
    if ((p->n > 0 && !y) || (p->n_cols > 0 && !x) || (p->nnz > 0 && !p->has_values)) return DDF_ERR_ARG;
    if (p->n == 0) {
        p->last_launches = 0;
        return DDF_OK;
    }
    return ddf_launch_spmv_lp(p, x, y, vec_dtype, (cudaStream_t)stream);
}

ddf_status ddf_sptrsv_refine(ddf_plan_t p, const double* b, double* x, double tol, int32_t max_iter,
                             ddf_stream_t stream, int32_t* iters, double* relres) {
    ddf_nvtx_range nvtx_("ddf_sptrsv_refine");
    if (!p) return DDF_ERR_ARG;
    if (p->kind != DDF_SPTRSV) return DDF_ERR_WRONG_KIND;
    if (p->vdtype != DDF_F32 && p->vdtype != DDF_BF16) return DDF_ERR_ARG;
    if (!(tol >= 0.0) || max_iter < 0) return DDF_ERR_ARG;
    if (p->n > 0 && (!b || !x || !p->has_values)) return DDF_ERR_ARG;
    if (p->n > 0 && (const void*)b < (const void*)(x + p->n) && (const void*)x < (const void*)(b + p->n))
        return DDF_ERR_ARG;
    if (p->n == 0) {
        if (iters) *iters = 0;
        if (relres) *relres = 0.0;
        p->last_launches = 0;
        return DDF_OK;
    }
    return ddf_refine(p, b, x, tol, max_iter, (cudaStream_t)stream, iters, relres);
}

ddf_status ddf_get_status(ddf_plan_t p, ddf_stream_t stream) {
    if (!p) return DDF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t h = 0;
    DDF_CUDA_TRY(cudaMemcpyAsync(&h, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DDF_CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(int32_t), s));
    DDF_CUDA_TRY(cudaStreamSynchronize(s));
    return (ddf_status)h;
}

ddf_status ddf_plan_stats(ddf_plan_t p, ddf_plan_stats_t* st) {
    if (!p || !st) return DDF_ERR_ARG;
    if (!p->stats_ready) {
        ddf_status e = ddf_compute_stats(p);
        if (e) return e;
    }
    *st = p->stats;
    return DDF_OK;
}

ddf_status ddf_plan_export(ddf_plan_t p, int64_t* records, int64_t* ncodelets, int32_t* seq,
                           int32_t* part_ptr, int32_t* depth, int64_t* gs) {
    if (!p || !ncodelets || !depth) return DDF_ERR_ARG;
    *ncodelets = p->ncod;
    *depth = p->depth;
    cudaStream_t s = p->stream;
    int32_t n = p->n;
    if (records && p->ncod > 0) {
        std::vector<dcod> h((size_t)p->ncod);
        DDF_CUDA_TRY(cudaMemcpyAsync(h.data(), p->cod, h.size() * sizeof(dcod), cudaMemcpyDeviceToHost, s));
        DDF_CUDA_TRY(cudaStreamSynchronize(s));
        for (size_t i = 0; i < h.size(); ++i) {
            const dcod& c = h[i];
            int64_t* r = records + 12 * i;
            r[0] = c.part;
            r[1] = c.type;
            r[2] = c.q0;
            r[3] = c.m;
            r[4] = c.n;
            r[5] = (c.flags & DC_F_STRIDED) ? 1 : 0;
            r[6] = c.rho;
            r[7] = (c.flags & DC_G_STRIDED) ? 1 : 0;
            r[8] = c.gamma;
            r[9] = c.h0;
            r[10] = c.delta;
            r[11] = c.sigma;
        }
    }
    if (seq && n > 0) {
        if (p->seq) {
            DDF_CUDA_TRY(cudaMemcpyAsync(seq, p->seq, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
        } else {
            for (int32_t i = 0; i < n; ++i) seq[i] = i;
        }
    }
    if (part_ptr) DDF_CUDA_TRY(cudaMemcpyAsync(part_ptr, p->part_ptr, (size_t)(p->depth + 1) * 4,
                                               cudaMemcpyDeviceToHost, s));
    if (gs && n > 0) {
        std::vector<int32_t> h((size_t)n);
        DDF_CUDA_TRY(cudaMemcpyAsync(h.data(), p->starts, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
        DDF_CUDA_TRY(cudaStreamSynchronize(s));
        for (int32_t i = 0; i < n; ++i) gs[i] = h[i];
    }
    DDF_CUDA_TRY(cudaStreamSynchronize(s));
    return DDF_OK;
}

void ddf_plan_destroy(ddf_plan_t p) {
    if (!p) return;
    // the frees are ordered on the plan's stream after the work queued there
    // (work that may still be running), so nothing waits here
    release(p);
    (void)cudaGetLastError();
    delete p;
}

int32_t ddf_last_launches(ddf_plan_t p) { return p ? p->last_launches : 0; }

int64_t ddf_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

ddf_status ddf_debug_fail_alloc(int64_t k) {
    g_alloc_countdown.store(k < 0 ? -1 : k, std::memory_order_relaxed);
    return DDF_OK;
}

ddf_status ddf_debug_set_dependency(ddf_plan_t p, int64_t k, int32_t col) {
    if (!p || p->kind != DDF_SPTRSV || k < 0 || k >= p->npts || col < 0 || col >= p->n) return DDF_ERR_ARG;
    DDF_CUDA_TRY(cudaMemcpyAsync(p->col + k, &col, sizeof(int32_t), cudaMemcpyHostToDevice, p->stream));
    DDF_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return DDF_OK;
}

}  // extern "C"
