// Batched and multi-RHS execution.
//
// A batch of independent matrices is inspected as one block-diagonal matrix:
// its partitions and codelets are those of Alg. 1 on that matrix, so every
// level of a batched SpTRSV holds the rows of all matrices at that level.
//
// The multi-RHS executors run the same codelets with a different lane map:
// one warp runs one row at a time and lane k owns right-hand side k, so
// every lane does one multiply-add per point and no reduction is needed.
// A row's points are read 32 at a time (lane t loads point t's value and
// column) and broadcast with shuffles; the right-hand sides of one column are
// contiguous, so a warp reads them with one coalesced access.
#include <vector>

#include "ddf_internal.cuh"

namespace {

constexpr int NRHS_MAX = 32;

__global__ void k_add_offset(int32_t* __restrict__ a, int64_t n, int32_t add) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] += add;
}

template <typename TX>
struct RB;
template <>
struct RB<double> {
    using U = unsigned long long;
    static constexpr U SENT = DDF_SENTINEL;
    static constexpr U CANON = DDF_CANON_NAN;
    static __device__ __forceinline__ U ld(const void* p) { return ddf_ld_relaxed_u64(p); }
    static __device__ __forceinline__ void st(void* p, U v) { ddf_st_relaxed_u64(p, v); }
    static __device__ __forceinline__ double val(U v) { return __longlong_as_double((long long)v); }
    static __device__ __forceinline__ U bits(double v) { return (U)__double_as_longlong(v); }
};
template <>
struct RB<float> {
    using U = uint32_t;
    static constexpr U SENT = 0xFFFFFFFFu;
    static constexpr U CANON = 0x7FC00000u;
    static __device__ __forceinline__ U ld(const void* p) { return ddf_ld_relaxed_u32(p); }
    static __device__ __forceinline__ void st(void* p, U v) { ddf_st_relaxed_u32(p, v); }
    static __device__ __forceinline__ float val(U v) { return __uint_as_float(v); }
    static __device__ __forceinline__ U bits(float v) { return __float_as_uint(v); }
};

// Column of point i1 of row i0 of codelet C (the three access functions of h).
__device__ __forceinline__ int32_t point_col(const dcod& C, const int32_t* __restrict__ col, int32_t i0,
                                             int32_t kb, int32_t i1) {
    const int32_t hb = C.h0 + C.delta * i0;
    if (C.type == DDF_BLAS) return hb + C.sigma * i1;
    if (C.type == DDF_PSC1) return hb + (col[C.sref + i1] - C.h0);
    return col[kb + i1];
}

// y_r[k] = sum over the row's points of a * x_col[k], k = lane < nrhs.
// Point i1's value is val[kb + i1 * vs] (vs > 1 for rows of SpMV value tiles).
template <typename TV, typename TX>
__device__ __forceinline__ TX row_mrhs(const dcod& C, int32_t i0, const int32_t* __restrict__ st,
                                      const int32_t* __restrict__ col, const TV* __restrict__ val,
                                      const TX* __restrict__ X, int32_t nrhs, int lane, int32_t vs = 1,
                                      int32_t vb = -1) {
    const int32_t q = C.q0 + i0;
    int32_t kb, L;
    if (C.type == DDF_PSC2) {
        kb = st[q];
        L = st[q + 1] - kb;
    } else {
        kb = vb >= 0 ? vb : C.g0 + C.gamma * i0;
        L = C.n;
    }
    TX acc = 0;
    for (int32_t p0 = 0; p0 < L; p0 += 32) {
        const int32_t i1 = p0 + lane;
        TX pv = 0;
        int32_t pj = 0;
        if (i1 < L) {
            pv = ddf_cvt<TX>(__ldcs(val + kb + (int64_t)i1 * vs));
            pj = point_col(C, col, i0, kb, i1);
        }
        const int32_t cnt = min(32, L - p0);
#pragma unroll 8
        for (int32_t t = 0; t < cnt; ++t) {
            const TX a = __shfl_sync(0xffffffffu, pv, t);
            const int32_t j = __shfl_sync(0xffffffffu, pj, t);
            if (lane < nrhs) acc += a * __ldg(X + (int64_t)j * nrhs + lane);
        }
    }
    return acc;
}

template <typename TV, typename TX>
__global__ void __launch_bounds__(DDF_CTA_THREADS)
k_spmm(const dcod* __restrict__ cod, const dunit* __restrict__ units, int64_t nunits,
       const int32_t* __restrict__ st, const int32_t* __restrict__ col, const TV* __restrict__ val,
       const TX* __restrict__ X, TX* __restrict__ Y, int32_t nrhs) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nunits; u += nw) {
        const dunit U = units[u];
        const int32_t c0 = U.cod;
        const int32_t ncods = U.i0b < 0 ? -U.i0b : 1;
        for (int32_t c = 0; c < ncods; ++c) {
            const dcod C = cod[c0 + c];
            const int32_t b0 = U.i0b < 0 ? 0 : U.i0b;
            const int32_t e0 = U.i0b < 0 ? C.m : U.i0e;
            for (int32_t i0 = b0; i0 < e0; ++i0) {
                const TX acc = row_mrhs<TV, TX>(C, i0, st, col, val, X, nrhs, lane);
                if (lane < nrhs) Y[(int64_t)(C.f0 + C.rho * i0) * nrhs + lane] = acc;
            }
        }
    }
}

// Rows of SpMV value tiles (point-major values), one warp per tile.
template <typename TV, typename TX>
__global__ void __launch_bounds__(DDF_CTA_THREADS)
k_spmm_tile(const dcod* __restrict__ cod, const dtile* __restrict__ tiles, int64_t ntiles,
            const int32_t* __restrict__ st, const int32_t* __restrict__ col, const TV* __restrict__ val,
            const TX* __restrict__ X, TX* __restrict__ Y, int32_t nrhs) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nw) {
        const dtile T = tiles[t];
        const int32_t w = (int32_t)(T.meta & 7u) + 1;
        for (int32_t r = 0; r < w; ++r) {
            const dcod C = cod[T.cod + (int32_t)((T.meta >> (3 + 3 * r)) & 7u)];
            const int32_t i0 = T.q + r - C.q0;
            const TX acc = row_mrhs<TV, TX>(C, i0, st, col, val, X, nrhs, lane, w, T.vb + r);
            if (lane < nrhs) Y[(int64_t)(C.f0 + C.rho * i0) * nrhs + lane] = acc;
        }
    }
}

template <typename U>
__global__ void k_fill_m(U* __restrict__ x, int64_t n, U pattern, uint32_t* __restrict__ ticket) {
    int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) {
        ticket[0] = 0u;
        ticket[1] = 0u;
    }
    for (int64_t i = i0; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = pattern;
}

template <typename TX>
__device__ __noinline__ TX wait_m(const TX* p, int32_t* status, uint32_t* abort_flag, int64_t cap_ns) {
    using B = RB<TX>;
    uint64_t t0 = ddf_globaltimer();
    uint32_t it = 0, ns = 32;
    while (true) {
        typename B::U v = B::ld(p);
        if (v != B::SENT) return B::val(v);
        ++it;
        if (it > 16) {
            __nanosleep(ns);
            ns = min(ns * 2, 128u);
        }
        if ((it & 15u) == 0) {
            if (ddf_ld_relaxed_s32(abort_flag) != 0) return B::val(B::CANON);
            if ((int64_t)(ddf_globaltimer() - t0) > cap_ns) {
                ddf_set_status(status, DDF_ERR_TIMEOUT);
                atomicExch(abort_flag, 1u);
                return B::val(B::CANON);
            }
        }
    }
}

constexpr int SM_E = 8;   // points of a row whose loads are in flight together

// Multi-RHS forward substitution over the level-ordered plan.  Each CTA
// takes the next chunk of upc work units from the ticket when it starts, so
// every unit it waits on belongs to a CTA that already runs (no co-residency
// needed, hence no cooperative launch).  Row x[r][k] is ready once it no
// longer holds the fill pattern; lane k waits on its own element, and the
// lanes of a warp read one row of X with one coalesced access.
template <typename TV, typename TX>
__global__ void __launch_bounds__(DDF_CTA_THREADS)
k_sptrsm(const dcod* __restrict__ cod, const dunit* __restrict__ units, int64_t nunits, int32_t upc,
         const int32_t* __restrict__ seq, const int32_t* __restrict__ st, const int32_t* __restrict__ col,
         const TV* __restrict__ val, const TX* __restrict__ dinv, const TX* __restrict__ B, TX* X, int32_t nrhs,
         uint32_t* ticket, int32_t* status, int64_t cap_ns) {
    using RBx = RB<TX>;
    __shared__ uint32_t chunk;
    if (threadIdx.x == 0) chunk = atomicAdd(ticket, 1u);
    __syncthreads();
    uint32_t* abort_flag = ticket + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t ub = (int64_t)chunk * upc;
    const int64_t ue = min(ub + (int64_t)upc, nunits);
    for (int64_t u = ub + w; u < ue; u += DDF_WARPS_PER_CTA) {
        const dunit U = units[u];
        const dcod C = cod[U.cod];
        for (int32_t i0 = U.i0b; i0 < U.i0e; ++i0) {
            const int32_t q = C.q0 + i0;
            const int32_t r = (C.flags & DC_F_STRIDED) ? C.f0 + C.rho * i0 : seq[q];
            int32_t kb, L;
            if (C.type == DDF_PSC2) {
                kb = st[q];
                L = st[q + 1] - kb;
            } else {
                kb = C.g0 + C.gamma * i0;
                L = C.n;
            }
            const TX bv = lane < nrhs ? B[(int64_t)r * nrhs + lane] : (TX)0;
            const TX di = dinv[q];
            TX acc = 0;
            for (int32_t p0 = 0; p0 < L; p0 += 32) {
                const int32_t i1 = p0 + lane;
                TX pv = 0;
                int32_t pj = 0;
                if (i1 < L) {
                    pv = ddf_cvt<TX>(val[kb + i1]);
                    pj = point_col(C, col, i0, kb, i1);
                }
                const int32_t cnt = min(32, L - p0);
                // the loads of up to SM_E points are issued before any is checked,
                // so one L2 round trip covers them
                for (int32_t t0 = 0; t0 < cnt; t0 += SM_E) {
                    typename RBx::U xv[SM_E];
                    TX av[SM_E];
                    int32_t jv[SM_E];
#pragma unroll
                    for (int e = 0; e < SM_E; ++e) {
                        const int32_t t = min(t0 + e, cnt - 1);
                        av[e] = __shfl_sync(0xffffffffu, pv, t);
                        jv[e] = __shfl_sync(0xffffffffu, pj, t);
                        xv[e] = (lane < nrhs && t0 + e < cnt) ? RBx::ld(X + (int64_t)jv[e] * nrhs + lane)
                                                             : (typename RBx::U)0;
                    }
                    if (lane < nrhs) {
#pragma unroll
                        for (int e = 0; e < SM_E; ++e) {
                            if (t0 + e >= cnt) break;
                            const TX xj = (xv[e] != RBx::SENT)
                                              ? RBx::val(xv[e])
                                              : wait_m<TX>(X + (int64_t)jv[e] * nrhs + lane, status, abort_flag, cap_ns);
                            acc += av[e] * xj;
                        }
                    }
                }
            }
            if (lane < nrhs) {
                const TX xr = (bv - acc) * di;
                typename RBx::U bits = RBx::bits(xr);
                if (bits == RBx::SENT) bits = RBx::CANON;
                RBx::st(X + (int64_t)r * nrhs + lane, bits);
            }
        }
    }
}

unsigned grid_units(int64_t nunits, int sm) {
    int64_t ctas = (nunits + DDF_WARPS_PER_CTA - 1) / DDF_WARPS_PER_CTA;
    int64_t cap = (int64_t)sm * 32;
    return (unsigned)std::max<int64_t>(1, std::min(ctas, cap));
}

template <typename TV, typename TX>
ddf_status launch_spmm(ddf_plan_s* p, const TV* val, const TX* X, TX* Y, int32_t nrhs, cudaStream_t s) {
    const int sm = p->sm_count > 0 ? p->sm_count : 152;
    int launches = 0;
    for (int t = 0; t < 3; ++t) {
        if (p->nunits[t] <= 0) continue;
        k_spmm<TV, TX><<<grid_units(p->nunits[t], sm), DDF_CTA_THREADS, 0, s>>>(
            p->cod, p->units[t], p->nunits[t], p->starts, p->col, val, X, Y, nrhs);
        ddf_count_launch();
        ++launches;
    }
    for (int t = 0; t < 2; ++t) {
        if (p->ntiles[t] <= 0) continue;
        k_spmm_tile<TV, TX><<<grid_units(p->ntiles[t], sm), DDF_CTA_THREADS, 0, s>>>(
            p->cod, p->tiles[t], p->ntiles[t], p->starts, p->col, val, X, Y, nrhs);
        ddf_count_launch();
        ++launches;
    }
    p->last_launches = launches;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

template <typename TV, typename TX>
ddf_status launch_sptrsm(ddf_plan_s* p, const TV* val, const TX* dinv, const TX* B, TX* X, int32_t nrhs,
                         cudaStream_t s) {
    using RBx = RB<TX>;
    const int sm = p->sm_count > 0 ? p->sm_count : 152;
    const int64_t ne = (int64_t)p->n * nrhs;
    k_fill_m<typename RBx::U><<<ddf_grid(ne > 0 ? ne : 1, 256, (unsigned)sm * 8), 256, 0, s>>>(
        (typename RBx::U*)X, ne, RBx::SENT, p->ticket);
    ddf_count_launch();
    int launches = 1;
    const int64_t nu = p->nunits[0];
    if (nu > 0) {
        const int32_t upc = p->units_per_cta > 0 ? p->units_per_cta : DDF_WARPS_PER_CTA;
        const int64_t ctas = (nu + upc - 1) / upc;
        k_sptrsm<TV, TX><<<(unsigned)ctas, DDF_CTA_THREADS, 0, s>>>(p->cod, p->units[0], nu, upc, p->seq,
                                                                    p->starts, p->col, val, dinv, B, X, nrhs,
                                                                    p->ticket, p->status, p->opts.spin_cap_ns);
        ddf_count_launch();
        ++launches;
    }
    p->last_launches = launches;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

ddf_status run_multi(ddf_plan_s* p, const void* in, void* out, int32_t nrhs, ddf_dtype dtype, cudaStream_t s) {
    if (p->kind == DDF_SPMV) {
        if (dtype == DDF_F64) return launch_spmm<double, double>(p, p->val, (const double*)in, (double*)out, nrhs, s);
        return launch_spmm<float, float>(p, (const float*)p->val_lp, (const float*)in, (float*)out, nrhs, s);
    }
    if (dtype == DDF_F64)
        return launch_sptrsm<double, double>(p, p->val, p->dinv, (const double*)in, (double*)out, nrhs, s);
    return launch_sptrsm<float, float>(p, (const float*)p->val_lp, p->dinv_lp, (const float*)in, (float*)out, nrhs,
                                       s);
}

ddf_status check_multi(ddf_plan_s* p, const void* in, void* out, int32_t nrhs, ddf_dtype dtype) {
    if (!p) return DDF_ERR_ARG;
    if (nrhs < 1 || nrhs > NRHS_MAX) return DDF_ERR_ARG;
    if (dtype != DDF_F64 && dtype != DDF_F32) return DDF_ERR_ARG;
    if (dtype == DDF_F32 && p->vdtype != DDF_F32) return DDF_ERR_ARG;
    if (p->nnz > 0 && !p->has_values) return DDF_ERR_ARG;
    if ((p->n > 0 || p->n_cols > 0) && (!in || !out)) return DDF_ERR_ARG;
    return DDF_OK;
}

}  // namespace

extern "C" {

ddf_status ddf_inspect_batch(const ddf_csr* mats, int32_t count, ddf_kind kind, const ddf_opts* o,
                             ddf_stream_t stream, ddf_plan_t* out) {
    ddf_nvtx_range nvtx_("ddf_inspect_batch");
    if (!out) return DDF_ERR_ARG;
    *out = nullptr;
    if (!mats || count < 1 || (kind != DDF_SPMV && kind != DDF_SPTRSV)) return DDF_ERR_ARG;
    {
        ddf_opts opts;
        if (o) opts = *o;
        else ddf_opts_default(&opts);
        if (opts.window_t < 1 || opts.window_t > DDF_MAX_T || !(opts.allowed_types & DDF_ALLOW_PSC2) ||
            (opts.allowed_types & ~DDF_ALLOW_ALL))
            return DDF_ERR_ARG;
    }
    int64_t N = 0, NC = 0, NNZ = 0;
    bool vals = mats[0].values != nullptr;
    for (int32_t i = 0; i < count; ++i) {
        const ddf_csr& A = mats[i];
        if (A.n_rows < 0 || A.n_cols < 0 || A.nnz < 0 || !A.rowptr || (A.nnz > 0 && !A.colidx)) return DDF_ERR_ARG;
        if (kind == DDF_SPTRSV && A.n_rows != A.n_cols) return DDF_ERR_NOT_SQUARE;
        if ((A.values != nullptr) != vals) return DDF_ERR_ARG;   // values for all matrices or for none
        if (!A.on_device && (A.rowptr[0] != 0 || (int64_t)A.rowptr[A.n_rows] != A.nnz)) return DDF_ERR_UNSORTED;
        N += A.n_rows;
        NC += A.n_cols;
        NNZ += A.nnz;
    }
    if (N > 0x7fffffffll - 1 || NC > 0x7fffffffll || NNZ > 0x7fffffffll) return DDF_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    ddf_plan_s* p = nullptr;
    ddf_status st = ddf_new_plan(kind, o, s, (int32_t)N, (int32_t)NC, NNZ, &p);
    if (st) return st;
    int32_t* rp = nullptr;
    int32_t* ci = nullptr;
    double* v = nullptr;
    st = ddf_alloc(&rp, N + 1, s);
    if (!st) st = ddf_alloc(&ci, NNZ, s);
    if (!st && vals) st = ddf_alloc(&v, NNZ, s);
    const int sm = p->sm_count > 0 ? p->sm_count : 152;
    int64_t r0 = 0, c0 = 0, z0 = 0;
    for (int32_t i = 0; i < count && !st; ++i) {
        const ddf_csr& A = mats[i];
        const cudaMemcpyKind k = A.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        // rowptr of matrix i (its last entry equals the next matrix's first once offset)
        if (cudaMemcpyAsync(rp + r0, A.rowptr, sizeof(int32_t) * ((size_t)A.n_rows + 1), k, s) != cudaSuccess)
            st = DDF_ERR_CUDA;
        if (!st && A.nnz > 0 &&
            cudaMemcpyAsync(ci + z0, A.colidx, sizeof(int32_t) * (size_t)A.nnz, k, s) != cudaSuccess)
            st = DDF_ERR_CUDA;
        if (!st && vals && A.nnz > 0 &&
            cudaMemcpyAsync(v + z0, A.values, sizeof(double) * (size_t)A.nnz, k, s) != cudaSuccess)
            st = DDF_ERR_CUDA;
        if (!st && z0 > 0) {
            k_add_offset<<<ddf_grid((int64_t)A.n_rows + 1, 256, (unsigned)sm * 4), 256, 0, s>>>(
                rp + r0, (int64_t)A.n_rows + 1, (int32_t)z0);
            ddf_count_launch();
        }
        if (!st && c0 > 0 && A.nnz > 0) {
            k_add_offset<<<ddf_grid(A.nnz, 256, (unsigned)sm * 4), 256, 0, s>>>(ci + z0, A.nnz, (int32_t)c0);
            ddf_count_launch();
        }
        r0 += A.n_rows;
        c0 += A.n_cols;
        z0 += A.nnz;
    }
    if (!st && cudaGetLastError() != cudaSuccess) st = DDF_ERR_CUDA;
    if (st) {
        (void)cudaGetLastError();
        ddf_free(rp, s);
        ddf_free(ci, s);
        ddf_free(v, s);
        ddf_plan_destroy(p);
        return st;
    }
    return ddf_finish_plan(p, rp, ci, v, s, out);
}

ddf_status ddf_spmm(ddf_plan_t p, const void* X, void* Y, int32_t nrhs, ddf_dtype dtype, ddf_stream_t stream) {
    ddf_nvtx_range nvtx_("ddf_spmm");
    ddf_status st = check_multi(p, X, Y, nrhs, dtype);
    if (st) return st;
    if (p->kind != DDF_SPMV) return DDF_ERR_WRONG_KIND;
    if (p->n == 0) {
        p->last_launches = 0;
        return DDF_OK;
    }
    return run_multi(p, X, Y, nrhs, dtype, (cudaStream_t)stream);
}

ddf_status ddf_sptrsm(ddf_plan_t p, const void* B, void* X, int32_t nrhs, ddf_dtype dtype, ddf_stream_t stream) {
    ddf_nvtx_range nvtx_("ddf_sptrsm");
    ddf_status st = check_multi(p, B, X, nrhs, dtype);
    if (st) return st;
    if (p->kind != DDF_SPTRSV) return DDF_ERR_WRONG_KIND;
    const size_t bytes = (size_t)p->n * nrhs * (dtype == DDF_F64 ? 8 : 4);
    if (p->n > 0 && (const char*)B < (const char*)X + bytes && (const char*)X < (const char*)B + bytes)
        return DDF_ERR_ARG;
    if (p->n == 0) {
        p->last_launches = 0;
        return DDF_OK;
    }
    return run_multi(p, B, X, nrhs, dtype, (cudaStream_t)stream);
}

ddf_status ddf_tune(ddf_plan_t p, const void* in, void* out, int32_t nrhs, ddf_dtype dtype, ddf_stream_t stream,
                    int32_t* best_unit_nnz) {
    ddf_nvtx_range nvtx_("ddf_tune");
    ddf_status st = check_multi(p, in, out, nrhs, dtype);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    DDF_CUDA_TRY(cudaEventCreate(&e0));
    DDF_CUDA_TRY(cudaEventCreate(&e1));
    // SpMV: tile size of the work units; SpTRSV: work units per CTA ticket
    const int32_t cand_spmv[] = {64, 128, 256, 512, 1024, 2048};
    const int32_t cand_trsv[] = {8, 16, 32, 64};
    const bool spmv = p->kind == DDF_SPMV;
    const int nc = spmv ? 6 : 4;
    float best = 3.0e38f;
    int32_t pick = spmv ? p->opts.unit_nnz : p->units_per_cta;
    for (int c = 0; c < nc && !st; ++c) {
        if (spmv) {
            p->opts.unit_nnz = cand_spmv[c];
            st = ddf_build_units(p, s);
        } else {
            p->units_per_cta = cand_trsv[c];
        }
        if (st) break;
        float ms = 0.0f;
        for (int rep = 0; rep < 3 && !st; ++rep) {     // warm-up, then the fastest of two timed runs
            cudaEventRecord(e0, s);
            st = run_multi(p, in, out, nrhs, dtype, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = DDF_ERR_CUDA;
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep == 1 || (rep == 2 && t < ms)) ms = t;
        }
        if (!st && ms < best) {
            best = ms;
            pick = spmv ? cand_spmv[c] : cand_trsv[c];
        }
    }
    if (spmv) {
        p->opts.unit_nnz = pick;
        if (!st) st = ddf_build_units(p, s);
    } else {
        p->units_per_cta = pick;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!st && cudaStreamSynchronize(s) != cudaSuccess) st = DDF_ERR_CUDA;
    if (best_unit_nnz) *best_unit_nnz = pick;
    return st;
}

}  // extern "C"
