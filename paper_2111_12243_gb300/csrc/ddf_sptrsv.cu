// SpTRSV executor: forward substitution L x = b over the level-ordered plan.
//
// Partitions (levels) run in order and the codelets of one level together
// (Sec. IV-A: partitions in sequence, codelets of a partition in parallel),
// without a barrier between levels: every row waits only for the rows it
// reads.  The ready flag of row j is x[j] itself: the call first fills x with
// a NaN pattern that arithmetic never produces, and a row is ready once its
// entry holds anything else.  One 64-bit load therefore both checks the flag
// and fetches the value.
//
// Work units are ordered by level.  The solve is one persistent cooperative
// launch: warp gw of W co-resident warps runs units gw, gw + W, gw + 2W, ...
// in increasing order.  A unit waits only on units of earlier levels, which
// have smaller indices; by induction on the unit index every wait ends,
// because all W warps are resident (cooperative launch) and each runs its
// units in order.  Each wait is still bounded by spin_cap_ns (globaltimer);
// when it runs out the kernel latches DDF_ERR_TIMEOUT in the status word,
// stops waiting anywhere, and completes with NaN in the rows concerned.
//
// The solve is templated on the value type TV and the vector type TX: FP64
// for ddf_sptrsv, and FP32 vectors with FP32 or BF16 values for the
// low-precision solves of ddf_sptrsv_refine (the flag pattern is then the
// 32-bit NaN 0xFFFFFFFF).
#include "ddf_internal.cuh"

namespace {

constexpr int SMAX = 4;   // points per lane held in registers before the dependency reads

// Bit-level view of the vector type: the ready-flag pattern is a NaN that
// arithmetic never produces; a result equal to it is stored as the canonical NaN.
template <typename TX>
struct XBits;
template <>
struct XBits<double> {
    using U = unsigned long long;
    static constexpr U SENT = DDF_SENTINEL;
    static constexpr U CANON = DDF_CANON_NAN;
    static __device__ __forceinline__ U ld(const void* p) { return ddf_ld_relaxed_u64(p); }
    static __device__ __forceinline__ void st(void* p, U v) { ddf_st_relaxed_u64(p, v); }
    static __device__ __forceinline__ double val(U v) { return __longlong_as_double((long long)v); }
    static __device__ __forceinline__ U bits(double v) { return (U)__double_as_longlong(v); }
};
template <>
struct XBits<float> {
    using U = uint32_t;
    static constexpr U SENT = 0xFFFFFFFFu;
    static constexpr U CANON = 0x7FC00000u;
    static __device__ __forceinline__ U ld(const void* p) { return ddf_ld_relaxed_u32(p); }
    static __device__ __forceinline__ void st(void* p, U v) { ddf_st_relaxed_u32(p, v); }
    static __device__ __forceinline__ float val(U v) { return __uint_as_float(v); }
    static __device__ __forceinline__ U bits(float v) { return __float_as_uint(v); }
};

template <typename U>
__global__ void k_fill(U* __restrict__ x, int64_t n, U pattern, uint32_t* __restrict__ ticket) {
    int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) {
        ticket[0] = 0u;   // work ticket
        ticket[1] = 0u;   // abort flag of this call
    }
    for (int64_t i = i0; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = pattern;
}

// Bounded wait for x[j]: a few immediate polls, then exponential backoff
// (32 ns doubling to 128 ns) so that waiting warps do not flood L2.
template <typename TX>
__device__ __noinline__ TX wait_x(const TX* p, int32_t* status, uint32_t* abort_flag, int64_t cap_ns) {
    using B = XBits<TX>;
    uint64_t t0 = ddf_globaltimer();
    uint32_t it = 0, ns = 32;
    while (true) {
        typename B::U v = B::ld(p);
        if (v != B::SENT) return B::val(v);
        ++it;
        if (it > 32) {
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

// Read x[j] once it is ready (plain relaxed load first, bounded wait after).
template <typename TX>
__device__ __forceinline__ TX dep(const TX* x, int32_t j, int32_t* status, uint32_t* abort_flag, int64_t cap_ns) {
    using B = XBits<TX>;
    typename B::U v = B::ld(x + j);
    if (v != B::SENT) return B::val(v);
    return wait_x<TX>(x + j, status, abort_flag, cap_ns);
}

// One warp per work unit; a unit is the rows one warp pass covers (32 / v
// rows, v lanes per row).  Everything that does not depend on x (descriptor,
// row index, values, columns, b, 1/L_ii) is loaded before the first
// dependency is read, and the reads of all dependencies of a lane are issued
// together, so a unit waiting on an earlier level only pays the flag hop.
template <typename TV, typename TX>
__global__ void __launch_bounds__(DDF_CTA_THREADS, 4)
k_sptrsv(const dcod* __restrict__ cod, const dunit* __restrict__ units, int64_t nunits,
         const int32_t* __restrict__ seq, const int32_t* __restrict__ st, const int32_t* __restrict__ col,
         const TV* __restrict__ val, const TX* __restrict__ dinv, const TX* __restrict__ b, TX* x,
         uint32_t* ticket, int32_t* status, int64_t cap_ns) {
    using B = XBits<TX>;
    uint32_t* abort_flag = ticket + 1;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nunits; u += nw) {
        const dunit U = units[u];
        const dcod C = cod[U.cod];
        const int v = U.v;
        const int lg = __ffs(v) - 1;
        const int rpw = 32 >> lg;
        const int sub = lane >> lg;
        const int li = lane & (v - 1);
        for (int32_t ib = U.i0b; ib < U.i0e; ib += rpw) {
            const int32_t i0 = ib + sub;
            const bool act = i0 < U.i0e;
            const int32_t q = C.q0 + i0;
            int32_t r = 0, kb = 0, L = 0, hb = 0;
            TX bv = 0, di = 0;
            TX vv[SMAX];
            int32_t jj[SMAX];
#pragma unroll
            for (int k = 0; k < SMAX; ++k) {
                vv[k] = 0;
                jj[k] = -1;
            }
            if (act) {
                r = (C.flags & DC_F_STRIDED) ? C.f0 + C.rho * i0 : seq[q];
                if (C.type == DDF_PSC2) {
                    kb = st[q];
                    L = st[q + 1] - kb;
                } else {
                    kb = C.g0 + C.gamma * i0;
                    L = C.n;
                }
                hb = C.h0 + C.delta * i0;
                bv = b[r];
                di = dinv[q];
#pragma unroll
                for (int k = 0; k < SMAX; ++k) {
                    const int32_t i1 = li + k * v;
                    if (i1 < L) {
                        vv[k] = ddf_cvt<TX>(val[kb + i1]);
                        jj[k] = (C.type == DDF_BLAS)   ? hb + C.sigma * i1
                                : (C.type == DDF_PSC1) ? hb + (col[C.sref + i1] - C.h0)
                                                       : col[kb + i1];
                    }
                }
            }
            TX acc = 0;
            // Read the dependencies held in registers; while some are not
            // ready, one lane of the warp waits on its first missing value and
            // the others re-read after it arrives, so a waiting warp costs one
            // poller instead of one per lane.
            typename B::U xv[SMAX];
#pragma unroll
            for (int k = 0; k < SMAX; ++k) xv[k] = jj[k] >= 0 ? B::ld(x + jj[k]) : (typename B::U)0;
            while (true) {
                int miss = -1;
#pragma unroll
                for (int k = SMAX - 1; k >= 0; --k)
                    if (jj[k] >= 0 && xv[k] == B::SENT) miss = k;
                const unsigned pending = __ballot_sync(0xffffffffu, miss >= 0);
                if (!pending) break;
                if (lane == __ffs(pending) - 1) {
                    TX w = wait_x<TX>(x + jj[miss], status, abort_flag, cap_ns);
                    xv[miss] = B::bits(w) == B::SENT ? B::CANON : B::bits(w);
                }
                __syncwarp();
                if (ddf_ld_relaxed_s32(abort_flag) != 0) {
#pragma unroll
                    for (int k = 0; k < SMAX; ++k)
                        if (jj[k] >= 0 && xv[k] == B::SENT) xv[k] = B::CANON;
                } else {
#pragma unroll
                    for (int k = 0; k < SMAX; ++k)
                        if (jj[k] >= 0 && xv[k] == B::SENT) xv[k] = B::ld(x + jj[k]);
                }
            }
            if (act) {
#pragma unroll
                for (int k = 0; k < SMAX; ++k)
                    if (jj[k] >= 0) acc += vv[k] * B::val(xv[k]);
                for (int32_t i1 = li + SMAX * v; i1 < L; i1 += v) {
                    const int32_t j = (C.type == DDF_BLAS)   ? hb + C.sigma * i1
                                      : (C.type == DDF_PSC1) ? hb + (col[C.sref + i1] - C.h0)
                                                             : col[kb + i1];
                    acc += ddf_cvt<TX>(val[kb + i1]) * dep<TX>(x, j, status, abort_flag, cap_ns);
                }
            }
            for (int o = v >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (act && li == 0) {
                TX xr = (bv - acc) * di;
                typename B::U bits = B::bits(xr);
                if (bits == B::SENT) bits = B::CANON;
                B::st(x + r, bits);
            }
        }
    }
}

template <typename TV, typename TX>
ddf_status launch_solve(ddf_plan_s* p, const TV* val, const TX* dinv, const TX* b, TX* x, cudaStream_t s) {
    using B = XBits<TX>;
    int64_t n = p->n;
    int sm = p->sm_count > 0 ? p->sm_count : 152;
    k_fill<typename B::U><<<ddf_grid(n > 0 ? n : 1, 256, (unsigned)sm * 8), 256, 0, s>>>(
        (typename B::U*)x, n, B::SENT, p->ticket);
    ddf_count_launch();
    int launches = 1;
    int64_t nu = p->nunits[0];
    if (nu > 0) {
        int per_sm = 0;
        DDF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sptrsv<TV, TX>, DDF_CTA_THREADS, 0));
        if (per_sm < 1) per_sm = 1;
        int64_t ctas = (nu + DDF_WARPS_PER_CTA - 1) / DDF_WARPS_PER_CTA;
        if (ctas > (int64_t)per_sm * sm) ctas = (int64_t)per_sm * sm;
        const dcod* a_cod = p->cod;
        const dunit* a_units = p->units[0];
        const int32_t* a_seq = p->seq;
        const int32_t* a_st = p->starts;
        const int32_t* a_col = p->col;
        uint32_t* a_ticket = p->ticket;
        int32_t* a_status = p->status;
        int64_t a_cap = p->opts.spin_cap_ns;
        void* args[] = {(void*)&a_cod, (void*)&a_units, (void*)&nu, (void*)&a_seq, (void*)&a_st, (void*)&a_col,
                        (void*)&val, (void*)&dinv, (void*)&b, (void*)&x, (void*)&a_ticket, (void*)&a_status,
                        (void*)&a_cap};
        DDF_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_sptrsv<TV, TX>, dim3((unsigned)ctas),
                                                 dim3(DDF_CTA_THREADS), args, 0, s));
        ddf_count_launch();
        ++launches;
    }
    p->last_launches = launches;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

}  // namespace

ddf_status ddf_launch_sptrsv(ddf_plan_s* p, const double* b, double* x, cudaStream_t s) {
    return launch_solve<double, double>(p, p->val, p->dinv, b, x, s);
}

// Low-precision solve of a refinement step: FP32 vectors, FP32 or BF16 values.
ddf_status ddf_launch_sptrsv_lp(ddf_plan_s* p, const float* b, float* x, cudaStream_t s) {
    if (p->vdtype == DDF_F32) return launch_solve<float, float>(p, (const float*)p->val_lp, p->dinv_lp, b, x, s);
    if (p->vdtype == DDF_BF16)
        return launch_solve<__nv_bfloat16, float>(p, (const __nv_bfloat16*)p->val_lp, p->dinv_lp, b, x, s);
    return DDF_ERR_ARG;
}
