// SpMV executor y = A x: one kernel per codelet type (Sec. IV-B, Listing 3).
//
// A warp runs one work unit (rows [i0b, i0e) of one codelet) with v lanes
// per row (v a power of two): lane li of the row group handles the points
// i1 = li, li + v, ...; the row sum is reduced with xor shuffles inside the
// group and written once.  The three kernels differ only in how they form
// the column h(i0, i1):
//   BLAS   h0 + delta*i0 + sigma*i1          no index loads
//   PSC I  h0 + delta*i0 + s[i1]             s loaded once per unit (first row's columns)
//   PSC II col[g(i0, i1)]                    one index per point, row extents from starts
// Values of BLAS / PSC I codelets sit at g0 + gamma*i0 + i1: consecutive rows
// are contiguous, so a row group's loads are coalesced.
#include "ddf_internal.cuh"

namespace {

constexpr int SMAX = 4;   // s entries kept in registers per lane (n <= 4 v)

template <int TYPE>
__global__ void __launch_bounds__(DDF_CTA_THREADS)
k_spmv(const dcod* __restrict__ cod, const dunit* __restrict__ units, int64_t nunits,
       const int32_t* __restrict__ st, const int32_t* __restrict__ col, const double* __restrict__ val,
       const double* __restrict__ x, double* __restrict__ y) {
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
        int32_t sreg[SMAX];
        if (TYPE == DDF_PSC1) {
#pragma unroll
            for (int k = 0; k < SMAX; ++k) {
                int32_t i1 = li + k * v;
                sreg[k] = (i1 < C.n) ? __ldg(col + C.sref + i1) - C.h0 : 0;
            }
        }
        for (int32_t ib = U.i0b; ib < U.i0e; ib += rpw) {
            const int32_t i0 = ib + sub;
            const bool act = i0 < U.i0e;
            double acc = 0.0;
            int32_t r = 0;
            if (act) {
                r = C.f0 + C.rho * i0;
                if (TYPE == DDF_BLAS) {
                    const double* vp = val + (C.g0 + C.gamma * i0);
                    const int32_t hb = C.h0 + C.delta * i0;
#pragma unroll 8
                    for (int32_t i1 = li; i1 < C.n; i1 += v) acc += __ldcs(vp + i1) * __ldg(x + hb + C.sigma * i1);
                } else if (TYPE == DDF_PSC1) {
                    const double* vp = val + (C.g0 + C.gamma * i0);
                    const int32_t hb = C.h0 + C.delta * i0;
                    if (C.n <= SMAX * v) {
#pragma unroll
                        for (int k = 0; k < SMAX; ++k) {
                            int32_t i1 = li + k * v;
                            if (i1 < C.n) acc += __ldcs(vp + i1) * __ldg(x + hb + sreg[k]);
                        }
                    } else {
                        const int32_t* sp = col + C.sref;
#pragma unroll 8
                        for (int32_t i1 = li; i1 < C.n; i1 += v)
                            acc += __ldcs(vp + i1) * __ldg(x + hb + (__ldg(sp + i1) - C.h0));
                    }
                } else {
                    const int32_t q = C.q0 + i0;
                    const int32_t kb = st[q], ke = st[q + 1];
#pragma unroll 4
                    for (int32_t k = kb + li; k < ke; k += v) acc += __ldcs(val + k) * __ldg(x + __ldcs(col + k));
                }
            }
            for (int o = v >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (act && li == 0) y[r] = acc;
        }
    }
}

unsigned grid_for(int64_t nunits, int sm_count) {
    int64_t ctas = (nunits + DDF_WARPS_PER_CTA - 1) / DDF_WARPS_PER_CTA;
    int64_t cap = (int64_t)sm_count * 32;
    if (ctas > cap) ctas = cap;
    if (ctas < 1) ctas = 1;
    return (unsigned)ctas;
}

}  // namespace

ddf_status ddf_launch_spmv(ddf_plan_s* p, const double* x, double* y, cudaStream_t s) {
    int launches = 0;
    int sm = p->sm_count > 0 ? p->sm_count : 152;
    if (p->nunits[DDF_BLAS] > 0) {
        k_spmv<DDF_BLAS><<<grid_for(p->nunits[0], sm), DDF_CTA_THREADS, 0, s>>>(
            p->cod, p->units[0], p->nunits[0], p->starts, p->col, p->val, x, y);
        ddf_count_launch();
        ++launches;
    }
    if (p->nunits[DDF_PSC1] > 0) {
        k_spmv<DDF_PSC1><<<grid_for(p->nunits[1], sm), DDF_CTA_THREADS, 0, s>>>(
            p->cod, p->units[1], p->nunits[1], p->starts, p->col, p->val, x, y);
        ddf_count_launch();
        ++launches;
    }
    if (p->nunits[DDF_PSC2] > 0) {
        k_spmv<DDF_PSC2><<<grid_for(p->nunits[2], sm), DDF_CTA_THREADS, 0, s>>>(
            p->cod, p->units[2], p->nunits[2], p->starts, p->col, p->val, x, y);
        ddf_count_launch();
        ++launches;
    }
    p->last_launches = launches;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}
