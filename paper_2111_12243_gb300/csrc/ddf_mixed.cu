// Mixed precision: low-precision copies of a plan's values, and SpTRSV with
// iterative refinement (FP32 / BF16 solves, FP64 residual and update).
//
//   x0 = solve_lp(b)                     low precision, FP32 vectors
//   repeat: r = b - L x                  FP64 (values, x, b and the sums)
//           stop when ||r||_2 <= tol ||b||_2
//           d = solve_lp(r);  x += d     correction in low precision, update in FP64
//
// The low-precision solve is the same codelet executor as the FP64 one
// (k_sptrsv instantiated for FP32 vectors), so every refinement step pays the
// dependency chain of the level sets again: the method trades bytes per solve
// for more solves.
#include <math.h>
#include <string.h>

#include "ddf_internal.cuh"

namespace {

template <typename T>
__global__ void k_to_lowp(const double* __restrict__ in, T* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = ddf_from_float<T>((float)in[i]);
}

__global__ void k_d2f(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__device__ __forceinline__ void block_add(double v, double* acc) {
    __shared__ double part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(acc, v);
    }
}

// ||b||^2 and b rounded to FP32 (right-hand side of the first solve)
__global__ void k_rhs(const double* __restrict__ b, float* __restrict__ blp, int64_t n, double* __restrict__ nrm) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[i];
        blp[i] = (float)v;
        s += v * v;
    }
    block_add(s, nrm);
}

// r = b - L x in FP64 over the level-ordered copy: position q holds row
// seq[q], its off-diagonal entries starts[q] .. starts[q+1] and L_qq = diag[q].
// Also ||r||^2 and r rounded to FP32.  A thread sums a row of up to
// RES_LONG off-diagonal entries by itself (one FP64 multiply-add per entry,
// no reduction); longer rows (the power-law matrix has rows of thousands of
// entries) are collected by a ballot and summed by the whole warp, lanes
// striding over the entries.  The sum of squares goes to nrm[1]; thread 0
// also copies the plan's status word into nrm[2], so that one copy returns
// the norms and the solve's status.
constexpr int32_t RES_LONG = 64;

__global__ void k_residual(int32_t n, const int32_t* __restrict__ seq, const int32_t* __restrict__ st,
                           const int32_t* __restrict__ col, const double* __restrict__ val,
                           const double* __restrict__ diag, const double* __restrict__ b,
                           const double* __restrict__ x, double* __restrict__ r, float* __restrict__ rlp,
                           double* __restrict__ nrm, const int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) reinterpret_cast<int32_t*>(nrm + 2)[0] = *status;
    double s2 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the loop runs the same number of times on every lane of a warp
    const int64_t q_end = ((int64_t)n + 31) / 32 * 32;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q_end; q += stride) {
        const bool in = q < n;
        int32_t a = 0, e = 0, row = 0;
        if (in) {
            row = seq[q];
            a = st[q];
            e = st[q + 1];
        }
        const bool lng = in && e - a > RES_LONG;
        double acc = 0.0;
        if (in && !lng) {
            acc = diag[q] * x[row];
            for (int32_t k = a; k < e; ++k) acc += val[k] * x[col[k]];
        }
        // long rows: the warp sums each in turn
        for (unsigned m = __ballot_sync(0xffffffffu, lng); m; m &= m - 1) {
            const int src = __ffs(m) - 1;
            const int32_t la = __shfl_sync(0xffffffffu, a, src), le = __shfl_sync(0xffffffffu, e, src);
            double part = 0.0;
            for (int32_t k = la + lane; k < le; k += 32) part += val[k] * x[col[k]];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == src) acc = diag[q] * x[row] + part;
        }
        if (in) {
            const double rv = b[row] - acc;
            r[row] = rv;
            rlp[row] = (float)rv;
            s2 += rv * rv;
        }
    }
    block_add(s2, nrm + 1);
}

// x = d (first step) or x += d, FP64 update of an FP32 correction
__global__ void k_update(double* __restrict__ x, const float* __restrict__ d, int64_t n, int first) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = first ? (double)d[i] : x[i] + (double)d[i];
}

unsigned gs(int64_t n, int sm) { return ddf_grid(n > 0 ? n : 1, 256, (unsigned)sm * 8); }

}  // namespace

// Build (or refresh, after new values) the low-precision copies of a plan.
ddf_status ddf_make_lowp(ddf_plan_s* p, cudaStream_t s) {
    const int dt = p->opts.store_dtype;
    if (dt == DDF_F64) return DDF_OK;
    const int sm = p->sm_count > 0 ? p->sm_count : 152;
    const int64_t nv = p->kind == DDF_SPMV ? p->nnz : p->npts;
    p->vdtype = dt;
    if (!p->val_lp && nv > 0) {
        ddf_status st = dt == DDF_F32 ? ddf_alloc((float**)&p->val_lp, nv + DDF_TAIL_PAD, s)
                                      : ddf_alloc((__nv_bfloat16**)&p->val_lp, nv + DDF_TAIL_PAD, s);
        if (st) return st;
    }
    if (p->kind == DDF_SPTRSV && p->n > 0) {
        ddf_status st = DDF_OK;
        if (!p->dinv_lp) st = ddf_alloc(&p->dinv_lp, p->n, s);
        if (!st && !p->r64) st = ddf_alloc(&p->r64, p->n, s);
        if (!st && !p->rlp) st = ddf_alloc(&p->rlp, p->n, s);
        if (!st && !p->xlp) st = ddf_alloc(&p->xlp, p->n, s);
        if (!st && !p->nrm) st = ddf_alloc(&p->nrm, 3, s);   // ||b||^2, ||r||^2, status word
        if (st) return st;
    }
    if (!p->has_values) return DDF_OK;
    if (nv > 0) {
        if (dt == DDF_F32) k_to_lowp<float><<<gs(nv, sm), 256, 0, s>>>(p->val, (float*)p->val_lp, nv);
        else k_to_lowp<__nv_bfloat16><<<gs(nv, sm), 256, 0, s>>>(p->val, (__nv_bfloat16*)p->val_lp, nv);
        ddf_count_launch();
    }
    if (p->kind == DDF_SPTRSV && p->n > 0) {
        k_d2f<<<gs(p->n, sm), 256, 0, s>>>(p->dinv, p->dinv_lp, p->n);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

ddf_status ddf_refine(ddf_plan_s* p, const double* b, double* x, double tol, int32_t max_iter, cudaStream_t s,
                      int32_t* iters, double* relres) {
    const int64_t n = p->n;
    const int sm = p->sm_count > 0 ? p->sm_count : 152;
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    int launches = 0;
    DDF_CUDA_TRY(cudaMemsetAsync(p->nrm, 0, 2 * sizeof(double), s));
    k_rhs<<<gs(n, sm), 256, 0, s>>>(b, p->rlp, n, p->nrm);
    ddf_count_launch();
    ++launches;
    ddf_status st = ddf_launch_sptrsv_lp(p, p->rlp, p->xlp, s);
    if (st) return st;
    launches += p->last_launches;
    k_update<<<gs(n, sm), 256, 0, s>>>(x, p->xlp, n, 1);
    ddf_count_launch();
    ++launches;
    double h[3] = {0.0, 0.0, 0.0};
    double nb = 0.0, rel = 0.0;
    int32_t it = 0;
    for (;; ++it) {
        DDF_CUDA_TRY(cudaMemsetAsync(p->nrm + 1, 0, sizeof(double), s));
        k_residual<<<gs(n, sm), 256, 0, s>>>((int32_t)n, p->seq, p->starts, p->col, p->val, p->diag, b, x, p->r64,
                                            p->rlp, p->nrm, p->status);
        ddf_count_launch();
        ++launches;
        // the norms and the solve's status word in one copy, one wait per step
        DDF_CUDA_TRY(cudaMemcpyAsync(h, p->nrm, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        DDF_CUDA_TRY(cudaStreamSynchronize(s));
        int32_t stw = 0;
        memcpy(&stw, &h[2], sizeof(int32_t));
        if (stw) {
            p->last_launches = launches;
            return (ddf_status)stw;
        }
        nb = sqrt(h[0]);
        rel = nb > 0.0 ? sqrt(h[1]) / nb : sqrt(h[1]);
        if (rel <= tol || it >= max_iter) break;
        st = ddf_launch_sptrsv_lp(p, p->rlp, p->xlp, s);
        if (st) return st;
        launches += p->last_launches;
        k_update<<<gs(n, sm), 256, 0, s>>>(x, p->xlp, n, 0);
        ddf_count_launch();
        ++launches;
    }
    DDF_CUDA_TRY(cudaGetLastError());
    p->last_launches = launches;
    if (iters) *iters = it;
    if (relres) *relres = rel;
    return rel <= tol ? DDF_OK : DDF_ERR_NOT_CONVERGED;
}
