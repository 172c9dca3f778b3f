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
// Also ||r||^2 (into nrm[1]) and r rounded to FP32.  The positions are cut
// into groups of 32; a group of T points runs on NT threads (a warp, or the
// whole CTA when T > RES_WARP_MAX), thread t adding the products of the
// points [t K, (t + 1) K), K = ceil(T / NT), row by row with fused
// multiply-adds in point order, four points' loads in flight at a time.  A
// scan over the threads carries the partial sums of rows that cross stretch
// boundaries to the thread where each row ends, so any mix of row lengths
// (the power-law matrix has rows of thousands of entries next to rows of
// one) spreads evenly over the threads, and every sum has a fixed order.
// Thread 0 also copies the plan's status word into nrm[2], so that one copy
// returns the norms and the solve's status.
constexpr int RES_ROWS = 32;
constexpr int RES_WARP_MAX = 2048;
constexpr int RES_THREADS = 256;

struct ResArgs {
    const int32_t* seq;
    const int32_t* st;
    const int32_t* col;
    const double* val;
    const double* diag;
    const double* b;
    const double* x;
    double* r;
    float* rlp;
};

__device__ __forceinline__ void res_finish(const ResArgs& A, int32_t q, double sum, double& s2) {
    const int32_t row = A.seq[q];
    const double rv = A.b[row] - (A.diag[q] * A.x[row] + sum);
    A.r[row] = rv;
    A.rlp[row] = (float)rv;
    s2 += rv * rv;
}

// One group of R positions starting at qa, its points (relative to st[qa])
// bounded by srow[0 .. R]; NT threads, t = this thread's index among them.
// wb / wa: per-warp scan totals (NT > 32 only).
template <int NT>
__device__ __forceinline__ void res_group(const ResArgs& A, int32_t qa, int32_t R, const int32_t* srow, int t,
                                          double* wb, int32_t* wa, double& s2) {
    const int lane = t & 31;
    const int32_t ka = A.st[qa];
    const int32_t T = srow[R];
    if (t < R && srow[t + 1] == srow[t]) res_finish(A, qa + t, 0.0, s2);   // rows without off-diagonals
    const int32_t K = (T + NT - 1) / NT;
    const int32_t e0 = min(t * K, T), e1 = min(e0 + K, T);
    double hp = 0.0, tp = 0.0;
    int32_t hr = 0, tr = 0;
    bool cont = false, single = true;
    if (e0 < e1) {
        int32_t lo = 0, hi = R - 1;   // the row holding point e0: the last row starting at or before it
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (srow[mid] <= e0) lo = mid;
            else hi = mid - 1;
        }
        int32_t rr = lo;
        hr = rr;
        cont = srow[rr] < e0;
        int32_t e = e0;
        while (true) {
            const int32_t end = min(srow[rr + 1], e1);
            double acc = 0.0;
            int32_t k = e;
            for (; k + 4 <= end; k += 4) {
                const int64_t z = (int64_t)ka + k;
                const double v0 = A.val[z], v1 = A.val[z + 1], v2 = A.val[z + 2], v3 = A.val[z + 3];
                const double x0 = A.x[A.col[z]], x1 = A.x[A.col[z + 1]], x2 = A.x[A.col[z + 2]],
                             x3 = A.x[A.col[z + 3]];
                acc = fma(v0, x0, acc);
                acc = fma(v1, x1, acc);
                acc = fma(v2, x2, acc);
                acc = fma(v3, x3, acc);
            }
            for (; k < end; ++k) acc = fma(A.val[(int64_t)ka + k], A.x[A.col[(int64_t)ka + k]], acc);
            if (rr == hr) hp = acc;
            if (end == e1) {
                tr = rr;
                tp = acc;
                break;
            }
            if (rr != hr) res_finish(A, qa + rr, acc, s2);   // a row inside the stretch
            single = false;
            e = end;
            do {
                ++rr;
            } while (srow[rr + 1] == srow[rr]);   // skip rows without points (a later row holds point e)
        }
    }
    // carry_out(t) = tp(t) + [single(t) and cont(t)] carry_out(t - 1): a scan over the threads
    double cb = tp;
    bool ca = single && cont && e0 < e1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double pb = __shfl_up_sync(0xffffffffu, cb, o);
        const bool pa = __shfl_up_sync(0xffffffffu, ca, o);
        if (lane >= o) {
            if (ca) cb += pb;
            ca = ca && pa;
        }
    }
    double cin;
    if constexpr (NT == 32) {
        const double prev = __shfl_up_sync(0xffffffffu, cb, 1);
        cin = (lane > 0 && cont) ? prev : 0.0;
    } else {
        const int w = t >> 5;
        if (lane == 31) {
            wb[w] = cb;
            wa[w] = ca;
        }
        __syncthreads();
        double cw = 0.0;   // carry into this warp, warps combined in index order
        for (int i = 0; i < w; ++i) cw = wb[i] + (wa[i] ? cw : 0.0);
        const double out = cb + (ca ? cw : 0.0);
        const double prev = __shfl_up_sync(0xffffffffu, out, 1);
        cin = cont ? (lane > 0 ? prev : cw) : 0.0;
        __syncthreads();
    }
    if (e0 < e1) {
        if (!single) {
            res_finish(A, qa + hr, hp + cin, s2);   // the head row ended in the stretch
            if (srow[tr + 1] == e1) res_finish(A, qa + tr, tp, s2);
        } else if (srow[hr + 1] == e1) {
            res_finish(A, qa + hr, hp + cin, s2);
        }
    }
}

__global__ void __launch_bounds__(RES_THREADS)
k_residual(int32_t n, ResArgs A, double* __restrict__ nrm, const int32_t* __restrict__ status) {
    constexpr int NWARP = RES_THREADS / 32;
    __shared__ int32_t srow_w[NWARP][RES_ROWS + 1];
    __shared__ int32_t srow_c[RES_ROWS + 1];
    __shared__ int32_t heavy[RES_THREADS];
    __shared__ int32_t nheavy;
    __shared__ double wb[NWARP];
    __shared__ int32_t wa[NWARP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) reinterpret_cast<int32_t*>(nrm + 2)[0] = *status;
    double s2 = 0.0;
    const int64_t ngroups = ((int64_t)n + RES_ROWS - 1) / RES_ROWS;
    auto group_points = [&](int64_t g) {
        const int32_t qa = (int32_t)(g * RES_ROWS);
        const int32_t R = min(RES_ROWS, n - qa);
        return A.st[qa + R] - A.st[qa];
    };
    // groups of more than RES_WARP_MAX points: one CTA each.  This CTA looks
    // at groups blockIdx.x + i gridDim.x, 256 values of i at a time, and runs
    // the heavy ones among them (the long rows of a power-law matrix sit at
    // its deep levels, so heavy groups cluster in level order: the stride
    // spreads them over the CTAs).
    for (int64_t i0 = 0; (int64_t)blockIdx.x + i0 * gridDim.x < ngroups; i0 += RES_THREADS) {
        if (threadIdx.x == 0) nheavy = 0;
        __syncthreads();
        const int64_t g = (int64_t)blockIdx.x + (i0 + threadIdx.x) * gridDim.x;
        if (g < ngroups && group_points(g) > RES_WARP_MAX) heavy[atomicAdd(&nheavy, 1)] = (int32_t)g;
        __syncthreads();
        const int32_t nh = nheavy;
        for (int32_t h = 0; h < nh; ++h) {
            const int32_t qa = heavy[h] * RES_ROWS;
            const int32_t R = min(RES_ROWS, n - qa);
            if ((int)threadIdx.x <= R) srow_c[threadIdx.x] = A.st[qa + threadIdx.x] - A.st[qa];
            __syncthreads();
            res_group<RES_THREADS>(A, qa, R, srow_c, threadIdx.x, wb, wa, s2);
            __syncthreads();
        }
    }
    // the other groups: one warp each
    int32_t* srow = srow_w[w];
    const int64_t nw = ((int64_t)gridDim.x * RES_THREADS) >> 5;
    for (int64_t g = ((int64_t)blockIdx.x * RES_THREADS + threadIdx.x) >> 5; g < ngroups; g += nw) {
        const int32_t qa = (int32_t)(g * RES_ROWS);
        const int32_t R = min(RES_ROWS, n - qa);
        for (int32_t i = lane; i <= R; i += 32) srow[i] = A.st[qa + i] - A.st[qa];
        __syncwarp();
        if (srow[R] <= RES_WARP_MAX) res_group<32>(A, qa, R, srow, lane, nullptr, nullptr, s2);
        __syncwarp();
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
        const ResArgs ra{p->seq, p->starts, p->col, p->val, p->diag, b, x, p->r64, p->rlp};
        k_residual<<<ddf_grid(((n + 31) / 32) * 32, RES_THREADS, (unsigned)sm * 8), RES_THREADS, 0, s>>>(
            (int32_t)n, ra, p->nrm, p->status);
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
