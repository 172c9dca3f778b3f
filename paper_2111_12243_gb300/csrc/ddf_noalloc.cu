// ddf_sptrsv_csr_noalloc: a lower-triangular solve for callers that cannot
// allocate device memory.  It works directly on the caller's CSR arrays (no
// plan: building a plan allocates) and keeps its scratch in one file-scope
// device array instead of memory obtained from cudaMalloc.
//
// Scratch layout (32-bit words): [0] work ticket, [1] status, [2] abort flag,
// [NA_HDR + r] = number of the call that finished row r.  Call numbers start
// at 1 and grow with every call on the device, so the per-row flags never need
// clearing; only the three header words are reset per call.  Every call on a
// device uses the same array, so calls that overlap on the GPU race.
#include <atomic>

#include "ddf_internal.cuh"

namespace {

constexpr int NA_HDR = 64;                      // header words (keeps the flags 256-byte aligned)
constexpr int NA_CHUNK = 32 * DDF_WARPS_PER_CTA;  // rows per CTA ticket (one row per lane slot)
constexpr int NA_RPW = NA_CHUNK / DDF_WARPS_PER_CTA;

__device__ __align__(256) uint32_t ddf_noalloc_scratch[NA_HDR + DDF_NOALLOC_MAX_ROWS];

// Per device ordinal: the number of the last call, so that row flags left by
// earlier calls (which the array keeps) never match the current call's.
std::atomic<uint32_t> g_epoch[64];

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until row j of this call is finished (flag == epoch).
__device__ bool na_wait(const uint32_t* flag, uint32_t epoch, uint32_t* hdr, int64_t cap_ns) {
    uint64_t t0 = ddf_globaltimer();
    uint32_t it = 0, ns = 32;
    while (true) {
        if (ld_acquire_u32(flag) == epoch) return true;
        ++it;
        if (it > 8) {
            __nanosleep(ns);
            ns = min(ns * 2, 256u);
        }
        if ((it & 15u) == 0) {
            if (ddf_ld_relaxed_s32(hdr + 2) != 0) return false;
            if ((int64_t)(ddf_globaltimer() - t0) > cap_ns) {
                atomicCAS(hdr + 1, 0u, (uint32_t)DDF_ERR_TIMEOUT);
                atomicExch(hdr + 2, 1u);
                return false;
            }
        }
    }
}

// Forward substitution in row order.  Each CTA takes the next chunk of
// NA_CHUNK rows from the ticket; warp w solves rows [w*NA_RPW, (w+1)*NA_RPW)
// of the chunk one after the other, lanes over the row's entries.  Values of
// the chunk's rows are also kept in shared memory, so dependencies inside
// the chunk are read there; dependencies on earlier chunks wait on the
// scratch flags.  Every row waited on has a smaller index, hence belongs to
// this CTA or to a CTA that already holds a ticket: the waits end.  Indices
// are checked before use: a malformed row latches an error and contributes
// nothing instead of reading out of bounds.
__global__ void __launch_bounds__(DDF_CTA_THREADS)
k_sptrsv_noalloc(int32_t n, int64_t nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                 const double* __restrict__ v, const double* __restrict__ b, double* x, uint32_t* scratch,
                 uint32_t epoch, int64_t cap_ns) {
    __shared__ uint32_t chunk;
    __shared__ double sx[NA_CHUNK];
    __shared__ int32_t sready[NA_CHUNK];
    uint32_t* hdr = scratch;
    uint32_t* flag = scratch + NA_HDR;
    if (threadIdx.x == 0) chunk = atomicAdd(hdr, 1u);
    for (int i = threadIdx.x; i < NA_CHUNK; i += blockDim.x) sready[i] = 0;
    __syncthreads();
    volatile int32_t* vr = sready;
    volatile double* vx = sx;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)chunk * NA_CHUNK;
    for (int rr = 0; rr < NA_RPW; ++rr) {
        const int64_t r = base + (int64_t)w * NA_RPW + rr;
        if (r >= n) break;
        const int32_t a = rp[r], e = rp[r + 1];
        bool bad = a < 0 || e <= a || (int64_t)e > nnz;
        const int32_t last = bad ? -1 : ci[e - 1];
        if (!bad && last != (int32_t)r) bad = true;
        double acc = 0.0;
        if (!bad) {
            for (int32_t k = a + lane; k < e - 1; k += 32) {
                const int32_t j = ci[k];
                if (j < 0 || (int64_t)j >= r) {      // not strictly below the diagonal
                    atomicCAS(hdr + 1, 0u, (uint32_t)DDF_ERR_NOT_LOWER);
                    continue;
                }
                double xj;
                if ((int64_t)j >= base) {
                    const int32_t lj = j - (int32_t)base;
                    uint64_t t0 = 0;
                    uint32_t it = 0;
                    while (vr[lj] == 0) {
                        if ((++it & 255u) == 0) {
                            if (t0 == 0) t0 = ddf_globaltimer();
                            if (ddf_ld_relaxed_s32(hdr + 2) != 0) break;
                            if ((int64_t)(ddf_globaltimer() - t0) > cap_ns) {
                                atomicCAS(hdr + 1, 0u, (uint32_t)DDF_ERR_TIMEOUT);
                                atomicExch(hdr + 2, 1u);
                                break;
                            }
                        }
                    }
                    // pairs with the writer's fence between its value and flag stores
                    __threadfence_block();
                    xj = vx[lj];
                } else {
                    if (ld_acquire_u32(flag + j) != epoch) na_wait(flag + j, epoch, hdr, cap_ns);
                    xj = __ldcg(x + j);
                }
                acc += v[k] * xj;
            }
        } else {
            if (lane == 0) atomicCAS(hdr + 1, 0u, (uint32_t)DDF_ERR_MISSING_DIAG);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            double d = bad ? 0.0 : v[e - 1];
            if (!bad && d == 0.0) atomicCAS(hdr + 1, 0u, (uint32_t)DDF_ERR_ZERO_DIAG);
            double xr = (b[r] - acc) / d;
            x[r] = xr;
            vx[r - base] = xr;
            __threadfence_block();
            vr[r - base] = 1;
            st_release_u32(flag + r, epoch);
        }
        __syncwarp();
    }
}

// The device address of the scratch array in the current context.  In host
// code the array's name is only a host-side stand-in, so the kernel must be
// given this address instead.  The lookup runs on every call (it allocates
// nothing once the module is loaded), so a context that was reset or replaced
// since an earlier call never receives a stale address.  The first lookup in
// a context loads the library's module, which is where the array is created.
ddf_status scratch_address(uint32_t** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, ddf_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        (void)cudaGetLastError();
        return DDF_ERR_CUDA;
    }
    *out = (uint32_t*)p;
    return DDF_OK;
}

}  // namespace

extern "C" ddf_status ddf_sptrsv_csr_noalloc(int32_t n, int64_t nnz, const int32_t* rowptr,
                                             const int32_t* colidx, const double* values,
                                             const double* b, double* x, int64_t spin_cap_ns,
                                             ddf_stream_t stream) {
    ddf_nvtx_range nvtx_("ddf_sptrsv_csr_noalloc");
    if (n < 0 || nnz < 0 || nnz > 0x7fffffffll || spin_cap_ns <= 0) return DDF_ERR_ARG;
    if (n > DDF_NOALLOC_MAX_ROWS) return DDF_ERR_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return DDF_ERR_CUDA;
    }
    // the set-up comes before the n == 0 return, so that an empty call is the
    // warm-up that loads the module (and creates the array) ahead of time
    uint32_t* scratch = nullptr;
    ddf_status st = scratch_address(&scratch);
    if (st) return st;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_sptrsv_noalloc) != cudaSuccess) {
        (void)cudaGetLastError();
        return DDF_ERR_CUDA;
    }
    if (n == 0) return DDF_OK;
    if (!rowptr || !colidx || !values || !b || !x) return DDF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t epoch = g_epoch[dev].fetch_add(1u) + 1u;
    if (epoch == 0u) {
        // the call counter wrapped: forget every old row flag once
        DDF_CUDA_TRY(cudaMemsetAsync(scratch + NA_HDR, 0, sizeof(uint32_t) * DDF_NOALLOC_MAX_ROWS, s));
        epoch = g_epoch[dev].fetch_add(1u) + 1u;
    }
    DDF_CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * 3, s));
    const unsigned ctas = (unsigned)((n + NA_CHUNK - 1) / NA_CHUNK);
    k_sptrsv_noalloc<<<ctas, DDF_CTA_THREADS, 0, s>>>(n, nnz, rowptr, colidx, values, b, x, scratch, epoch,
                                                     spin_cap_ns);
    ddf_count_launch();
    DDF_CUDA_TRY(cudaGetLastError());
    uint32_t h = 0;
    DDF_CUDA_TRY(cudaMemcpyAsync(&h, scratch + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    DDF_CUDA_TRY(cudaStreamSynchronize(s));
    return (ddf_status)h;
}
