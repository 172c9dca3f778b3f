// Device primitives used by the inspector: exclusive prefix sums and a stable
// LSD radix sort of (uint32 key, int32 value) pairs.
#include "ddf_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;   // 4096

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Block-wide exclusive scan of one tile held in shared memory (blocked per thread).
template <typename TIn>
__global__ void k_tile_sums(const TIn* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        if (k < n) acc += (int64_t)in[k];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) wsum[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int i = 0; i < SCAN_THREADS / 32; ++i) t += wsum[i];
        sums[blockIdx.x] = t;
    }
}

template <typename TIn>
__global__ void k_tile_scan(const TIn* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                            int64_t* __restrict__ out) {
    __shared__ int64_t tile[SCAN_TILE];
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        tile[i] = (k < n) ? (int64_t)in[k] : 0;
    }
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t loc[SCAN_ITEMS];
    int64_t t = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        loc[j] = t;
        t += tile[threadIdx.x * SCAN_ITEMS + j];
    }
    int64_t incl = warp_incl_scan(t, lane);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t v = (lane < SCAN_THREADS / 32) ? wsum[lane] : 0;
        v = warp_incl_scan(v, lane);
        if (lane < SCAN_THREADS / 32) wsum[lane] = v;
    }
    __syncthreads();
    int64_t pre = offs[blockIdx.x] + (incl - t) + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) tile[threadIdx.x * SCAN_ITEMS + j] = pre + loc[j];
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        if (k < n) out[k] = tile[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = offs[gridDim.x];
}

// Exclusive scan of at most one tile (n <= SCAN_TILE) by one CTA; out[n] is
// the total.
template <typename TIn>
__global__ void k_scan_one(const TIn* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
    __shared__ int64_t tile[SCAN_TILE];
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) tile[i] = (i < n) ? (int64_t)in[i] : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t loc[SCAN_ITEMS];
    int64_t t = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        loc[j] = t;
        t += tile[threadIdx.x * SCAN_ITEMS + j];
    }
    const int64_t incl = warp_incl_scan(t, lane);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t v = (lane < SCAN_THREADS / 32) ? wsum[lane] : 0;
        v = warp_incl_scan(v, lane);
        if (lane < SCAN_THREADS / 32) wsum[lane] = v;
    }
    __syncthreads();
    const int64_t pre = (incl - t) + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) tile[threadIdx.x * SCAN_ITEMS + j] = pre + loc[j];
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS)
        if (i < n) out[i] = tile[i];
    if (threadIdx.x == 0) out[n] = wsum[SCAN_THREADS / 32 - 1];
}

template <typename TIn>
ddf_status scan_impl(const TIn* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        DDF_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return DDF_OK;
    }
    if (n <= SCAN_TILE) {
        k_scan_one<TIn><<<1, SCAN_THREADS, 0, s>>>(in, n, out);
        ddf_count_launch();
        DDF_CUDA_TRY(cudaGetLastError());
        return DDF_OK;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t* sums = nullptr;
    int64_t* offs = nullptr;
    ddf_status st = ddf_alloc(&sums, nb, s);
    if (st) return st;
    st = ddf_alloc(&offs, nb + 1, s);
    if (st) { ddf_free(sums, s); return st; }
    k_tile_sums<TIn><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums);
    ddf_count_launch();
    st = scan_impl<int64_t>(sums, offs, nb, s);
    if (!st) {
        k_tile_scan<TIn><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, offs, out);
        ddf_count_launch();
    }
    ddf_free(sums, s);
    ddf_free(offs, s);
    if (st) return st;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
constexpr int RS_WARPS = 8;
constexpr int RS_STEPS = 8;
constexpr int RS_TILE = RS_WARPS * 32 * RS_STEPS;   // 2048 elements per CTA

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                             int32_t* __restrict__ ghist, int64_t ntiles) {
    __shared__ int32_t h[RS_WARPS][256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * 32 * RS_STEPS;
    for (int st = 0; st < RS_STEPS; ++st) {
        int64_t i = base + st * 32 + lane;
        if (i < n) atomicAdd(&h[w][(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int32_t t = 0;
        for (int k = 0; k < RS_WARPS; ++k) t += h[k][d];
        ghist[(int64_t)d * ntiles + blockIdx.x] = t;
    }
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                                int shift, const int64_t* __restrict__ goff, int64_t ntiles) {
    __shared__ int32_t h[RS_WARPS][256];
    __shared__ int64_t base[RS_WARPS][256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t b0 = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * 32 * RS_STEPS;
    for (int st = 0; st < RS_STEPS; ++st) {
        int64_t i = b0 + st * 32 + lane;
        if (i < n) atomicAdd(&h[w][(kin[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int64_t run = goff[(int64_t)d * ntiles + blockIdx.x];
        for (int k = 0; k < RS_WARPS; ++k) {
            base[k][d] = run;
            run += h[k][d];
        }
    }
    __syncthreads();
    unsigned lt = (1u << lane) - 1u;
    for (int st = 0; st < RS_STEPS; ++st) {
        int64_t i = b0 + st * 32 + lane;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t d = valid ? ((key >> shift) & 255u) : (256u + (unsigned)lane);
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid) {
            int64_t pos = base[w][d] + __popc(peers & lt);
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) base[w][d] += __popc(peers);
        __syncwarp();
    }
}

}  // namespace

ddf_status ddf_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, s);
}

ddf_status ddf_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}

// Sort (keys, vals) by key, stably; results replace the inputs.
ddf_status ddf_radix_sort_u32(uint32_t* keys, int32_t* vals, int64_t n, uint32_t max_key,
                              cudaStream_t s) {
    if (n <= 1 || max_key == 0) return DDF_OK;
    int passes = 0;
    for (uint32_t m = max_key; m; m >>= 8) ++passes;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    uint32_t* k2 = nullptr;
    int32_t* v2 = nullptr;
    int32_t* hist = nullptr;
    int64_t* goff = nullptr;
    ddf_status st = ddf_alloc(&k2, n, s);
    if (!st) st = ddf_alloc(&v2, n, s);
    if (!st) st = ddf_alloc(&hist, 256 * ntiles, s);
    if (!st) st = ddf_alloc(&goff, 256 * ntiles + 1, s);
    uint32_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    for (int p = 0; p < passes && !st; ++p) {
        int shift = 8 * p;
        k_radix_hist<<<(unsigned)ntiles, RS_WARPS * 32, 0, s>>>(ka, n, shift, hist, ntiles);
        ddf_count_launch();
        st = ddf_scan_i32_to_i64(hist, goff, 256 * ntiles, s);
        if (st) break;
        k_radix_scatter<<<(unsigned)ntiles, RS_WARPS * 32, 0, s>>>(ka, va, kb, vb, n, shift, goff,
                                                                  ntiles);
        ddf_count_launch();
        uint32_t* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    if (!st && ka != keys) {
        cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, va, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    }
    ddf_free(k2, s);
    ddf_free(v2, s);
    ddf_free(hist, s);
    ddf_free(goff, s);
    if (st) return st;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}
