// Internal declarations shared by the CUDA translation units of libddf.so.
// Nothing here is part of the public ABI (include/ddf.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ddf.h"

#define DDF_MAX_T 512          // largest mining window t (local mask of 512 bits)
#define DDF_WARPS_PER_CTA 8
#define DDF_CTA_THREADS (32 * DDF_WARPS_PER_CTA)
#define DDF_SOLVE_CTAS_PER_SM 2   // resident CTAs per SM of the level-set solve (measured: 1 and 4 are slower)
#define DDF_SOLVE_PTS 2           // points per lane the level-set solve holds in registers: a solve
                                  // unit gives a row of L points ceil(L / DDF_SOLVE_PTS) lanes
// Coarsened solve: a partition is cut into chunks of at most DDF_BLK_ROWS_CAP
// rows and DDF_BLK_ENT_CAP points, the unit staged into shared memory; a row
// longer than DDF_BLK_ENT_CAP is a chunk of its own, run from global memory.
#define DDF_BLK_ROWS_CAP 64
#define DDF_TAIL_PAD 8            // spare elements after val / col / val_lp
#define DDF_BLK_ENT_CAP 768
#define DDF_BLK_CHAIN_LANES 256   // threads of the chain role
#define DDF_BLK_PROD_PER_LANE 8   // points per producer lane per batch
#define DDF_BLK_CHAIN_PER_LANE 1  // in-block points per chain lane (more lanes per row shorten
                                  // the dependent chain, which sets the chunk's latency)
// chunk_meta bits
#define DDF_CK_VCHAIN(m) ((m) & 0xff)
#define DDF_CK_VPROD(m) (((m) >> 8) & 0xff)
#define DDF_CK_PSC2 (1 << 16)
#define DDF_CK_DIRECT (1 << 17)

// Executor codelet descriptor (64 bytes).  Access functions of the codelet's
// rows i0 in [0, m) and points i1 in [0, n):
//   f(i0)     = f0 + rho*i0            (F_STRIDED)   else seq[q0 + i0]
//   g(i0, i1) = g0 + gamma*i0 + i1     (G_STRIDED)   else starts[q0 + i0] + i1
//   h(i0, i1) = h0 + delta*i0 + sigma*i1              (BLAS)
//             = h0 + delta*i0 + (col[sref + i1] - h0) (PSC I: s = first row's columns)
//             = col[g(i0, i1)]                         (PSC II)
struct dcod {
    int32_t q0, m, n, type;
    int32_t part, flags;
    int32_t f0, rho;
    int32_t g0, gamma;
    int32_t h0, delta, sigma, sref;
    int32_t pad0, pad1;
};
static_assert(sizeof(dcod) == 64, "dcod layout");

enum { DC_F_STRIDED = 1, DC_G_STRIDED = 2, DC_TILED = 4 };

// SpMV value tiles.  Consecutive BLAS / PSC I codelets of one type and one
// row length n <= DDF_TILE_NMAX whose rows follow each other form a run
// (dcod.pad0 = first position of the run, pad1 = one past its last; flag
// DC_TILED).  A run is cut into tiles of DDF_TILE_ROWS consecutive rows from
// its first position, and each tile's w x n values (the same range of the
// plan's value array that the rows occupy in CSR order) are stored point-major:
// point i1 of row r of the tile at tile base + i1 * w + r.  The executor then
// runs one lane per row, and the lanes of a tile read one contiguous stretch
// per point.
#define DDF_TILE_ROWS 8
#define DDF_TILE_NMAX 256
#define DDF_LONG_ROW 1024   // SpMV PSC II rows longer than this run one CTA per row

// One tile of the SpMV executor: rows q .. q + w - 1, values from vb (the
// tile's first row's CSR offset); row q + r belongs to codelet
// cod + ((meta >> (3 + 3 r)) & 7), and w = (meta & 7) + 1.
struct dtile {
    int32_t q, cod, vb;
    uint32_t meta;
};
static_assert(sizeof(dtile) == 16, "dtile layout");

// Executor work unit: rows [i0b, i0e) of codelet `cod`, processed by one warp
// with `v` lanes per row (a power of two, 1..32).
struct dunit {
    int32_t cod, i0b, i0e, v;
};
static_assert(sizeof(dunit) == 16, "dunit layout");

// The plan: every pointer is device memory owned by the plan.
struct ddf_plan_s {
    ddf_kind kind;
    ddf_opts opts;
    int device;
    cudaStream_t stream;          // stream the plan was built on (used to free it)
    int32_t n, n_cols, depth;
    int64_t nnz;                  // entries of the inspected CSR
    int64_t npts;                 // iteration points (SpTRSV: off-diagonal entries)
    int has_values;
    // executor layout ("sequence CSR"): positions q, starts[q] .. starts[q+1]
    int32_t* starts;              // SpMV: CSR rowptr copy; SpTRSV: level-ordered off-diagonal starts
    int32_t* col;                 // columns in that layout
    double* val;                  // values in that layout
    int32_t* seq;                 // SpTRSV: row at each position (level order); SpMV: NULL
    int32_t* part_ptr;            // [depth + 1]
    double* dinv;                 // SpTRSV: 1 / L_ii per position
    int32_t* orig_rowptr;         // SpTRSV: rowptr of the inspected matrix (for ddf_update_values)
    int32_t* orig_rowend;         // SpTRSV with lower_of_input: end of each row's lower part
                                  // (owned); NULL when the input is L itself (ends: orig_rowptr + 1)
    // codelets and units
    dcod* cod;
    int64_t ncod;
    int64_t ncod_type[3];
    dunit* units[3];              // SpMV: one list per type (codelets not in tiles); SpTRSV:
                                  // units[0] = all, level order
    int64_t nunits[3];
    int32_t* unit_q;              // SpTRSV: first position of each unit of units[0]
    // SpTRSV batch plans, the multi-RHS solve's work items (NULL: the units
    // themselves): ranges of positions (units[0] split where the matrix
    // changes) and segments of long rows
    int32_t* mrhs_q;              // first position of each item
    int2* mrhs_seg;               // (segment of its row, first partial-sum slot of the row); x = -1: a range
    int32_t* mrhs_order;          // the items in the solve's ticket order
    int64_t mrhs_nr;              // items
    double* mrhs_part;            // partial sums of the segments: 32 slots of 8 bytes per segment
    uint32_t* mrhs_cnt;           // segments finished, per long row (at its first slot)
    int64_t mrhs_ns;              // partial-sum slots
    int32_t* mrhs_moff;           // first row of each matrix of the batch (saved with the plan)
    int32_t mrhs_nmat;
    int32_t* long_q;              // SpMV: positions of the PSC II rows of more than DDF_LONG_ROW
                                  // points (each a one-row unit of units[2], run one CTA per row)
    int64_t nlong;
    dtile* tiles[2];              // SpMV: tiles of tiled BLAS / PSC I codelets (DC_TILED)
    int64_t ntiles[2];
    // device scratch / status
    int32_t* status;              // device status word (ddf_status)
    uint32_t* ticket;             // SpTRSV: work ticket
    int32_t last_launches;
    int32_t mrhs_units_per_ticket;   // ddf_sptrsm: work units per warp ticket (ddf_tune picks it)
    int32_t sm_count;
    // mixed precision (store_dtype != DDF_F64): low-precision copies and the
    // refinement scratch of a SpTRSV plan
    int32_t vdtype;
    void* val_lp;                 // values in store_dtype, same layout as val
    float* dinv_lp;               // SpTRSV: 1 / L_ii rounded to FP32
    double* diag;                 // SpTRSV: L_ii in FP64 (residual)
    double* r64;                  // residual b - L x (row order)
    float* rlp;                   // residual rounded to FP32 (right-hand side of a correction)
    float* xlp;                   // low-precision solution / correction
    double* nrm;                  // ||b||^2, ||r||^2 (FP64 accumulators) and a copy of the status word
    // coarsened SpTRSV plans (opts.coarsen_rows = R > 0): partitions are the
    // (block of R rows, level) pairs; part_ptr then has depth + 1 entries with
    // depth = number of partitions, and nlevels is the depth of G
    int32_t nlevels;              // SpTRSV: depth of G
    int32_t nblocks;              // coarsened: ceil(n / R); 0 otherwise
    int32_t* blk_ptr;             // [nblocks + 1] first partition of each block
    int32_t* esplit;              // [n] entries of position q with a column before its block
    int32_t* qcod;                // [n] codelet holding position q
    int64_t nchunks;              // coarsened: chunks of all partitions
    int32_t* chunk_q0;            // [nchunks + 1] first position of each chunk
    int32_t* chunk_meta;          // [nchunks] lanes per row and flags (DDF_CK_*)
    int32_t* blk_chunk;           // [nblocks + 1] first chunk of each block
    // statistics, computed on the first ddf_plan_stats call
    int32_t stats_ready;
    ddf_plan_stats_t stats;
};

#define DDF_SENTINEL 0xFFFFFFFFFFFFFFFFull   // fill pattern of x during a solve (a NaN)
#define DDF_CANON_NAN 0x7FF8000000000000ull

#define DDF_CUDA_TRY(call)                         \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            (void)cudaGetLastError();              \
            return e_ == cudaErrorMemoryAllocation ? DDF_ERR_OOM : DDF_ERR_CUDA; \
        }                                          \
    } while (0)

// value conversions used by the templated executors
template <typename TA>
__device__ __forceinline__ TA ddf_cvt(double v) { return (TA)v; }
template <typename TA>
__device__ __forceinline__ TA ddf_cvt(float v) { return (TA)v; }
template <typename TA>
__device__ __forceinline__ TA ddf_cvt(__nv_bfloat16 v) { return (TA)__bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T ddf_from_float(float v) { return (T)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 ddf_from_float<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ---------------------------------------------------------------------------
// memory-model helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ddf_ld_relaxed_u64(const void* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void ddf_st_relaxed_u64(void* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ddf_ld_relaxed_u32(const void* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void ddf_st_relaxed_u32(void* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t ddf_ld_relaxed_s32(const void* p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void ddf_st_relaxed_s32(void* p, int32_t v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ddf_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void ddf_set_status(int32_t* status, int32_t code) {
    atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// host-side launchers implemented in the .cu files
// ---------------------------------------------------------------------------
// ddf_scan.cu
ddf_status ddf_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
ddf_status ddf_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
ddf_status ddf_radix_sort_u32(uint32_t* keys, int32_t* vals, int64_t n, uint32_t max_key,
                              cudaStream_t s);
// ddf_inspect.cu
ddf_status ddf_build_plan(ddf_plan_s* p, const int32_t* rowptr, const int32_t* colidx,
                          const double* values, cudaStream_t s);
ddf_status ddf_gather_values(ddf_plan_s* p, const double* values, cudaStream_t s);
ddf_status ddf_compute_stats(ddf_plan_s* p);
ddf_status ddf_build_units(ddf_plan_s* p, cudaStream_t s);
ddf_status ddf_mark_tiles(ddf_plan_s* p, cudaStream_t s);
ddf_status ddf_build_unit_q(ddf_plan_s* p, cudaStream_t s);
// ddf_batch.cu: the multi-RHS solve's work items of a batch plan whose matrices start at rows moff[0 .. count - 1]
ddf_status ddf_build_mrhs_items(ddf_plan_s* p, const int32_t* moff, int32_t count, cudaStream_t s);
ddf_status ddf_build_long_rows(ddf_plan_s* p, cudaStream_t s);
// ddf_capi.cu
ddf_status ddf_new_plan(ddf_kind kind, const ddf_opts* o, cudaStream_t s, int32_t n, int32_t n_cols, int64_t nnz,
                        ddf_plan_s** out);
// borrowed: ci / v belong to the caller (read only during this call, not freed)
ddf_status ddf_finish_plan(ddf_plan_s* p, int32_t* rp, int32_t* ci, double* v, cudaStream_t s, ddf_plan_t* out,
                           bool borrowed = false);
// ddf_spmv.cu
ddf_status ddf_launch_spmv(ddf_plan_s* p, const double* x, double* y, cudaStream_t s);
ddf_status ddf_launch_spmv_lp(ddf_plan_s* p, const void* x, void* y, int vec_dtype, cudaStream_t s);
// ddf_sptrsv.cu
ddf_status ddf_launch_sptrsv(ddf_plan_s* p, const double* b, double* x, cudaStream_t s);
ddf_status ddf_launch_sptrsv_lp(ddf_plan_s* p, const float* b, float* x, cudaStream_t s);
// ddf_mixed.cu
ddf_status ddf_make_lowp(ddf_plan_s* p, cudaStream_t s);
ddf_status ddf_refine(ddf_plan_s* p, const double* b, double* x, double tol, int32_t max_iter, cudaStream_t s,
                      int32_t* iters, double* relres);

// process-wide count of kernel launches (ddf_capi.cu)
void ddf_count_launch(int64_t k = 1);

// test hook of ddf_debug_fail_alloc (ddf_capi.cu): true for the one device
// allocation that is to fail as if the device were out of memory
bool ddf_alloc_injected_failure();

// NVTX range around an entry point (header-only NVTX 3: a no-op unless a
// profiling tool is attached)
struct ddf_nvtx_range {
    explicit ddf_nvtx_range(const char* name);
    ~ddf_nvtx_range();
};

// device allocation helpers (stream-ordered)
template <typename T>
static inline ddf_status ddf_alloc(T** ptr, int64_t count, cudaStream_t s) {
    *ptr = nullptr;
    if (count <= 0) return DDF_OK;
    if (ddf_alloc_injected_failure()) return DDF_ERR_OOM;
    cudaError_t e = cudaMallocAsync((void**)ptr, (size_t)count * sizeof(T), s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *ptr = nullptr;
        return e == cudaErrorMemoryAllocation ? DDF_ERR_OOM : DDF_ERR_CUDA;
    }
    return DDF_OK;
}
template <typename T>
static inline void ddf_free(T*& ptr, cudaStream_t s) {
    if (ptr) (void)cudaFreeAsync((void*)ptr, s);
    ptr = nullptr;
}

static inline unsigned ddf_grid(int64_t work, int per_block, unsigned cap = 0x7fffffffu) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > (int64_t)cap) g = cap;
    return (unsigned)g;
}
