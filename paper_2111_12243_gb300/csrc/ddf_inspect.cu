// DDF inspector on the GPU (Alg. 1 of the paper).
//
//   computeAccessFunctions  implicit: position q of a partition sequence has
//                           f(q) = seq[q], g(q,i1) = starts[q] + i1,
//                           h(q,i1) = col[starts[q] + i1]           (Sec. III-A)
//   findDependencies        SpTRSV: level of every row, longest path (k_levels)
//   partitionIterationSpace SpTRSV: rows sorted by (level, row) (radix sort);
//                           SpMV: one partition with every row      (Sec. IV-A)
//   ComputeFOPD             first order partial differences per position and
//                           between consecutive positions (k_features, Sec. III-D)
//   GetConsecutiveIterations regions of t consecutive positions of a partition
//   BLAS_first / PSCI_first / PSCII_first / min_cost / append
//                           one thread per region (k_mine, k_emit)
//
// Every step is deterministic: counts come from per-region work followed by
// prefix sums, and the level order from a stable radix sort.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ddf_internal.cuh"

namespace {

enum : uint8_t { FL_HSTR = 1, FL_EQLEN = 2, FL_TRANS = 4, FL_LINK = 8 };
enum { MK_NONE = -1 };

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
// One thread per row; every violation found is reported with atomicMin, so
// the result is the smallest error code present.
__global__ void k_validate(int32_t n, int32_t n_cols, int64_t nnz, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, const double* __restrict__ v, int kind,
                           int32_t* __restrict__ err, int lanes) {
    // `lanes` consecutive threads per row: lane li checks the entries
    // a + li, a + li + lanes, ... (coalesced), each against the next entry
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lg = __ffs(lanes) - 1, li = (int)(t & (lanes - 1));
    const int64_t r = t >> lg;
    if (t == 0 && (rp[0] != 0 || (int64_t)rp[n] != nnz)) atomicMin(err, (int)DDF_ERR_UNSORTED);
    if (r >= n) return;
    const int32_t a = rp[r], b = rp[r + 1];
    if (a < 0 || b < a || (int64_t)b > nnz) {
        if (li == 0) atomicMin(err, (int)DDF_ERR_UNSORTED);
        return;
    }
    bool out = false, order = false;
#pragma unroll 4
    for (int32_t k = a + li; k < b; k += lanes) {
        const int32_t c = ci[k];
        out |= c < 0 || c >= n_cols;
        if (k + 1 < b) order |= ci[k + 1] <= c;
    }
    // a row with several faults reports the smallest code, as the matrix
    // does across rows (atomicMin)
    if (out) atomicMin(err, (int)DDF_ERR_OUT_OF_RANGE);
    if (order) atomicMin(err, (int)DDF_ERR_UNSORTED);
    if (kind == DDF_SPTRSV && li == 0 && !out && !order) {
        if (b == a) atomicMin(err, (int)DDF_ERR_MISSING_DIAG);
        else if (ci[b - 1] > r) atomicMin(err, (int)DDF_ERR_NOT_LOWER);
        else if (ci[b - 1] != r) atomicMin(err, (int)DDF_ERR_MISSING_DIAG);
        else if (v != nullptr && v[b - 1] == 0.0) atomicMin(err, (int)DDF_ERR_ZERO_DIAG);
    }
}

// lower_of_input: the end of the lower part of each row of a validated
// square matrix (its columns increase, so the part is a prefix: the first
// entry with a column above the row ends it), and that part's diagonal
// checks.  Rows that failed validation get an empty part.
__global__ void k_lower_end(int32_t n, int64_t nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, int32_t* __restrict__ re, int32_t* __restrict__ err) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t a = rp[r], b = rp[r + 1];
    if (a < 0 || b < a || (int64_t)b > nnz) {
        re[r] = a < 0 ? 0 : a;
        return;
    }
    int32_t lo = a, hi = b;   // first k in [a, b) with ci[k] > r, else b
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (ci[mid] > r) hi = mid;
        else lo = mid + 1;
    }
    re[r] = lo;
    if (lo == a || ci[lo - 1] != r) atomicMin(err, (int)DDF_ERR_MISSING_DIAG);
    else if (v != nullptr && v[lo - 1] == 0.0) atomicMin(err, (int)DDF_ERR_ZERO_DIAG);
}

__global__ void k_set2(int32_t* __restrict__ a, int32_t v0, int32_t v1) {
    a[0] = v0;
    a[1] = v1;
}

__global__ void k_fill_i32(int32_t* __restrict__ a, int64_t n, int32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_iota_u32(int32_t* __restrict__ a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

__global__ void k_i64_to_i32(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

// ---------------------------------------------------------------------------
// findDependencies: level[i] = 1 + max level of its off-diagonal columns
// ---------------------------------------------------------------------------
constexpr int LEV_CHUNK = 1024;                               // rows per CTA ticket (a multiple of 1024)
constexpr int LEV_MAXSEG = 256;                               // longest run one warp takes at once

// Bounded wait on a level written by another CTA: a few immediate polls, then
// exponential backoff so that waiting warps do not flood L2 with requests.
__device__ int32_t wait_level(const int32_t* p, int32_t* status, int64_t cap_ns) {
    uint64_t t0 = ddf_globaltimer();
    uint32_t it = 0, ns = 32;
    while (true) {
        int32_t v = ddf_ld_relaxed_s32(p);
        if (v >= 0) return v;
        ++it;
        if (it > 4) {
            __nanosleep(ns);
            ns = min(ns * 2, 512u);
        }
        if ((it & 15u) == 0) {
            if (ddf_ld_relaxed_s32(status) != 0) return 0;
            if ((int64_t)(ddf_globaltimer() - t0) > cap_ns) {
                ddf_set_status(status, DDF_ERR_TIMEOUT);
                return 0;
            }
        }
    }
}

// Bounded wait on a level written by another warp of this CTA.  The wait
// sleeps between polls: a warp spinning on shared memory would otherwise take
// issue slots from the warp of its SM that computes the awaited row.
__device__ int32_t wait_level_smem(volatile int32_t* p, int32_t* status, int64_t cap_ns) {
    uint64_t t0 = ddf_globaltimer();
    uint32_t it = 0;
    while (true) {
        int32_t v = *p;
        if (v >= 0) return v;
        if (++it > 32) __nanosleep(32);
        if ((it & 63u) == 0) {
            if (ddf_ld_relaxed_s32(status) != 0) return 0;
            if ((int64_t)(ddf_globaltimer() - t0) > cap_ns) {
                ddf_set_status(status, DDF_ERR_TIMEOUT);
                return 0;
            }
        }
    }
}

// Each CTA takes the next chunk of LEV_CHUNK consecutive rows from a ticket and
// cuts it into runs: a run starts at every row that does not read the row just
// before it (the start of a grid line of a stencil, for instance) and at least
// every LEV_MAXSEG rows.  Warps take runs in increasing order from a counter
// and compute a run's rows in order, so a chain that follows the rows stays on
// one warp while the next run, which only waits for the rows it reads, starts
// on another.  Levels of the chunk's rows are also kept in shared memory: a
// dependency inside the chunk costs a shared-memory read instead of an L2
// round trip.  Rows are software pipelined: while row r is reduced, the
// column indices of row r + 1 and the levels of its dependencies outside the
// chunk are already in flight.  Every row waited on has a smaller index, so it
// belongs to a run that a running warp has taken, or to a CTA that already
// holds a ticket and runs: the waits end.  Large chunks keep many rows in
// flight per resident thread: with one row per thread too few planes of a
// 3-D stencil are resident for the wavefront to pipeline.
constexpr int LEV_WARPS = 16;                                 // warps per CTA

constexpr int LEV_PF = 2;   // dependencies per lane prefetched (rows of up to 64 off-diagonals)

__device__ __forceinline__ void lev_prefetch(int32_t a, int32_t b, int lane, int64_t base,
                                             const int32_t* __restrict__ ci, const int32_t* lev,
                                             int32_t* j, int32_t* l) {
#pragma unroll
    for (int k = 0; k < LEV_PF; ++k) {
        const int32_t kk = a + lane + 32 * k;
        j[k] = kk < b ? ci[kk] : -1;
    }
#pragma unroll
    for (int k = 0; k < LEV_PF; ++k)
        l[k] = (j[k] >= 0 && (int64_t)j[k] < base) ? ddf_ld_relaxed_s32(lev + j[k]) : -1;
}

__global__ void __launch_bounds__(32 * LEV_WARPS)
k_levels(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ re, const int32_t* __restrict__ ci,
         int32_t* lev, uint32_t* ticket, int32_t* maxlev, int32_t* status, int64_t cap_ns) {
    __shared__ int32_t chunk, nruns, next;
    __shared__ int32_t wmax[LEV_WARPS];
    __shared__ int32_t slev[LEV_CHUNK];
    __shared__ uint32_t scut[LEV_CHUNK / 32];
    __shared__ int32_t rstart[LEV_CHUNK + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        chunk = (int32_t)atomicAdd(ticket, 1u);
        next = 0;
    }
    for (int i = threadIdx.x; i < LEV_CHUNK; i += blockDim.x) slev[i] = -1;
    __syncthreads();
    const int64_t base = (int64_t)chunk * LEV_CHUNK;
    const int32_t rlen = (int32_t)min((int64_t)LEV_CHUNK, (int64_t)n - base);
    // run starts: rows that do not read the previous row, and every LEV_MAXSEG rows
    for (int bt = w; bt < LEV_CHUNK / 32; bt += LEV_WARPS) {
        const int32_t o = bt * 32 + lane;
        bool cut = false;
        if (o < rlen) {
            const int64_t r = base + o;
            const int32_t e = re[r] - 1;   // the diagonal is last
            cut = (o % LEV_MAXSEG) == 0 || !(e > rp[r] && ci[e - 1] == (int32_t)(r - 1));
        }
        const unsigned m = __ballot_sync(0xffffffffu, cut);
        if (lane == 0) scut[bt] = m;
    }
    __syncthreads();
    if (w == 0) {
        // positions of the set bits, in order (LEV_WPL consecutive words per lane)
        constexpr int LEV_WPL = LEV_CHUNK / 1024;
        int c = 0;
#pragma unroll
        for (int i = 0; i < LEV_WPL; ++i) c += __popc(scut[lane * LEV_WPL + i]);
        int pre = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += t;
        }
        int k = pre - c;
#pragma unroll
        for (int i = 0; i < LEV_WPL; ++i)
            for (uint32_t m = scut[lane * LEV_WPL + i]; m; m &= m - 1)
                rstart[k++] = 32 * (lane * LEV_WPL + i) + __ffs(m) - 1;
        if (lane == 31) {
            nruns = pre;
            rstart[pre] = rlen;
        }
    }
    __syncthreads();
    volatile int32_t* vs = slev;
    int32_t mymax = 0;
    while (true) {
        int32_t u = 0;
        if (lane == 0) u = atomicAdd(&next, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= nruns) break;
        const int32_t ua = rstart[u], ub = rstart[u + 1];
        for (int32_t sb = ua; sb < ub; sb += 32) {
            // row extents of the next (up to) 32 rows of the run, one per lane
            const int64_t r0 = base + sb;
            const int cnt = min(32, ub - sb);
            int32_t ra_l = 0, rb_l = 0;
            if (lane < cnt) {
                ra_l = rp[r0 + lane];
                rb_l = re[r0 + lane] - 1;   // the diagonal is last: not a dependency
            }
            int32_t cj[LEV_PF], cl[LEV_PF];
            {
                const int32_t a = __shfl_sync(0xffffffffu, ra_l, 0), b = __shfl_sync(0xffffffffu, rb_l, 0);
                lev_prefetch(a, b, lane, base, ci, lev, cj, cl);
            }
            for (int rr = 0; rr < cnt; ++rr) {
                const int64_t r = r0 + rr;
                const int32_t a = __shfl_sync(0xffffffffu, ra_l, rr), b = __shfl_sync(0xffffffffu, rb_l, rr);
                // next row's columns and external levels go out now
                int32_t nj[LEV_PF], nl[LEV_PF];
                {
                    const bool more = rr + 1 < cnt;
                    const int32_t na = __shfl_sync(0xffffffffu, ra_l, (rr + 1) & 31);
                    const int32_t nb = __shfl_sync(0xffffffffu, rb_l, (rr + 1) & 31);
                    lev_prefetch(na, more ? nb : na, lane, base, ci, lev, nj, nl);
                }
                int32_t m = -1;
#pragma unroll
                for (int k = 0; k < LEV_PF; ++k) {
                    const int32_t jj = cj[k];
                    if (jj < 0) continue;
                    int32_t lj;
                    if ((int64_t)jj >= base) {
                        lj = vs[jj - base];
                        if (lj < 0) lj = wait_level_smem(vs + (jj - base), status, cap_ns);
                    } else {
                        lj = cl[k];
                        if (lj < 0) lj = wait_level(lev + jj, status, cap_ns);
                    }
                    m = max(m, lj);
                }
                for (int32_t k = a + lane + 32 * LEV_PF; k < b; k += 32) {   // rows longer than the prefetch
                    const int32_t jj = ci[k];
                    int32_t lj;
                    if ((int64_t)jj >= base) {
                        lj = vs[jj - base];
                        if (lj < 0) lj = wait_level_smem(vs + (jj - base), status, cap_ns);
                    } else {
                        lj = ddf_ld_relaxed_s32(lev + jj);
                        if (lj < 0) lj = wait_level(lev + jj, status, cap_ns);
                    }
                    m = max(m, lj);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) {
                    vs[r - base] = m + 1;
                    ddf_st_relaxed_s32(lev + r, m + 1);
                }
                mymax = max(mymax, m + 1);
                __syncwarp();
#pragma unroll
                for (int k = 0; k < LEV_PF; ++k) {
                    cj[k] = nj[k];
                    cl[k] = nl[k];
                }
            }
        }
    }
    if (lane == 0) wmax[w] = mymax;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int k = 0; k < LEV_WARPS; ++k) t = max(t, wmax[k]);
        atomicMax(maxlev, t);
    }
}

// part_ptr[l] = first position of level l in the sorted order (every level
// between 0 and depth-1 holds at least one row).
__global__ void k_part_ptr(int32_t n, const uint32_t* __restrict__ ls, int32_t* __restrict__ pp,
                           int32_t depth) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    if (q == 0) pp[depth] = n;
    if (q == 0 || ls[q] != ls[q - 1]) pp[ls[q]] = (int32_t)q;
}

// ---------------------------------------------------------------------------
// Coarsened partitions (LBC-style, Sec. IV-A): rows in blocks of R consecutive
// rows; inside a block, one partition per level.  The level order is sorted a
// second time, stably, by block, which gives (block, level, row).
// ---------------------------------------------------------------------------
__global__ void k_block_key(int32_t n, const int32_t* __restrict__ seq, int32_t R, uint32_t* __restrict__ key) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) key[q] = (uint32_t)(seq[q] / R);
}

// flag[q] = 1 where a partition starts: the block or the level changes.
__global__ void k_coarse_flags(int32_t n, const int32_t* __restrict__ seq, const uint32_t* __restrict__ key,
                               const int32_t* __restrict__ lev, int32_t* __restrict__ flag) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    flag[q] = (q == 0 || key[q] != key[q - 1] || lev[seq[q]] != lev[seq[q - 1]]) ? 1 : 0;
}

// part_ptr / blk_ptr from the exclusive scan `off` of the flags; pid[q] is the
// partition of position q (the mining step's partition key).
__global__ void k_coarse_fill(int32_t n, const uint32_t* __restrict__ key, const int32_t* __restrict__ flag,
                              const int64_t* __restrict__ off, int32_t npart, int32_t nblocks,
                              int32_t* __restrict__ pp, int32_t* __restrict__ bp, uint32_t* __restrict__ pid) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int32_t id = (int32_t)(off[q + 1] - 1);
    pid[q] = (uint32_t)id;
    if (flag[q]) {
        pp[id] = (int32_t)q;
        if (q == 0 || key[q] != key[q - 1]) bp[key[q]] = id;
    }
    if (q == 0) {
        pp[npart] = n;
        bp[nblocks] = npart;
    }
}

// esplit[q]: how many of position q's off-diagonal columns lie before the first
// row of its block (they are read from other blocks; the rest from this one).
// Columns are increasing inside a row.
__global__ void k_esplit(int32_t n, const int32_t* __restrict__ seq, const int32_t* __restrict__ st,
                         const int32_t* __restrict__ col, int32_t R, int32_t* __restrict__ es) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int32_t base = (seq[q] / R) * R;
    int32_t lo = st[q], hi = st[q + 1];
    const int32_t a = lo;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < base) lo = mid + 1;
        else hi = mid;
    }
    es[q] = lo - a;
}

// qcod[q] = codelet covering position q.
__global__ void k_qcod(int64_t ncod, const dcod* __restrict__ cod, int32_t* __restrict__ qc) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncod) return;
    const int32_t q0 = cod[c].q0, m = cod[c].m;
    for (int32_t i = 0; i < m; ++i) qc[q0 + i] = (int32_t)c;
}

__device__ __forceinline__ int32_t pow2_at_least(int32_t need) {
    int32_t v = 1;
    while (v < need && v < 32) v <<= 1;
    return v;
}

__device__ __forceinline__ int32_t pow2_at_most(int32_t lim) {
    int32_t v = 1;
    while (v * 2 <= lim && v < 32) v <<= 1;
    return v;
}

// Chunks of the coarsened solve: each partition is cut greedily, in position
// order, into runs of at most DDF_BLK_ROWS_CAP rows and DDF_BLK_ENT_CAP points;
// a row with more points than that is a chunk of its own ("direct").  One
// thread per partition; write == false only counts.
template <bool write>
__device__ int32_t chunk_partition(int32_t a, int32_t b, const int32_t* __restrict__ st,
                                   const int32_t* __restrict__ es, const int32_t* __restrict__ qc,
                                   const dcod* __restrict__ cod, int32_t* __restrict__ cq0,
                                   int32_t* __restrict__ cmeta) {
    int32_t k = 0;
    int32_t q = a;
    while (q < b) {
        const int32_t c0 = q;
        int32_t rows = 0, ents = 0, mi = 0, ml = 0, flags = 0;
        const int32_t L0 = st[q + 1] - st[q];
        if (L0 > DDF_BLK_ENT_CAP) {
            rows = 1;
            mi = L0 - es[q];
            ml = L0;
            flags = DDF_CK_DIRECT;
            ++q;
        } else {
            while (q < b && rows < DDF_BLK_ROWS_CAP) {
                const int32_t L = st[q + 1] - st[q];
                if (L > DDF_BLK_ENT_CAP || ents + L > DDF_BLK_ENT_CAP) break;
                ents += L;
                ++rows;
                mi = max(mi, L - es[q]);
                ml = max(ml, L);
                if (write && cod[qc[q]].type == DDF_PSC2) flags |= DDF_CK_PSC2;
                ++q;
            }
        }
        if (write) {
            const int32_t vch = min(pow2_at_most(DDF_BLK_CHAIN_LANES / rows),
                                    pow2_at_least((mi + DDF_BLK_CHAIN_PER_LANE - 1) / DDF_BLK_CHAIN_PER_LANE));
            const int32_t vpr = pow2_at_least((ml + DDF_BLK_PROD_PER_LANE - 1) / DDF_BLK_PROD_PER_LANE);
            cq0[k] = c0;
            cmeta[k] = vch | (vpr << 8) | flags;
        }
        ++k;
    }
    return k;
}

__global__ void k_chunk_count(int32_t npart, const int32_t* __restrict__ pp, const int32_t* __restrict__ st,
                              const int32_t* __restrict__ es, int32_t* __restrict__ cnt) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npart) return;
    cnt[g] = chunk_partition<false>(pp[g], pp[g + 1], st, es, nullptr, nullptr, nullptr, nullptr);
}

__global__ void k_chunk_fill(int32_t npart, const int32_t* __restrict__ pp, const int32_t* __restrict__ st,
                             const int32_t* __restrict__ es, const int32_t* __restrict__ qc,
                             const dcod* __restrict__ cod, const int64_t* __restrict__ coff, int32_t n,
                             int32_t* __restrict__ cq0, int32_t* __restrict__ cmeta) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npart) return;
    const int64_t o = coff[g];
    chunk_partition<true>(pp[g], pp[g + 1], st, es, qc, cod, cq0 + o, cmeta + o);
    if (g == 0) cq0[coff[npart]] = n;
}

__global__ void k_blk_chunk(int32_t nblocks, const int32_t* __restrict__ bp, const int64_t* __restrict__ coff,
                            int32_t* __restrict__ bc) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b <= nblocks) bc[b] = (int32_t)coff[bp[b]];
}

// ---------------------------------------------------------------------------
// SpTRSV relayout: off-diagonal columns and values of the rows in level order
// ---------------------------------------------------------------------------
// rp[r] .. re[r]: row r of L, its diagonal last (re = rp + 1 when the input is
// L itself; the end of the lower part of each row when L is read from A)
__global__ void k_rel_lens(int32_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ re, int32_t* __restrict__ lens) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    int32_t r = perm[q];
    lens[q] = re[r] - rp[r] - 1;
}

// Copies the off-diagonal columns (col != NULL) and values (vals != NULL) of
// the rows in level order, and 1 / L_qq (and L_qq when diag != NULL).  A warp
// takes 32 consecutive positions, whose outputs are one contiguous stretch
// st[q0] .. st[q0 + 32]: lane l finds the source of output element o = l, l +
// 32, ... by a binary search over the positions' output starts (staged in
// shared memory), so the writes are coalesced and the reads of a row's
// points are contiguous across lanes.
constexpr int REL_THREADS = 256;

__global__ void __launch_bounds__(REL_THREADS)
k_rel_gather(int32_t n, const int32_t* __restrict__ perm, const int32_t* __restrict__ rp,
             const int32_t* __restrict__ re, const int32_t* __restrict__ ci, const double* __restrict__ vals,
             const int32_t* __restrict__ st, int32_t* __restrict__ col, double* __restrict__ val,
             double* __restrict__ dinv, double* __restrict__ diag) {
    __shared__ int32_t sd_all[REL_THREADS / 32][32];
    __shared__ int32_t sa_all[REL_THREADS / 32][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t* sd = sd_all[w];
    int32_t* sa = sa_all[w];
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gq = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gq * 32 < n; gq += nw) {
        const int64_t q0 = gq * 32;
        const int32_t R = (int32_t)min((int64_t)32, (int64_t)n - q0);
        const int64_t q = q0 + lane;
        int32_t a = 0, d = 0;
        if (lane < R) {
            const int32_t r = perm[q];
            a = rp[r];
            const int32_t e = re[r] - 1;   // the diagonal is last
            d = st[q];
            if (vals) {
                const double dv = vals[e];
                dinv[q] = 1.0 / dv;
                if (diag) diag[q] = dv;
            }
        }
        const int32_t d0 = __shfl_sync(0xffffffffu, d, 0);
        const int32_t dend = st[q0 + R];
        sd[lane] = d - d0;
        sa[lane] = a;
        __syncwarp();
        const int32_t T = dend - d0;
#pragma unroll 4
        for (int32_t o = lane; o < T; o += 32) {
            int32_t lo = 0, hi = R - 1;   // the last position whose output starts at or before o
            while (lo < hi) {
                const int32_t mid = (lo + hi + 1) >> 1;
                if (sd[mid] <= o) lo = mid;
                else hi = mid - 1;
            }
            const int32_t src = sa[lo] + (o - sd[lo]);
            if (col) col[d0 + o] = ci[src];
            if (vals) val[d0 + o] = vals[src];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// regions (GetConsecutiveIterations): windows of t positions of each partition
// ---------------------------------------------------------------------------
__global__ void k_region_counts(int32_t nparts, const int32_t* __restrict__ pp, int32_t t,
                                int32_t* __restrict__ rc) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nparts) return;
    int32_t sz = pp[l + 1] - pp[l];
    rc[l] = (sz + t - 1) / t;
}

// One thread per region g: its partition is the last p with roff[p] <= g.
__global__ void k_region_fill(int32_t nparts, const int32_t* __restrict__ pp, int32_t t,
                              const int64_t* __restrict__ roff, int64_t nreg, int32_t* __restrict__ ra,
                              int32_t* __restrict__ rb, int32_t* __restrict__ rpart) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nreg) return;
    int32_t lo = 0, hi = nparts - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (roff[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const int32_t a = pp[lo] + (int32_t)(g - roff[lo]) * t;
    ra[g] = a;
    rb[g] = min(a + t, pp[lo + 1]);
    rpart[g] = lo;
}

// ---------------------------------------------------------------------------
// ComputeFOPD
// ---------------------------------------------------------------------------
struct Feat {
    const uint8_t* fl;
    const int32_t *sig, *dF, *dG, *dH;
    const int32_t* st;
};

// v lanes per position: the checks over a row's points are split across the
// lanes and combined with warp votes inside the group of v lanes.
__global__ void k_features(int32_t n, const int32_t* __restrict__ seq, const int32_t* __restrict__ st,
                           const int32_t* __restrict__ col, const uint32_t* __restrict__ lsorted,
                           uint8_t* __restrict__ fl, int32_t* __restrict__ sig, int32_t* __restrict__ dF,
                           int32_t* __restrict__ dG, int32_t* __restrict__ dH, int lanes) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lg = __ffs(lanes) - 1, li = (int)(t & (lanes - 1));
    const int64_t q = t >> lg;
    const bool act = q < n;
    int32_t a = 0, L = 0, s = 0, ap = 0, Lp = 0, d0 = 0;
    bool link = false;
    if (act) {
        a = st[q];
        L = st[q + 1] - a;
        link = q > 0 && (lsorted == nullptr || lsorted[q] == lsorted[q - 1]);
        if (L >= 2) s = col[a + 1] - col[a];
        if (link) {
            ap = st[q - 1];
            Lp = a - ap;
            if (L == Lp && L > 0) d0 = col[a] - col[ap];
        }
    }
    bool ok = true, tr = true;
    if (act) {
        const int32_t* h = col + a;
        for (int32_t i = 1 + li; i + 1 < L; i += lanes)
            if (h[i + 1] - h[i] != s) {
                ok = false;
                break;
            }
        if (link && L == Lp) {
            const int32_t* hp = col + ap;
            for (int32_t i = 1 + li; i < L; i += lanes)
                if (h[i] - hp[i] != d0) {
                    tr = false;
                    break;
                }
        }
    }
    // AND over the group of v lanes
    const unsigned gm = (lanes == 32) ? 0xffffffffu : (((1u << lanes) - 1u) << (threadIdx.x & 31 & ~(lanes - 1)));
    {
        const unsigned bo = __ballot_sync(0xffffffffu, !ok), bt = __ballot_sync(0xffffffffu, !tr);
        ok = (bo & gm) == 0;
        tr = (bt & gm) == 0;
    }
    if (!act || li != 0) return;
    uint8_t f = 0;
    if (ok) f |= FL_HSTR;
    int32_t df = 0, dg = 0, dh = 0;
    if (link) {
        f |= FL_LINK;
        df = seq ? seq[q] - seq[q - 1] : 1;
        dg = a - ap;
        if (L == Lp) {
            f |= FL_EQLEN;
            if (tr) {
                f |= FL_TRANS;
                dh = d0;
            }
        }
    }
    fl[q] = f;
    sig[q] = s;
    dF[q] = df;
    dG[q] = dg;
    dH[q] = dh;
}

// ---------------------------------------------------------------------------
// mining strategies (one warp per region)
//
// The warp first turns the region's FOPD features into 512-bit predicate
// masks over the local positions i = q - a (one ballot per 32 positions):
//   hstr   row i has evenly spaced columns (Delta_i1 h constant)
//   ok     link (i-1, i): equal lengths and a translated pattern
//   same   ok at i and i-1 with the same strides (Delta_i0 of f, g, h)
//   chF    Delta_i0 f changes at i        chG  Delta_i0 g changes at i
//   neq    rows i-1 and i differ in length
// The three greedy strategies then run on lane 0 as bit scans over these
// masks: each step jumps to the next candidate position, so a region costs
// O(pieces) instead of O(t) per strategy.  The decisions are the same as
// the position-by-position definition (and as the oracle's).
// ---------------------------------------------------------------------------
struct Weights {
    int64_t op, cl, idx;
};

constexpr int MW = DDF_MAX_T / 32;    // 32-bit words per region mask
constexpr int MINE_WARPS = 4;

struct RegionMasks {
    uint32_t hstr[MW], ok[MW], same[MW], chF[MW], chG[MW], neq[MW], cov[MW];
    int32_t st[DDF_MAX_T + 1];        // starts[a + i] - starts[a]
};

// smallest j in [from, end) whose bit equals `want`, else end
__device__ __forceinline__ int32_t next_bit(const uint32_t* m, int32_t from, int32_t end, bool want) {
    if (from >= end) return end;
    int32_t w = from >> 5;
    uint32_t word = want ? m[w] : ~m[w];
    word &= ~0u << (from & 31);
    const int32_t wl = (end - 1) >> 5;
    while (true) {
        if (word) {
            int32_t pos = (w << 5) + __ffs(word) - 1;
            return pos < end ? pos : end;
        }
        if (++w > wl) return end;
        word = want ? m[w] : ~m[w];
    }
}

__device__ __forceinline__ bool any_bit(const uint32_t* m, int32_t from, int32_t end) {
    return next_bit(m, from, end, true) < end;
}

__device__ __forceinline__ void set_bits(uint32_t* m, int32_t from, int32_t end) {
    for (int32_t i = from; i < end;) {
        int32_t w = i >> 5, b = i & 31;
        int32_t k = min(32 - b, end - i);
        uint32_t bits = (k == 32) ? ~0u : (((1u << k) - 1u) << b);
        m[w] |= bits;
        i += k;
    }
}

// maximal run from i with f, g strided and a shared s (PSC I form)
__device__ __forceinline__ int32_t ext_run(const RegionMasks& R, int32_t i, int32_t end) {
    int32_t i1 = i + 1;
    if (i1 >= end || !((R.ok[i1 >> 5] >> (i1 & 31)) & 1u)) return i1;
    return next_bit(R.same, i + 2, end, false);
}

__device__ __forceinline__ bool run_F(const RegionMasks& R, int32_t i, int32_t j) {
    return !any_bit(R.chF, i + 2, j);
}
__device__ __forceinline__ bool run_G(const RegionMasks& R, int32_t i, int32_t j) {
    return !any_bit(R.neq, i + 1, j) && !any_bit(R.chG, i + 2, j);
}

// Eq. 1: c = w_op |p| + w_cl + w_idx (|s_f| + |s_g| + |s_h|)
__device__ int64_t piece_cost(const RegionMasks& R, int type, int32_t i, int32_t j, const Weights& w) {
    int64_t m = j - i;
    int64_t p = (int64_t)R.st[j] - R.st[i];
    int64_t sf = 0, sg = 0, sh = 0;
    if (type == DDF_PSC1) sh = R.st[i + 1] - R.st[i];
    if (type == DDF_PSC2) {
        sf = run_F(R, i, j) ? 0 : m;
        sg = run_G(R, i, j) ? 0 : m;
        sh = p;
    }
    return w.op * p + w.cl + w.idx * (sf + sg + sh);
}

struct Sink {
    const RegionMasks* R;
    int8_t* mark;       // global marks of the region (NULL: cost only)
    int32_t* plen;
    int64_t cost;
    int32_t pieces;
    __device__ void put(int type, int32_t i, int32_t j, const Weights& w) {
        cost += piece_cost(*R, type, i, j, w);
        if (mark) {
            int flags = (run_F(*R, i, j) ? 4 : 0) | (run_G(*R, i, j) ? 8 : 0);
            mark[i] = (int8_t)(type | flags);
            plen[i] = j - i;
        }
        ++pieces;
    }
};

__device__ void leftovers(const RegionMasks& R, int32_t len, const Weights& w, Sink& out) {
    int32_t q = next_bit(R.cov, 0, len, false);
    while (q < len) {
        int32_t e = next_bit(R.cov, q, len, true);
        out.put(DDF_PSC2, q, e, w);
        q = next_bit(R.cov, e, len, false);
    }
}

__device__ void clear_cov(RegionMasks& R) {
    for (int k = 0; k < MW; ++k) R.cov[k] = 0u;
}

__device__ void blas_first(RegionMasks& R, int32_t len, int allowed, const Weights& w, Sink& out) {
    clear_cov(R);
    int32_t q = next_bit(R.hstr, 0, len, true);            // maximal BLAS runs
    while (q < len) {
        int32_t q1 = ext_run(R, q, len);
        out.put(DDF_BLAS, q, q1, w);
        set_bits(R.cov, q, q1);
        q = next_bit(R.hstr, q1, len, true);
    }
    if (allowed & DDF_ALLOW_PSC1) {                        // PSC I runs in the gaps
        q = next_bit(R.cov, 0, len, false);
        while (q < len) {
            const int32_t v = next_bit(R.cov, q, len, true);
            int32_t u = q;
            while (u < v) {
                int32_t u1 = ext_run(R, u, v);
                if (u1 - u >= 2) {
                    out.put(DDF_PSC1, u, u1, w);
                    set_bits(R.cov, u, u1);
                    u = u1;
                } else {
                    // next start that can extend: ok at its successor
                    int32_t nx = next_bit(R.ok, u + 2, v, true);
                    u = (nx < v) ? nx - 1 : v;
                }
            }
            q = next_bit(R.cov, v, len, false);
        }
    }
    leftovers(R, len, w, out);
}

__device__ void psc1_first(RegionMasks& R, int32_t len, int allowed, const Weights& w, Sink& out) {
    clear_cov(R);
    int32_t q = 0;
    while (q < len) {
        int32_t q1 = ext_run(R, q, len);
        if (q1 - q >= 2) {
            bool h = (R.hstr[q >> 5] >> (q & 31)) & 1u;
            out.put((h && (allowed & DDF_ALLOW_BLAS)) ? DDF_BLAS : DDF_PSC1, q, q1, w);
            set_bits(R.cov, q, q1);
            q = q1;
        } else {
            int32_t nx = next_bit(R.ok, q + 2, len, true);
            q = (nx < len) ? nx - 1 : len;
        }
    }
    leftovers(R, len, w, out);
}

// Pass 1: build the masks, choose the strategy of least total cost (ties:
// BLAS_first, then PSCI_first), and record its pieces at their first
// position: mark (type | F << 2 | G << 3), plen (rows) and lidx (index of the
// piece inside the region).
__global__ void __launch_bounds__(32 * MINE_WARPS)
k_mine(int64_t nreg, const int32_t* __restrict__ ra, const int32_t* __restrict__ rb, Feat F, int allowed,
       Weights w, int8_t* __restrict__ mark, int32_t* __restrict__ plen, int32_t* __restrict__ lidx,
       int32_t* __restrict__ cnt) {
    __shared__ RegionMasks RM[MINE_WARPS];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * MINE_WARPS + wi;
    if (r >= nreg) return;
    RegionMasks& R = RM[wi];
    const int32_t a = ra[r], len = rb[r] - a;
    const int32_t s0 = F.st[a];
    int32_t pdF = 0, pdG = 0, pdH = 0;
    bool pok = false;
    for (int32_t c = 0; c * 32 < len; ++c) {
        const int32_t i = c * 32 + lane;
        const bool valid = i < len;
        const int64_t q = (int64_t)a + i;
        uint8_t f = valid ? F.fl[q] : 0;
        int32_t df = valid ? F.dF[q] : 0, dg = valid ? F.dG[q] : 0, dh = valid ? F.dH[q] : 0;
        // values of position i - 1 (lane 0 takes them from the previous chunk)
        int32_t udF = __shfl_up_sync(0xffffffffu, df, 1);
        int32_t udG = __shfl_up_sync(0xffffffffu, dg, 1);
        int32_t udH = __shfl_up_sync(0xffffffffu, dh, 1);
        bool ok = valid && i >= 1 && (f & FL_EQLEN) && (f & FL_TRANS);
        bool uok = __shfl_up_sync(0xffffffffu, ok, 1);
        if (lane == 0) {
            udF = pdF;
            udG = pdG;
            udH = pdH;
            uok = pok;
        }
        bool same = ok && i >= 2 && uok && df == udF && dg == udG && dh == udH;
        uint32_t bh = __ballot_sync(0xffffffffu, valid && (f & FL_HSTR));
        uint32_t bo = __ballot_sync(0xffffffffu, ok);
        uint32_t bs = __ballot_sync(0xffffffffu, same);
        uint32_t bf = __ballot_sync(0xffffffffu, valid && i >= 2 && df != udF);
        uint32_t bg = __ballot_sync(0xffffffffu, valid && i >= 2 && dg != udG);
        uint32_t bn = __ballot_sync(0xffffffffu, valid && i >= 1 && !(f & FL_EQLEN));
        if (lane == 0) {
            R.hstr[c] = bh;
            R.ok[c] = bo;
            R.same[c] = bs;
            R.chF[c] = bf;
            R.chG[c] = bg;
            R.neq[c] = bn;
        }
        pdF = __shfl_sync(0xffffffffu, df, 31);
        pdG = __shfl_sync(0xffffffffu, dg, 31);
        pdH = __shfl_sync(0xffffffffu, dh, 31);
        pok = __shfl_sync(0xffffffffu, ok, 31);
    }
    for (int32_t i = lane; i <= len; i += 32) R.st[i] = F.st[a + i] - s0;
    for (int32_t i = lane; i < len; i += 32) mark[a + i] = (int8_t)MK_NONE;
    __syncwarp();
    if (lane == 0) {
        int64_t C[3];
        int best = -1;
        for (int st = 0; st < 3; ++st) {
            if (st == 0 && !(allowed & DDF_ALLOW_BLAS)) continue;
            if (st == 1 && !(allowed & DDF_ALLOW_PSC1)) continue;
            Sink k{&R, nullptr, nullptr, 0, 0};
            if (st == 0) blas_first(R, len, allowed, w, k);
            else if (st == 1) psc1_first(R, len, allowed, w, k);
            else k.put(DDF_PSC2, 0, len, w);
            C[st] = k.cost;
            if (best < 0 || C[st] < C[best]) best = st;
        }
        Sink k{&R, mark + a, plen + a, 0, 0};
        if (best == 0) blas_first(R, len, allowed, w, k);
        else if (best == 1) psc1_first(R, len, allowed, w, k);
        else k.put(DDF_PSC2, 0, len, w);
        cnt[r] = k.pieces;
    }
    __syncwarp();
    // codelets are appended in position order: the local index of a piece is
    // the number of piece starts before it in the region
    int32_t before = 0;
    for (int32_t c = 0; c * 32 < len; ++c) {
        const int32_t i = c * 32 + lane;
        const bool start = i < len && mark[a + i] != (int8_t)MK_NONE;
        const uint32_t bal = __ballot_sync(0xffffffffu, start);
        if (start) lidx[a + i] = before + __popc(bal & ((1u << lane) - 1u));
        before += __popc(bal);
    }
}

// Pass 2 (cList.append): the lanes of a warp walk the region's positions and
// write the codelet of every piece start at off[region] + its local index.
__global__ void __launch_bounds__(32 * MINE_WARPS)
k_emit(int64_t nreg, const int32_t* __restrict__ ra, const int32_t* __restrict__ rb,
       const int32_t* __restrict__ rpart, Feat F, const int32_t* __restrict__ seq,
       const int32_t* __restrict__ col, const int8_t* __restrict__ mark, const int32_t* __restrict__ plen,
       const int32_t* __restrict__ lidx, const int64_t* __restrict__ off, dcod* __restrict__ out) {
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * MINE_WARPS + wi;
    if (r >= nreg) return;
    const int32_t a = ra[r], b = rb[r];
    const int64_t o = off[r];
    for (int32_t q = a + lane; q < b; q += 32) {
        const int mk = mark[q];
        if (mk == MK_NONE) continue;
        const int type = mk & 3;
        const bool fs = (mk & 4) != 0, gs = (mk & 8) != 0;
        const int32_t m = plen[q];
        const int32_t L = F.st[q + 1] - F.st[q];
        dcod c;
        c.q0 = q;
        c.m = m;
        c.n = (type == DDF_PSC2) ? -1 : L;
        c.type = type;
        c.part = rpart[r];
        c.flags = (fs ? DC_F_STRIDED : 0) | (gs ? DC_G_STRIDED : 0);
        c.f0 = seq ? seq[q] : q;
        c.rho = (fs && m >= 2) ? F.dF[q + 1] : 0;
        c.g0 = F.st[q];
        c.gamma = (gs && m >= 2) ? F.dG[q + 1] : 0;
        c.h0 = (type != DDF_PSC2 && L >= 1) ? col[F.st[q]] : 0;
        c.delta = (type != DDF_PSC2 && m >= 2) ? F.dH[q + 1] : 0;
        c.sigma = (type == DDF_BLAS && L >= 2) ? F.sig[q] : 0;
        c.sref = F.st[q];
        c.pad0 = c.pad1 = 0;
        out[o + lidx[q]] = c;
    }
}

// ---------------------------------------------------------------------------
// executor work units
// ---------------------------------------------------------------------------
constexpr int64_t SPMV_WARP_SPAN = 4096;   // bytes of values one SpMV warp pass spans

__device__ __forceinline__ int32_t pow2_ceil32(int32_t x) {
    int32_t v = 1;
    while (v < x && v < 32) v <<= 1;
    return v;
}

// Units of one codelet.  BLAS / PSC I: rows split evenly, v = lanes per row.
// PSC II: consecutive rows while the unit stays within unit_nnz points.
// one_pass (SpTRSV): a unit is what one warp covers in a single pass, i.e.
// 32 / v rows with v lanes for DDF_SOLVE_PTS points each, so that a solve
// unit waits on its dependencies only once.
template <bool WRITE>
__device__ int32_t make_units(const dcod& c, int32_t ci, const int32_t* __restrict__ st,
                              int32_t unit_nnz, bool one_pass, dunit* out) {
    int32_t cnt = 0;
    if (c.type != DDF_PSC2) {
        int32_t n = c.n;
        int32_t v, rows;
        if (one_pass) {
            v = pow2_ceil32(n > 0 ? (n + DDF_SOLVE_PTS - 1) / DDF_SOLVE_PTS : 1);
            rows = 32 / v;
        } else {
            // SpMV: the fewest lanes per row whose warp footprint (32/v rows of
            // n values) stays within SPMV_WARP_SPAN bytes.  Fewer lanes per row
            // means fewer shuffle-reduction additions: the FP64 pipe, not HBM,
            // is the first limit of an FP64 SpMV on this part.
            v = 1;
            while (v < 32 && (int64_t)(32 / v) * n * 8 > SPMV_WARP_SPAN) v <<= 1;
            int32_t rpw = 32 / v;
            rows = rpw * max(1, (n > 0) ? unit_nnz / (rpw * n) : 32);
        }
        for (int32_t i = 0; i < c.m; i += rows) {
            if (WRITE) out[cnt] = dunit{ci, i, min(i + rows, c.m), v};
            ++cnt;
        }
        return cnt;
    }
    int32_t i = 0;
    while (i < c.m) {
        int32_t j = i;
        if (one_pass) {
            int32_t v = pow2_ceil32(max((st[c.q0 + i + 1] - st[c.q0 + i] + DDF_SOLVE_PTS - 1) / DDF_SOLVE_PTS, 1));
            j = i + 1;
            while (j < c.m) {
                int32_t v2 = max(v, pow2_ceil32(max((st[c.q0 + j + 1] - st[c.q0 + j] + DDF_SOLVE_PTS - 1) /
                                                        DDF_SOLVE_PTS, 1)));
                if (v2 * (j - i + 1) > 32) break;
                v = v2;
                ++j;
            }
            if (WRITE) out[cnt] = dunit{ci, i, j, v};
            ++cnt;
            i = j;
            continue;
        }
        int64_t pts = 0;
        while (j < c.m && j - i < 256) {
            int32_t L = st[c.q0 + j + 1] - st[c.q0 + j];
            if (j > i && pts + L > unit_nnz) break;
            pts += L;
            ++j;
        }
        int32_t avg = (int32_t)((pts + (j - i) - 1) / (j - i));
        if (WRITE) out[cnt] = dunit{ci, i, j, pow2_ceil32(avg > 0 ? avg : 1)};
        ++cnt;
        i = j;
    }
    return cnt;
}

// SpMV BLAS / PSC I codelets smaller than one unit are grouped: consecutive
// codelets of one type and one row length whose rows are contiguous share a
// work unit (encoded with i0b = -count, i0e = total rows), so that a warp
// amortises its descriptor loads over several small codelets.
constexpr int32_t GROUP_MAX_ROWS = 256;
constexpr int32_t GROUP_MAX_CODELETS = 32;

__device__ __forceinline__ int32_t spmv_lanes(int32_t n) {
    int32_t v = 1;
    while (v < 32 && (int64_t)(32 / v) * n * 8 > SPMV_WARP_SPAN) v <<= 1;
    return v;
}
__device__ __forceinline__ int32_t spmv_unit_rows(int32_t n, int32_t unit_nnz) {
    int32_t rpw = 32 / spmv_lanes(n);
    return rpw * max(1, (n > 0) ? unit_nnz / (rpw * n) : 32);
}
__device__ __forceinline__ bool groupable(const dcod& c, int32_t unit_nnz) {
    return c.type != DDF_PSC2 && !(c.flags & DC_TILED) && c.m < spmv_unit_rows(c.n, unit_nnz);
}
__device__ __forceinline__ bool linked(const dcod& p, const dcod& c, int32_t unit_nnz) {
    return groupable(p, unit_nnz) && groupable(c, unit_nnz) && p.type == c.type && p.n == c.n &&
           p.q0 + p.m == c.q0;
}

// Group units led by codelet i (which starts a chain of linked codelets).
template <bool WRITE>
__device__ int32_t make_groups(const dcod* __restrict__ cod, int64_t ncod, int64_t i, int32_t unit_nnz,
                               dunit* out) {
    const dcod c0 = cod[i];
    const int32_t cap = min(GROUP_MAX_ROWS, 4 * spmv_unit_rows(c0.n, unit_nnz));
    const int32_t v = spmv_lanes(c0.n);
    int32_t cnt = 0;
    int64_t g = i;
    int32_t rows = c0.m, k = 1;
    dcod prev = c0;
    for (int64_t j = i + 1;; ++j) {
        bool more = j < ncod;
        dcod cj;
        if (more) {
            cj = cod[j];
            more = linked(prev, cj, unit_nnz);
        }
        if (!more || rows + cj.m > cap || k == GROUP_MAX_CODELETS) {
            if (WRITE) out[cnt] = (k == 1) ? dunit{(int32_t)g, 0, rows, v} : dunit{(int32_t)g, -k, rows, v};
            ++cnt;
            if (!more) break;
            g = j;
            rows = 0;
            k = 0;
        }
        rows += cj.m;
        ++k;
        prev = cj;
    }
    return cnt;
}

__global__ void k_unit_counts(int64_t ncod, const dcod* __restrict__ cod, const int32_t* __restrict__ st,
                              int32_t unit_nnz, int split_types, int32_t* __restrict__ c0,
                              int32_t* __restrict__ c1, int32_t* __restrict__ c2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncod) return;
    dcod c = cod[i];
    int32_t k;
    if (c.flags & DC_TILED) {
        k = 0;   // executed through its tiles
    } else if (split_types && groupable(c, unit_nnz)) {
        // members of a chain add nothing; the chain's first codelet makes its groups
        k = (i > 0 && linked(cod[i - 1], c, unit_nnz)) ? 0 : make_groups<false>(cod, ncod, i, unit_nnz, nullptr);
    } else {
        k = make_units<false>(c, (int32_t)i, st, unit_nnz, !split_types, nullptr);
    }
    if (!split_types) {
        c0[i] = k;
        return;
    }
    c0[i] = c.type == DDF_BLAS ? k : 0;
    c1[i] = c.type == DDF_PSC1 ? k : 0;
    c2[i] = c.type == DDF_PSC2 ? k : 0;
}

__global__ void k_unit_write(int64_t ncod, const dcod* __restrict__ cod, const int32_t* __restrict__ st,
                             int32_t unit_nnz, int split_types, const int64_t* __restrict__ o0,
                             const int64_t* __restrict__ o1, const int64_t* __restrict__ o2,
                             dunit* __restrict__ u0, dunit* __restrict__ u1, dunit* __restrict__ u2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncod) return;
    dcod c = cod[i];
    if (c.flags & DC_TILED) return;
    dunit* dst;
    if (!split_types) dst = u0 + o0[i];
    else if (c.type == DDF_BLAS) dst = u0 + o0[i];
    else if (c.type == DDF_PSC1) dst = u1 + o1[i];
    else dst = u2 + o2[i];
    if (split_types && groupable(c, unit_nnz)) {
        if (!(i > 0 && linked(cod[i - 1], c, unit_nnz))) make_groups<true>(cod, ncod, i, unit_nnz, dst);
        return;
    }
    make_units<true>(c, (int32_t)i, st, unit_nnz, !split_types, dst);
}

__device__ __forceinline__ bool long_unit(const dunit& U, const dcod* __restrict__ cod,
                                          const int32_t* __restrict__ st) {
    if (U.i0b < 0 || U.i0e - U.i0b != 1) return false;
    const int32_t q = cod[U.cod].q0 + U.i0b;
    return st[q + 1] - st[q] > DDF_LONG_ROW;
}
__global__ void k_long_flags(int64_t nu, const dunit* __restrict__ units, const dcod* __restrict__ cod,
                             const int32_t* __restrict__ st, int32_t* __restrict__ flag) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < nu) flag[u] = long_unit(units[u], cod, st);
}
__global__ void k_long_write(int64_t nu, const dunit* __restrict__ units, const dcod* __restrict__ cod,
                             const int32_t* __restrict__ flag, const int64_t* __restrict__ off,
                             int32_t* __restrict__ lq) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < nu && flag[u]) lq[off[u]] = cod[units[u].cod].q0 + units[u].i0b;
}

__global__ void k_unit_q(int64_t nu, const dunit* __restrict__ units, const dcod* __restrict__ cod,
                         int32_t* __restrict__ uq) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < nu) uq[u] = cod[units[u].cod].q0 + units[u].i0b;
}

// ---------------------------------------------------------------------------
// SpMV value tiles (runs of codelets executed one lane per row)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool tile_eligible(const dcod& c) {
    return c.type != DDF_PSC2 && c.n >= 0 && c.n <= DDF_TILE_NMAX && c.m >= 1;
}
// c continues the run of p: same type and row length, next positions
__device__ __forceinline__ bool tile_linked(const dcod& p, const dcod& c) {
    return tile_eligible(p) && tile_eligible(c) && p.type == c.type && p.n == c.n && p.q0 + p.m == c.q0;
}

// head[c] = 1 when codelet c starts a run
__global__ void k_run_heads(int64_t ncod, const dcod* __restrict__ cod, int32_t* __restrict__ head) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncod) return;
    const dcod C = cod[c];
    head[c] = tile_eligible(C) && !(c > 0 && tile_linked(cod[c - 1], C));
}

// First and one-past-last position of every run (rid = run index, from the
// exclusive scan of the heads), then every codelet of a run records both.
__global__ void k_run_bounds(int64_t ncod, const dcod* __restrict__ cod, const int64_t* __restrict__ rid,
                             int32_t* __restrict__ rs, int32_t* __restrict__ re) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncod) return;
    const dcod C = cod[c];
    if (!tile_eligible(C)) return;
    const int64_t r = rid[c + 1] - 1;   // inclusive count of heads - 1
    if (rid[c + 1] != rid[c]) rs[r] = C.q0;
    if (!(c + 1 < ncod && tile_linked(C, cod[c + 1]))) re[r] = C.q0 + C.m;
}

__global__ void k_run_apply(int64_t ncod, dcod* __restrict__ cod, const int64_t* __restrict__ rid,
                            const int32_t* __restrict__ rs, const int32_t* __restrict__ re) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncod) return;
    dcod& C = cod[c];
    if (!tile_eligible(C)) return;
    const int64_t r = rid[c + 1] - 1;
    C.pad0 = rs[r];
    C.pad1 = re[r];
    C.flags |= DC_TILED;
}

// Tiles that start inside codelet c: starts pad0 + k * DDF_TILE_ROWS in [q0, q0 + m).
__device__ __forceinline__ void tile_range(const dcod& C, int32_t* k0, int32_t* k1) {
    const int32_t T = DDF_TILE_ROWS;
    *k0 = (C.q0 - C.pad0 + T - 1) / T;
    *k1 = (C.q0 + C.m - C.pad0 + T - 1) / T;
}

__global__ void k_tile_counts(int64_t ncod, const dcod* __restrict__ cod, int32_t* __restrict__ c0,
                              int32_t* __restrict__ c1) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncod) return;
    const dcod C = cod[c];
    int32_t k = 0;
    if (C.flags & DC_TILED) {
        int32_t k0, k1;
        tile_range(C, &k0, &k1);
        k = k1 - k0;
    }
    c0[c] = C.type == DDF_BLAS ? k : 0;
    c1[c] = C.type == DDF_PSC1 ? k : 0;
}

__global__ void k_tile_write(int64_t ncod, const dcod* __restrict__ cod, const int32_t* __restrict__ st,
                             const int64_t* __restrict__ o0, const int64_t* __restrict__ o1,
                             dtile* __restrict__ t0, dtile* __restrict__ t1) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncod) return;
    const dcod C = cod[c];
    if (!(C.flags & DC_TILED)) return;
    dtile* dst = C.type == DDF_BLAS ? t0 + o0[c] : t1 + o1[c];
    int32_t k0, k1;
    tile_range(C, &k0, &k1);
    for (int32_t k = k0; k < k1; ++k) {
        const int32_t tq = C.pad0 + k * DDF_TILE_ROWS;
        const int32_t w = min(DDF_TILE_ROWS, C.pad1 - tq);
        uint32_t meta = (uint32_t)(w - 1);
        int64_t cc = c;
        int32_t end = C.q0 + C.m;
        for (int32_t r = 0; r < w; ++r) {
            while (tq + r >= end) {   // the run's next codelet (at most 7 steps in a tile)
                ++cc;
                const dcod N = cod[cc];
                end = N.q0 + N.m;
            }
            meta |= (uint32_t)(cc - c) << (3 + 3 * r);
        }
        dst[k - k0] = dtile{tq, (int32_t)c, st[tq], meta};
    }
}

// Values of every codelet outside tiles, copied in CSR order (one warp per codelet).
__global__ void k_copy_untiled(int64_t ncod, const dcod* __restrict__ cod, const int32_t* __restrict__ st,
                               const double* __restrict__ src, double* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncod; c += nw) {
        const dcod C = cod[c];
        if (C.flags & DC_TILED) continue;
        const int32_t a = st[C.q0], b = st[C.q0 + C.m];
        for (int32_t k = a + lane; k < b; k += 32) dst[k] = src[k];
    }
}

// Values of each tile point-major: point i1 of row r at vb + i1 * w + r (one warp per tile).
__global__ void k_tile_permute(int64_t ntiles, const dtile* __restrict__ tiles, const dcod* __restrict__ cod,
                               const double* __restrict__ src, double* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nw) {
        const dtile T = tiles[t];
        const int32_t w = (int32_t)(T.meta & 7u) + 1;
        const int32_t n = cod[T.cod].n;
        const int32_t tot = w * n;
        for (int32_t e = lane; e < tot; e += 32) {
            const int32_t i1 = e / w, r = e - i1 * w;
            dst[(int64_t)T.vb + e] = src[(int64_t)T.vb + (int64_t)r * n + i1];
        }
    }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    template <typename T>
    ddf_status get(T** p, int64_t n) {
        ddf_status st = ddf_alloc(p, n, s);
        if (!st && *p) ptrs.push_back((void*)*p);
        return st;
    }
    ~Scratch() {
        for (void* p : ptrs) (void)cudaFreeAsync(p, s);
    }
};

template <typename T>
ddf_status d2h(T* host, const T* dev, int64_t n, cudaStream_t s) {
    if (n <= 0) return DDF_OK;
    DDF_CUDA_TRY(cudaMemcpyAsync(host, dev, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost, s));
    DDF_CUDA_TRY(cudaStreamSynchronize(s));
    return DDF_OK;
}

#define TRY(x)                         \
    do {                               \
        ddf_status t_ = (x);           \
        if (t_ != DDF_OK) return t_;   \
    } while (0)

constexpr int TPB = 256;

// Lanes per row for the per-row inspector kernels: the smallest power of two
// at least the mean row length, at most `cap`.
int lanes_for_mean(int64_t entries, int64_t rows, int cap = 32) {
    const int64_t mean = rows > 0 ? (entries + rows - 1) / rows : 1;
    int v = 1;
    while (v < cap && v < mean) v <<= 1;
    return v;
}


// CSR validation: at most 4 lanes per row (inspect(L) of elasticity 64^3:
// 2.22 ms with 32 lanes per row, 2.10 ms with 4, 2.14 ms with one)
constexpr int VALIDATE_MAX_LANES = 4;

void fill_stats(ddf_plan_s* p, const std::vector<dcod>& hc) {
    ddf_plan_stats_t& S = p->stats;
    memset(&S, 0, sizeof(S));
    S.kind = p->kind;
    S.n_rows = p->n;
    S.n_cols = p->n_cols;
    S.depth = p->depth;
    S.levels = p->kind == DDF_SPTRSV ? p->nlevels : 0;
    S.blocks = p->nblocks;
    // SpTRSV: the entries of L (with lower_of_input, fewer than the input's)
    S.nnz = p->kind == DDF_SPTRSV ? p->npts + p->n : p->nnz;
    S.points = p->npts;
    int64_t psc2_nof = 0, s_entries = 0;
    std::vector<int32_t> hst;
    for (const dcod& c : hc) {
        S.ncodelets[c.type]++;
        S.rows[c.type] += c.m;
        if (c.type == DDF_PSC1) s_entries += c.n;
        if (c.type == DDF_PSC2 && !(c.flags & DC_F_STRIDED)) psc2_nof += c.m;
    }
    S.nunits = p->nunits[0] + p->nunits[1] + p->nunits[2] + p->ntiles[0] + p->ntiles[1];
    (void)psc2_nof;
    (void)s_entries;
}

}  // namespace

// Build the plan from device copies of the CSR arrays (rowptr/colidx/values,
// values may be NULL).  SpMV keeps the three arrays as its value layout.
ddf_status ddf_build_plan(ddf_plan_s* p, const int32_t* rowptr, const int32_t* colidx,
                          const double* values, cudaStream_t s) {
    const int32_t n = p->n;
    const int kind = p->kind;
    Scratch tmp{s, {}};
    int32_t* err = nullptr;
    TRY(tmp.get(&err, 1));
    int32_t big = 0x7fffffff;
    DDF_CUDA_TRY(cudaMemcpyAsync(err, &big, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    // row ends of L: rowptr + 1, or (lower_of_input) the end of each row's
    // lower part, computed after the general checks of the input
    const bool lower = kind == DDF_SPTRSV && p->opts.lower_of_input;
    const int32_t* rowend = rowptr + 1;
    const int gl = lanes_for_mean(p->nnz, n, VALIDATE_MAX_LANES);
    k_validate<<<ddf_grid(((int64_t)n + 1) * gl, TPB), TPB, 0, s>>>(n, p->n_cols, p->nnz, rowptr, colidx, values,
                                                                   lower ? (int)DDF_SPMV : kind, err, gl);
    ddf_count_launch();
    if (lower && n > 0) {
        TRY(ddf_alloc(&p->orig_rowend, n, s));
        k_lower_end<<<ddf_grid(n, TPB), TPB, 0, s>>>(n, p->nnz, rowptr, colidx, values, p->orig_rowend, err);
        ddf_count_launch();
        rowend = p->orig_rowend;
    }
    DDF_CUDA_TRY(cudaGetLastError());
    int32_t herr = 0;
    TRY(d2h(&herr, err, 1, s));
    if (herr != 0x7fffffff) return (ddf_status)herr;

    const int32_t* seq = nullptr;        // identity for SpMV
    uint32_t* lsorted = nullptr;         // level of each position (SpTRSV)
    if (kind == DDF_SPMV) {
        p->starts = const_cast<int32_t*>(rowptr);
        p->col = const_cast<int32_t*>(colidx);
        p->val = const_cast<double*>(values);
        p->depth = n > 0 ? 1 : 0;
        p->npts = p->nnz;
        TRY(ddf_alloc(&p->part_ptr, 2, s));
        k_set2<<<1, 1, 0, s>>>(p->part_ptr, 0, n);
        ddf_count_launch();
    } else {
        // findDependencies: sync-free levels
        int32_t* lev = nullptr;
        uint32_t* tick = nullptr;
        int32_t* maxlev = nullptr;
        TRY(tmp.get(&lev, n));
        TRY(tmp.get(&tick, 1));
        TRY(tmp.get(&maxlev, 2));   // [0] largest level, [1] a copy of the status word
        k_fill_i32<<<ddf_grid(n, TPB, 4096), TPB, 0, s>>>(lev, n, -1);
        ddf_count_launch();
        DDF_CUDA_TRY(cudaMemsetAsync(tick, 0, sizeof(uint32_t), s));
        DDF_CUDA_TRY(cudaMemsetAsync(maxlev, 0, sizeof(int32_t), s));
        DDF_CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(int32_t), s));
        if (n > 0) {
            k_levels<<<ddf_grid(n, LEV_CHUNK), 32 * LEV_WARPS, 0, s>>>(n, rowptr, rowend, colidx, lev, tick,
                                                                       maxlev, p->status, p->opts.spin_cap_ns);
            ddf_count_launch();
        }
        DDF_CUDA_TRY(cudaGetLastError());
        DDF_CUDA_TRY(cudaMemcpyAsync(maxlev + 1, p->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        int32_t hm[2] = {0, 0};
        TRY(d2h(hm, maxlev, 2, s));
        const int32_t hmax = hm[0], hstat = hm[1];
        if (hstat) return (ddf_status)hstat;
        p->depth = n > 0 ? hmax + 1 : 0;   // hmax is the largest level
        p->nlevels = p->depth;
        // partitionIterationSpace: rows sorted by (level, row)
        TRY(ddf_alloc(&p->seq, n, s));
        TRY(tmp.get(&lsorted, n));
        DDF_CUDA_TRY(cudaMemcpyAsync(lsorted, lev, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        k_iota_u32<<<ddf_grid(n, TPB, 4096), TPB, 0, s>>>(p->seq, n);
        ddf_count_launch();
        TRY(ddf_radix_sort_u32(lsorted, p->seq, n, (uint32_t)(p->depth > 0 ? p->depth - 1 : 0), s));
        const int32_t R = p->opts.coarsen_rows;
        if (R > 0 && n > 0) {
            // coarsened: stable second sort by block, partitions = (block, level)
            p->nblocks = (int32_t)(((int64_t)n + R - 1) / R);
            uint32_t* key = nullptr;
            int32_t* flag = nullptr;
            int64_t* foff = nullptr;
            TRY(tmp.get(&key, n));
            TRY(tmp.get(&flag, n));
            TRY(tmp.get(&foff, (int64_t)n + 1));
            k_block_key<<<ddf_grid(n, TPB), TPB, 0, s>>>(n, p->seq, R, key);
            ddf_count_launch();
            TRY(ddf_radix_sort_u32(key, p->seq, n, (uint32_t)(p->nblocks - 1), s));
            k_coarse_flags<<<ddf_grid(n, TPB), TPB, 0, s>>>(n, p->seq, key, lev, flag);
            ddf_count_launch();
            TRY(ddf_scan_i32_to_i64(flag, foff, n, s));
            int64_t npart = 0;
            TRY(d2h(&npart, foff + n, 1, s));
            p->depth = (int32_t)npart;
            TRY(ddf_alloc(&p->part_ptr, npart + 1, s));
            TRY(ddf_alloc(&p->blk_ptr, (int64_t)p->nblocks + 1, s));
            k_coarse_fill<<<ddf_grid(n, TPB), TPB, 0, s>>>(n, key, flag, foff, p->depth, p->nblocks, p->part_ptr,
                                                         p->blk_ptr, lsorted);
            ddf_count_launch();
        } else {
            TRY(ddf_alloc(&p->part_ptr, (int64_t)p->depth + 1, s));
            if (n > 0) {
                k_part_ptr<<<ddf_grid(n, TPB), TPB, 0, s>>>(n, lsorted, p->part_ptr, p->depth);
                ddf_count_launch();
            }
            else DDF_CUDA_TRY(cudaMemsetAsync(p->part_ptr, 0, sizeof(int32_t), s));
        }
        // level-ordered copy of the off-diagonal entries
        int32_t* lens = nullptr;
        int64_t* st64 = nullptr;
        TRY(tmp.get(&lens, n));
        TRY(tmp.get(&st64, (int64_t)n + 1));
        if (n > 0) {
            k_rel_lens<<<ddf_grid(n, TPB), TPB, 0, s>>>(n, p->seq, rowptr, rowend, lens);
            ddf_count_launch();
        }
        TRY(ddf_scan_i32_to_i64(lens, st64, n, s));
        // validated: every row of L holds exactly one diagonal entry, stored last
        int64_t npts = p->nnz - n;
        if (lower) TRY(d2h(&npts, st64 + n, 1, s));
        p->npts = npts;
        TRY(ddf_alloc(&p->starts, (int64_t)n + 1, s));
        k_i64_to_i32<<<ddf_grid(n + 1, TPB, 4096), TPB, 0, s>>>(st64, p->starts, (int64_t)n + 1);
        ddf_count_launch();
        // DDF_TAIL_PAD spare elements: the coarsened solve stages ranges of
        // these arrays with 16-byte-granular bulk copies
        TRY(ddf_alloc(&p->col, npts + DDF_TAIL_PAD, s));
        TRY(ddf_alloc(&p->val, npts + DDF_TAIL_PAD, s));
        TRY(ddf_alloc(&p->dinv, n, s));
        if (p->opts.store_dtype != DDF_F64) TRY(ddf_alloc(&p->diag, n, s));
        if (n > 0) {
            const unsigned cap = (unsigned)(p->sm_count > 0 ? p->sm_count : 152) * 8;
            k_rel_gather<<<ddf_grid(((int64_t)n + 31) / 32 * 32, REL_THREADS, cap), REL_THREADS, 0, s>>>(
                n, p->seq, rowptr, rowend, colidx, values, p->starts, p->col, p->val, p->dinv, p->diag);
            ddf_count_launch();
        }
        DDF_CUDA_TRY(cudaGetLastError());
        if (p->nblocks > 0) {
            TRY(ddf_alloc(&p->esplit, n, s));
            k_esplit<<<ddf_grid(n, TPB), TPB, 0, s>>>(n, p->seq, p->starts, p->col, R, p->esplit);
            ddf_count_launch();
        }
        // keep the inspected rowptr for ddf_update_values
        p->orig_rowptr = const_cast<int32_t*>(rowptr);
    }
    p->has_values = values != nullptr;

    // regions
    int32_t nparts = p->depth;
    int32_t t = p->opts.window_t;
    int32_t* rc = nullptr;
    int64_t* roff = nullptr;
    TRY(tmp.get(&rc, nparts));
    TRY(tmp.get(&roff, (int64_t)nparts + 1));
    if (nparts > 0) {
        k_region_counts<<<ddf_grid(nparts, TPB), TPB, 0, s>>>(nparts, p->part_ptr, t, rc);
        ddf_count_launch();
    }
    TRY(ddf_scan_i32_to_i64(rc, roff, nparts, s));
    int64_t nreg = 0;
    TRY(d2h(&nreg, roff + nparts, 1, s));
    int32_t *ra = nullptr, *rb = nullptr, *rpart = nullptr;
    TRY(tmp.get(&ra, nreg));
    TRY(tmp.get(&rb, nreg));
    TRY(tmp.get(&rpart, nreg));
    if (nparts > 0) {
        k_region_fill<<<ddf_grid(nreg, TPB), TPB, 0, s>>>(nparts, p->part_ptr, t, roff, nreg, ra, rb, rpart);
        ddf_count_launch();
    }

    // ComputeFOPD
    uint8_t* fl = nullptr;
    int32_t *sig = nullptr, *dF = nullptr, *dG = nullptr, *dH = nullptr;
    TRY(tmp.get(&fl, n));
    TRY(tmp.get(&sig, n));
    TRY(tmp.get(&dF, n));
    TRY(tmp.get(&dG, n));
    TRY(tmp.get(&dH, n));
    seq = p->seq;
    if (n > 0) {
        const int fv = 1;   // one lane per position measured fastest
        k_features<<<ddf_grid((int64_t)n * fv, TPB), TPB, 0, s>>>(n, seq, p->starts, p->col, lsorted, fl, sig, dF,
                                                                 dG, dH, fv);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    Feat F{fl, sig, dF, dG, dH, p->starts};
    Weights w{p->opts.w_op, p->opts.w_codelet, p->opts.w_index};

    // mining and append
    int8_t* mark = nullptr;
    int32_t *plen = nullptr, *lidx = nullptr;
    int32_t* cnt = nullptr;
    int64_t* off = nullptr;
    TRY(tmp.get(&mark, n));
    TRY(tmp.get(&plen, n));
    TRY(tmp.get(&lidx, n));
    TRY(tmp.get(&cnt, nreg));
    TRY(tmp.get(&off, nreg + 1));
    if (nreg > 0) {
        k_mine<<<ddf_grid(nreg, MINE_WARPS), 32 * MINE_WARPS, 0, s>>>(nreg, ra, rb, F, p->opts.allowed_types, w,
                                                                    mark, plen, lidx, cnt);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    TRY(ddf_scan_i32_to_i64(cnt, off, nreg, s));
    int64_t ncod = 0;
    TRY(d2h(&ncod, off + nreg, 1, s));
    p->ncod = ncod;
    TRY(ddf_alloc(&p->cod, ncod, s));
    if (nreg > 0) {
        k_emit<<<ddf_grid(nreg, MINE_WARPS), 32 * MINE_WARPS, 0, s>>>(nreg, ra, rb, rpart, F, seq, p->col, mark,
                                                                    plen, lidx, off, p->cod);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    if (p->nblocks > 0) {
        TRY(ddf_alloc(&p->qcod, n, s));
        if (ncod > 0) {
            k_qcod<<<ddf_grid(ncod, TPB), TPB, 0, s>>>(ncod, p->cod, p->qcod);
            ddf_count_launch();
        }
        // chunks of the coarsened solve
        const int32_t np = p->depth;
        int32_t* ccnt = nullptr;
        int64_t* coff = nullptr;
        TRY(tmp.get(&ccnt, np));
        TRY(tmp.get(&coff, (int64_t)np + 1));
        k_chunk_count<<<ddf_grid(np, 128), 128, 0, s>>>(np, p->part_ptr, p->starts, p->esplit, ccnt);
        ddf_count_launch();
        TRY(ddf_scan_i32_to_i64(ccnt, coff, np, s));
        int64_t nck = 0;
        TRY(d2h(&nck, coff + np, 1, s));
        p->nchunks = nck;
        TRY(ddf_alloc(&p->chunk_q0, nck + 1, s));
        TRY(ddf_alloc(&p->chunk_meta, nck, s));
        TRY(ddf_alloc(&p->blk_chunk, (int64_t)p->nblocks + 1, s));
        k_chunk_fill<<<ddf_grid(np, 128), 128, 0, s>>>(np, p->part_ptr, p->starts, p->esplit, p->qcod, p->cod,
                                                       coff, n, p->chunk_q0, p->chunk_meta);
        ddf_count_launch();
        k_blk_chunk<<<ddf_grid((int64_t)p->nblocks + 1, TPB), TPB, 0, s>>>(p->nblocks, p->blk_ptr, coff,
                                                                          p->blk_chunk);
        ddf_count_launch();
        DDF_CUDA_TRY(cudaGetLastError());
    }

    // executor units (SpMV: runs of short-row BLAS / PSC I codelets go to tiles)
    TRY(ddf_mark_tiles(p, s));
    TRY(ddf_build_units(p, s));
    p->stats_ready = 0;
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

// SpMV: the tile lists of the DC_TILED codelets (BLAS in tiles[0], PSC I in tiles[1]).
static ddf_status build_tiles(ddf_plan_s* p, cudaStream_t s) {
    Scratch tmp{s, {}};
    const int64_t ncod = p->ncod;
    for (int k = 0; k < 2; ++k) {
        ddf_free(p->tiles[k], s);
        p->ntiles[k] = 0;
    }
    if (ncod <= 0) return DDF_OK;
    int32_t *c0 = nullptr, *c1 = nullptr;
    int64_t *o0 = nullptr, *o1 = nullptr, *t2 = nullptr;
    TRY(tmp.get(&c0, ncod));
    TRY(tmp.get(&c1, ncod));
    TRY(tmp.get(&o0, ncod + 1));
    TRY(tmp.get(&o1, ncod + 1));
    TRY(tmp.get(&t2, 2));
    k_tile_counts<<<ddf_grid(ncod, TPB), TPB, 0, s>>>(ncod, p->cod, c0, c1);
    ddf_count_launch();
    DDF_CUDA_TRY(cudaGetLastError());
    TRY(ddf_scan_i32_to_i64(c0, o0, ncod, s));
    TRY(ddf_scan_i32_to_i64(c1, o1, ncod, s));
    DDF_CUDA_TRY(cudaMemcpyAsync(t2, o0 + ncod, 8, cudaMemcpyDeviceToDevice, s));
    DDF_CUDA_TRY(cudaMemcpyAsync(t2 + 1, o1 + ncod, 8, cudaMemcpyDeviceToDevice, s));
    int64_t tot[2] = {0, 0};
    TRY(d2h(tot, t2, 2, s));
    for (int k = 0; k < 2; ++k) {
        p->ntiles[k] = tot[k];
        TRY(ddf_alloc(&p->tiles[k], tot[k], s));
    }
    if (tot[0] + tot[1] > 0) {
        k_tile_write<<<ddf_grid(ncod, TPB), TPB, 0, s>>>(ncod, p->cod, p->starts, o0, o1, p->tiles[0],
                                                        p->tiles[1]);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

// SpMV: mark the runs of codelets that are executed in tiles (DC_TILED, run
// bounds in pad0 / pad1).  The codelets are in position order.
ddf_status ddf_mark_tiles(ddf_plan_s* p, cudaStream_t s) {
    Scratch tmp{s, {}};
    const int64_t ncod = p->ncod;
    if (p->kind != DDF_SPMV || ncod <= 0) return DDF_OK;
    int32_t* head = nullptr;
    int64_t* rid = nullptr;
    int32_t *rs = nullptr, *re = nullptr;
    TRY(tmp.get(&head, ncod));
    TRY(tmp.get(&rid, ncod + 1));
    TRY(tmp.get(&rs, ncod));
    TRY(tmp.get(&re, ncod));
    k_run_heads<<<ddf_grid(ncod, TPB), TPB, 0, s>>>(ncod, p->cod, head);
    ddf_count_launch();
    DDF_CUDA_TRY(cudaGetLastError());
    TRY(ddf_scan_i32_to_i64(head, rid, ncod, s));
    k_run_bounds<<<ddf_grid(ncod, TPB), TPB, 0, s>>>(ncod, p->cod, rid, rs, re);
    ddf_count_launch();
    k_run_apply<<<ddf_grid(ncod, TPB), TPB, 0, s>>>(ncod, p->cod, rid, rs, re);
    ddf_count_launch();
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

// (Re)build the executor work units of a plan from its codelets with the
// plan's current unit_nnz (SpMV: one list per codelet type; SpTRSV: one list
// in level order).
ddf_status ddf_build_units(ddf_plan_s* p, cudaStream_t s) {
    Scratch tmp{s, {}};
    const int kind = p->kind;
    const int64_t ncod = p->ncod;
    for (int k = 0; k < 3; ++k) {
        ddf_free(p->units[k], s);
        p->nunits[k] = 0;
    }
    int split = kind == DDF_SPMV;
    int32_t *c0 = nullptr, *c1 = nullptr, *c2 = nullptr;
    int64_t *o0 = nullptr, *o1 = nullptr, *o2 = nullptr;
    TRY(tmp.get(&c0, ncod));
    TRY(tmp.get(&o0, ncod + 1));
    if (split) {
        TRY(tmp.get(&c1, ncod));
        TRY(tmp.get(&c2, ncod));
        TRY(tmp.get(&o1, ncod + 1));
        TRY(tmp.get(&o2, ncod + 1));
    }
    if (ncod > 0) {
        k_unit_counts<<<ddf_grid(ncod, TPB), TPB, 0, s>>>(ncod, p->cod, p->starts, p->opts.unit_nnz,
                                                         split, c0, c1, c2);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    TRY(ddf_scan_i32_to_i64(c0, o0, ncod, s));
    if (split) {
        TRY(ddf_scan_i32_to_i64(c1, o1, ncod, s));
        TRY(ddf_scan_i32_to_i64(c2, o2, ncod, s));
    }
    int64_t tot[3] = {0, 0, 0};
    if (split) {
        int64_t* t3 = nullptr;
        TRY(tmp.get(&t3, 3));
        DDF_CUDA_TRY(cudaMemcpyAsync(t3, o0 + ncod, 8, cudaMemcpyDeviceToDevice, s));
        DDF_CUDA_TRY(cudaMemcpyAsync(t3 + 1, o1 + ncod, 8, cudaMemcpyDeviceToDevice, s));
        DDF_CUDA_TRY(cudaMemcpyAsync(t3 + 2, o2 + ncod, 8, cudaMemcpyDeviceToDevice, s));
        TRY(d2h(tot, t3, 3, s));
    } else {
        TRY(d2h(&tot[0], o0 + ncod, 1, s));
    }
    for (int k = 0; k < 3; ++k) {
        p->nunits[k] = tot[k];
        TRY(ddf_alloc(&p->units[k], tot[k], s));
    }
    if (ncod > 0) {
        k_unit_write<<<ddf_grid(ncod, TPB), TPB, 0, s>>>(ncod, p->cod, p->starts, p->opts.unit_nnz, split,
                                                        o0, o1, o2, p->units[0], p->units[1], p->units[2]);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    if (split) {
        TRY(build_tiles(p, s));
        TRY(ddf_build_long_rows(p, s));
    } else {
        TRY(ddf_build_unit_q(p, s));
    }
    return DDF_OK;
}

// SpMV: the PSC II rows of more than DDF_LONG_ROW points, in unit order (each
// is a one-row unit: a unit closes before a row that would take it past
// unit_nnz points).
ddf_status ddf_build_long_rows(ddf_plan_s* p, cudaStream_t s) {
    Scratch tmp{s, {}};
    ddf_free(p->long_q, s);
    p->nlong = 0;
    const int64_t nu = p->nunits[2];
    if (p->kind != DDF_SPMV || nu <= 0) return DDF_OK;
    int32_t* flag = nullptr;
    int64_t* off = nullptr;
    TRY(tmp.get(&flag, nu));
    TRY(tmp.get(&off, nu + 1));
    k_long_flags<<<ddf_grid(nu, TPB), TPB, 0, s>>>(nu, p->units[2], p->cod, p->starts, flag);
    ddf_count_launch();
    DDF_CUDA_TRY(cudaGetLastError());
    TRY(ddf_scan_i32_to_i64(flag, off, nu, s));
    int64_t nl = 0;
    TRY(d2h(&nl, off + nu, 1, s));
    p->nlong = nl;
    TRY(ddf_alloc(&p->long_q, nl, s));
    if (nl > 0) {
        k_long_write<<<ddf_grid(nu, TPB), TPB, 0, s>>>(nu, p->units[2], p->cod, flag, off, p->long_q);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

// SpTRSV: the first position of each work unit (the solve's first load level).
ddf_status ddf_build_unit_q(ddf_plan_s* p, cudaStream_t s) {
    ddf_free(p->unit_q, s);
    const int64_t nu = p->nunits[0];
    TRY(ddf_alloc(&p->unit_q, nu, s));
    if (nu > 0) {
        k_unit_q<<<ddf_grid(nu, TPB), TPB, 0, s>>>(nu, p->units[0], p->cod, p->unit_q);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    return DDF_OK;
}

// Plan statistics, computed on first request from a host copy of the
// descriptors and the starts array (not part of inspection).
ddf_status ddf_compute_stats(ddf_plan_s* p) {
    cudaStream_t s = p->stream;
    const int32_t n = p->n;
    const int64_t ncod = p->ncod;
    std::vector<dcod> hc((size_t)ncod);
    TRY(d2h(hc.data(), p->cod, ncod, s));
    for (int k = 0; k < 3; ++k) p->ncod_type[k] = 0;
    for (const dcod& c : hc) p->ncod_type[c.type]++;
    fill_stats(p, hc);
    std::vector<int32_t> hst((size_t)n + 1);
    TRY(d2h(hst.data(), p->starts, (int64_t)n + 1, s));
    ddf_plan_stats_t& S = p->stats;
    int64_t sentries = 0, psc2_idx_rows = 0, perm_rows = 0;
    for (const dcod& c : hc) {
        int64_t pts = (int64_t)hst[c.q0 + c.m] - hst[c.q0];
        S.ops[c.type] += pts;
        if (c.type == DDF_PSC1) sentries += c.n;
        if (c.type == DDF_PSC2) psc2_idx_rows += c.m + 1;
        if (!(c.flags & DC_F_STRIDED)) perm_rows += c.m;
    }
    for (int32_t q = 0; q < n; ++q) S.max_row_len = std::max<int64_t>(S.max_row_len, hst[q + 1] - hst[q]);
    int64_t desc = 64 * ncod;   // codelet descriptors (work units are a scheduling detail)
    if (p->kind == DDF_SPMV) {
        S.bytes_exec = 8 * S.points + 8 * (int64_t)p->n_cols + 8 * (int64_t)n + 4 * S.ops[DDF_PSC2] +
                       4 * psc2_idx_rows + 4 * sentries + desc;
    } else {
        S.bytes_exec = 8 * S.points + 8 * (int64_t)n /*dinv*/ + 8 * (int64_t)n /*b*/ +
                       16 * (int64_t)n /*x fill + write*/ + 4 * S.ops[DDF_PSC2] + 4 * psc2_idx_rows +
                       4 * perm_rows + 4 * sentries + desc;
    }
    p->stats_ready = 1;
    return DDF_OK;
}

// New values in the original CSR order, same pattern.
// SpMV: CSR order, except the tiles' values, which are stored point-major.
// values and the plan's array must not overlap.
ddf_status ddf_gather_values(ddf_plan_s* p, const double* values, cudaStream_t s) {
    if (p->kind == DDF_SPMV) {
        if (p->nnz > 0) {
            if (p->ntiles[0] + p->ntiles[1] == 0) {
                DDF_CUDA_TRY(cudaMemcpyAsync(p->val, values, (size_t)p->nnz * 8, cudaMemcpyDeviceToDevice, s));
            } else {
                const unsigned cap = (unsigned)(p->sm_count > 0 ? p->sm_count : 152) * 64;
                k_copy_untiled<<<ddf_grid(p->ncod * 32, TPB, cap), TPB, 0, s>>>(p->ncod, p->cod, p->starts,
                                                                               values, p->val);
                ddf_count_launch();
                for (int t = 0; t < 2; ++t) {
                    if (p->ntiles[t] <= 0) continue;
                    k_tile_permute<<<ddf_grid(p->ntiles[t] * 32, TPB, cap), TPB, 0, s>>>(
                        p->ntiles[t], p->tiles[t], p->cod, values, p->val);
                    ddf_count_launch();
                }
            }
        }
        DDF_CUDA_TRY(cudaGetLastError());
        p->has_values = 1;
        return DDF_OK;
    }
    int32_t n = p->n;
    if (n > 0) {
        const int32_t* re = p->orig_rowend ? p->orig_rowend : p->orig_rowptr + 1;
        const unsigned cap = (unsigned)(p->sm_count > 0 ? p->sm_count : 152) * 8;
        k_rel_gather<<<ddf_grid(((int64_t)n + 31) / 32 * 32, REL_THREADS, cap), REL_THREADS, 0, s>>>(
            n, p->seq, p->orig_rowptr, re, nullptr, values, p->starts, nullptr, p->val, p->dinv, p->diag);
        ddf_count_launch();
    }
    DDF_CUDA_TRY(cudaGetLastError());
    p->has_values = 1;
    return DDF_OK;
}
